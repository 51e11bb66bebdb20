"""Closed-form states used to pin the oracle and, at full size, the GPU path.  TEST INFRASTRUCTURE ONLY.

* Bell / GHZ (paper section V, the GHZ benchmark: one Hadamard then a CNOT chain):
  (|0...0> + |1...1>) / sqrt(2).
* Uniform superposition: Hadamard (printed in section II-A) on every qubit of |0...0> gives 2^(-n/2).
* QFT of a basis state |x> (section V, the QFT benchmark; the discrete Fourier transform of a
  basis vector): amplitude of |y> is 2^(-n/2) exp(+2 pi i x y / 2^n).  The product x*y is taken
  modulo 2^n in exact integer arithmetic before the phase is formed, so the value is accurate to
  fp64 rounding at any n.
* Grover search (section V: the oracle flips the marked state's phase, the diffusion amplifies
  it): the amplitudes after r rounds, from the standard two-dimensional rotation argument.
"""
from __future__ import annotations

import math

import numpy as np


def ghz(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = psi[-1] = 1.0 / np.sqrt(2.0)
    return psi


def uniform(n: int) -> np.ndarray:
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


def qft_amplitudes(n: int, x: int, ys) -> np.ndarray:
    """<y| QFT |x> for the given y (array-like of ints), exact phase reduction mod 2^n."""
    ys = np.asarray(ys, dtype=np.uint64)
    mask = np.uint64((1 << n) - 1) if n < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    # x*y mod 2^n without overflow: split y into 16-bit limbs
    xv = int(x) & ((1 << n) - 1)
    prod = np.zeros_like(ys)
    for shift in range(0, 64, 16):
        limb = (ys >> np.uint64(shift)) & np.uint64(0xFFFF)
        term = (limb * np.uint64(xv & 0xFFFFFFFFFFFF)) & mask if n <= 48 else None
        if term is None:
            raise ValueError("n too large for this helper")
        prod = (prod + ((term << np.uint64(shift)) & mask)) & mask
    frac = prod.astype(np.float64) / float(1 << n)
    return (2.0 ** (-n / 2.0)) * np.exp(2j * np.pi * frac)


def qft_state(n: int, x: int) -> np.ndarray:
    return qft_amplitudes(n, x, np.arange(1 << n, dtype=np.uint64))


def grover_amplitudes(n: int, rounds: int) -> tuple:
    """(marked amplitude, every other amplitude) after `rounds` Grover rounds from H|0...0> whose
    diffusion is H(I - 2|0><0|)H = I - 2|s><s| (the textbook operator times -1): with
    sin t = 2^(-n/2), the textbook iterate rotates by 2t in span{|m>, |m_perp>}, and the extra
    sign gives (-1)^r sin((2r+1)t) on |m> and (-1)^r cos((2r+1)t)/sqrt(2^n - 1) elsewhere."""
    t = math.asin(2.0 ** (-n / 2))
    sgn = -1.0 if rounds % 2 else 1.0
    return sgn * math.sin((2 * rounds + 1) * t), sgn * math.cos((2 * rounds + 1) * t) / math.sqrt(2.0 ** n - 1)
