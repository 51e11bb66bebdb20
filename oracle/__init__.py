"""Complex128 CPU oracle for the fused-gate state-vector path.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product library never does, and shares no code with it.

Every function here follows the plain definition of the state-vector method (paper section II-A):

* ``apply_gate`` / ``run_circuit`` -- Eq. 3 applied gate by gate, unfused, in circuit order
  (C loop in ``sv_oracle.c``; one OpenMP ``parallel for`` over independent groups at most).
* ``norm`` -- sum of |c_i|^2 (condition under Eq. 1) in fp64.
* ``sample`` -- inverse-CDF lookup of given uniforms in the |c_i|^2 distribution (Eq. 1: |c_i|^2
  is the probability of observing basis state i).
* ``expval_pauli`` -- <psi|P|psi> for a Pauli string P (the ExpectationValue routine of
  section IV, read as an expectation value): each single-qubit Pauli factor applied to a copy of
  psi with ``apply_gate`` (Eq. 3), then the fp64 inner product with psi.
* ``fidelity`` / ``l2_error`` -- the acceptance metrics, fp64.

Conventions: amplitude index bit q <-> qubit q (qubit 0 is the least-significant bit); a gate's
matrix is 2^k x 2^k, row-major, with local index bit j <-> ``gate.targets[j]``; controls act as
"apply only where every control bit is 1" (the sentence after Eq. 3).

Gate objects are duck-typed: anything with ``.targets`` (sequence of int), ``.controls``
(sequence of int, may be empty) and ``.matrix`` (2^k x 2^k complex array).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsv_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only: it runs on x86-64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c_dp = ctypes.POINTER(ctypes.c_double)
        c_ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_apply_gate.argtypes = [c_dp, ctypes.c_int, ctypes.c_int, c_ip, ctypes.c_int,
                                          c_ip, c_dp, ctypes.c_int]
        lib.oracle_apply_gate.restype = ctypes.c_int
        lib.oracle_norm.argtypes = [c_dp, ctypes.c_int]
        lib.oracle_norm.restype = ctypes.c_double
        lib.oracle_norm_c64.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        lib.oracle_norm_c64.restype = ctypes.c_double
        lib.oracle_sample_probs.argtypes = [c_dp, ctypes.c_int64, c_dp, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_sample_probs.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def basis_state(n: int, index: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def apply_gate(psi: np.ndarray, n: int, gate, threads: int = 1) -> None:
    """Apply one (possibly controlled) gate to ``psi`` in place (Eq. 3)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    tg = np.ascontiguousarray(np.asarray(gate.targets, dtype=np.int32))
    ct = np.ascontiguousarray(np.asarray(tuple(gate.controls), dtype=np.int32).reshape(-1))
    if ct.size == 0:
        ct = np.zeros(1, dtype=np.int32)
        nc = 0
    else:
        nc = int(len(gate.controls))
    U = np.ascontiguousarray(np.asarray(gate.matrix, dtype=np.complex128))
    k = len(gate.targets)
    assert U.shape == (1 << k, 1 << k)
    rc = _load().oracle_apply_gate(_dptr(psi.view(np.float64)), n, k,
                                   tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nc,
                                   ct.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   _dptr(U.view(np.float64)), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_apply_gate rejected gate targets={gate.targets} controls={gate.controls}")


def run_circuit(n: int, gates, init_index: int = 0, threads: int = 1, psi: np.ndarray | None = None) -> np.ndarray:
    """Start from |init_index> (or a given state) and apply every gate in order, unfused."""
    if psi is None:
        psi = basis_state(n, init_index)
    for g in gates:
        apply_gate(psi, n, g, threads)
    return psi


def norm(psi: np.ndarray) -> float:
    """sum |c_i|^2 in fp64 (complex128 state, or complex64 state widened exactly)."""
    n = int(psi.size).bit_length() - 1
    if psi.dtype == np.complex64:
        a = np.ascontiguousarray(psi)
        return float(_load().oracle_norm_c64(a.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n))
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().oracle_norm(_dptr(a.view(np.float64)), n))


def probabilities(psi: np.ndarray) -> np.ndarray:
    a = np.asarray(psi).astype(np.complex128)
    return a.real * a.real + a.imag * a.imag


def sample(psi: np.ndarray, uniforms: np.ndarray) -> np.ndarray:
    """out[s] = smallest i with p_0+...+p_i > u_s * sum(p), p = |c|^2 in fp64."""
    p = np.ascontiguousarray(probabilities(psi))
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.zeros(u.size, dtype=np.uint64)
    rc = _load().oracle_sample_probs(_dptr(p), p.size, _dptr(u), u.size,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    assert rc == 0
    return out


PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


class _OneQubit:
    def __init__(self, q, m):
        self.targets = (int(q),)
        self.controls = ()
        self.matrix = m


def expval_pauli(psi: np.ndarray, n: int, terms, threads: int = 1) -> complex:
    """<psi|P|psi> for P = the tensor product of the single-qubit Paulis in ``terms``
    ({qubit: 'X' | 'Y' | 'Z' | 'I'}; identity on every other qubit), complex128, not normalised."""
    phi = np.array(psi, dtype=np.complex128, copy=True)
    for q, s in dict(terms).items():
        apply_gate(phi, n, _OneQubit(q, PAULI[str(s).upper()]), threads)
    return complex(np.vdot(np.asarray(psi, dtype=np.complex128), phi))


def fidelity(psi_ref: np.ndarray, psi: np.ndarray) -> float:
    """F = |<ref|psi>|^2 / (||ref||^2 ||psi||^2), accumulated in fp64."""
    a = np.asarray(psi_ref).astype(np.complex128).ravel()
    b = np.asarray(psi).astype(np.complex128).ravel()
    ov = np.vdot(a, b)
    return float(abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def l2_error(psi_ref: np.ndarray, psi: np.ndarray) -> float:
    """||psi - psi_ref||_2 without phase alignment, fp64."""
    a = np.asarray(psi_ref).astype(np.complex128).ravel()
    b = np.asarray(psi).astype(np.complex128).ravel()
    return float(np.linalg.norm(b - a))
