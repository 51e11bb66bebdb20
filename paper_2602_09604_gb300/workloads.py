"""Seeded synthetic circuits (input data only; no simulation arithmetic lives here).

Both the CUDA path and the complex128 oracle consume these gate lists; this module is the only
thing they share.  Each gate is a :class:`Gate` with fp64 complex matrices.

Conventions (the paper fixes the gate kinds of its five benchmarks in section V but not their
exact layout; the readings below are this library's):

* amplitude index bit q <-> qubit q; a gate's local matrix index bit j <-> ``targets[j]``;
* grid qubits are numbered row-major over the kept sites, q = r * cols + c before any removal;
* coupler patterns on a rectangular grid: A = horizontal (r,c)-(r,c+1) with c even,
  B = horizontal with c odd, C = vertical (r,c)-(r+1,c) with r even, D = vertical with r odd;
  cycle i uses pattern "ABCDCDAB"[i % 8];
* a cycle is one single-qubit layer (sqrt(X), sqrt(Y), sqrt(W); the first cycle draws uniformly
  from all three, later cycles from the two that differ from that qubit's previous gate) followed
  by one fSim(pi/2, pi/6) layer on the cycle's couplers;
* sqrt(G) for G in {X, Y, W=(X+Y)/sqrt(2)} is the principal square root,
  (1+i)/2 * I + (1-i)/2 * G (G has eigenvalues +-1, and the principal root of -1 is i);
* QFT (section V): for j = n-1 .. 0: H(j), then CP(2 pi / 2^(j-m+1)) on (m, j) for m = j-1 .. 0;
  then SWAP(q, n-1-q) for q < n/2.  Its closed form is QFT|x> = 2^(-n/2) sum_y e^{+2 pi i x y/2^n}|y>.
* GHZ (section V): H on qubit 0, then CNOT(control q, target q+1) for q = 0 .. n-2.
* hardware-efficient ansatz: per layer RZ(phi) then RY(theta) on every qubit (angles uniform on
  [0, 2 pi)), then a CZ ladder CZ(q, q+1) for q = 0 .. n-2.
* Grover (section V): H on every qubit, then per round an oracle (X on the qubits where the
  marked index has a 0, a Z on qubit n-1 controlled by qubits 0 .. n-2, the same X layer) and a
  diffusion (H, X on every qubit, the same multi-controlled Z, X, H).  The diffusion is
  H (I - 2|0><0|) H = I - 2|s><s|, the textbook operator times -1 (the oracle's closed form
  follows from that).
* Quantum volume (section V): `depth` layers (default n); each draws a random permutation of the
  qubits and, on every pair (p[2i], p[2i+1]), applies Haar-random single-qubit unitaries and
  CNOTs: (A1, A2), CNOT, (B1, B2), CNOT, (C1, C2), CNOT, (D1, D2), CNOT controlled by the first.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
W = (X + Y) / math.sqrt(2.0)


def principal_sqrt_pm1(G: np.ndarray) -> np.ndarray:
    """Principal square root of an involution G (eigenvalues +-1): (1+i)/2 I + (1-i)/2 G."""
    return 0.5 * (1 + 1j) * I2 + 0.5 * (1 - 1j) * G


SQRT_X = principal_sqrt_pm1(X)
SQRT_Y = principal_sqrt_pm1(Y)
SQRT_W = principal_sqrt_pm1(W)
ONE_QUBIT_SET = (("sqrt_x", SQRT_X), ("sqrt_y", SQRT_Y), ("sqrt_w", SQRT_W))


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def cphase(lam: float) -> np.ndarray:
    return np.diag([1, 1, 1, np.exp(1j * lam)]).astype(np.complex128)


SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)


def ry(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(phi: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)]).astype(np.complex128)


@dataclass(frozen=True)
class Gate:
    targets: tuple
    matrix: np.ndarray = field(compare=False, repr=False)
    controls: tuple = ()
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.targets)

    def dagger(self) -> "Gate":
        return Gate(self.targets, np.ascontiguousarray(self.matrix.conj().T), self.controls, self.name + "^dg")


def inverse(gates) -> list:
    return [g.dagger() for g in reversed(list(gates))]


# ----------------------------------------------------------------------------- grid random circuits
@dataclass(frozen=True)
class Grid:
    rows: int
    cols: int
    dropped: tuple = ()          # (r, c) sites removed from the grid

    def sites(self):
        return [(r, c) for r in range(self.rows) for c in range(self.cols) if (r, c) not in self.dropped]

    def qubit_of(self):
        return {s: q for q, s in enumerate(self.sites())}

    @property
    def n(self) -> int:
        return len(self.sites())


def coupler_pattern(grid: Grid, pattern: str):
    qo = grid.qubit_of()
    out = []
    for r in range(grid.rows):
        for c in range(grid.cols):
            if pattern in "AB":
                if c + 1 < grid.cols and (c % 2 == (0 if pattern == "A" else 1)):
                    a, b = (r, c), (r, c + 1)
                else:
                    continue
            else:
                if r + 1 < grid.rows and (r % 2 == (0 if pattern == "C" else 1)):
                    a, b = (r, c), (r + 1, c)
                else:
                    continue
            if a in qo and b in qo:
                out.append(tuple(sorted((qo[a], qo[b]))))
    return out


PATTERN_SEQUENCE = "ABCDCDAB"
GRID_16 = Grid(4, 4)
GRID_28 = Grid(4, 7)
GRID_30 = Grid(5, 6)
GRID_32 = Grid(4, 8)
GRID_33 = Grid(6, 6, dropped=((5, 3), (5, 4), (5, 5)))


def random_grid_circuit(grid: Grid, cycles: int, seed: int, theta: float = math.pi / 2,
                        phi: float = math.pi / 6) -> list:
    rng = np.random.default_rng(seed)
    n = grid.n
    prev = [-1] * n
    fs = fsim(theta, phi)
    gates = []
    for cyc in range(cycles):
        for q in range(n):
            if prev[q] < 0:
                choice = int(rng.integers(0, 3))
            else:
                others = [i for i in range(3) if i != prev[q]]
                choice = others[int(rng.integers(0, 2))]
            prev[q] = choice
            name, m = ONE_QUBIT_SET[choice]
            gates.append(Gate((q,), m, (), name))
        for a, b in coupler_pattern(grid, PATTERN_SEQUENCE[cyc % len(PATTERN_SEQUENCE)]):
            gates.append(Gate((a, b), fs, (), "fsim"))
    return gates


# ----------------------------------------------------------------------------- textbook circuits
def qft_circuit(n: int) -> list:
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate((j,), H, (), "h"))
        for m in range(j - 1, -1, -1):
            gates.append(Gate((m, j), cphase(2 * math.pi / 2 ** (j - m + 1)), (), "cp"))
    for q in range(n // 2):
        gates.append(Gate((q, n - 1 - q), SWAP, (), "swap"))
    return gates


def ghz_circuit(n: int, controlled: bool = True) -> list:
    """H(0) then CNOT chain.  With controlled=True the CNOT is X with a control qubit (exercises
    control folding); otherwise it is the dense 4x4 on (control, target)."""
    gates = [Gate((0,), H, (), "h")]
    cnot_dense = np.array([[1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0], [0, 1, 0, 0]], dtype=np.complex128)
    for q in range(n - 1):
        if controlled:
            gates.append(Gate((q + 1,), X, (q,), "cnot"))
        else:
            gates.append(Gate((q, q + 1), cnot_dense, (), "cnot"))   # local bit0=control q
    return gates


def hea_circuit(n: int, layers: int, rng: np.random.Generator) -> list:
    gates = []
    for _ in range(layers):
        for q in range(n):
            phi = float(rng.uniform(0, 2 * math.pi))
            theta = float(rng.uniform(0, 2 * math.pi))
            gates.append(Gate((q,), rz(phi), (), "rz"))
            gates.append(Gate((q,), ry(theta), (), "ry"))
        for q in range(n - 1):
            gates.append(Gate((q, q + 1), CZ, (), "cz"))
    return gates


def hea_batch(count: int = 256, n_lo: int = 10, n_hi: int = 20, layers: int = 8, seed: int = 5):
    """[(n, gates)] for `count` independent circuits with n ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [(int(n), hea_circuit(int(n), layers, rng)) for n in ns]


# ----------------------------------------------------------------------------- random unitaries
def grover_circuit(n: int, marked: int, rounds: int) -> list:
    assert n >= 2 and 0 <= marked < (1 << n)
    mcz = Gate((n - 1,), Z, tuple(range(n - 1)), "mcz")
    gates = [Gate((q,), H, (), "h") for q in range(n)]
    for _ in range(rounds):
        flips = [Gate((q,), X, (), "x") for q in range(n) if not (marked >> q) & 1]
        gates += flips + [mcz] + flips
        gates += [Gate((q,), H, (), "h") for q in range(n)] + [Gate((q,), X, (), "x") for q in range(n)]
        gates += [mcz]
        gates += [Gate((q,), X, (), "x") for q in range(n)] + [Gate((q,), H, (), "h") for q in range(n)]
    return gates


def qv_circuit(n: int, depth: int | None = None, seed: int = 0) -> list:
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(n if depth is None else depth):
        perm = [int(q) for q in rng.permutation(n)]
        for i in range(n // 2):
            a, b = perm[2 * i], perm[2 * i + 1]
            for layer in range(4):
                gates.append(Gate((a,), random_unitary(2, rng), (), "u"))
                gates.append(Gate((b,), random_unitary(2, rng), (), "u"))
                if layer < 3:
                    gates.append(Gate((b,), X, (a,), "cx"))
    return gates


def random_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitary: QR of a complex Gaussian matrix with the phases of R's diagonal removed."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_gate(n: int, k: int, rng: np.random.Generator, targets=None) -> Gate:
    if targets is None:
        targets = tuple(int(t) for t in rng.choice(n, size=k, replace=False))
    return Gate(tuple(targets), random_unitary(1 << k, rng), (), f"rand{k}")


def random_state(n: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# named workloads ------------------------------------------------------------------------------
def circuit_16q():
    """4x4 grid, 14 cycles, seed 1 (308 gates)."""
    return GRID_16.n, random_grid_circuit(GRID_16, 14, seed=1)


def circuit_30q_grid(cycles: int = 20, seed: int = 2):
    return GRID_30.n, random_grid_circuit(GRID_30, cycles, seed=seed)


def qft_basis_index(n: int, seed: int) -> int:
    return int(np.random.default_rng(seed).integers(0, 1 << n))
