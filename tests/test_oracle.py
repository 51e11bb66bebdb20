"""Pins for the complex128 oracle: brute force, closed forms, invariants, paper-printed numbers.

Every test here is CPU-only.  The pins are chosen so that a transposed matrix, a reversed target
order, a conjugated gate, a dropped control or a wrong sign fails at least one of them (the last
test plants each of those mistakes and checks that it is caught)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute, closed_forms
from paper_2602_09604_gb300 import workloads as wl
from paper_2602_09604_gb300 import costs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def _random_gates(n, count, rng, kmax=4, with_controls=True):
    gates = []
    for _ in range(count):
        k = int(rng.integers(1, min(kmax, n) + 1))
        qs = [int(q) for q in rng.permutation(n)]
        targets = tuple(qs[:k])
        nc = int(rng.integers(0, min(2, n - k) + 1)) if with_controls else 0
        controls = tuple(qs[k:k + nc])
        gates.append(wl.Gate(targets, wl.random_unitary(1 << k, rng), controls, "r"))
    return gates


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9])
def test_oracle_matches_brute_force(n):
    rng = np.random.default_rng(100 + n)
    gates = _random_gates(n, 12, rng)
    init = int(rng.integers(0, 1 << n))
    a = oracle.run_circuit(n, gates, init)
    b = brute.run_circuit(n, gates, init)
    assert np.max(np.abs(a - b)) < 1e-12


def test_oracle_threads_do_not_change_result():
    rng = np.random.default_rng(7)
    n = 12
    gates = _random_gates(n, 10, rng, kmax=3)
    a = oracle.run_circuit(n, gates, 5, threads=1)
    b = oracle.run_circuit(n, gates, 5, threads=4)
    assert np.array_equal(a, b)


def test_cnot_index_convention_by_hand():
    # CNOT with control qubit 0 and target qubit 1: |q1 q0> = |01> (index 1) -> |11> (index 3)
    g = wl.Gate((1,), wl.X, (0,), "cnot")
    for init, expect in [(0, 0), (1, 3), (2, 2), (3, 1)]:
        psi = oracle.run_circuit(2, [g], init)
        assert abs(psi[expect] - 1.0) < 1e-15 and np.sum(np.abs(psi) ** 2) == pytest.approx(1.0)
    # the same gate written densely on targets (0, 1): local bit 0 = qubit 0 = control
    dense = wl.ghz_circuit(2, controlled=False)[1]
    for init, expect in [(0, 0), (1, 3), (2, 2), (3, 1)]:
        psi = oracle.run_circuit(2, [dense], init)
        assert abs(psi[expect] - 1.0) < 1e-15


def test_target_order_is_local_bit_order():
    rng = np.random.default_rng(3)
    U = wl.random_unitary(4, rng)
    # swapping local bits 0 and 1 of the matrix == swapping the target list
    perm = [0, 2, 1, 3]
    Up = U[np.ix_(perm, perm)]
    n = 5
    psi0 = wl.random_state(n, rng)
    a = oracle.run_circuit(n, [wl.Gate((1, 4), U)], psi=psi0.copy())
    b = oracle.run_circuit(n, [wl.Gate((4, 1), Up)], psi=psi0.copy())
    assert np.max(np.abs(a - b)) < 1e-13
    c = oracle.run_circuit(n, [wl.Gate((4, 1), U)], psi=psi0.copy())
    assert np.max(np.abs(a - c)) > 1e-3


@pytest.mark.parametrize("n", [1, 4, 9])
def test_one_qubit_gate_equals_tensordot(n):
    rng = np.random.default_rng(11 + n)
    psi0 = wl.random_state(n, rng)
    for q in range(n):
        U = wl.random_unitary(2, rng)
        a = oracle.run_circuit(n, [wl.Gate((q,), U)], psi=psi0.copy())
        b = brute.apply_1q_tensordot(psi0, n, q, U)
        assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("n", [1, 3, 10, 14])
def test_hadamard_everywhere_is_uniform(n):
    psi = oracle.run_circuit(n, [wl.Gate((q,), wl.H) for q in range(n)], 0)
    assert np.max(np.abs(psi - closed_forms.uniform(n))) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 8, 13])
@pytest.mark.parametrize("controlled", [True, False])
def test_bell_and_ghz(n, controlled):
    gates = wl.ghz_circuit(n, controlled=controlled)
    assert len(gates) == n
    psi = oracle.run_circuit(n, gates, 0)
    assert np.max(np.abs(psi - closed_forms.ghz(n))) < 1e-15


def test_qft_closed_form_helper_is_the_dft():
    # reduces to the textbook DFT: sqrt(N) * ifft(e_x)
    for n in (1, 3, 6, 11):
        N = 1 << n
        for x in (0, 1, N - 1, N // 3):
            e = np.zeros(N, dtype=np.complex128)
            e[x] = 1
            ref = math.sqrt(N) * np.fft.ifft(e)
            assert np.max(np.abs(closed_forms.qft_state(n, x) - ref)) < 1e-12
    # exact phase reduction at large n: y = 2^(n-1), x odd -> phase pi
    n = 34
    amp = closed_forms.qft_amplitudes(n, 3, [1 << (n - 1)])[0]
    assert abs(amp - (-(2.0 ** (-n / 2)))) < 1e-20


@pytest.mark.parametrize("n", [1, 2, 5, 10, 13])
def test_qft_circuit_matches_closed_form(n):
    gates = wl.qft_circuit(n)
    assert len(gates) == n + n * (n - 1) // 2 + n // 2
    x = wl.qft_basis_index(n, seed=n)
    psi = oracle.run_circuit(n, gates, x)
    assert np.max(np.abs(psi - closed_forms.qft_state(n, x))) < 1e-12


def test_norm_and_unitarity_invariants():
    rng = np.random.default_rng(21)
    n = 11
    gates = _random_gates(n, 20, rng, kmax=5)
    psi = oracle.run_circuit(n, gates, 17)
    assert oracle.norm(psi) == pytest.approx(1.0, abs=1e-13)
    exact = math.fsum((psi.real ** 2 + psi.imag ** 2).tolist())
    assert abs(oracle.norm(psi) - exact) <= (1 << n) * 2.2e-16
    back = oracle.run_circuit(n, wl.inverse(gates), psi=psi.copy())
    e = np.zeros(1 << n, dtype=np.complex128)
    e[17] = 1
    assert np.max(np.abs(back - e)) < 1e-13


def test_norm_c64_widening():
    rng = np.random.default_rng(5)
    psi = wl.random_state(8, rng).astype(np.complex64)
    ref = float(np.sum(psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2))
    assert oracle.norm(psi) == pytest.approx(ref, rel=1e-15)


def test_sample_inverse_cdf_by_hand():
    psi = np.sqrt(np.array([0.1, 0.2, 0.3, 0.4])).astype(np.complex128)
    u = np.array([0.0, 0.0999, 0.35, 0.61, 0.99, 0.5999])
    out = oracle.sample(psi, u)
    assert out.tolist() == [0, 0, 2, 3, 3, 2]
    # exact boundary: cumsum_0 = 0.25 is not > 0.25, so index 1
    psi2 = np.full(4, 0.5, dtype=np.complex128)
    assert oracle.sample(psi2, np.array([0.25, 0.2499999, 0.75]))[:].tolist() == [1, 0, 3]


def test_sample_ghz_and_chi_square():
    from scipy import stats
    n = 10
    psi = oracle.run_circuit(n, wl.ghz_circuit(n), 0)
    rng = np.random.default_rng(9)
    u = rng.random(20000)
    out = oracle.sample(psi, u)
    assert set(np.unique(out).tolist()) <= {0, (1 << n) - 1}
    frac = np.mean(out == 0)
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / u.size)
    # chi-square on a random 6-qubit state
    p = oracle.probabilities(wl.random_state(6, rng))
    psi6 = np.sqrt(p).astype(np.complex128)
    u = rng.random(200000)
    counts = np.bincount(oracle.sample(psi6, u).astype(np.int64), minlength=64)
    chi = stats.chisquare(counts, p / p.sum() * u.size)
    assert chi.pvalue > 1e-4


def test_fidelity_and_error_metrics():
    rng = np.random.default_rng(2)
    a = wl.random_state(6, rng)
    assert oracle.fidelity(a, a * np.exp(0.7j)) == pytest.approx(1.0, abs=1e-14)
    assert oracle.l2_error(a, a) == 0.0
    b = wl.random_state(6, rng)
    assert oracle.fidelity(a, b) == pytest.approx(abs(np.vdot(a, b)) ** 2, rel=1e-12)


def test_paper_printed_numbers():
    gold = json.load(open(GOLDEN))
    Hp = np.array(gold["hadamard"]["matrix_times_sqrt2"], dtype=float) / math.sqrt(2)
    assert np.allclose(wl.H, Hp, atol=1e-15)
    assert costs.flops_per_group(gold["flops_per_group_1q"]["k"]) == gold["flops_per_group_1q"]["flops"]
    nv = gold["arithmetic_intensity"]["num_vals"]
    for case in gold["arithmetic_intensity"]["cases"]:
        assert abs(costs.ai_paper(case["f"], nv) - case["ai"]) <= case["abs_tol"]
    for n in (5, 16, 30, 34):
        assert costs.state_bytes(n) == 2 ** (n + gold["memory_bytes"]["log2_bytes_minus_n"])
    assert len(wl.ghz_circuit(17)) == 17 * gold["ghz_gate_count"]["gates_per_qubit"]


def test_gate_library_definitions():
    for G, R in ((wl.X, wl.SQRT_X), (wl.Y, wl.SQRT_Y), (wl.W, wl.SQRT_W)):
        assert np.allclose(R @ R, G, atol=1e-15)
        assert np.allclose(R.conj().T @ R, np.eye(2), atol=1e-15)
        assert np.all(np.linalg.eigvals(R).real >= -1e-15)      # principal root
    F = wl.fsim(math.pi / 2, math.pi / 6)
    assert np.allclose(F.conj().T @ F, np.eye(4), atol=1e-15)
    assert np.allclose(wl.ry(0.3) @ wl.ry(-0.3), np.eye(2))
    # RY(theta) = exp(-i theta Y / 2), RZ(phi) = exp(-i phi Z / 2)
    from scipy.linalg import expm
    assert np.allclose(wl.ry(0.9), expm(-0.45j * wl.Y), atol=1e-14)
    assert np.allclose(wl.rz(1.3), expm(-0.65j * wl.Z), atol=1e-14)


def test_planted_mistakes_are_caught():
    """Each plausible oracle mistake, planted on the CPU, fails a pin above."""
    rng = np.random.default_rng(77)
    n = 6
    gates = _random_gates(n, 8, rng, kmax=3)
    good = brute.run_circuit(n, gates, 3)

    def differs(bad_gates):
        return np.max(np.abs(oracle.run_circuit(n, bad_gates, 3) - good)) > 1e-6

    assert differs([wl.Gate(g.targets, g.matrix.T, g.controls) for g in gates])            # transposed
    assert differs([wl.Gate(g.targets[::-1], g.matrix, g.controls) for g in gates])        # bit order
    assert differs([wl.Gate(g.targets, g.matrix.conj(), g.controls) for g in gates])       # conjugated
    assert differs([wl.Gate(g.targets, g.matrix, ()) for g in gates])                      # dropped control
    # a sign error in the QFT phase fails the closed form
    x = 5
    bad = [wl.Gate(g.targets, g.matrix.conj(), g.controls) if g.name == "cp" else g for g in wl.qft_circuit(5)]
    assert np.max(np.abs(oracle.run_circuit(5, bad, x) - closed_forms.qft_state(5, x))) > 1e-3


# Hand-computed values for the acceptance metrics (F = |<ref|psi>|^2 / (||ref||^2 ||psi||^2) and
# ||psi - ref||_2, the bar the GPU path is held to).  Each value below was worked out on paper.
_L2_CASES = [
    ([1, 0], [0, 1], math.sqrt(2)),                 # |0> vs |1>: sqrt(1 + 1)
    ([1, 0], [1j, 0], math.sqrt(2)),                # |i - 1| = sqrt(2)
    ([0], [3 + 4j], 5.0),                           # a single 3-4-5 amplitude
    ([1, 1j], [1j, 1], 2.0),                        # |i - 1|^2 + |1 - i|^2 = 4
    ([0.5, 0.5, 0.5, 0.5], [0.5, 0.5, 0.5, -0.5], 1.0),   # one sign flipped: |-1| = 1
]
_F_CASES = [
    ([1, 0], [1, 1], 0.5),                          # F(|0>, |+>) = 1/2 (|+> unnormalised)
    ([1, 0], [0, 1], 0.0),                          # orthogonal
    ([1, 1j], [1, 1j], 1.0),                        # the same state: conj matters (no conj gives 0)
    ([1, 1j], [1, 1], 0.5),                         # <a|b> = 1 - i: |1 - i|^2 / (2 * 2) = 2/4
    ([2, 0, 0], [0.5, 0.5 * math.sqrt(3), 0], 0.25),   # cos^2(pi/3), ref not normalised
    ([1, 0], [1j, 0], 1.0),                         # a global phase does not count
]


@pytest.mark.parametrize("a,b,want", _L2_CASES)
def test_l2_error_hand_values(a, b, want):
    assert oracle.l2_error(np.array(a, complex), np.array(b, complex)) == pytest.approx(want, abs=1e-15)
    assert oracle.l2_error(np.array(b, complex), np.array(a, complex)) == pytest.approx(want, abs=1e-15)


@pytest.mark.parametrize("a,b,want", _F_CASES)
def test_fidelity_hand_values(a, b, want):
    assert oracle.fidelity(np.array(a, complex), np.array(b, complex)) == pytest.approx(want, abs=1e-15)
    assert oracle.fidelity(np.array(b, complex), np.array(a, complex)) == pytest.approx(want, abs=1e-15)


def test_metric_mistakes_are_caught():
    """Plausible mistakes in the two metrics, planted here on the CPU, each fail a hand value."""
    def l2_no_sqrt(a, b):                      # squared norm
        return float(np.sum(np.abs(np.asarray(b) - np.asarray(a)) ** 2))

    def l2_max(a, b):                          # max-norm instead of the 2-norm
        return float(np.max(np.abs(np.asarray(b) - np.asarray(a))))

    def l2_real_only(a, b):                    # imaginary parts dropped
        return float(np.linalg.norm(np.real(np.asarray(b) - np.asarray(a))))

    def f_no_conj(a, b):                       # <a|b> without the conjugate
        a, b = np.asarray(a, complex), np.asarray(b, complex)
        return float(abs(np.dot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))

    def f_no_norm(a, b):                       # overlap not normalised
        return float(abs(np.vdot(np.asarray(a, complex), np.asarray(b, complex))) ** 2)

    def f_no_square(a, b):                     # |<a|b>| instead of its square
        a, b = np.asarray(a, complex), np.asarray(b, complex)
        return float(abs(np.vdot(a, b)) / math.sqrt(np.vdot(a, a).real * np.vdot(b, b).real))

    for bad in (l2_no_sqrt, l2_max, l2_real_only):
        assert any(abs(bad(np.array(a, complex), np.array(b, complex)) - w) > 1e-6 for a, b, w in _L2_CASES), bad
    for bad in (f_no_conj, f_no_norm, f_no_square):
        assert any(abs(bad(np.array(a, complex), np.array(b, complex)) - w) > 1e-6 for a, b, w in _F_CASES), bad
