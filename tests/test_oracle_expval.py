"""Pins for the oracle's Pauli expectation value <psi|P|psi> (the ExpectationValue routine of
section IV read as an expectation value): brute force with the full 2^n x 2^n Kronecker matrix
(independent of the oracle's gate loop), closed forms on basis, uniform, GHZ and |+i> states,
Hermiticity, the identity string, and a planted sign mistake in Y.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import binding as bm
from paper_2602_09604_gb300 import workloads as wl

P1 = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
      "Z": np.array([[1, 0], [0, -1]])}


def kron_string(n, terms):
    """Full matrix of the string: qubit q acts on bit q, so qubit 0 is the rightmost factor."""
    m = np.eye(1, dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        m = np.kron(m, P1[terms.get(q, "I")])
    return m


def random_terms(n, rng):
    return {int(q): "IXYZ"[int(rng.integers(0, 4))] for q in range(n) if rng.random() < 0.6}


@pytest.mark.parametrize("n", [1, 3, 5])
def test_brute_force_kronecker(n):
    rng = np.random.default_rng(40 + n)
    psi = wl.random_state(n, rng).astype(np.complex128)
    for _ in range(30):
        t = random_terms(n, rng)
        want = np.vdot(psi, kron_string(n, t) @ psi)
        got = oracle.expval_pauli(psi, n, t)
        assert abs(got - want) <= 1e-12, t


def test_basis_states():
    n = 6
    for x in (0, 1, 0b101101, 63):
        psi = oracle.basis_state(n, x)
        for zs in (0b1, 0b110, 0b101011, 0b111111):
            t = {q: "Z" for q in range(n) if (zs >> q) & 1}
            assert oracle.expval_pauli(psi, n, t) == pytest.approx((-1) ** bin(x & zs).count("1"))
        assert oracle.expval_pauli(psi, n, {2: "X"}) == 0
        assert oracle.expval_pauli(psi, n, {0: "Y", 4: "Z"}) == 0


def test_uniform_state():
    n = 5
    psi = closed_forms.uniform(n)
    assert oracle.expval_pauli(psi, n, {0: "X", 3: "X", 4: "X"}) == pytest.approx(1.0)
    assert oracle.expval_pauli(psi, n, {1: "Y"}) == pytest.approx(0.0)
    assert oracle.expval_pauli(psi, n, {2: "Z"}) == pytest.approx(0.0)


def test_ghz_correlations():
    n = 4
    psi = closed_forms.ghz(n)
    ev = lambda t: oracle.expval_pauli(psi, n, t)
    assert ev({0: "Z", 3: "Z"}) == pytest.approx(1.0)
    assert ev({0: "Z"}) == pytest.approx(0.0)
    assert ev({q: "X" for q in range(n)}) == pytest.approx(1.0)
    assert ev({0: "Y", 1: "Y", 2: "X", 3: "X"}) == pytest.approx(-1.0)
    assert ev({q: "Y" for q in range(n)}) == pytest.approx(1.0)


def test_plus_i_state_fixes_the_sign_of_y():
    psi = np.array([1, 1j]) / np.sqrt(2)
    assert oracle.expval_pauli(psi, 1, {0: "Y"}) == pytest.approx(1.0)
    assert oracle.expval_pauli(psi, 1, {0: "X"}) == pytest.approx(0.0)
    assert oracle.expval_pauli(psi, 1, {0: "Z"}) == pytest.approx(0.0)


def test_hermitian_and_identity():
    n = 7
    rng = np.random.default_rng(3)
    psi = 1.7 * wl.random_state(n, rng).astype(np.complex128)
    for _ in range(20):
        assert abs(oracle.expval_pauli(psi, n, random_terms(n, rng)).imag) <= 1e-12
    assert oracle.expval_pauli(psi, n, {}) == pytest.approx(oracle.norm(psi))


def test_planted_y_sign_is_caught(monkeypatch):
    monkeypatch.setitem(oracle.PAULI, "Y", np.conj(oracle.PAULI["Y"]))
    psi = np.array([1, 1j]) / np.sqrt(2)
    assert oracle.expval_pauli(psi, 1, {0: "Y"}) != pytest.approx(1.0)
    n = 3
    psi = wl.random_state(n, np.random.default_rng(1)).astype(np.complex128)
    t = {0: "Y", 2: "X"}
    assert abs(oracle.expval_pauli(psi, n, t) - np.vdot(psi, kron_string(n, t) @ psi)) > 1e-6


def test_mask_encoding():
    assert bm.pauli_masks({0: "X", 3: "Y", 5: "Z", 7: "I"}) == (0b1001, 0b101000)
    with pytest.raises(ValueError):
        bm.pauli_masks({0: "Q"})
