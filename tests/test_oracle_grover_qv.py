"""Pins for the Grover and quantum-volume workloads (section V) run through the oracle, which also
pin the oracle's handling of many controls: Grover's amplitudes after r rounds have a closed form
(sin / cos of (2r+1)t with sin t = 2^(-n/2)); a Grover circuit whose multi-controlled Z lost one
control misses it; quantum-volume circuits preserve the norm and their inverse returns |0...0>.
CPU only."""
import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import workloads as wl


@pytest.mark.parametrize("n", [3, 5, 8, 10])
def test_grover_closed_form(n):
    marked = (0b1011011011 * 7) % (1 << n)
    for r in range(0, int(np.pi / 4 * 2 ** (n / 2)) + 2):
        psi = oracle.run_circuit(n, wl.grover_circuit(n, marked, r), 0)
        a, b = closed_forms.grover_amplitudes(n, r)
        assert abs(psi[marked] - a) <= 1e-12
        assert np.max(np.abs(np.delete(psi, marked) - b)) <= 1e-12


def test_grover_optimal_rounds_find_the_marked_state():
    n, marked = 10, 613
    r = int(np.floor(np.pi / 4 * 2 ** (n / 2)))
    psi = oracle.run_circuit(n, wl.grover_circuit(n, marked, r), 0)
    assert abs(psi[marked]) ** 2 > 0.99


def test_dropped_control_is_caught():
    n, marked = 6, 22
    gates = []
    for g in wl.grover_circuit(n, marked, 2):
        if g.name == "mcz":
            g = wl.Gate(g.targets, g.matrix, g.controls[1:], "mcz")
        gates.append(g)
    psi = oracle.run_circuit(n, gates, 0)
    a, _ = closed_forms.grover_amplitudes(n, 2)
    assert abs(psi[marked] - a) > 1e-3


@pytest.mark.parametrize("n", [4, 7])
def test_qv_norm_and_inverse(n):
    gates = wl.qv_circuit(n, seed=3)
    assert len(gates) == n * (n // 2) * 11
    psi = oracle.run_circuit(n, gates, 0)
    assert abs(oracle.norm(psi) - 1.0) <= 1e-12
    back = oracle.run_circuit(n, wl.inverse(gates), 0, psi=psi.copy())
    assert abs(back[0] - 1.0) <= 1e-12
