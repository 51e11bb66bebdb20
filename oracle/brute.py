"""Brute-force full-unitary simulation for tiny n (n <= 10).  TEST INFRASTRUCTURE ONLY.

An independent construction of the same physics as ``sv_oracle.c``: instead of looping over
amplitude groups (Eq. 3), every gate is embedded into the full 2^n x 2^n operator with Kronecker
products (Eq. 4: gates on disjoint qubits compose by tensor product) and a basis permutation, the
operators are multiplied together, and the product is applied to the initial vector.  A mistake
in either construction (bit order, operand order, a missed target) shows up as disagreement.
"""
from __future__ import annotations

import numpy as np


def controlled_matrix(U: np.ndarray, n_controls: int) -> np.ndarray:
    """Matrix on (targets..., controls...) local bits: U where every control bit is 1, else I.

    Local index = t + 2^k * c with t the target part and c the control part (controls above)."""
    k = int(U.shape[0]).bit_length() - 1
    if n_controls == 0:
        return np.array(U, dtype=np.complex128)
    dim = 1 << (k + n_controls)
    M = np.eye(dim, dtype=np.complex128)
    all_on = (1 << n_controls) - 1
    lo = all_on << k
    M[lo:lo + (1 << k), lo:lo + (1 << k)] = U
    return M


def permutation_matrix(n: int, order) -> np.ndarray:
    """P with P|i> = |i'>, where bit j of i' is bit order[j] of i (order is a permutation of 0..n-1)."""
    N = 1 << n
    P = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        ip = 0
        for j, q in enumerate(order):
            ip |= ((i >> q) & 1) << j
        P[ip, i] = 1.0
    return P


def full_operator(n: int, gate) -> np.ndarray:
    """2^n x 2^n operator of one gate: P^T (I_rest (x) U_local) P."""
    qubits = list(gate.targets) + list(gate.controls)
    U = controlled_matrix(np.asarray(gate.matrix, dtype=np.complex128), len(gate.controls))
    rest = [q for q in range(n) if q not in qubits]
    order = qubits + rest                       # new bit j <- old qubit order[j]
    P = permutation_matrix(n, order)
    big = np.kron(np.eye(1 << len(rest), dtype=np.complex128), U)   # U acts on the low new bits
    return P.conj().T @ big @ P


def circuit_unitary(n: int, gates) -> np.ndarray:
    W = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        W = full_operator(n, g) @ W
    return W


def run_circuit(n: int, gates, init_index: int = 0) -> np.ndarray:
    if n > 10:
        raise ValueError("brute force is for n <= 10")
    W = circuit_unitary(n, gates)
    return W[:, init_index].copy()


def apply_1q_tensordot(psi: np.ndarray, n: int, q: int, U: np.ndarray) -> np.ndarray:
    """Special case: a one-qubit gate on qubit q, as a tensordot over the reshaped state.

    Viewing the state as an array of shape (2^(n-q-1), 2, 2^q), axis 1 is bit q."""
    t = np.asarray(psi, dtype=np.complex128).reshape(1 << (n - q - 1), 2, 1 << q)
    out = np.einsum("ab,ibj->iaj", np.asarray(U, dtype=np.complex128), t)
    return out.reshape(-1)
