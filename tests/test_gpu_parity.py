"""GPU parity: the CUDA path (through the C ABI) against the complex128 oracle.

Tolerances (fp32 state, fp32 fused matrices, fp32 FMA accumulation; the paper's acceptance is
agreement with a reference simulator to 1e-6):
  * fidelity F >= 1 - 1e-6 and ||psi - psi_ref||_2 <= 1e-4 for whole circuits;
  * per element |delta| <= 1e-5 for a single fused gate on a normalised state: each output is a
    2^(k+1)-term fp32 FMA chain over inputs of modulus <= 1, plus one fp32 rounding of the
    matrix, so |delta| <= (2^(k+1) + 2) * 2^-24 ~ 8e-6 at k = 6.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F_TOL = 1e-6
L2_TOL = 1e-4
ELEM_TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_09604_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def DS(B):
    from paper_2602_09604_gb300.state import DeviceState
    return DeviceState


def threads():
    return oracle.default_threads()


def run_gpu(B, DS, n, gates, max_k, init=0, psi0=None, **kw):
    st = DS(n)
    if psi0 is not None:
        st.load(psi0)
    else:
        st.init(init)
    f = B.sv_fuse_circuit(gates, n, max_k=max_k, **kw)
    try:
        st.apply(f)
        out = st.store()
    finally:
        B.sv_fused_free(f)
        st.free()
    return out


def assert_close(ref, got, elem_tol=None):
    F = oracle.fidelity(ref, got)
    err = oracle.l2_error(ref, got)
    assert F >= 1 - F_TOL, (F, err)
    assert err <= L2_TOL, (F, err)
    if elem_tol is not None:
        assert np.max(np.abs(ref - got.astype(np.complex128))) <= elem_tol


def target_sets(n, k, rng):
    """Target sets covering every class: all low (<5), all high (>=5), mixed, edges."""
    sets = []
    if k <= 5 and n >= k:
        sets.append(tuple(int(t) for t in rng.choice(min(5, n), size=k, replace=False)) if min(5, n) >= k else None)
    if n - 5 >= k:
        sets.append(tuple(int(t) for t in 5 + rng.choice(n - 5, size=k, replace=False)))
        sets.append(tuple(range(n - k, n)))                     # topmost qubits
    if n >= 6 and k >= 2:
        lo = int(rng.integers(0, 5))
        rest = [q for q in range(5, n)]
        hi = [int(t) for t in rng.choice(rest, size=min(k - 1, len(rest)), replace=False)]
        t = [lo] + hi
        while len(t) < k:
            t.append(int(rng.choice([q for q in range(5) if q not in t])))
        sets.append(tuple(t))
    sets.append(tuple(int(t) for t in rng.choice(n, size=k, replace=False)))
    return [s for s in sets if s is not None and len(set(s)) == k]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 11, 16, 21])
def test_single_fused_gate_every_k_and_class(B, DS, n):
    rng = np.random.default_rng(1000 + n)
    psi0 = wl.random_state(n, rng).astype(np.complex64)
    for k in range(1, min(6, n) + 1):
        for tg in target_sets(n, k, rng):
            g = wl.random_gate(n, k, rng, targets=tg)
            ref = psi0.astype(np.complex128)
            oracle.apply_gate(ref, n, g)
            got = run_gpu(B, DS, n, [g], max_k=k, psi0=psi0)
            assert_close(ref, got, ELEM_TOL)


@pytest.mark.parametrize("force", ["mixed", "low"])
def test_tile_kernel_on_any_targets(B, DS, force):
    """The shared-memory tile kernel is correct for every target set, not only the ones it is
    chosen for (forced path)."""
    rng = np.random.default_rng(7)
    n = 14
    psi0 = wl.random_state(n, rng).astype(np.complex64)
    path = B.PATH_MIXED if force == "mixed" else B.PATH_LOW
    for k in range(1, 7):
        for tg in target_sets(n, k, rng):
            g = wl.random_gate(n, k, rng, targets=tg)
            ref = psi0.astype(np.complex128)
            oracle.apply_gate(ref, n, g)
            got = run_gpu(B, DS, n, [g], max_k=k, psi0=psi0, force_path=path)
            assert_close(ref, got, ELEM_TOL)


@pytest.mark.parametrize("max_k", [1, 2, 3, 4, 5, 6])
def test_grid_circuit_16q_every_max_k(B, DS, max_k):
    n, gates = wl.circuit_16q()
    ref = oracle.run_circuit(n, gates, 0, threads=threads())
    got = run_gpu(B, DS, n, gates, max_k)
    assert_close(ref, got)


def test_grid_circuit_22q(B, DS):
    n, gates = wl.GRID_16.n, None
    grid = wl.Grid(4, 6)
    n = grid.n - 2          # 22 qubits: drop two corner sites
    grid = wl.Grid(4, 6, dropped=((3, 4), (3, 5)))
    gates = wl.random_grid_circuit(grid, 12, seed=4)
    ref = oracle.run_circuit(n, gates, 0, threads=threads())
    for max_k in (2, 4, 6):
        assert_close(ref, run_gpu(B, DS, n, gates, max_k))


def test_qft_20q_closed_form(B, DS):
    n = 20
    x = wl.qft_basis_index(n, seed=20)
    got = run_gpu(B, DS, n, wl.qft_circuit(n), 5, init=x)
    assert_close(closed_forms.qft_state(n, x), got, ELEM_TOL)


def test_ghz_and_controls(B, DS):
    for n in (3, 9, 24):
        got = run_gpu(B, DS, n, wl.ghz_circuit(n, controlled=True), 4)
        assert_close(closed_forms.ghz(n), got, ELEM_TOL)


def test_hea_circuit_matches_oracle(B, DS):
    rng = np.random.default_rng(55)
    for n in (10, 13, 17):
        gates = wl.hea_circuit(n, 8, rng)
        ref = oracle.run_circuit(n, gates, 0, threads=threads())
        assert_close(ref, run_gpu(B, DS, n, gates, 4))


def test_layout_roundtrip_and_init(B, DS):
    rng = np.random.default_rng(3)
    for n in (1, 4, 5, 6, 13):
        psi = wl.random_state(n, rng).astype(np.complex64)
        st = DS(n)
        st.load(psi)
        assert np.array_equal(st.store(), psi)
        x = int(rng.integers(0, 1 << n))
        st.init(x)
        e = np.zeros(1 << n, dtype=np.complex64)
        e[x] = 1
        assert np.array_equal(st.store(), e)
        st.free()


def test_norm_matches_oracle(B, DS):
    rng = np.random.default_rng(11)
    for n in (1, 3, 5, 9, 17, 22):
        psi = (wl.random_state(n, rng) * (0.5 + rng.random())).astype(np.complex64)
        st = DS(n)
        st.load(psi)
        got = st.norm()
        ref = oracle.norm(psi)       # same complex64 values, widened exactly, fp64 sum
        assert abs(got - ref) <= 1e-12 * max(ref, 1.0), (n, got, ref)
        st.free()


def _check_samples(psi64, u, got):
    """Compare with the oracle on the same complex64 values.  Every GPU sample must be valid (its
    cumulative-probability interval contains u * total, up to fp64 summation-order noise), and it
    may differ from the oracle's only when u * total sits within that noise of a boundary."""
    ref = oracle.sample(psi64, u)
    p = oracle.probabilities(psi64)
    c = np.cumsum(p)
    total = c[-1]
    tol = 1e-12 * total
    t = u * total
    g = got.astype(np.int64)
    lo = np.where(g > 0, c[np.maximum(g - 1, 0)], 0.0)
    hi = c[g]
    assert np.all(lo - tol <= t) and np.all(t < hi + tol)
    bad = np.nonzero(ref != got)[0]
    for s in bad:
        i = int(ref[s])
        edge = min(abs(c[i] - t[s]), abs((c[i - 1] if i else 0.0) - t[s]))
        assert edge <= tol, (s, int(got[s]), i)
    return ref


def test_sample_matches_oracle(B, DS):
    rng = np.random.default_rng(12)
    for n in (1, 4, 5, 12, 16, 19):
        psi = wl.random_state(n, rng).astype(np.complex64)
        st = DS(n)
        st.load(psi)
        u = rng.random(3000)
        u[:4] = [0.0, 0.5, 0.999999999, 1e-300]
        got = st.sample(u)
        _check_samples(psi, u, got)
        st.free()


def test_sample_ghz_and_zero_probability_entries(B, DS):
    n = 20
    st = DS(n)
    st.init(0)
    f = B.sv_fuse_circuit(wl.ghz_circuit(n), n, max_k=4)
    st.apply(f)
    B.sv_fused_free(f)
    u = np.random.default_rng(2).random(4096)
    got = st.sample(u)
    assert set(np.unique(got).tolist()) <= {0, (1 << n) - 1}
    _check_samples(st.store(), u, got)
    st.free()


def test_timing_records(B, DS):
    n, gates = wl.circuit_16q()
    st = DS(n)
    st.init(0)
    f = B.sv_fuse_circuit(gates, n, max_k=3)
    rec = st.apply(f, timings=True)
    assert len(rec) == B.sv_fused_count(f)
    for i, r in enumerate(rec):
        info = B.sv_fused_get_info(f, i)
        assert r["us"] > 0 and r["k"] == info["k"] and r["path"] == info["path"]
        assert r["target_mask"] == sum(1 << t for t in info["targets"])
    B.sv_fused_free(f)
    st.free()


def test_errors_are_reported_not_crashing(B, DS):
    import torch
    buf = torch.empty(64, dtype=torch.float32, device="cuda")
    with pytest.raises(B.SvError) as e:
        B.sv_alloc(10, buf.data_ptr(), buf.numel() * 4, 0)
    assert e.value.code == B.SV_ENOMEM
    with pytest.raises(B.SvError):
        B.sv_alloc(10, buf.data_ptr() + 4, 1 << 20, 0)          # misaligned
    st = DS(6)
    f = B.sv_fuse_circuit([wl.Gate((0,), wl.H)], 7)
    with pytest.raises(B.SvError) as e:
        st.apply(f)
    assert e.value.code == B.SV_ESTATE
    B.sv_fused_free(f)
    with pytest.raises(B.SvError):
        st.sample(np.array([1.5]))
    with pytest.raises(B.SvError):
        B.sv_init(st.h, 1 << 6)
    st.free()


# ------------------------------------------------------------------- full size (30 qubits)
def test_30q_grid_inverse_returns_to_zero(B, DS):
    """At the benchmark's size no complex128 state is kept; the circuit followed by its inverse
    must return |0...0> (unitarity), and the norm must stay 1."""
    n, gates = wl.circuit_30q_grid()
    st = DS(n)
    st.init(0)
    for mk in (4,):
        f = B.sv_fuse_circuit(gates, n, max_k=mk)
        st.apply(f)
        B.sv_fused_free(f)
        assert abs(st.norm() - 1.0) < 1e-4
        fi = B.sv_fuse_circuit(wl.inverse(gates), n, max_k=mk)
        st.apply(fi)
        B.sv_fused_free(fi)
    samples = st.sample(np.linspace(0, 0.999, 64))
    assert np.all(samples == 0)
    import torch
    amp0 = complex(st.buf[0].item(), st.buf[32].item())
    assert abs(amp0) ** 2 >= 1 - 1e-4
    st.free()


def test_30q_qft_sampled_amplitudes(B, DS):
    n = 30
    x = wl.qft_basis_index(n, seed=30)
    st = DS(n)
    st.init(x)
    f = B.sv_fuse_circuit(wl.qft_circuit(n), n, max_k=4)
    st.apply(f)
    B.sv_fused_free(f)
    rng = np.random.default_rng(30)
    idx = rng.integers(0, 1 << n, size=1 << 16).astype(np.uint64)
    import torch
    o = torch.from_numpy(((idx >> np.uint64(5)) << np.uint64(6) | (idx & np.uint64(31))).astype(np.int64)).cuda()
    re = st.buf[o].double().cpu().numpy()
    im = st.buf[o + 32].double().cpu().numpy()
    got = re + 1j * im
    ref = closed_forms.qft_amplitudes(n, x, idx)
    scale = 2.0 ** (n / 2)
    assert np.max(np.abs(got - ref)) * scale < 1e-4      # relative to the amplitude size 2^(-n/2)
    assert abs(st.norm() - 1.0) < 1e-4
    st.free()
