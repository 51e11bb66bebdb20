"""Complex128 states against the complex128 oracle: single fused gates of every k and target
class (with kept controls), random circuits with many-control gates at every fusion size, Grover
and QFT closed forms, layout round trip, norm and sampling, all to ~1e-12 (fp64 arithmetic, so the
two sides differ only by summation order); then the 30-qubit benchmark circuit in complex128 as
the reference for the complex64 tensor-core path at full size."""
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2602_09604_gb300",
                     "cost_model_gb300.bin")


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


def c128_state(n):
    from paper_2602_09604_gb300.state import DeviceState
    return DeviceState(n, c128=True)


def rand_c128(n, rng):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [1, 3, 5, 6, 9, 14])
def test_single_gates_every_k(B, n):
    rng = np.random.default_rng(60 + n)
    psi0 = rand_c128(n, rng)
    for k in range(1, min(n, 6) + 1):
        for _ in range(3):
            g = wl.random_gate(n, k, rng)
            st = c128_state(n)
            st.load(psi0)
            f = B.sv_fuse_circuit([g], n, max_k=6, mode=B.FUSE_NONE)
            st.apply(f)
            got = st.store()
            B.sv_fused_free(f)
            st.free()
            ref = psi0.copy()
            oracle.apply_gate(ref, n, g)
            assert np.max(np.abs(got - ref)) <= 1e-13, (n, k, g.targets)


@pytest.mark.parametrize("n,max_k", [(8, 1), (12, 2), (15, 3), (17, 4), (13, 6)])
def test_random_circuits_with_controls(B, n, max_k):
    rng = np.random.default_rng(n * 3 + max_k)
    gates = []
    for _ in range(80):
        k = int(rng.integers(1, 4))
        nc = int(rng.integers(0, 6)) if rng.random() < 0.4 else 0
        qs = [int(q) for q in rng.permutation(n)]
        gates.append(wl.Gate(tuple(qs[:k]), wl.random_unitary(1 << k, rng), tuple(qs[k:k + nc])))
    st = c128_state(n)
    st.init(5)
    f = B.sv_fuse_circuit(gates, n, max_k=max_k)
    st.apply(f)
    B.sv_fused_free(f)
    got = st.store()
    ref = oracle.run_circuit(n, gates, 5, threads=oracle.default_threads())
    assert np.max(np.abs(got - ref)) <= 1e-12
    assert abs(st.norm() - 1.0) <= 1e-12
    st.free()


def test_grover_and_qft_closed_forms(B):
    n, marked, r = 14, 0x2A5C, 5
    st = c128_state(n)
    st.init(0)
    f = B.sv_fuse_circuit(wl.grover_circuit(n, marked, r), n, max_k=3)
    st.apply(f)
    B.sv_fused_free(f)
    got = st.store()
    a, b = closed_forms.grover_amplitudes(n, r)
    assert abs(got[marked] - a) <= 1e-12
    assert np.max(np.abs(np.delete(got, marked) - b)) <= 1e-12
    x = 9001
    st.init(x)
    f = B.sv_fuse_circuit(wl.qft_circuit(n), n, max_k=4)
    st.apply(f)
    B.sv_fused_free(f)
    got = st.store()
    assert np.max(np.abs(got - closed_forms.qft_state(n, x))) <= 1e-12
    st.free()


def test_layout_norm_and_sampling(B):
    n = 16
    rng = np.random.default_rng(8)
    psi = rand_c128(n, rng) * 1.5
    st = c128_state(n)
    st.load(psi)
    assert np.array_equal(st.store(), psi)                 # exact round trip
    assert abs(st.norm() - oracle.norm(psi)) <= 1e-12
    u = rng.random(512)
    s = st.sample(u)
    want = oracle.sample(psi, u)
    diff = np.nonzero(s != want)[0]
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    for i in diff:   # only where fp64 summation order moves a boundary
        assert abs(cdf[min(s[i], want[i])] - u[i] * cdf[-1]) <= 1e-12
    assert len(diff) <= 2
    st.free()
    with pytest.raises(B.SvError):
        st2 = c128_state(8)
        st2.init(0)
        B.sv_expval_pauli(st2.h, [0], [1])


def test_bench_circuit_c128_reference_for_tensor_cores(B):
    import torch
    from paper_2602_09604_gb300.state import DeviceState
    n, gates = wl.circuit_30q_grid()
    ref = c128_state(n)
    ref.init(0)
    f = B.sv_fuse_circuit(gates, n, max_k=3)
    ref.apply(f)
    B.sv_fused_free(f)
    assert abs(ref.norm() - 1.0) <= 1e-10
    model = B.sv_mlp_load(MODEL) if os.path.exists(MODEL) else None
    kw = dict(max_k=6, precision=B.PREC_BF16X3, tc_min_k=4,
              mode=B.FUSE_LEARNED if model is not None else B.FUSE_GREEDY, model=model)
    st = DeviceState(n)
    st.init(0)
    f = B.sv_fuse_circuit(gates, n, **kw)
    st.apply(f)
    B.sv_fused_free(f)
    ov = torch.zeros((), dtype=torch.complex128, device="cuda")
    d2 = torch.zeros((), dtype=torch.float64, device="cuda")
    nb = torch.zeros((), dtype=torch.float64, device="cuda")
    step = 1 << 26
    for lo in range(0, st.buf.numel(), step):
        a = ref.buf[lo:lo + step].view(-1, 2, 32)
        b = st.buf[lo:lo + step].view(-1, 2, 32).double()
        ca = torch.complex(a[:, 0], a[:, 1])
        cb = torch.complex(b[:, 0], b[:, 1])
        ov += (ca.conj() * cb).sum()
        d2 += ((ca - cb).abs() ** 2).sum()
        nb += (cb.abs() ** 2).sum()
    fid = float(ov.abs() ** 2 / nb)
    err = float(d2.sqrt())
    out = os.environ.get("SV_REPORT_DIR")
    if out:
        import json
        with open(os.path.join(out, "c128_reference_30q.json"), "w") as fh:
            json.dump({"fidelity": fid, "l2_error": err}, fh)
    assert fid >= 1 - 1e-6 and err <= 1e-4, (fid, err)
    if model is not None:
        B.sv_mlp_free(model)
    st.free()
    ref.free()
