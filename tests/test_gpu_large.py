"""33- and 34-qubit runs (64 GiB and 128 GiB complex64 states): the learned partition against fixed
greedy fusion at every max size, with correctness from properties that hold at any size.

* 33 qubits: 6x6 grid minus sites (5,3), (5,4), (5,5), 24 cycles.  The circuit followed by its
  inverse must return |0...0> (unitarity).
* 34 qubits: QFT of a seeded basis state; sampled amplitudes against the closed form
  2^(-n/2) exp(2 pi i x y / 2^n), and the norm.  The learned partition must beat the best fixed
  size by at least 3% here (the deferred-diagonal order gives fewer passes).
With SV_REPORT_DIR set, the timings go to <SV_REPORT_DIR>/large_runs.json.
"""
import json
import os

import numpy as np
import pytest

from oracle import closed_forms
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2602_09604_gb300",
                     "cost_model_gb300.bin")
REPORT = {}


@pytest.fixture(scope="module")
def env():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    from paper_2602_09604_gb300.state import DeviceState
    m = binding.sv_mlp_load(MODEL)
    yield binding, DeviceState, m
    binding.sv_mlp_free(m)
    out = os.environ.get("SV_REPORT_DIR")
    if out and REPORT:
        with open(os.path.join(out, "large_runs.json"), "w") as fh:
            json.dump(REPORT, fh, indent=1)


def variants(B, m):
    v = [("learned_bf16x3", dict(max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, model=m)),
         ("plain_fp32_k4", dict(max_k=4))]
    v += [(f"greedy_k{k}_bf16x3", dict(max_k=k, precision=B.PREC_BF16X3, tc_min_k=4)) for k in range(2, 7)]
    return v


def time_variants(B, st, n, gates, m, init=0):
    import time
    res = {}
    for label, kw in variants(B, m):
        t0 = time.perf_counter()
        f = B.sv_fuse_circuit(gates, n, **kw)
        fuse_s = time.perf_counter() - t0
        st.init(init)
        rec = st.apply(f, timings=True)
        res[label] = {"device_s": sum(r["us"] for r in rec) / 1e6, "fused_gates": len(rec), "fuse_host_s": fuse_s}
        B.sv_fused_free(f)
    return res


def test_33q_grid_learned_vs_fixed(env):
    B, DS, m = env
    n, gates = wl.GRID_33.n, wl.random_grid_circuit(wl.GRID_33, 24, seed=4)
    assert n == 33
    st = DS(n)
    res = time_variants(B, st, n, gates, m)
    # correctness: learned forward then learned inverse returns |0...0>
    kw = dict(max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, model=m)
    f = B.sv_fuse_circuit(gates, n, **kw)
    fi = B.sv_fuse_circuit(wl.inverse(gates), n, **kw)
    st.init(0)
    st.apply(f)
    norm_fwd = st.norm()
    st.apply(fi)
    amp0 = complex(st.buf[0].item(), st.buf[32].item())
    B.sv_fused_free(f)
    B.sv_fused_free(fi)
    st.free()
    REPORT["grid33"] = {"gates": len(gates), "variants": res, "norm_after_circuit": norm_fwd,
                        "p0_after_inverse": abs(amp0) ** 2}
    assert abs(norm_fwd - 1) < 1e-4
    assert abs(amp0) ** 2 >= 1 - 1e-4
    best_fixed = min(v["device_s"] for k, v in res.items() if k.startswith("greedy"))
    assert res["learned_bf16x3"]["device_s"] <= 1.03 * best_fixed, res
    assert res["learned_bf16x3"]["device_s"] < res["plain_fp32_k4"]["device_s"]


def _qft_samples(st, n, x, seed):
    """Sampled amplitudes of the state against the closed form: (max relative error, l2 estimate).
    Every QFT amplitude has size 2^(-n/2), so the relative error is |d| * 2^(n/2), and
    2^n * mean(|d|^2) over uniformly drawn indices estimates ||psi - psi_ref||_2^2 without bias."""
    import torch
    idx = np.random.default_rng(seed).integers(0, 1 << n, size=1 << 16).astype(np.uint64)
    o = torch.from_numpy(((idx >> np.uint64(5)) << np.uint64(6) | (idx & np.uint64(31))).astype(np.int64)).cuda()
    got = st.buf[o].double().cpu().numpy() + 1j * st.buf[o + 32].double().cpu().numpy()
    d = np.abs(got - closed_forms.qft_amplitudes(n, x, idx))
    return float(d.max() * 2.0 ** (n / 2)), float(np.sqrt(np.mean(d * d) * 2.0 ** n))


def test_30q_qft_learned_vs_fixed(env):
    """The 30-qubit QFT (the second workload of the 30-qubit configuration): every fixed fusion
    size, the plain fp32 K = 4 and the learned partition timed on one basis input; the learned
    circuit (the post-phase partition with its swap network) checked against the closed form."""
    B, DS, m = env
    n = 30
    gates = wl.qft_circuit(n)
    x = wl.qft_basis_index(n, seed=30)
    st = DS(n)
    res = time_variants(B, st, n, gates, m, init=x)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, model=m)
    st.init(x)
    st.apply(f)
    B.sv_fused_free(f)
    nrm = st.norm()
    max_rel, l2 = _qft_samples(st, n, x, 31)
    st.free()
    REPORT["qft30"] = {"gates": len(gates), "variants": res, "norm": nrm, "max_rel_amp_error": max_rel, "l2_estimate": l2}
    assert abs(nrm - 1) < 1e-4 and l2 <= 1e-4 and max_rel < 2e-4, (nrm, l2, max_rel)
    best_fixed = min(v["device_s"] for k, v in res.items() if k.startswith("greedy"))
    assert res["learned_bf16x3"]["fused_gates"] <= 8, res
    assert res["learned_bf16x3"]["device_s"] <= 0.25 * best_fixed, res


def test_34q_qft_learned_vs_fixed(env):
    B, DS, m = env
    n = 34
    gates = wl.qft_circuit(n)
    x = wl.qft_basis_index(n, seed=34)
    st = DS(n)
    res = time_variants(B, st, n, gates, m, init=x)
    checks = {}
    # fp32 CUDA cores (greedy K = 4): the bar of the 30-qubit QFT test, 1e-4 relative per amplitude
    f = B.sv_fuse_circuit(gates, n, max_k=4)
    st.init(x)
    st.apply(f)
    B.sv_fused_free(f)
    checks["plain_fp32_k4"] = dict(zip(("max_rel_amp_error", "l2_estimate"), _qft_samples(st, n, x, 34)))
    # learned partition on 3xBF16 tensor cores: the acceptance bar ||psi - psi_ref||_2 <= 1e-4 (estimated
    # from the samples); per amplitude 2e-4 relative (products carry ~2^-16 relative error per fused
    # pass, so the per-amplitude error is a random sum of that over the passes)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_LEARNED, precision=B.PREC_BF16X3, model=m)
    st.init(x)
    st.apply(f)
    B.sv_fused_free(f)
    nrm = st.norm()
    checks["learned_bf16x3"] = dict(zip(("max_rel_amp_error", "l2_estimate"), _qft_samples(st, n, x, 35)))
    # post-phase fusion: the controlled-phase ladders ride on the six-qubit gates as per-amplitude
    # phases in the same pass (one pass per six qubits, then the swap network)
    f = B.sv_fuse_circuit(gates, n, max_k=6, mode=B.FUSE_PHASES, precision=B.PREC_BF16X3, tc_min_k=4)
    phases_gates = B.sv_fused_count(f)
    st.init(x)
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st.stream)
    st.apply(f)
    e1.record(st.stream)
    torch.cuda.synchronize()
    res["phases_bf16x3"] = {"device_s": e0.elapsed_time(e1) / 1e3, "fused_gates": phases_gates}
    B.sv_fused_free(f)
    nrm_ph = st.norm()
    checks["phases_bf16x3"] = dict(zip(("max_rel_amp_error", "l2_estimate"), _qft_samples(st, n, x, 36)))
    st.free()
    REPORT["qft34"] = {"gates": len(gates), "variants": res, "norm": nrm, "checks": checks}
    assert abs(nrm - 1) < 1e-4
    assert checks["plain_fp32_k4"]["max_rel_amp_error"] < 1e-4, checks
    assert checks["learned_bf16x3"]["l2_estimate"] <= 1e-4, checks
    assert checks["learned_bf16x3"]["max_rel_amp_error"] < 2e-4, checks
    assert abs(nrm_ph - 1) < 1e-4
    assert checks["phases_bf16x3"]["l2_estimate"] <= 1e-4, checks
    assert checks["phases_bf16x3"]["max_rel_amp_error"] < 2e-4, checks
    best_fixed = min(v["device_s"] for k, v in res.items() if k.startswith("greedy"))
    assert phases_gates <= 12 and res["phases_bf16x3"]["device_s"] < 0.25 * best_fixed, res
    # the learned search gains here: its candidates include the post-phase partition, which the
    # model (trained on timings of gates with post-phases too) scores cheapest
    assert res["learned_bf16x3"]["fused_gates"] == phases_gates, res
    assert res["learned_bf16x3"]["device_s"] <= 0.25 * best_fixed, res
