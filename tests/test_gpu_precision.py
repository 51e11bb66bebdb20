"""Precision of every arithmetic mode on grid circuits (the random-circuit recipe, 20 cycles).

* 28 qubits (4x7 grid, seed 3), against the complex128 oracle: fused at max 5 and 6 qubits, fp32
  CUDA cores and 3xBF16 tensor cores must meet F >= 1 - 1e-6 and ||psi - psi_ref||_2 <= 1e-4;
  TF32 is the fast, lower-precision mode and is reported (its per-gate error is ~3e-4).
* 28 qubits, the exact launch configuration the benchmark times (learned fusion with the light
  cone on n - 2 qubits fused apart, started from |0...0> through sv_init_apply, 3xBF16 tensor cores
  for fused gates of 4 or more qubits), element by element against the oracle.
* 32 qubits (4x8 grid, seed 6; a 32 GiB complex64 state): the same modes and sizes against the
  library's complex128 state (64 GiB, fp64 arithmetic; it matches the oracle to 1e-12 wherever
  the oracle fits), F and ||psi - psi_ref||_2 computed in fp64 on the device.
With SV_REPORT_DIR set, the measured numbers are written to <SV_REPORT_DIR>/precision_28q.json,
bench_path_28q.json and precision_32q.json.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl
from devmetrics import device_metrics

pytestmark = pytest.mark.gpu
MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2602_09604_gb300",
                     "cost_model_gb300.bin")
MODES = (("fp32", 0), ("bf16x3", 2), ("tf32", 1))   # name, SV_PREC_*


def _report(name, data):
    out = os.environ.get("SV_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, name), "w") as fh:
            json.dump(data, fh, indent=1)
    print(json.dumps(data))


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def grid28():
    n, gates = wl.GRID_28.n, wl.random_grid_circuit(wl.GRID_28, 20, seed=3)
    assert n == 28
    return n, gates, oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())


def test_precision_modes_28q(B, grid28):
    from paper_2602_09604_gb300.state import DeviceState
    n, gates, ref = grid28
    st = DeviceState(n)
    report = {"workload": "4x7 grid, 20 cycles, seed 3", "n": n, "gates": len(gates), "modes": {}}
    for name, prec in MODES:
        for mk in (5, 6):
            f = B.sv_fuse_circuit(gates, n, max_k=mk, precision=prec, tc_min_k=4)
            st.init(0)
            rec = st.apply(f, timings=True)
            got = st.store()
            F = oracle.fidelity(ref, got)
            err = oracle.l2_error(ref, got)
            report["modes"][f"{name}_k{mk}"] = {"fidelity": F, "l2_error": err, "fused_gates": len(rec),
                                                "device_ms": sum(r["us"] for r in rec) / 1e3}
            B.sv_fused_free(f)
            if name in ("fp32", "bf16x3"):
                assert F >= 1 - 1e-6 and err <= 1e-4, (name, mk, F, err)
            else:
                assert F >= 0.99, (name, mk, F)
    st.free()
    _report("precision_28q.json", report)


def test_bench_path_28q_vs_oracle(B, grid28):
    """The benchmark's launch configuration, element by element against the oracle.  Bar: the
    acceptance bar F >= 1 - 1e-6 and ||psi - psi_ref||_2 <= 1e-4, and per element
    |d_i| <= 5e-4 * max(|ref_i|, 2^(-n/2)).  The rounding error of a fused pass scales with the
    input's norm, not with the output amplitude, so an error of total norm 1e-4 spread over 2^n
    amplitudes is ~1e-4 * 2^(-n/2) per amplitude (rms); the largest of 2^28 such (Rayleigh-like)
    values is about sqrt(ln 2^28) = 4.4 times the rms, which the factor 5 allows."""
    from paper_2602_09604_gb300.state import DeviceState
    n, gates, ref = grid28
    model = B.sv_mlp_load(MODEL) if os.path.exists(MODEL) else None
    kw = dict(max_k=6, precision=B.PREC_BF16X3, tc_min_k=4,
              mode=B.FUSE_LEARNED if model is not None else B.FUSE_GREEDY, model=model)
    f = B.sv_fuse_circuit(gates, n, **kw, start_qubits=n - 2)
    st = DeviceState(n)
    rec = B.sv_init_apply(st.h, 0, f, True)
    B.sv_device_status()
    got = st.store()
    small = sum(1 for r in rec if r["path"] == B.PATH_AUTO)
    B.sv_fused_free(f)
    if model is not None:
        B.sv_mlp_free(model)
    st.free()
    d = np.abs(got.astype(np.complex128) - ref)
    rel = d / np.maximum(np.abs(ref), 2.0 ** (-n / 2))
    F = oracle.fidelity(ref, got)
    err = oracle.l2_error(ref, got)
    _report("bench_path_28q.json", {
        "workload": "4x7 grid, 20 cycles, seed 3", "n": n, "fusion": "learned" if model else "greedy",
        "start_qubits": n - 2, "fused_gates": len(rec), "small_state_gates": small,
        "fidelity": F, "l2_error": err, "max_abs_error": float(d.max()), "max_rel_error": float(rel.max())})
    assert small > 0                       # the lazy start really ran gates on the small state
    assert F >= 1 - 1e-6 and err <= 1e-4, (F, err)
    assert float(rel.max()) <= 5e-4, float(rel.max())


def test_precision_modes_32q(B):
    """Config 3's 32-qubit half against the complex128 GPU state (no complex128 oracle fits)."""
    from paper_2602_09604_gb300.state import DeviceState
    n, gates = wl.GRID_32.n, wl.random_grid_circuit(wl.GRID_32, 20, seed=6)
    assert n == 32
    ref = DeviceState(n, c128=True)
    ref.init(0)
    fr = B.sv_fuse_circuit(gates, n, max_k=3)
    ref.apply(fr)
    B.sv_fused_free(fr)
    B.sv_device_status()
    st = DeviceState(n)
    report = {"workload": "4x8 grid, 20 cycles, seed 6", "n": n, "gates": len(gates),
              "reference": "complex128 GPU state, greedy K = 3, fp64", "modes": {}}
    for name, prec in MODES:
        for mk in (5, 6):
            f = B.sv_fuse_circuit(gates, n, max_k=mk, precision=prec, tc_min_k=4)
            st.init(0)
            rec = st.apply(f, timings=True)
            B.sv_device_status()
            m = device_metrics(ref.buf, st.buf)
            m.update(fused_gates=len(rec), device_ms=sum(r["us"] for r in rec) / 1e3)
            report["modes"][f"{name}_k{mk}"] = m
            B.sv_fused_free(f)
            if name in ("fp32", "bf16x3"):
                assert m["fidelity"] >= 1 - 1e-6 and m["l2_error"] <= 1e-4, (name, mk, m)
            else:
                assert m["fidelity"] >= 0.99, (name, mk, m)
    assert abs(device_metrics(ref.buf, ref.buf)["norm"] - 1.0) < 1e-12
    st.free()
    ref.free()
    _report("precision_32q.json", report)
