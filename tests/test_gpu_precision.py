"""Precision of every arithmetic mode against the complex128 oracle on a 28-qubit grid circuit.

4x7 grid, 20 cycles (the random-circuit recipe), fused at max 5 and 6 qubits.  fp32 CUDA cores and
3xBF16 tensor cores must meet F >= 1 - 1e-6 and ||psi - psi_ref||_2 <= 1e-4; TF32 is the fast,
lower-precision mode and is reported (its per-gate error is ~3e-4).  With SV_REPORT_DIR set, the
measured numbers are written to <SV_REPORT_DIR>/precision_28q.json.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_precision_modes_28q():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding as B
    from paper_2602_09604_gb300.state import DeviceState

    n, gates = wl.GRID_28.n, wl.random_grid_circuit(wl.GRID_28, 20, seed=3)
    assert n == 28
    ref = oracle.run_circuit(n, gates, 0, threads=oracle.default_threads())
    st = DeviceState(n)
    report = {"workload": "4x7 grid, 20 cycles, seed 3", "n": n, "gates": len(gates), "modes": {}}
    for name, prec in (("fp32", B.PREC_FP32), ("bf16x3", B.PREC_BF16X3), ("tf32", B.PREC_TF32)):
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
    out = os.environ.get("SV_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_28q.json"), "w") as fh:
            json.dump(report, fh, indent=1)
    print(json.dumps(report))
