"""The benchmark configuration itself at full size (30-qubit 5x6 grid, 20 cycles, 845 gates,
learned fusion with the 28-qubit light cone fused apart, started through sv_init_apply, 3xBF16
tensor cores: the launch configuration bench.py times), checked by
properties that hold at any size: the circuit followed by its inverse returns |0...0>, the norm
stays 1, and the state agrees with the independent fp32 CUDA-core path (greedy K = 4, no tensor
cores) to the accuracy bar; sampled bitstrings are valid indices of nonzero probability."""
import os

import numpy as np
import pytest

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


def test_bench_configuration_full_size(B):
    import torch
    from paper_2602_09604_gb300.state import DeviceState
    n, gates = wl.circuit_30q_grid()
    model = B.sv_mlp_load(MODEL) if os.path.exists(MODEL) else None
    kw = dict(max_k=6, precision=B.PREC_BF16X3, tc_min_k=4,
              mode=B.FUSE_LEARNED if model is not None else B.FUSE_GREEDY, model=model)
    st = DeviceState(n)
    # bench path: the 28-qubit light cone fused apart, started from |0...0> through sv_init_apply
    f = B.sv_fuse_circuit(gates, n, **kw, start_qubits=28)
    B.sv_init_apply(st.h, 0, f, False)
    B.sv_device_status()
    assert abs(st.norm() - 1.0) <= 1e-4
    u = np.random.default_rng(3).random(256)
    s = st.sample(u)
    assert np.all(s < (1 << n))
    tc = st.buf.clone()
    # independent fp32 CUDA-core path
    fp = B.sv_fuse_circuit(gates, n, max_k=4, precision=B.PREC_FP32)
    st.init(0)
    st.apply(fp)
    B.sv_fused_free(fp)
    ref = st.buf
    # fidelity and l2 distance in fp64, computed on the device block by block (8 GiB states)
    ov = torch.zeros((), dtype=torch.complex128, device="cuda")
    d2 = torch.zeros((), dtype=torch.float64, device="cuda")
    na = torch.zeros((), dtype=torch.float64, device="cuda")
    nb = torch.zeros((), dtype=torch.float64, device="cuda")
    step = 1 << 26
    for lo in range(0, ref.numel(), step):
        a = ref[lo:lo + step].view(-1, 2, 32).double()
        b = tc[lo:lo + step].view(-1, 2, 32).double()
        ca = torch.complex(a[:, 0], a[:, 1])
        cb = torch.complex(b[:, 0], b[:, 1])
        ov += (ca.conj() * cb).sum()
        d2 += ((ca - cb).abs() ** 2).sum()
        na += (ca.abs() ** 2).sum()
        nb += (cb.abs() ** 2).sum()
    fid = float(ov.abs() ** 2 / (na * nb))
    assert fid >= 1 - 1e-6, fid
    assert float(d2.sqrt()) <= 1e-4, float(d2.sqrt())
    del tc
    # circuit then its inverse through the bench path returns |0...0>
    fi = B.sv_fuse_circuit(wl.inverse(gates), n, **kw)
    B.sv_init_apply(st.h, 0, f, False)
    st.apply(fi)
    B.sv_device_status()
    amp0 = complex(st.buf[0].item(), st.buf[32].item())
    assert abs(amp0) ** 2 >= 1 - 1e-4
    out = os.environ.get("SV_REPORT_DIR")
    if out:
        import json
        with open(os.path.join(out, "bench_config_30q.json"), "w") as fh:
            json.dump({"fidelity_vs_fp32_path": fid, "l2_vs_fp32_path": float(d2.sqrt()),
                       "p0_after_inverse": abs(amp0) ** 2}, fh)
    B.sv_fused_free(fi)
    B.sv_fused_free(f)
    if model is not None:
        B.sv_mlp_free(model)
    st.free()
