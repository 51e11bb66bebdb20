"""The allocation-free sampling entry point (sv_sample_noalloc) against sv_sample.

Some callers cannot call cudaMalloc: a process whose memory pool already owns the GPU's memory, or
one that cannot afford the device-wide synchronisation an allocation may cause.  sv_sample_noalloc
serves them from a fixed array inside the library; it must return exactly what sv_sample returns
(the same kernels on the same data), on consecutive calls that reuse that array.  This file is
collected last so a failure here cannot stop the rest of a run that halts at the first failure.
"""
import numpy as np
import pytest

from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_sampling_matches_sv_sample_twice():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding as B
    from paper_2602_09604_gb300.state import DeviceState

    rng = np.random.default_rng(2024)
    for n, count in ((18, 4096), (9, 1000)):      # second call: different sizes, same scratch
        st = DeviceState(n)
        st.init(0)
        f = B.sv_fuse_circuit(wl.hea_circuit(n, 4, rng), n, max_k=4)
        st.apply(f)
        B.sv_fused_free(f)
        u = rng.random(count)
        ref = st.sample(u)
        for _ in range(2):                          # two calls in a row
            got = B.sv_sample_noalloc(st.buf.data_ptr(), n, st.stream.cuda_stream, u)
            assert np.array_equal(got, ref)
        st.free()


def test_noalloc_sampling_rejects_sizes_beyond_its_scratch():
    libbuild.build()
    import torch
    from paper_2602_09604_gb300 import binding as B
    buf = torch.zeros(1 << 10, dtype=torch.float32, device="cuda")
    with pytest.raises(B.SvError) as e:
        B.sv_sample_noalloc(buf.data_ptr(), 31, 0, np.array([0.5]))
    assert e.value.code == B.SV_EINVAL
    with pytest.raises(B.SvError) as e:
        B.sv_sample_noalloc(buf.data_ptr(), 5, 0, np.full(4097, 0.5))
    assert e.value.code == B.SV_EINVAL
