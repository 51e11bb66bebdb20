"""sv_sample_norm (samples and norm from one read pass) equals sv_sample and sv_norm: the same
samples, the norm to fp64 summation-order noise; norm only with no samples; complex128 too."""
import numpy as np
import pytest

import oracle
from paper_2602_09604_gb300 import build as libbuild
from paper_2602_09604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    libbuild.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2602_09604_gb300 import binding
    return binding


@pytest.mark.parametrize("n,c128", [(3, False), (12, False), (22, False), (13, True)])
def test_sample_norm_matches_separate_calls(B, n, c128):
    from paper_2602_09604_gb300.state import DeviceState
    rng = np.random.default_rng(n)
    psi = wl.random_state(n, rng).astype(np.complex128) * 1.25
    st = DeviceState(n, c128=c128)
    st.load(psi)
    u = rng.random(300)
    s1 = B.sv_sample(st.h, u)
    n1 = B.sv_norm(st.h)
    s2, n2 = B.sv_sample_norm(st.h, u)
    assert np.array_equal(s1, s2)
    assert abs(n1 - n2) <= 1e-13 * n1
    _, n3 = B.sv_sample_norm(st.h, [])
    assert n3 == n2
    ref = oracle.norm(st.store().astype(np.complex128))
    assert abs(n2 - ref) <= 1e-12 * ref
    st.free()
