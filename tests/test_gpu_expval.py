"""Pauli expectation values on the GPU against the oracle: seeded random states at sizes from one
zero-padded block to several thousand blocks, strings covering every mask case the kernel
distinguishes (identity, pure Z, X inside a block, X across blocks, Y-heavy, more than eight strings
sharing one x mask, i.e. several read passes); then 30-qubit properties (basis state, GHZ) at the
full size and determinism."""
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


def strings_for(n, rng, count=40):
    out = [{}, {0: "Z"}, {n - 1: "X"}, {q: "Z" for q in range(n)}, {q: "Y" for q in range(min(n, 6))}]
    if n > 1:
        out += [{0: "X", 1: "Y"}, {0: "Y", n - 1: "Y"}]
    if n > 6:
        out += [{5: "X", 6: "Z"}, {2: "X", 7: "Y", 3: "Z"}]
    # nine strings with one shared x mask (two read passes for that mask)
    shared = {q: "X" for q in range(0, n, 3)}
    for i in range(9):
        t = dict(shared)
        for q in range(1, n, 3):
            if (i >> (q % 4)) & 1:
                t[q] = "Z"
        if i % 2 and 0 in t:
            t[0] = "Y"
        out.append(t)
    while len(out) < count:
        out.append({int(q): "XYZ"[int(rng.integers(0, 3))] for q in range(n) if rng.random() < 0.4})
    return out


@pytest.mark.parametrize("n", [3, 5, 6, 12, 17, 22])
def test_expval_matches_oracle(B, n):
    from paper_2602_09604_gb300.state import DeviceState
    rng = np.random.default_rng(100 + n)
    psi = wl.random_state(n, rng)                       # complex64, unit norm
    st = DeviceState(n)
    st.load(psi)
    strings = strings_for(n, rng)
    got = st.expval(strings)
    ref64 = psi.astype(np.complex128)
    threads = oracle.default_threads()
    for t, g in zip(strings, got):
        want = oracle.expval_pauli(ref64, n, t, threads)
        assert abs(g - want.real) <= 2e-6, (n, t, g, want)
    again = st.expval(strings)
    assert np.array_equal(got, again)                   # fixed reduction order
    st.free()


def test_expval_full_size_properties(B):
    from paper_2602_09604_gb300.state import DeviceState
    n = 30
    st = DeviceState(n)
    x = 0b101100111000011110000011111001
    st.init(x)
    zs = [0b1, 1 << 29, (1 << 30) - 1, 0b1010101 << 20]
    strings = [{q: "Z" for q in range(n) if (z >> q) & 1} for z in zs] + [{7: "X"}, {0: "Y", 29: "Z"}]
    got = st.expval(strings)
    want = [(-1) ** bin(x & z).count("1") for z in zs] + [0.0, 0.0]
    assert np.allclose(got, want, atol=1e-12)
    # GHZ through the product path
    f = B.sv_fuse_circuit(wl.ghz_circuit(n), n, max_k=4)
    st.init(0)
    st.apply(f)
    B.sv_fused_free(f)
    got = st.expval([{0: "Z", 29: "Z"}, {0: "Z"}, {q: "X" for q in range(n)},
                     {**{q: "X" for q in range(n)}, 0: "Y", 1: "Y"}, {}])
    assert np.allclose(got, [1.0, 0.0, 1.0, -1.0, 1.0], atol=2e-5)
    st.free()


def test_expval_rejects_bad_masks(B):
    from paper_2602_09604_gb300.state import DeviceState
    st = DeviceState(8)
    st.init(0)
    with pytest.raises(B.SvError) as e:
        B.sv_expval_pauli(st.h, [1 << 8], [0])
    assert e.value.code == B.SV_EINVAL
    assert B.sv_expval_pauli(st.h, [], []).size == 0
    st.free()
