"""The allocation-free TPIILU apply, for callers that cannot allocate device
memory (memory owned by another runtime or a fixed pool, or a loop where
allocation is not allowed).

It is called through the C ABI and compared with the regular iiluk_apply,
bit for bit (the tolerance every parity test here uses), on two calls in a
row: the second call must not depend on what the first left in the shared
static scratch.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import _lib as L
from paper_0803_0048_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("side,k", [(40, 2), (700, 1)], ids=["2d_40x40_k2", "2d_700x700_k1"])
def test_noalloc_apply_matches_regular_apply_twice(side, k):
    """n = 1,600 (a few CTAs) and n = 490,000 (near half the scratch's
    2^20 rows, thousands of CTAs)."""
    lib = L.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = W.conv_diff(side, 2, (20.0, 20.0))
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.colind).cuda()
    av = torch.from_numpy(A.val).cuda()
    S = P.symbolic(rp, ci, k)
    M = P.iiluk_build(P.numeric(S, av))
    frp, fci, _, fdg = S.pattern()
    g = M.values()
    for call, seed in enumerate((11, 12)):
        p = torch.from_numpy(W.uniform(W.stream_key(seed, "na"), np.arange(A.n), -1, 1)).cuda()
        want = M.apply(p)
        got = torch.full_like(p, float("nan"))
        st = lib.iiluk_apply_noalloc(A.n, _ptr(frp), _ptr(fci), _ptr(fdg), _ptr(g), _ptr(p),
                                     _ptr(got), stream)
        assert st == L.OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        g_bits = got.cpu().numpy().view(np.int64)
        w_bits = want.cpu().numpy().view(np.int64)
        assert np.array_equal(g_bits, w_bits), f"call {call}: results differ"


def test_noalloc_apply_rejects_sizes_beyond_its_scratch():
    lib = L.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(2, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.iiluk_apply_noalloc((1 << 20) + 1, _ptr(idx), _ptr(col), _ptr(idx), _ptr(one),
                                 _ptr(one), _ptr(one), stream)
    assert st == L.ENOMEM
