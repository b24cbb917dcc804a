"""The numeric phase's multipliers and the sweeps' division by u_ii are
computed on the integer pipes (a fixed-point reciprocal of the divisor from
an fp32 seed and two Newton steps, then an exact remainder correction)
instead of by the FP64 division.  The method is exact only if the quotient
always comes out as IEEE's correctly rounded one, so it is pinned here
against the host's IEEE division (numpy), bit for bit, through iluk_div_rn
(the same device functions), on inputs chosen to stress it: random operands
over the whole exponent range, random normal operands with normal
quotients (the integer path), quotients next to a rounding midpoint, extreme
significands (reciprocal seeds at both ends of their range, rounding carries
into the exponent), quotients at the edges of the normal range (overflow to
infinity, underflow to subnormals, which fall back to IEEE division), and
special values.
"""
import numpy as np
import pytest
import torch

import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def _from_parts(sign, exp, mant):
    """Doubles from sign bits, biased exponents and 52-bit mantissas."""
    u = (sign.astype(np.uint64) << np.uint64(63)) | (exp.astype(np.uint64) << np.uint64(52)) \
        | (mant.astype(np.uint64) & np.uint64((1 << 52) - 1))
    return u.view(np.float64)


def _check(a, b):
    with np.errstate(all="ignore"):
        want = a / b
    got = P.div_rn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    nan_w, nan_g = np.isnan(want), np.isnan(got)
    assert np.array_equal(nan_w, nan_g)
    ok = ~nan_w
    bad = np.flatnonzero(_bits(want[ok]) != _bits(got[ok]))
    assert bad.size == 0, (f"{bad.size} quotients differ, first: "
                           f"{a[ok][bad[0]]!r} / {b[ok][bad[0]]!r} = {want[ok][bad[0]]!r}, "
                           f"got {got[ok][bad[0]]!r}")


def _draws(tag, n):
    return W.draws_u64(W.stream_key(41, tag), np.arange(n))


def test_random_operands_whole_range():
    n = 1 << 22
    ra, rb = _draws("a", n), _draws("b", n)
    a = _from_parts(ra >> np.uint64(63), (ra >> np.uint64(52)) % np.uint64(2047), ra)
    b = _from_parts(rb >> np.uint64(63), (rb >> np.uint64(52)) % np.uint64(2047), rb)
    _check(a, b)


def test_random_operands_normal_quotients():
    n = 1 << 23
    ra, rb = _draws("fa", n), _draws("fb", n)
    ea = np.uint64(523) + (ra >> np.uint64(52)) % np.uint64(1001)
    eb = np.uint64(523) + (rb >> np.uint64(52)) % np.uint64(1001)
    _check(_from_parts(ra >> np.uint64(63), ea, ra), _from_parts(rb >> np.uint64(63), eb, rb))


def test_quotients_at_the_edges_of_the_normal_range():
    # biased quotient exponents -2..3 and 2043..2048 around the subnormal and
    # overflow boundaries, with random significands (some round up across
    # the boundary)
    n = 1 << 20
    ra, rb, rs = _draws("ea", n), _draws("eb", n), _draws("es", n)
    eb = np.uint64(1000) + rb % np.uint64(47)
    shift = rs % np.uint64(12)  # target exponent offset
    lo = (eb.astype(np.int64) - 1023 + 1 + (shift.astype(np.int64) - 3)).clip(1, 2046)
    hi = (eb.astype(np.int64) - 1023 + 2046 + (shift.astype(np.int64) - 8)).clip(1, 2046)
    ea = np.where(rs & np.uint64(1 << 40), lo, hi).astype(np.uint64)
    _check(_from_parts(ra >> np.uint64(63), ea, ra), _from_parts(rb >> np.uint64(63), eb, rb))


def test_quotients_near_a_midpoint():
    # a = b*q + b*(ulp(q)/2): a / b lies within a few ulps of the midpoint
    # between q and its successor, where a faithful first guess most often
    # needs the correction step to round the right way.
    n = 1 << 22
    rq, rb = _draws("q", n), _draws("qb", n)
    q = _from_parts(np.zeros(n, np.uint64), np.uint64(1023) + rq % np.uint64(40), rq >> np.uint64(4))
    b = _from_parts(rb >> np.uint64(63), np.uint64(1003) + (rb >> np.uint64(52)) % np.uint64(41), rb)
    a = b * q + b * (np.spacing(q) / 2)
    _check(a, b)


def test_extreme_mantissas():
    # mantissas of all ones, all zeros and one bit away from either, paired
    # every way: the reciprocal's tail and the remainder are then extreme
    ms = [0, 1, 2, (1 << 52) - 1, (1 << 52) - 2, 1 << 51, (1 << 51) - 1, (1 << 51) + 1]
    vals = []
    for e in (1021, 1022, 1023, 1024, 1025):
        for m in ms:
            vals.append(_from_parts(np.zeros(1, np.uint64), np.array([e], np.uint64),
                                    np.array([m], np.uint64))[0])
    vals = np.array(vals + [-v for v in vals])
    a, b = np.meshgrid(vals, vals, indexing="ij")
    _check(a.ravel().copy(), b.ravel().copy())


def test_range_edges_and_special_values():
    edges = []
    for e in (1, 2, 3, 622, 623, 624, 1022, 1023, 1024, 1422, 1423, 1424, 2044, 2045, 2046):
        for m in (0, 1, (1 << 52) - 1, 0x8000000000000):
            edges.append(_from_parts(np.zeros(1, np.uint64), np.array([e], np.uint64),
                                     np.array([m], np.uint64))[0])
    specials = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                2.225073858507201e-308, 1.7976931348623157e308, -1.7976931348623157e308, 1.0,
                -1.0, 3.0, 0.1, 1e-300, 1e300]
    vals = np.array(edges + edges + specials + [-x for x in edges], dtype=np.float64)
    a, b = np.meshgrid(vals, vals, indexing="ij")
    _check(a.ravel().copy(), b.ravel().copy())
