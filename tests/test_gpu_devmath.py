"""The refined FP64 reciprocal and reciprocal square root of the eigensolvers,
and the bit-level double-float split of the double-float kernels.

rcp64 and rsqrt64 start from the hardware estimates and take two
Newton-Raphson steps.  Over their stated domain, |x| in [2^-1022, 2^1022],
rcp64 must be within one ulp and rsqrt64 within two ulps of the correctly
rounded results, here computed exactly on the host with 60-digit decimal
arithmetic (CUDA's IEEE division is checked to be that correctly rounded
value).  Outside that domain the estimate flushes subnormals: the header
states the results there (0 for huge inputs, not finite for subnormal ones),
which are checked too.  The split's hi word is the input cut to 24
significant bits and hi + lo (exact in FP64) must equal the input to 2^-48
relative wherever lo stays in FP32's normal range.
"""

import ctypes
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_05559_gb300 import build
    build.build()
    import paper_1905_05559_gb300 as hm
    return hm


def _run(hm, x):
    lib = hm.load()
    xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    out = torch.full((6, x.size), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.hess_check_devmath(ctypes.c_void_p(xd.data_ptr()), x.size, ctypes.c_void_p(out.data_ptr()),
                                None)
    assert st == 0, hm.last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ulps(a, b):
    """|a - b| in units in the last place, for finite doubles of equal sign."""
    ia = np.abs(a).view(np.int64)
    ib = np.abs(b).view(np.int64)
    assert np.all(np.sign(a) == np.sign(b))
    return np.abs(ia - ib)


def _inputs(seed=0, n=6000):
    rng = np.random.default_rng(seed)
    # exponents spread over the whole domain, random mantissas
    e = rng.integers(-1022, 1022, size=n)
    m = rng.uniform(1.0, 2.0, size=n)
    x = np.ldexp(m, e)
    x = np.clip(x, np.ldexp(1.0, -1022), np.ldexp(1.0, 1022))
    # the domain's edges, powers of two and their neighbours
    edges = [np.ldexp(1.0, -1022), np.ldexp(1.0, 1022), 1.0, 2.0, 0.5, 3.0, 1.0 / 3.0]
    edges += [np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), np.nextafter(np.ldexp(1.0, -1022), 1.0)]
    x = np.concatenate([x, np.array(edges), 1.0 + rng.uniform(0, 1e-12, 64)])
    return x


def _exact(x, f):
    getcontext().prec = 60
    return np.array([float(f(Decimal(float(v)))) for v in x])


def test_rcp64_within_one_ulp_of_correct_rounding(hm):
    x = _inputs(0)
    for sign in (1.0, -1.0):
        xs = sign * x
        out = _run(hm, xs)
        ref = _exact(xs, lambda d: Decimal(1) / d)
        assert np.array_equal(out[1], ref)  # CUDA's division is correctly rounded
        assert _ulps(out[0], ref).max() <= 1


def test_rsqrt64_within_two_ulps_of_correct_rounding(hm):
    x = _inputs(1)
    out = _run(hm, x)
    ref = _exact(x, lambda d: Decimal(1) / d.sqrt())
    u = _ulps(out[2], ref)
    assert u.max() <= 2
    assert np.mean(u <= 1) >= 0.9
    # 1/sqrt(x) by two correctly rounded operations is itself within one ulp
    assert _ulps(out[3], ref).max() <= 1


def test_outside_the_domain_results_are_zero_or_not_finite(hm):
    sub = np.array([np.ldexp(1.0, -1030), np.ldexp(1.0, -1074), 1e-310])
    big = np.array([np.ldexp(1.5, 1022), np.ldexp(1.0, 1023), 1.5e308])
    out = _run(hm, np.concatenate([sub, big]))
    assert not np.isfinite(out[0][:3]).any()
    assert np.all(out[0][3:] == 0.0)


def test_double_float_split_from_bits(hm):
    rng = np.random.default_rng(3)
    n = 4000
    e = rng.integers(-74, 128, size=n)
    x = np.ldexp(rng.uniform(1.0, 2.0, size=n), e) * rng.choice([-1.0, 1.0], size=n)
    x = np.concatenate([x, [1.0, -1.0, 3.0, 1.0 / 3.0, np.nextafter(1.0, 2.0), np.ldexp(1.0, -74),
                            np.ldexp(1.9999999999, 127)]])
    out = _run(hm, x)
    hi, lo = out[4], out[5]
    # hi: x with its significand cut to 24 bits (toward zero, same sign)
    trunc = (x.view(np.int64) & ~np.int64((1 << 29) - 1)).view(np.float64)
    assert np.array_equal(hi, trunc)
    assert np.all(np.abs(lo) <= np.ldexp(np.abs(hi), -23))
    err = np.abs((hi + lo) - x) / np.abs(x)
    assert err.max() <= 2.0 ** -48, err.max()
    # below FP32's normal range: both words 0; in between, hi stays exact
    tiny = np.array([0.0, -0.0, np.ldexp(1.0, -127), np.ldexp(1.5, -200), 1e-300])
    out = _run(hm, tiny)
    assert np.all(out[4] == 0.0) and np.all(out[5] == 0.0)
    mid = np.ldexp(rng.uniform(1.0, 2.0, size=200), rng.integers(-126, -74, size=200))
    out = _run(hm, mid)
    assert np.array_equal(out[4], (mid.view(np.int64) & ~np.int64((1 << 29) - 1)).view(np.float64))
    assert (np.abs(out[4] + out[5] - mid) / mid).max() <= 2.0 ** -23
