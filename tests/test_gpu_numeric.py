"""The kernels' hand-written numeric helpers on the GPU against the IEEE-754
operations they replace (numpy's conversions, ldexp and division are those
operations, correctly rounded), through the es_dg_debug_numeric test hook:
subnormals, ties, the ends of the float range, infinities, NaNs, powers of two
and random values over the whole exponent range."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D2F, F2D, LDEXP, RCP, RCP_LO, D2F_TAIL, F2D_POS = range(7)
FMIN = float(np.finfo(np.float32).tiny)     # 2^-126
FMAX = float(np.finfo(np.float32).max)


@pytest.fixture(scope="module")
def run():
    import torch

    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    lib = _lib.load()

    def call(which, x, k=0):
        x = np.ascontiguousarray(x)
        out_dtype = np.float32 if which in (D2F, D2F_TAIL) else np.float64
        xin = torch.from_numpy(x).cuda()
        out = torch.empty(x.shape, dtype=torch.float32 if out_dtype == np.float32 else torch.float64,
                          device="cuda")
        rc = lib.es_dg_debug_numeric(which, C.c_void_p(xin.data_ptr()), C.c_void_p(out.data_ptr()),
                                     x.size, k, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        return out.cpu().numpy()
    return call


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def random_doubles(rng, n, emin, emax):
    e = rng.integers(emin, emax + 1, size=n)
    m = rng.uniform(1.0, 2.0, size=n)
    s = rng.choice([-1.0, 1.0], size=n)
    return s * np.ldexp(m, e)


def test_d2f(run):
    rng = np.random.default_rng(1)
    f = random_doubles(rng, 20000, -126, 127).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    ties = f + np.sign(f) * 0.5 * ulp                   # halfway: round to even
    near = f + np.sign(f) * ulp * rng.uniform(-0.49, 0.49, size=f.size)
    # the helper's domain is |x| < 2^128: FLT_MAX and the values that round past it
    # (to +-inf) are inside; infinities, NaNs and larger magnitudes are not
    edge = np.array([FMAX, -FMAX, FMAX * (1 + 2.0 ** -25), FMAX * (1 + 2.0 ** -23),
                     2.0 ** 128 * (1 - 2.0 ** -30), FMIN, -FMIN, FMIN * (1 + 2.0 ** -30), 1.0, -1.0,
                     2.0 ** 127, 2.0 ** -126, 0.0, -0.0, 1e-300, -1e-300, 5e-324])
    pw2 = np.ldexp(1.0, np.arange(-126, 128)).astype(np.float64)
    x = np.concatenate([random_doubles(rng, 20000, -126, 127), ties, near, edge, pw2, -pw2])
    got = run(D2F, x)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    want = np.where(np.abs(x) < FMIN, np.copysign(np.float32(0), x).astype(np.float32), want)
    assert np.array_equal(bits(got), bits(want)), x[bits(got) != bits(want)][:8]


def test_f2d(run):
    rng = np.random.default_rng(2)
    u = rng.integers(0, 2 ** 32, size=50000, dtype=np.uint64).astype(np.uint32)
    x = np.concatenate([u.view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, FMIN, -FMIN, FMAX, -FMAX, 1e-40,
                                  -1e-44], dtype=np.float32)])
    got = run(F2D, x)
    with np.errstate(invalid="ignore"):  # signalling NaNs among the random patterns
        want = x.astype(np.float64)
    sub = (np.abs(x) < FMIN) & ~np.isnan(x)
    want[sub] = np.copysign(0.0, x[sub].astype(np.float64))
    ok = (bits(got) == bits(want)) | (np.isnan(got) & np.isnan(want))
    assert ok.all(), x[~ok][:8]


@pytest.mark.parametrize("k", [-2, -1, 1, 2])
def test_ldexp(run, k):
    rng = np.random.default_rng(3 + k)
    dmin = float(np.finfo(np.float64).tiny)
    x = np.concatenate([random_doubles(rng, 20000, -1022, 1023),
                        np.array([dmin, -dmin, 2 * dmin, np.finfo(np.float64).max, 0.0, -0.0,
                                  np.inf, -np.inf, 5e-324, 1.0, -3.0])])
    got = run(LDEXP, x, k)
    with np.errstate(over="ignore", under="ignore"):
        want = np.ldexp(x, k)
    flush = (np.abs(x) < dmin) | (np.abs(want) < dmin)
    want[flush] = np.copysign(0.0, x[flush])
    assert np.array_equal(bits(got), bits(want)), x[bits(got) != bits(want)][:8]
    assert np.isnan(run(LDEXP, np.array([np.nan]), k)).all()


def test_rcp(run):
    rng = np.random.default_rng(4)
    x = np.concatenate([random_doubles(rng, 50000, -1000, 1000),
                        np.ldexp(1.0, np.arange(-1000, 1001)), rng.uniform(0.5, 2.0, 20000)])
    want = 1.0 / x
    ulp = np.spacing(np.abs(want))
    err = np.abs(run(RCP, x) - want) / ulp
    assert err.max() <= 1.0, err.max()
    rel = np.abs(run(RCP_LO, x) - want) / np.abs(want)
    assert rel.max() <= 2.0 ** -38, rel.max()


def test_series_tail_conversions(run):
    rng = np.random.default_rng(5)
    u = np.concatenate([rng.uniform(0.0, 1e-4, 20000), np.abs(random_doubles(rng, 20000, -126, 127)),
                        np.array([0.0, FMIN, FMIN * 0.999, 1e-40, 2.0 ** 127, 1.5])])
    got = run(D2F_TAIL, u).astype(np.float64)
    # truncation toward zero: never above u, less than one float ulp below it
    normal = u >= FMIN
    assert np.all(got[~normal] == 0.0)
    gu, uu = got[normal], u[normal]
    assert np.all(gu <= uu)
    assert np.all(uu - gu < np.spacing(gu.astype(np.float32)).astype(np.float64))
    exact = uu.astype(np.float32).astype(np.float64) == uu
    assert np.array_equal(gu[exact], uu[exact])
    f = np.abs(random_doubles(rng, 20000, -126, 127)).astype(np.float32)
    assert np.array_equal(run(F2D_POS, f), f.astype(np.float64))
