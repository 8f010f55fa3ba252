"""The step kernel's own exp, logarithm and reciprocal against CUDA's exp,
log and IEEE division: at most 2 ulp apart on the ranges the rates use,
identical on the special values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_exp_and_reciprocal():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-700, 700, 200000), rng.uniform(-1, 1, 100000),
                        rng.uniform(-511.9, 511.9, 100000),
                        np.array([0.0, -0.0, 1e-300, -1e-300, 511.99, -511.99, 512.0, -512.0, 709.0,
                                  -708.0, 710.0, -746.0, np.inf, -np.inf, np.nan, 1.0, -1.0])])
    dev = torch.device("cuda")
    xd = torch.tensor(x, device=dev)
    outs = [torch.empty_like(xd) for _ in range(4)]
    rc = chem.lib().chem_selftest_math(len(x), xd.data_ptr(), *[o.data_ptr() for o in outs], None)
    assert rc == 0
    ye, yr, re, rr = [o.cpu().numpy() for o in outs]
    fin = np.isfinite(yr) & (yr > 0) & (np.abs(x) < 700)
    ulp = np.abs(ye[fin] - yr[fin]) / np.spacing(yr[fin])
    assert ulp.max() <= 2.0, ulp.max()
    spec = ~np.isfinite(x) | (np.abs(x) >= 512)
    assert np.array_equal(ye[spec], yr[spec], equal_nan=True)
    assert ye[x == -np.inf][0] == 0.0 and np.isnan(ye[np.isnan(x)][0])
    nz = np.isfinite(x) & (np.abs(x) > 1e-300)
    ulp_r = np.abs(re[nz] - rr[nz]) / np.spacing(np.abs(rr[nz]))
    assert ulp_r.max() <= 1.0


def test_split_exponential_and_scaling():
    """The equilibrium constants' exponent arithmetic: exp(x) = y 2^k with y
    within 2 ulp of exp(x - k ln 2) (extended precision) on |x| < 2^22 (a
    species' g/RT can pass 1000 at low temperature), the saturated forms
    beyond, and v 2^k against ldexp with the stated flushes."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-1023.9, 1023.9, 200000), rng.uniform(-5, 5, 50000),
                        rng.uniform(-4.1e6, 4.1e6, 20000),
                        np.array([0.0, -0.0, 511.99, -511.99, 512.0, -512.0, 1023.99, -1023.99,
                                  1024.0, -1024.0, 5000.0, -5000.0, 4194303.9, -4194303.9,
                                  4194304.0, -4194304.0, 1e300, -1e300, np.inf, -np.inf, np.nan])])
    vals = np.concatenate([rng.uniform(1, 2, 100000) * 2.0 ** rng.integers(-1000, 1000, 100000),
                           -rng.uniform(1, 2, 1000),
                           np.array([0.0, -0.0, 5e-324, -1e-310, np.inf, -np.inf, np.nan, 1.0, 1.0, 1.0, 1.0])])
    ks = np.concatenate([rng.integers(-2200, 2200, 100000), rng.integers(-60, 60, 1000),
                         np.array([5, 5, 100, 3000, -4, 4, 1, 1023, 1024, -1022, -1023])]).astype(np.int32)
    m = max(len(x), len(vals))
    x = np.resize(x, m) if len(x) < m else x
    vals = np.concatenate([vals, np.ones(m - len(vals))])
    ks = np.concatenate([ks, np.zeros(m - len(ks), np.int32)])
    dev = torch.device("cuda")
    xd, vd = torch.tensor(x, device=dev), torch.tensor(vals, device=dev)
    kd = torch.tensor(ks, device=dev)
    ym, ys = torch.empty_like(xd), torch.empty_like(xd)
    yp = torch.empty(m, dtype=torch.int32, device=dev)
    rc = chem.lib().chem_selftest_scaled_exp(m, xd.data_ptr(), ym.data_ptr(), yp.data_ptr(), vd.data_ptr(),
                                             kd.data_ptr(), ys.data_ptr(), None)
    assert rc == 0
    ym, yp, ys = ym.cpu().numpy(), yp.cpu().numpy(), ys.cpu().numpy()
    # split exponential
    inr = np.isfinite(x) & (np.abs(x) < 2.0 ** 22)
    assert np.all((ym[inr] >= 0.99) & (ym[inr] <= 2.01))
    # reference exp(x - k ln 2): in long double below 1024 (its error there
    # stays under half an ulp of a double even with an 80-bit long double),
    # in 40-digit decimal arithmetic on a sample above
    small = inr & (np.abs(x) < 1024)
    ld = np.longdouble
    ref = np.exp(x[small].astype(ld) - yp[small].astype(ld) * np.log(ld(2)))
    ulp = np.abs(ym[small].astype(ld) - ref) / np.spacing(ref.astype(np.float64)).astype(ld)
    assert float(ulp.max()) <= 2.0, float(ulp.max())
    import decimal
    ctx = decimal.Context(prec=40)
    ln2 = ctx.ln(decimal.Decimal(2))
    big = np.nonzero(inr & ~small)[0]
    for i in big[:: max(1, len(big) // 3000)]:
        r = ctx.exp(ctx.subtract(decimal.Decimal(float(x[i])), ctx.multiply(decimal.Decimal(int(yp[i])), ln2)))
        rf = float(r)
        assert abs(decimal.Decimal(float(ym[i])) - r) <= 2 * decimal.Decimal(float(np.spacing(rf))), (x[i], ym[i], rf)
    out = np.isfinite(x) & (np.abs(x) >= 2.0 ** 22) | np.isinf(x)
    assert np.all(ym[out] == 1.0) and np.all(np.abs(yp[out]) == 2 ** 24)
    assert np.all(np.sign(yp[out]) == np.sign(x[out]))
    assert np.isnan(ym[np.isnan(x)]).all()
    # power-of-two scaling
    tiny = np.finfo(np.float64).tiny
    normal = np.isfinite(vals) & (np.abs(vals) >= tiny)
    with np.errstate(over="ignore", under="ignore"):
        ref = np.ldexp(vals, ks)
    ok = normal & (np.abs(ref) >= tiny) & np.isfinite(ref)
    assert np.array_equal(ys[ok], ref[ok])
    under = normal & (np.abs(ref) < tiny)
    assert np.all(ys[under] == 0.0) and np.array_equal(np.signbit(ys[under]), np.signbit(vals[under]))
    over = normal & ~np.isfinite(ref)
    assert np.all(np.isinf(ys[over])) and np.array_equal(np.sign(ys[over]), np.sign(vals[over]))
    keep = ~normal
    assert np.array_equal(ys[keep], vals[keep], equal_nan=True)


def test_log_of_temperatures():
    """The kernels' table-driven logarithm (Tang's method) within 2 ulp of
    CUDA's log and of the host's, on the temperature-recovery bracket and
    across its domain x >= 2, including table points and midpoints."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    rng = np.random.default_rng(2)
    j = np.arange(129)
    x = np.concatenate([rng.uniform(200.0, 6000.0, 300000),
                        np.exp(rng.uniform(np.log(2.0), 700.0, 100000)),
                        rng.uniform(2.0, 2.01, 20000),
                        (1.0 + j / 128.0) * 1024.0, (1.0 + (j + 0.5) / 128.0) * 256.0,
                        (1.0 + (j + 0.5) / 128.0) * 2.0, np.array([2.0, 200.0, 6000.0, 2.0 ** 1020])])
    dev = torch.device("cuda")
    xd = torch.tensor(x, device=dev)
    y, yr = torch.empty_like(xd), torch.empty_like(xd)
    assert chem.lib().chem_selftest_log(len(x), xd.data_ptr(), y.data_ptr(), yr.data_ptr(), None) == 0
    y, yr = y.cpu().numpy(), yr.cpu().numpy()
    for ref in (yr, np.log(x)):
        ulp = np.abs(y - ref) / np.spacing(np.abs(ref))
        w = int(np.argmax(ulp))
        assert ulp.max() <= 2.0, (ulp.max(), x[w], y[w], ref[w])
