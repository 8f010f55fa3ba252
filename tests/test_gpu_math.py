"""The step kernel's own exp and reciprocal against CUDA's exp and IEEE
division: at most 2 ulp apart on the ranges the rates use, identical on the
special values."""
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
