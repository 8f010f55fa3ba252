"""Mixed-precision path (Jacobian, D entries and LU in FP32; rates, sources,
residual, update and temperature in FP64) against the FP64 oracle."""
import os

import numpy as np
import pytest

import parity as P
from paper_1110_4903_gb300 import synth

pytestmark = pytest.mark.gpu
THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return t


def _stats(rg, eg, og, rr, er, oo, rho0):
    ok = oo["status"] == 0
    same = ok & (og["substeps"] == oo["substeps"]) & (og["failures"] == oo["failures"])
    rel9 = np.abs(rg - rr) / np.maximum(np.abs(rr), 1e-9 * rho0.sum(0)[None, :])
    relT = np.abs(og["T"] - oo["T"]) / oo["T"]
    return dict(n=len(ok), status_equal=float((og["status"] == oo["status"]).mean()),
                frac_same=float(same.mean()),
                max_rel_same=float(rel9[:, same].max()) if same.any() else 0.0,
                max_relT_same=float(relT[same].max()) if same.any() else 0.0,
                max_rel_all=float(rel9[:, ok].max()), max_relT_all=float(relT[ok].max()),
                iters_ratio=float(og["newton_iters"][ok].sum() / max(1, oo["newton_iters"][ok].sum())))


@pytest.mark.parametrize("wl,ncell,opts", [("h2air-1k", 1024, dict(max_halvings=0)),
                                           ("h2air-1M", 512, {}), ("hc36-256k", 128, {})])
def test_mixed_against_oracle(torch, wl, ncell, opts):
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    idx = np.arange(ncell) * 1637 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    c = chem.Chem(m, precision=chem.MIXED, **opts)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS, **opts, **P.MIXED_OPTS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
    st = _stats(rg, eg, og, rr, er, oo, rho)
    print(wl, st)
    assert st["status_equal"] == 1.0
    assert st["max_rel_same"] <= P.TOL_MIXED and st["max_relT_same"] <= P.TOL_MIXED
    assert st["frac_same"] >= 0.9
    c.close()


@pytest.mark.parametrize("wl,ncell,lanes", [("h2air-1M", 1000, 2), ("h2air-1M", 1000, 4), ("h2air-1M", 1000, 8),
                                            ("h2air-1M", 1000, 16), ("h2air-1M", 1000, 32),
                                            ("hc36-256k", 64, 8), ("hc36-256k", 64, 16)])
def test_mixed_every_lane_width(torch, wl, ncell, lanes):
    # every FP32 kernel instantiation against the oracle under the same
    # Newton control: the elimination's row splits (fewer columns than lanes),
    # the per-lane-count gather layouts and the shuffle argmax of G < 32
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    idx = np.arange(ncell) * 997 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    c = chem.Chem(m, precision=chem.MIXED, lanes_per_cell=lanes)
    assert c.lanes(chem.MIXED) == lanes
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS, **P.MIXED_OPTS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T, ld=ncell + 3)
    st = _stats(rg, eg, og, rr, er, oo, rho)
    assert st["status_equal"] == 1.0
    assert st["max_rel_same"] <= P.TOL_MIXED and st["max_relT_same"] <= P.TOL_MIXED
    assert st["frac_same"] >= 0.85
    c.close()
