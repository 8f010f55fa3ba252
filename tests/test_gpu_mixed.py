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


@pytest.mark.parametrize("wl,sample", [("hc36-256k", 96), ("hc36-front-2M", 96)])
def test_mixed_full_size_sampled(torch, wl, sample):
    """The benchmark's headline path at full size in its launch configuration:
    every cell conserves mass and energy, a random sample matches the oracle
    under the same Newton control."""
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    c = chem.Chem(m, precision=chem.MIXED)
    dev = torch.device("cuda")
    T = torch.tensor(f.T, device=dev)
    Y = torch.tensor(f.Y, device=dev)
    rho = torch.zeros_like(Y)
    e = torch.zeros_like(T)
    c.state_from_tpy(T, torch.tensor(f.P, device=dev), Y, rho, e)
    rho0, e0 = rho.clone(), e.clone()
    n = f.n
    T_out = torch.zeros_like(T)
    outs = [torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(4)]
    c.advance(rho, e, dt, T_in=T, T_out=T_out, status=outs[0], newton_iters=outs[1], substeps=outs[2],
              failures=outs[3])
    torch.cuda.synchronize()
    ef = torch.tensor(P.oracle.OracleMech(m).ef(), device=dev)
    st, it, su, fa = (t.cpu().numpy() for t in outs)
    # conservation: BE conserves mass and U = e + sum e_f rho exactly at its
    # root; the mixed path stops an accepted substep up to kappa x tolerance
    # away from the root (contraction-rate stop), so each accepted substep may
    # leave kappa (rtol + ns atol_rel) of relative mass or energy, carried on
    bound = 1e-13 + torch.tensor(su, device=dev, dtype=torch.float64) * P.MIXED_OPTS["conv_kappa"] * (
        1e-10 + m.ns * 1e-12)
    assert (((rho.sum(0) - rho0.sum(0)).abs() / rho0.sum(0)) <= bound).all()
    U0, U1 = e0 + ef @ rho0, e + ef @ rho
    assert (((U1 - U0).abs() / (e0.abs() + ef.abs() @ rho0.abs())) <= bound).all()
    assert (st == 0).mean() >= 0.9999
    rng = np.random.default_rng(321)
    idx = np.sort(rng.choice(n, sample, replace=False))
    r0, e0s = rho0[:, idx].cpu().numpy(), e0[idx].cpu().numpy()
    rr, er, oo = P.oracle_reference(m, r0, e0s, dt, f.T[idx], threads=THREADS, **P.MIXED_OPTS)
    og = dict(T=T_out[idx].cpu().numpy(), status=st[idx], newton_iters=it[idx], substeps=su[idx],
              failures=fa[idx])
    s = _stats(rho[:, idx].cpu().numpy(), e[idx].cpu().numpy(), og, rr, er, oo, r0)
    assert s["status_equal"] == 1.0
    assert s["max_rel_same"] <= P.TOL_MIXED and s["max_relT_same"] <= P.TOL_MIXED
    assert s["frac_same"] >= 0.85
    c.close()
