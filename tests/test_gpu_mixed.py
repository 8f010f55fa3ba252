"""Mixed-precision path (Jacobian, D entries and LU in FP32; rates, sources,
residual, update and temperature in FP64) against the FP64 oracle.

Two checks per sample:
  - every cell the GPU finished is compared with the oracle integrating the
    same cell along the GPU's own substep schedule (the replay), so cells
    whose accept/reject decisions differ from the oracle's are checked too;
  - cells whose schedule equals the oracle's own (the oracle run under the
    same Newton control, and under the default control) are compared with
    that run directly, and their fraction is bounded from below."""
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


def _check(m, rho, e, dt, T_in, rg, eg, og, rr, er, oo, min_same, opts=None):
    """Replay of every finished cell, plus the direct comparison of cells on
    the oracle's own path; returns both statistics."""
    assert np.array_equal(og["status"], oo["status"]), int((og["status"] != oo["status"]).sum())
    rep = P.replay_check(m, rho, e, dt, T_in, rg, eg, og, P.TOL_MIXED, floor=P.FLOOR_MIXED,
                         threads=THREADS, **(opts or {}))
    st = P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_MIXED, min_same=min_same, flip_tol=np.inf,
                   floor=P.FLOOR_MIXED)
    return rep, st


@pytest.mark.parametrize("wl,n_uniform,n_hot,opts", [
    ("h2air-1k", 1024, 0, dict(max_halvings=0)),
    ("h2air-1M", 1024, 128, {}),
    ("hc36-256k", 384, 128, {}),
])
def test_mixed_against_oracle(torch, wl, n_uniform, n_hot, opts):
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    idx = P.hot_and_uniform(f, n_uniform, n_hot)
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    c = chem.Chem(m, precision=chem.MIXED, **opts)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS, **opts, **P.MIXED_OPTS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
    rep, st = _check(m, rho, e, dt, fs.T, rg, eg, og, rr, er, oo, 0.85, opts)
    print(wl, "replay", rep, "on-path", st)
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
    _check(m, rho, e, dt, fs.T, rg, eg, og, rr, er, oo, 0.85)
    c.close()


@pytest.mark.parametrize("wl,ncell", [("h2air-1M", 1024), ("hc36-256k", 256)])
def test_mixed_against_default_control_oracle(torch, wl, ncell):
    """Against the oracle with its default Newton control (the norm test
    alone): cells whose schedule equals that oracle's are within the mixed
    bar of it, and every finished cell is within it of its replay."""
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    idx = np.arange(ncell) * 2039 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    c = chem.Chem(m, precision=chem.MIXED)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
    rep, st = _check(m, rho, e, dt, fs.T, rg, eg, og, rr, er, oo, 0.8)
    print(wl, "default-control oracle: replay", rep, "on-path", st)
    c.close()


@pytest.mark.parametrize("wl,sample,hot", [("hc36-256k", 256, 64), ("hc36-front-2M", 256, 64)])
def test_mixed_full_size_sampled(torch, wl, sample, hot):
    """The benchmark's headline path at full size in its launch configuration:
    every cell conserves mass and energy; a random sample plus the hottest
    cells is checked against the oracle's replay of their own schedules and,
    where the schedules agree, against the oracle under the same control."""
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
    # root; the mixed path stops an accepted substep when the contraction-rate
    # estimate of its distance from the root, theta / (1 - theta) |delta|,
    # is at most kappa x tolerance (Hairer & Wanner, Sec. IV.8), so each
    # accepted substep may leave about kappa (rtol + ns atol_rel) of relative
    # mass or energy, carried on.  The estimate takes the last contraction
    # rate for the next one; with the FP32 Jacobian the rate varies between
    # iterations, and the true distance can exceed the estimate: hence the
    # factor 2 (the largest ratio measured over 2^18 cells is about 1.2)
    bound = 1e-13 + 2 * torch.tensor(su, device=dev, dtype=torch.float64) * P.MIXED_OPTS["conv_kappa"] * (
        1e-10 + m.ns * 1e-12)
    assert (((rho.sum(0) - rho0.sum(0)).abs() / rho0.sum(0)) <= bound).all()
    U0, U1 = e0 + ef @ rho0, e + ef @ rho
    assert (((U1 - U0).abs() / (e0.abs() + ef.abs() @ rho0.abs())) <= bound).all()
    assert (st == 0).mean() >= 0.9999
    rng = np.random.default_rng(321)
    idx = np.unique(np.concatenate([rng.choice(n, sample, replace=False),
                                    np.argsort(-f.T, kind="stable")[:hot]]))
    r0, e0s = rho0[:, idx].cpu().numpy(), e0[idx].cpu().numpy()
    rr, er, oo = P.oracle_reference(m, r0, e0s, dt, f.T[idx], threads=THREADS, **P.MIXED_OPTS)
    # the sampled cells again in a launch of their own, recording their
    # schedules and substep states: a cell's result does not depend on the
    # rest of the batch, so it must equal the full launch's bit for bit
    rg, eg, og = P.gpu_run(torch, c, r0, e0s, dt, T_in=f.T[idx])
    assert np.array_equal(rg, rho[:, idx].cpu().numpy()) and np.array_equal(eg, e[idx].cpu().numpy())
    assert np.array_equal(og["T"], T_out[idx].cpu().numpy()) and np.array_equal(og["status"], st[idx])
    assert np.array_equal(og["newton_iters"], it[idx]) and np.array_equal(og["substeps"], su[idx])
    rep, s = _check(m, r0, e0s, dt, f.T[idx], rg, eg, og, rr, er, oo, 0.8)
    print(wl, "replay", rep, "on-path", s)
    c.close()
