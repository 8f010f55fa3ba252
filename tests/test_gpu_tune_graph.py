"""Autotuner and captured-graph steps (persistent work-stealing kernel under
a CUDA graph) on the uneven front field."""
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


@pytest.fixture(scope="module")
def front(torch):
    m, f, dt = synth.workload("hc36-front-2M")
    # a band-crossing strip of rows: cold gas, both tanh edges and the hot band
    rows = np.arange(0, 1024, 64)
    idx = (rows[:, None] * 2048 + np.arange(2048)[None, :]).reshape(-1)
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    return m, fs, rho, e, dt


def test_autotune_then_parity(torch, front):
    from paper_1110_4903_gb300 import chem
    m, fs, rho, e, dt = front
    dev = torch.device("cuda")
    c = chem.Chem(m, precision=chem.MIXED)
    r = torch.tensor(rho, device=dev)
    ev = torch.tensor(e, device=dev)
    T = torch.tensor(fs.T, device=dev)
    lanes, wpb = c.autotune(r, ev, dt, T_in=T, precision=chem.MIXED)
    assert lanes in (8, 16, 32) and 1 <= wpb <= 10
    assert c.lanes(chem.MIXED) == lanes
    assert np.array_equal(r.cpu().numpy(), rho)        # the tuner worked on a copy
    # parity of the tuned shape on a sample containing band cells
    idx = np.concatenate([np.arange(0, rho.shape[1], 811)[:40], np.where(fs.T > 2500)[0][:40]])
    rr, er, oo = P.oracle_reference(m, rho[:, idx], e[idx], dt, fs.T[idx], threads=THREADS, **P.MIXED_OPTS)
    rg, eg, og = P.gpu_run(torch, c, rho[:, idx], e[idx], dt, T_in=fs.T[idx])
    P.replay_check(m, rho[:, idx], e[idx], dt, fs.T[idx], rg, eg, og, P.TOL_MIXED, floor=P.FLOOR_MIXED,
                   threads=THREADS)
    P.compare(rg, eg, og, rr, er, oo, rho[:, idx], P.TOL_MIXED, min_same=0.9, flip_tol=np.inf,
              floor=P.FLOOR_MIXED)
    c.close()


def test_graph_steps_match_plain_steps(torch, front):
    from paper_1110_4903_gb300 import chem
    m, fs, rho, e, dt = front
    dev = torch.device("cuda")
    c = chem.Chem(m)
    r_g = torch.tensor(rho, device=dev)
    e_g = torch.tensor(e, device=dev)
    st = torch.zeros(e.shape[0], dtype=torch.int32, device=dev)
    g = c.graph(r_g, e_g, dt, status=st)
    r_p = torch.tensor(rho, device=dev)
    e_p = torch.tensor(e, device=dev)
    before = c.launch_count()
    for step in range(2):
        g.launch()
        c.advance(r_p, e_p, dt)
        torch.cuda.synchronize()
        assert torch.equal(r_g, r_p) and torch.equal(e_g, e_p), step
    assert c.launch_count() - before == 4
    assert (st == 0).all()
    g.close()
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_segmented_equals_single_launch_and_oracle(torch, front, precision):
    """Domain-segmented execution (Sec. 5.2): launches over segments of the
    field give the single launch's results bit for bit, and a sample of the
    cells (band cells included) matches the oracle: directly where the
    substep schedules agree, through the replay of the GPU's schedule for
    every cell."""
    from paper_1110_4903_gb300 import chem
    m, fs, rho, e, dt = front
    dev = torch.device("cuda")
    prec = chem.MIXED if precision == "mixed" else chem.FP64
    c = chem.Chem(m, precision=prec)
    n = e.shape[0]
    T = torch.tensor(fs.T, device=dev)
    r1, e1 = torch.tensor(rho, device=dev), torch.tensor(e, device=dev)
    c.advance(r1, e1, dt, T_in=T)
    for seg in (4096, 5000, 32768):
        r2, e2 = torch.tensor(rho, device=dev), torch.tensor(e, device=dev)
        outs = [torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(4)]
        T_out = torch.zeros(n, dtype=torch.float64, device=dev)
        sc = torch.zeros((n, P.SCHED_WORDS), dtype=torch.int32, device=dev)
        ss = torch.zeros((n, P.SUBSTEP_STATES, m.ns + 1), dtype=torch.float64, device=dev)
        c.advance_segmented(r2, e2, dt, seg, T_in=T, T_out=T_out, status=outs[0], newton_iters=outs[1],
                            substeps=outs[2], failures=outs[3], schedule=sc, substep_states=ss)
        torch.cuda.synchronize()
        assert torch.equal(r1, r2) and torch.equal(e1, e2), seg
    idx = np.unique(np.concatenate([np.arange(0, n, 499)[:48], np.where(fs.T > 2500)[0][::37][:48]]))
    st, it, su, fa = (t.cpu().numpy()[idx] for t in outs)
    og = dict(T=T_out.cpu().numpy()[idx], status=st, newton_iters=it, substeps=su, failures=fa,
              schedule=sc.cpu().numpy().view(np.uint32)[idx], states=ss.cpu().numpy()[idx])
    rg, eg = r2.cpu().numpy()[:, idx], e2.cpu().numpy()[idx]
    opts = P.MIXED_OPTS if precision == "mixed" else {}
    tol = P.TOL_MIXED if precision == "mixed" else P.TOL_FP64
    floor = P.FLOOR_MIXED if precision == "mixed" else P.FLOOR
    rr, er, oo = P.oracle_reference(m, rho[:, idx], e[idx], dt, fs.T[idx], threads=THREADS, **opts)
    P.replay_check(m, rho[:, idx], e[idx], dt, fs.T[idx], rg, eg, og, tol, floor=floor, threads=THREADS)
    if precision == "mixed":
        P.compare(rg, eg, og, rr, er, oo, rho[:, idx], tol, min_same=0.85, flip_tol=np.inf, floor=floor)
    else:
        P.compare(rg, eg, og, rr, er, oo, rho[:, idx], tol)
    c.close()
