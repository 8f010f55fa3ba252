"""GPU-vs-oracle parity of the FP64 chemistry step through the C ABI."""
import os

import numpy as np
import pytest

import parity as P
import small_mechs
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
def h2air(torch):
    from paper_1110_4903_gb300 import chem
    m = synth.h2_air_9sp()
    c = chem.Chem(m)
    yield m, c
    c.close()


@pytest.fixture(scope="module")
def hc36(torch):
    from paper_1110_4903_gb300 import chem
    m = synth.hydrocarbon_36sp()
    c = chem.Chem(m)
    yield m, c
    c.close()


def test_config1_single_be_step_all_cells(torch, h2air):
    # 9 sp / 38 rxn, 1,024 cells, one dt = 1e-7 s BE step, no substepping
    m, _ = h2air
    from paper_1110_4903_gb300 import chem
    c = chem.Chem(m, max_halvings=0)
    mech, f, dt = synth.workload("h2air-1k")
    rho, e = P.initial_state(m, f)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, f.T, threads=THREADS, max_halvings=0)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=f.T)
    st = P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64, min_same=1.0)
    assert st["ok"] == f.n
    assert st["iters_equal"] >= 0.999
    c.close()


@pytest.mark.parametrize("lanes", [2, 4, 8, 16, 32])
def test_every_lane_width_ragged_sizes(torch, h2air, lanes):
    # 1,000 cells (ragged against every slot count), padded leading dimension
    m, c = h2air
    mech, f, _ = synth.workload("h2air-1M")
    idx = np.arange(1000) * 997 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    dt = 1e-6
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T, ld=1003, lanes=lanes)
    P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64)
    P.replay_check(m, rho, e, dt, fs.T, rg, eg, og, P.TOL_FP64, threads=THREADS)


def test_hc36_subset(torch, hc36):
    # 36 sp / 308 rxn, dt = 1e-6 s with adaptive substeps
    m, c = hc36
    mech, f, dt = synth.workload("hc36-256k")
    idx = np.arange(160) * 1637 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
    P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64)
    P.replay_check(m, rho, e, dt, fs.T, rg, eg, og, P.TOL_FP64, threads=THREADS)


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_hc36_lane_widths(torch, hc36, lanes):
    m, c = hc36
    mech, f, dt = synth.workload("hc36-256k")
    idx = np.arange(40) * 7919 % f.n
    fs = synth.subsample(f, idx)
    rho, e = P.initial_state(m, fs)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T, lanes=lanes)
    P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64)
    P.replay_check(m, rho, e, dt, fs.T, rg, eg, og, P.TOL_FP64, threads=THREADS)


def test_edge_cases(torch, h2air):
    m, c = h2air
    mech, f, _ = synth.workload("h2air-1k")
    fs = synth.subsample(f, np.arange(8))
    rho, e = P.initial_state(m, fs)
    # n = 0 is a no-op; n = 1 works
    rg, eg, og = P.gpu_run(torch, c, rho[:, :1], e[:1], 1e-7, T_in=fs.T[:1])
    rr, er, oo = P.oracle_reference(m, rho[:, :1], e[:1], 1e-7, fs.T[:1], threads=1)
    P.compare(rg, eg, og, rr, er, oo, rho[:, :1], P.TOL_FP64)
    # dt = 0: unchanged, status OK, temperature recovered
    rg, eg, og = P.gpu_run(torch, c, rho, e, 0.0)
    assert np.array_equal(rg, rho) and np.array_equal(eg, e) and (og["status"] == 0).all()
    np.testing.assert_allclose(og["T"], fs.T, rtol=1e-12)
    # bad inputs keep their values and report per-cell status
    r2, e2 = rho.copy(), e.copy()
    r2[0, 1] = np.nan                 # non-finite
    r2[:, 2] = 0.0                    # zero density
    e2[3] = 1e12                      # temperature far above the bracket
    e2[4] = -1e9                      # far below it
    rg, eg, og = P.gpu_run(torch, c, r2, e2, 1e-7)
    rr, er, oo = P.oracle_reference(m, r2, e2, 1e-7, None, threads=1)
    assert list(og["status"][1:5]) == [3, 3, 2, 2]
    assert np.array_equal(og["status"], oo["status"])
    assert np.array_equal(rg[:, 1:5], r2[:, 1:5], equal_nan=True)
    ok = og["status"] == 0
    rel = P.rel_species(rg[:, ok], rr[:, ok], rho[:, ok].sum(0))
    assert rel.max() <= P.TOL_FP64


def test_state_and_temperature_kernels(torch, hc36):
    m, c = hc36
    import oracle
    om = oracle.OracleMech(m)
    f = synth.uniform_field(m.ns, 777, 250.0, 5000.0, seed=17)
    rho_ref, e_ref = om.state_from_tpy(f.T, f.P, f.Y)
    dev = torch.device("cuda")
    T = torch.tensor(f.T, device=dev)
    Pp = torch.tensor(f.P, device=dev)
    Y = torch.tensor(f.Y, device=dev)
    rho = torch.zeros_like(Y)
    e = torch.zeros_like(T)
    c.state_from_tpy(T, Pp, Y, rho, e)
    Tout = torch.zeros_like(T)
    c.temperature(rho, e, Tout)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rho.cpu().numpy(), rho_ref, rtol=1e-14)
    np.testing.assert_allclose(e.cpu().numpy(), e_ref, rtol=1e-12, atol=1e-9 * np.abs(e_ref).max())
    np.testing.assert_allclose(Tout.cpu().numpy(), f.T, rtol=1e-12)


@pytest.mark.parametrize("wl,sample", [("h2air-1M", 512), ("hc36-256k", 96), ("hc36-front-2M", 96)])
def test_full_size_sampled(torch, wl, sample):
    """Full-size workloads in the benchmark's launch configuration: every
    cell is checked for conservation; a random sample against the oracle."""
    from paper_1110_4903_gb300 import chem
    m, f, dt = synth.workload(wl)
    c = chem.Chem(m)
    dev = torch.device("cuda")
    T = torch.tensor(f.T, device=dev)
    Pp = torch.tensor(f.P, device=dev)
    Y = torch.tensor(f.Y, device=dev)
    rho = torch.zeros_like(Y)
    e = torch.zeros_like(T)
    c.state_from_tpy(T, Pp, Y, rho, e)
    rho0 = rho.clone()
    e0 = e.clone()
    n = f.n
    T_out = torch.zeros_like(T)
    st = torch.zeros(n, dtype=torch.int32, device=dev)
    it = torch.zeros(n, dtype=torch.int32, device=dev)
    su = torch.zeros(n, dtype=torch.int32, device=dev)
    fa = torch.zeros(n, dtype=torch.int32, device=dev)
    c.advance(rho, e, dt, T_in=T, T_out=T_out, status=st, newton_iters=it, substeps=su, failures=fa)
    torch.cuda.synchronize()
    # conservation of mass and energy in every cell
    ef = torch.tensor(P.oracle.OracleMech(m).ef(), device=dev)
    mass_err = ((rho.sum(0) - rho0.sum(0)).abs() / rho0.sum(0)).max().item()
    U0 = e0 + ef @ rho0
    U1 = e + ef @ rho
    scale = e0.abs() + ef.abs() @ rho0.abs()
    en_err = ((U1 - U0).abs() / scale).max().item()
    assert mass_err <= 1e-13 and en_err <= 1e-13
    stat = st.cpu().numpy()
    assert (stat == 0).mean() >= 0.9999
    rng = np.random.default_rng(123)
    idx = np.unique(np.concatenate([rng.choice(n, sample, replace=False),
                                    np.argsort(-f.T, kind="stable")[:32]]))
    r0 = rho0[:, idx].cpu().numpy()
    e0s = e0[idx].cpu().numpy()
    rr, er, oo = P.oracle_reference(m, r0, e0s, dt, f.T[idx], threads=THREADS)
    # the sampled cells again in a launch of their own, recording their
    # schedules and substep states: bit-identical to the full launch
    rg, eg, og = P.gpu_run(torch, c, r0, e0s, dt, T_in=f.T[idx])
    assert np.array_equal(rg, rho[:, idx].cpu().numpy()) and np.array_equal(eg, e[idx].cpu().numpy())
    assert np.array_equal(og["T"], T_out[idx].cpu().numpy()) and np.array_equal(og["status"], stat[idx])
    assert np.array_equal(og["newton_iters"], it[idx].cpu().numpy())
    P.compare(rg, eg, og, rr, er, oo, r0, P.TOL_FP64)
    P.replay_check(m, r0, e0s, dt, f.T[idx], rg, eg, og, P.TOL_FP64, threads=THREADS)
    c.close()


@pytest.mark.parametrize("wl,ncell,dt", [("h2air-1k", 1024, 1e-7), ("hc36-256k", 128, 1e-9)])
def test_point_implicit_mode(torch, wl, ncell, dt):
    """The scheme exactly as printed (Eq. 29, one linearised step per
    substep, no Newton iteration): GPU against the oracle's same mode.  (On
    the 36-species field at dt = 1e-6 s one linearised step is so
    ill-conditioned that most cells fail the positivity check either way;
    1e-9 s keeps the linear step meaningful.)"""
    from paper_1110_4903_gb300 import chem
    m, f, _ = synth.workload(wl)
    fs = synth.subsample(f, np.arange(ncell) * 131 % f.n)
    rho, e = P.initial_state(m, fs)
    opts = dict(point_implicit=1, max_newton=1, max_halvings=0)
    c = chem.Chem(m, **opts)
    rr, er, oo = P.oracle_reference(m, rho, e, dt, fs.T, threads=THREADS, **opts)
    rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
    assert (og["newton_iters"][oo["status"] == 0] == 1).all()
    P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64, min_same=1.0)
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_maximum_species_count(torch, precision):
    """The largest mechanism the library takes: 64 species (65 x 65 systems,
    so every per-unknown loop runs three passes at 32 lanes per cell), 480
    reactions, against the oracle."""
    from paper_1110_4903_gb300 import chem
    m = synth.hydrocarbon_mechanism(64, 60, 20, 400, 64480, "hc-64sp-480r")
    f = synth.uniform_field(m.ns, 64, 900.0, 2800.0, seed=64)
    rho, e = P.initial_state(m, f)
    dt = 1e-6
    if precision == "fp64":
        c = chem.Chem(m)
        assert c.lanes(chem.FP64) == 32
        rr, er, oo = P.oracle_reference(m, rho, e, dt, f.T, threads=THREADS)
        rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=f.T)
        P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64)
        P.replay_check(m, rho, e, dt, f.T, rg, eg, og, P.TOL_FP64, threads=THREADS)
    else:
        c = chem.Chem(m, precision=chem.MIXED)
        rr, er, oo = P.oracle_reference(m, rho, e, dt, f.T, threads=THREADS, **P.MIXED_OPTS)
        rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=f.T)
        ok = oo["status"] == 0
        assert np.array_equal(og["status"], oo["status"]) and ok.mean() >= 0.95
        P.replay_check(m, rho, e, dt, f.T, rg, eg, og, P.TOL_MIXED, floor=P.FLOOR_MIXED,
                       threads=THREADS)
        P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_MIXED, min_same=0.8, flip_tol=np.inf,
                  floor=P.FLOOR_MIXED)
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coefficient_not_a_power_of_two(torch, precision):
    """3 A <=> A3 gives A a net coefficient of -3.  The kernels' list words hold
    coefficients that are signed powers of two, so the library splits it into
    -2 and -1.  The result agrees with the oracle, which uses the coefficient
    whole."""
    from paper_1110_4903_gb300 import chem
    m = small_mechs.trimer_chain()
    f = synth.uniform_field(m.ns, 96, 900.0, 2000.0, seed=33)
    rho, e = P.initial_state(m, f)
    dt = 1e-6
    if precision == "fp64":
        c = chem.Chem(m)
        rr, er, oo = P.oracle_reference(m, rho, e, dt, f.T, threads=THREADS)
        rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=f.T)
        st = P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_FP64)
        P.replay_check(m, rho, e, dt, f.T, rg, eg, og, P.TOL_FP64, threads=THREADS)
    else:
        c = chem.Chem(m, precision=chem.MIXED)
        rr, er, oo = P.oracle_reference(m, rho, e, dt, f.T, threads=THREADS, **P.MIXED_OPTS)
        rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=f.T)
        # every cell against the oracle replaying its own substep schedule;
        # on this small stiff system the FP32 elimination's slower Newton
        # convergence takes most cells along other halving sequences than
        # the oracle's own run, so only the cells on its schedule are
        # compared with that run
        P.replay_check(m, rho, e, dt, f.T, rg, eg, og, P.TOL_MIXED, floor=P.FLOOR_MIXED,
                       threads=THREADS)
        st = P.compare(rg, eg, og, rr, er, oo, rho, P.TOL_MIXED, min_same=0.0, flip_tol=np.inf,
                       floor=P.FLOOR_MIXED)
    assert st["ok"] == f.n
    # the cells react: every one moved away from its input
    assert (np.abs(rg - rho).max(axis=0) > 1e-6 * rho.sum(axis=0)).all()
    c.close()
