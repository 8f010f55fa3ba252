"""Pins for the oracle's backward-Euler step (Eq. 29 iterated by Newton) and
its substep control: closed forms for A <=> B and 2A <=> B, the point-implicit
step as printed, conservation, detailed balance at long times."""
import numpy as np
import pytest

import small_mechs as sm
from paper_1110_4903_gb300 import synth

R, PA = sm.R, sm.PA


def _isothermal_state(om, T, rhos):
    rho = np.array(rhos, np.float64)
    e = sum(rho[s] * om.species_esens(s, T) for s in range(om.ns))
    return rho, e


def test_isomer_single_step_closed_form(oracle_mod):
    # A <=> B, dH = 0: T is constant and BE is linear:
    #   A1 = (A0 + h kb (A0 + B0)) / (1 + h (kf + kb))
    om = oracle_mod.OracleMech(sm.isomer_pair(kf=1.0e4, a7A=5.0, a7B=5.7))
    kf, kb = 1.0e4, 1.0e4 / np.exp(0.7)
    rho, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    for h in (1e-6, 1e-4, 3e-3, 1.0):
        r1, e1, res = om.advance_cell(rho, e, h, 1200.0, oracle_mod.default_opts(max_halvings=0))
        assert res["status"] == 0 and res["substeps"] == 1
        assert res["newton_iters"] == 2          # exact step, then a zero update
        A1 = (rho[0] + h * kb * (rho[0] + rho[1])) / (1 + h * (kf + kb))
        assert r1[0] == pytest.approx(A1, rel=1e-13)
        assert r1[1] == pytest.approx(rho.sum() - A1, rel=1e-13)
        assert res["T"] == pytest.approx(1200.0, rel=1e-13)


def test_isomer_many_steps_converge_to_exponential(oracle_mod):
    om = oracle_mod.OracleMech(sm.isomer_pair(kf=1.0e4, a7A=5.0, a7B=5.7))
    kf, kb = 1.0e4, 1.0e4 / np.exp(0.7)
    rho0, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    t_end = 2e-4
    tot = rho0.sum()
    Aeq = tot * kb / (kf + kb)
    exact = Aeq + (rho0[0] - Aeq) * np.exp(-(kf + kb) * t_end)
    errs = []
    for nsteps in (50, 100, 200):
        r = rho0.copy()
        for _ in range(nsteps):
            r, e, res = om.advance_cell(r, e, t_end / nsteps, 1200.0)
            assert res["status"] == 0
        errs.append(abs(r[0] - exact))
    # backward Euler is first order: halving h halves the error
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_point_implicit_step_as_printed(oracle_mod):
    # Eq. 29 with one linearised step: (I - h dOmega/dQ) dQ = h Omega(Q0).
    # 2A <=> B is isothermal at constant e; by hand in concentrations a, b:
    #   f = kf a^2 - kb b,  da = -2 f h,  db = f h  (linearised)
    om = oracle_mod.OracleMech(sm.dimer_pair(A_cgs=1.0e10, a7A=4.0, a7B=12.0))
    W = om.mech.molar_mass
    kf = 1.0e4
    Kc = R * np.e / PA * np.exp(12.0 - 8.0)
    kb = kf / Kc
    T = 1800.0
    rho, e = _isothermal_state(om, T, [0.02, 0.005])
    a0, b0 = rho / W
    h = 2e-4
    f0 = kf * a0 ** 2 - kb * b0
    # Jacobian of (da/dt, db/dt) wrt (a, b): [[-4 kf a, 2 kb], [2 kf a, -kb]]
    M = np.eye(2) - h * np.array([[-4 * kf * a0, 2 * kb], [2 * kf * a0, -kb]])
    rhs = h * np.array([-2 * f0, f0])
    det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
    da = (rhs[0] * M[1, 1] - M[0, 1] * rhs[1]) / det
    db = (M[0, 0] * rhs[1] - rhs[0] * M[1, 0]) / det
    opts = oracle_mod.default_opts(point_implicit=1, max_newton=1, max_halvings=0)
    r1, e1, res = om.advance_cell(rho, e, h, T, opts)
    assert res["status"] == 0 and res["newton_iters"] == 1
    assert r1[0] / W[0] == pytest.approx(a0 + da, rel=1e-12)
    assert r1[1] / W[1] == pytest.approx(b0 + db, rel=1e-12)
    assert e1 == pytest.approx(e, rel=1e-14)


def test_halving_budget_counts(oracle_mod):
    # with one Newton iteration and a convergence test, no substep can be
    # accepted (the first update is never below tolerance): every level
    # fails once, then the cell fails and keeps its input
    om = oracle_mod.OracleMech(sm.isomer_pair())
    rho, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    opts = oracle_mod.default_opts(max_newton=1, max_halvings=6)
    r1, e1, res = om.advance_cell(rho, e, 1e-3, 1200.0, opts)
    assert res["status"] == oracle_mod.NEWTON_FAILED
    assert res["failures"] == 7 and res["newton_iters"] == 7 and res["substeps"] == 0
    np.testing.assert_array_equal(r1, rho)
    assert e1 == e


def test_bad_inputs(oracle_mod):
    om = oracle_mod.OracleMech(sm.isomer_pair())
    rho, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    _, _, res = om.advance_cell(np.array([np.nan, 0.01]), e, 1e-6)
    assert res["status"] == oracle_mod.BAD_INPUT
    _, _, res = om.advance_cell(np.array([0.0, 0.0]), e, 1e-6)
    assert res["status"] == oracle_mod.BAD_INPUT
    _, _, res = om.advance_cell(rho, e, -1e-6)
    assert res["status"] == oracle_mod.BAD_INPUT
    r1, e1, res = om.advance_cell(rho, e, 0.0)
    assert res["status"] == 0 and res["newton_iters"] == 0
    np.testing.assert_array_equal(r1, rho)
    _, _, res = om.advance_cell(rho, 1e12, 1e-6)
    assert res["status"] == oracle_mod.T_FAILED


@pytest.mark.parametrize("wl", ["h2air-1k", "hc36-256k"])
def test_conservation_per_step(oracle_mod, wl):
    # BE preserves linear invariants and J satisfies them: total mass,
    # element moles and U = e + sum_s rho_s e_s(T_ref) are conserved
    mech, f, dt = synth.workload(wl)
    om = oracle_mod.OracleMech(mech)
    idx = np.arange(0, f.n, f.n // 12)[:12]
    fs = synth.subsample(f, idx)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    r1, e1, out = om.advance_batch(rho, e, dt, T_in=fs.T, threads=4)
    assert np.all(out["status"] == 0)
    ef = om.ef()
    np.testing.assert_allclose(r1.sum(0), rho.sum(0), rtol=1e-13)
    el0 = mech.elem_comp.T @ (rho / mech.molar_mass[:, None])
    el1 = mech.elem_comp.T @ (r1 / mech.molar_mass[:, None])
    np.testing.assert_allclose(el1, el0, rtol=1e-12)
    U0 = e + ef @ rho
    U1 = e1 + ef @ r1
    scale = np.abs(e) + np.abs(ef) @ np.abs(rho)
    assert np.all(np.abs(U1 - U0) <= 1e-13 * scale)
    assert np.any(np.abs(r1 - rho).max(0) > 1e-6 * rho.sum(0))  # it did react


def test_detailed_balance_at_long_times(oracle_mod):
    # after many long BE steps every reaction sits at equilibrium:
    # K_f prod [X]^nu' = K_b prod [X]^nu'' (Eq. 24-25 with Q_r = 0)
    mech = synth.h2_air_9sp()
    om = oracle_mod.OracleMech(mech)
    f = synth.uniform_field(mech.ns, 2, 1500.0, 2500.0, seed=21)
    rho, e = om.state_from_tpy(f.T, f.P, f.Y)
    for i in range(2):
        r, ei, T = rho[:, i].copy(), e[i], f.T[i]
        for h in np.geomspace(1e-8, 1.0, 200):
            r, ei, res = om.advance_cell(r, ei, h, T)
            assert res["status"] == 0
            T = res["T"]
        kf, Kc, kb = om.rate_constants(T)
        c = r / mech.molar_mass
        for rr in range(mech.nr):
            Pf = np.prod([c[mech.reac_sp[rr, j]] ** mech.reac_nu[rr, j] for j in range(3)
                          if mech.reac_sp[rr, j] >= 0])
            Pb = np.prod([c[mech.prod_sp[rr, j]] ** mech.prod_nu[rr, j] for j in range(3)
                          if mech.prod_sp[rr, j] >= 0])
            fwd, rev = kf[rr] * Pf, kb[rr] * Pb
            if max(fwd, rev) > 1e-200:
                assert abs(np.log(fwd) - np.log(rev)) <= 1e-8, (rr, fwd, rev)


@pytest.mark.parametrize("wl", ["h2air-1k", "hc36-256k"])
@pytest.mark.parametrize("kappa", [0.01, 1.0])
def test_rate_stop_stays_within_its_bound(oracle_mod, wl, kappa):
    # the contraction-rate stop (Hairer & Wanner, Solving ODEs II, Sec. IV.8)
    # promises that the iterate it accepts is within kappa * tolerance of the
    # Newton limit; the iterate converged to norm <= 1 one step further stands
    # in for that limit.  It never needs more iterations than the plain test.
    mech, f, dt = synth.workload(wl)
    om = oracle_mod.OracleMech(mech)
    idx = np.linspace(0, f.n - 1, 48).astype(int)
    fs = synth.subsample(f, idx)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    h = dt / 4
    r0, e0, a = om.advance_batch(rho, e, h, T_in=fs.T,
                                 opts=oracle_mod.default_opts(conv_kappa=0.0, max_halvings=0))
    r1, e1, b = om.advance_batch(rho, e, h, T_in=fs.T,
                                 opts=oracle_mod.default_opts(conv_kappa=kappa, max_halvings=0))
    ok = (a["status"] == 0) & (b["status"] == 0)
    assert ok.sum() >= 12
    tol = 1e-10 * np.abs(r0) + 1e-12 * r0.sum(0)
    assert (np.abs(r1 - r0) / tol)[:, ok].max() <= kappa
    assert (b["newton_iters"] <= a["newton_iters"])[ok].all()
    assert (b["newton_iters"] < a["newton_iters"])[ok].sum() >= 4
