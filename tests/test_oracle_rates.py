"""Pins for the oracle's rate expressions, Sec. 3.2: Arrhenius forward rate
(Eq. 23), equilibrium constant (Eq. 24), progress rate with third body
(Eq. 25), species production (Eq. 26) and mass conservation (Eq. 27)."""
import numpy as np
import pytest

import small_mechs as sm
from paper_1110_4903_gb300 import synth

R, PA = sm.R, sm.PA


@pytest.fixture(scope="module")
def gen_mechs(oracle_mod):
    return [oracle_mod.OracleMech(synth.h2_air_9sp()), oracle_mod.OracleMech(synth.hydrocarbon_36sp())]


def test_isomer_equilibrium_constant_closed_form(oracle_mod):
    om = oracle_mod.OracleMech(sm.isomer_pair(kf=1.0e4, a7A=5.0, a7B=5.7))
    for T in (300.0, 999.0, 1000.0, 1700.0, 4000.0):
        kf, Kc, kb = om.rate_constants(T)
        assert kf[0] == pytest.approx(1.0e4, rel=1e-15)
        assert Kc[0] == pytest.approx(np.exp(0.7), rel=1e-14)
        assert kb[0] == pytest.approx(1.0e4 / np.exp(0.7), rel=1e-14)


def test_dimer_equilibrium_constant_closed_form(oracle_mod):
    # K_c = (R e / P_a) exp(a7_B - 2 a7_A), m^3/mol, for every T
    om = oracle_mod.OracleMech(sm.dimer_pair(A_cgs=1.0e10, a7A=4.0, a7B=3.0))
    for T in (400.0, 1500.0, 3000.0):
        kf, Kc, kb = om.rate_constants(T)
        assert kf[0] == pytest.approx(1.0e4, rel=1e-14)          # 1e10 cm^3 -> 1e4 m^3
        assert Kc[0] == pytest.approx(R * np.e / PA * np.exp(3.0 - 8.0), rel=1e-13)


def test_cgs_to_si_by_order(oracle_mod):
    # beta = E = 0: K_f is A in SI, A_cgs * (1e-6)^(m - 1), m incl. third body
    m = sm.third_body_twin()
    m.arr_beta[:] = 0.0
    m.arr_Ea[:] = 0.0
    om = oracle_mod.OracleMech(m)
    kf, _, _ = om.rate_constants(1234.0)
    assert kf[0] == pytest.approx(1e12 * 1e-6, rel=1e-14)
    assert kf[1] == pytest.approx(1e18 * 1e-12, rel=1e-14)


def _fd_dlog(f, T, h=1e-3):
    d1 = (np.log(f(T + h)) - np.log(f(T - h))) / (2 * h)
    d2 = (np.log(f(T + h / 2)) - np.log(f(T - h / 2))) / h
    return (4 * d2 - d1) / 3


def test_arrhenius_and_van_t_hoff_derivatives(gen_mechs):
    # d ln K_f/dT = beta/T + E/(R T^2); d ln K_c/dT = dH0/(R T^2) - sum(nu)/T
    for om in gen_mechs:
        m = om.mech
        nu = np.zeros((m.nr, m.ns))
        for r in range(m.nr):
            for j in range(3):
                if m.reac_sp[r, j] >= 0:
                    nu[r, m.reac_sp[r, j]] -= m.reac_nu[r, j]
                if m.prod_sp[r, j] >= 0:
                    nu[r, m.prod_sp[r, j]] += m.prod_nu[r, j]
        for T in (700.0, 1400.0, 2600.0):
            kf_fd = _fd_dlog(lambda t: om.rate_constants(t)[0], T)
            Kc_fd = _fd_dlog(lambda t: om.rate_constants(t)[1], T)
            h_RT = np.array([om.thermo(s, T)[1] for s in range(m.ns)])
            dH_RT = nu @ h_RT
            kf_ex = m.arr_beta / T + m.arr_Ea / (R * T * T)
            Kc_ex = dH_RT / T - nu.sum(1) / T
            assert np.abs(kf_fd - kf_ex).max() <= 1e-7 * np.abs(kf_ex).max()
            assert np.abs(Kc_fd - Kc_ex).max() <= 1e-6 * np.abs(Kc_ex).max()


def test_third_body_factor_is_total_concentration(oracle_mod):
    # all efficiencies 1: C_M = sum_s [X_s] = P / (R T) (Eq. 5)
    om = oracle_mod.OracleMech(sm.third_body_twin())
    for T, P in ((900.0, 101325.0), (2100.0, 5e5)):
        Y = np.array([[0.2], [0.3], [0.5]])
        rho, e = om.state_from_tpy(np.array([T]), np.array([P]), Y)
        Q = om.progress(T, rho[:, 0])
        assert Q[1] / Q[0] == pytest.approx(P / (R * T), rel=1e-13)


def test_mass_action_orders(oracle_mod):
    # Q for 2A <=> B: K_f [A]^2 - K_b [B]; scaling [A] by 2 with [B] = 0 gives x4
    om = oracle_mod.OracleMech(sm.dimer_pair())
    W = om.mech.molar_mass
    q1 = om.progress(1500.0, np.array([0.01, 0.0]))[0]
    q2 = om.progress(1500.0, np.array([0.02, 0.0]))[0]
    assert q2 / q1 == pytest.approx(4.0, rel=1e-14)
    kf, _, kb = om.rate_constants(1500.0)
    assert q1 == pytest.approx(kf[0] * (0.01 / W[0]) ** 2, rel=1e-14)
    q3 = om.progress(1500.0, np.array([0.0, 0.05]))[0]
    assert q3 == pytest.approx(-kb[0] * 0.05 / W[1], rel=1e-14)


def _random_states(om, n, seed):
    f = synth.uniform_field(om.ns, n, 800.0, 3000.0, seed=seed)
    rho, e = om.state_from_tpy(f.T, f.P, f.Y)
    return rho, f.T


def test_mass_and_element_conservation_of_sources(gen_mechs):
    # Eq. 27: sum_s wdot_s = 0; each element: sum_s n_se wdot_s / M_s = 0;
    # energy: sum_s e_s(T_ref) wdot_s + Omega_e = 0
    for om in gen_mechs:
        m = om.mech
        ef = om.ef()
        rho, T = _random_states(om, 20, seed=7)
        for i in range(rho.shape[1]):
            w = om.source(rho[:, i], T[i])
            scale = np.abs(w[:-1]).sum()
            assert abs(w[:-1].sum()) <= 1e-14 * scale
            el = m.elem_comp.T @ (w[:-1] / m.molar_mass)
            el_scale = m.elem_comp.T @ np.abs(w[:-1] / m.molar_mass)
            assert np.all(np.abs(el) <= 1e-13 * el_scale + 1e-300)
            assert abs((ef * w[:-1]).sum() + w[-1]) <= 1e-14 * np.abs(ef * w[:-1]).sum()


def test_generated_mechanisms_are_element_balanced(gen_mechs):
    for om in gen_mechs:
        m = om.mech
        for r in range(m.nr):
            v = np.zeros(m.ne, np.int64)
            for j in range(3):
                if m.reac_sp[r, j] >= 0:
                    v -= m.reac_nu[r, j] * m.elem_comp[m.reac_sp[r, j]]
                if m.prod_sp[r, j] >= 0:
                    v += m.prod_nu[r, j] * m.elem_comp[m.prod_sp[r, j]]
            assert not v.any()


def test_equilibrium_constants_as_products_over_factor_slots(oracle_mod):
    # The kernels form 1/K_c (Eq. 24) as a product over the reaction's factor
    # slots (species listed with repetition, up to three per side) of each
    # product's exp(g/RT - ln(P_a/RT)) and each reactant's inverse: that is
    # exp(dG/RT) (RT/P_a)^dnu because dnu is the number of product factors
    # minus reactant factors, and a species on both sides cancels.
    for mech in (synth.h2_air_9sp(), synth.hydrocarbon_36sp()):
        om = oracle_mod.OracleMech(mech)
        for T in (300.0, 800.0, 1500.0, 2800.0, 5000.0):
            g = np.array([om.thermo(s, T)[1] - om.thermo(s, T)[2] for s in range(mech.ns)])
            L = np.log(PA / (R * T))
            _, Kc, _ = om.rate_constants(T)
            for r in range(mech.nr):
                ex = 0.0
                for j in range(3):
                    if mech.prod_sp[r, j] >= 0:
                        ex += mech.prod_nu[r, j] * (g[mech.prod_sp[r, j]] - L)
                    if mech.reac_sp[r, j] >= 0:
                        ex -= mech.reac_nu[r, j] * (g[mech.reac_sp[r, j]] - L)
                # the exponent sums terms of size |g| up to a few hundred
                tol = 1e-15 * (np.abs(g).max() + abs(L)) * 8
                assert abs(ex - np.log(1.0 / Kc[r])) <= tol, (mech.name, T, r)
