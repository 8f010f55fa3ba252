"""Pins for the oracle's thermodynamics and temperature recovery (Eq. 3 energy
definition, NASA-7 species data): quadrature of cp, closed forms of
constant-cp species, continuity at T_mid, Dalton's law (Eq. 5)."""
import numpy as np
import pytest
from scipy.integrate import quad

import small_mechs as sm
from paper_1110_4903_gb300 import synth

R = sm.R


@pytest.fixture(scope="module")
def mechs(oracle_mod):
    return [oracle_mod.OracleMech(synth.h2_air_9sp()), oracle_mod.OracleMech(synth.hydrocarbon_36sp())]


def test_enthalpy_and_entropy_are_integrals_of_cp(mechs):
    # h(T2) - h(T1) = int cp dT and s(T2) - s(T1) = int cp/T dT, across T_mid
    for om in mechs:
        for s in range(0, om.ns, 5):
            for T1, T2 in ((300.0, 900.0), (700.0, 2500.0), (1000.0, 4000.0), (250.0, 5800.0)):
                cp = lambda T: om.thermo(s, T)[0]
                dh = quad(cp, T1, T2, points=[1000.0], epsabs=0, epsrel=1e-13)[0]
                ds = quad(lambda T: cp(T) / T, T1, T2, points=[1000.0], epsabs=0, epsrel=1e-13)[0]
                h1, h2 = T1 * om.thermo(s, T1)[1], T2 * om.thermo(s, T2)[1]
                s1, s2 = om.thermo(s, T1)[2], om.thermo(s, T2)[2]
                assert abs((h2 - h1) - dh) <= 1e-10 * max(abs(dh), abs(h1), abs(h2))
                assert abs((s2 - s1) - ds) <= 1e-10 * max(abs(ds), abs(s1), abs(s2))


def test_internal_energy_is_integral_of_cv(mechs):
    for om in mechs:
        for s in range(0, om.ns, 7):
            for T1, T2 in ((300.0, 1500.0), (900.0, 3000.0)):
                de = quad(lambda T: om.species_cv(s, T), T1, T2, points=[1000.0], epsabs=0,
                          epsrel=1e-13)[0]
                got = om.species_e(s, T2) - om.species_e(s, T1)
                assert abs(got - de) <= 1e-10 * abs(de)
                # e = h - R T / M, i.e. e_sens(T_ref) = 0
                assert om.species_esens(s, sm.TREF) == 0.0


def test_continuity_at_t_mid(mechs):
    for om in mechs:
        for s in range(om.ns):
            lo = om.thermo(s, 1000.0)              # tie goes to the low range
            hi = om.thermo(s, np.nextafter(1000.0, 2000.0))
            for a, b in zip(lo, hi):
                assert abs(a - b) <= 1e-11 * max(1.0, abs(a))


def test_range_selection_closed_form(oracle_mod):
    om = oracle_mod.OracleMech(sm.two_range_species())
    assert om.thermo(0, 900.0)[0] == 3.5
    assert om.thermo(0, 1000.0)[0] == 3.5
    assert om.thermo(0, 1100.0)[0] == 4.5


def test_constant_cp_energy_and_temperature_recovery(oracle_mod):
    mech = sm.const_cp_mixture()
    om = oracle_mod.OracleMech(mech)
    W = mech.molar_mass
    a1 = mech.nasa7[:, 0, 0]
    rho = np.array([0.01, 0.2, 0.05])
    for T in (250.0, 298.15, 800.0, 2345.6, 5500.0):
        for s in range(3):
            exact = R / W[s] * (a1[s] - 1.0) * (T - sm.TREF)
            assert abs(om.species_esens(s, T) - exact) <= 1e-12 * max(1.0, abs(exact)) * 10
        e = sum(rho[s] * R / W[s] * (a1[s] - 1.0) * (T - sm.TREF) for s in range(3))
        for guess in (1500.0, 210.0, 5900.0, -1.0, np.nan):
            rc, Tr, it = om.recover_T(rho, e, guess)
            assert rc == 0
            assert abs(Tr - T) <= 1e-12 * T
            assert it <= 50


def test_temperature_recovery_out_of_range_fails(oracle_mod):
    mech = sm.const_cp_mixture()
    om = oracle_mod.OracleMech(mech)
    W = mech.molar_mass
    a1 = mech.nasa7[:, 0, 0]
    rho = np.array([0.01, 0.2, 0.05])
    for T in (150.0, 7000.0):
        e = sum(rho[s] * R / W[s] * (a1[s] - 1.0) * (T - sm.TREF) for s in range(3))
        rc, _, _ = om.recover_T(rho, e)
        assert rc != 0


def test_state_from_tpy_obeys_dalton(mechs):
    # Eq. 5: P = sum_s rho_s R T / M_s, and sum_s rho_s = rho
    for om in mechs:
        f = synth.uniform_field(om.ns, 50, 900.0, 2800.0, seed=11, P=2.0e5)
        rho, e = om.state_from_tpy(f.T, f.P, f.Y)
        P = (rho / om.mech.molar_mass[:, None]).sum(0) * R * f.T
        np.testing.assert_allclose(P, f.P, rtol=1e-13)
        np.testing.assert_allclose(rho / rho.sum(0), f.Y, rtol=1e-13)
        for i in range(5):
            rc, T, _ = om.recover_T(rho[:, i], e[i], 1500.0)
            assert rc == 0 and abs(T - f.T[i]) <= 1e-12 * f.T[i]
