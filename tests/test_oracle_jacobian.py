"""Pins for the oracle's analytic Jacobian d(wdot, Omega_e)/d(rho, e), the
dOmega/dQ of Eq. 29: central finite differences with Richardson
extrapolation of the source through the temperature recovery, plus the
column identities inherited from mass and energy conservation."""
import numpy as np
import pytest

import small_mechs as sm
from paper_1110_4903_gb300 import synth


def _source_of_state(om, x):
    rc, T, _ = om.recover_T(x[:-1], x[-1], 1500.0)
    assert rc == 0
    return om.source(x[:-1], T)


def _col_scales(x):
    rho_tot = x[:-1].sum()
    xs = np.maximum(np.abs(x), 1e-2 * rho_tot)
    xs[-1] = max(abs(x[-1]), 1e5 * rho_tot)
    return xs


def _fd_jacobian(om, x):
    n = x.shape[0]
    xs = _col_scales(x)
    J = np.zeros((n, n))
    for k in range(n):
        h = 1e-4 * xs[k]

        def d(hh):
            xp, xm = x.copy(), x.copy()
            xp[k] += hh
            xm[k] -= hh
            return (_source_of_state(om, xp) - _source_of_state(om, xm)) / (2 * hh)
        J[:, k] = (4 * d(h / 2) - d(h)) / 3
    return J


def _check(J, Jfd, x, tol):
    """Norm-wise relative error of the column-scaled Jacobian, separately
    for the species rows and the energy row (their units differ)."""
    ns = J.shape[0] - 1
    xs = _col_scales(x)
    for rows in (slice(0, ns), slice(ns, ns + 1)):
        A = J[rows] * xs[None, :]
        B = Jfd[rows] * xs[None, :]
        scale = np.abs(A).max()
        assert np.abs(A - B).max() <= tol * scale + 1e-300


@pytest.mark.parametrize("builder", [sm.isomer_pair, sm.dimer_pair, sm.third_body_twin])
def test_small_mechanisms_fd(oracle_mod, builder):
    # the dimer with a7_B = 12 keeps K_b [B] within a few decades of
    # K_f [A]^2, so the differences do not cancel to noise
    mech = builder(a7B=12.0) if builder is sm.dimer_pair else builder()
    if builder is sm.isomer_pair:
        # give the pair different heats so temperature columns matter
        mech.nasa7[1, :, 5] += 300.0
        mech.arr_Ea[:] = 5e4
        mech.arr_beta[:] = 0.7
    om = oracle_mod.OracleMech(mech)
    f = synth.uniform_field(om.ns, 3, 900.0, 2500.0, seed=3)
    rho, e = om.state_from_tpy(f.T, f.P, f.Y)
    for i in range(3):
        x = np.concatenate([rho[:, i], [e[i]]])
        rc, T, _ = om.recover_T(x[:-1], x[-1], 1500.0)
        J = om.jacobian(x[:-1], T)
        _check(J, _fd_jacobian(om, x), x, 1e-7)


def test_h2air_mechanism_fd(oracle_mod):
    om = oracle_mod.OracleMech(synth.h2_air_9sp())
    f = synth.uniform_field(om.ns, 3, 1000.0, 2500.0, seed=5)
    rho, e = om.state_from_tpy(f.T, f.P, f.Y)
    for i in range(3):
        x = np.concatenate([rho[:, i], [e[i]]])
        rc, T, _ = om.recover_T(x[:-1], x[-1], 1500.0)
        _check(om.jacobian(x[:-1], T), _fd_jacobian(om, x), x, 1e-7)


def test_column_identities(oracle_mod):
    # d/dx_k of (sum_s wdot_s) = 0 and of (sum_s e_s^f wdot_s + Omega_e) = 0
    for mech in (synth.h2_air_9sp(), synth.hydrocarbon_36sp()):
        om = oracle_mod.OracleMech(mech)
        ef = om.ef()
        f = synth.uniform_field(om.ns, 4, 800.0, 2800.0, seed=9)
        rho, e = om.state_from_tpy(f.T, f.P, f.Y)
        for i in range(4):
            J = om.jacobian(rho[:, i], f.T[i])
            ns = om.ns
            colsum = J[:ns].sum(0)
            assert np.all(np.abs(colsum) <= 1e-13 * np.abs(J[:ns]).sum(0) + 1e-300)
            en = ef @ J[:ns] + J[ns]
            assert np.all(np.abs(en) <= 1e-13 * np.abs(ef[:, None] * J[:ns]).sum(0) + 1e-300)


def test_reduced_species_system_equals_full_solve(oracle_mod):
    # The kernels solve the Newton system of Eq. 29 on the species unknowns:
    # with the energy row of I - hJ equal to [e_f, 1] - e_f (species rows)
    # (the identity above), the energy equation reduces to the conservation
    # law de = -R_E - e_f . drho, R_E = (x_e - x0_e) + e_f . (x_s - x0_s),
    # and the species rows become (A_sk - a_s e_f,k) drho_k = -F_s + a_s R_E
    # (a_s = A_s,e).  On the oracle's Jacobians the reduced solution solves
    # the full (N_s+1)-unknown system with a componentwise backward error
    # at rounding level (smaller than a direct LU of the badly scaled full
    # system reaches), and matches that direct solution within its
    # conditioning.
    rng = np.random.default_rng(3)
    for mech in (synth.h2_air_9sp(), synth.hydrocarbon_36sp()):
        om = oracle_mod.OracleMech(mech)
        ns = om.ns
        ef = om.ef()
        f = synth.uniform_field(ns, 6, 900.0, 2800.0, seed=11)
        rho, e = om.state_from_tpy(f.T, f.P, f.Y)
        for i in range(6):
            x = np.append(rho[:, i], e[i])
            rc, T, _ = om.recover_T(x[:-1], x[-1], f.T[i])
            assert rc == 0
            J = om.jacobian(x[:-1], T)
            w = om.source(x[:-1], T)
            x0 = x * (1 + 1e-3 * rng.standard_normal(ns + 1))
            for h in (1e-9, 1e-7, 1e-5):
                A = np.eye(ns + 1) - h * J
                b = -(x - x0 - h * w)
                full = np.linalg.solve(A, b)
                RE = (x[ns] - x0[ns]) + ef @ (x[:ns] - x0[:ns])
                a = A[:ns, ns]
                Ar = A[:ns, :ns] - np.outer(a, ef)
                br = b[:ns] + a * RE
                drho = np.linalg.solve(Ar, br)
                de = -RE - ef @ drho
                red = np.append(drho, de)
                r = A @ red - b
                bw = np.max(np.abs(r) / (np.abs(A) @ np.abs(red) + np.abs(b)))
                assert bw <= 1e-11, (mech.name, i, h, bw)
                assert np.all(np.abs(red - full) <= 1e-6 * np.abs(full)), (mech.name, i, h)
                # the right-hand side's conservation: b_e + e_f . b_s = -R_E
                # (the sources cancel: Omega_e = -e_f . wdot)
                assert abs(b[ns] + ef @ b[:ns] + RE) <= 1e-12 * (abs(b[ns]) + np.abs(ef * b[:ns]).sum())
