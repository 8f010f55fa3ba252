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
