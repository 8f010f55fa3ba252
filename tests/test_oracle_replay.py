"""Pins for the oracle's replay mode: one cell integrated along a GIVEN
sequence of accepted and rejected substep attempts (the schedule another
integrator took), each accepted attempt's backward-Euler system (Eq. 29
iterated by Newton) solved to the norm test.

Backward Euler has one solution per sequence of substep sizes, so a replay
is pinned by (1) the closed form of A <=> B composed over the substep sizes a
schedule implies, with those sizes derived here from the halve-on-failure /
double-on-success rule; (2) the oracle's own runs, whose recorded schedule
must replay to the same bits; (3) the inconsistent schedules it must refuse."""
import numpy as np
import pytest

import small_mechs as sm
from paper_1110_4903_gb300 import synth


def _isothermal_state(om, T, rhos):
    rho = np.array(rhos, np.float64)
    e = sum(rho[s] * om.species_esens(s, T) for s in range(om.ns))
    return rho, e


def _bits(accepted):
    words = np.zeros(8, np.uint32)
    for a, acc in enumerate(accepted):
        if acc:
            words[a // 32] |= np.uint32(1 << (a % 32))
    return words


def _substep_sizes(accepted, dt, max_halvings=20):
    """Substep sizes of the accepted attempts: time in units of dt 2^-20,
    h = dt 2^-level with the level raised until the substep fits the time
    left, +1 after a rejected attempt, -1 after an accepted one."""
    total = 1 << max_halvings
    t, level, hs = 0, 0, []
    for acc in accepted:
        while (total >> level) > total - t:
            level += 1
        if acc:
            hs.append(dt * 2.0 ** -level)
            t += total >> level
            level = max(0, level - 1)
        else:
            level += 1
    assert t == total
    return hs


@pytest.mark.parametrize("accepted", [
    [1],
    [0, 1, 1],
    [0, 0, 1, 1, 1],             # dt/4, dt/2 (doubled), the last dt/4
    [0, 1, 0, 1, 1],
    [0, 0, 0, 1, 1, 1, 1],
    [0, 1, 0, 0, 1, 1, 1],
])
def test_isomer_replay_closed_form(oracle_mod, accepted):
    # A <=> B with dH = 0 is linear and isothermal: one BE substep h maps
    #   A -> (A + h kb (A + B)) / (1 + h (kf + kb)),  A + B fixed
    om = oracle_mod.OracleMech(sm.isomer_pair(kf=1.0e4, a7A=5.0, a7B=5.7))
    kf, kb = 1.0e4, 1.0e4 / np.exp(0.7)
    rho, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    dt = 3e-4
    hs = _substep_sizes(accepted, dt)
    A, tot = rho[0], rho.sum()
    for h in hs:
        A = (A + h * kb * tot) / (1 + h * (kf + kb))
    r1, e1, res = om.advance_cell_replay(rho, e, dt, _bits(accepted), len(accepted), 1200.0)
    assert res["status"] == 0
    assert res["substeps"] == sum(accepted) and res["failures"] == len(accepted) - sum(accepted)
    assert r1[0] == pytest.approx(A, rel=1e-13)
    assert r1[1] == pytest.approx(tot - A, rel=1e-13)
    assert res["T"] == pytest.approx(1200.0, rel=1e-13)


@pytest.mark.parametrize("wl", ["h2air-1M", "hc36-256k", "hc36-front-2M"])
def test_replay_of_own_schedule_is_exact(oracle_mod, wl):
    # the oracle's accepted attempts converged within its iteration limit, so
    # a replay without the divergence check takes the same Newton iterates
    mech, f, dt = synth.workload(wl)
    om = oracle_mod.OracleMech(mech)
    idx = np.linspace(0, f.n - 1, 24).astype(int)
    if wl == "hc36-front-2M":
        idx = np.argsort(-f.T)[:24]          # the hot band: many halvings
    fs = synth.subsample(f, idx)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    for kappa in (0.0, 0.01):
        r1, e1, o = om.advance_batch(rho, e, dt, T_in=fs.T, threads=4, schedule=True, states_cap=32,
                                     opts=oracle_mod.default_opts(conv_kappa=kappa))
        assert (o["status"] == 0).all()
        if wl != "h2air-1M":
            assert (o["failures"] > 0).sum() >= 3
        na = o["substeps"] + o["failures"]
        # accepted bits and counts agree
        nbits = np.array([sum(bin(int(w)).count("1") for w in row) for row in o["schedule"]])
        assert np.array_equal(nbits, o["substeps"])
        r2, e2, o2 = om.advance_batch_replay(rho, e, dt, o["schedule"], na, T_in=fs.T, threads=4,
                                             opts=oracle_mod.replay_opts(conv_kappa=kappa))
        assert (o2["status"] == 0).all()
        assert np.array_equal(r2, r1) and np.array_equal(e2, e1)
        assert np.array_equal(o2["T"], o["T"])
        # guided by the oracle's own states after each accepted substep, each
        # substep's Newton starts at (kappa = 0) or near (kappa > 0) its root
        # and converges back to it within the tolerance
        assert (o["substeps"] <= 32).all()
        r3, e3, o3 = om.advance_batch_replay(rho, e, dt, o["schedule"], na, T_in=fs.T, threads=4,
                                             opts=oracle_mod.replay_opts(), guides=o["states"])
        assert (o3["status"] == 0).all()
        rel = np.abs(r3 - r1) / np.maximum(np.abs(r1), 1e-12 * rho.sum(0)[None, :])
        assert rel.max() <= 1e-10
        np.testing.assert_allclose(o3["T"], o["T"], rtol=1e-12)
        # the states the oracle recorded are its own: the last one is the result
        last = o["states"][np.arange(len(na)), o["substeps"] - 1]
        assert np.array_equal(last[:, :-1].T, r1) and np.array_equal(last[:, -1], e1)


def test_replay_refuses_inconsistent_schedules(oracle_mod):
    om = oracle_mod.OracleMech(sm.isomer_pair())
    rho, e = _isothermal_state(om, 1200.0, [0.03, 0.01])
    MISMATCH, NOCONV = oracle_mod.REPLAY_MISMATCH, oracle_mod.REPLAY_NOT_CONVERGED
    cases = [
        ([0, 1], MISMATCH),              # half of dt done, schedule ends
        ([1, 1], MISMATCH),              # an attempt after dt is reached
        ([0] * 21 + [1], MISMATCH),      # level beyond max_halvings = 20
        ([], MISMATCH),                  # nothing done
    ]
    for acc, want in cases:
        r1, e1, res = om.advance_cell_replay(rho, e, 1e-3, _bits(acc), len(acc), 1200.0)
        assert res["status"] == want, acc
        np.testing.assert_array_equal(r1, rho)
        assert e1 == e
    # an accepted attempt whose system cannot meet the norm test in one
    # iteration (the first update is never below tolerance)
    r1, e1, res = om.advance_cell_replay(rho, e, 1e-3, _bits([1]), 1, 1200.0,
                                         opts=oracle_mod.replay_opts(max_newton=1))
    assert res["status"] == NOCONV
    np.testing.assert_array_equal(r1, rho)
    # dt = 0 takes no attempt
    r1, e1, res = om.advance_cell_replay(rho, e, 0.0, _bits([]), 0, 1200.0)
    assert res["status"] == 0
    np.testing.assert_array_equal(r1, rho)


def test_replay_of_a_different_schedule_is_another_valid_step(oracle_mod):
    # forcing extra halvings on a reacting cell gives a different BE
    # discretisation: it still conserves mass and U = e + sum e_f rho, and
    # it differs from the cell's own result by the first-order truncation
    mech, f, dt = synth.workload("hc36-256k")
    om = oracle_mod.OracleMech(mech)
    fs = synth.subsample(f, np.array([int(np.argmax(f.T))]))
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    r1, e1, o = om.advance_batch(rho, e, dt, T_in=fs.T, schedule=True)
    assert o["status"][0] == 0
    na = int(o["substeps"][0] + o["failures"][0])
    own = [(int(o["schedule"][0, a // 32]) >> (a % 32)) & 1 for a in range(na)]
    # one more rejection before the cell's own schedule, which is then cut
    # where it reaches dt, or continued with accepted attempts until it does
    total = 1 << 20
    forced, t, level = [0], 0, 1
    for acc in own + [1] * 64:
        while (total >> level) > total - t:
            level += 1
        forced.append(acc)
        if acc:
            t += total >> level
            level = max(0, level - 1)
        else:
            level += 1
        if t == total:
            break
    assert forced != own
    r2, e2, o2 = om.advance_cell_replay(rho[:, 0], e[0], dt, _bits(forced), len(forced), fs.T[0])
    assert o2["status"] == 0
    ef = om.ef()
    assert abs(r2.sum() - rho[:, 0].sum()) <= 1e-13 * rho[:, 0].sum()
    U0, U2 = e[0] + ef @ rho[:, 0], e2 + ef @ r2
    assert abs(U2 - U0) <= 1e-13 * (abs(e[0]) + np.abs(ef) @ np.abs(rho[:, 0]))
    d = np.abs(r2 - r1[:, 0]).max() / rho[:, 0].sum()
    assert 1e-12 < d < 1e-1
