"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

import oracle
from paper_1110_4903_gb300 import synth

# Tolerances (relative error, per result).  FP64: the oracle's own results
# move by ~1e-12 under a 1-ulp perturbation of the inputs at these
# conditionings, so 1e-10 leaves two decades.  Species use a floor of
# 1e-12 of the cell density below which differences are absolute.
TOL_FP64 = 1e-10
TOL_MIXED = 1e-6
FLOOR = 1e-12
# The mixed path's floor: its Newton iterations stop at the same tolerances
# as the FP64 path's (rtol 1e-10, atol 1e-12 rho) but converge linearly, so
# trace species carry absolute differences near atol; 1e-9 rho keeps those
# below the 1e-6 bar.
FLOOR_MIXED = 1e-9
# The mixed path's default Newton control (the library accepts by the
# contraction estimate with safety factor 0.01 there, and by the norm test
# alone on the FP64 path); mixed results are compared with the oracle run
# under the same control, so that substep decisions can be matched.
MIXED_OPTS = dict(conv_kappa=0.01)
SCHED_WORDS = 8
SUBSTEP_STATES = 32


def gpu_run(torch, ch, rho, e, dt, T_in=None, n_cells=None, ld=None, schedule=True, **kw):
    """Runs the chemistry step on the device; returns host copies (and, with
    schedule=True, the per-cell substep schedule as og["schedule"], [n, 8]
    uint32, and the states after accepted substeps as og["states"],
    [n, 32, ns+1])."""
    dev = torch.device("cuda")
    n = e.shape[0] if n_cells is None else n_cells
    ld = rho.shape[1] if ld is None else ld
    r = torch.zeros((rho.shape[0], ld), dtype=torch.float64, device=dev)
    r[:, : rho.shape[1]] = torch.tensor(rho, device=dev)
    ev = torch.tensor(e, device=dev)
    Tt = None if T_in is None else torch.tensor(T_in, device=dev)
    T_out = torch.zeros(n, dtype=torch.float64, device=dev)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    it = torch.zeros(n, dtype=torch.int32, device=dev)
    su = torch.zeros(n, dtype=torch.int32, device=dev)
    fa = torch.zeros(n, dtype=torch.int32, device=dev)
    sc = torch.full((n, SCHED_WORDS), -1, dtype=torch.int32, device=dev) if schedule else None
    ss = torch.full((n, SUBSTEP_STATES, rho.shape[0] + 1), float("nan"), dtype=torch.float64,
                    device=dev) if schedule else None
    ch.advance(r, ev, dt, n_cells=n, T_in=Tt, T_out=T_out, status=st, newton_iters=it,
               substeps=su, failures=fa, schedule=sc, substep_states=ss, **kw)
    torch.cuda.synchronize()
    out = dict(T=T_out.cpu().numpy(), status=st.cpu().numpy(), newton_iters=it.cpu().numpy(),
               substeps=su.cpu().numpy(), failures=fa.cpu().numpy())
    if schedule:
        out["schedule"] = sc.cpu().numpy().view(np.uint32)
        out["states"] = ss.cpu().numpy()
    return r[:, : rho.shape[1]].cpu().numpy(), ev.cpu().numpy(), out


def rel_species(r_gpu, r_ref, rho_tot, floor=FLOOR):
    return np.abs(r_gpu - r_ref) / np.maximum(np.abs(r_ref), floor * rho_tot[None, :])


def same_path(og, oo):
    """Cells both sides finished along the same substep schedule: equal
    counts, and equal accepted-attempt bits where both records exist."""
    ok = (oo["status"] == 0) & (og["status"] == 0)
    same = ok & (og["substeps"] == oo["substeps"]) & (og["failures"] == oo["failures"])
    if "schedule" in og and "schedule" in oo:
        same &= (og["schedule"] == oo["schedule"]).all(1)
    return same


def compare(r_gpu, e_gpu, og, r_ref, e_ref, oo, rho0, tol, min_same=0.9999, flip_tol=1e-6,
            floor=FLOOR):
    """Element-wise comparison.  Returns a dict of statistics; asserts the
    bar: statuses equal, cells with identical decision paths (the same
    substep schedule) within tol, at least `min_same` of cells on identical
    paths, the rest within flip_tol."""
    rho_tot = rho0.sum(0)
    assert np.array_equal(og["status"], oo["status"]), (
        "status differs in %d cells" % int((og["status"] != oo["status"]).sum()))
    ok = oo["status"] == 0
    same = same_path(og, oo)
    rel = rel_species(r_gpu, r_ref, rho_tot, floor)
    relT = np.abs(og["T"] - oo["T"]) / np.abs(oo["T"])
    e_scale = np.abs(e_ref) + np.abs(rho0).sum(0) * 1e6
    rel_e = np.abs(e_gpu - e_ref) / e_scale
    frac_same = same.sum() / max(1, ok.sum())
    stats = dict(n=len(ok), ok=int(ok.sum()), same=int(same.sum()), frac_same=float(frac_same),
                 max_rel_species=float(rel[:, same].max()) if same.any() else 0.0,
                 max_rel_T=float(relT[same].max()) if same.any() else 0.0,
                 max_rel_e=float(rel_e[same].max()) if same.any() else 0.0,
                 iters_equal=float((og["newton_iters"] == oo["newton_iters"])[ok].mean()) if ok.any() else 1.0)
    if same.any():
        assert rel[:, same].max() <= tol, stats
        assert relT[same].max() <= tol, stats
        assert rel_e[same].max() <= tol, stats
    assert frac_same >= min_same, stats
    flip = ok & ~same
    if flip.any():
        assert rel[:, flip].max() <= flip_tol, stats
    # failed cells keep their input exactly
    bad = ~ok
    if bad.any():
        assert np.array_equal(r_gpu[:, bad], rho0[:, bad])
    return stats


def replay_check(mech, rho0, e0, dt, T_in, r_gpu, e_gpu, og, tol, floor=FLOOR, threads=8,
                 **opts):
    """Every cell the GPU finished, against the oracle integrating the same
    cell along the GPU's own substep schedule (oracle.advance_batch_replay:
    each accepted attempt's backward-Euler system solved to the norm test,
    Newton started from the GPU's state after that substep where
    og["states"] holds it, so that where a system has several roots the
    oracle takes the GPU's).  Asserts that every replay succeeds and every
    result (species, T, e) is within tol; returns the statistics."""
    ok = og["status"] == 0
    na = og["substeps"] + og["failures"]
    assert (na[ok] <= 32 * SCHED_WORDS).all()
    guides = og.get("states")
    if guides is not None:
        assert (og["substeps"][ok] <= SUBSTEP_STATES).all()
        guides = guides[ok]
    om = oracle.OracleMech(mech)
    rr, er, orp = om.advance_batch_replay(rho0[:, ok], e0[ok], dt, og["schedule"][ok], na[ok],
                                          T_in=None if T_in is None else np.asarray(T_in)[ok],
                                          opts=oracle.replay_opts(**opts), threads=threads,
                                          guides=guides)
    bad = orp["status"] != 0
    assert not bad.any(), "replay failed in %d cells (statuses %s)" % (
        int(bad.sum()), sorted(set(orp["status"][bad].tolist())))
    rho_tot = rho0[:, ok].sum(0)
    rel = rel_species(r_gpu[:, ok], rr, rho_tot, floor)
    relT = np.abs(og["T"][ok] - orp["T"]) / orp["T"]
    e_scale = np.abs(er) + np.abs(rho0[:, ok]).sum(0) * 1e6
    rel_e = np.abs(e_gpu[ok] - er) / e_scale
    stats = dict(replayed=int(ok.sum()), max_rel_species=float(rel.max()) if ok.any() else 0.0,
                 p99_rel_species=float(np.percentile(rel.max(0), 99)) if ok.any() else 0.0,
                 max_rel_T=float(relT.max()) if ok.any() else 0.0,
                 max_rel_e=float(rel_e.max()) if ok.any() else 0.0)
    assert stats["max_rel_species"] <= tol, stats
    assert stats["max_rel_T"] <= tol, stats
    assert stats["max_rel_e"] <= tol, stats
    return stats


def oracle_reference(mech, rho, e, dt, T_in, threads=8, schedule=True, **opts):
    om = oracle.OracleMech(mech)
    return om.advance_batch(rho, e, dt, T_in=T_in, opts=oracle.default_opts(**opts), threads=threads,
                            schedule=schedule)


def initial_state(mech, f):
    om = oracle.OracleMech(mech)
    return om.state_from_tpy(f.T, f.P, f.Y)


def hot_and_uniform(f, n_uniform, n_hot, stride=1637):
    """Indices of a strided uniform sample plus the hottest cells."""
    idx = np.unique(np.concatenate([np.arange(n_uniform) * stride % f.n,
                                    np.argsort(-f.T, kind="stable")[:n_hot]]))
    return idx
