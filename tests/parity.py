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
# The mixed path's default Newton control (the library accepts by the
# contraction estimate with safety factor 0.01 there, and by the norm test
# alone on the FP64 path); mixed results are compared with the oracle run
# under the same control, so that substep decisions can be matched.
MIXED_OPTS = dict(conv_kappa=0.01)


def gpu_run(torch, ch, rho, e, dt, T_in=None, n_cells=None, ld=None, **kw):
    """Runs the chemistry step on the device; returns host copies."""
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
    ch.advance(r, ev, dt, n_cells=n, T_in=Tt, T_out=T_out, status=st, newton_iters=it,
               substeps=su, failures=fa, **kw)
    torch.cuda.synchronize()
    return (r[:, : rho.shape[1]].cpu().numpy(), ev.cpu().numpy(),
            dict(T=T_out.cpu().numpy(), status=st.cpu().numpy(), newton_iters=it.cpu().numpy(),
                 substeps=su.cpu().numpy(), failures=fa.cpu().numpy()))


def rel_species(r_gpu, r_ref, rho_tot):
    return np.abs(r_gpu - r_ref) / np.maximum(np.abs(r_ref), FLOOR * rho_tot[None, :])


def compare(r_gpu, e_gpu, og, r_ref, e_ref, oo, rho0, tol, min_same=0.9999, flip_tol=1e-6):
    """Element-wise comparison.  Returns a dict of statistics; asserts the
    bar: statuses equal, cells with identical decision paths (substeps and
    failed attempts) within tol, at least `min_same` of cells on identical
    paths, the rest within flip_tol."""
    rho_tot = rho0.sum(0)
    assert np.array_equal(og["status"], oo["status"]), (
        "status differs in %d cells" % int((og["status"] != oo["status"]).sum()))
    ok = oo["status"] == 0
    same = ok & (og["substeps"] == oo["substeps"]) & (og["failures"] == oo["failures"])
    rel = rel_species(r_gpu, r_ref, rho_tot)
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


def oracle_reference(mech, rho, e, dt, T_in, threads=8, **opts):
    om = oracle.OracleMech(mech)
    return om.advance_batch(rho, e, dt, T_in=T_in, opts=oracle.default_opts(**opts), threads=threads)


def initial_state(mech, f):
    om = oracle.OracleMech(mech)
    return om.state_from_tpy(f.T, f.P, f.Y)
