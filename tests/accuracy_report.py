"""Accuracy of the GPU chemistry step against the FP64 oracle, per workload
and precision: max and 99th-percentile relative error of species densities,
temperature and energy, over a sample of cells.  Not a test (it asserts
nothing); run it on a GPU machine:

    python tests/accuracy_report.py [--cells N]

Species use the tests' floor (1e-12 of the cell density) below which
differences count as absolute.  "same path" are the cells whose substep
schedule (the accepted / rejected sequence of attempts) equals the
oracle's; every finished cell is also compared with the oracle integrating
it along the GPU's own schedule (the replay), which covers the cells that
took a different, equally valid halving sequence.  Uniform and hottest
cells are reported separately.
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import parity as P  # noqa: E402
from paper_1110_4903_gb300 import synth  # noqa: E402


def samples(f, n, seed=0):
    """n uniformly spread cells, and the n hottest (the stiff ones)."""
    if n >= f.n:
        return {"all": np.arange(f.n)}
    rng = np.random.default_rng(seed)
    return {"uniform": np.sort(rng.choice(f.n, n, replace=False)),
            "hottest": np.sort(np.argsort(-f.T, kind="stable")[:n])}


def _q(a):
    a = a.max(0) if a.ndim == 2 else a
    return (float(a.max()), float(np.percentile(a, 99))) if a.size else (0.0, 0.0)


def replay(mech, rho0, e0, dt, T_in, og, threads, **opts):
    """The oracle along the GPU's own schedule, for the cells it finished."""
    ok = og["status"] == 0
    om = P.oracle.OracleMech(mech)
    na = og["substeps"] + og["failures"]
    return om.advance_batch_replay(rho0[:, ok], e0[ok], dt, og["schedule"][ok], na[ok], T_in=T_in[ok],
                                   threads=threads, opts=P.oracle.replay_opts(**opts),
                                   guides=og["states"][ok])


def stats(rho0, rg, eg, og, rr, er, oo, rep, floor):
    ok = og["status"] == 0
    same = P.same_path(og, oo)
    out = dict(cells=int(len(ok)), status_equal=bool(np.array_equal(og["status"], oo["status"])),
               same_path=float(same.sum() / max(1, ok.sum())))
    rel = P.rel_species(rg, rr, rho0.sum(0), floor)
    relT = np.abs(og["T"] - oo["T"]) / np.abs(oo["T"])
    out["same_path_species_max"], out["same_path_species_p99"] = _q(rel[:, same])
    out["same_path_T_max"], _ = _q(relT[same])
    # every finished cell against the replay of its own schedule
    rp, ep, orp = rep
    good = orp["status"] == 0
    out["replay_failed"] = int((~good).sum())
    relr = P.rel_species(rg[:, ok][:, good], rp[:, good], rho0[:, ok][:, good].sum(0), floor)
    relTr = np.abs(og["T"][ok][good] - orp["T"][good]) / orp["T"][good]
    rele = np.abs(eg[ok][good] - ep[good]) / (np.abs(ep[good]) + np.abs(rho0[:, ok][:, good]).sum(0) * 1e6)
    out["all_cells_species_max"], out["all_cells_species_p99"] = _q(relr)
    out["all_cells_T_max"], out["all_cells_T_p99"] = _q(relTr)
    out["all_cells_e_max"], _ = _q(rele)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=1024)
    args = ap.parse_args()
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    threads = min(16, os.cpu_count() or 1)
    report = []
    for wl in ("h2air-1k", "h2air-1M", "hc36-256k", "hc36-front-2M"):
        mech, f, dt = synth.workload(wl)
        opts = dict(max_halvings=0) if wl == "h2air-1k" else {}
        for part, idx in samples(f, args.cells).items():
            fs = synth.subsample(f, idx)
            rho, e = P.initial_state(mech, fs)
            for prec, name, tol in ((chem.FP64, "fp64", P.TOL_FP64), (chem.MIXED, "mixed", P.TOL_MIXED)):
                c = chem.Chem(mech, precision=prec, **opts)
                rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
                c.close()
                rep = replay(mech, rho, e, dt, fs.T, og, threads, **opts)
                # the oracle under the path's own Newton control, and (mixed)
                # under the default control as well
                ctls = [("own", P.MIXED_OPTS if name == "mixed" else {})]
                if name == "mixed":
                    ctls.append(("default", {}))
                for ctl_name, ctl in ctls:
                    rr, er, oo = P.oracle_reference(mech, rho, e, dt, fs.T, threads=threads, **opts, **ctl)
                    for floor in (P.FLOOR, P.FLOOR_MIXED):
                        s = stats(rho, rg, eg, og, rr, er, oo, rep, floor)
                        s.update(workload=wl, sample=part, precision=name, tolerance=tol,
                                 oracle_control=ctl_name, species_floor=floor)
                        report.append(s)
                        print(json.dumps(s), flush=True)


if __name__ == "__main__":
    main()
