"""Accuracy of the GPU chemistry step against the FP64 oracle, per workload
and precision: max and 99th-percentile relative error of species densities,
temperature and energy, over a sample of cells.  Not a test (it asserts
nothing); run it on a GPU machine:

    python tests/accuracy_report.py [--cells N]

Species use the tests' floor (1e-12 of the cell density) below which
differences count as absolute.  "same path" are the cells whose substep
decisions (accepted substeps and failed attempts) equal the oracle's; the
others took a different, equally valid halving sequence and are reported
separately.
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


def sample(f, n, seed=0):
    """n cells: half uniformly spread, half the hottest (the stiff ones)."""
    if n >= f.n:
        return np.arange(f.n)
    rng = np.random.default_rng(seed)
    hot = np.argsort(f.T)[-4 * n:]
    idx = np.unique(np.concatenate([rng.choice(f.n, n // 2, replace=False), rng.choice(hot, n - n // 2, replace=False)]))
    return np.sort(idx)


def stats(rg, eg, og, rr, er, oo, rho0):
    ok = oo["status"] == 0
    same = ok & (og["substeps"] == oo["substeps"]) & (og["failures"] == oo["failures"])
    rel = P.rel_species(rg, rr, rho0.sum(0))
    relT = np.abs(og["T"] - oo["T"]) / np.abs(oo["T"])
    rel_e = np.abs(eg - er) / (np.abs(er) + np.abs(rho0).sum(0) * 1e6)

    def q(a, m):
        a = a[..., m].ravel() if a.ndim == 2 else a[m]
        return (float(a.max()), float(np.percentile(a, 99))) if a.size else (0.0, 0.0)

    out = dict(cells=int(len(ok)), status_equal=bool(np.array_equal(og["status"], oo["status"])),
               same_path=float(same.sum() / max(1, ok.sum())))
    for name, a in (("species", rel), ("T", relT), ("e", rel_e)):
        mx, p99 = q(a, same)
        out[name + "_max"] = mx
        out[name + "_p99"] = p99
    flip = ok & ~same
    if flip.any():
        out["other_path_species_max"] = float(rel[:, flip].max())
        out["other_path_T_max"] = float(relT[flip].max())
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
        fs = synth.subsample(f, sample(f, args.cells))
        rho, e = P.initial_state(mech, fs)
        opts = dict(max_halvings=0) if wl == "h2air-1k" else {}
        for prec, name, tol in ((chem.FP64, "fp64", P.TOL_FP64), (chem.MIXED, "mixed", P.TOL_MIXED)):
            # the oracle under the path's own Newton control
            ctl = P.MIXED_OPTS if name == "mixed" else {}
            rr, er, oo = P.oracle_reference(mech, rho, e, dt, fs.T, threads=threads, **opts, **ctl)
            c = chem.Chem(mech, precision=prec, **opts)
            rg, eg, og = P.gpu_run(torch, c, rho, e, dt, T_in=fs.T)
            c.close()
            s = stats(rg, eg, og, rr, er, oo, rho)
            s.update(workload=wl, precision=name, tolerance=tol)
            report.append(s)
            print(json.dumps(s), flush=True)


if __name__ == "__main__":
    main()
