"""Operator-split reacting flow in one dimension (Eq. 4): each fluid step is
a convection half -- a stand-in first-order upwind advection of the
conserved densities (rho_s, e) at constant velocity on a periodic domain,
in plain torch operations -- followed by the chemistry half on the GPU
through the library (a captured-graph chemistry step when the buffers stay
fixed).  Domain totals of mass and of U = e + sum_s rho_s e_f,s are
conserved by both halves.

  python -m paper_1110_4903_gb300.coupled_demo [--cells 4096] [--steps 20]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def initial_field(mech, cells):
    """A hot kernel (2400 K, with a small pool of H, O and OH radicals) in
    cold H2-air reactants at 1 atm: (T [cells], P [cells], Y [ns, cells])."""
    x = np.arange(cells) / cells
    g = np.exp(-((x - 0.5) / 0.05) ** 2)
    T = 400.0 + 2000.0 * g
    Y = np.zeros((mech.ns, cells))
    names = mech.species
    rad = {"H": 2e-4, "O": 1e-3, "OH": 2e-3}
    for sp, y in rad.items():
        Y[names.index(sp)] = y * g
    rest = 1.0 - Y.sum(0)
    Y[names.index("H2")] = 0.028 * rest
    Y[names.index("O2")] = 0.226 * rest
    Y[names.index("N2")] = 0.746 * rest
    return T, np.full(cells, 101325.0), Y


def advect(rho, e, c, roll):
    """The convection half: first-order upwind advection of the conserved
    densities at Courant number c on a periodic domain, in place, for torch
    tensors or numpy arrays (`roll(a, shift, axis)`): a <- a - c (a - a[i-1]),
    each element by the same IEEE operations on either."""
    rho -= c * (rho - roll(rho, 1, 1))
    e -= c * (e - roll(e, 1, 0))


def run(cells=4096, steps=20, cfl=0.5, dx=50e-6, u=500.0, precision=1, use_graph=True):
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1110_4903_gb300 import chem, synth
    mech = synth.h2_air_9sp()
    ch = chem.Chem(mech, precision=precision)
    dev = torch.device("cuda")
    T, P, Y = initial_field(mech, cells)
    Tt = torch.tensor(T, device=dev)
    rho = torch.empty((mech.ns, cells), dtype=torch.float64, device=dev)
    e = torch.empty(cells, dtype=torch.float64, device=dev)
    ch.state_from_tpy(Tt, torch.tensor(P, device=dev), torch.tensor(Y, device=dev), rho, e)
    rho0, e0 = rho.clone(), e.clone()
    dt = cfl * dx / u
    ef = torch.tensor(ch.formation_energies(), device=dev)
    status = torch.zeros(cells, dtype=torch.int32, device=dev)
    T_out = torch.zeros(cells, dtype=torch.float64, device=dev)
    g = ch.graph(rho, e, dt, T_out=T_out, status=status) if use_graph else None
    m0 = rho.sum().item()
    U0 = (e.sum() + (ef[:, None] * rho).sum()).item()
    c = u * dt / dx
    hist = []

    def troll(a, shift, axis):
        return torch.roll(a, shift, dims=axis if a.dim() > 1 else 0)

    for n in range(steps):
        # convection half: upwind, conservative, periodic
        advect(rho, e, c, troll)
        # chemistry half
        if g is not None:
            g.launch()
        else:
            ch.advance(rho, e, dt, T_out=T_out, status=status)
        torch.cuda.synchronize()
        hist.append({"step": n + 1, "T_max": float(T_out.max()), "T_min": float(T_out.min()),
                     "failed_cells": int((status != 0).sum()), "mass": float(rho.sum()),
                     "U": float(e.sum() + (ef[:, None] * rho).sum())})
    if g is not None:
        g.close()
    ch.close()
    scale = float(e.abs().sum() + (ef.abs()[:, None] * rho.abs()).sum())
    return {"cells": cells, "steps": steps, "dt": dt, "c": c, "mass_drift": abs(hist[-1]["mass"] - m0) / m0,
            "energy_drift": abs(hist[-1]["U"] - U0) / scale, "history": hist,
            "rho0": rho0.cpu().numpy(), "e0": e0.cpu().numpy(), "rho": rho.cpu().numpy(),
            "e": e.cpu().numpy(), "T": T_out.cpu().numpy()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=20)
    args = ap.parse_args()
    out = run(args.cells, args.steps)
    print(json.dumps({k: v for k, v in out.items() if k in ("cells", "steps", "dt", "mass_drift", "energy_drift")}))
    for h in out["history"]:
        print(json.dumps(h))


if __name__ == "__main__":
    main()
