"""Domain segmentation overhead (Sec. 5.2): one chemistry step of a
128 x 128 field issued as 1, 2, 4, ... launches over segments of the grid
(chem_advance_segmented), timed with CUDA events.  One JSON line per case.

  python -m paper_1110_4903_gb300.segment_bench [--segments 1,2,4,8,16,32]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--segments", default="1,2,4,8,16,32")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem, synth
    mech = synth.hydrocarbon_36sp()
    f = synth.front_field(mech, nx=args.nx, ny=args.ny, band=8)
    n = f.n
    dev = torch.device("cuda")
    ch = chem.Chem(mech, precision=chem.MIXED)
    rho0 = torch.empty((mech.ns, n), dtype=torch.float64, device=dev)
    e0 = torch.empty(n, dtype=torch.float64, device=dev)
    ch.state_from_tpy(torch.tensor(f.T, device=dev), torch.tensor(f.P, device=dev),
                      torch.tensor(f.Y, device=dev), rho0, e0)
    base = None
    for nseg in [int(s) for s in args.segments.split(",")]:
        seg = -(-n // nseg)
        times = []
        for rep in range(1 + args.reps):
            rho, e = rho0.clone(), e0.clone()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ch.advance_segmented(rho, e, 1e-6, seg if nseg > 1 else 0)
            b.record()
            torch.cuda.synchronize()
            if rep:
                times.append(a.elapsed_time(b))
        t = min(times)
        base = base or t
        print(json.dumps({"case": "segmented", "cells": n, "segments": nseg, "cells_per_segment": seg,
                          "ms": t, "relative": t / base}), flush=True)
    ch.close()


if __name__ == "__main__":
    main()
