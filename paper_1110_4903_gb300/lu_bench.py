"""Batched dense solves on the GPU: the kinetics-only experiment of Sec. 5.2
(Gaussian elimination over many independent N_s x N_s systems).  The
global-memory kernels (matrices in HBM; a thread per system, or a block of
warps per 32 systems when there are few), in the scalar rounding order and
contracted (FMA), against the on-chip kernel (one warp per system, matrix in
shared memory).  One JSON line per case, with the fraction of the measured
HBM bandwidth (by the paper's byte count of the elimination) and of the FP64
pipe (by the operation count, divisions as one).

  python -m paper_1110_4903_gb300.lu_bench [--sizes 10,37,100,200] [--bytes 2e9]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HBM_PEAK_GBS = 6677.8          # measured copy bandwidth of this GB300 pool
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 pipe: two lane-operations per clock per SM (a warp instruction every
# 16 cycles), whatever the instruction (FMA, multiply or add)
FP64_PIPE_TOPS = 152 * 2 * 2.07e9 / 1e12


def flops(n):
    """FP64 operations of one factorisation and one solve (divide = 1).
    Without FMA contraction each is one FP64 pipe instruction, except the
    divisions (n (n + 1) / 2 of them), which take several."""
    lu = sum((n - j - 1) + 2 * (n - j - 1) * (n - j - 1) for j in range(n))
    return lu + 2 * n * n


def global_bytes(n):
    """HBM bytes of the global-memory elimination of one system: pivot
    search reads the column, each step reads and writes the trailing block
    and reads the pivot row; then the matrix is read for the substitutions
    (b: read and written per step as well)."""
    b = 0
    for j in range(n):
        m = n - j - 1
        b += (n - j) * 8                 # pivot column
        b += (m * (m + 1) + (m + 1)) * 8  # trailing block + multipliers read
        b += (m * (m + 1)) * 8           # trailing block written
        b += 2 * 8                       # right-hand side
    b += n * n * 8 + 4 * n * 8           # substitutions
    return b


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10,25,37,50,100,150,200")
    ap.add_argument("--bytes", default="5e8,4e9", help="matrix bytes per case (comma list)")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    dev = torch.device("cuda")
    for n, nbytes in [(int(s), float(b)) for s in args.sizes.split(",") for b in args.bytes.split(",")]:
        n_sys = int(min(nbytes / (8 * n * n), 1 << 22))
        rng = np.random.default_rng(n)
        base = torch.tensor(rng.standard_normal((n, n)), device=dev)
        for method, name in ((chem.LU_GLOBAL, "global"), (chem.LU_GLOBAL_FMA, "global_fma"),
                             (chem.LU_ONCHIP, "onchip")):
            glob = method in (chem.LU_GLOBAL, chem.LU_GLOBAL_FMA)
            if method == chem.LU_ONCHIP and n * (n + 1) * 8 > 227 * 1024:
                continue
            # diagonally shifted random systems, built on the device
            if glob:
                A0 = (torch.randn((n, n, n_sys), dtype=torch.float64, device=dev) +
                      0.5 * n ** 0.5 * torch.eye(n, dtype=torch.float64, device=dev)[:, :, None])
                b0 = torch.randn((n, n_sys), dtype=torch.float64, device=dev)
            else:
                A0 = (torch.randn((n_sys, n, n), dtype=torch.float64, device=dev) +
                      0.5 * n ** 0.5 * torch.eye(n, dtype=torch.float64, device=dev)[None])
                b0 = torch.randn((n_sys, n), dtype=torch.float64, device=dev)
            A = torch.empty_like(A0)
            b = torch.empty_like(b0)
            info = torch.zeros(n_sys, dtype=torch.int32, device=dev)
            times = []
            for rep in range(1 + args.reps):
                A.copy_(A0)
                b.copy_(b0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                chem.batched_solve(method, A, b, None, info)
                e1.record()
                torch.cuda.synchronize()
                if rep:
                    times.append(e0.elapsed_time(e1) * 1e-3)
            t = min(times)
            fl = flops(n) * n_sys
            by = (global_bytes(n) if glob else 2 * 8 * (n * n + n)) * n_sys
            line = {"case": "batched_solve", "method": name, "n": n, "systems": n_sys,
                    "seconds": t, "systems_per_s": n_sys / t, "gflops": fl / t / 1e9,
                    "hbm_gbs": by / t / 1e9, "hbm_frac": by / t / 1e9 / HBM_PEAK_GBS,
                    "fp64_pipe_frac": fl / t / 1e12 / FP64_PIPE_TOPS,
                    "roofline": ({"bound": "hbm", "achieved": by / t / 1e9, "peak": HBM_PEAK_GBS,
                                  "unit": "GB/s", "frac": by / t / 1e9 / HBM_PEAK_GBS}
                                 if glob else
                                 {"bound": "alu", "achieved": fl / t / 1e12, "peak": FP64_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": fl / t / 1e12 / FP64_PEAK_TFLOPS}),
                    "singular": int((info != 0).sum().item())}
            print(json.dumps(line), flush=True)
            del A0, b0, A, b


if __name__ == "__main__":
    main()
