"""Benchmark of the batched implicit chemistry step (one JSON line on stdout).

A step is one chemistry advance (all cells, dt = 1e-6 s) of the 36-species /
308-reaction workload on 2^18 cells, inputs resident in HBM; the state is
restored from a pristine device copy before every step and L2 is flushed
(256 MiB write) before every step.  `value` is whole-job cell-updates/s;
`e2e` is the same through chem_advance_host with pinned host buffers (copies
inside the timed region).  `--impl reference` times the CPU oracle instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "chemistry cell-updates/s at 36 sp/308 rxn (mixed vs FP64) + p50/p99 request latency"
WORKLOAD = "hc36-256k"
WORKLOAD_DESC = ("synthetic 36 sp / 308 rxn mechanism (4 elements, 40 third-body, 12 pressure-"
                 "independent unimolecular), 2^18 constant-volume cells, T U[900, 2800] K, 1 atm, "
                 "Dirichlet(1) mass fractions, one dt = 1e-6 s backward-Euler chemistry step with "
                 "adaptive substeps")
# DRAM bytes (read + write) of one launch of the step kernel on the default
# workload (2^18 cells, state and tables cold after the L2 flush), from a
# single-pass ncu capture of a full-size launch of the current kernels
# (dram__bytes_read.sum + dram__bytes_write.sum; part of the state written
# back is still in L2 when the kernel ends).  Other workloads report null.
MEASURED_TRAFFIC = {"mixed": 80.06e6 + 29.98e6, "fp64": 80.23e6 + 34.77e6}
# FP64-pipe utilisation of the step kernels from ncu
# (sm__pipe_fp64_cycles_active, share of active cycles), captured on the
# first 16,384 cells of the default workload (a full launch is too long for
# a multi-pass capture).
MEASURED_FP64_PIPE = {"mixed": 0.597, "fp64": 0.805}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk x 2 x max clock
FP64_PEAK_PROBE_TFLOPS = 1.193                    # DFMA timing probe on this GPU model
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FFMA/clk x 2 x max clock


def work_model(mech):
    """Algorithmic work of one Newton iteration of one cell, exponentials
    counted apart from the flops (FMA = 2 flop).

    fp64_path: the per-iteration count of the method as written -- thermo
    25 N_s, rates 20 R + 2 N_s R_tb, Jacobian 84 R + 12 N_s R_tb + 5 n^2 +
    2 n N_s, Gaussian elimination on the n = N_s + 1 unknowns of Eq. 29
    2 n^3/3 + 2 n^2, residual 3 n -- plus 2 R exponentials (K_f and K_e).

    mixed_fp64 / mixed_fp32: the mixed-precision path's split, counted from
    the mechanism's structure: what it keeps in FP64 (NASA-7 h, s, g and
    energies, two temperature-recovery iterations' energy sums, rate
    constants and progress rates, species sources, residual, update and
    convergence norm) and what it moves to FP32 (heat capacities and the
    recovery's derivative, the Jacobian's rate factors, D entries and
    gather, the elimination).

    The kernels do less for the same result: K_b comes from per-species
    exponentials (one exp per reaction plus one per species, `exp_kernel`),
    and the energy unknown is eliminated through total-energy conservation
    (N_s unknowns)."""
    ns, nr = mech.ns, mech.nr
    n = ns + 1
    ntb = int(np.asarray(mech.third_body).astype(bool).sum())
    nu = np.zeros((nr, ns), np.int64)
    for r in range(nr):
        for j in range(3):
            if mech.reac_sp[r, j] >= 0:
                nu[r, mech.reac_sp[r, j]] -= mech.reac_nu[r, j]
            if mech.prod_sp[r, j] >= 0:
                nu[r, mech.prod_sp[r, j]] += mech.prod_nu[r, j]
    nD = j_ent = sp_ent = 0
    for r in range(nr):
        cols = {int(s) for s in mech.reac_sp[r] if s >= 0} | {int(s) for s in mech.prod_sp[r] if s >= 0}
        if mech.third_body[r]:
            cols |= {s for s in range(ns) if mech.tb_eff[r, s] != 1.0}
        rows = int((nu[r] != 0).sum())
        nD += len(cols)
        j_ent += len(cols) * rows
        sp_ent += rows
    fp64_path = (25 * ns + (20 * nr + 2 * ns * ntb) + (84 * nr + 12 * ns * ntb + 5 * n * n + 2 * n * ns) +
                 (2 * n ** 3 // 3 + 2 * n * n) + 3 * n)
    thermo, thermo_cp = 28 * ns, 10 * ns          # h, s, g, e | c_p, rho c_v
    trec_e, trec_cv = 2 * 14 * ns, 2 * 13 * ns    # two recovery iterations: e(T) | c_v(T)
    rates_src = 30 * nr                          # rate constants, progress rates (exp apart)
    rates_jac = 10 * nr                          # C_M K_f, C_M K_b, dQ/dT
    d_entries = 8 * nD
    gather_src = 2 * sp_ent + 2 * ns
    gather_jac = 4 * sp_ent + 4 * ns
    jac = 6 * ns * n + 2 * j_ent + 2 * nD + 6 * n
    lu = sum(2 * (n - j - 1) * (n - j) + (n - j - 1) + 1 for j in range(n)) + n * n
    update, update_norm = 6 * n, 3 * n
    mixed_fp64 = thermo + trec_e + rates_src + gather_src + update + update_norm
    mixed_fp32 = thermo_cp + trec_cv + rates_jac + d_entries + gather_jac + jac + lu
    return dict(fp64_path=fp64_path, mixed_fp64=mixed_fp64, mixed_fp32=mixed_fp32,
                exp_method=2 * nr, exp_kernel=nr + ns, nD=nD, j_ent=j_ent, ntb=ntb)


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.p = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="chem_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()
        self._rows = self._read()
        if self.path:
            try:
                os.unlink(self.path)
            except OSError:
                pass

    def _read(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        return rows

    def summary(self):
        if self.p is None:
            return None
        rows = getattr(self, "_rows", [])
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_init(args):
    from paper_1110_4903_gb300 import replicas
    return replicas.init()


def barrier_max(world, value, device):
    from paper_1110_4903_gb300 import replicas
    return replicas.max_over_ranks(value, device) if world > 1 else value


def cpu_baseline(sample_cells=4096, threads=None, single=True):
    """The oracle on the host cores over a bounded, stratified sample of the
    workload (every 64th cell)."""
    import oracle
    from paper_1110_4903_gb300 import synth
    mech, f, dt = synth.workload(WORKLOAD)
    idx = np.arange(0, f.n, max(1, f.n // sample_cells))[:sample_cells]
    fs = synth.subsample(f, idx)
    om = oracle.OracleMech(mech)
    rho, e = om.state_from_tpy(fs.T, fs.P, fs.Y)
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    _, _, out = om.advance_batch(rho, e, dt, T_in=fs.T, threads=threads)
    el = time.perf_counter() - t0
    res = dict(value=len(idx) / el, unit="cell-updates/s", cores=threads, kind="oracle",
               sample="%d cells (every %dth of the 2^18-cell workload), one dt step each, %.1f s wall"
                      % (len(idx), f.n // sample_cells, el),
               newton_iters_mean=float(out["newton_iters"].mean()))
    if single:
        # one host thread, the comparison point of the paper's single-core runs
        n1 = max(1, sample_cells // 16)
        t0 = time.perf_counter()
        om.advance_batch(rho[:, :n1], e[:n1], dt, T_in=fs.T[:n1], threads=1)
        el1 = time.perf_counter() - t0
        res["single_thread"] = dict(value=n1 / el1, unit="cell-updates/s", cores=1,
                                    sample="first %d of those cells, %.1f s wall" % (n1, el1))
    return res


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    steps = []
    cb = None
    for i in range(args.warmup + args.steps):
        res = cpu_baseline(sample_cells=args.ref_cells, single=False)
        if i >= args.warmup:
            steps.append(res)
        cb = res
    value = statistics.mean(s["value"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * args.ref_cells / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample_cells": args.ref_cells},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"],
                             "value": value, "unit": "cell-updates/s"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_path(torch, ch, rho0, e0, T_in, dt, precision, steps, warmup, flush, stream, want_stats,
              graph=False):
    """Times `steps` advances (after `warmup`) on `stream`; returns per-step
    kernel-only and whole-step times (ms) and per-cell counters.  With
    graph=True each step is a launch of a captured graph of the step."""
    n = e0.shape[0]
    rho = torch.empty_like(rho0)
    e = torch.empty_like(e0)
    st = torch.empty(n, dtype=torch.int32, device=e0.device)
    it = torch.empty(n, dtype=torch.int32, device=e0.device)
    g = None
    if graph:
        g = ch.graph(rho, e, dt, T_in=T_in, status=st, newton_iters=it, precision=precision)
    step_ms, kern_ms = [], []
    with torch.cuda.stream(stream):
        for i in range(warmup + steps):
            flush.fill_(float(i))                      # evict L2 (256 MiB write)
            a = torch.cuda.Event(enable_timing=True)
            k0 = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rho.copy_(rho0)
            e.copy_(e0)
            k0.record(stream)
            if g is not None:
                g.launch(stream)
            else:
                ch.advance(rho, e, dt, T_in=T_in, status=st, newton_iters=it, precision=precision,
                           stream=stream)
            b.record(stream)
            if i >= warmup:
                step_ms.append((a, k0, b))
        stream.synchronize()
    if g is not None:
        g.close()
    tot = [a.elapsed_time(b) for a, k0, b in step_ms]
    ker = [k0.elapsed_time(b) for a, k0, b in step_ms]
    stats = None
    if want_stats:
        stats = dict(status_ok=float((st == 0).float().mean().item()),
                     newton_iters=int(it.sum().item()),
                     newton_iters_mean=float(it.float().mean().item()),
                     newton_iters_max=int(it.max().item()),
                     newton_iters_hist=torch.bincount(it.clamp(0, 64).long(), minlength=65).tolist())
    return tot, ker, stats


SERVE_STALL_S = 120.0   # a serving run that completes nothing for this long is an error


def _stalled(t_last_done):
    if time.perf_counter() - t_last_done > SERVE_STALL_S:
        raise RuntimeError("request server made no progress for %.0f s" % SERVE_STALL_S)


def _wait_done(srv, ticket):
    res = srv.wait(ticket, timeout_us=int(SERVE_STALL_S * 1e6))
    if res is None:
        raise RuntimeError("request %d did not finish within %.0f s" % (ticket, SERVE_STALL_S))
    return res


def serving_run(torch, chem, synth, device, n_requests, rate_frac=0.7, budget_bytes=0, seed=5,
                n_sims=128, max_inflight=64):
    """Poisson stream of chemistry requests from many simulations (9 or 36
    species with probability 1/2, 1k-256k cells log-uniform, dt log-uniform
    1e-8..1e-5 s) against a request server; states are resident on the
    device.  The rate is rate_frac x the capacity measured by a saturating
    burst first.  Returns throughput and latency percentiles."""
    rng = np.random.default_rng(seed)
    mechs = [synth.h2_air_9sp(), synth.hydrocarbon_36sp()]
    handles = [chem.Chem(m, precision=chem.MIXED) for m in mechs]
    sims = []
    for i in range(n_sims):
        k = i % 2
        n = int(np.exp(rng.uniform(np.log(1024), np.log(262144))))
        f = synth.uniform_field(mechs[k].ns, n, 900.0, 2800.0, seed=10_000 + i)
        T = torch.tensor(f.T, device=device)
        rho = torch.empty((mechs[k].ns, n), dtype=torch.float64, device=device)
        e = torch.empty(n, dtype=torch.float64, device=device)
        handles[k].state_from_tpy(T, torch.tensor(f.P, device=device),
                                  torch.tensor(f.Y, device=device), rho, e)
        sims.append((k, n, rho, e))
    torch.cuda.synchronize()
    srv = chem.Server(budget_bytes=budget_bytes, max_inflight=max_inflight)
    busy = {}

    def pick(k, draw):
        cands = [i for i in range(n_sims) if sims[i][0] == k and i not in busy]
        return cands[int(draw * len(cands)) % len(cands)] if cands else None

    progress = [time.perf_counter()]

    def retire():
        for i, t in list(busy.items()):
            r = srv.poll(t)
            if r.state in (chem.REQ_DONE, chem.REQ_FAILED, chem.REQ_CANCELLED):
                done.append((t, r, sims[i][1]))
                del busy[i]
                progress[0] = time.perf_counter()
        if busy:
            _stalled(progress[0])

    # capacity: a saturating burst
    done = []
    t0 = time.perf_counter()
    burst = 64
    for j in range(burst):
        k = j % 2
        i = pick(k, rng.uniform())
        busy[i] = srv.submit(handles[k], sims[i][2], sims[i][3],
                             float(np.exp(rng.uniform(np.log(1e-8), np.log(1e-5)))))
    while busy:
        retire()
        time.sleep(0.0005)
    cap_rps = burst / (time.perf_counter() - t0)
    rate = rate_frac * cap_rps
    # the stream
    reqs = synth.poisson_requests(n_requests, rate, seed=seed)
    done = []
    arrivals = {}
    cells = 0
    t_start = time.perf_counter()
    srv_t0 = None
    for q in reqs:
        while time.perf_counter() - t_start < q["t"]:
            retire()
            time.sleep(0.0002)
        i = pick(q["mech"], rng.uniform())
        while i is None:          # every simulation of this mechanism is in flight
            retire()
            time.sleep(0.0002)
            i = pick(q["mech"], rng.uniform())
        t = srv.submit(handles[q["mech"]], sims[i][2], sims[i][3], q["dt"])
        busy[i] = t
        arrivals[t] = time.perf_counter() - (t_start + q["t"])   # client-side delay
        cells += sims[i][1]
    while busy:
        retire()
        time.sleep(0.0002)
    wall = time.perf_counter() - t_start
    # latency from the scheduled arrival (server clock offset from the submit stamp)
    lat, wait = [], []
    for t, r, n in done:
        if t in arrivals:
            lat.append(r.t_done - r.t_submit + max(0.0, arrivals[t]))
            wait.append(r.t_start - r.t_submit)
    lat, wait = np.array(lat), np.array(wait)
    st = srv.stats()
    srv.close()
    for h in handles:
        h.close()
    return {"requests": len(lat), "rate_rps": rate, "capacity_rps": cap_rps, "rate_frac": rate_frac,
            "cell_updates_per_s": cells / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "admission_wait_p99_ms": float(np.percentile(wait, 99) * 1e3),
            "requests_waiting_over_1ms": int((wait > 1e-3).sum()),
            "budget_bytes": st["budget_bytes"], "max_inflight": max_inflight,
            "kernel_instances_launched": st["launches"], "failed": st["failed"]}


def serving_background(torch, chem, synth, device, n_small=48, seed=7):
    """Small requests arriving while a large one runs: one 2^18-cell request
    of the 36-species mechanism, then n_small requests (1k-16k cells, 9 or
    36 species alternately, dt 1e-6 s) at Poisson times spread over the large
    request's own duration.  Reports the small requests' latency (submit to
    done, host clock) and device span (first claim to last cell, device
    clock), and the large request's span alone and in the mix."""
    rng = np.random.default_rng(seed)
    mechs = {9: synth.h2_air_9sp(), 36: synth.hydrocarbon_36sp()}
    hs = {k: chem.Chem(m, precision=chem.MIXED) for k, m in mechs.items()}

    def state(k, n, sd):
        f = synth.uniform_field(mechs[k].ns, n, 900.0, 2800.0, seed=sd)
        rho = torch.empty((mechs[k].ns, n), dtype=torch.float64, device=device)
        e = torch.empty(n, dtype=torch.float64, device=device)
        hs[k].state_from_tpy(torch.tensor(f.T, device=device), torch.tensor(f.P, device=device),
                             torch.tensor(f.Y, device=device), rho, e)
        return rho, e

    big = state(36, 1 << 18, 20_000)
    smalls = [(k, state(k, int(np.exp(rng.uniform(np.log(1024), np.log(16384)))), 20_001 + i))
              for i, k in enumerate([9, 36] * (n_small // 2))]
    torch.cuda.synchronize()
    srv = chem.Server()
    r, e = big[0].clone(), big[1].clone()
    res = _wait_done(srv, srv.submit(hs[36], r, e, 1e-6))
    span_alone = (res.dev_last_ns - res.dev_first_ns) * 1e-9
    gaps = rng.exponential(0.8 * span_alone / n_small, n_small)
    r, e = big[0].clone(), big[1].clone()
    tb = srv.submit(hs[36], r, e, 1e-6)
    t0 = time.perf_counter()
    tickets = []
    for (k, (rs, es)), at in zip(smalls, np.cumsum(gaps)):
        while time.perf_counter() - t0 < at:
            time.sleep(0.0002)
        tickets.append(srv.submit(hs[k], rs, es, 1e-6))
    rb = _wait_done(srv, tb)
    lat, span, before = [], [], 0
    for t in tickets:
        q = _wait_done(srv, t)
        lat.append(q.t_done - q.t_submit)
        span.append((q.dev_last_ns - q.dev_first_ns) * 1e-9)
        before += q.dev_last_ns < rb.dev_last_ns
    st = srv.stats()
    srv.close()
    for h in hs.values():
        h.close()
    lat, span = np.array(lat), np.array(span)
    return {"large_cells": 1 << 18, "small_requests": n_small,
            "small_p50_ms": float(np.percentile(lat, 50) * 1e3),
            "small_p99_ms": float(np.percentile(lat, 99) * 1e3),
            "small_device_span_p50_ms": float(np.percentile(span, 50) * 1e3),
            "small_device_span_p99_ms": float(np.percentile(span, 99) * 1e3),
            "small_finished_before_large": int(before),
            "large_span_alone_ms": span_alone * 1e3,
            "large_span_in_mix_ms": (rb.dev_last_ns - rb.dev_first_ns) * 1e-6,
            "kernel_instances_launched": st["launches"], "failed": st["failed"]}


def serving_sweep(args):
    """The request stream at several loads (fractions of the measured
    capacity, overload included) and HBM budgets (one small enough to force
    queueing); one JSON line with a record per run."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem, synth
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    runs = []
    for frac in (0.5, 0.8, 1.0, 1.3):
        runs.append(serving_run(torch, chem, synth, device, args.serving_requests, frac, 0))
    # the largest request (2^18 cells, 36 species) holds about 81 MB: at 90
    # MiB no two large requests are in flight together, so admission waits
    for budget in (256 << 20, 90 << 20):
        runs.append(serving_run(torch, chem, synth, device, args.serving_requests, 0.7, budget))
    bg = serving_background(torch, chem, synth, device)
    print(json.dumps({"metric": "request latency of the chemistry server (Poisson arrivals)",
                      "unit": "ms", "requests_per_run": args.serving_requests, "runs": runs,
                      "small_requests_during_a_large_one": bg}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-cells", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: time FP64 and mixed, headline = mixed")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per cell (0: the library's choice)")
    ap.add_argument("--workload", default=WORKLOAD, help="named workload of synth.workload")
    ap.add_argument("--graph", action="store_true", help="time captured-graph steps")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch shape first")
    ap.add_argument("--cells", type=int, default=0,
                    help="time the first CELLS cells only (a smaller case for profiling)")
    ap.add_argument("--serving-requests", type=int, default=120,
                    help="requests in the serving stream (0: skip the serving run)")
    ap.add_argument("--serving-rate", type=float, default=0.7, help="load as a fraction of capacity")
    ap.add_argument("--serving-budget", type=int, default=0, help="server HBM budget in bytes")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="only the request server: loads 0.5-1.2 of capacity and two HBM budgets")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.serving_sweep:
        if rank == 0:
            serving_sweep(args)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem, synth

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    mech, f, dt = synth.workload(args.workload)
    if args.cells:
        f = synth.subsample(f, np.arange(min(args.cells, f.n)))
    wm = work_model(mech)
    stream = torch.cuda.Stream(device)
    handles = {}
    for name, prec in (("fp64", chem.FP64), ("mixed", chem.MIXED)):
        if args.precision in ("both", name):
            handles[name] = chem.Chem(mech, lanes_per_cell=args.lanes, precision=prec)
    head_name = "mixed" if "mixed" in handles else "fp64"
    head = handles[head_name]
    with torch.cuda.stream(stream):
        T = torch.tensor(f.T, device=device)
        Pp = torch.tensor(f.P, device=device)
        Y = torch.tensor(f.Y, device=device)
        rho0 = torch.empty_like(Y)
        e0 = torch.empty_like(T)
        head.state_from_tpy(T, Pp, Y, rho0, e0, stream=stream)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    stream.synchronize()
    n = f.n

    results = {}
    clk = None
    gpu_launches = 0
    wall = 0.0
    for name, ch in handles.items():
        prec = chem.MIXED if name == "mixed" else chem.FP64
        shape = None
        if args.autotune:
            shape = ch.autotune(rho0, e0, dt, T_in=T, precision=prec, stream=stream)
        # untimed statistics launch: Newton iterations for the work model
        _, _, stats = time_path(torch, ch, rho0, e0, T, dt, prec, 1, 0, flush, stream, True)
        launches0 = ch.launch_count()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as ck:
            t0 = time.perf_counter()
            tot, ker, _ = time_path(torch, ch, rho0, e0, T, dt, prec, args.steps, args.warmup, flush,
                                    stream, False, graph=args.graph)
            torch.cuda.synchronize()
            w = time.perf_counter() - t0
        launches = (ch.launch_count() - launches0) * args.steps // (args.steps + args.warmup)
        step_ms = barrier_max(world, statistics.mean(tot), device)
        kern_ms = barrier_max(world, statistics.mean(ker), device)
        it = stats["newton_iters"]
        ksec = kern_ms * 1e-3
        flop64 = wm["fp64_path"] if name == "fp64" else wm["mixed_fp64"]
        a64 = it * flop64 / ksec / 1e12
        bytes_launch = n * (16 * (mech.ns + 1) + 8)
        full_default = args.workload == WORKLOAD and not args.cells
        roof = {"bound": "alu", "achieved": a64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": a64 / FP64_PEAK_TFLOPS,
                "traffic": MEASURED_TRAFFIC[name] if full_default else None,
                "traffic_unit": "bytes per launch (DRAM read + write)",
                "kernel": "chem::be_kernel<%d,%s>" % (ch.lanes(prec), "double" if name == "fp64" else "float"),
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe, the binding "
                               "pipe; MEASURED_PEAKS.json has no FP64 figure); a DFMA timing probe "
                               "measured %.3f TFLOP/s" % FP64_PEAK_PROBE_TFLOPS,
                "work_model": ("%d FP64 flop per Newton iteration, %s, exponentials apart; %d Newton "
                               "iterations per launch" % (
                                   flop64, "the method's count (thermo, rates, Jacobian, elimination on "
                                   "N_s+1 unknowns, residual)" if name == "fp64" else
                                   "the part the mixed path keeps in FP64", it)),
                "exp": {"method_per_iter": wm["exp_method"], "kernel_per_iter": wm["exp_kernel"],
                        "method_rate_G_per_s": it * wm["exp_method"] / ksec / 1e9,
                        "evaluated_rate_G_per_s": it * wm["exp_kernel"] / ksec / 1e9},
                "ncu_fp64_pipe_busy": MEASURED_FP64_PIPE[name] if full_default else None,
                "hbm_gbs": bytes_launch / ksec / 1e9}
        if name == "mixed":
            a32 = it * wm["mixed_fp32"] / ksec / 1e12
            roof["fp32"] = {"achieved": a32, "peak": FP32_PEAK_TFLOPS, "frac": a32 / FP32_PEAK_TFLOPS,
                            "unit": "TFLOP/s",
                            "work_model": "%d FP32 flop per Newton iteration (Jacobian, elimination, "
                                          "heat capacities)" % wm["mixed_fp32"],
                            "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz"}
        results[name] = dict(value=world * n / (step_ms * 1e-3), ms_per_step=step_ms,
                             kernel_ms_per_step=kern_ms, lanes_per_cell=ch.lanes(prec),
                             newton_iters_mean=stats["newton_iters_mean"],
                             newton_iters_max=stats["newton_iters_max"],
                             cells_ok=stats["status_ok"], roofline=roof)
        if shape is not None:
            results[name]["autotuned_warps_per_block"] = shape[1]
        if args.workload != WORKLOAD:
            # Newton iterations per cell: histogram over 0..63, 64 = 64 or more
            results[name]["newton_iters_hist"] = stats["newton_iters_hist"]
        if ch is head:
            clk = ck.summary()
            gpu_launches = launches
            wall = w

    e2e = None
    if not args.no_e2e:
        rho_h = torch.empty((mech.ns, n), dtype=torch.float64, pin_memory=True).numpy()
        e_h = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        rho_src = rho0.cpu().numpy()
        e_src = e0.cpu().numpy()
        times = []
        for i in range(1 + 2):
            rho_h[...] = rho_src
            e_h[...] = e_src
            t1 = time.perf_counter()
            head.advance_host(rho_h, e_h, dt)
            t2 = time.perf_counter()
            if i >= 1:
                times.append(t2 - t1)
        e2e_s = barrier_max(world, statistics.mean(times), device)
        e2e = {"value": world * n / e2e_s, "unit": "cell-updates/s",
               "h2d_bytes_per_step": int(n * (mech.ns + 1) * 8),
               "d2h_bytes_per_step": int(n * (mech.ns + 1) * 8),
               "api": "chem_advance_host (pinned host buffers, synchronous), %s" % head_name,
               "steps": len(times)}

    serving = None
    if args.serving_requests > 0 and not args.cells:
        serving = serving_run(torch, chem, synth, device, args.serving_requests, args.serving_rate,
                              args.serving_budget)
        serving["small_requests_during_a_large_one"] = serving_background(torch, chem, synth, device)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        cb.pop("newton_iters_mean", None)

    if rank == 0:
        hr = results[head_name]
        line = {"metric": METRIC, "value": hr["value"], "unit": "cell-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": hr["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if head_name == "fp64" else "f32+f64", "data": "synthetic",
                "config": {"workload": (WORKLOAD_DESC if args.workload == WORKLOAD else args.workload)
                           if not args.cells else "first %d cells of: %s" % (n, args.workload),
                           "cells": n, "precision": head_name,
                           "lanes_per_cell": hr["lanes_per_cell"],
                           "l2": "flushed (256 MiB write) before every step; state restored from "
                                 "a device copy inside the step",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "graph": bool(args.graph), "autotuned": bool(args.autotune)},
                "kernel_ms_per_step": hr["kernel_ms_per_step"], "wall_s": wall,
                "newton_iters_mean": hr["newton_iters_mean"],
                "newton_iters_max": hr["newton_iters_max"], "cells_ok": hr["cells_ok"],
                "roofline": hr["roofline"], "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clk, "serving": serving}
        for name, r in results.items():
            line[name] = {k: v for k, v in r.items()}
        if "fp64" in results and "mixed" in results:
            line["mixed_over_fp64"] = results["mixed"]["value"] / results["fp64"]["value"]
        print(json.dumps(line), flush=True)
    for ch in handles.values():
        ch.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
