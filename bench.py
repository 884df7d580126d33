"""Benchmark: N-1 scenarios/s of the batched GB300 screen on the 10,000-bus
synthetic grid (every single-branch outage; mismatch <= 1e-4 p.u.).

One step = one gpcg_n1_screen over all outages of the grid, with the grid,
base case and outage list resident on the device.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpcg|reference]

Under torchrun every rank screens the full outage list of its own copy of
the grid (weak scaling: no data-path collective), rank 0 reports.  The
reference arm (--impl reference) times the CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N-1 scenarios/sec at 10k buses (mismatch≤1e-4 p.u.), batched vs plain; HBM GB/s %"
WORKLOAD = "grid10k"


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def algorithmic_bytes(info, iters, w, n_bus, n_branch):
    """Bytes the method must move per screen (per-unit figures: 15 w n per
    inner PCG iteration, 32 n per outer half-iteration's FP64 mismatch,
    16 n + 8 m for the flows, plus the shared matrix and factor bytes per
    iteration amortised over the scenarios)."""
    outer = iters[:, 0].astype(np.float64)
    inP = iters[:, 1].astype(np.float64)
    inQ = iters[:, 2].astype(np.float64)
    S = iters.shape[0]
    vec = 15.0 * w * (inP.sum() * info["n_p"] + inQ.sum() * info["n_q"])
    mis = 32.0 * n_bus * (2.0 * outer + 1.0).sum()
    flows = S * (16.0 * n_bus + 8.0 * n_branch)
    mats = (inP.sum() * (info["nnz_p"] + 2 * info["nnz_lp"]) +
            inQ.sum() * (info["nnz_q"] + 2 * info["nnz_lq"])) * (w + 4) / max(S, 1)
    return vec + mis + flows + mats


def island_split(g, iters):
    """Mean iterations of the outages that island buses (the bridges) and of
    the rest, outage k being branch k: the islanding scenarios' extra inner
    iterations are reported, not asserted."""
    from paper_1803_03290_gb300 import binding
    br = binding.analyze(g)["bridge"][:iters.shape[0]].astype(bool)
    out = {"outages": int(br.sum())}
    for key, sel in (("islanding", br), ("other", ~br)):
        if sel.any():
            out[key] = {"mean_outer": round(float(iters[sel, 0].mean()), 3),
                        "mean_inner_P": round(float(iters[sel, 1].mean()), 3),
                        "mean_inner_Q": round(float(iters[sel, 2].mean()), 3)}
    return out


def fp64_operations(g, iters):
    """FP64 operations (an FMA counts once) the screen's FP64 parts take per
    launch, from the kernel's arithmetic: per full P mismatch 4 per adjacency
    entry and 7 per non-slack bus (+2 per PQ bus for dQ), per Q mismatch 4
    per adjacency entry and 6 per PQ bus, per angle update 12 per non-slack
    bus (the exact rotation of e + jf), per |V| update 2 per PQ bus (e and f
    scaled), the first P mismatch 1 per non-slack bus (the base case's is
    stored), and 16 per branch for the flows and loading; k outer iterations
    take k full P mismatches, k Q mismatches and k updates of each kind."""
    bt = np.asarray(g.bus_type)
    deg = np.bincount(np.r_[g.f, g.t], minlength=g.n_bus)
    nP, nQ = int((bt != 2).sum()), int((bt == 0).sum())
    AP, AQ = int(deg[bt != 2].sum()), int(deg[bt == 0].sum())
    per_outer = (4 * AP + 7 * nP + 2 * nQ) + (4 * AQ + 6 * nQ) + 12 * nP + 2 * nQ
    k = iters[:, 0].astype(np.float64)
    return float((k * per_outer).sum() + iters.shape[0] * (nP + 16 * g.n_branch))


FP64_PEAK_GOPS = 625.0  # nominal 1.25 TFLOP/s of GB300 with an FMA as 2 FLOP


# DRAM bytes per launch of the N-1 kernel on the default grid10k workload
# (dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture of the
# timed screens, taken by hand and recorded here), valid only for the kernel
# sources with this digest and the launch shape it was taken with; the bench
# line labels it as such.
KERNEL_TRAFFIC = {"sha256": "5c65860d6f4d99dd6095f335cd505f3268e05e415e21923246480d59bb078b1b", "bytes": 178.25e9,
                  "knobs": {"tile": 2, "ctas_per_sm": 5, "tail_rows": [241, 236]}}
KERNEL_SOURCES = ("fdpf.cu", "fdpf_kernel.cuh", "fdpf_ops.cuh", "fdpf.h", "common.cuh")


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1803_03290_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bench_grid(args, point=0):
    """The named workload's synthetic grid, with ``--xfmr-frac`` of its
    branches made transformers (drawn after the rest: the grid is otherwise
    the same).  ``point`` > 0 is another operating point of the same grid:
    every load scaled by 1 + 0.02 point (the rank's share of a multi-point
    study when several GPUs run)."""
    from gridgen import CONFIGS, config_grid, make_grid
    lam = getattr(args, "load_scale", 0.0) or 0.0
    if args.xfmr_frac <= 0 and lam <= 0 and point == 0:
        return config_grid(args.config)
    kw = dict(CONFIGS[args.config])
    if lam > 0:
        kw["load_scale"] = lam
    kw["load_scale"] *= 1.0 + 0.02 * point
    g = make_grid(gen_share=1.0, xfmr_frac=args.xfmr_frac, **kw)
    g.meta["config"] = args.config
    return g


def xfmr_note(args):
    note = f", {100 * args.xfmr_frac:g} % transformers" if args.xfmr_frac > 0 else ""
    if getattr(args, "load_scale", 0.0) > 0:
        note += f", loads scaled by {args.load_scale:g}"
    return note


def run_gpcg(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1803_03290_gb300 as gp

    # weak scaling over GPUs: rank r screens every outage of operating point
    # r of the grid (its loads scaled by 1 + 0.02 r), so the units -- pairs of
    # operating point and outage -- are sharded by point with no collective
    g = bench_grid(args, rank if world > 1 else 0)
    prec = {"fp32": gp.BATCHED_FP32, "fp64": gp.BATCHED_FP64,
            "fp16f": gp.BATCHED_FP32_F16}[args.precision]
    pc = {"exact": gp.PRECOND_EXACT, "ic0": gp.PRECOND_IC0, "jacobi": gp.PRECOND_JACOBI}[args.precond]
    knobs = dict(tile=args.tile, ctas_per_sm=args.ctas_per_sm, tail_rows=args.tail_rows)
    c = gp.GPCG(g, precision=prec, precond=pc, tol=1e-4, **knobs)
    c.base_solve()
    info = c.info()
    S = g.n_branch if args.n_outages <= 0 else min(args.n_outages, g.n_branch)
    outages = torch.arange(S, dtype=torch.int32, device=dev)
    n, m = g.n_bus, g.n_branch
    # one screen call for all outages, or (--chunk K) one call per chunk of K
    # outages into the same output buffers (each chunk size replays its graph)
    K = S if args.chunk <= 0 else min(args.chunk, S)
    out = {
        "theta": torch.empty((K, n), dtype=torch.float64, device=dev),
        "V": torch.empty((K, n), dtype=torch.float64, device=dev),
        "flow": torch.empty((K, m), dtype=torch.float64, device=dev),
        "iters": torch.empty((K, 3), dtype=torch.int32, device=dev),
        "status": torch.empty((K,), dtype=torch.int32, device=dev),
        "max_loading": torch.empty((K,), dtype=torch.float64, device=dev),
        "n_overload": torch.empty((K,), dtype=torch.int32, device=dev),
    }
    all_iters = torch.empty((S, 3), dtype=torch.int32, device=dev)
    all_status = torch.empty((S,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    # --streams N (with --chunk): N contexts, each with its own stream and
    # buffers, take the chunks in turn, so a chunk's kernel fills the SMs
    # that the previous chunk's draining kernel has left
    NS = max(1, args.streams) if K < S else 1
    ctxs, streams, outs = [c], [stream], [out]
    for _ in range(NS - 1):
        ci = gp.GPCG(g, precision=prec, precond=pc, tol=1e-4, **knobs)
        ci.base_solve()
        ctxs.append(ci)
        streams.append(torch.cuda.Stream(device=dev))
        outs.append({key: torch.empty_like(v) for key, v in out.items()})

    def screen_all(timings=None):
        if NS > 1:
            start = torch.cuda.Event()
            start.record(stream)
            for st in streams[1:]:
                st.wait_event(start)
        for j, k0 in enumerate(range(0, S, K)):
            k1 = min(S, k0 + K)
            cj, sj, oj = ctxs[j % NS], streams[j % NS], outs[j % NS]
            o = {key: v[:k1 - k0] for key, v in oj.items()}
            cj.n1_screen_device(outages[k0:k1], o, sj)
            with torch.cuda.stream(sj):
                all_iters[k0:k1].copy_(o["iters"])
                all_status[k0:k1].copy_(o["status"])
            if timings is not None and NS == 1:
                torch.cuda.synchronize()
                timings.append(cj.last_timings())
        if NS > 1:
            for st in streams[1:]:
                done = torch.cuda.Event()
                done.record(st)
                stream.wait_event(done)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    for _ in range(args.warmup):
        screen_all()
    torch.cuda.synchronize()
    info = c.info()  # the tile width the autotuner chose on the first call
    step_ms, kern_ms = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            chunk_ms = []
            ev0.record(stream)
            screen_all(chunk_ms if K < S else None)
            ev1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            if NS > 1:  # concurrent chunks: the step's span stands for the kernel time
                kern_ms.append((0.0, step_ms[-1]))
            elif K < S:
                kern_ms.append((sum(t[0] for t in chunk_ms), sum(t[1] for t in chunk_ms)))
            else:
                kern_ms.append(c.last_timings())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    from paper_1803_03290_gb300.shard import max_over_ranks
    total_ms = max_over_ranks(float(sum(step_ms)), device=dev)
    value = world * S * args.steps / (total_ms / 1e3)
    iters = all_iters.cpu().numpy()
    status = all_status.cpu().numpy()

    # end to end through the public C ABI with host buffers (pinned): outage
    # list in, results out -- the screening summary (status, iterations, max
    # loading, overload count) and, separately, every output of the screen
    # (also angles, magnitudes, flows and island labels)
    hout = np.arange(S, dtype=np.int32)

    def e2e_run(names):
        shapes = {"theta": ((S, n), torch.float64), "V": ((S, n), torch.float64),
                  "flow": ((S, m), torch.float64), "label": ((S, n), torch.int32),
                  "iters": ((S, 3), torch.int32), "status": ((S,), torch.int32),
                  "max_loading": ((S,), torch.float64), "n_overload": ((S,), torch.int32)}
        bufs = {k: torch.empty(*shapes[k][:1], dtype=shapes[k][1], pin_memory=True)
                for k in names}
        ms = []
        if world > 1:
            dist.barrier()
        for k in range(args.steps + 1):
            t0 = time.perf_counter()
            c.n1_screen(hout, out=bufs)
            dt = (time.perf_counter() - t0) * 1e3
            if k:
                ms.append(dt)
        # the slowest rank's mean step time (each rank screens its own point)
        mean_ms = max_over_ranks(statistics.mean(ms), device=dev)
        return {"value": world * S / (mean_ms / 1e3), "unit": "scenarios/s",
                "h2d_bytes_per_step": int(hout.nbytes),
                "d2h_bytes_per_step": int(sum(b.numel() * b.element_size() for b in bufs.values())),
                "outputs": ", ".join(names)}

    e2e = e2e_run(("iters", "status", "max_loading", "n_overload"))
    e2e_full = None
    if not args.e2e_summary_only:
        e2e_full = e2e_run(("theta", "V", "flow", "label", "iters", "status", "max_loading",
                            "n_overload"))

    # plain per-scenario FP64 PCG on a sample (one scenario per launch sequence)
    plain = None
    if args.plain_sample > 0 and rank == 0:
        c.set_options(precision=gp.PLAIN_FP64)
        ps = min(args.plain_sample, S)
        samp = np.random.default_rng(7).choice(S, ps, replace=False).astype(np.int32)
        c.n1_screen(samp[:4], outputs=("status",))
        t0 = time.perf_counter()
        c.n1_screen(samp, outputs=("status",))
        dt = time.perf_counter() - t0
        plain = {"value": ps / dt, "unit": "scenarios/s",
                 "sample": f"{ps} seeded outages of {args.config}, FP64, one scenario at a time "
                           f"over the whole GPU"}
        c.set_options(precision=prec)

    w = 8 if prec == gp.BATCHED_FP64 else 4
    algo = algorithmic_bytes(info, iters, w, n, m)
    fd_ms = statistics.mean(k[1] for k in kern_ms)
    peak, peak_kind = load_peaks()
    achieved = algo / (fd_ms / 1e3) / 1e9
    default_workload = (args.config == "grid10k" and args.precision == "fp32" and
                        args.xfmr_frac == 0 and args.chunk <= 0 and args.load_scale <= 0 and
                        args.precond == "exact" and args.n_outages <= 0)
    shape = {"tile": info["tile"], "ctas_per_sm": info["ctas_per_sm"],
             "tail_rows": [info["tail_rows_p"], info["tail_rows_q"]]}
    traffic = (KERNEL_TRAFFIC["bytes"] if default_workload and shape == KERNEL_TRAFFIC["knobs"]
               and kernel_digest() == KERNEL_TRAFFIC["sha256"] else None)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_source": ("recorded ncu capture of these kernel sources" if traffic
                               else None),
            "kernel": "fdpf_tiles_kernel", "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": int(algo), "kernel_ms": round(fd_ms, 3),
            "islands_kernel_ms": round(statistics.mean(k[0] for k in kern_ms), 3)}
    if w == 4:  # FP32 inner solves: the FP64 work is the mismatch, updates and flows
        f64 = fp64_operations(g, iters)
        roof["fp64_pipe"] = {"ops_per_launch": int(f64),
                             "achieved_gops": round(f64 / (fd_ms / 1e3) / 1e9, 1),
                             "peak_gops": FP64_PEAK_GOPS,
                             "frac": round(f64 / (fd_ms / 1e3) / 1e9 / FP64_PEAK_GOPS, 4),
                             "peak_source": "nominal (1.25 TFLOP/s, FMA = 2 FLOP)"}
    n_chunks = (S + K - 1) // K
    if n_chunks > 1:  # bytes and kernel time summed over the step's launches
        roof["launches_per_step"] = n_chunks
    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_baseline(g, args.cpu_sample)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "scenarios/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w == 4 else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: {n} buses, {m} branches{xfmr_note(args)}, "
                                   f"{S} single-branch "
                                   f"outages{f' in chunks of {K}' if n_chunks > 1 else ''}"
                                   f"{f' on {NS} streams' if NS > 1 else ''}, "
                                   f"tol 1e-4 p.u., {args.precond} base-case preconditioner, "
                                   f"{args.precision} inner PCG, FP64 mismatch/flows"
                                   f"{f'; {world} operating points (loads x 1 + 0.02 r), one per GPU' if world > 1 else ''}",
                       "n_bus": n, "n_branch": m, "scenarios": S, "tile": info["tile"],
                       "ctas_per_sm": info["ctas_per_sm"],
                       "tail_rows": [info["tail_rows_p"], info["tail_rows_q"]],
                       "knobs": {0: "options", 1: "autotuner probes",
                                 2: "autotuner cache"}[info["tuned"]],
                       "chunk": K, "streams": NS,
                       "l2": "flushed between steps (512 MiB write)",
                       "precond": args.precond, "precision": args.precision},
            "e2e": e2e, "e2e_full": e2e_full, "gpu_launches": 2 * n_chunks * args.steps,
            "roofline": roof, "cpu_baseline": cpu, "plain": plain,
            "clocks": clk.summary(),
            "scenarios": {"converged": int((status == 0).sum()), "island_no_gen": int((status == 3).sum()),
                          "maxiter": int((status == 1).sum()), "diverged": int((status == 2).sum()),
                          "mean_outer": float(iters[:, 0].mean()),
                          "mean_inner_P": float(iters[:, 1].mean()),
                          "mean_inner_Q": float(iters[:, 2].mean()),
                          "islanding": island_split(g, iters)},
        }
        print(json.dumps(line), flush=True)
    for ci in ctxs:
        ci.close()
    if world > 1:
        dist.destroy_process_group()


_DC_GRID = None


def _dc_init(name):
    global _DC_GRID
    from gridgen import config_grid
    _DC_GRID = config_grid(name)


def _dc_chunk(outs):
    from oracle import dc
    dc.dc_screen(_DC_GRID, outs)
    return len(outs)


def _gen_chunk(args):
    name, xf, buses = args
    from oracle import powerflow as pf
    from oracle import screen
    g = bench_grid(argparse.Namespace(config=name, xfmr_frac=xf))
    th0, V0, _, _, _ = pf.base_case(g, tol=1e-10, max_outer=200)
    t0 = time.perf_counter()
    screen.n1_screen(g, th0, V0, buses, tol=1e-4, processes=1, kind="generator")
    return time.perf_counter() - t0


def run_gen(args):
    """The N-1 screen of generator outages: every PV bus's generator trips in
    turn (the bus becomes PQ with its load, the lost generation is
    re-dispatched); the same persistent kernel with a B'' extension row."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1803_03290_gb300 as gp
    g = bench_grid(args)
    prec = {"fp32": gp.BATCHED_FP32, "fp64": gp.BATCHED_FP64,
            "fp16f": gp.BATCHED_FP32_F16}[args.precision]
    c = gp.GPCG(g, precision=prec, tol=1e-4)
    c.base_solve()
    pv = np.flatnonzero(g.bus_type == 1).astype(np.int32)
    if args.n_outages > 0:
        pv = pv[:args.n_outages]
    S, n, m = pv.size, g.n_bus, g.n_branch
    buses = torch.from_numpy(pv).to(dev)
    out = {"iters": torch.empty(S, 3, dtype=torch.int32, device=dev),
           "status": torch.empty(S, dtype=torch.int32, device=dev),
           "max_loading": torch.empty(S, dtype=torch.float64, device=dev)}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    for _ in range(args.warmup):
        c.n1_gen_screen_device(buses, out)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms, kern_ms = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record()
            c.n1_gen_screen_device(buses, out)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            kern_ms.append(c.last_timings())
    value = S * args.steps / (sum(ms) / 1e3)
    e2e_ms = []
    for k in range(args.steps + 1):
        t0 = time.perf_counter()
        c.n1_gen_screen(pv, outputs=("status", "max_loading", "iters"))
        if k:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    status = out["status"].cpu().numpy()
    iters = out["iters"].cpu().numpy()
    info = c.info()
    w = 8 if prec == gp.BATCHED_FP64 else 4
    # the extension row adds one row to every B'' pass
    info_x = dict(info, n_q=info["n_q"] + 1)
    algo = algorithmic_bytes(info_x, iters, w, n, m)
    fd_ms = statistics.mean(k[1] for k in kern_ms)
    peak, peak_kind = load_peaks()
    achieved = algo / (fd_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None,
            "kernel": "fdpf_tiles_kernel (generator outages)", "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": int(algo), "kernel_ms": round(fd_ms, 3),
            "setup_kernel_ms": round(statistics.mean(k[0] for k in kern_ms), 3)}
    cpu = None
    if args.cpu_sample > 0:
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0))
        k = min(args.cpu_sample, S)
        sample = np.random.default_rng(12).choice(pv, k, replace=False)
        chunks = [ch for ch in np.array_split(sample, cores) if len(ch)]
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(len(chunks)) as pool:
            solve_s = pool.map(_gen_chunk, [(args.config, args.xfmr_frac, ch) for ch in chunks])
        wall = time.perf_counter() - t0
        cpu = {"value": round(k / max(solve_s), 2), "unit": "scenarios/s", "cores": len(chunks),
               "kind": "oracle",
               "sample": f"{k} seeded generator outages, tol 1e-4 p.u., one process per core "
                         f"(solve time of the slowest process; {wall:.1f} s wall with set-up)"}
    line = {"metric": "N-1 generator-outage scenarios/sec at 10k buses (mismatch<=1e-4 p.u.)",
            "value": round(value, 1), "unit": "scenarios/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sum(ms) / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec != gp.BATCHED_FP64 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.config}: {n} buses, {m} branches{xfmr_note(args)}, "
                                   f"generator outages of all {S} PV buses, tol 1e-4 p.u., "
                                   f"exact base-case preconditioner, {args.precision} inner PCG",
                       "scenarios": S, "l2": "flushed between steps (512 MiB write)"},
            "e2e": {"value": round(S / (statistics.mean(e2e_ms) / 1e3), 1), "unit": "scenarios/s",
                    "h2d_bytes_per_step": 4 * S, "d2h_bytes_per_step": 24 * S},
            "gpu_launches": 2 * args.steps, "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "scenarios": {"converged": int((status == 0).sum()),
                          "no_gen": int((status == 3).sum()),
                          "maxiter": int((status == 1).sum()),
                          "diverged": int((status == 2).sum()),
                          "mean_outer": float(iters[:, 0].mean()),
                          "mean_inner_P": float(iters[:, 1].mean()),
                          "mean_inner_Q": float(iters[:, 2].mean())}}
    print(json.dumps(line), flush=True)
    c.close()


def _adj_chunk(args):
    name, outs = args
    from gridgen import config_grid
    from oracle import adjoint
    g = config_grid(name)
    t0 = time.perf_counter()
    adjoint.loss_and_grad(g, outs, g.P_sched, 1.0 / g.x)
    return time.perf_counter() - t0


def run_adjoint(args):
    """The adjoint workload: loss and gradients (w.r.t. the bus injections and
    the branch susceptances) of the smooth overload penalty summed over every
    single-branch outage of the DC model -- per scenario one batched PCG for
    theta and one with the symmetric B'_s for lambda, then the sums."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1803_03290_gb300 as gp
    from gridgen import config_grid
    name = args.config if args.config != WORKLOAD else "grid2k"
    g = config_grid(name)
    c = gp.GPCG(g)
    S = g.n_branch if args.n_outages <= 0 else min(args.n_outages, g.n_branch)
    n, m = g.n_bus, g.n_branch
    outages = torch.arange(S, dtype=torch.int32, device=dev)
    P = torch.from_numpy(g.P_sched.astype(np.float64)).to(dev)
    b = torch.from_numpy((1.0 / g.x).astype(np.float64)).to(dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gP = torch.empty(n, dtype=torch.float64, device=dev)
    gb = torch.empty(m, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    for _ in range(args.warmup):
        c.n1_adjoint_device(outages, P, b, loss, gP, gb)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record()
            c.n1_adjoint_device(outages, P, b, loss, gP, gb)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    value = S * args.steps / (sum(ms) / 1e3)
    hout = np.arange(S, dtype=np.int32)
    e2e_ms = []
    for k in range(args.steps + 1):
        t0 = time.perf_counter()
        c.n1_adjoint(hout, g.P_sched, 1.0 / g.x)
        if k:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    cpu = None
    if args.cpu_sample > 0:
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0))
        k = min(args.cpu_sample, S)
        sample = np.random.default_rng(14).choice(S, k, replace=False)
        chunks = [ch for ch in np.array_split(sample, cores) if len(ch)]
        with mp.get_context("spawn").Pool(len(chunks)) as pool:
            secs = pool.map(_adj_chunk, [(name, ch) for ch in chunks])
        cpu = {"value": round(k / max(secs), 2), "unit": "scenarios/s", "cores": len(chunks),
               "kind": "oracle",
               "sample": f"{k} seeded outages (loss and both gradients), one process per core "
                         f"(time of the slowest process)"}
    line = {"metric": "N-1 overload-penalty adjoint scenarios/sec at 2k buses (loss + dL/dP + dL/db)",
            "value": round(value, 1), "unit": "scenarios/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sum(ms) / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{name}: {n} buses, {m} branches, all {S} single-branch "
                                   f"outages, DC model, softplus^2 overload penalty, FP64 "
                                   f"batched PCG with the exact base-case preconditioner",
                       "scenarios": S, "l2": "flushed between steps (512 MiB write)"},
            "e2e": {"value": round(S / (statistics.mean(e2e_ms) / 1e3), 1), "unit": "scenarios/s",
                    "h2d_bytes_per_step": 4 * S + 8 * (n + m),
                    "d2h_bytes_per_step": 8 * (1 + n + m)},
            "gpu_launches": None, "roofline": None, "cpu_baseline": cpu,
            "clocks": clk.summary(), "loss": float(loss.item())}
    print(json.dumps(line), flush=True)
    c.close()


def run_dc(args):
    """The DC (P-theta) quick screen of every outage: one batched PCG solve per
    scenario (plus one FP64 refinement step of FP32 solves), flows, loading."""
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1803_03290_gb300 as gp
    from gridgen import config_grid
    g = config_grid(args.config)
    prec = {"fp32": gp.BATCHED_FP32, "fp64": gp.BATCHED_FP64,
            "fp16f": gp.BATCHED_FP32_F16}[args.precision]
    c = gp.GPCG(g, precision=prec)
    info = c.info()
    S = g.n_branch if args.n_outages <= 0 else min(args.n_outages, g.n_branch)
    n, m = g.n_bus, g.n_branch
    outages = torch.arange(S, dtype=torch.int32, device=dev)
    out = {"iters": torch.empty(S, dtype=torch.int32, device=dev),
           "status": torch.empty(S, dtype=torch.int32, device=dev),
           "max_loading": torch.empty(S, dtype=torch.float64, device=dev)}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    for _ in range(args.warmup):
        c.n1_dc_screen_device(outages, out)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record()
            c.n1_dc_screen_device(outages, out)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    value = S * args.steps / (sum(ms) / 1e3)
    it = out["iters"].cpu().numpy().astype(np.float64)
    hout = np.arange(S, dtype=np.int32)
    e2e_ms = []
    for k in range(args.steps + 1):
        t0 = time.perf_counter()
        r = c.n1_dc_screen(hout, outputs=("status", "max_loading"))
        if k:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    w = 8 if prec == gp.BATCHED_FP64 else 4
    refine = 0.0 if w == 8 else 40.0 * info["n_p"]     # FP64 residual and update per scenario
    algo = (15.0 * w * info["n_p"] * it.sum() +
            S * (8.0 * info["n_p"] + refine + 8.0 * n + 16.0 * n + 8.0 * m) +
            it.sum() * (info["nnz_p"] + 2 * info["nnz_lp"]) * (w + 4) / max(S, 1))
    peak, peak_kind = load_peaks()
    achieved = algo / (statistics.mean(ms) / 1e3) / 1e9
    cpu = None
    if args.cpu_sample > 0:
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0))
        k = min(args.cpu_sample, m)
        outs = np.random.default_rng(11).choice(m, k, replace=False)
        chunks = [ch for ch in np.array_split(outs, cores) if len(ch)]
        with mp.get_context("spawn").Pool(cores, initializer=_dc_init,
                                          initargs=(args.config,)) as pool:
            pool.map(_dc_chunk, [ch[:1] for ch in chunks])  # every worker warmed
            t0 = time.perf_counter()
            pool.map(_dc_chunk, chunks)
            dt = time.perf_counter() - t0
        cpu = {"value": round(k / dt, 2), "unit": "scenarios/s", "cores": cores,
               "kind": "oracle",
               "sample": f"{k} seeded outages, direct solve per scenario, "
                         f"one process per core ({dt:.1f} s wall)"}
    line = {"metric": "DC (P-theta) N-1 quick-screen scenarios/sec at 10k buses", "value": round(value, 1),
            "unit": "scenarios/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(ms) / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w == 4 else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: {n} buses, {m} branches, {S} single-branch "
                                   f"outages, DC model, exact base-case preconditioner, "
                                   f"{args.precision} PCG", "l2": "flushed between steps (512 MiB write)"},
            "e2e": {"value": S / (statistics.mean(e2e_ms) / 1e3), "unit": "scenarios/s",
                    "h2d_bytes_per_step": int(hout.nbytes),
                    "d2h_bytes_per_step": int(r["status"].nbytes + r["max_loading"].nbytes)},
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "dc_tiles_kernel", "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": int(algo)},
            "cpu_baseline": cpu, "clocks": clk.summary(),
            "scenarios": {"ok": int((r["status"] == 0).sum()), "island_no_gen": int((r["status"] == 3).sum()),
                          "mean_iters": float(it.mean())}}
    print(json.dumps(line), flush=True)
    c.close()


def cpu_baseline(g, sample):
    """The oracle, as it stands, on a seeded sample of outages, all host cores."""
    from oracle import powerflow as pf
    from oracle import screen
    cores = len(os.sched_getaffinity(0))
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-10, max_outer=200)
    sample = min(sample, g.n_branch)
    outs = np.random.default_rng(11).choice(g.n_branch, sample, replace=False)
    t0 = time.perf_counter()
    screen.n1_screen(g, th0, V0, outs, tol=1e-4, max_outer=50, processes=cores)
    dt = time.perf_counter() - t0
    return {"value": round(sample / dt, 2), "unit": "scenarios/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample} seeded outages of the same grid, tol 1e-4 p.u., "
                      f"one process per core ({dt:.1f} s wall)"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from oracle import powerflow as pf
    from oracle import screen
    g = bench_grid(args)
    cores = len(os.sched_getaffinity(0))
    th0, V0, _, st, _ = pf.base_case(g, tol=1e-10, max_outer=200)
    per_step = min(args.ref_sample, g.n_branch)
    rng = np.random.default_rng(13)
    for _ in range(args.warmup):
        screen.n1_screen(g, th0, V0, rng.choice(g.n_branch, min(cores, per_step), replace=False),
                         tol=1e-4, processes=cores)
    times = []
    for _ in range(args.steps):
        outs = rng.choice(g.n_branch, per_step, replace=False)
        t0 = time.perf_counter()
        screen.n1_screen(g, th0, V0, outs, tol=1e-4, processes=cores)
        times.append(time.perf_counter() - t0)
    value = per_step * args.steps / sum(times)
    line = {"metric": METRIC, "value": round(value, 2), "unit": "scenarios/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.config}: {g.n_bus} buses, {g.n_branch} branches"
                                   f"{xfmr_note(args)}, "
                                   f"{per_step} seeded outages per step, tol 1e-4 p.u."},
            "cpu_baseline": {"value": round(value, 2), "unit": "scenarios/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{per_step} seeded outages per step, one process per core"},
            "e2e": {"value": round(value, 2), "unit": "scenarios/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpcg", choices=["gpcg", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16f"],
                    help="inner PCG: FP32, FP64, or FP32 vectors with a scaled FP16 factor")
    ap.add_argument("--precond", default="exact", choices=["exact", "ic0", "jacobi"])
    ap.add_argument("--tile", type=int, default=0, help="scenarios per tile (0: autotuned)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="tiles per SM (0: autotuned)")
    ap.add_argument("--tail-rows", type=int, default=0,
                    help="dense-tail cap of the substitutions (0: autotuned, -1: none)")
    ap.add_argument("--n-outages", type=int, default=0, help="screen only the first K outages (0 = all)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="screen the outages in calls of this many (0 = one call)")
    ap.add_argument("--streams", type=int, default=1,
                    help="with --chunk: contexts and streams that take the chunks in turn")
    ap.add_argument("--cpu-sample", type=int, default=400)
    ap.add_argument("--e2e-summary-only", action="store_true",
                    help="skip the end-to-end run that returns every output")
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--ref-sample", type=int, default=256)
    ap.add_argument("--load-scale", type=float, default=0.0,
                    help="loading factor lambda of the grid's loads (0: the workload's own)")
    ap.add_argument("--xfmr-frac", type=float, default=0.0,
                    help="make this fraction of the branches transformers (turns ratio "
                         "U[0.95, 1.05] at the from end); 0 = the plain workload")
    ap.add_argument("--workload", default="ac", choices=["ac", "dc", "gen", "adjoint"],
                    help="ac: the FDPF N-1 screen of branch outages (the headline); dc: the "
                         "P-theta quick screen; gen: the FDPF screen of generator outages; "
                         "adjoint: loss and gradients of the overload penalty (grid2k)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "dc":
        run_dc(args)
    elif args.workload == "gen":
        run_gen(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_gpcg(args)


if __name__ == "__main__":
    main()
