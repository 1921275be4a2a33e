#!/usr/bin/env python
"""Benchmark of the PLAS grid sort on GB300 (one JSON line on rank 0).

Metric: milliseconds per 1M x 14-D grid sort -- one complete sort of a
1024 x 1024 grid (N = 1,048,576) of 14 sort channels with 45 carried
channels, 3DGS-shaped synthetic data, default schedule, inputs resident in HBM.
A step is one full call of plas_sort (normalise, initial placement, every
iteration of the shrinking-radius schedule, permutation + carried gather).

  python bench.py [--steps K] [--warmup W] [--workload 3dgs-1024|3dgs-512|3dgs-1448|rgb-64|rgb-512]
  python bench.py --impl reference      # the CPU oracle on this host's cores
  python bench.py --workload rgb-512 --threshold-sweep   # VAD vs runtime over tol

Under torchrun (N > 1) every rank sorts its own replica (different seed): the
sort has no data-path exchange, so the job is N independent replicas and
'value' is the whole-job time per sort (max-over-ranks elapsed / sorts done).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "3dgs-1024": dict(side=1024, D=14, C=45, kind="3dgs",
               desc="1024x1024 grid (N=1,048,576), 14 sort + 45 carried fp32 channels, "
                    "3DGS-shaped synthetic attributes, seed 0, default schedule"),
    "3dgs-512": dict(side=512, D=14, C=45, kind="3dgs",
                 desc="512x512 grid (N=262,144), 14 sort + 45 carried fp32, 3DGS-shaped"),
    "3dgs-1448": dict(side=1448, D=14, C=45, kind="3dgs",
                 desc="1448x1448 grid (N=2,096,704), 14 sort + 45 carried fp32, 3DGS-shaped"),
    "rgb-64": dict(side=64, D=3, C=0, kind="rgb",
                 desc="64x64 grid (N=4096), 3 fp32 channels U[0,1)"),
    "rgb-512": dict(side=512, D=3, C=0, kind="rgb",
               desc="512x512 grid (N=262,144), 3 fp32 channels U[0,1) (paper's runtime test)"),
}
METRIC = "ms per 1M x 14-D grid sort"
FP32_FMA_LANES_PER_SM = 128  # sm_103a: 4 SM sub-partitions x 32 FP32 lanes

# Per-launch DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernel class, averaged over every launch of that class in one
# sort of the workload, from an ncu launch list of
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none -c 22000 --csv python bench.py --steps 1 --warmup 3
#       --no-cpu-baseline --no-serve --tune 12,96,4,0
# keyed by the sha1 of the target-pass sources it was taken on: a stale hash
# reports null.
NCU_TRAFFIC = {
    ("blur_cols", "3dgs-1024"): {"bytes_per_launch": 94084815, "src": "8c506d80d500"},
}
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _kernel_hash():
    """Hash of the sources of the target-pass kernels (the ring body lives in
    sweep_bodies.cuh): a stored ncu traffic figure is used only while they
    are unchanged."""
    h = hashlib.sha1()
    for name in ("fir_kernels.cu", "sweep_bodies.cuh"):
        with open(os.path.join(ROOT, "paper_2312_13299_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="plas_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [t.strip() for t in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows]
        util = [num(r[4]) for r in rows]
        loaded = [s for s, u in zip(sm, util) if s is not None and u is not None and u >= 50]
        if not loaded:
            loaded = [s for s in sm if s is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons, "samples": len(rows)}


def make_inputs(wl, seed=0):
    from paper_2312_13299_gb300 import synth
    n = wl["side"] * wl["side"]
    if wl["kind"] == "rgb":
        return synth.rgb_uniform(wl["side"], seed=seed), None
    return synth.gaussians_3dgs(n, seed=seed, with_carried=wl["C"] > 0)


def pass_fmas(length, r, other, D):
    t = 0
    for p in range(length):
        t += min(r, length - 1 - p) - max(-r, -p) + 1
    return t * other * D


def roofline(stats_list, peaks, peaks_src, clocks, wl):
    """Dominant kernel class of the timed steps and its achieved rate."""
    agg = {}
    for st in stats_list:
        for name, k in st["kernels"].items():
            a = agg.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            for f in a:
                a[f] += k[f]
    name = max(agg, key=lambda n: agg[n]["ms"])
    k = agg[name]
    total_ms = sum(a["ms"] for a in agg.values()) or 1.0
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = 152 * FP32_FMA_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hbm = peaks["hbm_gbs"]
    secs = k["ms"] / 1e3
    gbs = k["bytes"] / secs / 1e9 if secs > 0 else 0.0
    tfl = k["flops"] / secs / 1e12 if secs > 0 else 0.0
    if k["flops"] > 0 and tfl / fp32_peak_tflops > gbs / hbm:
        out = {"bound": "alu", "achieved": round(tfl, 3), "peak": round(fp32_peak_tflops, 2),
               "unit": "TFLOP/s", "frac": round(tfl / fp32_peak_tflops, 4),
               "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz"}
    else:
        out = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
               "frac": round(gbs / hbm, 4), "peak_source": f"{peaks_src} hbm_gbs"}
    tr = NCU_TRAFFIC.get((name, wl))
    out.update({"kernel": name, "traffic": (tr["bytes_per_launch"] if tr and tr["src"] == _kernel_hash() else None),
                "launches": int(k["launches"]), "avg_launch_us": round(k["ms"] * 1e3 / max(1, k["launches"]), 2),
                "share": round(k["ms"] / total_ms, 4)})
    per_kernel = {}
    for n, a in agg.items():
        s = a["ms"] / 1e3
        per_kernel[n] = {"launches": int(a["launches"]), "ms": round(a["ms"], 3),
                         "share": round(a["ms"] / total_ms, 4),
                         "GB/s": round(a["bytes"] / s / 1e9, 1) if s > 0 else None,
                         "TFLOP/s": round(a["flops"] / s / 1e12, 3) if s > 0 and a["flops"] else None}
    return out, per_kernel


def oracle_level_counts(workload):
    """Iterations per radius level of the complete oracle sort of this
    workload (data seed 0, Philox seed 0, default schedule), from the fixture
    that tests/golden/make_sort_goldens.py writes by running the oracle alone;
    None when no such fixture exists."""
    p = os.path.join(GOLDEN, f"oracle_sort_{workload}.json")
    if not os.path.exists(p):
        return None, p
    with open(p) as f:
        return json.load(f)["iterations_per_level"], p


def cpu_baseline(x_np, workload, wl, max_cpu_s=20.0):
    """The oracle's projected time per sort on this host's cores: all cores,
    and one thread (sampled at middle and small radii only, so that the
    bounded sample stays within seconds)."""
    import oracle
    counts, src = oracle_level_counts(workload)
    if counts is None:
        return {"value": None, "error": f"no oracle fixture {os.path.relpath(src, ROOT)}"}
    oracle.build()
    n_all = len(os.sched_getaffinity(0))
    oracle.set_num_threads(n_all)
    ms, sample, cpu_s = oracle_projection(x_np, wl, 0, counts, max_cpu_s=max_cpu_s)
    out = {"value": round(ms, 1), "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": sample, "cpu_seconds": round(cpu_s, 1), "projected": True,
           "level_counts": f"oracle fixture {os.path.relpath(src, ROOT)}"}
    oracle.set_num_threads(1)
    ms1, sample1, cpu1 = oracle_projection(x_np, wl, 0, counts, max_cpu_s=max_cpu_s,
                                           radii=(100.0, 10.0, 1.0))
    oracle.set_num_threads(n_all)
    out["one_thread"] = {"value": round(ms1, 1), "unit": "ms", "cores": 1, "sample": sample1,
                         "cpu_seconds": round(cpu1, 1), "projected": True}
    return out


def oracle_projection(x, wl, seed, level_counts, max_cpu_s=30.0, radii=None):
    """Bounded CPU-oracle sample -> projected ms for the whole sort.

    The oracle runs one and two iterations resumed at the first iteration of a
    few sampled levels, from its own random initial placement (the cost of an
    iteration depends on the radius and the block side, not on the grid's
    values, so no GPU state is needed).  The per-iteration cost at each
    sampled level (two-iteration minus one-iteration wall time) is fitted as
    a + b*FMAs and multiplied out over the per-level iteration counts of the
    schedule (level_counts, from the oracle's own complete run)."""
    import numpy as np
    import oracle
    side, D = wl["side"], wl["D"]
    N = side * side
    phis = oracle.levels(side, side)
    first_it = np.concatenate([[0], np.cumsum(level_counts)[:-1]])
    targets = list(radii) if radii else [phis[0], 100.0, 10.0, 1.0]
    sample_levels = sorted({int(np.argmin(np.abs(phis - t))) for t in targets})
    # the oracle's initial placement: Gaussian i at position pi0(i)
    perm0 = np.empty(N, np.int32)
    perm0[oracle.prp_table(seed, oracle.TAG_INIT, 0, N)] = np.arange(N, dtype=np.int32)
    pts = []
    t_start = time.time()
    for L in sample_levels:
        start = int(first_it[L])
        st = oracle.State()
        st.it, st.epoch, st.level = start, start, L
        times = []
        for n_it in (1, 2):
            t0 = time.perf_counter()
            oracle.sort(x, side, side, seed=seed, sched=oracle.default_schedule(max_iters=start + n_it),
                        perm_in=perm0, state=st, trace_cap=1)
            times.append(time.perf_counter() - t0)
        r = int(math.floor(phis[L]))
        fm = pass_fmas(side, min(r, side - 1), side, D) * 2
        pts.append((fm, max(times[1] - times[0], 1e-6), L))
        if time.time() - t_start > max_cpu_s:
            break
    A = np.array([[1.0, p[0]] for p in pts])
    y = np.array([p[1] for p in pts])
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    a, b = float(max(coef[0], 0.0)), float(max(coef[1], 0.0))
    total = 0.0
    for L, n in enumerate(level_counts):
        r = int(math.floor(phis[L]))
        total += n * (a + b * pass_fmas(side, min(r, side - 1), side, D) * 2)
    sample = (f"one and two oracle iterations resumed at levels {[p[2] for p in pts]} "
              f"(radii {[int(phis[p[2]]) for p in pts]}) from the oracle's own initial placement; "
              f"per-iteration cost fitted as a + b*FMAs and "
              f"projected over the schedule's {int(sum(level_counts))} iterations")
    return total * 1e3, sample, time.time() - t_start


def _dist_setup():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def _max_over_ranks(v, pg, device):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def _barrier(pg):
    if pg is not None:
        pg.barrier()


def run_plas(args):
    import numpy as np
    import torch
    import paper_2312_13299_gb300 as plas
    from paper_2312_13299_gb300 import build as _b
    world, rank, local, pg = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not _b.up_to_date():
        _b.build()
    plas.load()
    wl = WORKLOADS[args.workload]
    side, D, C = wl["side"], wl["D"], wl["C"]
    seed = rank
    x_np, car_np = make_inputs(wl, seed=seed)
    x = torch.from_numpy(x_np).to(dev)
    car = torch.from_numpy(car_np).to(dev) if car_np is not None else None
    ws = torch.empty(plas.sort_workspace_bytes(side, side, D, plas.Schedule(
        target_mode=1 if args.target == "box" else 0)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # launch shapes for this grid shape (the results do not depend on them):
    # measured by the autotuner, or pinned with --tune SMALL_BELOW,MEDIUM_BELOW,CTAS_PER_SM
    # (a profiler distorts the tuner's own timings, so profiled runs pin the
    # values a plain run chose)
    t_tune = time.perf_counter()
    if args.tune == "auto":
        tune = plas.autotune(side, side, D)
    else:
        sb, mb, per, *tma = (int(v) for v in args.tune.split(","))
        plas.set_tuning(side, side, D, fir_small_below=sb, fir_medium_below=mb,
                        assign_ctas_per_sm=per, large_tma=tma[0] if tma else None)
        tune = plas.get_tuning(side, side, D)
    t_tune = time.perf_counter() - t_tune

    tmode = 1 if args.target == "box" else 0

    def step(profile):
        return plas.sort(x, side, side, carried=car, seed=seed, workspace=ws,
                         schedule=plas.Schedule(profile=profile, target_mode=tmode), want_stats=True)

    for _ in range(args.warmup):
        step(False)

    def timed(profile):
        """K sorts bracketed by barrier + synchronize; CUDA events on the
        launching stream; clocks sampled meanwhile."""
        torch.cuda.synchronize()
        _barrier(pg)
        clocks = ClockSampler(local)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        _barrier(pg)
        e0.record(stream)
        sts = [step(profile).stats for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier(pg)
        ck = clocks.stop()
        return _max_over_ranks(e0.elapsed_time(e1), pg, dev), sts, ck

    # the measured value: plain sorts, no per-kernel events
    max_ms, stats_plain, ck = timed(False)
    ms_per_sort = max_ms / (args.steps * world)
    launches = int(sum(st["launches"] for st in stats_plain))
    # per-kernel durations for the roofline: the same K sorts again with a
    # CUDA event pair around every launch (their own timed region)
    n_prof = args.steps
    args_steps = args.steps
    args.steps = min(args.steps, 3)
    prof_ms, stats, ck_prof = timed(True)
    n_prof, args.steps = args.steps, args_steps

    # end to end: pinned host inputs in, permutation + carried out, per step
    xh = torch.from_numpy(x_np).pin_memory()
    ch = torch.from_numpy(car_np).pin_memory() if car_np is not None else None
    ph = torch.empty(side * side, dtype=torch.int32).pin_memory()
    coh = torch.empty_like(ch).pin_memory() if ch is not None else None
    xd = torch.empty_like(x)
    cd = torch.empty_like(car) if car is not None else None
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_e2e = max(1, min(args.steps, 3))

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        if cd is not None:
            cd.copy_(ch, non_blocking=True)
        r = plas.sort(xd, side, side, carried=cd, seed=seed, workspace=ws,
                      schedule=plas.Schedule(target_mode=tmode))
        ph.copy_(r.perm, non_blocking=True)
        if coh is not None:
            coh.copy_(r.carried, non_blocking=True)

    e2e_step()  # warm-up (untimed): the output tensors' first allocation
    torch.cuda.synchronize()
    _barrier(pg)
    e2.record(stream)
    for _ in range(n_e2e):
        e2e_step()
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(e2.elapsed_time(e3), pg, dev) / (n_e2e * world)
    h2d = x_np.nbytes + (car_np.nbytes if car_np is not None else 0)
    d2h = ph.numel() * 4 + (coh.numel() * 4 if coh is not None else 0)

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    peaks, psrc = _peaks()
    rl, per_kernel = roofline(stats, peaks, psrc, ck_prof or ck, args.workload)
    rl["timing"] = (f"CUDA events around every launch over {n_prof} further sorts "
                    f"({prof_ms / n_prof:.1f} ms per sort with the events)")
    st0 = stats_plain[-1]
    line = {
        "metric": METRIC, "value": round(ms_per_sort, 3), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded numpy; 3DGS-shaped attributes, no dataset)",
        "config": {"workload": wl["desc"], "grid": f"{side}x{side}", "N": side * side, "D": D,
                   "carried": C, "iterations_per_sort": st0["iterations"], "levels": st0["levels"],
                   "target": "box (fixed-point window mean, schedule.target_mode=1)" if tmode
                             else "gaussian (default)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2_policy": "working set (grid, target, row pass, inputs, carried) > 129 MB L2; no flush",
                   "tuning": {"fir_small_below": tune["fir_small_below"],
                              "fir_medium_below": tune["fir_medium_below"],
                              "assign_ctas_per_sm": tune["assign_ctas_per_sm"],
                              "source": "autotune" if args.tune == "auto" else "pinned",
                              "autotune_s": round(t_tune, 2)}},
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "roofline": rl,
        "kernels": per_kernel,
        "melem_iter_per_s": round(side * side * st0["iterations"] / (ms_per_sort / 1e3) / 1e6, 1),
        "clocks": ck,
    }
    if args.cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(x_np, args.workload, wl)
        except Exception as e:  # reported, never silently replaced
            line["cpu_baseline"] = {"value": None, "error": repr(e)}
    if args.serve_in_bench and world == 1:
        # the server's latency policy (fifo_fill) under Poisson arrivals and
        # its throughput policy (all) under a burst, each against plain
        try:
            pairs = [(pp.split(":")[0], [pp.split(":")[1]]) for pp in args.serve_pairs.split(",") if pp]
            line["serve"] = serve_compare(args.requests, [], [], args.sweeps, pairs=pairs)
        except Exception as e:  # reported, never silently replaced
            line["serve"] = {"error": repr(e)}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_reference(args):
    """The CPU oracle as it stands, timed on this host's cores (rank 0 only)."""
    import numpy as np
    world, rank, local, pg = _dist_setup()
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    import oracle
    oracle.build()
    wl = WORKLOADS[args.workload]
    x_np, _ = make_inputs(wl, seed=0)
    counts, src = oracle_level_counts(args.workload)
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no oracle fixture {os.path.relpath(src, ROOT)} for this workload"}), flush=True)
        if pg is not None:
            pg.destroy_process_group()
        return
    oracle.set_num_threads(len(os.sched_getaffinity(0)))
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample, _ = oracle_projection(x_np, wl, 0, counts, max_cpu_s=20.0)
        if i >= args.warmup:
            vals.append(v)
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded numpy; 3DGS-shaped attributes, no dataset)",
            "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample, "projected": True,
                             "level_counts": f"oracle fixture {os.path.relpath(src, ROOT)}"},
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def serve_compare(n, patterns, policies, sweeps, budget_bytes=40 * 10 ** 9, pairs=None):
    """Served stream against the plain path on one GPU: n requests (sides
    U{128..1024}, 14 sort + 45 carried channels, seeded) under an admission
    budget, through the server (continuous batching, one run per policy) and
    through the plain path (one plas_sort per request, first come first
    served).  Arrival patterns: 'poisson' at 0.8 x the plain path's capacity
    (mean service time of the side distribution, from a power-law fit of
    measured plain sorts), 'overload' Poisson at 1.25 x that capacity, and
    'burst' (every request at t = 0).  Latency = completion - arrival (host
    clock).  Every served result (permutation and carried attributes) is
    compared with the plain path's result of the same request."""
    import numpy as np
    import torch
    import paper_2312_13299_gb300 as plas
    from paper_2312_13299_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    fit_sides = [128, 384, 768]
    ts = []
    for side in fit_sides:
        xm, cm = synth.gaussians_3dgs(side * side, seed=999)
        xm_t, cm_t = torch.from_numpy(xm).to(dev), torch.from_numpy(cm).to(dev)
        plas.sort(xm_t, side, side, carried=cm_t)
        torch.cuda.synchronize()
        t = time.perf_counter()
        plas.sort(xm_t, side, side, carried=cm_t)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    b, loga = np.polyfit(np.log(fit_sides), np.log(ts), 1)
    mean_service = float(np.mean([math.exp(loga) * sd ** b for sd in range(128, 1025)]))
    rate = 0.8 / mean_service
    base = synth.request_stream(n, seed=0, rate_per_s=rate)
    inputs = []
    for i, (_, side) in enumerate(base):
        x, c = synth.gaussians_3dgs(side * side, seed=1000 + i)
        inputs.append((side, torch.from_numpy(x).to(dev), torch.from_numpy(c).to(dev), i))
    torch.cuda.synchronize()
    ref = {}

    def plain(arrivals):
        lat, t0, cells_iters = [], time.perf_counter(), 0
        for arr, (side, x, c, i) in zip(arrivals, inputs):
            while time.perf_counter() - t0 < arr:
                time.sleep(0.0005)
            r = plas.sort(x, side, side, carried=c, seed=i)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0 - arr)
            cells_iters += side * side * r.state["it"]
            ref[i] = (r.perm, r.carried)
        return lat, time.perf_counter() - t0, cells_iters, None

    def served(arrivals, policy):
        srv = plas.Server(14, mem_budget=budget_bytes, policy=policy)
        lat, t0, nxt, pending, cells_iters, same = {}, time.perf_counter(), 0, {}, 0, 0
        while len(lat) < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                side, x, c, i = inputs[nxt]
                pending[srv.submit(x, side, side, c, seed=i)] = (arrivals[nxt], side, i)
                nxt += 1
            if not pending:
                time.sleep(0.0005)
                continue
            for tk, res in srv.step(sweeps=sweeps):
                arr, side, i = pending.pop(tk)
                lat[tk] = time.perf_counter() - t0 - arr
                cells_iters += side * side * res.state["it"]
                if i in ref:
                    same += int(torch.equal(res.perm, ref[i][0]) and torch.equal(res.carried, ref[i][1]))
        wall = time.perf_counter() - t0
        srv.close()
        return list(lat.values()), wall, cells_iters, same

    def summary(lat, wall, ci, same):
        lat = np.array(lat) * 1e3
        out = {"p50_ms": round(float(np.percentile(lat, 50)), 1),
               "p99_ms": round(float(np.percentile(lat, 99)), 1),
               "mean_ms": round(float(lat.mean()), 1), "wall_s": round(wall, 2),
               "requests_per_s": round(n / wall, 3), "melem_iter_per_s": round(ci / wall / 1e6, 1)}
        if same is not None:
            out["results_equal_plain"] = f"{same}/{n}"
        return out

    pats = {"poisson": [a for a, _ in base], "overload": [a * 0.8 / 1.25 for a, _ in base],
            "burst": [0.0] * n}
    out = {}
    # (pattern, policies) to run; pairs overrides the full cross product
    plan = pairs if pairs else [(pat, policies) for pat in patterns]
    for pat, pols in plan:
        arr = pats[pat]
        out[pat] = {"plain": summary(*plain(arr))}
        for pol in pols:
            out[pat]["served_" + pol] = summary(*served(arr, pol))
    return {"workload": f"{n} requests, sides U{{128..1024}}, 14 sort + 45 carried fp32, "
                        f"{budget_bytes / 1e9:.0f} GB admission budget, seed 0",
            "poisson_rate_per_s": round(rate, 3),
            "plain_service_fit": f"t = {math.exp(loga):.3g} * side^{b:.2f} s "
                                 f"(mean {mean_service * 1e3:.0f} ms over the side distribution)",
            "sweeps_per_step": sweeps, "results": out}


def run_serve(args):
    """The served stream on its own JSON line (every policy and pattern)."""
    import paper_2312_13299_gb300 as plas
    plas.load()
    policies = [p for p in args.policies.split(",") if p]
    patterns = [p for p in args.patterns.split(",") if p]
    res = serve_compare(args.requests, patterns, policies, args.sweeps)
    first = policies[0] if policies else None
    head = res["results"].get("poisson", next(iter(res["results"].values()), {}))
    line = {"metric": "served p50/p99 latency of PLAS sort requests",
            "value": head.get("served_" + first, {}).get("p99_ms") if first else None,
            "unit": f"ms (p99, served, {first})", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic (seeded numpy; 3DGS-shaped attributes)",
            "config": {k: v for k, v in res.items() if k != "results"}, "results": res["results"]}
    print(json.dumps(line), flush=True)


def run_loss(args):
    """Smoothness loss (Sec. 3.2) on the 1024 x 1024 x 59 grid, sigma 1, 7 x 7:
    forward and hand-written backward, each timed with CUDA events over K
    launches after W warm-ups (inputs 247 MB > L2).  Algorithmic bytes: the
    forward reads x once (4 B/elem); the backward reads x and writes the
    gradient (8 B/elem)."""
    import torch
    import paper_2312_13299_gb300 as plas
    from paper_2312_13299_gb300 import synth
    plas.load()
    H = W = 1024
    x = torch.from_numpy(synth.loss_grid(H, W, seed=0).astype("float32")).cuda()
    C = x.shape[2]
    g = torch.ones((), device="cuda")
    peaks, psrc = _peaks()
    lam_paper = torch.from_numpy(synth.paper_smoothness_weights()).cuda()
    out = {}
    # the benchmark configuration (squared form, sigma 1, 7x7, unit weights)
    # and the paper's regulariser (Huber delta 1, kernel 5, sigma 3, weights
    # 0.09 opacity / 0.91 rotation)
    for name, fn, bpe in [("fwd", lambda: plas.smooth_loss_fwd(x), 4),
                          ("bwd", lambda: plas.smooth_loss_bwd(x, g), 8),
                          ("huber_paper_fwd", lambda: plas.smooth_loss_fwd(
                              x, 3.0, 5, lam_paper, huber_delta=1.0), 4),
                          ("huber_paper_bwd", lambda: plas.smooth_loss_bwd(
                              x, g, 3.0, 5, lam_paper, huber_delta=1.0), 8)]:
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps * 10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (args.steps * 10)
        gbs = bpe * H * W * C / (us * 1e-6) / 1e9
        out[name] = {"us": round(us, 1), "GB/s": round(gbs, 1), "frac": round(gbs / peaks["hbm_gbs"], 3)}
    line = {"metric": "smoothness loss fwd/bwd on 1024x1024x59 (sigma 1, 7x7)",
            "value": out["bwd"]["us"], "unit": "us (backward)", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32", "data": "synthetic (3DGS-shaped 14 + 45 channels)",
            "peak_hbm_gbs": peaks["hbm_gbs"], "peak_source": psrc, "results": out}
    print(json.dumps(line), flush=True)


def run_loss_loop(args):
    """The smoothness loss inside training (Sec. 3.2 with the sort of Sec. 3.1
    between steps) on the 1024 x 1024 x 59 grid: Adam (lr 1e-3) on the
    squared smoothness loss (sigma 1, 7 x 7) for --loop-steps steps; every 100
    steps the grid is re-sorted on its 14 sort channels (warm start from the
    current arrangement), and all 59 channels and both Adam moments follow
    the permutation.  Reported: ms per optimizer step (loss forward +
    hand-written backward + Adam update, CUDA events on the launching stream,
    re-sorts excluded), ms per re-sort and the loss before and after.  The
    loss and gradient against FP64 at every re-sort are checked by
    tests/test_gpu_loss.py::test_loss_loop_full_size_with_resorts."""
    import torch
    import paper_2312_13299_gb300 as plas
    from paper_2312_13299_gb300 import synth
    plas.load()
    H = W = 1024
    P = torch.from_numpy(synth.loss_grid(H, W, seed=0).reshape(H * W, -1).astype("float32")).cuda()
    P.requires_grad_(True)
    opt = torch.optim.Adam([P], lr=1e-3)
    stream = torch.cuda.current_stream()
    step_ms, sort_ms, losses = 0.0, [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for step in range(args.loop_steps):
        if step % 100 == 0:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.no_grad():
                r = plas.sort(P[:, :14].contiguous(), H, W, seed=step,
                              schedule=plas.Schedule(shuffle_init=(step == 0)))
                P.copy_(plas.gather_rows(P.detach(), r.perm))
                for v in (opt.state[P].values() if P in opt.state else []):
                    if torch.is_tensor(v) and v.dim() == 2:
                        v.copy_(plas.gather_rows(v, r.perm))
            torch.cuda.synchronize()
            sort_ms.append((time.perf_counter() - t0) * 1e3)
        e0.record(stream)
        opt.zero_grad(set_to_none=False)
        loss = plas.smooth_loss(P.reshape(H, W, -1), 1.0, 7)
        loss.backward()
        opt.step()
        e1.record(stream)
        e1.synchronize()
        step_ms += e0.elapsed_time(e1)
        if step == 0 or step == args.loop_steps - 1:
            losses.append(float(loss.item()))
    line = {"metric": "smoothness-loss training loop with re-sorts, 1024x1024x59",
            "value": round(step_ms / args.loop_steps, 4), "unit": "ms per optimizer step",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic (3DGS-shaped 14 + 45 channels)",
            "config": {"steps": args.loop_steps, "resort_every": 100, "optimizer": "Adam lr 1e-3",
                       "loss": "squared, sigma 1, 7x7, unit weights"},
            "resort_ms": [round(v, 1) for v in sort_ms], "loss_first": losses[0], "loss_last": losses[-1]}
    print(json.dumps(line), flush=True)


def run_threshold_sweep(args):
    """Sorting quality against runtime over the stall threshold (the
    break-threshold study of the supplementary), for the Gaussian and the box
    target: per (target, tol) and input seed (3 seeds), one warm-up sort and
    one CUDA-event-timed sort of the workload (default: 512 x 512 x 3
    U[0,1)) with autotuned launch shapes; reported are the means over the
    seeds of the time, the iterations and the VAD of the sorted grid on
    values x 255."""
    import torch
    import paper_2312_13299_gb300 as plas
    plas.load()
    wl = WORKLOADS[args.workload]
    side = wl["side"]
    plas.autotune(side, side, wl["D"])
    seeds = (0, 1, 2)
    xs = [torch.from_numpy(make_inputs(wl, seed=s)[0]).cuda() for s in seeds]
    tols = [float(t) for t in args.tols.split(",")]
    results = []
    for target in ("gaussian", "box"):
        for tol in tols:
            sch = plas.Schedule(tol=tol, target_mode=1 if target == "box" else 0)
            ms, its, vads = [], [], []
            for s, x in zip(seeds, xs):
                plas.sort(x, side, side, seed=s, schedule=sch)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r = plas.sort(x, side, side, seed=s, schedule=sch, want_sorted=True)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                its.append(int(r.state["it"]))
                vads.append(plas.grid_metrics(r.sorted.view(side, side, wl["D"]), scale=255.0)[1])
            results.append({"target": target, "tol": tol, "ms": round(statistics.mean(ms), 2),
                            "iterations": round(statistics.mean(its), 1),
                            "vad": round(statistics.mean(vads), 3),
                            "vad_per_seed": [round(v, 3) for v in vads]})
    vad0 = statistics.mean(plas.grid_metrics(x.view(side, side, wl["D"]), scale=255.0)[1]
                           for x in xs)
    line = {"metric": "VAD and ms per sort over the stall threshold", "workload": wl["desc"],
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic", "vad_unsorted": round(vad0, 2), "results": results}
    print(json.dumps(line), flush=True)


def run_stages(args):
    """Preparation before the sort (Sec. 3.1, Sec. 3.3) and quantisation
    after it (Sec. 3.3) on 1,100,000 raw Gaussians of 59 channels (14 sort +
    45 carried; N(0, 1.5) values, seed 0): activation of the 14 sort
    channels, largest-square selection on the opacity logits (channel 10, a
    strided column), row selection of the kept 1048^2 Gaussians, and their
    quantisation to 16-bit codes (q = 65536 for xyz, 256 otherwise) and back.
    Each stage is timed with CUDA events over 10*K calls after W warm-ups.
    Algorithmic bytes per call: activation 56 B read + 56 B written per
    Gaussian; selection 4 B read per Gaussian + 4 B written per kept one;
    row selection 236 B read + 236 B written + 4 B index per kept row;
    (de)quantisation 4 + 2 B per element."""
    import torch
    import paper_2312_13299_gb300 as plas
    plas.load()
    n, C = 1_100_000, 59
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    raw = torch.randn((n, C), generator=gen, device="cuda") * 1.5
    side, keep = plas.grid_select(raw[:, 10])
    kept = plas.select_rows(raw, keep)
    lo = kept.min(dim=0).values.cpu().tolist()
    hi = kept.max(dim=0).values.cpu().tolist()
    q = [65536] * 3 + [256] * (C - 3)
    codes = plas.quantize(kept, lo, hi, q)
    peaks, psrc = _peaks()
    m = side * side
    stages = [("activate_3dgs", lambda: plas.activate_3dgs(raw), 112 * n),
              ("grid_select", lambda: plas.grid_select(raw[:, 10]), 4 * n + 4 * m),
              ("select_rows", lambda: plas.select_rows(raw, keep), m * (8 * C + 4)),
              ("quantize", lambda: plas.quantize(kept, lo, hi, q), 6 * m * C),
              ("dequantize", lambda: plas.dequantize(codes, lo, hi, q), 6 * m * C)]
    out = {}
    for name, fn, nbytes in stages:
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = args.steps * 10
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        gbs = nbytes / (us * 1e-6) / 1e9
        out[name] = {"us": round(us, 2), "bytes": int(nbytes), "GB/s": round(gbs, 1),
                     "frac": round(gbs / peaks["hbm_gbs"], 3)}
    line = {"metric": "preparation and quantisation kernels, 1.1M raw Gaussians x 59 channels",
            "unit": "us per call", "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic N(0, 1.5) raw parameters", "side": side,
            "peak_hbm_gbs": peaks["hbm_gbs"], "peak_source": psrc,
            "timing": "CUDA events over 10*K back-to-back calls (inputs 260 MB > L2)",
            "results": out}
    print(json.dumps(line), flush=True)


def run_ncu_case(args):
    """A bounded launch sequence for profiler captures: the workload's inputs,
    one sort capped at --ncu-case iterations (all at the top radius levels)."""
    import torch
    import paper_2312_13299_gb300 as plas
    plas.load()
    wl = WORKLOADS[args.workload]
    side = wl["side"]
    x_np, _ = make_inputs(wl, seed=0)
    x = torch.from_numpy(x_np).cuda()
    if args.tune != "auto":  # pinned launch shapes (the default shapes otherwise)
        sb, mb, per, *tma = (int(v) for v in args.tune.split(","))
        plas.set_tuning(side, side, wl["D"], fir_small_below=sb, fir_medium_below=mb,
                        assign_ctas_per_sm=per, large_tma=tma[0] if tma else None)
    r = plas.sort(x, side, side, seed=0,
                  schedule=plas.Schedule(max_iters=args.ncu_case, phi0=args.phi0,
                                         target_mode=1 if args.target == "box" else 0),
                  trace_cap=(1 << 20) if args.trace_out else 0)
    torch.cuda.synchronize()
    if args.trace_out:
        # level of every iteration, to attribute a launch list to radius levels
        with open(args.trace_out, "w") as f:
            f.write(" ".join(str(int(v)) for v in r.trace_level.cpu().tolist()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="plas", choices=["plas", "reference"])
    ap.add_argument("--workload", default="3dgs-1024", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--target", default="gaussian", choices=["gaussian", "box"],
                    help="low-pass target of the sort: the Gaussian (default) or the box variant")
    ap.add_argument("--tune", default="auto", help="'auto' (run the autotuner) or "
                    "SMALL_BELOW,MEDIUM_BELOW,CTAS_PER_SM[,LARGE_TMA] to pin the launch shapes")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="ITERS",
                    help="run one sort of the workload capped at ITERS iterations and exit "
                         "(a small, bounded program for ncu captures; prints nothing)")
    ap.add_argument("--trace-out", default="", help="with --ncu-case: write the level of every "
                    "iteration to this file")
    ap.add_argument("--phi0", type=float, default=0.0, help="with --ncu-case: start radius "
                    "(0 = the schedule's default), to profile small radii directly")
    ap.add_argument("--serve", action="store_true",
                    help="served-stream benchmark (continuous batching vs plain), own JSON line")
    ap.add_argument("--loss-loop", action="store_true",
                    help="smoothness loss inside an Adam loop with a re-sort every 100 steps "
                         "(1024x1024x59), own JSON line")
    ap.add_argument("--loop-steps", type=int, default=1000)
    ap.add_argument("--loss", action="store_true",
                    help="smoothness-loss fwd/bwd benchmark on 1024x1024x59, own JSON line")
    ap.add_argument("--threshold-sweep", action="store_true",
                    help="VAD and runtime over the stall threshold, Gaussian and box target, "
                         "own JSON line (use with --workload rgb-512)")
    ap.add_argument("--tols", default="1e-2,3e-3,1e-3,3e-4,1e-4,3e-5,1e-5",
                    help="with --threshold-sweep: the thresholds")
    ap.add_argument("--stages", action="store_true",
                    help="preparation and quantisation kernel benchmark, own JSON line")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--sweeps", type=int, default=8, help="sweeps per server step")
    ap.add_argument("--policies", default="fifo_fill,shortest_first,all",
                    help="with --serve: server policies to run")
    ap.add_argument("--patterns", default="poisson,burst", help="with --serve: arrival patterns "
                    "(poisson = 0.8 x plain capacity, overload = 1.25 x, burst)")
    ap.add_argument("--no-serve", dest="serve_in_bench", action="store_false",
                    help="leave the served-stream comparison out of the default line")
    ap.add_argument("--serve-pairs", default="poisson:fifo_fill,burst:all",
                    help="PATTERN:POLICY pairs of the default line's served-stream comparison")
    args = ap.parse_args()
    if args.ncu_case > 0:
        run_ncu_case(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.loss:
        run_loss(args)
        return
    if args.loss_loop:
        run_loss_loop(args)
        return
    if args.threshold_sweep:
        run_threshold_sweep(args)
        return
    if args.stages:
        run_stages(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_plas(args)


if __name__ == "__main__":
    main()
