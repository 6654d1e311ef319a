#!/usr/bin/env python
"""Benchmark of the Gribov-copy enumerator on the 4D 4^4 compact U(1) workload.

Workload: 4D 4^4 periodic lattice (1024 links), eight von Mises orbits with
kappa_j = 0.5 + 1.5 j/7 (seeds 1-8), 2^20 random starts per orbit, mixed
precision (FP32 sweeps to max div^2 < 1e-10, FP64 polish to 1e-24),
overrelaxation omega = 1.7, FP64 Lanczos Faddeev-Popov test of every distinct
copy, FP64 dedup.
One step = the whole path (starts -> sweeps -> polish -> dedup -> FP test) for
all eight orbits' 2^20 starts, enqueued by one gc_enumerate_batch call as one
captured CUDA graph (fresh orbit objects every step).

Prints one JSON line.  `value` = converged copies per second with the orbits
resident on the device (CUDA events on the launch stream around the
gc_enumerate_batch call of each of the K timed steps); `e2e` = the same metric
through the C ABI with host buffers (link angles uploaded, distinct copies
read back into pinned arrays, every step; steps pipelined so that each step's
read-back runs beside the next step's kernels).  The plain FP64 path is timed
beside it as the same kind of batch on a sample of starts, and so are the same
steps with the FP32 Lanczos screen (`fp32_screen`).  `roofline` is the kernel
with the most time in isolated single-orbit passes, against the library's own
measured unit throughputs (`peaks`); `roofline.kernels` lists every kernel of
the step with its binding unit.
"""
from __future__ import annotations

import argparse
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

import numpy as np  # noqa: E402

import orbit_inputs as oi  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM traffic per start (read + write) of the two heavy kernels, from the ncu
# capture of the 65536-start 4^4 case recorded under profiles/ (None = not
# captured for the current kernel)
TRAFFIC_POLISH_PER_START = (1.34413568e8 + 2.15169792e8) / 65536  # profiles/polish_kernel_4d_L4.md (line polish)
TRAFFIC_RELAX_PER_START = (1.34264832e8 + 7.5560448e7) / 65536   # profiles/relax32_sheet_4d_L4.md
TRAFFIC_FPTEST_PER_COPY = (1.843584e8 + 3.775488e6) / 44636   # profiles/fp_test_pairs_4d_L4.md
# DRAM traffic per launch of the large-lattice leg's kernels (its own workload,
# 592 starts of 4D 16^4), from ncu: profiles/slab_traffic_4d_L16.md
TRAFFIC_SLAB_NEWTON1 = 2.92208894464e11 + 5.7204921344e10
TRAFFIC_SLAB_DSMEM32 = 2.1208832e7 + 2.71034368e8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--starts", type=int, default=1 << 20, help="starts per orbit (one step)")
    p.add_argument("--plain-starts", type=int, default=1 << 16)
    p.add_argument("--cpu-starts", type=int, default=1536)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-configs", action="store_true",
                   help="also time the oracle on configs 1 and 2 (a few minutes of host time)")
    p.add_argument("--check-every", type=int, default=4,
                   help="sweeps between residual checks when --autotune is 1")
    p.add_argument("--autotune", type=int, choices=[1, 2], default=2,
                   help="1: launch shapes only; 2: also the sweep-unroll depth")
    p.add_argument("--no-uneven", dest="uneven", action="store_false",
                   help="skip the uneven-batch leg (26 orbits of 13 lattice sizes in one graph)")
    p.add_argument("--no-large", dest="large", action="store_false",
                   help="skip the large-lattice leg (4D 16^4, hyperplane path)")
    p.add_argument("--serve-requests", type=int, default=100,
                   help="requests of each Poisson serving leg, above and below capacity (0 skips them)")
    return p.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, flags in rows for n, v in zip(names, flags) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------
# CPU legs: the oracle on host cores
# ----------------------------------------------------------------------------

def oracle_sample(orbit, n_starts, start0=0):
    """Whole oracle pipeline on a bounded sample; returns (converged, seconds, threads)."""
    import oracle
    t = time.perf_counter()
    relaxed, cp = oracle.enumerate_copies(orbit.d, orbit.L, orbit.phi, 1, orbit.orbit_id,
                                          n_starts, omega=1.7, eps=1e-24, start0=start0)
    dt = time.perf_counter() - t
    return int((relaxed.status == oracle.CONVERGED).sum()), dt, oracle.max_threads()


def oracle_configs():
    """The oracle on configs 1 and 2 (one thread and all host cores): config 1
    whole pipeline; config 2 (3D 6^3, one orbit) its C relaxation, all 10^5
    starts on all cores and 4096 of them on one thread (the oracle's Python
    dedup is quadratic in the copies, so the full config-2 pipeline is not
    timed)."""
    import oracle
    n_all = oracle.max_threads()   # a thread count, once set, stays: pass it explicitly
    out = {"cores": n_all}
    w1 = oi.workload_2d_4x4()
    o = w1.orbits[0]
    for nt in (1, n_all):
        t = time.perf_counter()
        rel, cp = oracle.enumerate_copies(o.d, o.L, o.phi, 1, o.orbit_id, w1.n_starts, w1.omega,
                                          w1.eps, nthreads=nt)
        dt = time.perf_counter() - t
        key = "config1_1thread" if nt == 1 and n_all > 1 else "config1_all_cores"
        out[key] = {"starts": w1.n_starts, "seconds": dt,
                    "converged_per_s": int((rel.status == oracle.CONVERGED).sum()) / dt,
                    "site_updates_per_s": float(rel.sweeps.sum()) * o.L ** o.d / dt,
                    "distinct": int(len(cp.F)), "pipeline": "whole"}
    w2 = oi.workload_3d_6cubed()
    o = w2.orbits[0]
    for nt, n in ((1, 4096), (n_all, w2.n_starts)):
        t = time.perf_counter()
        rel = oracle.relax_starts(o.d, o.L, o.phi, 1, o.orbit_id, 0, n, w2.omega, w2.eps, nthreads=nt)
        dt = time.perf_counter() - t
        key = "config2_1thread" if nt == 1 and n < w2.n_starts else "config2_all_cores"
        out[key] = {"starts": n, "seconds": dt,
                    "converged_per_s": int((rel.status == oracle.CONVERGED).sum()) / dt,
                    "site_updates_per_s": float(rel.sweeps.sum()) * o.L ** o.d / dt,
                    "pipeline": "relaxation (C, OpenMP over starts)"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = oi.workload_4d_4to4(args.starts)
    per_step = max(64, min(args.cpu_starts, 512))
    for k in range(args.warmup):
        oracle_sample(w.orbits[k % 8], 32, start0=10_000_000 + k)
    conv = 0
    secs = 0.0
    threads = 1
    for k in range(args.steps):
        c, dt, threads = oracle_sample(w.orbits[k % 8], per_step)
        conv += c
        secs += dt
    v = conv / secs
    sample = f"{per_step} starts of orbit k mod 8 per step (of 2^20), full oracle pipeline"
    out = {
        "impl": "reference", "metric": "converged_copies_per_s", "value": v,
        "unit": "copies/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "4d_L4_vonmises_x8", "lattice": "4^4", "orbits": 8,
                   "starts_per_orbit": per_step, "omega": 1.7, "eps": 1e-24},
        "cpu_baseline": {"value": v, "unit": "copies/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "copies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ----------------------------------------------------------------------------
# uneven batch: every (d, L) of the uneven sizes, two orbits each, in one graph
# ----------------------------------------------------------------------------

def uneven_leg(gb, torch, check_every, steps=2):
    # start counts: about 1e9 site updates per size, from the mean FP32 sweeps
    # per start of a 1000-start pilot of each size's first orbit
    mean_sweeps = {}
    for o in oi.workload_uneven().orbits[::2]:
        h = gb.gc_create_orbit(o.d, o.L, o.phi, o.orbit_id)
        gb.gc_enumerate_copies(h, 1000, 1.7, 1e-24,
                               gb.gc_options_default(precision=gb.GC_MIXED, check_every=check_every))
        mean_sweeps[(o.d, o.L)] = gb.gc_orbit_stats(h)["sweeps_fp32"] / 1000.0
        gb.gc_destroy_orbit(h)
    w = oi.workload_uneven(mean_sweeps=mean_sweeps)
    n_list = w.extra["n_starts"]
    side = torch.cuda.Stream()
    opt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=check_every,
                                fp_mode=gb.GC_FP_AUTO, stream=side, use_graph=1, autotune=2)
    ms, conv, upd = 0.0, 0, 0
    with torch.cuda.stream(side):
        for k in range(1 + steps):          # one untimed step: allocations, autotuning
            hs = [gb.gc_create_orbit(o.d, o.L, o.phi, o.orbit_id, n) for o, n in zip(w.orbits, n_list)]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(side)
            gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, opt)
            e1.record(side)
            e1.synchronize()
            sts = [gb.gc_orbit_stats(h) for h in hs]
            for h in hs:
                gb.gc_destroy_orbit(h)
            if k == 0:
                continue
            ms += e0.elapsed_time(e1)
            conv += sum(st["n_converged"] for st in sts)
            upd += sum(st["site_updates_fp32"] + st["site_updates_fp64"] for st in sts)
    return {"orbits": len(w.orbits), "starts_per_step": int(sum(n_list)),
            "shapes": {f"{o.d}D L{o.L}": n for o, n in list(zip(w.orbits, n_list))[::2]},
            "pilot_mean_sweeps": {f"{d_}D L{L_}": round(v, 1) for (d_, L_), v in mean_sweeps.items()},
            "site_updates_per_step": upd / steps,
            "value": conv / (ms / 1e3), "unit": "copies/s",
            "site_updates_per_s": upd / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
            "launch": "one gc_enumerate_batch per step as one CUDA graph, autotuned shapes and sweep-unroll depth"}


# ----------------------------------------------------------------------------
# large lattice: 4D 16^4, beyond shared memory (hyperplane path)
# ----------------------------------------------------------------------------

def large_lattice_leg(gb, torch, fp32_peak, d=4, L=16, n=592, runs=2):
    """One orbit of 4D 16^4 (65 536 sites, von Mises kappa = 1, seed 1), 592
    starts (four per SM) through the mixed path: FP32 hyperplane sweeps, the
    Newton polish, the FP64 cluster sweeps of the starts it leaves, final
    pass, dedup, fast-path region test.  Each run is timed with CUDA events on
    the launch stream around the enumerate call; per-stage times are the
    library's events.  HBM figures count algorithmic bytes: the FP32 sweeps
    move each start's state (8 B/site) in and out once per colour phase and
    read it once per residual check (the links, shared by all starts, stay in
    L2); an inner SOR sweep reads (2d + 1) FP32 coefficients per site and moves
    the correction (4 B/site) in and out once per phase.  The FP32 sweeps'
    time excludes the FP64 head sweeps before them (the library's event
    between the two, ms_starts); their FP32 work is 8d + 11 + 3/check_every
    operations per update, against the FP32 peak the bench measured."""
    V = L ** d
    phi = oi.von_mises_orbit(d, L, 1.0, 1)
    stream = torch.cuda.current_stream()
    opt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=4, fp_mode=gb.GC_FP_AUTO,
                                stream=stream)
    h = gb.gc_create_orbit(d, L, phi, 1)
    gb.gc_enumerate_copies(h, 64, 1.7, 1e-24, opt)            # allocations, first launches
    gb.gc_destroy_orbit(h)
    acc = {}
    ms = 0.0
    for _ in range(runs):
        h = gb.gc_create_orbit(d, L, phi, 1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gb.gc_enumerate_copies(h, n, 1.7, 1e-24, opt)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        st = gb.gc_orbit_stats(h)
        gb.gc_destroy_orbit(h)
        for k, v in st.items():
            acc[k] = acc.get(k, 0) + v
    # the plain FP64 path on a sample of the same orbit (hyperplane sweeps, bit-exact to the oracle)
    plain_n = 148
    popt = gb.gc_options_default(precision=gb.GC_FP64, check_every=1, fp_mode=gb.GC_FP_AUTO, stream=stream)
    h = gb.gc_create_orbit(d, L, phi, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gb.gc_enumerate_copies(h, plain_n, 1.7, 1e-24, popt)
    e1.record(stream)
    e1.synchronize()
    pst = gb.gc_orbit_stats(h)
    gb.gc_destroy_orbit(h)
    plain_value = pst["n_converged"] / (e0.elapsed_time(e1) / 1e3)
    hbm = json.load(open(PEAKS_FILE))["hbm_gbs"] if os.path.exists(PEAKS_FILE) else 6400.0
    relax_bytes = acc["sweeps_fp32"] * V * 32 + acc["sweeps_fp32"] / 4 * V * 8 + acc["n_starts"] * V * 8
    newton_ms = acc["ms_polish"] - acc["ms_polish_redo"]
    inner_bytes = acc["newton_inner_sweeps"] * V * (4 * (2 * d + 1) + 16)
    relax32_ms = acc["ms_relax"] - acc["ms_starts"]
    relax_gbs = relax_bytes / (relax32_ms / 1e3) / 1e9
    relax_tops = acc["sweeps_fp32"] * V * (8 * d + 11 + 3 / 4) / (relax32_ms / 1e3) / 1e12
    inner_gbs = inner_bytes / (newton_ms / 1e3) / 1e9
    return {"workload": f"{d}D {L}^{d} ({V} sites), von Mises kappa=1 seed 1, {n} starts, mixed, check_every 4",
            "runs": runs, "value": acc["n_converged"] / (ms / 1e3), "unit": "copies/s",
            "ms_per_run": ms / runs,
            "stage_ms": {"fp64_head": acc["ms_starts"] / runs, "relax_fp32": relax32_ms / runs,
                         "newton": newton_ms / runs,
                         "fp64_sweeps_and_final": acc["ms_polish_redo"] / runs,
                         "dedup": acc["ms_dedup"] / runs, "fp_test": acc["ms_fptest"] / runs},
            "converged": acc["n_converged"] // runs, "distinct": acc["n_distinct"] // runs,
            "sweeps_fp32_per_start": acc["sweeps_fp32"] / acc["n_starts"],
            "newton_steps_per_start": acc["newton_steps"] / acc["n_starts"],
            "inner_sweeps_per_start": acc["newton_inner_sweeps"] / acc["n_starts"],
            "fp64_fallback_starts": acc["polish_fallbacks"] // runs,
            "plain_fp64": {"starts": plain_n, "value": plain_value, "unit": "copies/s",
                           "sweeps_per_start": pst["sweeps_fp64"] / max(1, pst["n_starts"]),
                           "mixed_over_plain": (acc["n_converged"] / (ms / 1e3)) / plain_value},
            "relax_slab": {"kernel": "relax_dsmem_kernel<4> (8-CTA clusters, state in distributed shared memory)",
                           "bound": "latency", "achieved": relax_tops, "peak": fp32_peak,
                           "unit": "T FP32 lane ops/s", "frac": relax_tops / fp32_peak,
                           "ms": relax32_ms / runs, "traffic": TRAFFIC_SLAB_DSMEM32,
                           "hbm_equivalent": {"achieved": relax_gbs, "peak": hbm, "unit": "GB/s",
                                              "frac": relax_gbs / hbm, "bytes_per_update": 32 + 8 / 4},
                           "note": "latency-bound: each colour phase ends in a cluster barrier and reads "
                                   "neighbour planes from other CTAs' shared memory; the state stays in "
                                   "the cluster's shared memory and only the links come from L2, so DRAM "
                                   "(traffic, ncu) sees the starts' generation and write-back. "
                                   "hbm_equivalent: the state traffic the streamed form would move "
                                   "(34 B per update)"},
            "newton_inner": {"kernel": "slab_newton_kernel<4,·> (both stages)", "bound": "hbm",
                             "achieved": inner_gbs, "peak": hbm, "unit": "GB/s", "frac": inner_gbs / hbm,
                             "traffic": TRAFFIC_SLAB_NEWTON1,
                             "note": "over both Newton launches, the hard starts' cluster stage included; "
                                     "traffic = DRAM bytes of the one-CTA stage (ncu), as its algorithmic "
                                     "inner-sweep bytes predict"}}


# ----------------------------------------------------------------------------
# serving leg: Poisson arrivals at 200 requests/s of mixed-dimension requests
# ----------------------------------------------------------------------------

def serve_leg(gb, n_requests, opt, rate_hz=200.0, workers=16, seed=7):
    """n_requests Poisson arrivals at rate_hz through gc_server_*: latency
    (submission to completion, p50/p99/mean), achieved starts, converged
    copies and site updates per second over the span from the first
    submission to the last completion."""
    import threading
    reqs = oi.request_stream(n_requests, rate_hz=rate_hz, seed=seed)
    srv = gb.gc_server_create(workers, 0, opt)
    results = []
    tickets = []
    failures = []
    lock = threading.Lock()
    done = threading.Event()

    def collector():
        # collect in completion order (a result held until an earlier, longer
        # request finishes would keep its copy table on the device)
        outstanding = []
        seen = 0
        while True:
            with lock:
                outstanding += tickets[seen:]
                seen = len(tickets)
            if not outstanding:
                if done.is_set():
                    with lock:
                        if seen == len(tickets):
                            return
                time.sleep(0.0005)
                continue
            keep = []
            for t in outstanding:
                try:
                    status, latency, orb = gb.gc_server_wait(srv, t[0], 0.0)
                except gb.GribovError as e:
                    if e.code == gb.GC_ETIMEDOUT:
                        keep.append(t)
                        continue
                    raise
                if status != 0:
                    r = t[1]
                    failures.append(f"{r.d}D L={r.L} n={r.n_starts}: {gb.gc_last_error()}")
                conv = upd = 0
                if orb is not None:
                    st = gb.gc_orbit_stats(orb)
                    conv, upd = st["n_converged"], st["site_updates_fp32"] + st["site_updates_fp64"]
                    gb.gc_destroy_orbit(orb)
                results.append((status, latency, conv, upd, time.perf_counter()))
            outstanding = keep
            time.sleep(0.001)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    for r in reqs:
        wait = r.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tk = gb.gc_server_submit(srv, r.d, r.L, r.phi, r.seed, r.n_starts)
        with lock:
            tickets.append((tk, r))
    done.set()
    th.join()
    span = max(x[4] for x in results) - t0
    info = gb.gc_server_state(srv)
    gb.gc_server_destroy(srv)
    lat = np.array([x[1] for x in results])
    starts = sum(r.n_starts for r in reqs)
    return {"requests": n_requests, "rate_hz": rate_hz, "workers": workers,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()),
            "converged_copies_per_s": sum(x[2] for x in results) / span,
            "starts_per_s": starts / span, "site_updates_per_s": sum(x[3] for x in results) / span,
            "offered_starts_per_s": starts / reqs[-1].arrival_s,
            "failed": int(sum(1 for x in results if x[0] != 0)), "failures": failures[:5], "span_s": span,
            "loop_launches": info["loop_launches"], "admitted_on_device": info["admitted"],
            "mix": "dim in {2,3,4}, L from {4,6,8,12,16}/{4,5,6,8}/{3,4,5,6}, "
                   "n_starts log-uniform in [1e3, 1e6], von Mises(1.0) orbits"}


def serving_legs(gb, n_requests, opt):
    """The request stream at 200 requests/s (above the GPU's capacity for this
    mix: latency is mostly queueing), then the same mix at half the
    throughput that run achieved (below capacity: latency is service)."""
    over = serve_leg(gb, n_requests, opt, rate_hz=200.0)
    mean_n = (1e6 - 1e3) / math.log(1e3)                 # log-uniform [1e3, 1e6]
    low = 0.5 * over["starts_per_s"] / mean_n
    below = serve_leg(gb, n_requests, opt, rate_hz=low, seed=8)
    return {"above_capacity": over, "below_capacity": below}


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------

def stats_delta(a, b):
    return {k: b[k] - a[k] for k in b}


def run_ours(args):
    import torch
    import paper_1403_0555_b300 as gb
    from paper_1403_0555_b300.replicas import rank_seed, reduce_timing

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    gb.use_torch_allocator()
    stream = torch.cuda.current_stream()

    w = oi.workload_4d_4to4(args.starts)
    orbits = w.orbits
    d, L = 4, 4
    V = L ** d
    side = torch.cuda.Stream()
    # the first-region test of the workload: FP64 Lanczos for every distinct copy
    opt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=args.check_every,
                                fp_mode=gb.GC_FP_LANCZOS, stream=side, use_graph=1, autotune=args.autotune)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # weak scaling: with N > 1 every rank runs the whole eight-orbit workload
    # shape on orbits of its own seeds (no data-path collective)
    def step_orbits(k):
        if rank == 0:
            return orbits
        return [oi.Orbit(o.name, o.d, o.L, oi.von_mises_orbit(4, 4, oi.kappa_grid_4d()[j], rank_seed(rank, j)),
                         rank_seed(rank, j)) for j, o in enumerate(orbits)]

    def create(orbs):
        return [gb.gc_create_orbit(d, L, o.phi, o.orbit_id, args.starts) for o in orbs]

    n_list = [args.starts] * len(orbits)
    # launch shapes and sweep-unroll depth: tuned once (cached for every later
    # call), recorded in config
    h = gb.gc_create_orbit(d, L, orbits[0].phi, orbits[0].orbit_id)
    tuning = gb.gc_autotune(h, gb.GC_MIXED, mode=args.autotune)
    gb.gc_destroy_orbit(h)
    ce = tuning["check_every"] or args.check_every
    # warm-up: whole steps (allocations cached, autotuning done)
    with torch.cuda.stream(side):
        for k in range(args.warmup):
            hs = create(step_orbits(k))
            gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, opt)
            for h in hs:
                gb.gc_destroy_orbit(h)

    # --- device-resident timed region: K steps, each one graph launch of the
    # eight orbits' whole path.  Each step's orbits are created (link angles
    # uploaded) before its launch; CUDA events on the launch stream bracket the
    # batch call only, so `value` counts the enqueued work with inputs resident.
    with torch.cuda.stream(side):
        clk = ClockSampler(torch.cuda.current_device())
        barrier()
        clk.start()
        ms = 0.0
        stats = []
        n_distinct = None
        for k in range(args.steps):
            hs = create(step_orbits(k))
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(side)
            gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, opt)
            ev1.record(side)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            st_k = [gb.gc_orbit_stats(h) for h in hs]
            stats += st_k
            if n_distinct is None:
                n_distinct = [s_["n_distinct"] for s_ in st_k]
            for h in hs:
                gb.gc_destroy_orbit(h)
        barrier()
        clocks = clk.stop()
    tot = {k: sum(s_[k] for s_ in stats) for k in stats[0]}
    conv = tot["n_converged"]
    ms_max, conv_all = reduce_timing(dist, ms, conv, device="cuda")
    value = conv_all / (ms_max / 1000.0)
    upd = tot["site_updates_fp32"] + tot["site_updates_fp64"]

    # --- end to end through the C ABI with host buffers: link angles up, every
    # distinct copy (angles, F, first start, count, lambda_2, flag) back into
    # pinned host arrays allocated once, before the timed region
    cap = int(max(n_distinct) * 1.25) + 1024

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    def out_set():
        return {"F": pinned((cap,), torch.float64), "theta": pinned((cap, V), torch.float64),
                "first_start": pinned((cap,), torch.int64).view(np.uint64),
                "count": pinned((cap,), torch.int64).view(np.uint64),
                "lambda2": pinned((cap,), torch.float64), "region": pinned((cap,), torch.int32)}

    out_sets = [out_set(), out_set()]
    # Step k + 1 is enqueued (asynchronous batch) before step k's copies are
    # fetched, so the GPU always has the next step queued: each step's fetch
    # waits for that step, orders its copies on the step's stream, and leaves
    # the gathering and the device-to-host copies in flight
    # (gc_fetch_copies_async) beside the next step's kernels; gc_fetch_wait
    # completes them a step later.  Steps rotate over three streams, so that
    # destroying step k - 1's orbits (which synchronises their stream) never
    # waits for the step just enqueued.  Every step still uploads its link
    # angles and reads back all its distinct copies inside the timed region.
    e_streams = [torch.cuda.Stream() for _ in range(3)]
    e_opts = []
    for st_ in e_streams:
        eo = gb.gc_options_default(precision=gb.GC_MIXED, check_every=args.check_every,
                                   fp_mode=gb.GC_FP_LANCZOS, stream=st_, autotune=args.autotune)
        eo.async_ = 1
        e_opts.append(eo)
    acc = {"conv": 0, "h2d": 0, "d2h": 0}

    def e2e_launch(k):
        with torch.cuda.stream(e_streams[k % 3]):
            hs = []
            for o in step_orbits(k):
                phi = np.ascontiguousarray(o.phi)
                hs.append(gb.gc_create_orbit(d, L, phi, o.orbit_id, args.starts))
                acc["h2d"] += phi.nbytes
            gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, e_opts[k % 3])
        return hs

    def e2e_fetch(hs, bufs):
        for h in hs:
            acc["conv"] += gb.gc_orbit_stats(h)["n_converged"]
            try:
                res = gb.gc_fetch_copies(h, V, out=bufs, async_=True)
            except ValueError:          # more copies than the pinned arrays hold
                res = gb.gc_fetch_copies(h, V)
            acc["d2h"] += sum(res[k_].nbytes for k_ in ("F", "theta", "first_start", "count", "lambda2", "region"))

    def e2e_finish(hs):
        for h in hs:
            gb.gc_fetch_wait(h)
            gb.gc_destroy_orbit(h)

    def e2e_steps(nsteps):
        prev, older = e2e_launch(0), None
        for k in range(1, nsteps + 1):
            hs = e2e_launch(k) if k < nsteps else None
            if older is not None:
                e2e_finish(older)
            e2e_fetch(prev, out_sets[(k - 1) % 2])
            older, prev = prev, hs
        e2e_finish(older)

    e2e_steps(3)                        # warm-up of the three streams
    acc = {"conv": 0, "h2d": 0, "d2h": 0}
    barrier()
    t0 = time.perf_counter()
    e2e_steps(args.steps)
    e2e_conv, h2d, d2h = acc["conv"], acc["h2d"], acc["d2h"]
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_conv = reduce_timing(dist, e2e_s, e2e_conv, device="cuda")
    e2e = {"value": e2e_conv / e2e_s, "unit": "copies/s",
           "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
           "pipeline": "asynchronous batches on three streams, step k+1 enqueued before step k's fetch; "
                       "each step's copies ordered on the device after the step, gathered and copied to "
                       "the host (gc_fetch_copies_async) beside the next step's kernels; host wall clock "
                       "over all K steps"}

    # --- the same steps with the FP32 Lanczos screen (GC_FP_AUTO: FP64 only
    # for copies whose FP32 lambda_2 is at most 1e-3), a labelled variant
    sopt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=args.check_every,
                                 fp_mode=gb.GC_FP_AUTO, stream=side, use_graph=1, autotune=args.autotune)
    with torch.cuda.stream(side):
        hs = create(step_orbits(0))
        gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, sopt)      # warm-up step
        for h in hs:
            gb.gc_destroy_orbit(h)
        barrier()
        s_ms, s_conv = 0.0, 0
        for k in range(args.steps):
            hs = create(step_orbits(k))
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(side)
            gb.gc_enumerate_batch(hs, n_list, w.omega, w.eps, sopt)
            ev1.record(side)
            ev1.synchronize()
            s_ms += ev0.elapsed_time(ev1)
            s_conv += sum(gb.gc_orbit_stats(h)["n_converged"] for h in hs)
            for h in hs:
                gb.gc_destroy_orbit(h)
        barrier()
    s_ms_max, s_conv_all = reduce_timing(dist, s_ms, s_conv, device="cuda")
    screen_leg = {"value": s_conv_all / (s_ms_max / 1000.0), "unit": "copies/s",
                  "ms_per_step": s_ms_max / args.steps, "steps": args.steps,
                  "fp_test": "GC_FP_AUTO: FP32 Lanczos screen of every copy, FP64 Lanczos for those with "
                             "FP32 lambda_2 <= 1e-3"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # --- measured throughput of the arithmetic units (the roofline denominators)
    peaks = {"ffma": gb.gc_peak_probe(gb.GC_PEAK_FFMA, stream) / 1e12,
             "ffma2": gb.gc_peak_probe(gb.GC_PEAK_FFMA2, stream) / 1e12,
             "dfma": gb.gc_peak_probe(gb.GC_PEAK_DFMA, stream) / 1e12,
             "rsqrt": gb.gc_peak_probe(gb.GC_PEAK_RSQ, stream) / 1e12,
             "dfma_one_lane_per_warp": gb.gc_peak_probe(gb.GC_PEAK_DFMA_LANE1, stream) / 1e12,
             "unit": "T lane operations/s (packed f32x2 counts two)",
             "how": "gc_peak_probe: 4 CTAs x 256 threads per SM, 8 independent chains per thread, best of 3"}

    # --- plain FP64 path, run the way the headline step runs: the eight
    # orbits as one graph-captured gc_enumerate_batch call with the FP64
    # Lanczos test of every copy, plain_starts starts in all (an equal share
    # per orbit), launch shapes tuned (mode 1, result-neutral), so that
    # mixed_over_plain compares the precisions alone.  A first call of the
    # same size captures the graph and warms the allocator.
    pn = max(1, args.plain_starts // len(orbits))
    with torch.cuda.stream(side):
        h = gb.gc_create_orbit(d, L, orbits[0].phi, orbits[0].orbit_id)
        gb.gc_autotune(h, gb.GC_FP64, mode=1)
        gb.gc_destroy_orbit(h)
        popt = gb.gc_options_default(precision=gb.GC_FP64, check_every=args.check_every,
                                     fp_mode=gb.GC_FP_LANCZOS, stream=side, use_graph=1, autotune=1)
        hs = [gb.gc_create_orbit(d, L, o.phi, o.orbit_id, 2 * pn) for o in orbits]
        gb.gc_enumerate_batch(hs, [pn] * len(hs), w.omega, w.eps, popt)       # warm-up
        s0 = [gb.gc_orbit_stats(h) for h in hs]
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(side)
        gb.gc_enumerate_batch(hs, [pn] * len(hs), w.omega, w.eps, popt)
        p1.record(side)
        barrier()
        pms = p0.elapsed_time(p1)
        ps = [stats_delta(a_, gb.gc_orbit_stats(h)) for a_, h in zip(s0, hs)]
        for h in hs:
            gb.gc_destroy_orbit(h)
    p_conv = sum(x["n_converged"] for x in ps)
    p_upd = sum(x["site_updates_fp64"] for x in ps)
    plain = {"value": p_conv / (pms / 1000.0), "unit": "copies/s",
             "site_updates_per_s": p_upd / (pms / 1000.0),
             "sample": f"{pn} starts of each of the eight orbits, one graph-captured batch, FP64 Lanczos test",
             "mixed_over_plain": value / (p_conv / (pms / 1000.0))}

    # --- roofline of the dominant kernel.  Inside the timed batches the
    # orbits' kernels overlap, so each kernel's own duration is taken from
    # isolated single-orbit passes of the step's eight orbits (2^20 starts
    # each), with CUDA events on the launch stream around every kernel (the
    # library's per-stage events); each kernel's work and time are summed
    # over the eight launches, and the dominant kernel is the one with the
    # most time in the step.
    ropt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=ce,
                                 fp_mode=gb.GC_FP_LANCZOS, stream=stream)
    rs = None
    per_orbit_ms = []
    for o in orbits:
        h = gb.gc_create_orbit(d, L, o.phi, o.orbit_id, args.starts)
        gb.gc_enumerate_copies(h, args.starts, w.omega, w.eps, ropt)
        st = gb.gc_orbit_stats(h)
        gb.gc_destroy_orbit(h)
        per_orbit_ms.append({k: round(st[k], 2) for k in ("ms_starts", "ms_relax", "ms_polish", "ms_dedup",
                                                           "ms_fptest")}
                            | {"copies": st["n_distinct"]})
        rs = st if rs is None else {k: rs[k] + st[k] for k in rs}
    n_launch = len(orbits)
    # FP32 site updates of the bulk sweeps (the rest are polish fallbacks)
    rs_relax_updates = rs["sweeps_fp32"] * V
    # the relax stage holds the start draw (start32_kernel) and the FP32 sweeps
    stage_ms = {"start_draw": rs["ms_starts"], "relax_fp32": rs["ms_relax"] - rs["ms_starts"],
                "polish_fp64": rs["ms_polish"] - rs["ms_polish_redo"],
                "polish_redo": rs["ms_polish_redo"],
                "dedup": rs["ms_dedup"], "fp_test": rs["ms_fptest"]}
    # Per kernel: algorithmic operations over its isolated duration, against
    # the unit's throughput measured by gc_peak_probe on this GPU.
    #  * FP32 sweeps (relax32_sheet_kernel): FP32 pipe ops per site update, 8d
    #    for the staple's 2d complex products, 11 to blend and renormalise, and
    #    3 per site at a check (the residual reuses the update's staple);
    #  * line polish (polish_pairs_kernel): FP32 pipe ops per site, 12 (8d + 2)
    #    + 2 per double-float residual pass, 2d + 3 per inner SOR sweep,
    #    5d + 2d + 2 (weights, 1/D) + 58 (double-float rotation) per Newton
    #    step, 33 to promote, 8d + 11 per fallback FP32 update; its FP64 ops,
    #    the binding unit, 8d + 11 per site of the final pass (8d for the
    #    staple, 3 for the residual, 2 for the functional, 4 for the canonical
    #    copy, 2 to join the double-float halves);
    #  * first-region test (fp_test_pairs_kernel, FP64 Lanczos seeded by an
    #    FP32 Ritz vector): FP64 ops per site, 6d for the weights cos(phi^theta)
    #    (two complex products per link), 2d for the diagonal of M, 3 to
    #    normalise the seed, and per FP64 step 2d + 1 FMAs for M v and 6 more
    #    for the recurrence, alpha, mean, norm and the next vector (2d + 7);
    #    FP32 ops per site and FP32 step, 4d for M v (differences and FMAs)
    #    and 7 for the recurrence in the recording pass, 4d + 4 in the replay
    #    pass that sums the Ritz vector.
    # A packed f32x2 instruction does two lane operations, so the FP32 peak is
    # the larger of the scalar and packed FMA probes.
    fp32_peak = max(peaks["ffma"], peaks["ffma2"])
    fp64_peak = peaks["dfma"]
    fp32_per_update = 8 * d + 11 + 3 / ce
    sec = {k: v / 1e3 for k, v in stage_ms.items()}
    kernels = {}
    a_relax = rs["sweeps_fp32"] * V * fp32_per_update / sec["relax_fp32"] / 1e12
    kernels["relax_fp32"] = {"kernel": "relax32_sheet_kernel<8,1>", "bound": "alu", "achieved": a_relax,
                             "peak": fp32_peak, "unit": "T FP32 lane ops/s", "frac": a_relax / fp32_peak,
                             "ms": stage_ms["relax_fp32"], "launches": n_launch,
                             "traffic": TRAFFIC_RELAX_PER_START * args.starts}
    # The line polish (polish_pairs_kernel) and the CG instance rerunning the
    # starts it hands on (polish_kernel, a few hundred starts per step: a
    # latency tail that runs beside other orbits' kernels inside a batch) are
    # separate entries.  Newton steps, inner sweeps and FP64 passes are
    # counted by both kernels into shared counters and charged to the line
    # polish (the rerun starts add under 1 % to them); the fallback FP32 and
    # FP64 updates are the rerun's alone.
    fp32_pairs = (rs["df_residual_passes"] * V * (12 * (8 * d + 2) + 2)
                  + rs["newton_inner_sweeps"] * V * (2 * d + 3)
                  + rs["newton_steps"] * V * (7 * d + 2 + 58)
                  + rs["n_starts"] * V * 33)
    fp32_redo = (rs["site_updates_fp32"] - rs_relax_updates) * (8 * d + 11)
    fp32_ops = fp32_pairs + fp32_redo
    fp64_pairs = rs["fp64_residual_passes"] * V * (8 * d + 11)
    fp64_redo = rs["site_updates_fp64"] * (8 * d + 20)
    fp64_pol = fp64_pairs + fp64_redo
    t_pairs, t_redo = sec["polish_fp64"], sec["polish_redo"]
    a_pol = fp64_pairs / t_pairs / 1e12
    kernels["polish"] = {"kernel": "polish_pairs_kernel<4,4,12>", "bound": "alu",
                         "achieved": a_pol, "peak": fp64_peak, "unit": "T FP64 lane ops/s", "frac": a_pol / fp64_peak,
                         "fp32_frac": fp32_pairs / t_pairs / 1e12 / fp32_peak,
                         "ms": stage_ms["polish_fp64"], "launches": n_launch,
                         "traffic": TRAFFIC_POLISH_PER_START * args.starts}
    a_redo = fp64_redo / t_redo / 1e12 if t_redo > 0 else 0.0
    kernels["polish_redo"] = {"kernel": "polish_kernel<4,true> (CG instance, the handed-on starts)", "bound": "latency",
                              "achieved": a_redo, "peak": fp64_peak, "unit": "T FP64 lane ops/s",
                              "frac": a_redo / fp64_peak, "starts": rs["polish_redo_starts"],
                              "ms": stage_ms["polish_redo"], "launches": n_launch, "traffic": None,
                              "note": "one warp per start on a few SMs; its time is the slowest start's"}
    steps64 = rs["lanczos_steps_fp64"]
    steps32 = rs["lanczos_steps"] - steps64
    fp64_ops = rs["fp_tests_fp64"] * V * (8 * d + 3) + steps64 * V * (2 * d + 7)
    fp32_fp = steps32 * V * ((4 * d + 7) + (4 * d + 4))
    a_fp = fp64_ops / sec["fp_test"] / 1e12
    kernels["fp_test"] = {"kernel": "fp_test_pairs_kernel<4,4> (FP64 Lanczos from an FP32 Ritz vector)",
                          "bound": "alu", "achieved": a_fp,
                          "peak": fp64_peak, "unit": "T FP64 lane ops/s", "frac": a_fp / fp64_peak,
                          "fp32_frac": fp32_fp / sec["fp_test"] / 1e12 / fp32_peak,
                          "ms": stage_ms["fp_test"], "launches": n_launch,
                          "fp32_steps_per_copy": steps32 / max(1, rs["fp_tests"]),
                          "fp64_steps_per_copy": steps64 / max(1, rs["fp_tests_fp64"]),
                          "traffic": (TRAFFIC_FPTEST_PER_COPY * rs["fp_tests"] / n_launch
                                      if TRAFFIC_FPTEST_PER_COPY else None)}
    # the dominant kernel: the most time over the step's eight orbits
    dom = max(("relax_fp32", "polish", "polish_redo", "fp_test"), key=lambda k_: kernels[k_]["ms"])
    roof = dict(kernels[dom])
    roof["traffic_unit"] = "bytes per launch (DRAM read + write, ncu, scaled from the profiled case)"
    roof["peak_source"] = "measured on this GPU by gc_peak_probe (FFMA/FFMA2/DFMA), bench.py's peaks key"
    roof["ms_per_launch"] = roof["ms"] / n_launch
    roof["stage_ms_isolated"] = stage_ms
    roof["stage_ms_per_orbit"] = per_orbit_ms
    roof["polish_redo_starts"] = rs["polish_redo_starts"]
    roof["launch_starts"] = args.starts
    roof["isolated_passes"] = f"{n_launch} orbits x {args.starts} starts, one at a time; ms summed"
    roof["kernels"] = kernels
    # The step's algorithmic work charged at each unit's measured peak: the
    # kernels fill the SMs one after another (a batch overlaps only their
    # tails), so FP32 and FP64 time add; frac_serial compares that sum with
    # the measured step, frac_overlap the larger unit alone.  Dedup counts
    # its FP64 differences (2 per site of one comparison per converged start).
    fp32_all = rs["sweeps_fp32"] * V * fp32_per_update + fp32_ops + fp32_fp
    fp64_all = fp64_pol + fp64_ops + 2.0 * V * rs["n_converged"]
    t32 = fp32_all / (fp32_peak * 1e12) * 1e3
    t64 = fp64_all / (fp64_peak * 1e12) * 1e3
    step_ms = ms_max / args.steps
    path_roof = {"fp32_ms_at_peak": t32, "fp64_ms_at_peak": t64, "step_ms": step_ms,
                 "frac_serial": (t32 + t64) / step_ms, "frac_overlap": max(t32, t64) / step_ms,
                 "peaks": "measured FFMA2 and DFMA (peaks key)",
                 "work": "FP32 sweeps, polish (FP32 and FP64), first-region test (FP32 and FP64), dedup "
                         "differences; algorithmic operation counts as in roofline.kernels"}

    uneven = uneven_leg(gb, torch, args.check_every) if args.uneven else None
    large = large_lattice_leg(gb, torch, fp32_peak) if args.large else None

    serving = None
    if args.serve_requests > 0:
        sopt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=args.check_every,
                                     fp_mode=gb.GC_FP_AUTO)
        serving = serving_legs(gb, args.serve_requests, sopt)

    cpu_configs = oracle_configs() if args.cpu_configs else None

    cpu = None
    if not args.no_cpu_baseline:
        c, dt, threads = oracle_sample(orbits[0], args.cpu_starts)
        cpu = {"value": c / dt, "unit": "copies/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_starts} starts of the kappa=0.5 orbit, full oracle pipeline "
                         f"(FP64 relaxation, dense eigensolve per distinct copy), {dt:.1f} s"}

    out = {
        "metric": "converged_copies_per_s", "value": value, "unit": "copies/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "starts_per_step": len(orbits) * args.starts,
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "4d_L4_vonmises_x8", "lattice": "4^4", "orbits": 8,
                   "starts_per_orbit": args.starts, "omega": 1.7, "eps32": 1e-10, "eps": 1e-24,
                   "check_every": ce, "precision": "fp32 sweeps + fp64 polish",
                   "fp_test": "FP64 Lanczos for every distinct copy (GC_FP_LANCZOS)", "parallelism": f"weak x{world}", "launch": "one CUDA graph per step (8 orbits, 16 streams)",
                   "timed": "device events around each step's batch launch; orbit creation outside",
                   "tuning": tuning,
                   "l2": "working set > L2 (1 GiB staging per batch + copy pool)"},
        "site_updates_per_s": upd / (ms_max / 1000.0),
        "site_updates_fp32": tot["site_updates_fp32"], "site_updates_fp64": tot["site_updates_fp64"],
        "distinct_copies_per_orbit": n_distinct,
        "plain_fp64": plain,
        "batch_uneven": uneven,
        "large_lattice": large,
        "serving": serving,
        "roofline": roof, "path_roofline": path_roof,
        "peaks": peaks,
        "fp32_screen": screen_leg,
        "cpu_baseline": cpu,
        "cpu_baseline_configs": cpu_configs,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(tot["kernel_launches"]),
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
