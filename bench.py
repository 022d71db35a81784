#!/usr/bin/env python
"""Benchmark of the fused RD3Q81 stream-collide step (arXiv 2409.05114) on GB300.

One "step" = one lattice Boltzmann time step over the whole grid (pull streaming of all 81
populations on both sublattices, moments, temperature, App. B series equilibrium, BGK),
i.e. one launch of the fused kernel for a periodic case.  The headline workload is the
compressible Taylor-Green vortex at 512^3 (2 x 512^3 = 268M sites) with FP32 populations,
the point at which the HBM-roofline target is stated; TGV 128^3 and the FP64 / FP16 / BF16
storage variants are reported beside it.  Inputs live in HBM before the timed region; one
step moves 2 x 81 x 268M x 4 B = 174 GB, far above the 129 MB L2, so no L2 flush is needed.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
Multi-GPU: the method has no exchange step on this path (independent replicas), so N ranks
each advance their own replica ("scaling": "weak") with a barrier and max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM-roofline fraction, FP32/FP16 vs FP64 at stated error; served p50/p99"
Q = 81
BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=512, help="TGV grid edge of the headline workload")
    p.add_argument("--storage", default="f32", choices=sorted(BYTES))
    p.add_argument("--equilibrium", default="series", choices=["series", "series_exact_w", "entropic"],
                   help="for --quick runs: the equilibrium of the timed case")
    p.add_argument("--streaming", default="pingpong", choices=["pingpong", "aa"],
                   help="for --quick runs: two buffers, or one buffer updated in place (AA)")
    p.add_argument("--collision", default="bgk", choices=["bgk", "entropic"],
                   help="for --quick runs: BGK (alpha = 2) or the entropic alpha (needs --equilibrium entropic)")
    p.add_argument("--quick", action="store_true", help="headline only (no variants, e2e, CPU baseline)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-only", type=int, default=0, metavar="K",
                   help="time only the end-to-end path (K steps at --n, --storage) and print it (for profiling)")
    p.add_argument("--served-only", type=int, default=0, metavar="N",
                   help="run only the served mixed batch with N requests (no FP64 comparison)")
    return p.parse_args()


# ----------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_index_for_smi(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local_rank].strip()
    return str(local_rank)


KERNEL_SOURCES = ("stream_collide.cuh", "stream_collide_pair.cuh", "device_common.cuh", "lbm_internal.h", "rd3q81.h",
                  "sc_f32.cu", "sc_f16.cu", "sc_bf16.cu")


def kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2409_05114_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(storage: str, sites: int, eq: str = "series", collision: str = "bgk", streaming: str = "pingpong"):
    """DRAM bytes (read + write) of one fused-kernel launch, from the committed ncu record
    (bytes per site measured on a smaller grid, scaled by the sites; keyed by storage, plus
    "_entropic" for the exact-equilibrium kernel, "_elbm" for it with the entropic alpha and
    "_exactw" for the series equilibrium with exact temperature weights, then "_aa" for in-place
    streaming);
    None if the record is missing or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != kernel_source_sha():
        return None
    suffix = ("_elbm" if collision == "entropic" else "_entropic" if eq == "entropic"
              else "_exactw" if eq == "series_exact_w" else "") + ("_aa" if streaming == "aa" else "")
    k = rec.get("kernels", {}).get(storage + suffix)
    return None if k is None else int(round(k["dram_bytes_per_site"] * sites))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------

def tgv_fields_device(n: int, mach: float = 0.5):
    """TGV initial fields of workloads.taylor_green, generated on the device (same formulas)
    so that the 512^3 inputs need no host round trip."""
    import torch
    from paper_2409_05114_gb300 import workloads as W
    dev = torch.device("cuda")
    a = torch.arange(n, dtype=torch.float64, device=dev)
    k = 2.0 * math.pi / n
    U0 = mach * W.CS
    rho = torch.ones((2, n, n, n), dtype=torch.float64, device=dev)
    u = torch.empty((3, 2, n, n, n), dtype=torch.float64, device=dev)
    theta = torch.empty((2, n, n, n), dtype=torch.float64, device=dev)
    for s in (0, 1):
        X = (k * (a + 0.5 * s)).view(1, 1, n)
        Y = (k * (a + 0.5 * s)).view(1, n, 1)
        Z = (k * (a + 0.5 * s)).view(n, 1, 1)
        u[0, s] = U0 * torch.sin(X) * torch.cos(Y) * torch.cos(Z)
        u[1, s] = -U0 * torch.cos(X) * torch.sin(Y) * torch.cos(Z)
        u[2, s] = 0.0
        theta[s] = W.THETA0 + U0 ** 2 / 16.0 * (torch.cos(2 * X) + torch.cos(2 * Y)) * (torch.cos(2 * Z) + 2.0)
    return rho.reshape(-1), u.reshape(-1), theta.reshape(-1)


def time_steps(B, ctx, stream, steps: int, warmup: int, world: int, sampler=None):
    import torch
    B.lbm_step(ctx, warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    launches0 = B.lbm_launch_count(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.lbm_step(ctx, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    torch.cuda.synchronize()
    B.lbm_sync(ctx)
    ms = e0.elapsed_time(e1)
    return ms, B.lbm_launch_count(ctx) - launches0, clocks


def run_case(B, n: int, storage: str, steps: int, warmup: int, world: int, fp64_moments=False, sampler=None,
             eq="series", collision="bgk", streaming="pingpong"):
    """Creates a TGV n^3 context, times `steps` steps; returns a dict of measurements."""
    import torch
    from paper_2409_05114_gb300 import workloads as W
    stream = torch.cuda.Stream()
    cfg = B.make_config(n, n, n, 0.51 - 0.5, storage, fp64_moments=fp64_moments, stream=stream, equilibrium=eq,
                        collision=collision, streaming=streaming)
    ctx = B.lbm_create(cfg)
    try:
        rho, u, th = tgv_fields_device(n)
        torch.cuda.synchronize()
        B.lbm_init(ctx, rho, u, th)
        torch.cuda.synchronize()
        del rho, u, th
        ms, launches, clocks = time_steps(B, ctx, stream, steps, warmup, world, sampler)
    finally:
        B.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    ms = max_over_ranks(ms, world)
    sites = 2 * n ** 3
    per_step_s = ms / 1e3 / steps
    return {"sites": sites, "ms_per_step": ms / steps, "mlups": sites / per_step_s / 1e6,
            "bytes_per_site": 2 * Q * BYTES[storage], "launches": launches, "clocks": clocks,
            "gbs": 2 * Q * BYTES[storage] * sites / per_step_s / 1e9}


def run_e2e(B, n: int, storage: str, steps: int):
    """End to end through the C-ABI with host buffers.  Per step, one lbm_advance_fields call:
    equilibrium init from pinned host fields (H2D), one step, moments into pinned host arrays
    (D2H), the copies staged slab by slab and overlapped with the kernels.  The same work as
    three separate calls (lbm_init + lbm_step(1) + lbm_moments) is timed beside it."""
    import torch
    sites = 2 * n ** 3
    rho_d, u_d, th_d = tgv_fields_device(n)
    pin = lambda t: t.cpu().pin_memory()
    rho, u, th = pin(rho_d), pin(u_d), pin(th_d)
    del rho_d, u_d, th_d
    torch.cuda.empty_cache()
    orho = torch.empty(sites, dtype=torch.float64).pin_memory()
    ou = torch.empty(3 * sites, dtype=torch.float64).pin_memory()
    oth = torch.empty(sites, dtype=torch.float64).pin_memory()
    npv = lambda t: t.numpy()
    cfg = B.make_config(n, n, n, 0.01, storage, stream=torch.cuda.Stream())
    ctx = B.lbm_create(cfg)

    def fused():
        B.lbm_advance_fields(ctx, npv(rho), npv(u), npv(th), 1, npv(orho), npv(ou), npv(oth))

    def separate():
        B.lbm_init(ctx, npv(rho), npv(u), npv(th))
        B.lbm_step(ctx, 1)
        B.lbm_moments(ctx, npv(orho), npv(ou), npv(oth))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps

    try:
        dt = timed(fused)
        dt_sep = timed(separate)
    finally:
        B.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    return {"value": sites / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 5 * 8 * sites,
            "d2h_bytes_per_step": 5 * 8 * sites, "ms_per_step": dt * 1e3,
            "host_link_gbs": 2 * 5 * 8 * sites / dt / 1e9,
            "separate_calls": {"value": sites / dt_sep / 1e6, "ms_per_step": dt_sep * 1e3},
            "note": f"TGV {n}^3 {storage}: lbm_advance_fields(pinned host fields, 1 step, pinned host fields); "
                    "separate_calls = lbm_init + lbm_step(1) + lbm_moments on the same buffers"}


SERVED_BUDGET_GB = 32.0


def fp64_rate(B, wl, tau: float, eq: str, steps: int = 3):
    """MLUPS of per-case plain FP64 launches (lbm_step on an FP64 context, the same equilibrium)
    for one case shape: one warm-up step, then `steps` timed with CUDA events."""
    import torch
    stream = torch.cuda.Stream()
    ctx = B.lbm_create(B.make_config(wl.nx, wl.ny, wl.nz, tau, "f64", wl.faces, equilibrium=eq, stream=stream))
    try:
        B.lbm_init(ctx, np_flat(wl.rho), np_flat(wl.u), np_flat(wl.theta))
        B.lbm_step(ctx, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.lbm_step(ctx, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        B.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    return wl.sites * steps / (ms / 1e3) / 1e6


def np_flat(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def run_served(B, n_requests: int = 128, seed: int = 5114, compare_fp64: bool = True,
               budget_gb: float = SERVED_BUDGET_GB):
    """Served mixed batch (continuous batching, lbm_server_*): seeded Poisson arrivals of Sod-type
    shock tubes, Taylor-Green vortices at Ma 0.3-1.0 and Mach-2 blob flows (FP32 / FP16-offset
    storage, exact entropic equilibrium), each submitted at its arrival time to a server whose
    HBM budget the offered load exceeds, so that admission by footprint decides what is
    resident.  Reports time-to-solution p50/p99, aggregate MLUPS, the mean and peak resident
    fraction of the budget, and the per-case plain FP64 rate of the same list (each request's
    steps at the FP64 rate measured for its case shape, summed as if run one after another)."""
    import numpy as np
    import torch
    from paper_2409_05114_gb300 import workloads as W
    reqs = W.served_mix(n_requests, seed=seed)
    host = {}
    for r in reqs:
        if id(r.workload) not in host:
            host[id(r.workload)] = (np_flat(r.workload.rho), np_flat(r.workload.u), np_flat(r.workload.theta))
    budget = int(budget_gb * 1e9)
    srv = B.lbm_server_create(budget, 256)
    lat, status = [], []
    try:
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = t0 + r.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            wl = r.workload
            cfg = B.make_config(wl.nx, wl.ny, wl.nz, r.tau, r.storage, wl.faces, equilibrium=r.equilibrium)
            tickets.append(B.lbm_submit(srv, cfg, *host[id(wl)], r.nsteps))
        for t in tickets:
            if B.lbm_wait(srv, t, 1800.0) != B.LBM_OK:
                raise RuntimeError("served request did not finish")
            st, l = B.lbm_poll(srv, t)
            lat.append(l)
            status.append(st)
        wall = time.perf_counter() - t0
        stats = B.lbm_server_get_stats(srv)
    finally:
        B.lbm_server_destroy(srv)
    work_ok = sum(r.workload.sites * r.nsteps for r, st in zip(reqs, status) if st == B.LBM_OK)
    lat_s = sorted(lat)
    pct = lambda q: lat_s[min(len(lat_s) - 1, int(round(q * (len(lat_s) - 1))))]
    fams = {}
    for r in reqs:
        fams[r.family] = fams.get(r.family, 0) + 1
    out = {"requests": len(reqs), "completed_ok": sum(1 for x in status if x == B.LBM_OK),
           "unstable": sum(1 for x in status if x == B.LBM_EUNSTABLE),
           "p50_s": round(pct(0.5), 3), "p99_s": round(pct(0.99), 3), "max_s": round(lat_s[-1], 3),
           "aggregate_mlups": round(work_ok / wall / 1e6, 1), "wall_s": round(wall, 2), "site_updates": work_ok,
           "hbm_budget_gb": budget_gb,
           "mean_resident_frac": round(stats["resident_byte_seconds"] / max(stats["busy_seconds"], 1e-9) / budget, 3),
           "peak_resident_frac": round(stats["peak_resident_bytes"] / budget, 3),
           "offered_footprint_gb": round(sum(2 * 81 * r.workload.sites * (4 if r.storage == "f32" else 2)
                                             for r in reqs) / 1e9, 1),
           "ticks": stats["ticks"], "graph_launches": stats["graph_launches"],
           "families": fams, "storage": "f32/f16-offset (even odds)", "equilibrium": "exact entropic (Sec. III), BGK",
           "arrivals": f"Poisson, seed {seed}, mean {1e3 * 0.03:.0f} ms (all arrive within "
                       f"{reqs[-1].arrival_s:.1f} s: the GPU stays saturated)",
           "mix": "Sod tubes 256-2048x4x4 (rho 1|0.125, theta 1|0.8, tau_lb 0.6); TGV 32^3-192^3 Ma 0.3-1.0 "
                  "(Re 400, tau_lb >= 0.55); Mach-2 blobs 256x256x4-1024x256x4 (tau_lb 0.55); 200-2000 steps"}
    if not compare_fp64:
        return out
    rates, t_fp64 = {}, 0.0
    for r in reqs:
        key = (r.workload.name, r.tau)
        if key not in rates:
            rates[key] = fp64_rate(B, r.workload, r.tau, r.equilibrium)
        t_fp64 += r.workload.sites * r.nsteps / (rates[key] * 1e6)
    work_all = sum(r.workload.sites * r.nsteps for r in reqs)
    out.update({"fp64_per_case_mlups": round(work_all / t_fp64 / 1e6, 1), "fp64_per_case_s": round(t_fp64, 1),
                "speedup_vs_fp64_per_case": round((work_ok / wall) / (work_all / t_fp64), 2),
                "fp64_baseline": "per-case FP64 lbm_step, same equilibrium; each shape's rate timed over 3 steps "
                                 "(CUDA events), each request's steps at that rate, summed"})
    return out


def cpu_baseline(n: int = 128, steps: int = 1):
    """Times the FP64 oracle (as it stands) in a single-threaded subprocess: `steps` full
    oracle steps of the TGV n^3 workload."""
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W
wl = W.taylor_green({n})
f = O.init(wl.rho, wl.u, wl.theta)
t0 = time.perf_counter()
for _ in range({steps}):
    f = O.step(f, wl.paper_tau('lb'))
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "sites": wl.sites, "steps": {steps}}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if res.returncode != 0:
        return {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle", "error": res.stderr[-300:]}
    d = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": d["sites"] * d["steps"] / d["seconds"] / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} full FP64 oracle step(s) of the TGV {n}^3 workload ({d['sites']} sites), "
                      f"numpy single thread, {d['seconds']:.1f} s"}


def ours(args):
    import torch
    rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2409_05114_gb300 import binding as B
    if args.e2e_only:
        print(json.dumps({"e2e": run_e2e(B, args.n, args.storage, args.e2e_only)}), flush=True)
        return
    if args.served_only:
        print(json.dumps({"served": run_served(B, args.served_only)}), flush=True)
        return

    peak, peak_kind = measured_peaks()
    sampler = ClockSampler(gpu_index_for_smi(local))
    head = run_case(B, args.n, args.storage, args.steps, args.warmup, world, sampler=sampler, eq=args.equilibrium,
                    collision=args.collision, streaming=args.streaming)
    value = head["mlups"] * world
    achieved = head["gbs"]
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"f32": "f32", "f64": "f64", "f16": "f16-offset",
                                                          "bf16": "bf16-offset"}[args.storage],
        "data": "synthetic (compressible Taylor-Green vortex, Ma 0.5)",
        "config": {"workload": f"taylor_green_{args.n}^3", "sites": head["sites"], "storage": args.storage,
                   "equilibrium": args.equilibrium, "collision": args.collision,
                   "streaming": "pull, ping-pong" if args.streaming == "pingpong" else "AA (one buffer, in place)",
                   "tau_lb": 0.51, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (one step moves %.0f GB)" % (head["bytes_per_site"] * head["sites"] / 1e9)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": ncu_traffic(args.storage, head["sites"], args.equilibrium, args.collision,
                                                                 args.streaming),
                     "peak_source": f"{peak_kind} hbm_gbs (STREAM-style copy)",
                     "bytes_per_site": head["bytes_per_site"]},
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
    }
    if not args.quick and rank == 0:
        variants = {}
        for name, n, st, mom, eq, col, strm in (("tgv128_f32", 128, "f32", False, "series", "bgk", "pingpong"),
                                          ("tgv128_f64", 128, "f64", False, "series", "bgk", "pingpong"),
                                          ("tgv512_f16", 512, "f16", False, "series", "bgk", "pingpong"),
                                          ("tgv512_bf16", 512, "bf16", False, "series", "bgk", "pingpong"),
                                          ("tgv512_f32_fp64moments", 512, "f32", True, "series", "bgk", "pingpong"),
                                          ("tgv512_f32_exactw", 512, "f32", False, "series_exact_w", "bgk", "pingpong"),
                                          ("tgv512_f32_entropic", 512, "f32", False, "entropic", "bgk", "pingpong"),
                                          ("tgv512_f16_entropic", 512, "f16", False, "entropic", "bgk", "pingpong"),
                                          ("tgv128_f64_entropic", 128, "f64", False, "entropic", "bgk", "pingpong"),
                                          ("tgv512_f32_elbm", 512, "f32", False, "entropic", "entropic", "pingpong"),
                                          ("tgv512_f16_elbm", 512, "f16", False, "entropic", "entropic", "pingpong"),
                                          ("tgv512_f32_aa", 512, "f32", False, "series", "bgk", "aa"),
                                          ("tgv512_f16_aa", 512, "f16", False, "series", "bgk", "aa"),
                                          ("tgv512_f64_aa", 512, "f64", False, "series", "bgk", "aa")):
            if n == args.n and st == args.storage and not mom and eq == "series" and strm == args.streaming:
                continue
            r = run_case(B, n, st, max(5, args.steps // 2), 3, 1, fp64_moments=mom, eq=eq, collision=col,
                         streaming=strm)
            variants[name] = {"mlups": round(r["mlups"], 1), "gbs": round(r["gbs"], 1),
                              "roofline_frac": round(r["gbs"] / peak, 4), "ms_per_step": round(r["ms_per_step"], 4)}
        line["variants"] = variants
        line["e2e"] = run_e2e(B, args.n, args.storage, 3)
        try:
            line["served"] = run_served(B)
        except Exception as exc:  # report, do not lose the rest of the line
            line["served"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.quick and not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------------------

def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from oracle import rd3q81 as O
    from paper_2409_05114_gb300 import workloads as W
    n = 32
    wl = W.taylor_green(n)
    tau = wl.paper_tau("lb")
    f = O.init(wl.rho, wl.u, wl.theta)
    for _ in range(args.warmup):
        f = O.step(f, tau)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(f, tau)
    dt = time.perf_counter() - t0
    value = wl.sites * args.steps / dt / 1e6
    sample = f"each step = one full FP64 oracle step of TGV {n}^3 ({wl.sites} sites), same init recipe as the headline"
    line = {"metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"taylor_green_{args.n}^3 (oracle on a {n}^3 sample)", "sites": wl.sites},
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
