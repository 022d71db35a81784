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
    p.add_argument("--fp64-moments", action="store_true",
                   help="for --quick runs: FP64-quality moment sums and temperature recovery")
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


def ncu_traffic(storage: str, sites: int, eq: str = "series", collision: str = "bgk", streaming: str = "pingpong",
                fp64_moments: bool = False):
    """DRAM bytes (read + write) of one fused-kernel launch, from the committed ncu record
    (bytes per site measured on a smaller grid, scaled by the sites; keyed by storage, plus
    "_entropic" for the exact-equilibrium kernel, "_elbm" for it with the entropic alpha and
    "_exactw" for the series equilibrium with exact temperature weights, then "_fp64m" for
    FP64-quality moments and "_aa" for in-place streaming);
    None if the record is missing or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != kernel_source_sha():
        return None
    suffix = ("_elbm" if collision == "entropic" else "_entropic" if eq == "entropic"
              else "_exactw" if eq == "series_exact_w" else "") + ("_fp64m" if fp64_moments else "") + \
        ("_aa" if streaming == "aa" else "")
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


def run_workload(B, wl, tau: float, storage: str, steps: int, warmup: int, fp64_moments=False, eq="series",
                 collision="bgk", total_steps: int = 0):
    """Times `steps` steps of workload wl (initial fields from the host) after `warmup`, then runs
    on (untimed) to `total_steps` if that is larger; returns MLUPS and whether the whole run stayed
    stable (no site flagged rho <= 0, theta <= 0 or non-finite)."""
    import torch
    stream = torch.cuda.Stream()
    cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, fp64_moments=fp64_moments, stream=stream,
                        equilibrium=eq, collision=collision)
    ctx = B.lbm_create(cfg)
    stable = True
    try:
        B.lbm_init(ctx, np_flat(wl.rho), np_flat(wl.u), np_flat(wl.theta))
        torch.cuda.synchronize()
        B.lbm_step(ctx, warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.lbm_step(ctx, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        try:
            B.lbm_sync(ctx)
            rest = total_steps - warmup - steps
            while rest > 0 and stable:
                B.lbm_step(ctx, min(rest, 100))
                rest -= 100
                B.lbm_sync(ctx)
        except B.LbmUnstable:
            stable = False
    finally:
        B.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    per_step = ms / 1e3 / steps
    return {"mlups": wl.sites / per_step / 1e6, "gbs": 2 * Q * BYTES[storage] * wl.sites / per_step / 1e9,
            "ms_per_step": ms / steps, "stable": stable, "sites": wl.sites}


def workload_variants(B, peak: float):
    """The shock-tube, decaying-turbulence and Mach-2 workloads at their stated sizes."""
    from paper_2409_05114_gb300 import workloads as W
    out = {}
    sod = W.sod(512, 4, 4)
    r = run_workload(B, sod, sod.paper_tau("lb"), "f64", 200, 3, eq="entropic")
    out["sod512x4x4_f64_entropic"] = r
    hit = W.hit(256)
    for st in ("f32", "f16", "bf16"):
        # at tau_lb 0.505 the entropic alpha (Eq. (delH)) keeps FP32 stable for the 500 steps; the
        # series form (the one with FP64-quality moment sums) fails within a hundred
        out[f"hit256_{st}_entropic_alpha_500steps"] = run_workload(B, hit, hit.paper_tau("lb"), st, 10, 3,
                                                                   eq="entropic", collision="entropic",
                                                                   total_steps=500)
        out[f"hit256_{st}_series_fp64moments"] = run_workload(B, hit, hit.paper_tau("lb"), st, 10, 3,
                                                              fp64_moments=True, total_steps=100)
    del hit
    blob = W.mach2_blob()
    for st in ("f32", "f16"):
        out[f"mach2blob1024x256x4_{st}_entropic_2000steps"] = run_workload(B, blob, blob.paper_tau("lb"), st, 2000, 3,
                                                                           eq="entropic")
    for k, v in out.items():
        v["roofline_frac"] = round(v["gbs"] / peak, 4)
        v["mlups"] = round(v["mlups"], 1)
        v["gbs"] = round(v["gbs"], 1)
        v["ms_per_step"] = round(v["ms_per_step"], 4)
    return out


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


def run_served(B, n_requests: int = 100, seed: int = 5114, compare_fp64: bool = True,
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
           "backlog_resident_frac": round(stats["backlog_byte_seconds"] / max(stats["backlog_seconds"], 1e-9) / budget, 3),
           "backlog_share_of_busy": round(stats["backlog_seconds"] / max(stats["busy_seconds"], 1e-9), 3),
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


# ----------------------------------------------------------------------------------------
# the oracle leg: CPU baseline and the FP64-oracle errors (the only part that runs oracle/)
# ----------------------------------------------------------------------------------------

# Bounded oracle samples of the four workloads (sites x steps of one timed sample).
ORACLE_SAMPLES = {
    "sod512x4x4": ("W.sod(512, 4, 4)", "series", 24),
    "taylor_green32": ("W.taylor_green(32)", "series", 6),
    "hit32": ("W.hit(32)", "series", 6),
    "mach2blob128x32x4": ("W.mach2_blob(128, 32, 4)", "entropic", 2),
}

_ORACLE_SAMPLE_CODE = """
import sys, time, json
sys.path.insert(0, {root!r})
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W
wl = {make}
tau = wl.paper_tau('lb')
f = O.init(wl.rho, wl.u, wl.theta, eq={eq!r})
t0 = time.perf_counter()
for _ in range({steps}):
    f = O.step(f, tau, wl.oracle_bc_x(), eq={eq!r})
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "sites": wl.sites, "steps": {steps}}}))
"""


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_rate(name: str, procs: int = 1):
    """Runs the bounded oracle sample of workload `name` in `procs` concurrent single-threaded
    processes (fresh interpreters, independent samples); returns (summed MLUPS, seconds of one)."""
    make, eq, steps = ORACLE_SAMPLES[name]
    code = _ORACLE_SAMPLE_CODE.format(root=ROOT, make=make, eq=eq, steps=steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    rates, secs = [], []
    for p_ in ps:
        out, err = p_.communicate(timeout=1800)
        if p_.returncode != 0:
            raise RuntimeError(err[-300:])
        d = json.loads(out.strip().splitlines()[-1])
        rates.append(d["sites"] * d["steps"] / d["seconds"] / 1e6)
        secs.append(d["seconds"])
    return sum(rates), statistics.median(secs), d["sites"] * d["steps"]


def cpu_baseline():
    """The FP64 oracle as it stands, on the host cores: each workload's bounded sample in one
    single-threaded process, then in one process per core (independent samples, rates summed).
    The headline value is the all-core Taylor-Green figure."""
    cores = len(os.sched_getaffinity(0))
    per = {}
    for name in ORACLE_SAMPLES:
        r1, s1, work = oracle_sample_rate(name, 1)
        rn, sn, _ = oracle_sample_rate(name, cores)
        per[name] = {"mlups_1core": round(r1, 4), "mlups_all_cores": round(rn, 3), "seconds_per_sample_1core": round(s1, 2),
                     "site_updates_per_sample": work, "equilibrium": ORACLE_SAMPLES[name][1]}
    head = per["taylor_green32"]
    return {"value": head["mlups_all_cores"], "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "value_1core": head["mlups_1core"], "workloads": per,
            "sample": f"FP64 numpy oracle, one single-threaded process per core ({cores}) on independent samples, "
                      f"rates summed; each sample = the listed steps of one workload (TGV 32^3: "
                      f"{ORACLE_SAMPLES['taylor_green32'][2]} steps)"}


_ORACLE_FIELDS_CODE = """
import sys
sys.path.insert(0, {root!r})
import numpy as np
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W
wl = {make}
f = O.init(wl.rho, wl.u, wl.theta, eq={eq!r})
f = O.run(f, {tau!r}, {steps}, wl.oracle_bc_x(), eq={eq!r}, collision={col!r})
r, u, t = O.fields(f)
np.savez({path!r}, rho=r, u=u, theta=t)
"""

# Parity-size cases of each workload: (name, workload expression, paper tau expression, steps,
# equilibrium, collision, fp64_moments).
ORACLE_CASES = [
    ("sod128x4x4_entropic_40steps", "W.sod(128, 4, 4)", "W.paper_tau(0.6, 'lb')", 40, "entropic", "bgk", False),
    ("taylor_green32_series_100steps", "W.taylor_green(32)", "W.paper_tau(0.51, 'lb')", 100, "series", "bgk", False),
    ("hit16_series_fp64moments_20steps", "W.hit(16)", "W.paper_tau(0.505, 'lb')", 20, "series", "bgk", True),
    ("hit16_entropic_alpha_20steps", "W.hit(16)", "W.paper_tau(0.505, 'lb')", 20, "entropic", "entropic", False),
    ("mach2blob128x32x4_entropic_10steps", "W.mach2_blob(128, 32, 4)", "W.paper_tau(0.55, 'lb')", 10, "entropic", "bgk",
     False),
]
# The serving families at parity size (served FP32 and FP16, exact entropic equilibrium, BGK).
SERVED_CASES = [
    ("shock_tube64x4x4_20steps", "W.sod(64, 4, 4)", "W.paper_tau(0.6, 'lb')", 20),
    ("taylor_green16_ma1_20steps", "W.taylor_green(16, mach=1.0)", "W.tgv_served_tau(16, 1.0)", 20),
    ("mach2blob32x16x4_10steps", "W.mach2_blob(32, 16, 4)", "W.paper_tau(0.55, 'lb')", 10),
]


def oracle_errors(B):
    """Max relative errors of the library's fields against the FP64 oracle (rho and theta pointwise,
    u relative to max |u|) at parity sizes of each workload, for every storage precision, and of
    the served path (the serving families, through lbm_server_*).  The oracle references run in
    parallel single-threaded processes (no GPU) while the library's runs go on the GPU."""
    import numpy as np
    from paper_2409_05114_gb300 import workloads as W
    tmp = tempfile.mkdtemp(prefix="oracle_ref_")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    jobs = {}
    specs = [(n, mk, tau, st, eq, col) for n, mk, tau, st, eq, col, _ in ORACLE_CASES] + \
            [(n, mk, tau, st, "entropic", "bgk") for n, mk, tau, st in SERVED_CASES]
    for name, make, tau_expr, steps, eq, col in specs:
        path = os.path.join(tmp, name + ".npz")
        code = _ORACLE_FIELDS_CODE.format(root=ROOT, make=make, eq=eq, col=col, steps=steps, path=path,
                                          tau=float(eval(tau_expr, {"W": W})))
        jobs[name] = (subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.DEVNULL,
                                       stderr=subprocess.PIPE, text=True, env=env), path)

    def errs(ref, got):
        (r0, u0, t0), (r1, u1, t1) = ref, got
        umax = float(np.max(np.abs(u0))) or 1.0
        return {"rho": float(np.max(np.abs(r1 - r0) / np.abs(r0))), "u": float(np.max(np.abs(u1 - u0)) / umax),
                "theta": float(np.max(np.abs(t1 - t0) / np.abs(t0)))}

    def lib(wl, tau, storage, steps, eq, col, fp64_moments):
        cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, storage, wl.faces, fp64_moments=fp64_moments, equilibrium=eq,
                            collision=col)
        ctx = B.lbm_create(cfg)
        try:
            B.lbm_init(ctx, np_flat(wl.rho), np_flat(wl.u), np_flat(wl.theta))
            B.lbm_step(ctx, steps)
            S = wl.sites
            r, u, t = np.zeros(S), np.zeros(3 * S), np.zeros(S)
            B.lbm_moments(ctx, r, u, t)
        except B.LbmUnstable:
            return None
        finally:
            B.lbm_destroy(ctx)
        shp = (2, wl.nz, wl.ny, wl.nx)
        return r.reshape(shp), u.reshape((3,) + shp), t.reshape(shp)

    got = {}
    for name, make, tau_expr, steps, eq, col, mom in ORACLE_CASES:
        wl, tau = eval(make, {"W": W}), float(eval(tau_expr, {"W": W}))
        got[name] = {st: lib(wl, tau, st, steps, eq, col, mom and st != "f64") for st in ("f64", "f32", "f16", "bf16")}
    served_got = {}
    srv = B.lbm_server_create(4 << 30, 16)
    try:
        tickets = []
        for name, make, tau_expr, steps in SERVED_CASES:
            wl, tau = eval(make, {"W": W}), float(eval(tau_expr, {"W": W}))
            for st in ("f32", "f16"):
                cfg = B.make_config(wl.nx, wl.ny, wl.nz, tau, st, wl.faces, equilibrium="entropic")
                tickets.append((name, st, wl, B.lbm_submit(srv, cfg, np_flat(wl.rho), np_flat(wl.u), np_flat(wl.theta),
                                                           steps)))
        for name, st, wl, t in tickets:
            if B.lbm_wait(srv, t, 600.0) != B.LBM_OK:
                raise RuntimeError("served accuracy case did not finish")
            S = wl.sites
            r, u, th = np.zeros(S), np.zeros(3 * S), np.zeros(S)
            status, _ = B.lbm_poll(srv, t, r, u, th)
            shp = (2, wl.nz, wl.ny, wl.nx)
            served_got.setdefault(name, {})[st] = ((r.reshape(shp), u.reshape((3,) + shp), th.reshape(shp))
                                                   if status == B.LBM_OK else None)
    finally:
        B.lbm_server_destroy(srv)
    refs = {}
    for name, (proc, path) in jobs.items():
        _, err = proc.communicate(timeout=1800)
        if proc.returncode != 0:
            raise RuntimeError(f"oracle reference {name} failed: {err[-300:]}")
        z = np.load(path)
        refs[name] = (z["rho"], z["u"], z["theta"])
        os.unlink(path)
    os.rmdir(tmp)
    rnd = lambda d: {k: float(f"{v:.3g}") for k, v in d.items()}
    out = {name: {st: (rnd(errs(refs[name], g)) if g is not None else "unstable") for st, g in per.items()}
           for name, per in got.items()}
    served = {name: {st: (rnd(errs(refs[name], g)) if g is not None else "unstable") for st, g in per.items()}
              for name, per in served_got.items()}
    return out, served


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
    head = run_case(B, args.n, args.storage, args.steps, args.warmup, world, fp64_moments=args.fp64_moments,
                    sampler=sampler, eq=args.equilibrium, collision=args.collision, streaming=args.streaming)
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
                                                                 args.streaming, args.fp64_moments),
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
                                          ("tgv512_f16_fp64moments", 512, "f16", True, "series", "bgk", "pingpong"),
                                          ("tgv512_bf16_fp64moments", 512, "bf16", True, "series", "bgk", "pingpong"),
                                          ("tgv512_f32_aa_fp64moments", 512, "f32", True, "series", "bgk", "aa"),
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
        line["workloads"] = workload_variants(B, peak)
        line["e2e"] = run_e2e(B, args.n, args.storage, 3)
        try:
            line["served"] = run_served(B)
        except Exception as exc:  # report, do not lose the rest of the line
            line["served"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.quick and not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = cpu_baseline()
        try:
            line["oracle_errors"], served_acc = oracle_errors(B)
            if isinstance(line.get("served"), dict):
                line["served"]["accuracy_vs_fp64_oracle"] = served_acc
        except Exception as exc:  # report, do not lose the rest of the line
            line["oracle_errors"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------------------

def reference(args):
    """The reference arm: the FP64 oracle as it stands, one single-threaded process per host core,
    each advancing its own TGV 32^3 sample (the headline workload's recipe) through W warm-up and
    K timed oracle steps; the value sums the processes' rates.  No GPU is used."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2409_05114_gb300 import workloads as W
    n = 32
    cores = len(os.sched_getaffinity(0))
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import rd3q81 as O
from paper_2409_05114_gb300 import workloads as W
wl = W.taylor_green({n})
tau = wl.paper_tau('lb')
f = O.init(wl.rho, wl.u, wl.theta)
for _ in range({args.warmup}):
    f = O.step(f, tau)
t0 = time.perf_counter()
for _ in range({args.steps}):
    f = O.step(f, tau)
print(json.dumps({{"seconds": time.perf_counter() - t0, "sites": wl.sites}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(cores)]
    rates, secs = [], []
    for p_ in ps:
        out, err = p_.communicate(timeout=3600)
        if p_.returncode != 0:
            raise RuntimeError(err[-300:])
        d = json.loads(out.strip().splitlines()[-1])
        rates.append(d["sites"] * args.steps / d["seconds"] / 1e6)
        secs.append(d["seconds"])
    value = sum(rates)
    sites = 2 * n ** 3
    sample = (f"each step = one full FP64 oracle step of TGV {n}^3 ({sites} sites, same init recipe as the "
              f"headline) in each of {cores} single-threaded processes (one per host core), rates summed")
    line = {"metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.median(secs) / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"taylor_green_{args.n}^3 (oracle on {cores} x {n}^3 samples)", "sites": sites},
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
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
