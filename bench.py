"""Benchmark: arc x constant-latitude intersections on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sphx|reference]

A step is one dense call (sphx_intersect_gca_constlat) over the
ill-conditioned workload of 10^6 arcs (40 % short, 30 % near-tangent, 20 %
near-pole, 10 % near-antipodal), inputs resident in HBM; the L2 cache is
flushed (a 256 MiB write) between timed steps. The headline mode is the
integer-limb evaluation (SPHX_MODE_WIDE_INT, within 1 ulp of the exact
result); FP64-EFT (the paper's AccuX), direct FP64 and float-float are timed
the same way beside it. Under torchrun each rank runs its own
independently seeded batch (weak scaling, no data-path collective); the step
time is the maximum over ranks.

``--impl reference`` times the exact-rational CPU oracle, as it stands, on
the host's cores over bounded samples of the same workload.

Prints one JSON line (rank 0).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2510_09892_gb300 import workloads as W  # noqa: E402

METRIC = "arc–latitude intersections/sec at ≤4-ulp error, EFT vs direct FP64, % HBM roofline"
UNIT = "intersections/s"
N_ARCS = 1_000_000
WORKLOAD = ("ill-conditioned FP64-EFT stress, 10^6 arcs: 40% short (log-uniform 1e-10..1e-2 rad), "
            "30% nearly tangent (z0 within 1e-12 of the z-extremum), 20% near-pole "
            "(|z| > 1-1e-6), 10% near-antipodal")
# algorithmic work per arc of the dense call (both roots and the on-arc test)
BYTES_PER_ARC = 7 * 8 + 6 * 8 + 4   # 56 B in, 48 B points + 4 B count out
FP64_OPS_PER_ARC = {"eft": 465, "direct": 70}  # one op = add/mul/fma/div/sqrt
# thread instructions per arc of dense_kernel<WIDE> (ncu smsp__inst_executed.sum x 32
# / arcs on the 10^6-arc stress workload): the integer-limb method's work per arc
INST_PER_ARC = {"wide": 2351}
# DRAM bytes (read + write) of one launch of the headline kernel over the 10^6
# stress arcs, from the same ncu capture (writes still in L2 at kernel end are
# not counted)
TRAFFIC_PER_LAUNCH = {"wide": 58.238e6 + 9.188e6}
ISSUE_SLOTS_PER_SM_CLK = 4 * 32  # 4 schedulers, one warp instruction each per clock
SM_MAX_MHZ = 2070.0
DTYPES = {"wide": "u32 limbs (128/96-bit mantissas), f64 in/out", "eft": "f64",
          "direct": "f64", "ff32": "f32 pairs + f64",
          "adaptive": "f64 with a running error bound, u32 limbs where it fails"}
L2_FLUSH_BYTES = 256 << 20
ADAPTIVE_GATES = (4.0, 64.0, 2.0 ** 20)  # ulp per component; 4 is the adaptive mode's own
CPU_SAMPLE = 32_768            # arcs per oracle step


# ------------------------------------------------------------- host logic --
def dist_env():
    """(rank, world, local_rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard_seed(base: int, rank: int) -> int:
    """Seed of rank's batch: rank 0 runs the published workload seed itself."""
    return base if rank == 0 else int(np.random.SeedSequence([base, rank]).generate_state(1)[0])


def reduce_max(value: float, device=None) -> float:
    """Maximum of a float over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 100 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # wait (at most 3 s) for the first sample so the timed region is covered
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < 3.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ reference arm --
def oracle_rate(A, B, z, pool) -> float:
    """Arcs per second of the exact oracle over the given arcs, on the pool."""
    from oracle import exact
    n = len(z)
    chunk = max(1, n // (4 * pool._processes))
    jobs = [(A[i:i + chunk].tolist(), B[i:i + chunk].tolist(), z[i:i + chunk].tolist())
            for i in range(0, n, chunk)]
    t0 = time.perf_counter()
    pool.map(exact._batch_worker, jobs)
    return n / (time.perf_counter() - t0)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    A, B, z = W.stress_arcs(N_ARCS)
    with mp.get_context("spawn").Pool(cores) as pool:
        rates = []
        for step in range(args.warmup + args.steps):
            lo = (step * CPU_SAMPLE) % (N_ARCS - CPU_SAMPLE)
            r = oracle_rate(A[lo:lo + CPU_SAMPLE], B[lo:lo + CPU_SAMPLE], z[lo:lo + CPU_SAMPLE],
                            pool)
            if step >= args.warmup:
                rates.append(r)
    value = CPU_SAMPLE / statistics.mean([CPU_SAMPLE / r for r in rates])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * CPU_SAMPLE / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "exact rational (Python int), rounded to f64",
        "data": "synthetic", "config": config_dict(args, args.mode),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{CPU_SAMPLE} consecutive arcs of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, mode):
    return {"workload": WORKLOAD, "arcs_per_gpu": N_ARCS, "mode": mode,
            "seed": W.DEFAULT_SEED + 1, "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"independent batches, {args.gpus} GPU(s)"}


# ------------------------------------------------------------------ GPU arm --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sphx", choices=["sphx", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the ragged (regridding) leg reported beside the headline")
    ap.add_argument("--mode", default="wide", choices=["wide", "eft", "direct", "ff32"],
                    help="headline evaluation mode (the others are timed beside it)")
    ap.add_argument("--zonal-only", action="store_true",
                    help="run only the zonal-mean leg and print its JSON (for profiling)")
    ap.add_argument("--ragged-only", action="store_true",
                    help="run only the cubed-sphere regridding leg and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.zonal_only or args.ragged_only:
        import torch
        from paper_2510_09892_gb300 import sphx
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        if args.zonal_only:
            line = {"zonal_mean": zonal_leg(sphx, torch, dev, args, args.mode)}
        else:
            line = {"ragged_regridding": ragged_leg(sphx, torch, dev, args, args.mode)}
        print(json.dumps(line), flush=True)
        return

    rank, world, local = dist_env()
    # the process pools start before CUDA does ('spawn' regardless)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()
    mesh_pool = None
    if rank == 0 and not args.no_ragged:
        import multiprocessing as mp
        mesh_pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))

    import torch
    import torch.distributed as dist
    from paper_2510_09892_gb300 import sphx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    A, B, z = W.stress_arcs(N_ARCS, seed=shard_seed(W.DEFAULT_SEED + 1, rank))
    tA, tB, tz = (torch.from_numpy(v).to(dev) for v in (A, B, z))
    pts = torch.empty((N_ARCS, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.empty((N_ARCS,), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed(mode, steps, warmup):
        """Mean kernel time (ms) of `steps` dense calls, L2 flushed before each."""
        ms = []
        with torch.cuda.stream(stream):
            for i in range(warmup + steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, mode, stream)
                e1.record(stream)
                if i >= warmup:
                    ms.append((e0, e1))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in ms]

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_FP64) / 2  # FMA/s = FP64 op slots/s
    fp32_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_FP32) / 2
    int32_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_INT32)
    head = args.mode
    others = [m for m in ("wide", "eft", "direct", "ff32") if m != head]

    # warm-up of every mode, then the headline timed region
    for mode in [head] + others:
        timed(mode, 1, args.warmup)
    barrier()
    torch.cuda.synchronize()
    # the sampler runs through every timed leg (headline, other modes, e2e)
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        head_ms = timed(head, args.steps, 0)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall
        gpu_launches = args.steps  # one dense_kernel launch per step
        step_ms = reduce_max(statistics.mean(head_ms), dev)
        value = world * N_ARCS / (step_ms * 1e-3)

        modes = {head: {"value": value, "ms_per_step": step_ms}}
        for mode in others:
            m = reduce_max(statistics.mean(timed(mode, args.steps, 0)), dev)
            modes[mode] = {"value": world * N_ARCS / (m * 1e-3), "ms_per_step": m}
        e2e = e2e_leg(sphx, torch, dev, A, B, z, args, head)
        # the timed legs last well under a second, shorter than the sampling
        # period: keep the headline kernel running for 1.5 s more so that the
        # clock samples describe the GPU under this load (not timed)
        soak_end = time.perf_counter() + 1.5
        while time.perf_counter() < soak_end:
            timed(head, 50, 0)
    clk = clocks.summary()
    clk["window"] = "timed legs plus a 1.5 s soak of the headline kernel right after"

    arcs = arcs_leg(sphx, torch, dev, args, flush) if rank == 0 else None
    adaptive = adaptive_leg(sphx, torch, dev, args, flush, (A, B, z)) if rank == 0 else None
    ragged = ragged_leg(sphx, torch, dev, args, head) if rank == 0 and not args.no_ragged else None
    zonal = zonal_leg(sphx, torch, dev, args, head) if rank == 0 and not args.no_ragged else None
    meshes = (meshes_leg(sphx, torch, dev, args, head, mesh_pool)
              if rank == 0 and not args.no_ragged else None)

    # hits per step, from one more headline call's outputs
    sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, head)
    hits = int(torch.clamp(cnt, min=0).sum().item())

    hbm_peak = measured_hbm_peak()

    def hbm_roof(ms):
        gbs = BYTES_PER_ARC * N_ARCS / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "unit": "GB/s", "achieved": gbs, "peak": hbm_peak,
                "frac": gbs / hbm_peak, "traffic": None,
                "note": "108 B per arc (56 in, 52 out) against the measured copy bandwidth "
                        "(MEASURED_PEAKS.json, of measured)"}

    def alu_roof(ms, ops_per_arc, peak, pipe):
        rate = ops_per_arc * N_ARCS / (ms * 1e-3)
        measured = "issue" not in pipe
        return {"bound": "alu", "unit": "Tops/s", "achieved": rate / 1e12, "peak": peak / 1e12,
                "frac": rate / peak, "traffic": None,
                "note": f"{pipe}: {ops_per_arc} operations per arc against "
                        + ("the pipe's rate measured live by sphx_probe_fma_rate (of measured)"
                           if measured else
                           "4 x 32 lanes x SMs x the 2070 MHz maximum SM clock (derived)")}

    head_kernel_ms = statistics.mean(head_ms)
    issue_peak = ISSUE_SLOTS_PER_SM_CLK * sm_count * SM_MAX_MHZ * 1e6
    if head in INST_PER_ARC:
        roofline = alu_roof(head_kernel_ms, INST_PER_ARC[head], issue_peak,
                            "instruction issue (4 warp instructions per SM per clock)")
    elif head in FP64_OPS_PER_ARC:
        roofline = alu_roof(head_kernel_ms, FP64_OPS_PER_ARC[head], fp64_peak, "FP64 pipe")
    else:
        roofline = hbm_roof(head_kernel_ms)
    roofline["kernel"] = f"dense_kernel<{head}>"
    roofline["traffic"] = TRAFFIC_PER_LAUNCH.get(head)
    per_mode_roofs = {"hbm": {m: hbm_roof(modes[m]["ms_per_step"])["frac"] for m in modes}}
    per_mode_roofs["fp64_pipe"] = {m: alu_roof(modes[m]["ms_per_step"], FP64_OPS_PER_ARC[m],
                                               fp64_peak, "FP64")["frac"]
                                   for m in modes if m in FP64_OPS_PER_ARC}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "ms_per_step_stats": {"mean": statistics.mean(head_ms),
                              "median": statistics.median(head_ms), "best": min(head_ms),
                              "worst": max(head_ms), "steps": len(head_ms),
                              "note": "this rank's CUDA-event times of the timed steps"},
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": config_dict(args, head), "e2e": e2e, "gpu_launches": gpu_launches,
        "clocks": clk, "roofline": roofline, "roofline_hbm": hbm_roof(head_kernel_ms),
        "roofline_frac_by_mode": per_mode_roofs,
        "modes": modes,
        "eft_over_direct_time": modes["eft"]["ms_per_step"] / modes["direct"]["ms_per_step"],
        "hits_per_step": hits, "timed_wall_s": t_wall,
        "peaks": {"fp64_fma_per_s": fp64_peak, "fp32_fma_per_s": fp32_peak,
                  "int32_imad_per_s": int32_peak, "hbm_gbs": hbm_peak},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if arcs is not None:
        line["arc_x_arc"] = arcs
    if adaptive is not None:
        line["adaptive_filter"] = adaptive
    if ragged is not None:
        line["ragged_regridding"] = ragged
    if zonal is not None:
        line["zonal_mean"] = zonal
    if meshes is not None:
        line["ragged_meshes"] = meshes
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def arcs_leg(sphx, torch, dev, args, flush) -> dict:
    """Arc x arc intersections (not the headline): 10^6 pairs of great circle
    arcs (50 % uniform, 15 % short, 15 % nearly parallel circles, 10 % crossings
    near an endpoint, 10 % misses), each mode timed with CUDA events over
    `steps` calls, the L2 cache flushed before each."""
    A1, A2, B1, B2 = W.arc_pairs(1_000_000)
    t = [torch.from_numpy(v).to(dev) for v in (A1, A2, B1, B2)]
    n = len(A1)
    pts = torch.empty((n, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    cur = torch.cuda.current_stream(dev)
    res = {"workload": "10^6 arc pairs: 50% uniform, 15% short, 15% nearly parallel, "
                       "10% crossing near an endpoint, 10% misses", "pairs": n, "modes": {}}
    for mode in ("wide", "eft", "direct"):
        ms = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            sphx.sphx_intersect_gca_gca(*t, pts, cnt, mode, cur)
            e1.record(cur)
            if i >= args.warmup:
                ms.append((e0, e1))
        torch.cuda.synchronize()
        m = statistics.mean(a.elapsed_time(b) for a, b in ms)
        res["modes"][mode] = {"ms_per_step": m, "pairs_per_s": n / (m * 1e-3),
                              "hbm_frac": 148 * n / (m * 1e-3) / 1e9 / measured_hbm_peak()}
    res["hits"] = int(torch.clamp(cnt, min=0).sum().item())
    return res


def adaptive_leg(sphx, torch, dev, args, flush, stress) -> dict:
    """The adaptive filter (not the headline): on the 10^6 stress arcs and on
    10^6 well-conditioned arcs (uniform endpoints, arc length uniform in
    (0, pi/2), one latitude inside each arc's z-range), the time per dense call
    of the adaptive mode beside the integer-limb and direct FP64 forms, and the
    share of arcs the filter hands on to the integer-limb form."""
    cur = torch.cuda.current_stream(dev)
    res = {"workloads": {}}
    for name in ("stress", "uniform"):
        A, B, z = stress if name == "stress" else W.uniform_arcs(N_ARCS, seed=W.DEFAULT_SEED + 5)
        tA, tB, tz = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (A, B, z))
        n = len(z)
        pts = torch.empty((n, 2, 3), dtype=torch.float64, device=dev)
        cnt = torch.empty(n, dtype=torch.int32, device=dev)
        entry = {"arcs": n, "fallback_share": {}, "ms_per_step": {}}
        fb = torch.zeros(1, dtype=torch.int64, device=dev)
        calls = {"wide": lambda: sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "wide", cur),
                 "direct": lambda: sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "direct",
                                                                    cur)}
        for gate in ADAPTIVE_GATES:
            fb.zero_()
            sphx.sphx_intersect_gca_constlat_adaptive(tA, tB, tz, pts, cnt, gate, fb, cur)
            torch.cuda.synchronize()
            entry["fallback_share"][f"{gate:g} ulp"] = int(fb.item()) / n
            calls[f"adaptive, {gate:g} ulp"] = (
                lambda g=gate: sphx.sphx_intersect_gca_constlat_adaptive(tA, tB, tz, pts, cnt, g,
                                                                         None, cur))
        for key, call in calls.items():
            ms = []
            for i in range(args.warmup + args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(cur)
                call()
                e1.record(cur)
                if i >= args.warmup:
                    ms.append((e0, e1))
            torch.cuda.synchronize()
            entry["ms_per_step"][key] = statistics.mean(a.elapsed_time(b) for a, b in ms)
        res["workloads"][name] = entry
    return res


def ragged_leg(sphx, torch, dev, args, head) -> dict:
    """The regridding workload through the ragged call (not the headline): a
    cubed sphere with 1024 x 1024 cells per face (12 595 200 edges) against
    the 721 latitudes of a 0.25-degree grid. One step is the whole ragged
    sequence (candidate ranges, prefix sum, persistent intersection with
    compaction), replayed from the context's CUDA graph; the 605 MB of edges
    exceed L2, so no flush is needed. The launch shape is picked by
    sphx_autotune_ragged for each mode first."""
    A, B = W.cubed_sphere_edges(1024)
    lat = W.latlon_latitudes(721)
    E = len(A)
    d = {"A": torch.from_numpy(A).to(dev), "B": torch.from_numpy(B).to(dev),
         "eo": torch.tensor([0, E], dtype=torch.int64, device=dev),
         "lat": torch.from_numpy(lat).to(dev),
         "lo": torch.tensor([0, 721], dtype=torch.int64, device=dev)}
    lo = torch.empty(E, dtype=torch.int32, device=dev)
    hi = torch.empty(E, dtype=torch.int32, device=dev)
    sphx.sphx_candidate_ranges(d["A"], d["B"], d["eo"], d["lat"], d["lo"], lo, hi)
    pairs = int((hi - lo).sum().item())
    cap = 2 * pairs + 1024
    out = torch.empty(cap * 4, dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    res = {"workload": "cubed sphere N=1024 (12,595,200 edges) x 721 latitudes (0.25 deg)",
           "edges": E, "candidate_pairs": pairs, "modes": {}}
    cur = torch.cuda.current_stream(dev)
    with sphx.Context(dev.index or 0) as ctx:
        for mode in (head, "eft", "direct"):
            ctx.reset_tuning()
            tune_ms = sphx.sphx_autotune_ragged(ctx, d["A"], d["B"], d["eo"], d["lat"], d["lo"], out,
                                                total, mode, stream=cur)
            for _ in range(args.warmup):
                sphx.sphx_intersect_ragged(ctx, d["A"], d["B"], d["eo"], d["lat"], d["lo"], out,
                                           total, mode, stream=cur)
            if ctx.sync_status(cur) != sphx.OK:
                raise RuntimeError("ragged call reported an error")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            for _ in range(args.steps):
                sphx.sphx_intersect_ragged(ctx, d["A"], d["B"], d["eo"], d["lat"], d["lo"], out,
                                           total, mode, stream=cur)
            e1.record(cur)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            hits = int(total.item())
            res["hits"] = hits
            res["modes"][mode] = {
                "ms_per_step": ms, "edges_per_s": E / (ms * 1e-3),
                "pairs_per_s": pairs / (ms * 1e-3), "hits_per_s": hits / (ms * 1e-3),
                "hbm_frac": (48 * E + 32 * hits) / (ms * 1e-3) / 1e9 / measured_hbm_peak(),
                "tuning": ctx.get_tuning(), "autotune_best_ms": tune_ms}
    return res


def zonal_leg(sphx, torch, dev, args, head) -> dict:
    """The zonal-mean step (not the headline) on the regridding workload: the
    cubed sphere with 1024 x 1024 cells per face (6,291,456 node-indexed
    quadrilaterals) against the 721 latitudes of a 0.25-degree grid. One step
    is sphx_band_ranges (bands per cell, prefix sum), sphx_band_areas (area of
    every cell in every band it meets) and sphx_zonal_sums (per-band sums of
    field * area and area). The mesh (300 MB) exceeds L2, so no flush."""
    nodes, off, fn = W.cubed_sphere_cells(1024)
    lat = W.latlon_latitudes(721)
    F, nb = len(off) - 1, len(lat) - 1
    dn, do, df, dl = (torch.from_numpy(x).to(dev) for x in (nodes, off, fn, lat))
    field = torch.from_numpy(nodes[fn[0::4], 2].copy()).to(dev)  # z of each cell's first node
    lo = torch.empty(F, dtype=torch.int32, device=dev)
    hi = torch.empty(F, dtype=torch.int32, device=dev)
    ao = torch.empty(F + 1, dtype=torch.int64, device=dev)
    fa = torch.empty(nb, dtype=torch.float64, device=dev)
    aa = torch.empty(nb, dtype=torch.float64, device=dev)
    cur = torch.cuda.current_stream(dev)
    res = {"workload": "cubed sphere N=1024 (6,291,456 cells) x 721 latitudes (0.25 deg): "
                       "band ranges + band areas + zonal sums", "cells": F, "modes": {}}
    exact_bands = 2 * math.pi * np.diff(lat)
    with sphx.Context(dev.index or 0) as ctx:
        sphx.sphx_band_ranges(ctx, dn, do, df, dl, lo, hi, ao, stream=cur)
        entries = int(ao[-1].item())
        areas = torch.empty(entries, dtype=torch.float64, device=dev)
        res["band_entries"] = entries

        def step(mode, ev=None):
            sphx.sphx_band_ranges(ctx, dn, do, df, dl, lo, hi, ao, stream=cur)
            if ev is not None:
                ev[0].record(cur)
            sphx.sphx_band_areas(ctx, dn, do, df, dl, lo, hi, ao, areas, mode, stream=cur)
            if ev is not None:
                ev[1].record(cur)
            sphx.sphx_zonal_sums(ctx, lo, hi, ao, areas, field, len(lat), fa, aa, stream=cur)

        for mode in (head, "eft", "direct"):
            for _ in range(args.warmup):
                step(mode)
            if ctx.sync_status(cur) != sphx.OK:
                raise RuntimeError("band-area call reported an error")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            e0.record(cur)
            for i in range(args.steps):
                step(mode, kev[i])
            e1.record(cur)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            k_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
            cons = float(np.abs(aa.cpu().numpy() - exact_bands).max())
            res["modes"][mode] = {
                "ms_per_step": ms, "cells_per_s": F / (ms * 1e-3),
                "band_areas_per_s": entries / (ms * 1e-3), "area_kernel_ms": k_ms,
                "max_abs_band_total_error": cons}
    return res


def meshes_leg(sphx, torch, dev, args, head, pool) -> dict:
    """Ragged batching (not the headline): 512 independent polygon meshes of
    10^3 - 5x10^6 edges (log-uniform, ~3x10^8 edges in all) against per-mesh
    grids of 180 - 2881 latitudes, in one persistent launch replayed from a
    CUDA graph, with the launch shape picked by sphx_autotune_ragged; integer
    limbs, FP64-EFT and direct FP64."""
    E, L = W.ragged_sizes(512, 1e3, 5e6)
    eo = np.concatenate([[0], np.cumsum(E)]).astype(np.int64)
    lo_ = np.concatenate([[0], np.cumsum(L)]).astype(np.int64)
    lat = np.concatenate([W.latlon_latitudes(int(x)) for x in L])
    Et = int(eo[-1])
    tA = torch.empty((Et, 3), dtype=torch.float64, device=dev)
    tB = torch.empty((Et, 3), dtype=torch.float64, device=dev)
    seed = W.DEFAULT_SEED + 3
    with pool:
        for m, (A, B) in enumerate(pool.imap(W.ragged_mesh, [(m, int(E[m]), seed)
                                                            for m in range(len(E))])):
            tA[int(eo[m]):int(eo[m + 1])].copy_(torch.from_numpy(A))
            tB[int(eo[m]):int(eo[m + 1])].copy_(torch.from_numpy(B))
    teo = torch.from_numpy(eo).to(dev)
    tlo = torch.from_numpy(lo_).to(dev)
    tlat = torch.from_numpy(lat).to(dev)
    lo = torch.empty(Et, dtype=torch.int32, device=dev)
    hi = torch.empty(Et, dtype=torch.int32, device=dev)
    sphx.sphx_candidate_ranges(tA, tB, teo, tlat, tlo, lo, hi)
    pairs = int((hi - lo).sum().item())
    del lo, hi
    cap = pairs + pairs // 8 + 4096
    out = torch.empty(cap * 4, dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    res = {"workload": "512 polygon meshes, 1e3-5e6 edges each (log-uniform), 180-2881 "
                       "latitudes per mesh", "edges": Et, "candidate_pairs": pairs, "modes": {}}
    cur = torch.cuda.current_stream(dev)
    with sphx.Context(dev.index or 0) as ctx:
        for mode in (head, "eft", "direct"):
            ctx.reset_tuning()
            tune_ms = sphx.sphx_autotune_ragged(ctx, tA, tB, teo, tlat, tlo, out, total, mode,
                                                stream=cur)
            for _ in range(3):
                sphx.sphx_intersect_ragged(ctx, tA, tB, teo, tlat, tlo, out, total, mode,
                                           stream=cur)
            if ctx.sync_status(cur) != sphx.OK:
                raise RuntimeError("ragged call reported an error")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            steps = max(3, args.steps // 4)
            e0.record(cur)
            for _ in range(steps):
                sphx.sphx_intersect_ragged(ctx, tA, tB, teo, tlat, tlo, out, total, mode,
                                           stream=cur)
            e1.record(cur)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            hits = int(total.item())
            res["hits"] = hits
            res["modes"][mode] = {
                "ms_per_step": ms, "edges_per_s": Et / (ms * 1e-3),
                "pairs_per_s": pairs / (ms * 1e-3), "hits_per_s": hits / (ms * 1e-3),
                "hbm_frac": (48 * Et + 32 * hits) / (ms * 1e-3) / 1e9 / measured_hbm_peak(),
                "tuning": ctx.get_tuning(), "autotune_best_ms": tune_ms}
    del tA, tB, out
    torch.cuda.empty_cache()
    return res


def measured_hbm_peak() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure of the profiling recipe


def cpu_baseline_leg() -> dict:
    """The exact oracle, as it stands, on all host cores over a bounded sample."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = min(N_ARCS, 6000 * cores)  # ~0.6 s of oracle work per core
    A, B, z = W.stress_arcs(N_ARCS)
    with mp.get_context("spawn").Pool(cores) as pool:
        oracle_rate(A[:1024], B[:1024], z[:1024], pool)  # start the workers
        rate = oracle_rate(A[:n], B[:n], z[:n], pool)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} arcs of the 10^6-arc stress workload",
            "step_reference": step_reference_rates(A, B, z)}


def step_reference_rates(A, B, z) -> dict:
    """The paper's two FP64 forms as scalar C on one host core (the step
    reference, gcc -O2 -ffp-contract=off): direct Eq. 2.2 and AccuX
    (Algorithm 8), over the whole 10^6-arc stress workload. The paper reports
    AccuX about 9x slower than the direct form serially (Sec. 8)."""
    from oracle import steps
    steps.lib()  # build outside the timing
    out = {}
    for name, fn in (("direct", lambda: steps.direct(A, B, z)),
                     ("accux", lambda: steps.accux(A, B, z, variant=2))):
        best = float("inf")
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            best = min(best, time.perf_counter() - t0)
        out[name] = {"value": len(z) / best, "unit": UNIT, "cores": 1}
    out["accux_over_direct_time"] = out["direct"]["value"] / out["accux"]["value"]
    out["sample"] = "the whole 10^6-arc stress workload, one core, best of 3"
    return out


def e2e_leg(sphx, torch, dev, A, B, z, args, mode) -> dict:
    """Same metric through the C ABI from pinned HOST buffers
    (sphx_intersect_gca_constlat_host): every step moves the inputs in and the
    points and counts out; with page-locked buffers the kernel reads and writes
    host memory in place, so the transfers overlap the arithmetic."""
    n = len(z)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hz = torch.from_numpy(z).pin_memory()
    hP = torch.empty((n, 2, 3), dtype=torch.float64).pin_memory()
    hC = torch.empty((n,), dtype=torch.int32).pin_memory()
    cur = torch.cuda.current_stream(dev)
    with sphx.Context(dev.index or 0) as ctx:
        for _ in range(args.warmup):
            sphx.sphx_intersect_gca_constlat_host(ctx, hA, hB, hz, hP, hC, mode, cur)
        sphx.sphx_host_join(ctx, cur)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for _ in range(args.steps):
            sphx.sphx_intersect_gca_constlat_host(ctx, hA, hB, hz, hP, hC, mode, cur)
        sphx.sphx_host_join(ctx, cur)  # every step's results are back in host memory
        e1.record(cur)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_max(ms, dev)
    _, world, _ = dist_env()
    return {"value": world * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "h2d_bytes_per_step": n * 56, "d2h_bytes_per_step": n * 52,
            "path": "sphx_intersect_gca_constlat_host, pinned host buffers (read and written "
                    "in place by the kernel over NVLink-C2C)"}


if __name__ == "__main__":
    main()
