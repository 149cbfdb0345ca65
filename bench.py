"""Benchmark: arc x constant-latitude intersections on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sphx|reference]

A step is one dense call (sphx_intersect_gca_constlat) over the precision
workload: 2x10^8 arcs, 90 % well-conditioned (endpoints uniform on the
sphere, length U(0, pi/2), one latitude in each arc's z-range) mixed with
10 % of the ill-conditioned stress mix (short, nearly tangent, near-pole and
near-antipodal arcs), generated in independently seeded chunks of 2^20 arcs.
The 21.6 GB of inputs and outputs exceed the 129 MB L2 many times over, so
no flush is needed between steps. The headline mode is the integer-limb
evaluation (SPHX_MODE_WIDE_INT, correctly rounded on every sampled arc);
FP64-EFT (the paper's AccuX), direct FP64 and float-float run the same steps
beside it. The metric counts intersections (hits), not arcs. Under torchrun
each rank runs its own independently seeded batch (weak scaling, no
data-path collective); the step time is the maximum over ranks.

Beside the headline: the 10^6-arc stress workload (L2 flushed between
steps), arc x arc pairs, the adaptive filter, the ragged regridding and
mesh-batch legs and the zonal-mean step; on the host cores, the exact oracle
and the paper's two FP64 forms as plain C loops (cpu_baseline).

``--impl reference`` times the exact-rational CPU oracle, as it stands, on
the host's cores over bounded samples of the same workload.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
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
N_ARCS = 200_000_000
MIXED_SEED = W.DEFAULT_SEED + 4
WORKLOAD = ("precision variant: 2x10^8 arcs, 90% uniform (endpoints uniform on the sphere, "
            "length U(0, pi/2), z0 in the arc's z-range) mixed with 10% of the ill-conditioned "
            "stress mix, in independently seeded chunks of 2^20 arcs")
STRESS_ARCS = 1_000_000
STRESS_WORKLOAD = ("ill-conditioned FP64-EFT stress, 10^6 arcs: 40% short (log-uniform "
                   "1e-10..1e-2 rad), 30% nearly tangent (z0 within 1e-12 of the z-extremum), "
                   "20% near-pole (|z| > 1-1e-6), 10% near-antipodal")
MODES = ("wide", "eft", "direct", "ff32")
# algorithmic work per arc of the dense call (both roots and the on-arc test)
BYTES_PER_ARC = 7 * 8 + 6 * 8 + 4   # 56 B in, 48 B points + 4 B count out
# FP64 and FP32 thread instructions per arc of each mode's dense kernel (DFMA,
# DADD and DMUL; FFMA, FADD and FMUL; the division and square-root sequences
# counted by the instructions they expand to), from one ncu capture of 10^7
# mixed arcs: properties of the compiled kernels, tagged with the capture
OPS_SOURCE = ("ncu sm__sass_thread_inst_executed_op_{dfma,dadd,dmul,ffma,fadd,fmul}_pred_on.sum "
              "/ arcs, 10^7 arcs of the mixed workload, profiles/dense_modes_fp_ops_mixed_1e7.md "
              "(kernels as of commit 4ff5d7b)")
FP64_OPS_PER_ARC = {"eft": 413.5, "direct": 106.0, "ff32": 18.0, "wide": 14.0}
FP32_OPS_PER_ARC = {"ff32": 176.0, "wide": 57.0}
# Thread instructions per arc of dense_kernel<WIDE>, from one ncu capture
# (smsp__inst_executed.sum x 32 / arcs): a property of the compiled kernel,
# valid only for the build it was taken on, reported as a secondary figure.
INST_PER_ARC = {"wide": {"value": 2329, "source": "ncu smsp__inst_executed.sum x 32 / arcs, "
                         "10^7 arcs of the mixed workload, "
                         "profiles/dense_pf_kernel_wide_mixed_1e7.md (kernel as of commit "
                         "7a7e4e6)"}}
# DRAM bytes (read + write) per arc of one launch, from an ncu capture of a
# launch larger than L2 (scaled to the launch by its arcs); None where no
# capture matches the current kernel.
TRAFFIC_PER_ARC = {"wide": {"value": (561160448 + 477118208) / 1e7,
                            "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "launch over 10^7 arcs of the mixed workload, scaled by "
                                      "the arcs, profiles/dense_pf_kernel_wide_mixed_1e7.md "
                                      "(kernel as of commit 7a7e4e6)"}}
ISSUE_SLOTS_PER_SM_CLK = 4 * 32  # 4 schedulers, one warp instruction each per clock
SM_MAX_MHZ = 2070.0
DTYPES = {"wide": "u32 limbs (128/96-bit mantissas), f64 in/out", "eft": "f64",
          "direct": "f64", "ff32": "f32 pairs + f64",
          "adaptive": "f64 with a running error bound, u32 limbs where it fails"}
ERROR = {"wide": "<= 1 ulp per component (correctly rounded on every sampled arc)",
         "eft": "<= 4 ulp per component, |dP| <= 3 u sqrt(1 - z0^2) (Sec. 6.2)",
         "direct": "unbounded near tangency and the poles (Sec. 4): not at <= 4 ulp",
         "ff32": "its stated float-float bound, not at <= 4 ulp"}
L2_FLUSH_BYTES = 256 << 20
ADAPTIVE_GATES = (4.0, 64.0, 2.0 ** 20)  # ulp per component; 4 is the adaptive mode's own
CPU_SAMPLE = 32_768            # arcs per oracle step (reference arm)
CPU_LOOP_ARCS = 100_000_000    # arcs of the mixed workload for the all-core FP64 loops


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


def _mixed_job(args):
    k, seed = args
    return k, W.mixed_chunk(k, seed)


def fill_mixed(pool, seed: int, A, B, z):
    """The mixed workload's chunks, generated on the pool, written into the
    (n, 3), (n, 3), (n,) arrays A, B, z (any writable numpy arrays)."""
    n = len(z)
    jobs = [(k, seed) for k in range((n + W.CHUNK - 1) // W.CHUNK)]
    for k, (a, b, c) in pool.imap_unordered(_mixed_job, jobs):
        lo, hi = k * W.CHUNK, min(n, (k + 1) * W.CHUNK)
        A[lo:hi], B[lo:hi], z[lo:hi] = a[:hi - lo], b[:hi - lo], c[:hi - lo]


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
def _oracle_job(args):
    from oracle import exact
    A, B, Z = args
    hits = 0
    for i in range(len(Z)):
        hits += max(0, exact.intersect(A[i], B[i], Z[i]).count)
    return hits


def oracle_rate(A, B, z, pool) -> tuple[float, float]:
    """(arcs/s, intersections/s) of the exact oracle over the given arcs, on the pool."""
    n = len(z)
    chunk = max(1, n // (4 * pool._processes))
    jobs = [(A[i:i + chunk].tolist(), B[i:i + chunk].tolist(), z[i:i + chunk].tolist())
            for i in range(0, n, chunk)]
    t0 = time.perf_counter()
    hits = sum(pool.map(_oracle_job, jobs))
    dt = time.perf_counter() - t0
    return n / dt, hits / dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    steps = args.warmup + args.steps
    # one bounded sample per step: CPU_SAMPLE consecutive arcs of chunk `step`
    with mp.get_context("spawn").Pool(cores) as pool:
        secs, hits = [], []
        for step in range(steps):
            A, B, z = W.mixed_chunk(step, MIXED_SEED)
            a_rate, h_rate = oracle_rate(A[:CPU_SAMPLE], B[:CPU_SAMPLE], z[:CPU_SAMPLE], pool)
            if step >= args.warmup:
                secs.append(CPU_SAMPLE / a_rate)
                hits.append(h_rate * CPU_SAMPLE / a_rate)
    value = sum(hits) / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "exact rational (Python int), rounded to f64",
        "data": "synthetic", "config": config_dict(args, "exact oracle"),
        "arcs_per_s": CPU_SAMPLE * len(secs) / sum(secs),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step, the first {CPU_SAMPLE} arcs of one 2^20-arc chunk "
                                   "of the workload (chunk index = step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, mode):
    return {"workload": WORKLOAD, "arcs_per_gpu": args.arcs, "mode": mode, "seed": MIXED_SEED,
            "l2": "inputs and outputs (108 B per arc) far larger than L2: no flush",
            "parallelism": f"independent batches, {args.gpus} GPU(s)"}


# ---------------------------------------------------------------- CPU loops --
def cpu_loop_rate(fn, A, B, z, threads: int, chunk: int = 1 << 18) -> dict:
    """Arcs/s and intersections/s of a plain C loop (the step reference) over
    all arcs, split into `threads` contiguous ranges on host threads (the C
    calls release the interpreter lock, so the threads run in parallel)."""
    n = len(z)
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)

    def work(t):
        hits = 0
        for s in range(int(bounds[t]), int(bounds[t + 1]), chunk):
            e = min(int(bounds[t + 1]), s + chunk)
            c, _ = fn(A[s:e], B[s:e], z[s:e])
            hits += int(np.clip(c, 0, None).sum())
        return hits

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        hits = sum(ex.map(work, range(threads)))
    dt = time.perf_counter() - t0
    return {"value": hits / dt, "unit": UNIT, "arcs_per_s": n / dt, "cores": threads,
            "arcs": n}


def fp64_loops(stress, mixed) -> dict:
    """The paper's two FP64 forms as plain C loops (the step reference,
    gcc -O2 -ffp-contract=off): direct Eq. 2.2 and AccuX (Algorithm 8), on
    one core and on all host cores, over the whole 10^6-arc stress workload
    and over the first 10^8 arcs of the mixed workload."""
    from oracle import steps
    steps.lib()  # build outside the timing
    cores = os.cpu_count() or 1
    forms = {"direct": steps.direct, "accux": lambda A, B, z: steps.accux(A, B, z, variant=2)}
    out = {"cores": cores, "kind": "plain C loops of the step reference (gcc -O2 "
                                   "-ffp-contract=off), one arc per iteration"}
    for name, fn in forms.items():
        out[name] = {
            "stress_1e6_one_core": cpu_loop_rate(fn, *stress, threads=1),
            "stress_1e6_all_cores": cpu_loop_rate(fn, *stress, threads=cores),
            "mixed_all_cores": cpu_loop_rate(fn, *mixed, threads=cores),
        }
    out["accux_over_direct_time_one_core"] = (out["direct"]["stress_1e6_one_core"]["arcs_per_s"]
                                              / out["accux"]["stress_1e6_one_core"]["arcs_per_s"])
    return out


def cpu_oracle_leg(pool, A, B, z) -> dict:
    """The exact oracle, as it stands, on all host cores over a bounded sample."""
    cores = pool._processes
    n = min(len(z), 6000 * cores)  # ~0.6 s of oracle work per core
    oracle_rate(A[:1024], B[:1024], z[:1024], pool)  # start the workers
    a_rate, h_rate = oracle_rate(A[:n], B[:n], z[:n], pool)
    return {"value": h_rate, "unit": UNIT, "arcs_per_s": a_rate, "cores": cores,
            "kind": "oracle", "sample": f"first {n} arcs of the headline workload"}


# ------------------------------------------------------------------ GPU arm --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sphx", choices=["sphx", "reference"])
    ap.add_argument("--arcs", type=int, default=N_ARCS,
                    help="arcs per GPU of the headline workload (default: the 2x10^8 of the "
                         "precision comparison; smaller values are for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the ragged, mesh-batch and zonal legs reported beside the headline")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the headline mode on the headline workload (for profiling)")
    ap.add_argument("--mode", default="wide", choices=list(MODES),
                    help="headline evaluation mode (the others are timed beside it)")
    ap.add_argument("--zonal-only", action="store_true",
                    help="run only the zonal-mean leg and print its JSON (for profiling)")
    ap.add_argument("--ragged-only", action="store_true",
                    help="run only the cubed-sphere regridding leg and print its JSON (for profiling)")
    ap.add_argument("--meshes-only", action="store_true",
                    help="run only the 512-mesh ragged leg and print its JSON (for profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="ragged legs with the library's default launch shape (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    import multiprocessing as mp
    rank, world, local = dist_env()
    cores = max(1, (os.cpu_count() or 1) // world)
    pool = mp.get_context("spawn").Pool(cores)
    if args.zonal_only or args.ragged_only or args.meshes_only:
        import torch
        from paper_2510_09892_gb300 import sphx
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        if args.zonal_only:
            line = {"zonal_mean": zonal_leg(sphx, torch, dev, args, args.mode)}
        elif args.ragged_only:
            line = {"ragged_regridding": ragged_leg(sphx, torch, dev, args, args.mode)}
        else:
            line = {"ragged_meshes": meshes_leg(sphx, torch, dev, args, args.mode, pool)}
        pool.close()
        print(json.dumps(line), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_2510_09892_gb300 import sphx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    n = args.arcs
    seed = shard_seed(MIXED_SEED, rank)
    # the workload in page-locked host memory: the source of the device copy
    # and the host buffers of the end-to-end call
    hA = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    hB = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    hz = torch.empty((n,), dtype=torch.float64, pin_memory=True)
    t_gen = time.perf_counter()
    fill_mixed(pool, seed, hA.numpy(), hB.numpy(), hz.numpy())
    t_gen = time.perf_counter() - t_gen

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.headline_only:
        cpu = cpu_oracle_leg(pool, hA.numpy(), hB.numpy(), hz.numpy())
        stress = W.stress_arcs(STRESS_ARCS)
        m = min(n, CPU_LOOP_ARCS)
        cpu["fp64_loops"] = fp64_loops(stress, (hA.numpy()[:m], hB.numpy()[:m], hz.numpy()[:m]))
    tA, tB, tz = (t.to(dev) for t in (hA, hB, hz))
    pts = torch.empty((n, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.empty((n,), dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed(mode, steps, warmup):
        """CUDA-event times (ms) of `steps` dense calls over the whole batch on `stream`."""
        evs = []
        with torch.cuda.stream(stream):
            for i in range(warmup + steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, mode, stream)
                e1.record(stream)
                if i >= warmup:
                    evs.append((e0, e1))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def hits_of(mode):
        with torch.cuda.stream(stream):
            sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, mode, stream)
            h = int(torch.clamp(cnt, min=0).sum(dtype=torch.int64).item())
        return h

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_FP64) / 2  # FMA/s = FP64 op slots/s
    fp32_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_FP32) / 2
    int32_peak = sphx.sphx_probe_fma_rate(sphx.PIPE_INT32)
    head = args.mode
    others = [] if args.headline_only else [m for m in MODES if m != head]
    hbm_peak, hbm_src = measured_hbm_peak_src()

    # the dense grid of each mode, picked by the library's autotuner on these
    # arrays (untimed), then the warm-up steps
    dense_tuning = {}
    for mode in [head] + others:
        with torch.cuda.stream(stream):
            dense_tuning[mode] = sphx.sphx_autotune_dense(tA, tB, tz, pts, cnt, mode, stream)
        timed(mode, 1, args.warmup)
    barrier()
    torch.cuda.synchronize()
    # the sampler runs through every timed leg (headline, the other modes, e2e)
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        head_ms = timed(head, args.steps, 0)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall
        gpu_launches = args.steps  # one dense_kernel launch per step
        step_ms = reduce_max(statistics.mean(head_ms), dev)
        mode_ms = {head: step_ms}
        for mode in others:
            mode_ms[mode] = reduce_max(statistics.mean(timed(mode, args.steps, 0)), dev)
        e2e = None if args.headline_only else e2e_leg(sphx, torch, dev, hA, hB, hz, args, head)
    clk = clocks.summary()
    clk["window"] = "the timed steps of every mode and the end-to-end leg"

    modes = {}
    for mode, ms in mode_ms.items():
        h = hits_of(mode)
        hits_all = reduce_sum(h, dev)
        modes[mode] = {"value": hits_all / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                       "arcs_per_s": world * n / (ms * 1e-3), "hits_per_step": h,
                       "hbm_frac": BYTES_PER_ARC * n / (ms * 1e-3) / 1e9 / hbm_peak,
                       "error": ERROR[mode]}
        # the FP64 and FP32 pipes' rooflines: ops per arc x arcs/s against the
        # probes' FMA rates (one op per slot), with the source of the op counts
        if mode in FP64_OPS_PER_ARC:
            modes[mode]["fp64_pipe_frac"] = FP64_OPS_PER_ARC[mode] * n / (ms * 1e-3) / fp64_peak
        if mode in FP32_OPS_PER_ARC:
            modes[mode]["fp32_pipe_frac"] = FP32_OPS_PER_ARC[mode] * n / (ms * 1e-3) / fp32_peak
        modes[mode]["ops_source"] = OPS_SOURCE
    value = modes[head]["value"]
    if e2e is not None:
        e2e["value"] = reduce_sum(e2e["hits_per_step"], dev) / (e2e["ms_per_step"] * 1e-3)

    head_kernel_ms = statistics.mean(head_ms)
    gbs = BYTES_PER_ARC * n / (head_kernel_ms * 1e-3) / 1e9
    tpa = TRAFFIC_PER_ARC.get(head)
    roofline = {"bound": "hbm", "unit": "GB/s", "achieved": gbs, "peak": hbm_peak,
                "frac": gbs / hbm_peak, "traffic": None if tpa is None else tpa["value"] * n,
                "kernel": f"dense_pf_kernel<{head}>", "launch_ms": head_kernel_ms,
                "per_unit": f"{BYTES_PER_ARC} B per arc (56 in, 48 points + 4 count out) x "
                            f"{n} arcs per launch",
                "peak_source": hbm_src}
    if tpa is not None:
        roofline["traffic_source"] = tpa["source"]
    issue_peak = ISSUE_SLOTS_PER_SM_CLK * sm_count * SM_MAX_MHZ * 1e6
    roofline_issue = None
    if head in INST_PER_ARC:
        ipa = INST_PER_ARC[head]
        rate = ipa["value"] * n / (head_kernel_ms * 1e-3)
        roofline_issue = {"bound": "alu", "unit": "T instructions/s", "achieved": rate / 1e12,
                          "peak": issue_peak / 1e12, "frac": rate / issue_peak,
                          "instructions_per_arc": ipa["value"], "source": ipa["source"],
                          "peak_source": "4 warp instructions x 32 lanes x SMs x the 2070 MHz "
                                         "maximum SM clock (derived)"}
    if rank != 0:
        pool.close()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "ms_per_step_stats": {"mean": statistics.mean(head_ms),
                              "median": statistics.median(head_ms), "best": min(head_ms),
                              "worst": max(head_ms), "steps": len(head_ms),
                              "note": "this rank's CUDA-event times of the timed steps"},
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": config_dict(args, head), "arcs_per_s": modes[head]["arcs_per_s"],
        "hits_per_step": modes[head]["hits_per_step"], "e2e": e2e, "gpu_launches": gpu_launches,
        "clocks": clk, "roofline": roofline, "roofline_issue": roofline_issue,
        "modes": modes,
        "eft_over_direct_time": (modes["eft"]["ms_per_step"] / modes["direct"]["ms_per_step"]
                                 if "eft" in modes and "direct" in modes else None),
        "timed_wall_s": t_wall, "generate_s": t_gen,
        "dense_autotune_best_ms": dense_tuning,
        "peaks": {"fp64_fma_per_s": fp64_peak, "fp32_fma_per_s": fp32_peak,
                  "int32_imad_per_s": int32_peak, "hbm_gbs": hbm_peak, "hbm_source": hbm_src},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if not args.headline_only:
        del tA, tB, tz, pts, cnt
        torch.cuda.empty_cache()
        line["stress_1e6"] = stress_leg(sphx, torch, dev, args)
        line["arc_x_arc"] = arcs_leg(sphx, torch, dev, args)
        line["adaptive_filter"] = adaptive_leg(sphx, torch, dev, args)
        if not args.no_ragged:
            line["ragged_regridding"] = ragged_leg(sphx, torch, dev, args, head)
            line["zonal_mean"] = zonal_leg(sphx, torch, dev, args, head)
            line["ragged_meshes"] = meshes_leg(sphx, torch, dev, args, head, pool)
    pool.close()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def reduce_sum(value: int, device=None) -> int:
    """Sum of an integer over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return int(value)
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def _flushed_times(torch, dev, flush, call, steps, warmup):
    cur = torch.cuda.current_stream(dev)
    evs = []
    for i in range(warmup + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        call(cur)
        e1.record(cur)
        if i >= warmup:
            evs.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def stress_leg(sphx, torch, dev, args) -> dict:
    """The 10^6-arc ill-conditioned workload (not the headline): each mode's
    dense call timed with CUDA events, the L2 cache flushed (a 256 MiB write)
    before each call."""
    A, B, z = W.stress_arcs(STRESS_ARCS)
    tA, tB, tz = (torch.from_numpy(v).to(dev) for v in (A, B, z))
    pts = torch.empty((STRESS_ARCS, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.empty((STRESS_ARCS,), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    res = {"workload": STRESS_WORKLOAD, "arcs": STRESS_ARCS,
           "l2": "flushed between timed steps (256 MiB write)", "modes": {}}
    for mode in MODES:
        ms = _flushed_times(torch, dev, flush, lambda s, m=mode: sphx.sphx_intersect_gca_constlat(
            tA, tB, tz, pts, cnt, m, s), args.steps, args.warmup)
        hits = int(torch.clamp(cnt, min=0).sum().item())
        res["modes"][mode] = {"ms_per_step": ms, "value": hits / (ms * 1e-3), "unit": UNIT,
                              "arcs_per_s": STRESS_ARCS / (ms * 1e-3), "hits_per_step": hits,
                              "hbm_frac": BYTES_PER_ARC * STRESS_ARCS / (ms * 1e-3) / 1e9
                              / measured_hbm_peak()}
    return res


def arcs_leg(sphx, torch, dev, args) -> dict:
    """Arc x arc intersections (not the headline): 10^6 pairs of great circle
    arcs (50 % uniform, 15 % short, 15 % nearly parallel circles, 10 % crossings
    near an endpoint, 10 % misses), each mode timed with CUDA events over
    `steps` calls, the L2 cache flushed before each."""
    A1, A2, B1, B2 = W.arc_pairs(1_000_000)
    t = [torch.from_numpy(v).to(dev) for v in (A1, A2, B1, B2)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
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


def adaptive_leg(sphx, torch, dev, args) -> dict:
    """The adaptive filter (not the headline): on the 10^6 stress arcs and on
    10^6 well-conditioned arcs (uniform endpoints, arc length uniform in
    (0, pi/2), one latitude inside each arc's z-range), the time per dense call
    of the adaptive mode beside the integer-limb and direct FP64 forms, and the
    share of arcs the filter hands on to the integer-limb form."""
    cur = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    res = {"workloads": {}}
    for name in ("stress", "uniform"):
        A, B, z = (W.stress_arcs(STRESS_ARCS) if name == "stress"
                   else W.uniform_arcs(STRESS_ARCS, seed=W.DEFAULT_SEED + 5))
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
            tune_ms = None if args.no_autotune else sphx.sphx_autotune_ragged(
                ctx, d["A"], d["B"], d["eo"], d["lat"], d["lo"], out, total, mode, stream=cur)
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
            tune_ms = None if args.no_autotune else sphx.sphx_autotune_ragged(
                ctx, tA, tB, teo, tlat, tlo, out, total, mode, stream=cur)
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


def measured_hbm_peak_src() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "6.8 TB/s, the profiling recipe's fallback (of fallback)"


def measured_hbm_peak() -> float:
    return measured_hbm_peak_src()[0]


def e2e_leg(sphx, torch, dev, hA, hB, hz, args, mode) -> dict:
    """Same metric through the C ABI from page-locked HOST buffers
    (sphx_intersect_gca_constlat_host): every step moves the inputs in and the
    points and counts out; with page-locked buffers the kernel reads and writes
    host memory in place, so the transfers overlap the arithmetic."""
    n = len(hz)
    hP = torch.empty((n, 2, 3), dtype=torch.float64, pin_memory=True)
    hC = torch.empty((n,), dtype=torch.int32, pin_memory=True)
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
    hits = int(np.clip(hC.numpy(), 0, None).sum())
    del hP, hC
    return {"value": None, "unit": UNIT, "ms_per_step": ms, "hits_per_step": hits,
            "arcs_per_s": world * n / (ms * 1e-3),
            "h2d_bytes_per_step": n * 56, "d2h_bytes_per_step": n * 52,
            "path": "sphx_intersect_gca_constlat_host, page-locked host buffers (read and "
                    "written in place by the kernel over NVLink-C2C)"}


if __name__ == "__main__":
    main()
