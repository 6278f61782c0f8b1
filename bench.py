#!/usr/bin/env python3
"""Benchmark of the demag + LLG step on the 256x256x4 film.

Workload (the size-sweep film at 256x256x4): 4 nm cubic cells, Ms 8.6e5 A/m,
A 1.3e-11 J/m, Ku 5e2 J/m^3 (easy x), alpha 0.02, gamma_0 2.211e5, uniform
+x start, H_ext 2.5e4 A/m at 170 degrees in the xy plane, Euler dt 5e-14 s.
Synthetic data: the paper's own workload (muMAG standard problem 3) is not
reproduced; the seeded film stands in for it.

A step is one forward-Euler step (x R2C -> y/z FFT + tensor product ->
x C2R + field + LLG + Euler), i.e. one demag evaluation plus the update.
Every timed step starts with a cold L2: a 256 MiB buffer is overwritten
before it (outside the CUDA-event bracket).  `value` is cells*steps/s over
all ranks (replicas only: each rank integrates its own film; there is no
data-path collective).

--impl reference times the FP64 numpy oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = (256, 256, 4)
METRIC = "cells·steps/s and demag evals/s at 256×256×4; HBM GB/s fraction; vs oracle"
UNIT = "cells·steps/s"
FLUSH_BYTES = 256 << 20


def workload():
    from paper_1406_7459_gb300 import inputs
    w = dict(inputs.FILM_SWEEP)
    w["grid"] = GRID
    return w


def config_dict():
    w = workload()
    return {
        "workload": "film 256x256x4, 4 nm cells, Ku 5e2 easy x, alpha 0.02, uniform +x start, "
                    "H_ext 2.5e4 A/m at 170 deg, Euler dt 5e-14 s",
        "grid": list(GRID), "cell_m": list(w["cell"]), "padded": [512, 512, 8],
        "l2": "flushed before every timed step (256 MiB write)",
        "parallelism": "replicas",
    }


def algorithmic_bytes(grid):
    """Bytes each kernel must move at least once, FP32 SoA M (12 B/cell),
    complex64 x half-spectrum X = (Lx/2+1)*ny*nz per component (24 B per
    X element for three components).
    Three-pass model (the generic path and the reference accounting):
      pass 1 12N + 24X, plane 48X + 24Ks, pass 3 24X + 24N,
      Ks = (Lx/2+1)(Ly/2+1)(Lz/2+1) octant bins x 6 floats.
    Two-kernel power-of-two step (this benchmark):
      K_A plane 48X + 24Kd, K_B x-step 48X + 24N,
      Kd = (Lx/2+1)(Ly/2+1) nz coupling sets x 6 floats.
    Compulsory floor: M in and out (24N) plus the tensor spectrum once."""
    nx, ny, nz = grid
    L = [1 if n == 1 else 2 * n for n in grid]     # power-of-two grids here
    N = nx * ny * nz
    X = (L[0] // 2 + 1) * ny * nz
    Ks = (L[0] // 2 + 1) * (L[1] // 2 + 1) * (L[2] // 2 + 1)
    Kd = (L[0] // 2 + 1) * (L[1] // 2 + 1) * nz
    return {"pass1": 12 * N + 24 * X, "plane3": 48 * X + 24 * Ks, "pass3": 24 * X + 24 * N,
            "step3": 36 * N + 96 * X + 24 * Ks,
            "kA": 48 * X + 24 * Kd, "kB": 48 * X + 24 * N, "step2": 24 * N + 96 * X + 24 * Kd,
            "demag": 24 * N + 96 * X + 24 * Ks,
            "floor2": 24 * N + 24 * Kd, "floor3": 24 * N + 24 * Ks}


def algorithmic_flops(grid):
    """Nominal FP32 flops of one two-kernel step, counting a complex FFT of
    length n as 5 n log2 n and a pruned (zero-padded) transform of length 2n
    as two of length n:
      x forward and inverse: 3 ny nz / 2 row pairs, one pruned length-2nx
        transform each; y forward and inverse: 3 nz (nx + 1) lines of
        pruned length 2ny; direct z sum: 9 nz^2 complex-by-real
        multiply-adds (4 flops) per (kx, ky) bin of (nx + 1) x 2ny;
      field + LLG + Euler + renormalisation: 100 flops per cell."""
    import math
    nx, ny, nz = grid
    fft = lambda n: 5.0 * n * math.log2(n) if n > 1 else 0.0
    x = 2 * (3 * ny * nz / 2) * 2 * fft(nx)
    y = 2 * (3 * nz * (nx + 1)) * 2 * fft(ny)
    z = (nx + 1) * 2 * ny * 9 * nz * nz * 4
    return x + y + z + 100.0 * nx * ny * nz


def alu_peak_tflops(sm_mhz):
    """FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# Sources of the two step kernels: the DRAM traffic recorded under profiles/
# is reported only while these files hash to the value recorded with it.
STEP_KERNEL_SOURCES = ("fast_step.cuh", "fast_fft.cuh", "fft_device.cuh", "fast_passes.cuh", "bulk_copy.cuh",
                       "fast_step_x.cu", "fast_step_plane_a.cu", "fast_step_plane_b.cu")


def step_kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1406_7459_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, prof=None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when that capture was taken on other kernel sources."""
    prof = prof or os.path.join(ROOT, "profiles", "traffic_256x256x4.txt")
    try:
        rec = json.load(open(prof))
    except Exception:
        return None
    if rec.get("kernel_sources_sha16") != step_kernel_hash():
        return None
    return rec.get(kernel)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        # raw samples go to MM_CLOCKS_CSV when set, else to a temporary file
        # removed after parsing; the summary is part of the JSON line
        self.keep = bool(os.environ.get("MM_CLOCKS_CSV"))
        if self.keep:
            self.path = os.environ["MM_CLOCKS_CSV"]
        else:
            fd, self.path = tempfile.mkstemp(prefix="mm_clocks_", suffix=".csv")
            os.close(fd)
        self.fh = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.fh:
                self.fh.close()
            if not self.keep and os.path.exists(self.path):
                os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not self.keep:
            os.remove(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n, rank, ws):
    """Round-robin share of n independent samples for one rank (the samples
    are of uneven size; interleaving balances the ranks' cell counts)."""
    return list(range(rank, n, ws))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rate(seconds_budget=15.0, max_steps=None, workers=1):
    """Time the FP64 numpy oracle's Euler step on the same workload, on a
    bounded number of steps, with `workers` host threads for its demag
    evaluation (transforms and tensor product); returns
    (cells*steps/s, steps, seconds)."""
    from oracle import tensor as T, demag as D, llg as L
    from paper_1406_7459_gb300 import inputs
    w = workload()
    Lp = D.default_lengths(GRID)
    Kt = D.kernel_spectrum(T.tensor_octant(GRID, w["cell"]), Lp)
    M = inputs.uniform_m(GRID, w["Ms"], w["start"]).astype(np.float64)
    args = (w["dt"], w["cell"], w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"], w["H_ext"], Kt, Lp)
    prev = D.get_workers()
    D.set_workers(workers)
    try:
        M, _ = L.euler_step(M, *args)                # warm-up
        n, t0 = 0, time.perf_counter()
        while True:
            M, _ = L.euler_step(M, *args)
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds_budget or (max_steps and n >= max_steps):
                break
    finally:
        D.set_workers(prev)
    N = GRID[0] * GRID[1] * GRID[2]
    return N * n / el, n, el


def cpu_baseline_line(seconds_budget, max_steps=None):
    """The oracle on all host cores (the reported baseline) and on one core
    (beside it), each on a bounded sample of the same workload."""
    cores = host_cores()
    rate, n, el = oracle_rate(seconds_budget=seconds_budget, max_steps=max_steps, workers=cores)
    r1, n1, el1 = oracle_rate(seconds_budget=max(2.0, seconds_budget / 3), max_steps=max_steps, workers=1)
    return {"kind": "oracle", "value": rate, "unit": UNIT, "cores": cores,
            "sample": "%d FP64 Euler steps of the full 256x256x4 film (%.1f s) with %d host threads "
                      "(scipy.fft workers and a thread pool over the tensor product; the field "
                      "terms single-threaded numpy)" % (n, el, cores),
            "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                            "sample": "%d FP64 Euler steps (%.1f s), numpy FFT, one thread" % (n1, el1)}}


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    budget = args.ref_seconds if args.ref_seconds else min(120.0, max(10.0, 0.1 * args.steps))
    cb = cpu_baseline_line(budget, max_steps=args.steps)
    rate = cb["value"]
    N = GRID[0] * GRID[1] * GRID[2]
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * N / rate,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(),
        "cpu_baseline": cb,
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args, rank, ws):
    import torch
    from paper_1406_7459_gb300 import mm, inputs
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    w = workload()
    N = GRID[0] * GRID[1] * GRID[2]
    ctx = mm.mm_create(GRID, w["cell"], w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"])
    mm.mm_set_step_path(ctx, {"auto": mm.MM_STEP_AUTO, "graph": mm.MM_STEP_GRAPH,
                              "persistent": mm.MM_STEP_PERSISTENT}[args.step_path])
    step_path = "persistent" if mm.mm_get_step_path(ctx) == mm.MM_STEP_PERSISTENT else "graph"
    if args.tiled_copies:
        mm.mm_set_tiled_copies(ctx, args.tiled_copies)
    mm.mm_set_field(ctx, w["H_ext"])
    M0 = inputs.uniform_m(GRID, w["Ms"], w["start"]).reshape(-1)
    mm.mm_set_m(ctx, torch.from_numpy(M0).cuda())
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dt = w["dt"]
    K, W = args.steps, args.warmup

    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    sampler = ClockSampler(vis[local] if local < len(vis) else local)     # nvidia-smi numbering
    sampler.start()
    mm.mm_step(ctx, max(W, 3), dt)                   # warm-up (graph capture)
    torch.cuda.synchronize()
    # keep the clocks busy ~1 s so the sampler sees the load
    t_end = time.perf_counter() + (0.0 if args.quick else 1.0)
    while time.perf_counter() < t_end:
        mm.mm_step(ctx, 50, dt)
        torch.cuda.synchronize()

    # --- timed region: K steps, cold L2 before each, events around each step
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    barrier(ws)
    torch.cuda.synchronize()
    for s in range(K):
        flush.fill_(float(s))
        starts[s].record()
        mm.mm_step(ctx, 1, dt)
        ends[s].record()
    torch.cuda.synchronize()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    mm.mm_sync(ctx)

    # --- per-kernel durations (same cold-L2 protocol, kernels launched one
    # by one without programmatic overlap), for the roofline
    reps = min(K, 200)
    p1, p2, p3 = mm.mm_time_passes(ctx, reps, dt, flush)

    # --- demag evaluations per second (cold L2 per evaluation)
    Md = torch.empty(3 * N, device="cuda")
    mm.mm_get_m(ctx, Md)
    Hd = torch.empty_like(Md)
    de_s = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    de_e = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for s in range(reps):
        flush.fill_(float(s))
        de_s[s].record()
        mm.mm_demag_field(ctx, Md, Hd)
        de_e[s].record()
    torch.cuda.synchronize()
    demag_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(de_s, de_e))

    # --- steady state without flushing (L2-resident working set), context only;
    # long runs go through the multi-step graphs (captured here, both parities)
    for n_warm in (16, 1, 16):
        mm.mm_step(ctx, n_warm, dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mm.mm_step(ctx, K, dt)
    e1.record()
    torch.cuda.synchronize()
    warm_ms = e0.elapsed_time(e1) / K

    # --- context for the per-step number: what the same event pair costs
    # around one tiny kernel after the flush, and steps timed 16 per call
    # (L2 flushed before each call; the working set stays in L2 within it)
    tiny = torch.zeros(1, device="cuda")
    fa = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    fb = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for s in range(reps):
        flush.fill_(float(s))
        fa[s].record()
        tiny.zero_()
        fb[s].record()
    torch.cuda.synchronize()
    floor_us = 1e3 * statistics.mean(a.elapsed_time(b) for a, b in zip(fa, fb))
    r16 = min(K, 50)
    for s in range(r16):
        flush.fill_(float(s))
        fa[s].record()
        mm.mm_step(ctx, 16, dt)
        fb[s].record()
    torch.cuda.synchronize()
    call16_ms = statistics.mean(fa[s].elapsed_time(fb[s]) for s in range(r16)) / 16

    # --- end to end through the C ABI with host buffers
    Mh = torch.from_numpy(M0.copy()).pin_memory()
    Mo = torch.empty_like(Mh).pin_memory()
    ke = min(K, 200)
    e2e_t = 0.0
    for s in range(ke):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # one step of a host-resident state: its first kernel reads the
        # pinned input over the host link, its last writes the result back
        mm.mm_step_host(ctx, Mh, 1, dt, Mo)
        e2e_t += time.perf_counter() - t0
    # where an end-to-end call's time goes (context; after the e2e leg, so
    # that its timing is not perturbed): CUDA events on the context's stream
    # just before and after the call against its wall clock, and the same
    # step through device buffers
    kb = min(K, 50)
    span, wall, dev = [], [], []
    Md2 = torch.empty(3 * N, device="cuda")
    for s in range(kb):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ea.record()
        mm.mm_step_host(ctx, Mh, 1, dt, Mo)
        eb.record()
        wall.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
        span.append(ea.elapsed_time(eb) * 1e-3)
    Mdev = torch.from_numpy(M0.copy()).cuda()
    for s in range(kb):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mm.mm_set_m(ctx, Mdev)
        mm.mm_step(ctx, 1, dt)
        mm.mm_get_m(ctx, Md2)
        mm.mm_sync(ctx)
        dev.append(time.perf_counter() - t0)
    e2e_breakdown = {"calls": kb, "wall_us_median": 1e6 * statistics.median(wall),
                     "event_span_us_median": 1e6 * statistics.median(span),
                     "device_buffers_call_us_median": 1e6 * statistics.median(dev),
                     "what": "one mm_step_host call: wall clock, and CUDA events on its stream around it; "
                             "device buffers: mm_set_m + mm_step + mm_get_m + mm_sync from device memory"}
    clocks = sampler.stop()

    t_max = max_over_ranks(t_local, ws)
    e2e_max = max_over_ranks(e2e_t, ws)
    value = ws * N * K / t_max
    by = algorithmic_bytes(GRID)
    peak, peak_kind = measured_peaks()
    _, launches = mm.mm_plan_info(ctx)
    if launches == 2:
        passes = {"pass1_x_r2c_first_step_only": p1, "kA_plane_y_zsum_product": p2,
                  "kB_x_c2r_llg_euler_x_r2c": p3}
        kbytes = {"kA_plane_y_zsum_product": by["kA"], "kB_x_c2r_llg_euler_x_r2c": by["kB"]}
        step_bytes = by["step2"]
    else:
        passes = {"pass1_x_r2c": p1, "pass2_yz_plane": p2, "pass3_x_c2r_llg": p3}
        kbytes = {"pass1_x_r2c": by["pass1"], "pass2_yz_plane": by["plane3"], "pass3_x_c2r_llg": by["pass3"]}
        step_bytes = by["step3"]
    dom = max(kbytes, key=lambda k: passes[k])
    achieved = kbytes[dom] / (passes[dom] * 1e-3) / 1e9
    traffic = recorded_traffic(dom)
    step_ms_mean = 1e3 * t_max / K
    flops = algorithmic_flops(GRID)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu = {"flops_per_step": flops, "model": "two-kernel, 5 n log2 n per length-n FFT",
           "achieved_tflops": flops / (step_ms_mean * 1e-3) / 1e12,
           "peak_tflops": alu_peak_tflops(sm_mhz), "peak_basis": "152 SMs x 128 FP32 lanes x 2 x %g MHz" % sm_mhz}
    alu["frac"] = alu["achieved_tflops"] / alu["peak_tflops"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": step_ms_mean, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(),
        "demag_evals_per_s": ws * 1e3 / demag_ms,
        "step_hbm": {"algorithmic_bytes": step_bytes, "model": "two-kernel" if launches == 2 else "three-pass",
                     "gbs": step_bytes / (step_ms_mean * 1e-3) / 1e9,
                     "frac": step_bytes / (step_ms_mean * 1e-3) / 1e9 / peak,
                     "three_pass_model_bytes": by["step3"],
                     "three_pass_model_frac": by["step3"] / (step_ms_mean * 1e-3) / 1e9 / peak},
        "compulsory_bytes": {"bytes": by["floor2"] if launches == 2 else by["floor3"],
                             "what": "M in + M out + tensor spectrum in",
                             "frac_at_step_time": None},
        "alu": alu,
        "pass_ms": passes,
        "launches_per_step": launches if step_path == "graph" else "one launch per mm_step call",
        "step_path": step_path,
        "xstep_tiled_copies": mm.mm_get_tiled_copies(ctx),
        "steady_state_l2_resident": {"ms_per_step": warm_ms, "cells_steps_per_s": ws * N / (warm_ms * 1e-3)},
        "timing_context": {
            "event_pair_around_tiny_kernel_after_flush_us": floor_us,
            "flushed_16_step_calls": {"ms_per_step": call16_ms, "cells_steps_per_s": ws * N / (call16_ms * 1e-3),
                                      "what": "L2 flushed before each mm_step(ctx, 16) call, events around the call"}},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": kbytes[dom]},
        "gpu_launches": launches * K if step_path == "graph" else K,
        "clocks": clocks,
        "e2e": {"value": ws * N * ke / e2e_max, "unit": UNIT, "h2d_bytes_per_step": 12 * N,
                "d2h_bytes_per_step": 12 * N},
        "e2e_breakdown": e2e_breakdown,
    }
    cb = line["compulsory_bytes"]
    cb["frac_at_step_time"] = cb["bytes"] / (step_ms_mean * 1e-3) / 1e9 / peak
    if rank == 0 and ws == 1 and not (args.no_cpu_baseline or args.quick):
        line["cpu_baseline"] = cpu_baseline_line(args.cpu_seconds)
    mm.mm_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_sweep(args, rank, ws):
    """The film size sweep (64x64x4 ... 512x512x8, 200x60x3, plus the
    512x512x4 and 1024x1024x1 films): per grid the Euler step with the L2
    flushed before every timed step, the step with the working set left in
    L2 (one graph of many steps), and one demag evaluation after a flush."""
    import torch
    from paper_1406_7459_gb300 import mm, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = inputs.FILM_SWEEP
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    grids = list(inputs.FILM_SWEEP_GRIDS) + [(512, 512, 4), (1024, 1024, 1)]
    if args.sweep_grid:
        grids = [tuple(int(v) for v in g.split("x")) for g in args.sweep_grid.split(",")]
    K = max(20, min(args.steps, 200))

    def flushed(fn, reps):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for r in range(reps):
            flush.fill_(float(r))
            st[r].record()
            fn()
            en[r].record()
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in zip(st, en)) * 1e3

    points = []
    for grid in grids:
        n = grid[0] * grid[1] * grid[2]
        ctx = mm.mm_create(grid, w["cell"], w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"])
        mm.mm_set_m(ctx, torch.from_numpy(inputs.uniform_m(grid, w["Ms"], w["start"]).reshape(-1)).cuda())
        mm.mm_set_field(ctx, w["H_ext"])
        mm.mm_step(ctx, max(args.warmup, 3) + 32, w["dt"])
        torch.cuda.synchronize()
        step_us = flushed(lambda: mm.mm_step(ctx, 1, w["dt"]), K)
        mm.mm_step(ctx, 33, w["dt"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mm.mm_step(ctx, 320, w["dt"])
        e1.record()
        torch.cuda.synchronize()
        l2_us = e0.elapsed_time(e1) * 1e3 / 320
        Md = torch.empty(3 * n, device="cuda")
        mm.mm_get_m(ctx, Md)
        Hd = torch.empty_like(Md)
        demag_us = flushed(lambda: mm.mm_demag_field(ctx, Md, Hd), 50)
        points.append({"grid": list(grid), "launches_per_step": mm.mm_plan_info(ctx)[1],
                       "step_us_flushed": step_us, "cells_steps_per_s": n / (step_us * 1e-6),
                       "step_us_l2_resident": l2_us, "demag_us_flushed": demag_us})
        mm.mm_destroy(ctx)
    if rank == 0:
        print(json.dumps({"workload": "film size sweep, 4 nm cells, Ku 5e2 easy x, alpha 0.02, uniform +x start, "
                                      "H_ext 2.5e4 A/m at 170 deg, Euler dt 5e-14 s",
                          "metric": "us per Euler step / per demag evaluation", "dtype": "f32",
                          "data": "synthetic", "l2": "flushed (256 MiB write) before every flushed timing",
                          "points": points}))
    return 0


def run_cube(args, rank, ws):
    """Per-step time of the N^3 cube (N = 8..128) beside the paper's Table 1
    (context only: other hardware, other precision, a graphics-API path)."""
    import torch
    from paper_1406_7459_gb300 import mm, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = inputs.CUBE
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_table1.json")))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    points = []
    sizes = inputs.CUBE_SIZES if not args.cube_n else [int(v) for v in args.cube_n.split(",")]
    for n in sizes:
        if n not in inputs.CUBE_SIZES:
            raise SystemExit("--cube-n: %d is not one of %s" % (n, inputs.CUBE_SIZES))
        grid = (n, n, n)
        ctx = mm.mm_create(grid, w["cell"], w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"])
        mm.mm_set_m(ctx, torch.from_numpy(inputs.random_unit_m(grid, w["Ms"], w["seed"]).reshape(-1)).cuda())
        mm.mm_step(ctx, max(args.warmup, 3), w["dt"])
        torch.cuda.synchronize()
        K = max(20, min(args.steps, 200))
        tot = 0.0
        for s in range(K):
            flush.fill_(float(s))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            mm.mm_step(ctx, 1, w["dt"])
            b.record()
            b.synchronize()
            tot += a.elapsed_time(b)
        mm.mm_sync(ctx)
        ms = tot / K
        i = table["N"].index(n)
        points.append({"N": n, "cells": n ** 3, "ms_per_step": ms, "cells_steps_per_s": n ** 3 / (ms * 1e-3),
                       "launches_per_step": mm.mm_plan_info(ctx)[1],
                       "paper_gpu_ms": table["gpu_ms"][i], "paper_cpu_ms": table["cpu_ms"][i],
                       "vs_paper_gpu": table["gpu_ms"][i] / ms})
        mm.mm_destroy(ctx)
    if rank == 0:
        print(json.dumps({"workload": "cube N^3, 4 nm cells, Ku 5e2 easy x, alpha 0.5, random start, Euler "
                                      "dt 5e-14 s, L2 flushed before every timed step",
                          "metric": "ms per Euler step", "dtype": "f32", "data": "synthetic",
                          "points": points,
                          "paper_context": table["source"] + "; " + table["hardware"]["gpu"]}))
    return 0


def run_batch(args, rank, ws):
    """512 independent samples of uneven size (nx 16..256, ny 16..64,
    nz 1..2, random Ku, H_ext, alpha) stepped as one batch after the tile
    autotuner, against the same samples stepped one context at a time.  The
    batch working set (~0.7 GB) exceeds L2, so steps run back to back.
    Under torchrun each rank takes a round-robin share of the samples (no
    data-path collective; the ranks' cell counts are summed and their
    times max-reduced on the host)."""
    import torch
    from paper_1406_7459_gb300 import mm, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    samples = [inputs.batch_samples(512, seed=3)[i] for i in shard(512, rank, ws)]
    dt = 5e-14
    b = mm.mm_batch_create([s["grid"] for s in samples], [s["cell"] for s in samples],
                           [s["Ms"] for s in samples], [s["A"] for s in samples], [s["Ku"] for s in samples],
                           [s["alpha"] for s in samples], [s["gamma"] for s in samples])
    mm.mm_batch_set_field(b, [s["H_ext"] for s in samples])
    M = np.concatenate([s["M"].reshape(-1) for s in samples])
    mm.mm_batch_set_m(b, torch.from_numpy(M).cuda())
    choice, tune_ms = mm.mm_batch_autotune(b, dt)
    cells = mm.mm_batch_cells(b)
    K = max(10, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    path_ms, forms = {}, {}
    for name, path in (("graph", mm.MM_STEP_GRAPH), ("persistent", mm.MM_STEP_PERSISTENT)):
        mm.mm_batch_set_path(b, path)
        mm.mm_batch_step(b, max(args.warmup, 3), dt)
        barrier(ws)
        torch.cuda.synchronize()
        e0.record()
        mm.mm_batch_step(b, K, dt)
        e1.record()
        torch.cuda.synchronize()
        barrier(ws)
        mm.mm_batch_sync(b)
        path_ms[name] = max_over_ranks(e0.elapsed_time(e1) / K, ws)
        forms[name] = {0: "batched kernels replayed from a CUDA graph", 1: "one cooperative launch replayed from a CUDA graph",
                       2: "one cooperative launch issued directly"}.get(mm.mm_batch_launch_form(b), "?")
    batch_ms = path_ms["graph"]
    by = batch_bytes([s["grid"] for s in samples])
    by = {k: sum_over_ranks(float(v), ws) for k, v in by.items()}
    peak, peak_kind = measured_peaks()
    cells = int(sum_over_ranks(float(cells), ws))
    # the same samples, one context each, stepped one after another
    ctxs = []
    for s in samples:
        c = mm.mm_create(s["grid"], s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"], s["gamma"])
        mm.mm_set_field(c, s["H_ext"])
        mm.mm_set_m(c, torch.from_numpy(s["M"].reshape(-1)).cuda())
        mm.mm_step(c, 3, dt)
        ctxs.append(c)
    torch.cuda.synchronize()
    Ks = max(5, K // 10)
    e0.record()
    for _ in range(Ks):
        for c in ctxs:
            mm.mm_step(c, 1, dt)
    e1.record()
    torch.cuda.synchronize()
    single_ms = max_over_ranks(e0.elapsed_time(e1) / Ks, ws)
    for c in ctxs:
        mm.mm_destroy(c)
    if rank == 0:
        print(json.dumps({"workload": "batch of 512 samples, nx 16..256, ny 16..64, nz 1..2, Ku U[0,1e4], "
                                      "|H_ext| U[0,5e4] random direction, alpha U[0.01,0.5], Euler dt 5e-14 s",
                          "metric": "cells*steps/s over the batch", "dtype": "f32", "data": "synthetic",
                          "n_gpus": ws, "sharding": "round-robin samples per rank, no data-path collective",
                          "cells": cells, "batched_ms_per_step": batch_ms,
                          "batched_cells_steps_per_s": cells / (batch_ms * 1e-3),
                          "paths": {name: {"ms_per_step": ms, "cells_steps_per_s": cells / (ms * 1e-3),
                                           "algorithmic_bytes_per_step": by[name],
                                           "hbm_gbs": by[name] / (ms * 1e-3) / 1e9,
                                           "hbm_frac": by[name] / (ms * 1e-3) / 1e9 / peak,
                                           "launch": forms[name]}
                                    for name, ms in path_ms.items()},
                          "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
                          "byte_model": "per sample 24N + 96X + 24Ks (plane pass; update with the next x R2C "
                                        "fused); X = (Lx/2+1) ny nz, Ks = (Lx/2+1)(Ly/2+1)(Lz/2+1), FP32",
                          "one_context_at_a_time_ms_per_step": single_ms,
                          "one_context_at_a_time_cells_steps_per_s": cells / (single_ms * 1e-3),
                          "batching_gain": single_ms / batch_ms,
                          "autotune_choice": {"rows_pass1": choice[0], "rows_pass3": choice[1],
                                              "threads": choice[2], "planes_per_cta": choice[3]},
                          "autotune_ms_per_candidate": tune_ms,
                          "l2": "working set larger than L2; steps back to back"}))
    return 0


def padded_length(n):
    """The plan's padded FFT length: 1 for n = 1, 2n for a power of two,
    else the smallest 2^a 3^b 5^c >= 2n - 1."""
    if n == 1:
        return 1
    if n & (n - 1) == 0:
        return 2 * n
    m = 2 * n - 1
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def batch_bytes(grids):
    """Algorithmic bytes of one batch step summed over the samples: both
    paths run the plane pass and the update with the next x R2C fused
    (24N + 96X + 24Ks); the three-pass model (36N + 96X + 24Ks) beside it."""
    tot = {"graph": 0, "persistent": 0, "three_pass": 0}
    for nx, ny, nz in grids:
        Lx, Ly, Lz = padded_length(nx), padded_length(ny), padded_length(nz)
        N = nx * ny * nz
        X = (Lx // 2 + 1) * ny * nz
        Ks = (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1)
        tot["three_pass"] += 36 * N + 96 * X + 24 * Ks
        tot["graph"] += 24 * N + 96 * X + 24 * Ks
        tot["persistent"] += 24 * N + 96 * X + 24 * Ks
    return tot


def truncation_floor(h, m):
    """Relative L2 of the part of fields h (B, 3, H, W) (torch, device)
    outside the modes an FNO spectral path with m modes can carry: ky in
    {0..m-1} U {H-m..H-1}, kx < m, and their conjugate partners."""
    import torch
    H, W = h.shape[-2:]
    hf = torch.fft.fft2(h.double())
    keep = torch.zeros((H, W), dtype=torch.bool, device=h.device)
    ky = torch.cat([torch.arange(m), torch.arange(H - m, H)]).to(h.device)
    kx = torch.arange(m, device=h.device)
    keep[ky[:, None], kx[None, :]] = True
    keep[((-ky) % H)[:, None], ((-kx) % W)[None, :]] = True
    p = hf.abs() ** 2
    return float(torch.sqrt(p[..., ~keep].sum() / p.sum()))


def run_fno(args, rank, ws):
    """The surrogate network alone (256x256 film, width 32, 16x16 modes, 4
    layers; random weights and inputs at the surrogate's input scale): one
    inference forward pass (batch 1, replayed from its graph) back to back
    and with L2 flushed before each call, and one training step (forward,
    backward, Adam) at batch 8.  The x-mode transforms (2 per layer) run on
    the tensor cores."""
    import torch
    from paper_1406_7459_gb300 import mm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    H = W = 256
    C, m, L, Bt = 32, 16, 4, 8
    f = mm.mm_fno_create(H, W, width=C, modes=m, layers=L, max_batch=Bt, seed=1)
    g = torch.Generator(device="cuda").manual_seed(5)
    x1 = 1e-2 * torch.randn(1, 3 * H * W, device="cuda", generator=g)
    y1 = torch.empty_like(x1)
    xt = 1e-2 * torch.randn(Bt, 3 * H * W, device="cuda", generator=g)
    tt = torch.randn(Bt, 3 * H * W, device="cuda", generator=g)
    K = max(10, min(args.steps, 200))
    for _ in range(max(args.warmup, 3)):
        mm.mm_fno_forward(f, x1, y1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        mm.mm_fno_forward(f, x1, y1)
    e1.record()
    torch.cuda.synchronize()
    warm_ms = e0.elapsed_time(e1) / K
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    fl = []
    for s in range(K):
        flush.fill_(float(s))
        e0.record()
        mm.mm_fno_forward(f, x1, y1)
        e1.record()
        torch.cuda.synchronize()
        fl.append(e0.elapsed_time(e1))
    for _ in range(3):
        mm.mm_fno_train_step(f, xt, tt, 1e-4)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(K):
        mm.mm_fno_train_step(f, xt, tt, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / K
    tc_flop = L * 2 * (2.0 * C * H * 2 * m * W)              # x-mode forward and inverse GEMMs
    mix_flop = L * 2.0 * C * C * H * W
    line = {"metric": "FNO forward ms (batch 1) and training step ms (batch 8)", "workload":
            "FNO surrogate network alone, 256x256, width 32, 16x16 modes, 4 layers, BF16 / FP32 accumulate",
            "forward_ms_back_to_back": warm_ms, "forward_ms_l2_flushed": statistics.mean(fl),
            "train_step_ms_batch8": train_ms, "calls": K,
            "tensor_core_gflop_per_forward": tc_flop / 1e9, "cuda_core_channel_map_gflop_per_forward": mix_flop / 1e9,
            "data": "synthetic (random weights and inputs)"}
    mm.mm_fno_destroy(f)
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_surrogate(args, rank, ws):
    """FNO surrogate of H_demag on the 256x256x1 film (5x5x3 nm cells,
    alpha 0.02, random fields and starts): width 32, 16x16 retained modes,
    4 Fourier layers, BF16 with FP32 accumulation, trained on the GPU by the
    project's kernels on 20k (dM, H_demag(dM)) pairs drawn from solver
    trajectories (targets computed by the exact FFT demag as they are
    drawn), then used between exact refreshes every 8 steps with fallback
    above a 1e-3 relative residual, against the plain exact-demag steps."""
    import torch
    from paper_1406_7459_gb300 import mm, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    grid, cell, Ms, dt = (256, 256, 1), (5e-9, 5e-9, 3e-9), 8.6e5, 5e-14
    rng = np.random.default_rng(11)
    ctx = mm.mm_create(grid, cell, Ms, 1.3e-11, 0.0, 0.02, inputs.GAMMA0)
    N3 = 3 * ctx.N
    n_traj, T = 16, 160
    states = torch.empty((n_traj, T, N3), device="cuda")
    t0 = time.perf_counter()
    for tr in range(n_traj):
        d = rng.standard_normal(3)
        mm.mm_set_field(ctx, tuple(rng.uniform(0, 5e4) * d / np.linalg.norm(d)))
        mm.mm_set_m(ctx, torch.from_numpy(inputs.perturbed_m(grid, Ms, 700 + tr, 0.3).reshape(-1)).cuda())
        mm.mm_step(ctx, 40, dt)                      # let the start settle
        for s in range(T):
            mm.mm_step(ctx, 1, dt)
            mm.mm_get_m(ctx, states[tr, s])
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    modes = 16
    f = mm.mm_fno_create(256, 256, width=32, modes=modes, layers=4, max_batch=8, seed=1)
    B, iters = 8, 2500                               # 20k pairs
    X = torch.empty((B, N3), device="cuda")
    Y = torch.empty((B, N3), device="cuda")

    def draw(trs):
        """B pairs (dM / rms(dM), H_demag(dM) / rms(dM)) from trajectories trs."""
        tr = rng.choice(trs, B)
        t = rng.integers(0, T - 8, B)
        k = rng.integers(1, 9, B)
        for q in range(B):
            dM = (states[tr[q], t[q] + k[q]] - states[tr[q], t[q]]).contiguous()
            sc = torch.sqrt(torch.mean(dM * dM))
            mm.mm_demag_field(ctx, dM, Y[q])
            Y[q] /= sc
            X[q] = dM / sc

    train_trs, held_trs = np.arange(n_traj - 2), np.arange(n_traj - 2, n_traj)
    losses, floors = [], []
    t0 = time.perf_counter()
    for it in range(iters):
        draw(train_trs)
        if it % 250 == 0:
            floors.append(truncation_floor(Y.view(B, 3, 256, 256), modes))
        lr = 2e-3 if it < 1500 else (1e-3 if it < 2200 else 3e-4)
        losses.append(mm.mm_fno_train_step(f, X, Y, lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # relative error of the trained network on pairs of held-out trajectories
    held = []
    yh = torch.empty_like(X)
    for _ in range(8):
        draw(held_trs)
        mm.mm_fno_forward(f, X, yh)
        held += [float(torch.linalg.norm(yh[q] - Y[q]) / torch.linalg.norm(Y[q])) for q in range(B)]
    # evaluation: surrogate-assisted vs plain steps from a settled state
    M0 = states[0, T // 2].clone()
    # the regime where this network stays under the gate: short steps with a
    # refresh every 2 steps (the residual grows with the increment's field)
    small = {}
    for name, fn in (("network", f), ("frozen_field", None)):
        c = mm.mm_create(grid, cell, Ms, 1.3e-11, 0.0, 0.02, inputs.GAMMA0)
        mm.mm_set_field(c, (3e4, 1e4, 0.0))
        mm.mm_set_m(c, M0)
        if fn is None:
            fn = mm.mm_fno_create(256, 256, width=32, modes=modes, layers=4, max_batch=8, seed=1)
            mm.mm_fno_set_params(fn, np.zeros(mm.mm_fno_param_count(fn), np.float32))
        small[name] = mm.mm_step_surrogate(c, fn, 64, 1e-15, refresh=2, tol=1e-3)
        mm.mm_destroy(c)
    res = {}
    for name in ("surrogate", "plain"):
        c = mm.mm_create(grid, cell, Ms, 1.3e-11, 0.0, 0.02, inputs.GAMMA0)
        mm.mm_set_field(c, (3e4, 1e4, 0.0))
        mm.mm_set_m(c, M0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if name == "surrogate":
            st = mm.mm_step_surrogate(c, f, 256, dt, refresh=8, tol=1e-3)
        else:
            mm.mm_set_integrator(c, "euler")
            for _ in range(256):
                mm.mm_step(c, 1, dt)
            st = None
        e1.record()
        torch.cuda.synchronize()
        out = torch.empty(N3, device="cuda")
        mm.mm_get_m(c, out)
        mm.mm_sync(c)
        res[name] = (out, e0.elapsed_time(e1) / 256, st)
    dsur = (res["surrogate"][0] - M0).cpu().numpy()
    dpl = (res["plain"][0] - M0).cpu().numpy()
    traj_err = float(np.linalg.norm(dsur - dpl) / np.linalg.norm(dpl))
    # the size of a k-step increment's field against the field itself: the
    # residual at a refresh is about (network error) x rho(k)
    rho = {}
    c = mm.mm_create(grid, cell, Ms, 1.3e-11, 0.0, 0.02, inputs.GAMMA0)
    mm.mm_set_field(c, (3e4, 1e4, 0.0))
    hm, hd, mk = torch.empty(N3, device="cuda"), torch.empty(N3, device="cuda"), torch.empty(N3, device="cuda")
    mm.mm_demag_field(c, M0, hm)
    for k in (1, 7):
        mm.mm_set_m(c, M0)
        mm.mm_step(c, k, dt)
        mm.mm_get_m(c, mk)
        mm.mm_demag_field(c, (mk - M0).contiguous(), hd)
        rho[k] = float(torch.linalg.norm(hd) / torch.linalg.norm(hm))
    mm.mm_destroy(c)
    # cost of one surrogate evaluation against one exact demag evaluation
    xin = X[:1].contiguous()
    yout = torch.empty_like(xin)
    Hh = torch.empty(N3, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        mm.mm_fno_forward(f, xin, yout)
    e0.record()
    for _ in range(50):
        mm.mm_fno_forward(f, xin, yout)
    e1.record()
    torch.cuda.synchronize()
    fno_ms = e0.elapsed_time(e1) / 50
    e0.record()
    for _ in range(50):
        mm.mm_demag_field(ctx, M0, Hh)
    e1.record()
    torch.cuda.synchronize()
    exact_ms = e0.elapsed_time(e1) / 50
    if rank == 0:
        print(json.dumps({
            "workload": "FNO surrogate of H_demag, film 256x256x1, 5x5x3 nm, alpha 0.02; width 32, 16x16 modes, "
                        "4 layers, BF16 / FP32 accumulate; exact refresh every 8 steps, fallback above 1e-3",
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic (solver trajectories)",
            "training": {"pairs": B * iters, "iterations": iters, "batch": B, "loss_first": losses[0],
                         "loss_last_100_mean": float(np.mean(losses[-100:])), "seconds": t_train,
                         "trajectory_generation_seconds": t_data},
            "stepping": {"surrogate_ms_per_step": res["surrogate"][1], "plain_ms_per_step": res["plain"][1],
                         "gain_surrogate_over_plain": res["plain"][1] / res["surrogate"][1],
                         "stats": res["surrogate"][2], "trajectory_change_rel_err_vs_plain": traj_err},
            "short_steps_1e-15_refresh_2": small,
            "accuracy": {"network_rel_err_held_out_median": float(np.median(held)),
                         "truncation_floor_of_targets_mean": float(np.mean(floors)),
                         "increment_field_over_field": {"1_step": rho[1], "7_steps": rho[7]},
                         "gate": 1e-3,
                         "reading": "the refresh residual is about the network error times the increment "
                                    "ratio; the gate needs network error <= gate / ratio"},
            "one_evaluation_ms": {"fno_forward": fno_ms, "exact_fft_demag": exact_ms}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="film", choices=["film", "cube", "sweep", "batch", "surrogate", "fno"],
                    help="film: the 256x256x4 benchmark line; cube: the N^3 per-step curve; "
                         "sweep: the film size sweep; "
                         "batch: 512 uneven samples batched vs one at a time; surrogate: the FNO")
    ap.add_argument("--cube-n", default="",
                    help="cube workload: comma-separated subset of the sizes (default all)")
    ap.add_argument("--sweep-grid", default="",
                    help="sweep workload: comma-separated grids NXxNYxNZ instead of the sweep's own")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="time budget of the --impl reference oracle run (default 10-120 s by --steps)")
    ap.add_argument("--quick", action="store_true",
                    help="no clock warm-up loop and no CPU baseline (deterministic launch list for ncu)")
    ap.add_argument("--tiled-copies", type=int, default=0, choices=[0, 1, 2, 3],
                    help="x-step spectrum gather (1) / scatter (2) as tiled tensor copies (film workload)")
    ap.add_argument("--step-path", default="auto", choices=["auto", "graph", "persistent"],
                    help="film workload: how mm_step runs (mm_set_step_path)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, ws = dist_setup()
    if args.impl == "reference":
        rc = run_reference(args, rank, ws)
    elif args.workload == "cube":
        rc = run_cube(args, rank, ws)
    elif args.workload == "sweep":
        rc = run_sweep(args, rank, ws)
    elif args.workload == "batch":
        rc = run_batch(args, rank, ws)
    elif args.workload == "surrogate":
        rc = run_surrogate(args, rank, ws)
    elif args.workload == "fno":
        rc = run_fno(args, rank, ws)
    else:
        rc = run_gpu(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
