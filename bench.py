#!/usr/bin/env python
"""Throughput of the handheld multi-frame super-resolution path (align + merge).

Metric: merged raw MP/s = frames x raw megapixels of the burst / seconds per step, on the
12-MP workload (8 RGGB frames of 4032x3024, 1x RGB output), seeded synthetic input.
One step = hmfsr_align_merge on one burst (the alignment, and beside it the merge's
motion-free preparation, then the robustness and the accumulation).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {hmfsr,reference}]

With N > 1 (torchrun, one process per GPU) every rank merges its own burst (replicas:
the method has no exchange step); rank 0 prints one JSON line.  `--impl reference`
times the FP64 CPU oracle on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "merged raw MP/s (frames x MP / s) at 12MP x 8, align + merge"
UNIT = "MP/s"
WORKLOAD = "12mp"
# Per output pixel and frame, the arithmetic the method defines for the accumulation, one
# FP32 instruction per add, multiply or fused multiply-add:
#   per sample (9): offset d (2), products dx^2, dx dy, dy^2 (3), the quadratic form of
#     Eq. 2 (3), its exponent scale (1), numerator and denominator sums (2)    9 x 11 = 99
#   per frame: sampling position and window centre (4), bilinear Omega: weights (6) and
#     3 entries x 4 terms (12), its inverse (5), bilinear Rhat at the pixel's weights (4),
#     Rhat applied to the three channel sums (6)                                     37
# and 9 exponentials + 1 reciprocal on the MUFU.
ACC_FP32_OPS_PER_UNIT = 136
ACC_MUFU_PER_UNIT = 10
FALLBACK_HBM_GBS = 6800.0


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of every rank's x: a step of the whole job lasts as long as its
    slowest rank.  One rank: x itself."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mps(mp_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: each of `world` ranks merges its own burst of mp_per_rank
    frames x MP per step (replicas), all in ms_per_step (the slowest rank's)."""
    return world * mp_per_rank / (ms_per_step / 1e3)


def rank_seed(rank: int) -> int:
    """Seed of the burst rank `rank` merges: every rank works on its own input."""
    import burstgen
    return burstgen.SEED_BASE + 1 + 1000 * rank


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            return None
    return None


def kernel_traffic(name: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    if not os.path.exists(path):
        return None
    try:
        js = json.load(open(path))
        src = open(os.path.join(ROOT, "paper_1905_03277_gb300", "csrc", js["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != js["source_sha256_16"]:
            return None
        return js["dram_bytes_per_launch"]
    except Exception:
        return None


def bench_config(n: int, h: int, w: int, tile: int, world: int) -> dict:
    """The workload as both arms print it."""
    return {"workload": "12mp: 8 x 4032x3024 RGGB uint16 (12-bit), 1x RGB float32 output, align + merge",
            "frames": n, "height": h, "width": w, "scale": "1/1", "tile": tile,
            "l2": "no flush: the 195 MB burst read each step is larger than L2",
            "parallelism": "replicas" if world > 1 else "single"}


def measure_pipe_peaks(dev, n_sm: int, gpu_index: int) -> dict:
    """This GPU's FP32 FMA and MUFU ex2 issue rates (hmfsr_pipe_probe, CUDA events,
    2048 threads per SM, 10 launches of ~20 ms each per pipe), with the SM clock sampled
    meanwhile.  Lane-operations per second; per SM per clock = rate / (SMs x MHz)."""
    import ctypes

    import torch

    from paper_1905_03277_gb300 import _lib
    L = _lib.load()
    sink = torch.zeros(256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, pipe, iters in (("fp32_fma", _lib.PIPE_FP32_FMA, 20000), ("mufu_ex2", _lib.PIPE_MUFU_EX2, 2500)):
        ops = ctypes.c_double()
        launch = lambda: _lib.check(L.hmfsr_pipe_probe(pipe, n_sm * 8, iters, ctypes.c_void_p(sink.data_ptr()),
                                                       ctypes.byref(ops), ctypes.c_void_p(stream.cuda_stream)),
                                    "hmfsr_pipe_probe")
        launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        with ClockSampler(gpu_index) as clk:
            e0.record(stream)
            for _ in range(reps):
                launch()
            e1.record(stream)
            torch.cuda.synchronize()
        rate = ops.value * reps / (e0.elapsed_time(e1) / 1e3)
        c = clk.summary() or {}
        mhz = c.get("sm_mhz")
        out[name] = {"lane_ops_per_s": rate, "sm_mhz": mhz, "reasons": c.get("reasons"),
                     "per_sm_per_clk": rate / (n_sm * mhz * 1e6) if mhz else None}
    out["n_sm"] = n_sm
    out["how"] = ("hmfsr_pipe_probe: 8 blocks of 256 threads per SM, 8 independent chains of 16 dependent "
                  "operations per loop step per thread; 10 launches timed with CUDA events")
    return out


# -----------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# -----------------------------------------------------------------------------------------
def oracle_align_time(raw_np, cores):
    """Oracle alignment of the whole burst: (float32 motion, seconds)."""
    import oracle
    t0 = time.perf_counter()
    _, mf, _, _ = oracle.align(raw_np, n_threads=cores)
    return mf.astype("float32"), time.perf_counter() - t0


def oracle_merge_rows_time(raw_np, motion, params, scale, rows, cores):
    """Oracle merge of `rows` output rows in the middle of the frame: seconds."""
    import oracle
    n, h, w = raw_np.shape
    ho = (h * scale[0]) // scale[1]
    y0 = max(0, (ho - rows) // 2)
    t0 = time.perf_counter()
    oracle.merge(raw_np, motion, params, scale=scale, rows=(y0, y0 + rows), n_threads=cores)
    return time.perf_counter() - t0


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper's method written out plainly) on the
    host cores, one whole step per step -- the alignment of the 8-frame 12-MP burst and
    the merge of every output row -- on the GPU arm's workload and config."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import burstgen
    import oracle
    import torch
    # the input is rendered on the GPU when there is one (input generation only)
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    b = burstgen.make_burst(WORKLOAD, seed=rank_seed(0), device=gen_dev)
    raw_np = b["raw"].cpu().numpy()
    n, h, w = raw_np.shape
    scale = b["scale"]
    ho = (h * scale[0]) // scale[1]
    p = oracle.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
    cores = host_cores()
    mp = n * h * w / 1e6
    times = []
    for i in range(args.warmup + args.steps):
        motion, t_align = oracle_align_time(raw_np, cores)
        dt = t_align + oracle_merge_rows_time(raw_np, motion, p, scale, ho, cores)
        if i >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.mean(times)
    value = mp / (ms / 1e3)
    sample = (f"whole steps: per step, oracle alignment of the {n}-frame burst and oracle merge of all {ho} "
              f"output rows, on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(n, h, w, 16, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -----------------------------------------------------------------------------------------
# GPU arm
# -----------------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import burstgen
    import paper_1905_03277_gb300 as hm

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    hm.build()

    b = burstgen.make_burst(WORKLOAD, seed=rank_seed(rank), device=dev)
    raw = b["raw"]
    n, h, w = raw.shape
    scale = b["scale"]
    p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
    ap = hm.AlignParams(tile=p.tile)
    ho, wo = hm.out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    acc_ms, prep_ms, align_ms = [], [], []

    def step():
        # one call: the merge's motion-free preparation overlaps the alignment
        hm.align_merge(raw, p, scale, 0, ap, out=rgb)

    def step_phases():
        # the same work as three sequential calls, with events between the phases
        ev[0].record(stream)
        motion = hm.align(raw, 0, ap)
        ev[1].record(stream)
        ws = hm.merge_prepare(raw, motion, p)
        ev[2].record(stream)
        hm.merge_accumulate(raw, motion, ws, p, scale, out=rgb)
        ev[3].record(stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, inputs resident; the 195 MB burst is larger than the L2
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for _ in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    ms_step = elapsed / args.steps
    mp = n * h * w / 1e6
    value = whole_job_mps(mp, world, ms_step)

    # per-phase durations on the launching stream (separate pass, same work)
    for _ in range(min(args.steps, 10)):
        step_phases()
        torch.cuda.synchronize()
        align_ms.append(ev[0].elapsed_time(ev[1]))
        prep_ms.append(ev[1].elapsed_time(ev[2]))
        acc_ms.append(ev[2].elapsed_time(ev[3]))

    # end to end through the public API with host buffers: every step copies its burst in
    # from pinned host memory, aligns and merges it, and copies the RGB result back; the
    # pipeline overlaps one burst's copies with another's compute (two device slots)
    host_burst = raw.cpu().pin_memory()
    host_out = torch.empty((3, ho, wo), dtype=torch.float32, pin_memory=True)
    pipe = hm.AlignMergePipeline(tuple(raw.shape), p, scale, device=dev, depth=2)
    for _ in range(3):
        pipe.submit(host_burst, host_out)
    pipe.synchronize()
    torch.cuda.synchronize()
    e2e_steps = 30  # ~70 ms: the pipeline's fill and drain amortise
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(pipe.h2d)
    for _ in range(e2e_steps):
        pipe.submit(host_burst, host_out)
    e1.record(pipe.d2h)
    pipe.synchronize()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    del pipe
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = whole_job_mps(mp, world, e2e_ms)

    # noise-dependent tuning: the exact sum of a frame on the GPU (HBM-bound; the calls
    # rotate over the 8 frames, 195 MB > L2), then the parameters the base frame selects
    fsum = torch.empty(1, dtype=torch.int64, device=dev)
    for f in range(n):
        hm.frame_sum(raw, f, out=fsum)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    sum_reps = 4 * n
    t0.record(stream)
    for i in range(sum_reps):
        hm.frame_sum(raw, i % n, out=fsum)
    t1.record(stream)
    torch.cuda.synchronize()
    sum_us = t0.elapsed_time(t1) / sum_reps * 1e3
    tmp, tap, tsnr = hm.auto_params(raw, b["gain"], b["read"] ** 2, ref=0)
    frame_bytes = h * w * 2
    tuning = {"snr": tsnr, "tile": tap.tile, "k_detail": tmp.k_detail, "k_denoise": tmp.k_denoise,
              "frame_sum_us": sum_us, "frame_sum_gbs": frame_bytes / sum_us / 1e3,
              "hbm_frac": frame_bytes / sum_us / 1e3 / ((measured_peaks() or {}).get("hbm_gbs", FALLBACK_HBM_GBS)),
              "kernel": "k_frame_sum (hmfsr_frame_sum), 24.4 MB per 12-MP frame",
              "per_call": "the zeroing memset and the kernel, launched from Python back to back"}
    # Monte-Carlo noise statistics: the table for this burst's noise model (once per model)
    hm.noise_table(b["gain"], b["read"] ** 2, device=dev)
    torch.cuda.synchronize()
    t0.record(stream)
    ntab = hm.noise_table(b["gain"], b["read"] ** 2, device=dev)
    t1.record(stream)
    torch.cuda.synchronize()
    tuning["noise_table_ms"] = t0.elapsed_time(t1)
    # the whole merge with the closed form and with the table (inputs resident)
    tmotion = hm.align(raw, 0, ap)
    for fn in ("merge_ms", "merge_noise_ms"):
        call = (lambda: hm.merge(raw, tmotion, p, scale)) if fn == "merge_ms" else (
            lambda: hm.merge_noise(raw, tmotion, ntab, p, scale))
        call()
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(5):
            call()
        t1.record(stream)
        torch.cuda.synchronize()
        tuning[fn] = t0.elapsed_time(t1) / 5
    tuning["noise_table"] = (f"{ntab.shape[0]} levels x 4096 trials x 54 Philox-4x32-10 Irwin-Hall normals "
                             "(FP64 samples, rounding and clipping)")

    # bounded memory: the same merge a chunk of frames at a time (the running sums of every
    # output pixel kept in the workspace between chunks), against the resident merge
    bounded = {"chunk_frames": 2}
    crgb = hm.merge_chunked(raw, tmotion, p, scale, 0, chunk_frames=2)
    bounded["identical_to_resident"] = bool(torch.equal(crgb, hm.merge(raw, tmotion, p, scale)))
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(5):
        hm.merge_chunked(raw, tmotion, p, scale, 0, chunk_frames=2)
    t1.record(stream)
    torch.cuda.synchronize()
    bounded["chunked_merge_ms"] = t0.elapsed_time(t1) / 5
    bounded["resident_merge_ms"] = tuning["merge_ms"]
    for frames in (n, 4 * n):
        bounded[f"workspace_mb_{frames}_frames"] = {
            "resident": hm.workspace_size(hm._lib.OP_MERGE, (frames, h, w), p.tile, scale) / 1e6,
            "chunked": hm.chunked_workspace_size((frames, h, w), p.tile, scale, 2) / 1e6}
    del crgb

    # adjoint (fitting workload: 8 x 1024x1024 at 1.5x): forward with den, then backward
    fb = burstgen.make_burst("fit", seed=burstgen.SEED_BASE + 3 + 1000 * rank, device=dev)
    fraw = fb["raw"]
    fp = hm.MergeParams(noise_a=fb["gain"], noise_b=fb["read"] ** 2)
    fmotion = hm.align(fraw, 0, ap)
    fscale = fb["scale"]
    fho, fwo = hm.out_size(fraw.shape[1], fraw.shape[2], fscale)
    gup = torch.randn((3, fho, fwo), device=dev, generator=torch.Generator(device=dev).manual_seed(5))
    fev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd_ms, bwd_ms = [], []
    # the forward's planes stay in an adjoint-sized workspace, which the backward reuses
    fws = hm.backward_workspace(tuple(fraw.shape), fp.tile, fscale, dev)
    for i in range(8):
        fev[0].record(stream)
        frgb, fden = hm.merge(fraw, fmotion, fp, fscale, with_den=True, workspace=fws)
        fev[1].record(stream)
        hm.merge_backward(fraw, fmotion, fp, frgb, fden, gup, fscale, workspace=fws, prepared=True)
        fev[2].record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            fwd_ms.append(fev[0].elapsed_time(fev[1]))
            bwd_ms.append(fev[1].elapsed_time(fev[2]))

    # ragged batch: one persistent graph-captured launch vs per-burst align + merge
    batched = None
    if not args.no_batch:
        rb = burstgen.make_ragged_batch(args.batch_bursts, seed=burstgen.SEED_BASE + 4 + 1000 * rank, device=dev,
                                        ss=2)
        braw = [b["raw"] for b in rb]
        bparams = [hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2) for b in rb]
        bscales = [b["scale"] for b in rb]
        plan = hm.BatchPlan([tuple(r.shape) for r in braw], bparams, bscales, 0)
        brgb = plan.outputs(dev)
        tuned_ms, tune_log = plan.tune(braw, brgb)
        bmp = sum(r.shape[0] * r.shape[1] * r.shape[2] for r in braw) / 1e6
        be0, be1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        plan.run(braw, brgb, wait=True)
        reps = 3
        be0.record(stream)
        for _ in range(reps):
            plan.run(braw, brgb)
        be1.record(stream)
        plan.wait()
        batched_ms = be0.elapsed_time(be1) / reps
        prgb = plan.outputs(dev)

        def plain_pass():
            for r, pp, sc, out in zip(braw, bparams, bscales, prgb):
                mv_ = hm.align(r, 0, ap)
                ws_ = hm.merge_prepare(r, mv_, pp)
                hm.merge_accumulate(r, mv_, ws_, pp, sc, out=out)

        plain_pass()
        torch.cuda.synchronize()
        be0.record(stream)
        for _ in range(reps):
            plain_pass()
        be1.record(stream)
        torch.cuda.synchronize()
        plain_ms = be0.elapsed_time(be1) / reps
        identical = all(torch.equal(a, b_) for a, b_ in zip(brgb, prgb))
        batched = {"workload": f"{len(braw)} ragged bursts: 0.5-12 MP, 4:3 or 16:9, 4-15 frames, 1x/1.5x/2x, "
                               f"gain 0.5-8 (seeded)", "raw_mp_frames": bmp, "batched_ms": batched_ms,
                   "plain_ms": plain_ms, "batched_mps": bmp / (batched_ms / 1e3), "plain_mps": bmp / (plain_ms / 1e3),
                   "speedup": plain_ms / batched_ms, "identical_to_plain": identical,
                   "tuner_best_ms": tuned_ms, "tuner_ms": tune_log,
                   "plain_launches": sum(sum(hm.launches_per_call(r.shape[0], r.shape[1], r.shape[2]).values())
                                         for r in braw),
                   "mode": min(tune_log, key=tune_log.get)}
        del plan, brgb, prgb, braw, rb

    pipe_peaks = measure_pipe_peaks(dev, n_sm, local) if rank == 0 else None

    if rank == 0:
        units = ho * wo * n
        acc_s = statistics.median(acc_ms) / 1e3
        achieved = ACC_FP32_OPS_PER_UNIT * units / acc_s / 1e12
        clocks = clk.summary()
        fma, ex2 = pipe_peaks["fp32_fma"], pipe_peaks["mufu_ex2"]
        peak = fma["lane_ops_per_s"] / 1e12
        mufu_peak = ex2["lane_ops_per_s"] / 1e12
        roof = {"bound": "alu", "kernel": "k_merge_q1 (hmfsr_merge_accumulate: k_geo, k_merge_q1)", "achieved": achieved, "peak": peak,
                "unit": "T lane-ops/s", "frac": achieved / peak, "traffic": kernel_traffic("k_merge_12mp"),
                "peak_source": (f"measured: FP32 FMA issue rate of hmfsr_pipe_probe on this GPU ({n_sm} SMs, "
                                f"{fma['sm_mhz']} MHz sampled; {fma['per_sm_per_clk']:.1f} lane-ops per SM per clock)"),
                "ops_per_unit": ACC_FP32_OPS_PER_UNIT, "units_per_launch": units,
                "unit_of_work": "output pixel x frame; one lane-op per FP32 add, multiply or fused multiply-add",
                "mufu": {"achieved": ACC_MUFU_PER_UNIT * units / acc_s / 1e12, "peak": mufu_peak,
                         "frac": ACC_MUFU_PER_UNIT * units / acc_s / 1e12 / mufu_peak,
                         "peak_source": f"measured: ex2 issue rate of hmfsr_pipe_probe ({ex2['sm_mhz']} MHz sampled)"}}
        peaks = measured_peaks()
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            op = oracle.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
            raw_np = raw.cpu().numpy()
            cores = host_cores()
            motion_o, t_align = oracle_align_time(raw_np, cores)
            t_merge = oracle_merge_rows_time(raw_np, motion_o, op, scale, ho, cores)
            cpu = {"value": mp / (t_align + t_merge), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"the whole step once: oracle alignment of the 8-frame 12-MP burst ({t_align:.2f} s) "
                             f"+ oracle merge of all {ho} output rows ({t_merge:.2f} s)"}
        per_call = hm.launches_per_call(n, h, w, ap.n_levels, ap.tile, ap.radius[0])
        launches = args.steps * sum(per_call.values())
        merge_only_ms = statistics.median([p_ + a_ for p_, a_ in zip(prep_ms, acc_ms)])
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(n, h, w, p.tile, world),
                "roofline": roof, "cpu_baseline": cpu,
                "fp32_peak_measured": fma, "mufu_peak_measured": ex2,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(host_burst.numel() * 2),
                        "d2h_bytes_per_step": int(host_out.numel() * 4), "ms_per_step": e2e_ms,
                        "steps": e2e_steps, "api": "AlignMergePipeline (hmfsr_align_merge), 2 device slots: "
                                                   "one burst's copies overlap another's compute"},
                "gpu_launches": launches, "launches_per_step": per_call, "clocks": clocks,
                "breakdown_ms": {"align": statistics.median(align_ms), "merge_prepare": statistics.median(prep_ms),
                                 "merge_accumulate": statistics.median(acc_ms),
                                 "sequential_step": statistics.median(
                                     [a_ + p_ + c_ for a_, p_, c_ in zip(align_ms, prep_ms, acc_ms)]),
                                 "of": "the step's work as three sequential calls (hmfsr_align, "
                                       "hmfsr_merge_prepare, hmfsr_merge_accumulate), CUDA events between them"},
                "merge_only": {"value": mp / (merge_only_ms / 1e3), "unit": UNIT, "ms_per_step": merge_only_ms,
                               "of": "merge preparation + accumulation of each timed step (CUDA events), "
                                     "alignment excluded"},
                "hbm_peak_gbs": (peaks or {}).get("hbm_gbs", FALLBACK_HBM_GBS),
                "batched": batched,
                "snr_tuning": tuning,
                "bounded_memory": bounded,
                "adjoint": {"workload": "fit: 8 x 1024x1024 RGGB, 1.5x output",
                            "backward": "hmfsr_merge_backward_prepared (the forward's planes reused)",
                            "forward_ms": statistics.median(fwd_ms),
                            "backward_ms": statistics.median(bwd_ms),
                            "backward_over_forward": statistics.median(bwd_ms) / statistics.median(fwd_ms)}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_fit(args):
    """Adjoint workload: fit the eight tuning parameters (and the motion) of 16 bursts of
    8 x 1024x1024 (1.5x ground truth) with Adam; prints one JSON line."""
    import math

    import torch

    import burstgen
    import paper_1905_03277_gb300 as hm
    from paper_1905_03277_gb300.fit import fit

    dev = torch.device("cuda", 0)
    hm.build()
    bursts, gts = [], []
    for k in range(args.fit_bursts):
        b = burstgen.make_burst("fit", seed=burstgen.SEED_BASE + 3 + k, device=dev, with_gt=True)
        bursts.append(b["raw"])
        gts.append(b["gt"])
    base = hm.MergeParams(noise_a=1.0, noise_b=9.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    params, hist, _ = fit(bursts, gts, base, steps=args.fit_steps, scale=(3, 2))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    psnr = lambda mse: 10 * math.log10(4095.0 ** 2 / mse)
    print(json.dumps({"workload": f"fit: {args.fit_bursts} bursts x 8 x 1024x1024 RGGB, 1.5x ground truth, "
                                  f"{args.fit_steps} Adam steps (parameters and motion)",
                      "seconds": dt, "ms_per_step": 1000 * dt / args.fit_steps,
                      "loss_first": hist[0], "loss_last": hist[-1], "psnr_first_db": psnr(hist[0]),
                      "psnr_last_db": psnr(hist[-1]), "start": {k: getattr(base, k) for k in hm.PARAM_NAMES},
                      "fitted": {k: getattr(params, k) for k in hm.PARAM_NAMES}}), flush=True)
    return 0


def run_study_corruption(args):
    """Motion-robustness efficacy (Sec. 7.3) on synthetic bursts with ground truth: the
    PSNR of the merge, with the robustness and with it off (t = -1, so R = 1), as the
    alignment is corrupted in the two ways the paper describes.  Also the quadratic-fit
    subpixel step against Lucas-Kanade on the clean field.  One JSON line."""
    import math

    import numpy as np
    import torch

    import burstgen
    import paper_1905_03277_gb300 as hm

    dev = torch.device("cuda", 0)
    hm.build()
    scale, tile, crop = (3, 2), 16, 24
    ps, sigmas = (0.1, 0.2, 0.3, 0.4, 0.5), (0.05, 0.1, 0.15, 0.2, 0.25)
    rng = np.random.default_rng(burstgen.SEED_BASE + 70)

    def psnr(rgb, gt):
        d = (rgb - gt)[:, crop:-crop, crop:-crop].double()
        return 10.0 * math.log10(4095.0 ** 2 / float((d * d).mean()))

    def replace_tiles(m, frac, ref):
        # a fraction of each non-base frame's tiles get a vector that points at a different
        # area: displaced by one to three tiles along some axis
        m = m.copy()
        n, ty, tx, _ = m.shape
        for f in range(n):
            if f == ref:
                continue
            idx = rng.choice(ty * tx, size=int(round(frac * ty * tx)), replace=False)
            d = rng.integers(-3 * tile, 3 * tile + 1, size=(idx.size, 2))
            small = np.abs(d).max(axis=1) < tile
            while small.any():
                d[small] = rng.integers(-3 * tile, 3 * tile + 1, size=(int(small.sum()), 2))
                small = np.abs(d).max(axis=1) < tile
            flat = m[f].reshape(-1, 2)
            flat[idx] += d.astype(np.float32)
        return m

    def add_noise(m, sigma, ref):
        m = m.copy()
        keep = m[ref].copy()
        m += rng.normal(0.0, sigma, size=m.shape).astype(np.float32)
        m[ref] = keep
        return m

    rows = {"clean": [], "quadfit": [], "replace": {p: [] for p in ps}, "noise": {s: [] for s in sigmas}}
    n_bursts = 4
    for k in range(n_bursts):
        b = burstgen.make_burst("fit", seed=burstgen.SEED_BASE + 60 + k, device=dev, with_gt=True)
        raw, gt = b["raw"], b["gt"]
        on = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
        off = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2, t=-1.0)
        ap = hm.AlignParams(tile=tile)
        mv = hm.align(raw, 0, ap).cpu().numpy()

        def both(m):
            mt = torch.from_numpy(m).to(dev)
            return (psnr(hm.merge(raw, mt, on, scale), gt), psnr(hm.merge(raw, mt, off, scale), gt))

        rows["clean"].append(both(mv))
        rows["quadfit"].append(both(hm.align(raw, 0, ap, subpixel="quadfit").cpu().numpy()))
        for p in ps:
            rows["replace"][p].append(both(replace_tiles(mv, p, 0)))
        for sg in sigmas:
            rows["noise"][sg].append(both(add_noise(mv, sg, 0)))

    def mean2(v):
        a = np.array(v)
        return {"psnr_robust_db": float(a[:, 0].mean()), "psnr_no_robustness_db": float(a[:, 1].mean())}

    print(json.dumps({
        "study": "motion robustness efficacy (Sec. 7.3) on synthetic bursts",
        "workload": f"{n_bursts} bursts x 8 x 1024x1024 RGGB (fit workload), 1.5x, PSNR against the rendered "
                    f"ground truth inside a {crop}-px border",
        "clean_lk": mean2(rows["clean"]), "clean_quadfit": mean2(rows["quadfit"]),
        "tile_replacement": [dict(p=p, **mean2(rows["replace"][p])) for p in ps],
        "vector_noise_px": [dict(sigma=sg, **mean2(rows["noise"][sg])) for sg in sigmas],
        "corruption": "replacement: the tile's vector displaced by 1-3 tiles along some axis (a different area); "
                      "noise: N(0, sigma^2) raw px added to each component of each non-base tile's vector"}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("hmfsr", "reference"), default="hmfsr")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fit", action="store_true", help="run the parameter-fitting workload instead")
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch comparison")
    ap.add_argument("--batch-bursts", type=int, default=64)
    ap.add_argument("--fit-steps", type=int, default=200)
    ap.add_argument("--fit-bursts", type=int, default=16)
    ap.add_argument("--study", choices=("corruption",), help="run an evaluation study instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.fit:
        return run_fit(args)
    if args.study == "corruption":
        return run_study_corruption(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
