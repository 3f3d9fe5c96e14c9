#!/usr/bin/env python
"""Decode benchmark of the pWave++ path on GB300.

Metric: decoded MPix/s and p50/p99 decode latency. Workload (the batched
image configuration): a batch of 24 synthetic RGB 768x512 images (gradient +
rectangles + 1/f texture), 4-level CNN lifting, context model with 64
channels and the four-step LL model, quantiser steps {4, 8, 16, 32} (six
images each), random-init weights (seed 0). One step = one batched decode of
the 24 streams: stream parsing, CDF table bank, ConvLSTM + four-step context
passes with rANS decoding for all 13 subbands, dequantisation, inverse
lifting and colour conversion.

value: device-resident streams -> device images, CUDA events on the
library's stream, L2 flushed (256 MB write) between timed steps (outside the
events). e2e: the same decode through the C ABI from host streams to host
images, host wall clock around each call. roofline: the dominant kernel class
from the library's own CUDA-event timing. cpu_baseline: the CPU oracle
decoding a bounded sample (one 256x256 RGB crop of the workload).

Precision: FP8 by default (E4M3 3x3 context convolutions, BF16 elsewhere);
the other tensor-core class (BF16) is timed the same way under
"bf16_batched". gop: one 8-frame 1920x1080 GOP through pw_decode_gop (host in, host out).
fp32_single_image: the plain FP32 GPU path decoding the same
images one per call (its own FP32 streams, same q). serving: an open-loop run of the serving
workload's first 200 requests (Poisson arrivals at 200/s, mixed sizes from
256x256 to 2048x2048, gray/RGB) through the decode server, with p50/p99
latency (submit -> decoded host image) and MPix/s.

With --impl reference the CPU oracle is timed instead (each step decodes one
128x128 RGB crop of the workload) and one JSON line with "impl": "reference"
is printed. Multi-GPU (torchrun, N > 1): every rank decodes its own batch
(replicas, weak scaling); rank 0 prints the line.
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

BATCH = 24
H, W = 512, 768
QSTEPS = (4.0, 8.0, 16.0, 32.0)
WORKLOAD = "batch of 24 RGB 768x512 images, 4-level CNN lifting, 64-ch four-step context model, q in {4,8,16,32}"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(vals, world: int, dev=None):
    """Element-wise maximum of `vals` over the ranks (one all-reduce of a
    float64 tensor on `dev`); the values themselves when world == 1."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_mpix_per_s(world: int, pixels_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each decoded
    pixels_per_rank pixels, timed by the slowest of them (seconds)."""
    return world * pixels_per_rank / seconds / 1e6


def make_inputs(seed_base: int, batch: int):
    import synthetic as S
    imgs = [S.rgb_natural(H, W, seed=seed_base + i) for i in range(batch)]
    qs = [QSTEPS[i % 4] for i in range(batch)]
    return imgs, qs


def model_blob():
    import synthetic as S
    cfg = S.ModelConfig(levels=4, C=64, F=16, ll_mode=0)
    return S.pack_blob(cfg, S.random_model(cfg, 0))


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                pass
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
def cpu_oracle_decode_sample(crop: int):
    """Time the CPU oracle decoding one crop x crop RGB image of the workload."""
    import synthetic as S
    from oracle import codec as K
    blob = model_blob()
    img = S.rgb_natural(H, W, seed=1)[:crop, :crop]
    bs = K.encode_image(blob, img, q=8.0)
    t0 = time.perf_counter()
    K.decode_image(blob, bs)
    dt = time.perf_counter() - t0
    return crop * crop, dt


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    crop = 128
    for _ in range(args.warmup):
        cpu_oracle_decode_sample(crop)
    times = []
    for _ in range(args.steps):
        px, dt = cpu_oracle_decode_sample(crop)
        times.append(dt)
    total = sum(times)
    value = px * len(times) / total / 1e6
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": "decoded MPix/s", "value": value, "unit": "MPix/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": BATCH, "precision": "fp64 oracle",
                   "sample": f"one {crop}x{crop} RGB crop per step"},
        "cpu_baseline": {"value": value, "unit": "MPix/s", "cores": cores, "kind": "oracle",
                         "sample": f"{crop}x{crop} RGB crop of image 1, q=8, decode only"},
        "e2e": {"value": value, "unit": "MPix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)),
                       "p99": 1e3 * float(np.percentile(times, 99))},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def fp32_single_image(pw, local, imgs, qs, blob, stream_ptr):
    """The plain FP32 path decoding the workload one image per call.

    Its own FP32 streams (the precision class is part of the stream); the
    same images and quantiser steps, so the rate is essentially equal (bpp
    reported). Device streams -> device image, CUDA events around all calls.
    """
    import torch
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c32 = pw.Codec(local, "fp32", stream=stream_ptr)
    m32 = c32.load_model(blob)
    enc = []
    for img, q in zip(imgs, qs):
        enc.append(c32.encode_image(m32, img, q=q))
    bufs = [torch.from_numpy(np.frombuffer(b, dtype=np.uint8).copy()).to(dev) for b in enc]
    out = torch.empty((H, W, 3), dtype=torch.uint8, device=dev)

    def one(i):
        c32.decode_batch_device(m32, [bufs[i].data_ptr()], [len(enc[i])], out.data_ptr(), (H, W, 3))

    one(0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(len(enc)):
        one(i)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    n = len(enc)
    res = {"value": n * H * W / (ms / 1e3) / 1e6, "unit": "MPix/s", "images": n,
           "ms_per_image": ms / n, "bpp": 8.0 * sum(len(b) for b in enc) / (n * H * W),
           "path": "fp32 SIMT context model, one image per decode call"}
    m32.close()
    c32.close()
    return res


def batched_precision(pw, local, prec, imgs, qs, blob, stream_ptr, steps, warmup):
    """The same batched, device-resident decode in another precision class
    (its own streams; same images and q), timed the same way."""
    import torch
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c = pw.Codec(local, prec, stream=stream_ptr)
    m = c.load_model(blob)
    enc = [None] * len(imgs)
    for q in QSTEPS:
        idx = [i for i in range(len(imgs)) if qs[i] == q]
        if idx:
            for i, b in zip(idx, c.encode_batch(m, [imgs[i] for i in idx], q=q)):
                enc[i] = b
    lens = [len(b) for b in enc]
    offs = np.cumsum([0] + [(n + 255) // 256 * 256 for n in lens])
    host_all = np.zeros(int(offs[-1]), dtype=np.uint8)
    for i, b in enumerate(enc):
        host_all[offs[i]:offs[i] + lens[i]] = np.frombuffer(b, dtype=np.uint8)
    dev_all = torch.from_numpy(host_all).to(dev)
    ptrs = [dev_all.data_ptr() + int(offs[i]) for i in range(len(enc))]
    out = torch.empty((len(enc), H, W, 3), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        c.decode_batch_device(m, ptrs, lens, out.data_ptr(), (H, W, 3))
    torch.cuda.synchronize()
    times = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.decode_batch_device(m, ptrs, lens, out.data_ptr(), (H, W, 3))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    res = {"value": len(enc) * H * W / (ms / 1e3) / 1e6, "unit": "MPix/s", "ms_per_step": ms,
           "bpp": 8.0 * sum(lens) / (len(enc) * H * W)}
    m.close()
    c.close()
    return res


def gop_run(pw, codec, blob_low, blob_high, reps: int):
    """Video: one GOP of 8 synthetic 1920x1080 RGB frames (panned 1/f canvas +
    sprites), identity-motion temporal lifting, 8 temporal bands coded as
    images (low band with one model, the 7 high bands batched with another),
    q = 8. Host stream in, host frames out; host wall clock per decode."""
    import synthetic as S
    frames = S.video_gop(1080, 1920, 8, seed=3)
    ml, mh = codec.load_model(blob_low), codec.load_model(blob_high)
    gs = codec.encode_gop(ml, mh, frames, q=8.0)
    out = codec.decode_gop(ml, mh, gs, 8, (1080, 1920, 3))
    mse = float(np.mean((out.astype(np.float64) - frames) ** 2))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        codec.decode_gop(ml, mh, gs, 8, (1080, 1920, 3))
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(times))
    ml.close()
    mh.close()
    return {"workload": "1 GOP x 8 frames 1920x1080 RGB, 3 temporal levels, q=8", "frames": 8,
            "value": 8 * 1920 * 1080 / (ms / 1e3) / 1e6, "unit": "MPix/s",
            "ms_per_gop": ms, "bpp": 8.0 * len(gs) / (8 * 1920 * 1080),
            "psnr_db": 10 * np.log10(255.0 ** 2 / mse), "timing": "host wall clock, e2e"}


def serving_run(pw, codec, model, n_req: int, rate: float, lanes: int, max_batch: int,
                budget: int):
    """Open-loop serving: a Poisson stream of mixed-size decode requests.

    The first n_req requests of the serving workload (Poisson arrivals at
    `rate` per second, w and h log-uniform in [256, 2048] rounded down to a
    multiple of 16, gray/RGB 50/50, q uniform over {4, 8, 16, 32}); every
    image is a crop of a seeded synthetic canvas, pre-encoded by the GPU
    encoder. Requests are submitted at their arrival instants; latency is
    submit -> decoded image on the host (the server's own clock).
    """
    import synthetic as S
    reqs = S.request_stream(n=n_req, rate=rate, seed=7)
    rng = np.random.default_rng(7)
    canvas = {1: S.gray_sinusoids(2048, 2048, seed=7), 3: S.rgb_natural(2048, 2048, seed=7)}
    streams = []
    for r in reqs:
        y0 = int(rng.integers(0, 2048 - r["h"] + 1))
        x0 = int(rng.integers(0, 2048 - r["w"] + 1))
        img = np.ascontiguousarray(canvas[r["c"]][y0:y0 + r["h"], x0:x0 + r["w"]])
        streams.append(codec.encode_image(model, img, q=r["q"]))
    srv = pw.Server(codec, model, hbm_budget=budget, lanes=lanes, max_batch=max_batch)
    done = {}

    def collect():
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0005)
            done[i] = srv.poll(tickets[i], timeout_ms=600000) is not None

    tickets = [None] * len(reqs)
    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        dt = t0 + r["t"] - reqs[0]["t"] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(streams[i])
    th.join()
    st = srv.stats()
    srv.close()
    mpix = sum(r["w"] * r["h"] for r in reqs) / 1e6
    return {"requests": len(reqs), "rate_per_s": rate, "lanes": lanes, "max_batch": max_batch,
            "hbm_budget_gb": budget / 2**30, "mean_mpix_per_request": mpix / len(reqs),
            "completed": int(st["completed"]), "batches": int(st["batches"]),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mpix_per_s": st["mpix_per_s"],
            "offered_mpix_per_s": mpix / max(reqs[-1]["t"] - reqs[0]["t"], 1e-9),
            "all_ok": all(done.values())}


# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2405_12631_gb300 as pw

    stream = torch.cuda.current_stream(dev)
    codec = pw.Codec(local, args.precision, stream=stream.cuda_stream)
    blob = model_blob()
    model = codec.load_model(blob)
    BATCH = args.batch
    imgs, qs = make_inputs(1 + 1000 * rank, BATCH)
    streams = []
    for q in QSTEPS:
        idx = [i for i in range(BATCH) if qs[i] == q]
        if not idx:
            continue
        enc = codec.encode_batch(model, [imgs[i] for i in idx], q=q)
        streams += list(zip(idx, enc))
    streams = [s for _, s in sorted(streams, key=lambda t: t[0])]
    lens = [len(s) for s in streams]
    offs = np.cumsum([0] + [(n + 255) // 256 * 256 for n in lens])
    host_all = np.zeros(int(offs[-1]), dtype=np.uint8)
    for i, s in enumerate(streams):
        host_all[offs[i]:offs[i] + lens[i]] = np.frombuffer(s, dtype=np.uint8)
    dev_all = torch.from_numpy(host_all).to(dev)
    ptrs = [dev_all.data_ptr() + int(offs[i]) for i in range(BATCH)]
    out = torch.empty((BATCH, H, W, 3), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream_bytes = int(sum(lens))
    pixels = BATCH * H * W

    def step():
        codec.decode_batch_device(model, ptrs, lens, out.data_ptr(), (H, W, 3))

    def class_stats():
        stats = (pw.pw_kernel_stat * 32)()
        nst = pw.pw_ctx_kernel_stats(codec.ctx, stats, 32)
        return [{"name": stats[i].name.decode(), "launches": int(stats[i].launches),
                 "ms": float(stats[i].ms), "flops": float(stats[i].flops),
                 "bytes": float(stats[i].bytes)} for i in range(max(nst, 0))]

    for _ in range(max(args.warmup - 1, 0)):
        step()
    # the last warm-up step records every kernel class (the per-class
    # breakdown); the timed steps then record only the dominant class, whose
    # CUDA-event time gives the roofline figure without perturbing the rest
    pw.pw_ctx_profile(codec.ctx, 1)
    step()
    torch.cuda.synchronize()
    kern_all = class_stats()
    pw.pw_ctx_profile(codec.ctx, 0)
    dom_name = max(kern_all, key=lambda k: k["ms"])["name"] if kern_all else None
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if dom_name:
        pw.pw_ctx_profile_classes(codec.ctx, 1 << pw.pw_kernel_class(dom_name.encode()))
    l0 = codec.launches
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    sampler.stop()
    launches = codec.launches - l0
    kern = class_stats()     # the dominant class over the timed steps
    pw.pw_ctx_profile(codec.ctx, 0)
    total_ms = max_over_ranks([sum(times)], world, dev)[0]
    value = job_mpix_per_s(world, pixels * args.steps, total_ms / 1e3)

    # e2e: host streams -> host images through the C ABI
    e2e_times = []
    host_out = None
    if not args.no_e2e:
        for i in range(max(1, args.steps // 2)):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_out = codec.decode_batch(model, streams)
            e2e_times.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
    e2e_s, e2e_n = max_over_ranks([sum(e2e_times), len(e2e_times)], world, dev)
    e2e_value = job_mpix_per_s(world, pixels * e2e_n, e2e_s) if e2e_times else None

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    kern_sorted = sorted(kern_all, key=lambda k: -k["ms"])
    dom = kern[0] if kern else None
    clocks = sampler.summary()
    roofline = None
    if dom:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        if dom["name"].startswith("ctx") or dom["name"] == "lift_step":
            if args.precision in ("bf16", "fp8") and dom["name"].startswith("ctx"):
                tpeak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
                if args.precision == "fp8" and dom["name"] in ("ctx_conv3x3",
                                                               "ctx_lstm_gates_conv3x3"):
                    tpeak *= 2.0   # E4M3 convs: bf16 peak x the nominal fp8/bf16 ratio (2)
                cbound = "tensor"
            else:
                # FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock
                tpeak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
                cbound = "alu"
            # the bound is whichever roof the kernel's arithmetic intensity
            # (algorithmic FLOP per algorithmic HBM byte) hits first
            ridge = tpeak * 1e12 / (hbm * 1e9)
            ai = dom["flops"] / max(dom["bytes"], 1.0)
            if ai >= ridge:
                bound, unit, peak = cbound, "TFLOP/s", tpeak
                achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
            else:
                bound, unit, peak = "hbm", "GB/s", hbm
                achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        else:
            ai, ridge = None, None
            peak = hbm
            bound, unit = "hbm", "GB/s"
            achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak, "traffic": None, "kernel": dom["name"],
                    "timing": "CUDA events around this class's launches over the timed steps "
                              "(the only class recorded there)",
                    "flop_per_byte": ai, "ridge_flop_per_byte": ridge,
                    "peak_source": peak_kind + (" (derived: SMs x lanes x clock)"
                                                if bound == "alu" else "")}
    total_kernel_ms = sum(k["ms"] for k in kern_all) or 1.0
    line = {
        "metric": "decoded MPix/s", "value": value, "unit": "MPix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp8": "fp8-e4m3+bf16", "fp32": "f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if BATCH == 24 else WORKLOAD.replace("24", str(BATCH), 1),
                   "global_batch": BATCH * world, "image": "768x512 RGB",
                   "context_channels": 64, "levels": 4, "ll_mode": "four-step",
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) between timed steps",
                   "stream_bytes_per_step": stream_bytes,
                   "bpp": 8.0 * stream_bytes / pixels},
        "latency_ms": {"p50": float(np.percentile(times, 50)),
                       "p99": float(np.percentile(times, 99))},
        "e2e": {"value": e2e_value, "unit": "MPix/s",
                "h2d_bytes_per_step": stream_bytes, "d2h_bytes_per_step": pixels * 3},
        "gpu_launches": int(launches),
        "roofline": roofline,
        # per-class breakdown of one (profiled) warm-up step
        "kernels": [{"name": k["name"], "launches": k["launches"],
                     "ms_per_step": k["ms"],
                     "share": k["ms"] / total_kernel_ms} for k in kern_sorted],
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
        "wall_s_timed_region": t_wall,
    }
    if world == 1 and not args.no_compare:
        for p in ("fp8", "bf16"):
            if p != args.precision:
                line[f"{p}_batched"] = batched_precision(pw, local, p, imgs, qs, blob,
                                                         stream.cuda_stream, args.steps,
                                                         args.warmup)
    if not args.no_fp32 and world == 1:
        line["fp32_single_image"] = fp32_single_image(pw, local, imgs, qs, blob,
                                                      stream.cuda_stream)
    if not args.no_gop and world == 1:
        import synthetic as S
        cfg = S.ModelConfig(levels=4, C=64, F=16, ll_mode=0)
        line["gop"] = gop_run(pw, codec, blob, S.pack_blob(cfg, S.random_model(cfg, 1)), 3)
    if args.serve > 0 and world == 1:
        line["serving"] = serving_run(pw, codec, model, args.serve, 200.0, lanes=16,
                                      max_batch=8, budget=48 << 30)
    if not args.no_cpu and world == 1:
        px, dt = cpu_oracle_decode_sample(256)
        line["cpu_baseline"] = {"value": px / dt / 1e6, "unit": "MPix/s",
                                "cores": blas_threads(), "kind": "oracle",
                                "sample": "256x256 RGB crop of image 1, q=8, decode only"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("PW_BENCH_PRECISION", "fp8"),
                    choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="images per step (24 = the benchmark workload; smaller for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other tensor-core precision class")
    ap.add_argument("--no-gop", action="store_true", help="skip the video GOP leg")
    ap.add_argument("--no-fp32", action="store_true",
                    help="skip the FP32 single-image comparison")
    ap.add_argument("--serve", type=int, default=200,
                    help="requests of the open-loop serving run (0 = skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
