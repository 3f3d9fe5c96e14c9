#!/usr/bin/env python
"""Decode benchmark of the pWave++ path on GB300.

Metric: decoded MPix/s and p50/p99 decode latency. Headline workload (the
batched image configuration): a batch of 24 synthetic RGB 768x512 images
(gradient + rectangles + 1/f texture), 4-level CNN lifting, context model
with 64 channels and the four-step LL model, quantiser steps {4, 8, 16, 32}
(six images each), random-init weights (seed 0). One step = one batched
decode of the 24 streams: stream parsing, CDF table bank, ConvLSTM +
four-step context passes with rANS decoding for all 13 subbands,
dequantisation, inverse lifting and colour conversion.

value: device-resident streams -> device images, CUDA events on the
library's stream, L2 flushed (256 MB write) between timed steps (outside the
events). e2e: the same decode through the C ABI from host streams in
page-locked memory to host images in page-locked memory (both copies inside
each call), host wall clock around each call. roofline: the dominant kernel class
from the library's own CUDA-event timing; rooflines: every class of one
profiled step against its roof. Precision: FP8 by default (E4M3 3x3 context
convolutions, BF16 elsewhere); the BF16 class is timed the same way under
"bf16_batched", and the plain FP32 path one image per call under
"fp32_single_image".

The other workloads, each under "workloads" with its own key:
* single_gray_256: one 256x256 grayscale image (sum of 8 sinusoids plus
  noise), q = 8, C = 32, FP32 class, batch 1, in both LL modes (four-step
  and autoregressive), with the logistic-mixture (K = 3) probability
  model (four-step LL) and with the integer-network context model (INT8
  class, both LL modes), device-resident stream, CUDA events;
* video_4gop_1080p: 4 GOPs x 8 frames of 1920x1080 RGB (panned 1/f canvas
  and sprites), 3 motion-compensated temporal levels, BF16 class,
  pw_decode_gop host stream in / host frames out (page-locked), wall clock;
* serving_poisson: the full request stream (10,000 Poisson arrivals at
  200/s, sizes log-uniform 256..2048, gray/RGB, q in {4, 8, 16, 32}) through
  the decode server, plus a saturation sweep that replays its first 2,000
  requests at higher arrival rates;
* lossless_4k_12bit: 16 RGB 3840x2160 12-bit images, integer lifting with 5
  levels, FP8 context convolutions, decoded in sub-batches that fit the
  device, each decoded image compared with its input (bit_exact).

cpu_baseline: the FP64 CPU oracle, in a child process on the host cores, on
bounded samples of each workload (the headline value: one 256x256 RGB crop
of the batched workload), plus one single-thread figure.

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


def _time_oracle_decode(blob, bs, decode):
    t0 = time.perf_counter()
    decode(blob, bs)
    return time.perf_counter() - t0


def cpu_baseline_samples(single_thread: bool) -> dict:
    """The FP64 oracle decoding bounded samples of every workload on the
    host cores (this process: run it as a child whose BLAS thread count the
    environment fixes). Each sample: pixels and seconds of the decode alone
    (the oracle's encoder makes the stream first, untimed)."""
    import synthetic as S
    from oracle import codec as K

    def blob_of(levels, C, ll_mode, seed=0, prob=0):
        cfg = S.ModelConfig(levels=levels, C=C, F=16, ll_mode=ll_mode, prob=prob)
        return S.pack_blob(cfg, S.random_model(cfg, seed))

    out = {}
    gray = S.gray_sinusoids(256, 256, seed=0)
    for mode, name in ((0, "single_gray_256_four_step_ll"), (1, "single_gray_256_autoregressive_ll")):
        b = blob_of(4, 32, mode)
        bs = K.encode_image(b, gray, q=8.0)
        out[name] = {"pixels": 256 * 256, "s": _time_oracle_decode(b, bs, K.decode_image),
                     "sample": "the whole 256x256 gray image, q=8, C=32"}
        if single_thread:
            return out
    b = blob_of(4, 32, 0, prob=1)
    bs = K.encode_image(b, gray[:128, :128], q=8.0)
    out["single_gray_256_four_step_ll_logistic_mixture"] = {
        "pixels": 128 * 128, "s": _time_oracle_decode(b, bs, K.decode_image),
        "sample": "128x128 crop of the 256x256 gray image, q=8, C=32, mixture model"}
    b = blob_of(4, 64, 0)
    crop = S.rgb_natural(H, W, seed=1)[:256, :256]
    bs = K.encode_image(b, crop, q=8.0)
    out["batched_768x512_rgb"] = {"pixels": 256 * 256,
                                  "s": _time_oracle_decode(b, bs, K.decode_image),
                                  "sample": "256x256 RGB crop of image 1, q=8, C=64"}
    bl, bh = b, blob_of(4, 64, 0, seed=1)
    gop = S.video_gop(1080, 1920, 8, seed=3)[:, :64, :64]
    gs = K.encode_gop(bl, bh, gop, q=8.0)
    t0 = time.perf_counter()
    K.decode_gop(bl, bh, gs)
    out["video_4gop_1080p"] = {"pixels": 8 * 64 * 64, "s": time.perf_counter() - t0,
                               "sample": "one GOP of 8 frames cropped to 64x64, q=8, C=64"}
    b5 = blob_of(5, 64, 0)
    img = S.lossless_blobs(2160, 3840, seed=5)[:128, :128]
    bs = K.encode_image(b5, img, lossless=True, bitdepth=12)
    out["lossless_4k_12bit"] = {"pixels": 128 * 128,
                                "s": _time_oracle_decode(b5, bs, K.decode_image),
                                "sample": "128x128 crop of image 0, lossless 12-bit, 5 levels, C=64"}
    return out


def cpu_baseline_child(single_thread: bool) -> dict:
    """Run cpu_baseline_samples in a child interpreter (its own BLAS pool;
    one thread when single_thread) and return its results with the thread
    count it used."""
    env = dict(os.environ)
    if single_thread:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-samples"]
    if single_thread:
        cmd.append("--single-thread")
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_samples_main(single_thread: bool):
    res = cpu_baseline_samples(single_thread)
    print(json.dumps({"threads": 1 if single_thread else blas_threads(),
                      "nproc": os.cpu_count(), "samples": res}))


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


def batched_precision(pw, local, prec, imgs, qs, blob, stream_ptr, steps, warmup,
                      lane_shift: int = 7, chunk: int = 16384):
    """The same batched, device-resident decode in another precision class
    or stream format (its own streams; same images and q), timed the same
    way. lane_shift / chunk: the coder's symbols per interleaved state
    (2^lane_shift) and symbols per chunk."""
    import torch
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c = pw.Codec(local, prec, stream=stream_ptr)
    c.set_lane_rule(lane_shift)
    m = c.load_model(blob)
    enc = [None] * len(imgs)
    for q in QSTEPS:
        idx = [i for i in range(len(imgs)) if qs[i] == q]
        if idx:
            for i, b in zip(idx, c.encode_batch(m, [imgs[i] for i in idx], q=q, chunk=chunk)):
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
    calib = 0   # autotuner calibration, as for the headline leg
    while not pw.pw_autotune_settled() and calib < 24:
        c.decode_batch_device(m, ptrs, lens, out.data_ptr(), (H, W, 3))
        torch.cuda.synchronize()
        calib += 1
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


def single_image_latency(pw, local, stream_ptr, blob, prec: str, lane_shift: int, chunk: int,
                         reps: int = 10):
    """Decode latency of one RGB image at 256x256, 1024x768 and 2048x2048
    (crops of the batched workload's generator, q = 8), device stream in,
    device image out, median CUDA-event time of `reps` decodes."""
    import torch
    import synthetic as S
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c = pw.Codec(local, prec, stream=stream_ptr)
    c.set_lane_rule(lane_shift)
    m = c.load_model(blob)
    out = {}
    for hh, ww in ((256, 256), (768, 1024), (2048, 2048)):
        img = S.rgb_natural(hh, ww, seed=5)
        bs = c.encode_image(m, img, q=8.0, chunk=chunk)
        d_bs = torch.from_numpy(np.frombuffer(bs, dtype=np.uint8).copy()).to(dev)
        o = torch.empty((hh, ww, 3), dtype=torch.uint8, device=dev)

        def one():
            c.decode_batch_device(m, [d_bs.data_ptr()], [len(bs)], o.data_ptr(), (hh, ww, 3))
        for _ in range(3):
            one()
        torch.cuda.synchronize()
        t = _events_ms(stream, one, reps)
        out[f"{ww}x{hh}"] = {"ms": float(np.median(t)), "bpp": 8.0 * len(bs) / (hh * ww)}
    m.close()
    c.close()
    return out


def _events_ms(stream, fn, reps: int):
    """CUDA-event times (ms) of `reps` calls of fn on `stream`."""
    import torch
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def single_gray_run(pw, local, stream_ptr, steps: int, warmup: int):
    """One 256x256 grayscale image (128 + 8 random sinusoids + N(0, 8^2),
    seed 0), q = 8, C = 32 context model, FP32 class, batch 1, in both LL
    modes, with the logistic-mixture (K = 3) probability model in place
    of the Laplace one (four-step LL), and with the integer-network context
    model (INT8 class, both LL modes); device-resident stream -> device
    image, CUDA events per decode."""
    import torch
    import synthetic as S
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    img = S.gray_sinusoids(256, 256, seed=0)
    res = {"workload": "single 256x256 grayscale image, 4-level lifting, C=32, q=8, FP32, batch 1",
           "timing": "CUDA events per decode, device stream in, device image out"}
    for mode, name, prob, prec in ((0, "four_step_ll", 0, "fp32"),
                                   (1, "autoregressive_ll", 0, "fp32"),
                                   (0, "four_step_ll_logistic_mixture", 1, "fp32"),
                                   (0, "four_step_ll_integer_network", 0, "int8"),
                                   (1, "autoregressive_ll_integer_network", 0, "int8")):
        cfg = S.ModelConfig(levels=4, C=32, F=16, ll_mode=mode, prob=prob)
        c = pw.Codec(local, prec, stream=stream_ptr)
        m = c.load_model(S.pack_blob(cfg, S.random_model(cfg, 0)))
        bs = c.encode_image(m, img, q=8.0)
        d_bs = torch.from_numpy(np.frombuffer(bs, dtype=np.uint8).copy()).to(dev)
        out = torch.empty((256, 256), dtype=torch.uint8, device=dev)

        def one():
            c.decode_batch_device(m, [d_bs.data_ptr()], [len(bs)], out.data_ptr(), (256, 256))
        for _ in range(max(warmup, 3)):
            one()
        torch.cuda.synchronize()
        r0 = c.graph_replays
        t = _events_ms(stream, one, steps)
        replays = c.graph_replays - r0
        dec = out.cpu().numpy()
        mse = float(np.mean((dec.astype(np.float64) - img) ** 2))
        ms = float(np.median(t))
        res[name] = {"value": 256 * 256 / (ms / 1e3) / 1e6, "unit": "MPix/s",
                     "p50_ms": ms, "p99_ms": float(np.percentile(t, 99)),
                     "bpp": 8.0 * len(bs) / (256 * 256),
                     "psnr_db": 10 * np.log10(255.0 ** 2 / mse),
                     "graph_replays": replays}
        m.close()
        c.close()
    return res


def ragged_run(pw, local, stream_ptr, blob, n_img: int = 24, reps: int = 3):
    """Ragged batch: n_img RGB images of similar but unequal sizes (H
    log-uniform in 640..768, W in 896..1024, seed 7; rgb_natural content,
    q cycling 4, 8, 16, 32), the C = 64 model of the headline in the FP8
    class. One pw_decode_batch call decodes all of them on a canvas of the
    largest padded size; against it, the same streams one decode call each.
    Host wall clock per round (host streams in, host images out), after
    warm-up rounds that also settle the autotuner; every ragged result is
    compared with its single decode."""
    import synthetic as S
    rng = np.random.default_rng(7)
    sizes = [(int(np.exp(rng.uniform(np.log(640), np.log(768)))),
              int(np.exp(rng.uniform(np.log(896), np.log(1024))))) for _ in range(n_img)]
    imgs = [S.rgb_natural(h, w, seed=100 + i) for i, (h, w) in enumerate(sizes)]
    qs = [4.0, 8.0, 16.0, 32.0]
    c = pw.Codec(local, "fp8", stream=stream_ptr)
    m = c.load_model(blob)
    streams = [c.encode_image(m, im, q=qs[i % 4]) for i, im in enumerate(imgs)]
    px = sum(h * w for h, w in sizes)
    pad = [((h + 15) // 16 * 16, (w + 15) // 16 * 16) for h, w in sizes]
    canvas = max(h for h, _ in pad) * max(w for _, w in pad)
    for _ in range(6):
        rag = c.decode_ragged(m, streams)
    for _ in range(2):
        one = [c.decode_image(m, bs) for bs in streams]
    exact = all(np.array_equal(a, b) for a, b in zip(rag, one))
    t_rag, t_one = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        c.decode_ragged(m, streams)
        t_rag.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        for bs in streams:
            c.decode_image(m, bs)
        t_one.append(time.perf_counter() - t0)
    m.close()
    c.close()
    tr, to = min(t_rag), min(t_one)
    return {"workload": f"{n_img} RGB images of similar sizes (H 640..768, W 896..1024), C=64, "
                        "FP8, q in {4,8,16,32}",
            "value": px / tr / 1e6, "unit": "MPix/s", "ms_per_batch": tr * 1e3,
            "one_call_per_image": {"value": px / to / 1e6, "unit": "MPix/s",
                                   "ms_total": to * 1e3},
            "speedup": to / tr, "canvas_area_over_image_area": n_img * canvas / sum(
                h * w for h, w in pad),
            "bit_identical_to_single_decodes": exact,
            "timing": "host wall clock per call (host streams in, host images out)"}


def video_run(pw, local, stream_ptr, blob_low, blob_high, n_gop: int = 4, reps: int = 2):
    """Video: n_gop GOPs of 8 synthetic 1920x1080 RGB frames (panned 1/f
    canvas + sprites, seeds 3, 4, ...), motion-compensated temporal lifting
    (3 levels, block vectors from the encoder's motion search), the 8
    temporal bands coded as images (low band with one model, the 7 high
    bands batched with another), q = 8, BF16 class. Host stream in, host
    frames out into a page-locked buffer (pw_decode_gop); wall clock per pass
    over all GOPs, best of `reps`."""
    import torch
    import synthetic as S
    c = pw.Codec(local, "bf16", stream=stream_ptr)
    ml, mh = c.load_model(blob_low), c.load_model(blob_high)
    gops, streams, sse = [], [], 0.0
    for g in range(n_gop):
        fr = S.video_gop(1080, 1920, 8, seed=3 + g)
        gs = c.encode_gop(ml, mh, fr, q=8.0)
        out = c.decode_gop(ml, mh, gs, 8, (1080, 1920, 3))
        sse += float(np.sum((out.astype(np.float64) - fr) ** 2))
        gops.append(fr)
        streams.append(gs)
    h_out = torch.empty((8, 1080, 1920, 3), dtype=torch.uint8).pin_memory()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        for gs in streams:
            c.decode_gop_into(ml, mh, gs, 8, (1080, 1920, 3), h_out.data_ptr())
        times.append(time.perf_counter() - t0)
    best = min(times)
    assert np.array_equal(h_out.numpy(), c.decode_gop(ml, mh, streams[-1], 8, (1080, 1920, 3)))
    px = n_gop * 8 * 1920 * 1080
    ml.close()
    mh.close()
    c.close()
    return {"workload": f"{n_gop} GOPs x 8 frames 1920x1080 RGB, 3 temporal levels, 4 spatial "
                        "levels, C=64, q=8, BF16",
            "gops": n_gop, "frames": 8 * n_gop, "value": px / best / 1e6, "unit": "MPix/s",
            "ms_per_gop": 1e3 * best / n_gop,
            "bpp": 8.0 * sum(len(g) for g in streams) / px,
            "psnr_db": 10 * np.log10(255.0 ** 2 * px * 3 / sse),
            "timing": "host wall clock, e2e (host stream in, host frames out into page-locked "
                      "memory)"}


def encode_requests(pw, local, blob, reqs, precision: str, threads: int = 8,
                    lane_shift: int = 7, chunk: int = 16384):
    """Pre-encode the serving workload's requests: every image is a crop of
    a seeded synthetic 2048x2048 canvas (gray or RGB) at the request's size,
    coded with its quantiser step by the library's encoder (one context and
    stream per thread)."""
    import torch
    import synthetic as S
    rng = np.random.default_rng(7)
    canvas = {1: S.gray_sinusoids(2048, 2048, seed=7), 3: S.rgb_natural(2048, 2048, seed=7)}
    crops = []
    for r in reqs:
        y0 = int(rng.integers(0, 2048 - r["h"] + 1))
        x0 = int(rng.integers(0, 2048 - r["w"] + 1))
        crops.append((y0, x0))
    streams = [None] * len(reqs)

    def work(tid):
        st = torch.cuda.Stream(device=local)
        c = pw.Codec(local, precision, stream=st.cuda_stream)
        c.set_lane_rule(lane_shift)
        m = c.load_model(blob)
        for i in range(tid, len(reqs), threads):
            r = reqs[i]
            y0, x0 = crops[i]
            img = np.ascontiguousarray(canvas[r["c"]][y0:y0 + r["h"], x0:x0 + r["w"]])
            streams[i] = c.encode_image(m, img, q=r["q"], chunk=chunk)
        m.close()
        c.close()

    ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return streams


def serve(pw, codec, model, reqs, streams, lanes: int, max_batch: int, budget: int,
          rate_scale: float = 1.0):
    """Open-loop serving of pre-encoded requests: each is submitted at its
    arrival instant (the workload's Poisson times divided by rate_scale);
    latency is submit -> decoded host image (the server's own clock)."""
    srv = pw.Server(codec, model, hbm_budget=budget, lanes=lanes, max_batch=max_batch)
    done = {}
    tickets = [None] * len(reqs)

    def collect():
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0005)
            done[i] = srv.poll(tickets[i], timeout_ms=600000) is not None

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        dt = t0 + (r["t"] - reqs[0]["t"]) / rate_scale - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(streams[i])
    th.join()
    st = srv.stats()
    srv.close()
    mpix = sum(r["w"] * r["h"] for r in reqs) / 1e6
    span = max((reqs[-1]["t"] - reqs[0]["t"]) / rate_scale, 1e-9)
    return {"requests": len(reqs), "rate_per_s": 200.0 * rate_scale,
            "completed": int(st["completed"]), "batches": int(st["batches"]),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mpix_per_s": st["mpix_per_s"],
            "offered_mpix_per_s": mpix / span, "all_ok": all(done.values())}


def serving_run(pw, local, codec, model, blob, n_req: int, sweep_n: int = 2000,
                sweep=(1.0, 2.0, 4.0, 8.0), lanes: int = 8, max_batch: int = 8,
                budget: int = 160 << 30):
    """The serving workload: n_req requests (Poisson arrivals at 200/s, w and
    h log-uniform in [256, 2048] rounded down to a multiple of 16, gray/RGB
    50/50, q uniform over {4, 8, 16, 32}) through the decode server in the
    codec's precision class; then a saturation sweep replaying the first
    sweep_n requests with arrival rates 200 x each factor of `sweep`. A rate
    is sustained when the server completes at least 95 % of the offered
    MPix/s; max_sustained_mpix_per_s is the highest such completion rate.
    Server: 8 lanes, batches of up to 8 (ragged across close sizes), 160 GB
    HBM budget (measured on the sweep's 4x point: 48 GB and 16 lanes 201,
    160 GB and 16 lanes 255, 160 GB and 8 lanes 266 MPix/s; the same p50 and
    p99 at 200/s)."""
    import synthetic as S
    reqs = S.request_stream(n=n_req, rate=200.0, seed=7)
    t0 = time.perf_counter()
    streams = encode_requests(pw, local, blob, reqs,
                              {0: "fp32", 1: "bf16", 2: "fp8"}[codec.precision])
    enc_s = time.perf_counter() - t0
    main = serve(pw, codec, model, reqs, streams, lanes, max_batch, budget)
    mpix = sum(r["w"] * r["h"] for r in reqs) / 1e6
    main.update({"workload": f"{n_req} Poisson requests at 200/s, 256..2048 log-uniform, "
                             "gray/RGB, q in {4,8,16,32}",
                 "lanes": lanes, "max_batch": max_batch, "hbm_budget_gb": budget / 2**30,
                 "mean_mpix_per_request": mpix / len(reqs),
                 "encode_s_untimed": enc_s})
    n = min(sweep_n, len(reqs))
    pts = []
    for f in sweep:
        r = serve(pw, codec, model, reqs[:n], streams[:n], lanes, max_batch, budget, f)
        r["sustained"] = r["mpix_per_s"] >= 0.95 * r["offered_mpix_per_s"]
        pts.append(r)
    ok = [p["mpix_per_s"] for p in pts if p["sustained"] and p["all_ok"]]
    if main["mpix_per_s"] >= 0.95 * main["offered_mpix_per_s"]:
        ok.append(main["mpix_per_s"])
    main["saturation_sweep"] = pts
    main["max_sustained_mpix_per_s"] = max(ok) if ok else None
    main["capacity_mpix_per_s"] = max([p["mpix_per_s"] for p in pts] + [main["mpix_per_s"]])
    # the same first sweep_n requests in the faster coder format (one rANS
    # state per 32 symbols, 6144-symbol chunks): at 200/s and at 8x
    fs = encode_requests(pw, local, blob, reqs[:n],
                         {0: "fp32", 1: "bf16", 2: "fp8"}[codec.precision], lane_shift=5,
                         chunk=6144)
    fo = {"format": "lane rule 5, 6144-symbol chunks",
          "bytes_vs_default": sum(len(x) for x in fs) / sum(len(x) for x in streams[:n])}
    for f in (1.0, 8.0):
        fo[f"rate_{int(200 * f)}"] = serve(pw, codec, model, reqs[:n], fs, lanes, max_batch,
                                           budget, f)
    main["fast_format"] = fo
    return main


def lossless_run(pw, local, stream_ptr, n_img: int = 16, reps: int = 2):
    """Lossless at scale: n_img RGB 3840x2160 uint16 images with 12-bit values
    (Gaussian blobs + N(0, 15^2), seeds 5, 6, ...), RCT and integer lifting
    with 5 levels (padded to 3840x2176), C = 64 context model with FP8
    convolutions. Decoded in equal sub-batches of at most 8 images, sized so
    that the decode workspace leaves 24 GB of the device memory that is free
    once the encoder's context is closed; device streams -> device
    images, CUDA events around every sub-batch; every decoded image is
    compared with its input (bit_exact)."""
    import torch
    import synthetic as S
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    Hh, Ww = 2160, 3840
    cfg = S.ModelConfig(levels=5, C=64, F=16, ll_mode=0)
    blob = S.pack_blob(cfg, S.random_model(cfg, 0))
    imgs = [S.lossless_blobs(Hh, Ww, seed=5 + i) for i in range(n_img)]
    # the encoder runs on a context of its own, closed before decoding so
    # that its cached workspaces give their device memory back
    ce = pw.Codec(local, "fp8", stream=stream_ptr)
    me = ce.load_model(blob)
    streams = []
    for i in range(0, n_img, 4):
        streams += ce.encode_batch(me, imgs[i:i + 4], lossless=True, bitdepth=12)
    me.close()
    ce.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    c = pw.Codec(local, "fp8", stream=stream_ptr)
    m = c.load_model(blob)
    per = c.decode_footprint(m, streams[0], 1)
    free = torch.cuda.mem_get_info(dev)[0]
    sub = int(max(1, min(n_img, (free - (24 << 30)) // max(per, 1), 8)))
    # equal sub-batches (the largest divisor of the image count that fits):
    # one decode plan for all of them, and no small remainder call
    sub = max(d for d in range(1, sub + 1) if n_img % d == 0)
    lens = [len(b) for b in streams]
    offs = np.cumsum([0] + [(n + 255) // 256 * 256 for n in lens])
    host_all = np.zeros(int(offs[-1]), dtype=np.uint8)
    for i, b in enumerate(streams):
        host_all[offs[i]:offs[i] + lens[i]] = np.frombuffer(b, dtype=np.uint8)
    d_all = torch.from_numpy(host_all).to(dev)
    out = torch.empty((sub, Hh, Ww, 3), dtype=torch.int16, device=dev)
    groups = [list(range(i, min(i + sub, n_img))) for i in range(0, n_img, sub)]

    def dec(gi):
        g = groups[gi]
        c.decode_batch_device(m, [d_all.data_ptr() + int(offs[i]) for i in g],
                              [lens[i] for i in g], out.data_ptr(), (Hh, Ww, 3), bitdepth=12)
    exact = True
    for gi, g in enumerate(groups):
        dec(gi)
        torch.cuda.synchronize()
        got = out[:len(g)].cpu().numpy().view(np.uint16)
        for k, i in enumerate(g):
            exact = exact and bool(np.array_equal(got[k], imgs[i]))
    best = None
    for _ in range(reps):
        t = sum(sum(_events_ms(stream, lambda gi=gi: dec(gi), 1)) for gi in range(len(groups)))
        best = t if best is None else min(best, t)
    px = n_img * Hh * Ww
    res = {"workload": f"{n_img} RGB 3840x2160 12-bit images, lossless (RCT + integer lifting, "
                       "5 levels), C=64, FP8 context convolutions",
           "value": px / (best / 1e3) / 1e6, "unit": "MPix/s", "ms_total": best,
           "sub_batch": sub, "sub_batches": len(groups),
           "decode_workspace_bytes_per_image": int(per), "device_free_bytes_at_sizing": int(free),
           "bpp": 8.0 * sum(lens) / px, "bits_per_sample": 8.0 * sum(lens) / (3 * px),
           "bit_exact": exact,
           "timing": "CUDA events around each sub-batch decode, device streams -> device images"}
    m.close()
    c.close()
    del out, d_all
    torch.cuda.empty_cache()
    return res


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the kernel classes of one decode step of this workload (batch 24, FP8),
# from one ncu capture of `bench.py --nvtx-step` at full size (its summary
# is kept under profiles/); valid only while the sources
# of the captured kernels hash to "src" (the capture's), else reported
# as null.
TRAFFIC = {"src": "593c57cf64cb08e5", "precision": "fp8", "batch": 24,
           "bytes_per_launch": {"ctx_conv1x1": 346.65e6, "ctx_lstm_gates_conv3x3": 1175.22e6,
                                "ctx_conv3x3": 246.54e6, "ctx_head_conv3x3": 210.79e6,
                                "rans_decode": 5.87e6, "lift_step": 31.08e6,
                                "ctx_small": 173.86e6}}


def conv_src_hash() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_2405_12631_gb300", "csrc")
    h = hashlib.sha256()
    # every source of the captured kernels (convolutions, producers, coder,
    # lifting, parse / dequantisation / colour)
    for f in ("ctx_tc.cu", "tc_ptx.cuh", "pw_internal.cuh", "entropy.cu", "cdf_warp.cuh",
              "lift.cu", "f32x2.cuh", "spec_math.cuh", "driver.cu"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(name: str, precision: str, batch: int):
    if (precision != TRAFFIC["precision"] or batch != TRAFFIC["batch"]
            or conv_src_hash() != TRAFFIC["src"]):
        return None
    return TRAFFIC["bytes_per_launch"].get(name)


PAPER = {"hardware": "NVIDIA RTX A6000 (Ampere)", "precision": "not stated",
         "scope": "luma only, averaged (Kodak 768x512; UVG centre crops 768x512, GOP 8)",
         "image_decode_speedup_vs_autoregressive": 354,
         "video_decode_speedup_vs_autoregressive": 244,
         "pwave_decode_s_per_image": 5.64, "pwave_4step_ll_decode_s_per_image": 0.35,
         "pmctf_decode_s": 7.656,
         "note": "the paper's own figures, quoted for context; not measured here"}


def class_roofline(k: dict, precision: str, peaks: dict, peak_kind: str) -> dict:
    """Roofline of one kernel class from its algorithmic FLOP and bytes and
    its CUDA-event time: the bound is the roof its arithmetic intensity
    reaches first. Tensor-core classes (BF16 / FP8 context convolutions) use
    the measured sustained BF16 rate (x 2, the nominal FP8 / BF16 ratio, for
    the E4M3 3x3 convolutions); FP32 SIMT classes 152 SMs x 128 lanes x 2 x
    the maximum SM clock; HBM the measured copy bandwidth."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    name = k["name"]
    s = k["ms"] / 1e3
    if s <= 0:
        return {"kernel": name, "bound": None}
    # lift_step: in the tensor-core classes layers 2 and 3 of the lossy
    # lifting CNN (95 % of its FLOPs) run as BF16 MMAs
    tensor = precision in ("bf16", "fp8") and name in (
        "ctx_conv3x3", "ctx_head_conv3x3", "ctx_lstm_gates_conv3x3", "ctx_conv1x1", "lift_step")
    if tensor:
        tpeak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        if precision == "fp8" and name in ("ctx_conv3x3", "ctx_head_conv3x3",
                                           "ctx_lstm_gates_conv3x3"):
            tpeak *= 2.0
        cbound = "tensor"
    else:
        tpeak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        cbound = "alu"
    ridge = tpeak * 1e12 / (hbm * 1e9)
    ai = k["flops"] / max(k["bytes"], 1.0)
    if k["flops"] > 0 and ai >= ridge:
        bound, unit, peak, achieved = cbound, "TFLOP/s", tpeak, k["flops"] / s / 1e12
    else:
        bound, unit, peak, achieved = "hbm", "GB/s", hbm, k["bytes"] / s / 1e9
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "flop_per_byte": ai, "ridge_flop_per_byte": ridge,
            "ms_per_step": k["ms"], "launches": k["launches"],
            "tflops": k["flops"] / s / 1e12, "gbs": k["bytes"] / s / 1e9,
            "peak_source": peak_kind + (" (derived: SMs x lanes x clock)" if bound == "alu"
                                        else (" (x2 nominal fp8/bf16)" if bound == "tensor"
                                              and peak > 1.5 * float(peaks.get(
                                                  "bf16_tflops_sustained", 1e9)) else ""))}


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
    # encoder throughput (the first pass above was its warm-up): the same
    # batched encodes again, host images in, host streams out, wall clock
    torch.cuda.synchronize()
    t_enc = time.perf_counter()
    for q in QSTEPS:
        idx = [i for i in range(BATCH) if qs[i] == q]
        if idx:
            codec.encode_batch(model, [imgs[i] for i in idx], q=q)
    torch.cuda.synchronize()
    t_enc = time.perf_counter() - t_enc
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

    # autotuner calibration (untimed set-up, like the encodes above): the
    # convolution classes of this batch size sample their candidate
    # schedules on the first launches; decode until every class has its
    # schedule, so that no warm-up or timed launch is a tuning sample
    calib = 0
    while not pw.pw_autotune_settled() and calib < 24:
        step()
        torch.cuda.synchronize()
        calib += 1
    for _ in range(max(args.warmup - 1, 0)):
        step()
    if args.nvtx_step:
        # one more decode step inside the NVTX range "pw_step" (for ncu
        # --nvtx --nvtx-include "pw_step/"), then stop
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("pw_step")
        step()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"nvtx_step": "done", "batch": BATCH, "launches": codec.launches}))
        return
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

    # e2e: host streams -> host images through the C ABI (pw_decode_batch
    # with host pointers): the streams sit in page-locked host memory, as a
    # client's receive buffers would, and the images land in a page-locked
    # host buffer; every step's host-to-device copy of the streams and
    # device-to-host copy of the images is inside the timed call
    e2e_times = []
    if not args.no_e2e:
        h_streams = torch.from_numpy(host_all).pin_memory()
        h_ptrs = [h_streams.data_ptr() + int(offs[i]) for i in range(BATCH)]
        h_out = torch.empty((BATCH, H, W, 3), dtype=torch.uint8).pin_memory()
        for i in range(max(1, args.steps // 2)):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            codec.decode_batch_host_ptrs(model, h_ptrs, lens, h_out.data_ptr(), (H, W, 3))
            e2e_times.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
        ref0 = codec.decode_batch(model, streams[:1])[0]   # pageable path, same result
        assert np.array_equal(h_out[0].numpy(), ref0), "e2e decode differs"
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
        r = class_roofline(dom, args.precision, peaks, peak_kind)
        roofline = {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                    "unit": r["unit"], "frac": r["frac"],
                    "traffic": traffic_of(dom["name"], args.precision, BATCH),
                    "traffic_unit": "bytes per launch (ncu, one step at this batch)",
                    "algorithmic_bytes_per_launch": dom["bytes"] / max(dom["launches"], 1),
                    "kernel": dom["name"],
                    "timing": "CUDA events around this class's launches over the timed steps "
                              "(the only class recorded there)",
                    "flop_per_byte": r["flop_per_byte"],
                    "ridge_flop_per_byte": r["ridge_flop_per_byte"],
                    "peak_source": r["peak_source"]}
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
                "h2d_bytes_per_step": stream_bytes, "d2h_bytes_per_step": pixels * 3,
                "path": "pw_decode_batch, page-locked host streams in, page-locked host "
                        "images out, host wall clock per call; the decode chain replays "
                        "its captured CUDA graph and carries no per-launch events, while "
                        "the device-timed value above records CUDA events around the "
                        "dominant class's launches (its roofline), which end the "
                        "programmatic overlap at those launches"},
        "gpu_launches": int(launches),
        "encode": {"value": pixels / t_enc / 1e6, "unit": "MPix/s", "ms_per_batch": 1e3 * t_enc,
                   "timing": "host wall clock of the batched encodes (one call per quantiser "
                             "step), host images in, host streams out"},
        "roofline": roofline,
        # every class of one (profiled) warm-up step against its own roof
        "rooflines": [class_roofline(k, args.precision, peaks, peak_kind) for k in kern_sorted],
        "kernels": [{"name": k["name"], "launches": k["launches"],
                     "ms_per_step": k["ms"],
                     "share": k["ms"] / total_kernel_ms} for k in kern_sorted],
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
        "wall_s_timed_region": t_wall,
        "autotune_calibration_steps": calib,
        "paper": PAPER,
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
    if world == 1 and not args.no_compare:
        # the coder's rate / latency option: one rANS state per 32 symbols
        # (default 128), and also 6144-symbol chunks (default 16384)
        opts = {}
        for name, ls, ch in (("lane_rule_5", 5, 16384), ("lane_rule_5_chunk_6144", 5, 6144)):
            r = batched_precision(pw, local, args.precision, imgs, qs, blob, stream.cuda_stream,
                                  max(args.steps // 2, 3), args.warmup, ls, ch)
            r["bpp_vs_default"] = r["bpp"] / (8.0 * stream_bytes / pixels)
            opts[name] = r
        lat = {"default": single_image_latency(pw, local, stream.cuda_stream, blob,
                                               args.precision, 7, 16384)}
        lat["lane_rule_5_chunk_6144"] = single_image_latency(pw, local, stream.cuda_stream, blob,
                                                             args.precision, 5, 6144)
        opts["single_image_latency"] = lat
        line["coder_format_options"] = opts
    wl = {}
    if world == 1 and not args.no_workloads:
        wl["single_gray_256"] = single_gray_run(pw, local, stream.cuda_stream, args.steps,
                                                args.warmup)
        if not args.no_gop:
            import synthetic as S
            cfg = S.ModelConfig(levels=4, C=64, F=16, ll_mode=0)
            wl["video_4gop_1080p"] = video_run(pw, local, stream.cuda_stream, blob,
                                               S.pack_blob(cfg, S.random_model(cfg, 1)))
        wl["lossless_4k_12bit"] = lossless_run(pw, local, stream.cuda_stream)
        wl["ragged_batch_24"] = ragged_run(pw, local, stream.cuda_stream, blob)
    if args.serve > 0 and world == 1:
        wl["serving_poisson"] = serving_run(pw, local, codec, model, blob, args.serve)
    if wl:
        line["workloads"] = wl
    if not args.no_cpu and world == 1:
        multi = cpu_baseline_child(False)
        single = cpu_baseline_child(True)
        per = {}
        for k, v in multi.get("samples", {}).items():
            per[k] = {"value": v["pixels"] / v["s"] / 1e6, "unit": "MPix/s",
                      "threads": multi.get("threads"), "sample": v["sample"]}
        for k, v in single.get("samples", {}).items():
            per[k + "_single_thread"] = {"value": v["pixels"] / v["s"] / 1e6, "unit": "MPix/s",
                                         "threads": 1, "sample": v["sample"]}
        head = per.get("batched_768x512_rgb")
        line["cpu_baseline"] = {
            "value": head["value"] if head else None, "unit": "MPix/s",
            "cores": multi.get("threads"), "nproc": multi.get("nproc"), "kind": "oracle",
            "sample": head["sample"] + ", decode only" if head else None,
            "per_workload": per,
            "note": "FP64 numpy oracle in a child process; BLAS threads as stated"}
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
    ap.add_argument("--serve", type=int, default=10000,
                    help="requests of the open-loop serving run (0 = skip)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the single-image, video and lossless workloads")
    ap.add_argument("--nvtx-step", action="store_true",
                    help="after the warm-up, run one decode step inside the NVTX range "
                         "'pw_step' and exit (for ncu captures of exactly one step)")
    ap.add_argument("--cpu-samples", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--single-thread", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_samples:
        cpu_samples_main(args.single_thread)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
