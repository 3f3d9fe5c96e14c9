"""Seeded random-init weights and the flat weight-blob file format.

The paper trains one model per rate-distortion trade-off lambda (Section
4.1); trained weights are not available, so seeded random-init weights of the
same architecture stand in for them. This module only draws the numbers and
serialises them; the architecture that consumes them is implemented twice,
independently, by the oracle and by the CUDA library, which both look
tensors up by name in the blob.

Blob layout (little endian):
  0   char[4]  magic "PWMB"
  4   u32      version (1)
  8   u32      levels (number of wavelet decomposition levels)
  12  u32      C  (context-model channels)
  16  u32      F  (lifting CNN channels)
  20  u32      ll_mode (0: four-step LL model, 1: autoregressive LL model)
  24  u32      n_tensors
  28  u32      reserved (0)
  32  records, 64 bytes each: char name[40] (NUL padded), u32 ndim,
      u32 shape[4] (unused dims 1), u32 byte offset of the data from the
      blob start
  ... float32 data, each tensor starting on a 256-byte boundary
"""
from __future__ import annotations

import dataclasses
import struct

import numpy as np

MAGIC = b"PWMB"
VERSION = 1


@dataclasses.dataclass(frozen=True)
class ModelConfig:
    levels: int = 4
    C: int = 32
    F: int = 16
    ll_mode: int = 0  # 0 four-step LL, 1 autoregressive LL
    post: int = 0     # 1: the blob carries a post-processing CNN ("post.*")
    prob: int = 0     # 0: Laplace heads (2 outputs), 1: logistic mixture K = 3 (9)


def tensor_specs(cfg: ModelConfig):
    """(name, shape) of every parameter tensor, in blob order.

    Lifting predict/update CNNs (shared by all levels), one per direction
    (row, col) and operator (P, U): conv3x3 1->F, conv3x3 F->F, conv3x3 F->1;
    the same structure for the temporal lifting of GOPs ("tlift", P and U).
    With cfg.post, a post-processing CNN ("post", same structure) follows.
    Context prediction: ConvLSTM input conv (1->C, 3x3) and gate conv
    (2C->4C, 3x3, gate order i, f, o, g). Context fusion nets for subbands
    2..13 ("sb"), and either four-step nets for LL ("ll", ll_mode 0) or the
    autoregressive LL model ("ar", ll_mode 1). 1x1 weights are [Cout, Cin].
    Heads have 2 outputs (Laplace mean, scale pre-activation) or, with
    cfg.prob = 1 (four-step LL only), 9 (logistic mixture: 3 weight logits,
    3 means, 3 scale pre-activations).
    """
    C, F = cfg.C, cfg.F
    NH = 9 if cfg.prob else 2
    assert not (cfg.prob and cfg.ll_mode), "mixture heads need the four-step LL model"
    s = []
    for d in ("row", "col"):
        for op in ("P", "U"):
            p = f"lift.{d}.{op}."
            s += [(p + "w1", (F, 1, 3, 3)), (p + "b1", (F,)),
                  (p + "w2", (F, F, 3, 3)), (p + "b2", (F,)),
                  (p + "w3", (1, F, 3, 3)), (p + "b3", (1,))]
    for op in ("P", "U"):
        p = f"tlift.{op}."
        s += [(p + "w1", (F, 1, 3, 3)), (p + "b1", (F,)),
              (p + "w2", (F, F, 3, 3)), (p + "b2", (F,)),
              (p + "w3", (1, F, 3, 3)), (p + "b3", (1,))]
    if cfg.post:
        # post-processing CNN after the inverse transform (same structure)
        s += [("post.w1", (F, 1, 3, 3)), ("post.b1", (F,)),
              ("post.w2", (F, F, 3, 3)), ("post.b2", (F,)),
              ("post.w3", (1, F, 3, 3)), ("post.b3", (1,))]
    s += [("lstm.we", (C, 1, 3, 3)), ("lstm.be", (C,)),
          ("lstm.wg", (4 * C, 2 * C, 3, 3)), ("lstm.bg", (4 * C,))]
    sets = ["sb", "ll"] if cfg.ll_mode == 0 else ["sb"]
    for ns in sets:
        p = f"{ns}.s0."
        s += [(p + "win", (C, C)), (p + "bin", (C,)),
              (p + "w1", (C, C)), (p + "b1", (C,)),
              (p + "wdw", (C, 3, 3)), (p + "bdw", (C,)),
              (p + "w2", (C, C)), (p + "b2", (C,)),
              (p + "w3", (2 * C, C)), (p + "b3", (2 * C,)),
              (p + "w4", (C, 2 * C)), (p + "b4", (C,)),
              (p + "wh", (NH, C)), (p + "bh", (NH,))]
        for k in (1, 2, 3):
            p = f"{ns}.s{k}."
            s += [(p + "wa", (C, 1, 3, 3)), (p + "ba", (C,)),
                  (p + "wz", (C, 2 * C)), (p + "bz", (C,)),
                  (p + "w1", (C, C, 3, 3)), (p + "b1", (C,)),
                  (p + "w2", (C, C, 3, 3)), (p + "b2", (C,)),
                  (p + "wh", (NH, C)), (p + "bh", (NH,))]
    if cfg.ll_mode == 1:
        s += [("ar.w5", (C, 1, 5, 5)), ("ar.b5", (C,)),
              ("ar.w1", (C, C)), ("ar.b1", (C,)),
              ("ar.wh", (2, C)), ("ar.bh", (2,))]
    return s


def _init_scale(name: str, shape, cfg: ModelConfig) -> float:
    """Kaiming-uniform style bound for weight tensors, small for biases."""
    leaf = name.split(".")[-1]
    if leaf.startswith("b"):
        fan_in = 1
        return 0.05
    fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else 1
    base = np.sqrt(3.0 / max(fan_in, 1))
    if name.startswith("lift.") or name.startswith("tlift.") or name.startswith("post."):
        if leaf == "w1":          # input samples are of order +-128
            return base * (5.0 / 3.0) / 64.0
        if leaf == "w2":
            return base * (5.0 / 3.0)
        return base * 0.5         # residual output of order 1
    if name == "lstm.we" or name == "ar.w5" or leaf == "wa":
        return base * 0.25        # inputs are quantised symbols
    if leaf == "wh":
        return base * 0.1         # keeps initial means near zero
    if name == "lstm.wg":
        return base
    return base * np.sqrt(2.0)    # leaky-ReLU gain


def random_model(cfg: ModelConfig, seed: int = 0) -> dict:
    """Draw every tensor of `cfg` from a seeded PCG64 stream (float32).

    Heads get bias (0, softplus^-1(1.5)) so that initial scales are near 1.5
    quantisation steps (rates of a few bits per sample, as for a trained
    model at moderate quality), mixture heads equal weights, means 0 and
    scales 1; everything else is uniform in +-bound.
    """
    rng = np.random.default_rng(seed)
    out = {}
    for name, shape in tensor_specs(cfg):
        b = _init_scale(name, shape, cfg)
        t = rng.uniform(-b, b, shape).astype(np.float32)
        if name.endswith(".bh") and shape[0] == 2:
            t = np.array([0.0, np.log(np.expm1(1.5))], dtype=np.float32)
        elif name.endswith(".bh"):   # mixture: equal weights, mean 0, scale 1
            t = np.array([0.0] * 6 + [np.log(np.expm1(1.0))] * 3, dtype=np.float32)
        out[name] = t
    return out


def pack_blob(cfg: ModelConfig, tensors: dict) -> bytes:
    """Serialise `tensors` (named as in tensor_specs) into the blob format."""
    specs = tensor_specs(cfg)
    head = MAGIC + struct.pack("<7I", VERSION, cfg.levels, cfg.C, cfg.F,
                               cfg.ll_mode, len(specs), 0)
    rec_end = 32 + 64 * len(specs)
    off = (rec_end + 255) // 256 * 256
    recs, datas = [], []
    for name, shape in specs:
        t = np.ascontiguousarray(tensors[name], dtype="<f4")
        assert tuple(t.shape) == tuple(shape), (name, t.shape, shape)
        dims = list(shape) + [1] * (4 - len(shape))
        nm = name.encode("ascii")
        assert len(nm) < 40
        recs.append(nm.ljust(40, b"\0") + struct.pack("<6I", len(shape), *dims, off))
        datas.append((off, t.tobytes()))
        off = (off + t.nbytes + 255) // 256 * 256
    buf = bytearray(off)
    buf[:32] = head
    buf[32:rec_end] = b"".join(recs)
    for o, d in datas:
        buf[o:o + len(d)] = d
    return bytes(buf)
