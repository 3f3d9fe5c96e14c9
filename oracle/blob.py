"""Reader for the weight-blob file format (test infrastructure only).

Parses the little-endian "PWMB" container (header, 64-byte tensor records,
256-byte aligned float32 data) into a config dict and named float64 arrays.
Also computes the model hash that bitstreams carry to bind a stream to the
model that made it.
"""
from __future__ import annotations

import struct

import numpy as np


def read_blob(blob: bytes):
    """Return (cfg, tensors): cfg has levels, C, F, ll_mode; tensors are FP64."""
    if blob[:4] != b"PWMB":
        raise ValueError("not a weight blob")
    ver, levels, C, F, ll_mode, n, _ = struct.unpack_from("<7I", blob, 4)
    if ver != 1:
        raise ValueError("unsupported blob version")
    tensors = {}
    for i in range(n):
        rec = blob[32 + 64 * i: 32 + 64 * (i + 1)]
        name = rec[:40].split(b"\0", 1)[0].decode("ascii")
        ndim, d0, d1, d2, d3, off = struct.unpack_from("<6I", rec, 40)
        shape = (d0, d1, d2, d3)[:ndim]
        cnt = int(np.prod(shape))
        arr = np.frombuffer(blob, dtype="<f4", count=cnt, offset=off)
        tensors[name] = arr.reshape(shape).astype(np.float64)
    cfg = dict(levels=levels, C=C, F=F, ll_mode=ll_mode)
    return cfg, tensors


def model_hash(blob: bytes) -> int:
    """64-bit polynomial hash of the blob's little-endian u32 words.

    h = sum_i (w_i + 1) * P^(i+1) mod 2^64 with P = 0x100000001B3, where w_i
    is the i-th u32 word (the blob length is a multiple of 256 bytes).
    """
    w = np.frombuffer(blob, dtype="<u4").astype(np.uint64)
    P = np.uint64(0x100000001B3)
    with np.errstate(over="ignore"):
        pw = np.cumprod(np.full(w.shape[0], P, dtype=np.uint64), dtype=np.uint64)
        h = np.sum((w + np.uint64(1)) * pw, dtype=np.uint64)
    return int(h)
