"""pWave++ encode / decode and the bitstream container (test infrastructure).

Section 3.1 of the paper: one colour component at a time (YCbCr), learned
lifting DWT with 4 levels, scalar quantisation y~ = round(y * Delta) with
separate Delta_L (LL) and Delta_H (other subbands), dequantisation
y^ = y~ / Delta, coding of the subbands in a fixed order with the context
model of Section 3.2, and the inverse transform on the decoder side. Video
(Section 3.3): a GOP is split into temporal subbands that are coded
independently, the lowpass one with one model and the highpass ones with
another.

Readings where the paper is silent:
* colour: BT.601 full-range YCbCr for lossy RGB, the JPEG 2000 reversible
  colour transform (RCT) for lossless RGB; every component is level-shifted
  by 2^(bitdepth-1) before the transform;
* quantiser step q means Delta_L = Delta_H = 1/q (stored as FP32); the
  rounding decision is taken in FP32;
* images whose sides are not multiples of 2^levels are padded by whole-sample
  mirroring and cropped after decoding; output samples are floor(v + 1/2)
  (FP32), clipped to the bit depth;
* post-processing after the inverse transform (Section 3.1 names the module
  but not its layers): when the weight blob carries one ("post.*"), each
  reconstructed (padded, level-shifted) component plane x of a lossy image
  becomes x + CNN_post(x), CNN_post with the structure of the lifting CNN
  (conv3x3 1->F, tanh, conv3x3 F->F, tanh, conv3x3 F->1, zero padding);
  lossless images and the temporal bands of a GOP are not post-processed.

Bitstream ("PWBS", little endian): 64-byte header, then n_chunks + 1 u32
payload offsets, then the payload of rANS chunks in the order component,
subband (coding order), step; each step's positions (raster order) are split
into chunks of at most `chunk_symbols` symbols (see chunk_layout); a chunk of
n symbols is coded
with min(32, max(1, n >> s)) interleaved states (s = 7 unless header byte 52
says otherwise). In autoregressive-LL mode
the LL subband is one single-state chunk in raster order instead of four
steps.

  0 magic "PWBS"        4 u16 version (1)      6 u16 flags (1 lossless,
  8 u32 width          12 u32 height             2 autoregressive LL,
                                                 16 balanced chunks,
                                                 32 logistic-mixture
                                                 probability model; bits 2-3:
                                                 the precision class, which
                                                 the library records; 3 =
                                                 the integer-network context
                                                 model, which the oracle
                                                 writes and follows too)
 16 u8 ncomp           17 u8 levels            18 u8 bitdepth
 19 u8 colour (0 gray, 1 YCbCr, 2 RCT, 3 raw planes)
 20 f32 Delta_L        24 f32 Delta_H          28 u16 T   30 u8 log2 M
 31 u8 lanes           32 u32 chunk_symbols    36 u32 n_chunks
 40 u64 model hash     48 u32 payload bytes    52 u8 lane shift s: one
 interleaved state per 2^s symbols (0 = the default 7)      53..63 zero

GOP stream ("PWGP"): 0 magic, 4 u16 version, 6 u16 nframes, 8 u32 width,
12 u32 height, 16 u8 temporal levels, 17 u8 ncomp, 18 u16 zero, 20 u64 hash
of the lowpass model, 28 u64 hash of the highpass model; version 2 then
holds the block motion vectors of every temporal level and pair (the order
of lifting.gop_motion), each field ceil(Hp/16) x ceil(Wp/16) int8 pairs
(dy, dx) in raster order over the padded frame; then per temporal subband a
u32 length and a "PWBS" stream with colour 3. Version 1 (no vectors) is
zero motion.

Pins: decode(encode(x)) reproduces the quantised coefficients exactly and
the image to within the quantiser's reconstruction error, and exactly in
lossless mode (tests/test_oracle_codec.py); the YCbCr transform against the
BT.601 full-range matrices as JFIF prints them, the RCT against the JPEG
2000 definition, and the padding against an explicit whole-sample mirror
index table (tests/test_oracle_layer_pins.py).
"""
from __future__ import annotations

import struct

import numpy as np

from . import entropy as E
from . import intnet as I
from . import rans as R
from .blob import model_hash, read_blob
from .context import ContextModel, step_map, step_positions
from .lifting import (MC_BLOCK, Lifting, gop_luma, gop_motion, lift_cnn, net_of,
                      subband_shapes, temporal_forward, temporal_inverse)

LANES = 32
DEFAULT_CHUNK = 16384
f32 = np.float32

KR, KB = 0.299, 0.114
KG = 1.0 - KR - KB


class Model:
    """A parsed weight blob: lifting nets, context model, hash. integer:
    encode with the integer-network context model (oracle.intnet; streams
    say so in header bits 2-3 = 3, and decoding follows the stream)."""

    def __init__(self, blob: bytes, integer: bool = False):
        cfg, t = read_blob(blob)
        self.cfg = cfg
        self.levels = cfg["levels"]
        self.C = cfg["C"]
        self.ll_mode = cfg["ll_mode"]
        self.tensors = t
        self.lift = Lifting(t)
        self.post = net_of(t, "post.") if "post.w1" in t else None
        self.ctx = ContextModel(t, cfg["C"], cfg["ll_mode"])
        # logistic-mixture heads (9 outputs) instead of Laplace ones (2)
        self.mixture = cfg["ll_mode"] == 0 and t["sb.s0.wh"].shape[0] == 9
        self.hash = model_hash(blob)
        self.integer = integer
        self._intctx = None
        if integer and self.mixture:
            raise ValueError("the integer context model has Laplace heads")

    def int_context(self) -> I.IntContextModel:
        if self._intctx is None:
            self._intctx = I.IntContextModel(self.tensors, self.C, self.ll_mode)
        return self._intctx


# --------------------------------------------------------------------------
# colour
def colour_forward(img: np.ndarray, lossless: bool, bitdepth: int):
    """Image -> list of level-shifted component planes (FP64)."""
    off = float(1 << (bitdepth - 1))
    x = img.astype(np.float64)
    if x.ndim == 2:
        return [x - off], 0
    R_, G, B = x[:, :, 0], x[:, :, 1], x[:, :, 2]
    if lossless:
        Y = np.floor((R_ + 2 * G + B) / 4.0)
        return [Y - off, B - G, R_ - G], 2
    Y = KR * R_ + KG * G + KB * B
    Cb = (B - Y) / (2.0 * (1.0 - KB))
    Cr = (R_ - Y) / (2.0 * (1.0 - KR))
    return [Y - off, Cb, Cr], 1


def colour_inverse(planes, colour: int, bitdepth: int) -> np.ndarray:
    """Component planes -> image samples (FP64, before rounding)."""
    off = float(1 << (bitdepth - 1))
    if colour == 0:
        return planes[0] + off
    if colour == 2:
        Y, Cb, Cr = planes[0] + off, planes[1], planes[2]
        G = Y - np.floor((Cb + Cr) / 4.0)
        return np.stack([Cr + G, G, Cb + G], axis=2)
    Y, Cb, Cr = planes[0] + off, planes[1], planes[2]
    R_ = Y + 2.0 * (1.0 - KR) * Cr
    B = Y + 2.0 * (1.0 - KB) * Cb
    G = (Y - KR * R_ - KB * B) / KG
    return np.stack([R_, G, B], axis=2)


def to_samples(v: np.ndarray, bitdepth: int) -> np.ndarray:
    """floor(v + 1/2) decided in FP32, clipped to [0, 2^bitdepth - 1]."""
    r = np.floor((v.astype(f32) + f32(0.5)).astype(f32)).astype(np.float64)
    r = np.clip(r, 0, (1 << bitdepth) - 1)
    return r.astype(np.uint8 if bitdepth <= 8 else np.uint16)


def pad_plane(x: np.ndarray, mult: int) -> np.ndarray:
    """Whole-sample mirror padding up to multiples of `mult`."""
    h, w = x.shape
    H = -(-h // mult) * mult
    W = -(-w // mult) * mult

    def idx(n, N):
        i = np.arange(N)
        i = np.where(i < n, i, 2 * (n - 1) - i)
        return np.clip(i, 0, n - 1)

    return x[np.ix_(idx(h, H), idx(w, W))]


# --------------------------------------------------------------------------
# quantiser
def quantise(y: np.ndarray, delta32: np.float32) -> np.ndarray:
    """y~ = rint(y * Delta) with the decision taken in FP32."""
    return np.rint((y.astype(f32) * delta32).astype(f32)).astype(np.int64)


def dequantise(q: np.ndarray, delta32: np.float32) -> np.ndarray:
    """y^ = y~ / Delta (FP64)."""
    return q.astype(np.float64) / float(delta32)


# --------------------------------------------------------------------------
# context parameters
def int_params(t, j):
    """(mu, sigma) that the index decision maps exactly to (t, j): t / 16
    and the middle of scale bin j."""
    return (np.asarray(t, dtype=np.float64) / 16.0,
            E.sigma_of_bin(np.asarray(j)).astype(np.float64))


def context_params_all(model: Model, qsb: list):
    """Entropy parameters at every position of every subband, all symbols
    known: (mu, sigma) arrays, or for a mixture model [h, w, 9] arrays of
    (w_k, mu_k, sigma_k).

    Equivalent to what the decoder computes step by step, because each step
    only reads positions of earlier steps (the nets mask the rest).
    """
    if model.integer:
        return [int_params(t, j) for t, j in I.context_tj_all(model.int_context(), qsb)]
    cm = model.ctx
    out = []
    h = c = None
    for i, s in enumerate(qsb):
        s = s.astype(np.float64)
        H, W = s.shape
        if i == 0 and model.ll_mode == 1:
            out.append(cm.ar_params_all(s))
            continue
        if i == 0:
            l, ns = np.zeros((H, W, model.C)), "ll"
        else:
            up = qsb[i - 1].shape[0] < H
            h, c = cm.lstm(qsb[i - 1].astype(np.float64), h, c, up)
            l, ns = h, "sb"
        sm = step_map(H, W)
        if model.mixture:
            hd = np.zeros((H, W, E.MIX_K * 3))
            for k in range(4):
                hd = np.where((sm == k)[:, :, None], cm.step_head(k, s, l, ns), hd)
            out.append(E.mix_params(hd))
            continue
        mu = np.zeros((H, W))
        sg = np.zeros((H, W))
        for k in range(4):
            m, g = cm.step_params(k, s, l, ns)
            mu = np.where(sm == k, m, mu)
            sg = np.where(sm == k, g, sg)
        out.append((mu, sg))
    return out


# --------------------------------------------------------------------------
# chunk layout
def chunk_layout(shapes, ncomp: int, ll_ar: bool, S: int, balanced: bool = True,
                 lane_shift: int = 7):
    """List of (comp, subband, step, first, count, lanes) in stream order.

    step is -1 for the single-state autoregressive LL chunk. A step's n
    symbols (raster order) form ceil(n / S) chunks: balanced (flag 16 of
    the stream header), the first n mod k of the k chunks hold
    floor(n / k) + 1 symbols and the rest floor(n / k), so that no chunk's
    serial decode is longer than it needs to be; otherwise chunks of S
    symbols and a shorter last one.
    """
    out = []
    for comp in range(ncomp):
        for i, (h, w, _) in enumerate(shapes):
            if i == 0 and ll_ar:
                if h * w:
                    out.append((comp, 0, -1, 0, h * w, 1))
                continue
            sm = step_map(h, w)
            for k in range(4):
                n = int(np.count_nonzero(sm == k))
                if balanced:
                    nch = -(-n // S)
                    first = 0
                    for j in range(nch):
                        cnt = n // nch + (1 if j < n % nch else 0)
                        out.append((comp, i, k, first, cnt, chunk_lanes(cnt, lane_shift)))
                        first += cnt
                else:
                    for first in range(0, n, S):
                        cnt = min(S, n - first)
                        out.append((comp, i, k, first, cnt, chunk_lanes(cnt, lane_shift)))
    return out


def chunk_lanes(n: int, lane_shift: int = 7) -> int:
    """Interleaved states of a chunk of n symbols: one per 2^lane_shift
    symbols (128 by default; header byte 52 holds another choice), between 1
    and 32 (each state costs 4 bytes of flush)."""
    return min(LANES, max(1, n >> lane_shift))


def coding_tables(model: Model, par, ys, xs, bank):
    """Centres (ctr) and CDF tables ([n, NSYM + 1]) of the symbols at
    (ys, xs) of one subband; par is the subband's (mu, sigma), or its
    mixture parameters [h, w, 9] (w_k, mu_k, sigma_k)."""
    if model.mixture:
        ctr, q, j, g = E.mix_decision(par[ys, xs])
        return ctr, E.mix_tables(q, j, g).astype(np.int64)
    mu, sg = par
    ctr, phi, j = E.index_decision(mu[ys, xs], sg[ys, xs])
    return ctr, bank[E.table_id(phi, j)]


def _sym_positions(h, w, step):
    if step < 0:
        ys, xs = np.nonzero(np.ones((h, w), dtype=bool))
        return ys, xs
    return step_positions(h, w, step)


# --------------------------------------------------------------------------
# encode
def encode_planes(model: Model, planes: list, *, width: int, height: int,
                  bitdepth: int, colour: int, q: float = 8.0,
                  lossless: bool = False, chunk: int = DEFAULT_CHUNK, lane_shift: int = 7):
    """Encode level-shifted component planes (already padded)."""
    L = model.levels
    Hp, Wp = planes[0].shape
    shapes = subband_shapes(Hp, Wp, L)
    d32 = f32(1.0) if lossless else f32(1.0 / q)
    qcomp = []
    for x in planes:
        sb = model.lift.forward(x, L, lossless)
        qcomp.append([quantise(s, d32) for s in sb])
    return _encode_symbols(model, qcomp, shapes, width=width, height=height,
                           bitdepth=bitdepth, colour=colour, d32=d32,
                           lossless=lossless, chunk=chunk, lane_shift=lane_shift), qcomp


def _encode_symbols(model, qcomp, shapes, *, width, height, bitdepth, colour,
                    d32, lossless, chunk, params=None, lane_shift=7):
    """Entropy-code quantised subbands. params, if given, replaces the
    context model: params[comp][subband] = (mu, sigma) arrays of the
    subband's shape (index injection: the coder alone is then exercised on
    another implementation's entropy parameters; a mixture model's params
    are [h, w, 9] arrays of (w_k, mu_k, sigma_k) instead)."""
    bank = E.cdf_bank().astype(np.int64)
    ll_ar = model.ll_mode == 1
    if params is None:
        params = [context_params_all(model, qsb) for qsb in qcomp]
    layout = chunk_layout(shapes, len(qcomp), ll_ar, chunk, True, lane_shift)
    payload = []
    offsets = [0]
    for comp, i, k, first, n, nl in layout:
        h, w, _ = shapes[i]
        ys, xs = _sym_positions(h, w, k)
        ys, xs = ys[first:first + n], xs[first:first + n]
        ctr, tabs = coding_tables(model, params[comp][i], ys, xs, bank)
        vals = qcomp[comp][i][ys, xs]
        ops = [R.symbol_ops(int(vals[p] - ctr[p]), tabs[p]) for p in range(n)]
        st, words = R.encode_chunk(ops, nl)
        b = R.pack_chunk(st, words)
        payload.append(b)
        offsets.append(offsets[-1] + len(b))
    flags = ((1 if lossless else 0) | (2 if ll_ar else 0) | 16 | (32 if model.mixture else 0) |
             (12 if model.integer else 0))
    head = (b"PWBS" + struct.pack("<HHIIBBBBffHBBIIQI", 1, flags, width, height,
                                  len(qcomp), model.levels, bitdepth, colour,
                                  float(d32), float(d32), E.T, E.LOG2M, LANES,
                                  chunk, len(layout), model.hash, offsets[-1]))
    head = (head + bytes([0 if lane_shift == 7 else lane_shift])).ljust(64, b"\0")
    return head + np.asarray(offsets, dtype="<u4").tobytes() + b"".join(payload)


def encode_image(blob: bytes, img: np.ndarray, *, q: float = 8.0,
                 lossless: bool = False, bitdepth: int | None = None,
                 chunk: int = DEFAULT_CHUNK, lane_shift: int = 7,
                 integer: bool = False) -> bytes:
    """Encode an (h, w) or (h, w, 3) uint8/uint16 image (integer: with the
    integer-network context model)."""
    model = Model(blob, integer=integer)
    if bitdepth is None:
        bitdepth = 8 if img.dtype == np.uint8 else 16
    planes, colour = colour_forward(img, lossless, bitdepth)
    mult = 1 << model.levels
    planes = [pad_plane(p, mult) for p in planes]
    bs, _ = encode_planes(model, planes, width=img.shape[1], height=img.shape[0],
                          bitdepth=bitdepth, colour=colour, q=q,
                          lossless=lossless, chunk=chunk, lane_shift=lane_shift)
    return bs


# --------------------------------------------------------------------------
# decode
def parse_header(bs: bytes) -> dict:
    if bs[:4] != b"PWBS":
        raise ValueError("not a PWBS stream")
    (ver, flags, width, height, ncomp, levels, bitdepth, colour, dl, dh, T,
     log2m, lanes, chunk, nch, mhash, pbytes) = struct.unpack_from(
        "<HHIIBBBBffHBBIIQI", bs, 4)
    offs = np.frombuffer(bs, dtype="<u4", count=nch + 1, offset=64).astype(np.int64)
    base = 64 + 4 * (nch + 1)
    return dict(version=ver, lossless=bool(flags & 1), ll_ar=bool(flags & 2),
                balanced=bool(flags & 16), mixture=bool(flags & 32),
                integer=((flags >> 2) & 3) == 3,
                lane_shift=bs[52] or 7,
                width=width, height=height, ncomp=ncomp, levels=levels,
                bitdepth=bitdepth, colour=colour, delta_l=f32(dl), delta_h=f32(dh),
                T=T, log2m=log2m, lanes=lanes, chunk=chunk, n_chunks=nch,
                model_hash=mhash, payload_bytes=pbytes, offsets=offs,
                payload_base=base)


def encode_symbols_with_params(model: Model, qcomp: list, params: list, *, width: int,
                               height: int, bitdepth: int, colour: int, q: float = 8.0,
                               lossless: bool = False, chunk: int = DEFAULT_CHUNK,
                               lane_shift: int = 7) -> bytes:
    """A PWBS stream of the given quantised subbands (per component, coding
    order) coded with the given entropy parameters instead of the context
    model's (four-step subbands only)."""
    L = model.levels
    mult = 1 << L
    Hp = -(-height // mult) * mult
    Wp = -(-width // mult) * mult
    d32 = f32(1.0) if lossless else f32(1.0 / q)
    return _encode_symbols(model, qcomp, subband_shapes(Hp, Wp, L), width=width,
                           height=height, bitdepth=bitdepth, colour=colour, d32=d32,
                           lossless=lossless, chunk=chunk, params=params,
                           lane_shift=lane_shift)


def decode_symbols(model: Model, bs: bytes, params: list | None = None):
    """Decode the quantised subbands of every component (list of lists).

    params, if given, replaces the context model of the four-step subbands
    (params[comp][subband] = (mu, sigma) over the whole subband, or the
    mixture's [h, w, 9] (w_k, mu_k, sigma_k); only the values at each step's
    positions are read)."""
    hd = parse_header(bs)
    if hd["model_hash"] != model.hash:
        raise ValueError("stream was made with another model")
    if hd["mixture"] != model.mixture:
        raise ValueError("probability model of the stream and the model differ")
    integer = hd["integer"]
    if integer and hd["mixture"]:
        raise ValueError("integer context model streams use Laplace tables")
    ic = model.int_context() if integer else None
    L = hd["levels"]
    mult = 1 << L
    Hp = -(-hd["height"] // mult) * mult
    Wp = -(-hd["width"] // mult) * mult
    shapes = subband_shapes(Hp, Wp, L)
    layout = chunk_layout(shapes, hd["ncomp"], hd["ll_ar"], hd["chunk"], hd["balanced"],
                          hd["lane_shift"])
    if len(layout) != hd["n_chunks"]:
        raise ValueError("chunk count mismatch")
    bank = E.cdf_bank().astype(np.int64)
    cm = model.ctx
    offs = hd["offsets"]
    base = hd["payload_base"]
    chunks = {}
    for ci, (comp, i, k, first, n, nl) in enumerate(layout):
        chunks.setdefault((comp, i, k), []).append((ci, first, n, nl))
    out = []
    for comp in range(hd["ncomp"]):
        qsb = [np.zeros((h, w), dtype=np.int64) for h, w, _ in shapes]
        h_state = c_state = None
        for i, (H, W, _) in enumerate(shapes):
            s = qsb[i]
            if i == 0 and hd["ll_ar"]:
                for ci, first, n, nl in chunks.get((comp, 0, -1), []):
                    buf = bs[base + offs[ci]: base + offs[ci + 1]]
                    st, words = R.unpack_chunk(buf, nl)
                    cur = {}

                    def table_of(p, s=s, cur=cur, W=W):
                        y, x = divmod(p, W)
                        if integer:
                            mu, sg = int_params(*ic.ar_tj_at(s, y, x))
                        else:
                            mu, sg = cm.ar_params_at(s.astype(np.float64), y, x)
                        ctr, phi, j = E.index_decision(mu, sg)
                        cur[p] = int(ctr)
                        return bank[int(E.table_id(phi, j))]

                    def on_symbol(p, r, s=s, cur=cur, W=W):
                        y, x = divmod(p, W)
                        s[y, x] = cur[p] + r

                    _, used, xf = R.decode_chunk(st, words, n, nl, table_of, on_symbol)
                    _check_chunk(used, len(words), xf)
                continue
            if params is not None:
                l = ns = None
            elif integer and i == 0:
                l, ns = np.zeros((H, W, model.C), dtype=np.int64), "ll"
            elif integer:
                up = shapes[i - 1][0] < H
                h_state, c_state = ic.lstm(qsb[i - 1], h_state, c_state, up)
                l, ns = h_state, "sb"
            elif i == 0:
                l, ns = np.zeros((H, W, model.C)), "ll"
            else:
                up = shapes[i - 1][0] < H
                h_state, c_state = cm.lstm(qsb[i - 1].astype(np.float64),
                                           h_state, c_state, up)
                l, ns = h_state, "sb"
            for k in range(4):
                if params is not None:
                    par = params[comp][i]
                elif integer:
                    par = int_params(*ic.step_tj(k, s, l, ns))
                elif model.mixture:
                    par = E.mix_params(cm.step_head(k, s.astype(np.float64), l, ns))
                else:
                    par = cm.step_params(k, s.astype(np.float64), l, ns)
                ys, xs = step_positions(H, W, k)
                ctr, tabs = coding_tables(model, par, ys, xs, bank)
                for ci, first, n, nl in chunks.get((comp, i, k), []):
                    buf = bs[base + offs[ci]: base + offs[ci + 1]]
                    st, words = R.unpack_chunk(buf, nl)
                    r, used, xf = R.decode_chunk(
                        st, words, n, nl, lambda p, f=first: tabs[f + p])
                    _check_chunk(used, len(words), xf)
                    sl = slice(first, first + n)
                    s[ys[sl], xs[sl]] = ctr[sl] + np.asarray(r, dtype=np.int64)
        out.append(qsb)
    return hd, out


def _check_chunk(used, nwords, xf):
    if used != nwords or any(v != R.L for v in xf):
        raise ValueError("corrupt chunk")


def reconstruct_planes(model: Model, hd: dict, qcomp: list):
    """Dequantise and inverse-transform every component (padded planes)."""
    L = hd["levels"]
    out = []
    for qsb in qcomp:
        sb = [dequantise(q, hd["delta_l"] if i == 0 else hd["delta_h"])
              for i, q in enumerate(qsb)]
        out.append(model.lift.inverse(sb, L, hd["lossless"]))
    return out


def post_process(model: Model, hd: dict, planes: list) -> list:
    """x + CNN_post(x) per padded component plane (lossy images of a model
    with a post-processing net); the planes themselves otherwise."""
    if model.post is None or hd["lossless"]:
        return planes
    return [p + lift_cnn(p, model.post) for p in planes]


def decode_image(blob: bytes, bs: bytes) -> np.ndarray:
    """Decode a PWBS image stream to uint8/uint16 samples."""
    model = Model(blob)
    hd, qcomp = decode_symbols(model, bs)
    planes = post_process(model, hd, reconstruct_planes(model, hd, qcomp))
    h, w = hd["height"], hd["width"]
    planes = [p[:h, :w] for p in planes]
    v = colour_inverse(planes, hd["colour"], hd["bitdepth"])
    return to_samples(v, hd["bitdepth"])


# --------------------------------------------------------------------------
# GOPs (Section 3.3)
def encode_gop(blob_l: bytes, blob_h: bytes, frames: np.ndarray, *, q: float = 8.0,
               tlevels: int = 3, chunk: int = DEFAULT_CHUNK, motion: bool = True) -> bytes:
    """Encode nframes = 2^tlevels RGB (or gray) uint8 frames; motion=False
    writes a version-1 (zero-motion) stream."""
    ml, mh = Model(blob_l), Model(blob_h)
    nf = frames.shape[0]
    assert nf == 1 << tlevels
    h, w = frames.shape[1], frames.shape[2]
    comps = [colour_forward(frames[f], False, 8)[0] for f in range(nf)]
    nc = len(comps[0])
    mult = 1 << ml.levels
    mvs = None
    if motion:
        luma = [pad_plane(gop_luma(frames[f]), mult) for f in range(nf)]
        mvs = gop_motion(luma, tlevels)
    bands_per_comp = []
    for c in range(nc):
        fr = [pad_plane(comps[f][c], mult) for f in range(nf)]
        bands_per_comp.append(temporal_forward(fr, ml.tensors, tlevels, mvs))
    out = [b"PWGP" + struct.pack("<HHIIBBHQQ", 2 if motion else 1, nf, w, h, tlevels, nc, 0,
                                 ml.hash, mh.hash)]
    if motion:
        out.append(b"".join(np.asarray(v, dtype=np.int8).tobytes() for v in mvs))
    for b in range(nf):
        m = ml if b == 0 else mh
        planes = [bands_per_comp[c][b] for c in range(nc)]
        bs, _ = encode_planes(m, planes, width=w, height=h, bitdepth=8, colour=3,
                              q=q, lossless=False, chunk=chunk)
        out.append(struct.pack("<I", len(bs)) + bs)
    return b"".join(out)


def decode_gop(blob_l: bytes, blob_h: bytes, gs: bytes) -> np.ndarray:
    ml, mh = Model(blob_l), Model(blob_h)
    if gs[:4] != b"PWGP":
        raise ValueError("not a PWGP stream")
    ver, nf, w, h, tlevels, nc, _, hl, hh = struct.unpack_from("<HHIIBBHQQ", gs, 4)
    if ver not in (1, 2):
        raise ValueError("unsupported PWGP version")
    pos = 4 + struct.calcsize("<HHIIBBHQQ")
    mvs = None
    if ver == 2:
        mult = 1 << ml.levels
        nby = -(-(-(-h // mult) * mult) // MC_BLOCK)
        nbx = -(-(-(-w // mult) * mult) // MC_BLOCK)
        mvs = []
        for _ in range(nf - 1):
            n = nby * nbx * 2
            mvs.append(np.frombuffer(gs, dtype=np.int8, count=n, offset=pos)
                       .astype(np.int64).reshape(nby, nbx, 2))
            pos += n
    bands = []
    for b in range(nf):
        (n,) = struct.unpack_from("<I", gs, pos)
        pos += 4
        bs = gs[pos:pos + n]
        pos += n
        m = ml if b == 0 else mh
        hd, qcomp = decode_symbols(m, bs)
        bands.append(reconstruct_planes(m, hd, qcomp))
    frames = []
    per_comp = []
    for c in range(nc):
        per_comp.append(temporal_inverse([bands[b][c] for b in range(nf)],
                                         ml.tensors, tlevels, mvs))
    colour = 1 if nc == 3 else 0
    for f in range(nf):
        planes = [per_comp[c][f][:h, :w] for c in range(nc)]
        frames.append(to_samples(colour_inverse(planes, colour, 8), 8))
    return np.stack(frames)
