"""CNN lifting wavelet transform, FP64 (test infrastructure only).

Follows Section 3.1 and Fig. 2 of the paper: a 1-D lifting step splits a
signal into even and odd samples, predicts the odd samples from the even ones
(HP = odd - P(even)) and updates the even samples from the highpass
(LP = even + U(HP)); the inverse runs the same two steps backwards, so it
reconstructs perfectly for any P and U. A 2-D level applies the 1-D step
along rows first, then along columns. P and U are "residual CNN modules": a
fixed linear lifting filter plus a trainable CNN residual. With integer
rounding of the P and U outputs the transform maps integers to integers and
is losslessly invertible (the Fig. 2 caption).

Readings (the paper defers the filter details to its references):
* linear parts are the LeGall 5/3 filters: P_lin(e)[n] = (e[n] + e[n+1]) / 2
  and U_lin(h)[n] = (h[n-1] + h[n]) / 4, with whole-sample symmetric
  extension at both ends (e[N] = e[N-1], h[-1] = h[0]);
* the CNN residual is conv3x3(1->F), tanh, conv3x3(F->F), tanh,
  conv3x3(F->1), zero padding, applied to the 2-D array of even samples (for
  P) or of highpass samples (for U); one net per direction and operator,
  shared by all levels;
* integer mode takes floor(P) and floor(U + 1/2), decided in FP32, so
  that with the CNN residuals at zero it is exactly the reversible 5/3
  lifting of JPEG 2000;
* integer mode evaluates the CNN residual as a fixed sequence of FP32
  operations (lift_cnn_fp32, tanh32), because an integer lifting step
  reconstructs exactly only where encoder and decoder round the same value:
  the Fig. 2 caption's guarantee of perfect reconstruction then holds
  between any two implementations, not just within one. Each layer starts
  from its bias and adds, tap by tap in raster order and within a tap input
  channel by input channel, the product w * x, product and sum each rounded
  to FP32 (no fused multiply-add); v = P_lin + CNN is one FP32 addition.

Pins: perfect reconstruction for random weights, the exact integer round
trip, tanh32 within a few FP32 ulps of FP64 tanh and lift_cnn_fp32 within
FP32 rounding of the FP64 CNN, the LeGall 5/3 integer lifting of JPEG 2000 (CNN residual zero) checked
against a direct textbook formula, and the 2-D Haar basis functions for the
Haar special case (tests/test_oracle_lifting.py).

The temporal transform (Section 3.3) is the same lifting idea along the
frame axis: H = f_odd - P_t(MC(f_even)) and L = f_even + U_t(IMC(H)) with
P_t(v) = v + CNN(v) and U_t(v) = v / 2 + CNN(v) (Haar linear parts). The
predict step compensates motion: MC warps the even frame towards the odd
one with block motion vectors; the update step re-uses the same vectors to
map the highpass band back onto the even frame (inverse motion
compensation), so it filters along the motion trajectory. The paper defers
the motion model to its reference; the reading here:
* integer-pel block motion, 16 x 16 blocks on the padded frame grid, one
  vector (dy, dx) per block of the odd frame, |dy|, |dx| <= 16;
* MC(f)[y, x] = f[y + dy, x + dx] and IMC(h)[y, x] = h[y - dy, x - dx],
  (dy, dx) the vector of the block that contains (y, x), coordinates
  clamped to the frame; zero vectors give the identity transform;
* the vectors of temporal level l, pair m come from a full search between
  the original frames that the pair's two lowpass frames stand for (frames
  2^l m and 2^l m + 2^(l-1)) on an integer luma (the RCT luma
  floor((R + 2G + B) / 4) of the 8-bit samples, or the gray sample):
  minimum sum of absolute differences, ties to the smaller |dy| + |dx|,
  then the smaller dy, then the smaller dx.
The lifting structure makes the transform invertible for any vectors.
"""
from __future__ import annotations

import numpy as np

from .entropy import exp32

f32 = np.float32

def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Cross-correlation with zero padding ('same' size).

    x: [H, W, Cin], w: [Cout, Cin, kh, kw], b: [Cout] -> [H, W, Cout];
    out[y, x, o] = b[o] + sum_{i,dy,dx} w[o, i, dy, dx] x[y+dy-kh//2, x+dx-kw//2, i].
    """
    H, W, Cin = x.shape
    Cout, Cin2, kh, kw = w.shape
    assert Cin == Cin2
    ph, pw = kh // 2, kw // 2
    xp = np.zeros((H + 2 * ph, W + 2 * pw, Cin))
    xp[ph:ph + H, pw:pw + W, :] = x
    out = np.empty((H, W, Cout))
    out[...] = b
    for dy in range(kh):
        for dx in range(kw):
            out += xp[dy:dy + H, dx:dx + W, :] @ w[:, :, dy, dx].T
    return out


def lift_cnn(v: np.ndarray, net: dict) -> np.ndarray:
    """CNN residual of a predict/update filter on a 2-D array v -> same shape."""
    t = np.tanh(conv2d(v[:, :, None], net["w1"], net["b1"]))
    t = np.tanh(conv2d(t, net["w2"], net["b2"]))
    return conv2d(t, net["w3"], net["b3"])[:, :, 0]


# float32 nearest 1/n!, n = 3..11 (each written as its bit pattern's value)
_INV_FACT32 = {n: f32(float.fromhex(h)) for n, h in
               ((3, "0x1.555556p-3"), (4, "0x1.555556p-5"), (5, "0x1.111112p-7"),
                (6, "0x1.6c16c2p-10"), (7, "0x1.a01a02p-13"), (8, "0x1.a01a02p-16"),
                (9, "0x1.71de3ap-19"), (10, "0x1.27e4fcp-22"), (11, "0x1.ae6456p-26"))}


def tanh32(x: np.ndarray) -> np.ndarray:
    """tanh as a fixed sequence of correctly rounded FP32 operations.

    With a = |x| and z = -2a (exact), m = e^z - 1 is the degree-11 Taylor
    polynomial z + z^2/2! + ... + z^11/11! in Horner order (coefficients the
    float32 nearest 1/n!) when z >= -1, else exp32(z) - 1 (e^z <= 1/e there,
    so the subtraction does not cancel); then tanh(a) = -m / (2 + m), given
    the sign of x.
    """
    x = np.asarray(x, dtype=f32)
    a = np.abs(x)
    z = (f32(-2.0) * a).astype(f32)
    p = np.full_like(z, _INV_FACT32[11])
    for n in (10, 9, 8, 7, 6, 5, 4, 3):
        p = (p * z).astype(f32)
        p = (p + _INV_FACT32[n]).astype(f32)
    p = (p * z).astype(f32)
    p = (p + f32(0.5)).astype(f32)
    p = (p * z).astype(f32)
    p = (p + f32(1.0)).astype(f32)
    m_series = (p * z).astype(f32)
    m_exp = (exp32(np.minimum(z, f32(0.0))) - f32(1.0)).astype(f32)
    m = np.where(z >= f32(-1.0), m_series, m_exp).astype(f32)
    t = ((-m).astype(f32) / (f32(2.0) + m).astype(f32)).astype(f32)
    return np.copysign(t, x).astype(f32)


def conv3x3_fp32(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3 cross-correlation (as conv2d) in FP32 with a fixed
    order of separately rounded operations: acc = b, then for each tap (dy,
    dx) in raster order and each input channel i in ascending order
    acc = acc + w[o, i, dy, dx] * x[y + dy - 1, x + dx - 1, i]."""
    H, W, Cin = x.shape
    Cout = w.shape[0]
    w32 = np.asarray(w, dtype=f32)
    xp = np.zeros((H + 2, W + 2, Cin), dtype=f32)
    xp[1:H + 1, 1:W + 1, :] = x
    acc = np.empty((H, W, Cout), dtype=f32)
    acc[...] = np.asarray(b, dtype=f32)
    for dy in range(3):
        for dx in range(3):
            for i in range(Cin):
                prod = (xp[dy:dy + H, dx:dx + W, i:i + 1] * w32[:, i, dy, dx]).astype(f32)
                acc = (acc + prod).astype(f32)
    return acc


def lift_cnn_fp32(v: np.ndarray, net: dict) -> np.ndarray:
    """The CNN residual of lift_cnn evaluated as the integer-mode FP32
    operation sequence (float32 result)."""
    t = tanh32(conv3x3_fp32(np.asarray(v, dtype=f32)[:, :, None], net["w1"], net["b1"]))
    t = tanh32(conv3x3_fp32(t, net["w2"], net["b2"]))
    return conv3x3_fp32(t, net["w3"], net["b3"])[:, :, 0]


def net_of(tensors: dict, prefix: str) -> dict:
    return {k: tensors[prefix + k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")}


def _shift(a: np.ndarray, axis: int, delta: int) -> np.ndarray:
    """a[n + delta] along `axis`, clamped to the valid index range."""
    n = a.shape[axis]
    idx = np.clip(np.arange(n) + delta, 0, n - 1)
    return np.take(a, idx, axis=axis)


def round_int(v: np.ndarray, half: float) -> np.ndarray:
    """floor(v + half) with the decision taken in FP32 (the kernels'
    precision; the paper fixes none), returned as FP64 integers."""
    f32 = np.float32
    return np.floor((v.astype(f32) + f32(half)).astype(f32)).astype(np.float64)


def predict(e: np.ndarray, axis: int, net: dict | None, lossless: bool,
            linear: str = "53") -> np.ndarray:
    """P(e) = (e[n] + e[n+1]) / 2 + CNN_P(e); floor(P) in integer mode.

    linear="haar" replaces the linear part by P_lin(e)[n] = e[n].
    """
    v = e.copy() if linear == "haar" else 0.5 * (e + _shift(e, axis, +1))
    if net is not None and lossless:
        v = (v.astype(f32) + lift_cnn_fp32(e, net)).astype(f32).astype(np.float64)
    elif net is not None:
        v = v + lift_cnn(e, net)
    return round_int(v, 0.0) if lossless else v


def update(h: np.ndarray, axis: int, net: dict | None, lossless: bool,
           linear: str = "53") -> np.ndarray:
    """U(h) = (h[n-1] + h[n]) / 4 + CNN_U(h); floor(U + 1/2) in integer mode.

    linear="haar" replaces the linear part by U_lin(h)[n] = h[n] / 2.
    """
    v = 0.5 * h if linear == "haar" else 0.25 * (_shift(h, axis, -1) + h)
    if net is not None and lossless:
        v = (v.astype(f32) + lift_cnn_fp32(h, net)).astype(f32).astype(np.float64)
    elif net is not None:
        v = v + lift_cnn(h, net)
    return round_int(v, 0.5) if lossless else v


def lift_fwd(x: np.ndarray, axis: int, netP, netU, lossless: bool,
             linear: str = "53"):
    """One 1-D forward lifting step along `axis`: returns (LP, HP)."""
    n = x.shape[axis]
    assert n % 2 == 0
    e = np.take(x, np.arange(0, n, 2), axis=axis)
    o = np.take(x, np.arange(1, n, 2), axis=axis)
    hp = o - predict(e, axis, netP, lossless, linear)
    lp = e + update(hp, axis, netU, lossless, linear)
    return lp, hp


def lift_inv(lp: np.ndarray, hp: np.ndarray, axis: int, netP, netU,
             lossless: bool, linear: str = "53"):
    """Inverse of lift_fwd: undo the update, undo the predict, merge."""
    e = lp - update(hp, axis, netU, lossless, linear)
    o = hp + predict(e, axis, netP, lossless, linear)
    shape = list(e.shape)
    shape[axis] *= 2
    x = np.empty(shape)
    sl_e = [slice(None)] * x.ndim
    sl_o = [slice(None)] * x.ndim
    sl_e[axis] = slice(0, None, 2)
    sl_o[axis] = slice(1, None, 2)
    x[tuple(sl_e)] = e
    x[tuple(sl_o)] = o
    return x


class Lifting:
    """The four predict/update nets of the 2-D lifting transform."""

    def __init__(self, tensors: dict | None, linear: str = "53"):
        self.linear = linear
        if tensors is None:
            self.rP = self.rU = self.cP = self.cU = None
        else:
            self.rP = net_of(tensors, "lift.row.P.")
            self.rU = net_of(tensors, "lift.row.U.")
            self.cP = net_of(tensors, "lift.col.P.")
            self.cU = net_of(tensors, "lift.col.U.")

    def fwd_level(self, x: np.ndarray, lossless: bool):
        """One 2-D level: rows first, then columns -> (LL, HL, LH, HH).

        HL is the row-highpass / column-lowpass band, LH the row-lowpass /
        column-highpass band.
        """
        a = self.linear
        lo, hi = lift_fwd(x, 1, self.rP, self.rU, lossless, a)
        LL, LH = lift_fwd(lo, 0, self.cP, self.cU, lossless, a)
        HL, HH = lift_fwd(hi, 0, self.cP, self.cU, lossless, a)
        return LL, HL, LH, HH

    def inv_level(self, LL, HL, LH, HH, lossless: bool) -> np.ndarray:
        """Inverse of fwd_level: columns first, then rows."""
        a = self.linear
        lo = lift_inv(LL, LH, 0, self.cP, self.cU, lossless, a)
        hi = lift_inv(HL, HH, 0, self.cP, self.cU, lossless, a)
        return lift_inv(lo, hi, 1, self.rP, self.rU, lossless, a)

    def forward(self, x: np.ndarray, levels: int, lossless: bool):
        """Multi-level DWT; returns subbands in coding order.

        Order (Fig. 1 red arrows): LL_L, HL_L, LH_L, HH_L, HL_{L-1}, ...,
        HH_1, i.e. 3 * levels + 1 subbands.
        """
        details = []
        cur = x
        for _ in range(levels):
            cur, HL, LH, HH = self.fwd_level(cur, lossless)
            details.append((HL, LH, HH))
        out = [cur]
        for HL, LH, HH in reversed(details):
            out += [HL, LH, HH]
        return out

    def inverse(self, sb: list, levels: int, lossless: bool) -> np.ndarray:
        """Inverse of forward (subbands in coding order)."""
        cur = sb[0]
        for lv in range(levels):
            HL, LH, HH = sb[1 + 3 * lv: 4 + 3 * lv]
            cur = self.inv_level(cur, HL, LH, HH, lossless)
        return cur


def subband_shapes(h: int, w: int, levels: int):
    """(height, width, level) of each subband in coding order."""
    out = [(h >> levels, w >> levels, levels)]
    for lv in range(levels, 0, -1):
        out += [(h >> lv, w >> lv, lv)] * 3
    return out


def _tnet(tensors, op):
    return net_of(tensors, f"tlift.{op}.")


MC_BLOCK = 16
MC_RANGE = 16


def mc_warp(f: np.ndarray, mv: np.ndarray, sign: int, B: int = MC_BLOCK) -> np.ndarray:
    """out[y, x] = f[y + sign dy, x + sign dx], (dy, dx) = mv[y // B, x // B],
    coordinates clamped to the frame (sign +1: MC, -1: inverse MC)."""
    H, W = f.shape
    yy = np.arange(H)[:, None]
    xx = np.arange(W)[None, :]
    dy = mv[yy // B, xx // B, 0]
    dx = mv[yy // B, xx // B, 1]
    return f[np.clip(yy + sign * dy, 0, H - 1), np.clip(xx + sign * dx, 0, W - 1)]


def motion_search(cur: np.ndarray, ref: np.ndarray, B: int = MC_BLOCK,
                  R: int = MC_RANGE) -> np.ndarray:
    """Block motion vectors [ceil(H/B), ceil(W/B), 2] (int) of integer frame
    `cur` against `ref`: per block the (dy, dx) in [-R, R]^2 minimising
    sum |cur[y, x] - ref[clamp(y + dy), clamp(x + dx)]| over the block's
    pixels; ties to the smaller |dy| + |dx|, then dy, then dx."""
    H, W = cur.shape
    nby, nbx = -(-H // B), -(-W // B)
    cur = cur.astype(np.int64)
    ref = ref.astype(np.int64)
    yy = np.arange(H)[:, None]
    xx = np.arange(W)[None, :]
    best = np.full((nby, nbx, 4), np.iinfo(np.int64).max, dtype=np.int64)
    out = np.zeros((nby, nbx, 2), dtype=np.int64)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            d = np.zeros((nby * B, nbx * B), dtype=np.int64)
            d[:H, :W] = np.abs(cur - ref[np.clip(yy + dy, 0, H - 1), np.clip(xx + dx, 0, W - 1)])
            sad = d.reshape(nby, B, nbx, B).sum(axis=(1, 3))
            key = np.stack([sad, np.full_like(sad, abs(dy) + abs(dx)),
                            np.full_like(sad, dy), np.full_like(sad, dx)], axis=2)
            better = np.zeros((nby, nbx), dtype=bool)
            undecided = np.ones((nby, nbx), dtype=bool)
            for k in range(4):
                lt = key[:, :, k] < best[:, :, k]
                gt = key[:, :, k] > best[:, :, k]
                better |= undecided & lt
                undecided &= ~(lt | gt)
            best[better] = key[better]
            out[better] = (dy, dx)
    return out


def gop_luma(img: np.ndarray) -> np.ndarray:
    """Integer luma of an 8-bit frame for motion search: the gray sample, or
    floor((R + 2G + B) / 4)."""
    x = img.astype(np.int64)
    if x.ndim == 2:
        return x
    return (x[:, :, 0] + 2 * x[:, :, 1] + x[:, :, 2]) >> 2


def gop_motion(luma: list, tlevels: int) -> list:
    """Vectors of every temporal level and pair, in stream order: for level
    l = 1..T and pair m, motion_search(luma[2^l m + 2^(l-1)], luma[2^l m])."""
    n = len(luma)
    out = []
    for lv in range(1, tlevels + 1):
        for m in range(n >> lv):
            a = (1 << lv) * m
            out.append(motion_search(luma[a + (1 << (lv - 1))], luma[a]))
    return out


def temporal_forward(frames: list, tensors: dict, tlevels: int, mvs: list | None = None):
    """Temporal lifting over a GOP of 2^tlevels frames.

    mvs: the block vectors of every level and pair in the order of
    gop_motion (None: zero motion). Returns the temporal subbands in order
    [L_T, H_T, H_{T-1}..., H_1], the H bands of each level in frame order.
    """
    nP, nU = _tnet(tensors, "P"), _tnet(tensors, "U")
    cur = list(frames)
    highs = []
    k = 0
    for _ in range(tlevels):
        lows, hs = [], []
        for m in range(len(cur) // 2):
            fe, fo = cur[2 * m], cur[2 * m + 1]
            mv = mvs[k] if mvs is not None else None
            k += 1
            w = fe if mv is None else mc_warp(fe, mv, +1)
            h = fo - (w + lift_cnn(w, nP))
            v = h if mv is None else mc_warp(h, mv, -1)
            l = fe + (0.5 * v + lift_cnn(v, nU))
            lows.append(l)
            hs.append(h)
        highs.append(hs)
        cur = lows
    out = list(cur)
    for hs in reversed(highs):
        out += hs
    return out


def temporal_inverse(bands: list, tensors: dict, tlevels: int, mvs: list | None = None):
    """Inverse of temporal_forward (same vectors)."""
    nP, nU = _tnet(tensors, "P"), _tnet(tensors, "U")
    nf = 1 << tlevels
    starts = [0]
    for lv in range(1, tlevels + 1):
        starts.append(starts[-1] + (nf >> lv))      # first field of level lv + 1
    cur = [bands[0]]
    pos = 1
    for lv in range(tlevels, 0, -1):
        hs = bands[pos:pos + len(cur)]
        pos += len(cur)
        nxt = []
        for m, (l, h) in enumerate(zip(cur, hs)):
            mv = mvs[starts[lv - 1] + m] if mvs is not None else None
            v = h if mv is None else mc_warp(h, mv, -1)
            fe = l - (0.5 * v + lift_cnn(v, nU))
            w = fe if mv is None else mc_warp(fe, mv, +1)
            fo = h + (w + lift_cnn(w, nP))
            nxt += [fe, fo]
        cur = nxt
    return cur
