"""Integer-network context model (test infrastructure only).

The paper's context model (Section 3.2) runs in floating point, so two
implementations agree on a table index only up to rounding: near a
decision boundary they may differ (the float classes certify such
near-ties). Integer networks (Balle, Johnston and Minnen, "Integer networks
for data compression with latent-variable models", ICLR 2019) remove the
problem by construction: every operation of the network is integer
arithmetic with a fixed rounding rule, so encoder and decoder compute
identical parameters on any hardware. This module states that arithmetic
for the context model (ConvLSTM, the fusion nets of steps 1-4, the
autoregressive LL model, Laplace heads). The layer structure is the float
model's; this is the reading of how each layer is made integer:

* activations are integers with a fixed binary point: z, u, e, a (the
  fusion nets' and the ConvLSTM input's features) carry FA = 4 fractional
  bits and are clamped to [-127, 127] (+-7.94); h = l_i carries FH = 7
  (clamped to [-127, 127]); the cell state c carries 7 and is clamped to
  [-32767, 32767]; symbols enter as clamp(s, -127, 127);
* weights: the float weights of the blob, one scale per tensor: for a
  convolution whose input channels form groups with fractional bits fa_g
  (the ConvLSTM gates read [e (4), h (7)], the steps 2-4 1x1 reads
  [a (4), l (7)], the step 1 input 1x1 reads l (7)), k_g = the largest
  integer with max|w_g| 2^k_g <= WMAX = 56 (a zero group imposes nothing),
  the accumulator exponent S = min_g (k_g + fa_g), w_q = rint(w 2^(S -
  fa_g)) and b_q = rint(b 2^S), S lowered where needed so that
  max|b| 2^S <= 2^18 (bias-dominated layers keep their bias); the accumulator
  acc = b_q + sum w_q a then holds the output times 2^S exactly;
* requantisation to fa_out fractional bits: n = S - fa_out, rq(v) =
  floor((v + 2^(n-1)) / 2^n) for n > 0 (round half up), v 2^-n otherwise,
  then the clamp of the output; LeakyReLU acts on the accumulator:
  v >= 0 ? v : floor(v / 128) (slope 1/128);
* residual adds are integer adds of two FA = 4 values, clamped;
* ConvLSTM: the gate accumulators are requantised to FA, then hard
  sigmoid hs(x) = clamp(2x + 64, 0, 128) and hard tanh ht(x) =
  clamp(8x, -128, 128) (both with 7 fractional bits: 128 = 1.0);
  c = rq7(hs(f) c_prev + hs(i) ht(g)), h = clamp(rq7(hs(o) clamp(c, +-128)),
  +-127), rq7 the requantisation by 7 bits;
* head: t = clamp(rq(acc_mu) to 4 fractional bits, +-2^23) is 16 mu (the
  index decision's t directly); the scale output is read as a log-scale:
  j = clamp(rq(acc_rho) to 3 fractional bits + 24, 0, 127), the Laplace
  table's scale bin (sigma = 0.125 2^(j/8), so rho is log2 sigma);
  ctr, phi and the table follow from (t, j) as for the float classes.

Every intermediate value is an integer of magnitude below 2^24 (at most
2304 products of |w| <= 56 and |a| <= 127, plus |b| <= 2^18), so an
implementation may also evaluate the sums exactly in FP32.

Pins (tests/test_oracle_intnet.py): the requantisation, activations and
weight scaling on hand-worked values; the whole model against a separate
brute-force evaluation with explicit loops over positions, channels and
taps on tiny subbands; closed forms of the cell for saturated gates.
"""
from __future__ import annotations

import numpy as np

from .context import step_map

WMAX = 56
FA = 4
FH = 7
AMAX = 127
BMAX = 1 << 18
CMAX = 32767
J0 = 24


# --------------------------------------------------------------------------
# scalar definitions
def max_shift(m: float, lim: float = WMAX) -> int:
    """Largest integer k with m 2^k <= lim (m > 0), found exactly."""
    k = int(np.floor(np.log2(lim / m)))
    while m * 2.0 ** (k + 1) <= lim:
        k += 1
    while m * 2.0 ** k > lim:
        k -= 1
    return k


def quantise_conv(w: np.ndarray, b: np.ndarray, groups):
    """Integer weights of a convolution. w: [Cout, Cin, ...] float, b [Cout];
    groups: list of (first input channel, count, fa). Returns (w_q int64,
    b_q int64, S)."""
    S = None
    for c0, n, fa in groups:
        m = float(np.max(np.abs(w[:, c0:c0 + n])))
        if m > 0.0:
            k = max_shift(m) + fa
            S = k if S is None else min(S, k)
    if S is None:
        S = 30
    mb = float(np.max(np.abs(b))) if b.size else 0.0
    if mb > 0.0:
        S = min(S, max_shift(mb, BMAX))
    wq = np.zeros(w.shape, dtype=np.int64)
    for c0, n, fa in groups:
        wq[:, c0:c0 + n] = np.rint(w[:, c0:c0 + n] * 2.0 ** (S - fa)).astype(np.int64)
    bq = np.rint(b * 2.0 ** S).astype(np.int64)
    assert np.max(np.abs(wq)) <= WMAX
    return wq, bq, S


def rq(v, n: int):
    """Requantise integers v by n bits (round half up for n > 0)."""
    v = np.asarray(v, dtype=np.int64)
    if n > 0:
        return (v + (np.int64(1) << np.int64(n - 1))) >> np.int64(n)
    return v << np.int64(-n)


def lrelu_i(v):
    v = np.asarray(v, dtype=np.int64)
    return np.where(v >= 0, v, v >> np.int64(7))


def clampa(v, lim=AMAX):
    return np.clip(v, -lim, lim)


def hsig(x):
    return np.clip(2 * np.asarray(x, dtype=np.int64) + 64, 0, 128)


def htanh(x):
    return np.clip(8 * np.asarray(x, dtype=np.int64), -128, 128)


# --------------------------------------------------------------------------
# integer layers (exact int64)
def conv_i(x: np.ndarray, wq: np.ndarray, bq: np.ndarray) -> np.ndarray:
    """acc = b_q + conv(x, w_q), zero padding. x [H, W, Cin] int, w_q
    [Cout, Cin, k, k] (or [Cout, Cin] for 1x1) -> [H, W, Cout] int64.

    The products and sums are integers far below 2^53, so they are formed
    exactly in FP64 (numpy's matrix product) and returned as int64."""
    x = np.asarray(x, dtype=np.float64)
    wf = np.asarray(wq, dtype=np.float64)
    if wq.ndim == 2:
        return np.rint(x @ wf.T + bq).astype(np.int64)
    H, W, _ = x.shape
    k = wq.shape[2]
    r = k // 2
    xp = np.zeros((H + 2 * r, W + 2 * r, x.shape[2]))
    xp[r:r + H, r:r + W] = x
    out = np.zeros((H, W, wq.shape[0])) + bq
    for dy in range(k):
        for dx in range(k):
            out += xp[dy:dy + H, dx:dx + W, :] @ wf[:, :, dy, dx].T
    return np.rint(out).astype(np.int64)


def dw_i(x: np.ndarray, wq: np.ndarray, bq: np.ndarray) -> np.ndarray:
    """Depthwise 3x3 (w_q [C, 3, 3]), zero padding."""
    x = np.asarray(x, dtype=np.int64)
    H, W, C = x.shape
    xp = np.zeros((H + 2, W + 2, C), dtype=np.int64)
    xp[1:H + 1, 1:W + 1] = x
    out = np.zeros((H, W, C), dtype=np.int64) + bq
    for dy in range(3):
        for dx in range(3):
            out += xp[dy:dy + H, dx:dx + W, :] * wq[:, dy, dx]
    return out


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


class IntConv:
    """One quantised convolution: weights, bias, accumulator exponent."""

    def __init__(self, w, b, groups):
        self.wq, self.bq, self.S = quantise_conv(np.asarray(w), np.asarray(b), groups)

    def acc(self, x):
        return conv_i(x, self.wq, self.bq)

    def out(self, x, fa_out=FA, act=False):
        v = self.acc(x)
        if act:
            v = lrelu_i(v)
        return clampa(rq(v, self.S - fa_out))


AR_MASK = np.array([[1, 1, 1, 1, 1], [1, 1, 1, 1, 1], [1, 1, 0, 0, 0],
                    [0, 0, 0, 0, 0], [0, 0, 0, 0, 0]], dtype=np.float64)


class IntContextModel:
    """The integer context model of a float weight set: four-step nets for
    subbands 2..13 and either four-step nets (ll_mode 0) or the
    autoregressive model (ll_mode 1) for LL. The autoregressive model's
    layers in integer form: f1 = rq(lrelu(masked 5x5 conv of clamp(s))),
    f2 = rq(lrelu(1x1 f1)) (4 fractional bits each), head as the steps'."""

    def __init__(self, tensors: dict, C: int, ll_mode: int = 0):
        t = tensors
        self.C = C
        self.ll_mode = ll_mode
        self.we = IntConv(t["lstm.we"], t["lstm.be"], [(0, 1, 0)])
        self.wg = IntConv(t["lstm.wg"], t["lstm.bg"], [(0, C, FA), (C, C, FH)])
        self.nets = {}
        if ll_mode == 1:
            self.ar5 = IntConv(t["ar.w5"] * AR_MASK, t["ar.b5"], [(0, 1, 0)])
            self.ar1 = IntConv(t["ar.w1"], t["ar.b1"], [(0, C, FA)])
            self.arh = IntConv(t["ar.wh"], t["ar.bh"], [(0, C, FA)])
        for ns in (("sb", "ll") if ll_mode == 0 else ("sb",)):
            p = f"{ns}.s0."
            n0 = dict(
                win=IntConv(t[p + "win"], t[p + "bin"], [(0, C, FH)]),
                w1=IntConv(t[p + "w1"], t[p + "b1"], [(0, C, FA)]),
                w2=IntConv(t[p + "w2"], t[p + "b2"], [(0, C, FA)]),
                w3=IntConv(t[p + "w3"], t[p + "b3"], [(0, C, FA)]),
                w4=IntConv(t[p + "w4"], t[p + "b4"], [(0, 2 * C, FA)]),
                wh=IntConv(t[p + "wh"], t[p + "bh"], [(0, C, FA)]))
            wdw = t[p + "wdw"]
            dq, dbq, dS = quantise_conv(wdw[:, None], t[p + "bdw"], [(0, 1, FA)])
            n0["dw"] = (dq[:, 0], dbq, dS)
            nets = [n0]
            for k in (1, 2, 3):
                p = f"{ns}.s{k}."
                nets.append(dict(
                    wa=IntConv(t[p + "wa"], t[p + "ba"], [(0, 1, 0)]),
                    wz=IntConv(t[p + "wz"], t[p + "bz"], [(0, C, FA), (C, C, FH)]),
                    w1=IntConv(t[p + "w1"], t[p + "b1"], [(0, C, FA)]),
                    w2=IntConv(t[p + "w2"], t[p + "b2"], [(0, C, FA)]),
                    wh=IntConv(t[p + "wh"], t[p + "bh"], [(0, C, FA)])))
            self.nets[ns] = nets

    # --- context prediction ------------------------------------------------
    def lstm(self, s_prev: np.ndarray, h, c, up: bool):
        """One integer ConvLSTM step; h (7 fractional bits) and c (7) at the
        current resolution."""
        C = self.C
        x = clampa(np.asarray(s_prev, dtype=np.int64))
        if up:
            x = up2(x)
        H, W = x.shape
        if h is None:
            h = np.zeros((H, W, C), dtype=np.int64)
            c = np.zeros((H, W, C), dtype=np.int64)
        elif up:
            h, c = up2(h), up2(c)
        e = self.we.out(x[:, :, None])
        g = clampa(rq(self.wg.acc(np.concatenate([e, h], axis=2)), self.wg.S - FA))
        gi, gf, go, gg = g[..., 0:C], g[..., C:2 * C], g[..., 2 * C:3 * C], g[..., 3 * C:]
        c = clampa(rq(hsig(gf) * c + hsig(gi) * htanh(gg), FH), CMAX)
        h = clampa(rq(hsig(go) * np.clip(c, -128, 128), FH))
        return h, c

    # --- autoregressive LL ---------------------------------------------------
    def head_tj(self, hd: IntConv, acc):
        t = np.clip(rq(acc[..., 0], hd.S - 4), -(1 << 23), 1 << 23)
        j = np.clip(rq(acc[..., 1], hd.S - 3) + J0, 0, 127)
        return t, j

    def ar_tj_all(self, s: np.ndarray):
        """(t, j) of the autoregressive LL model at every position, all
        symbols known (only causal neighbours enter through the mask)."""
        sc = clampa(np.asarray(s, dtype=np.int64))
        f = self.ar5.out(sc[:, :, None], act=True)
        f = self.ar1.out(f, act=True)
        return self.head_tj(self.arh, self.arh.acc(f))

    def ar_tj_at(self, s: np.ndarray, y: int, x: int):
        """(t, j) at (y, x) from the causal neighbourhood only."""
        H, W = s.shape
        acc = self.ar5.bq.copy()
        for dy in range(3):
            for dx in range(5):
                if dy == 2 and dx >= 2:
                    continue
                yy, xx = y + dy - 2, x + dx - 2
                if 0 <= yy < H and 0 <= xx < W:
                    acc = acc + self.ar5.wq[:, 0, dy, dx] * int(np.clip(s[yy, xx], -AMAX, AMAX))
        f = clampa(rq(lrelu_i(acc), self.ar5.S - FA))
        f = clampa(rq(lrelu_i(self.ar1.wq @ f + self.ar1.bq), self.ar1.S - FA))
        t, j = self.head_tj(self.arh, self.arh.wq @ f + self.arh.bq)
        return int(t), int(j)

    # --- context fusion ------------------------------------------------------
    def step_tj(self, k: int, s: np.ndarray, l: np.ndarray, ns: str):
        """(t, j) of step k over the whole subband: t = 16 mu, j the scale
        bin; only positions of steps < k of s are read."""
        n = self.nets[ns][k]
        if k == 0:
            z = n["win"].out(l)
            u = n["w1"].out(z, act=True)
            dq, dbq, dS = n["dw"]
            u = clampa(rq(dw_i(u, dq, dbq), dS - FA))
            z = clampa(z + n["w2"].out(u))
            u = n["w3"].out(z, act=True)
            z = clampa(z + n["w4"].out(u))
        else:
            H, W = s.shape
            m = step_map(H, W) < k
            sc = np.where(m, clampa(np.asarray(s, dtype=np.int64)), 0)
            a = n["wa"].out(sc[:, :, None])
            z = n["wz"].out(np.concatenate([a, l], axis=2))
            u = n["w1"].out(z, act=True)
            z = clampa(z + n["w2"].out(u))
        return self.head_tj(n["wh"], n["wh"].acc(z))


def index_of(t, j):
    """(ctr, phi, j) of the Laplace table bank from (t, j)."""
    t = np.asarray(t, dtype=np.int64)
    ctr = (t + 8) >> 4
    return ctr, t - 16 * ctr, np.asarray(j, dtype=np.int64)


def context_tj_all(model: IntContextModel, qsb: list):
    """(t, j) at every position of every subband, all symbols known (the
    encoder's view; equal to what the decoder computes step by step)."""
    out = []
    h = c = None
    C = model.C
    for i, s in enumerate(qsb):
        H, W = s.shape
        if i == 0 and model.ll_mode == 1:
            out.append(model.ar_tj_all(s))
            continue
        if i == 0:
            l, ns = np.zeros((H, W, C), dtype=np.int64), "ll"
        else:
            up = qsb[i - 1].shape[0] < H
            h, c = model.lstm(qsb[i - 1], h, c, up)
            l, ns = h, "sb"
        sm = step_map(H, W)
        t = np.zeros((H, W), dtype=np.int64)
        j = np.zeros((H, W), dtype=np.int64)
        for k in range(4):
            tk, jk = model.step_tj(k, s, l, ns)
            t = np.where(sm == k, tk, t)
            j = np.where(sm == k, jk, j)
        out.append((t, j))
    return out
