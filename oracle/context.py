"""Parallel context model of pWave++, FP64 (test infrastructure only).

Section 3.2 and Figs. 3-5 of the paper. Subbands are coded in a fixed order
(Fig. 1). For subband i >= 2 a context prediction module, a convolutional
LSTM whose input is the previously coded subband, produces a hidden state
that serves as the long-term context l_i. A context fusion model then codes
the subband in four steps: each step covers one quarter of the positions,
taken from a "wide checkerboard" pattern, and estimates Laplace means and
scales from l_i plus the positions of earlier steps. Step 1 uses a
DepthConvBlock (a two-part residual block whose first part holds a depthwise
convolution); steps 2-4 use a two-layer residual block. The LL subband is
coded either by an autoregressive model (the pWave++ default) or by the same
four-step scheme without long-term context (the "4-step LL" variant of
Table 1).

The paper's figures that hold the layer specifications are not available,
so the layer structure below is a reading of the text:
* step pattern (period 2 rows x 4 columns): step 1 = {even row, x = 0 mod 4}
  and {odd row, x = 2 mod 4}; step 2 = step 1 shifted by two columns; step 3
  = {even row, x = 1 mod 4} and {odd row, x = 3 mod 4}; step 4 = the rest.
  This gives 0, 2, 6 and 8 coded neighbours in a 3x3 window, as the text
  states;
* ConvLSTM (Shi et al. 2015): e = conv3x3(1->C)(up(s_{i-1})),
  [i f o g] = conv3x3(2C->4C)([e, up(h)]), c = sig(f) c + sig(i) tanh(g),
  h = sig(o) tanh(c), l_i = h; h = c = 0 before subband 2; up() is nearest
  2x upsampling when the previous subband has half the resolution;
* step 1: z = 1x1(l); DepthConvBlock part 1: z += 1x1(dw3x3(lrelu(1x1(z))));
  part 2: z += 1x1(2C->C)(lrelu(1x1(C->2C)(z))); head 1x1(C->2);
* steps 2-4: a = conv3x3(1->C)(m_<k * s_i); z = 1x1(2C->C)([a, l_i]);
  z += conv3x3(lrelu(conv3x3(z))); head 1x1(C->2);
* head outputs (mu, rho) with scale sigma = softplus(rho); LeakyReLU slope
  0.01; zero padding for every convolution;
* autoregressive LL: masked 5x5 conv (taps strictly before the centre in
  raster order) 1->C, lrelu, 1x1 C->C, lrelu, 1x1 C->2.

Pins: the step partition (tiling, densities, 0/2/6/8 neighbour counts) and
causality by brute force, and the LSTM cell against its defining equations
(tests/test_oracle_context.py); the layer composition of both fusion nets
against closed forms for special weights - each skip connection, the [a, l]
order of the steps 2-4 fusion, the LeakyReLU slope, the orientation of the
spatial taps, the head and softplus - and the autoregressive LL model against
a single-tap closed form (tests/test_oracle_layer_pins.py). What stays
parity unpinned is the architecture itself (layer counts, widths, which
activation): the paper's figures that specify it are not available, so the
reading above is the specification.
"""
from __future__ import annotations

import numpy as np

from .lifting import conv2d

LRELU = 0.01


def lrelu(x):
    return np.where(x >= 0, x, LRELU * x)


def sigmoid(x):
    """Logistic function, written as (1 + tanh(x / 2)) / 2 (no overflow)."""
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def softplus(x):
    return np.where(x > 20.0, x, np.log1p(np.exp(np.minimum(x, 20.0))))


def step_map(h: int, w: int) -> np.ndarray:
    """Coding step (0..3) of every position of an h x w subband."""
    y = np.arange(h)[:, None] & 1
    x = np.arange(w)[None, :] & 3
    even = np.array([0, 2, 1, 3])   # x mod 4 -> step, even rows
    odd = np.array([1, 3, 0, 2])    # x mod 4 -> step, odd rows
    return np.where(y == 0, even[x], odd[x])


def step_positions(h: int, w: int, k: int):
    """(ys, xs) of the step-k positions in raster order."""
    ys, xs = np.nonzero(step_map(h, w) == k)
    return ys, xs


def conv1x1(x, w, b):
    return x @ w.T + b


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


class ContextModel:
    """Weights and forward passes of the context model."""

    def __init__(self, tensors: dict, C: int, ll_mode: int):
        self.t = tensors
        self.C = C
        self.ll_mode = ll_mode

    # --- context prediction (ConvLSTM) -----------------------------------
    def lstm(self, s_prev: np.ndarray, h, c, up: bool):
        """One ConvLSTM step; returns (h, c) at the current resolution."""
        t = self.t
        C = self.C
        x = upsample2(s_prev) if up else s_prev
        if h is None:
            H, W = x.shape
            h = np.zeros((H, W, C))
            c = np.zeros((H, W, C))
        elif up:
            h = upsample2(h)
            c = upsample2(c)
        e = conv2d(x[:, :, None], t["lstm.we"], t["lstm.be"])
        g = conv2d(np.concatenate([e, h], axis=2), t["lstm.wg"], t["lstm.bg"])
        gi, gf, go, gg = (g[:, :, 0:C], g[:, :, C:2 * C], g[:, :, 2 * C:3 * C],
                          g[:, :, 3 * C:4 * C])
        c = sigmoid(gf) * c + sigmoid(gi) * np.tanh(gg)
        h = sigmoid(go) * np.tanh(c)
        return h, c

    # --- context fusion ----------------------------------------------------
    def step_head(self, k: int, s: np.ndarray, l: np.ndarray, ns: str):
        """Raw head outputs of step k over the whole subband, [H, W, nh]
        (nh = 2: Laplace mean and scale pre-activation; 9: the logistic
        mixture's 3 weight logits, 3 means, 3 scale pre-activations)."""
        t = self.t
        p = f"{ns}.s{k}."
        if k == 0:
            z = conv1x1(l, t[p + "win"], t[p + "bin"])
            u = lrelu(conv1x1(z, t[p + "w1"], t[p + "b1"]))
            u = depthwise3x3(u, t[p + "wdw"], t[p + "bdw"])
            z = z + conv1x1(u, t[p + "w2"], t[p + "b2"])
            u = lrelu(conv1x1(z, t[p + "w3"], t[p + "b3"]))
            z = z + conv1x1(u, t[p + "w4"], t[p + "b4"])
        else:
            H, W = s.shape
            m = (step_map(H, W) < k).astype(np.float64)
            a = conv2d((m * s)[:, :, None], t[p + "wa"], t[p + "ba"])
            z = conv1x1(np.concatenate([a, l], axis=2), t[p + "wz"], t[p + "bz"])
            u = lrelu(conv2d(z, t[p + "w1"], t[p + "b1"]))
            z = z + conv2d(u, t[p + "w2"], t[p + "b2"])
        return conv1x1(z, t[p + "wh"], t[p + "bh"])

    def step_params(self, k: int, s: np.ndarray, l: np.ndarray, ns: str):
        """Entropy parameters (mu, sigma) of step k over the whole subband.

        s is the current subband (only positions of steps < k are read: the
        rest is masked to zero here); l the long-term context [H, W, C];
        ns selects the net set ("sb" for subbands 2..13, "ll" for the
        four-step LL model). Returns two [H, W] arrays.
        """
        out = self.step_head(k, s, l, ns)
        return out[:, :, 0], softplus(out[:, :, 1])

    # --- autoregressive LL ---------------------------------------------------
    def ar_mask(self):
        m = np.zeros((5, 5))
        m[:2, :] = 1.0
        m[2, :2] = 1.0
        return m

    def ar_params_all(self, s: np.ndarray):
        """AR LL parameters at every position, given all symbols (encoder)."""
        t = self.t
        w5 = t["ar.w5"] * self.ar_mask()[None, None]
        f = lrelu(conv2d(s[:, :, None], w5, t["ar.b5"]))
        f = lrelu(conv1x1(f, t["ar.w1"], t["ar.b1"]))
        out = conv1x1(f, t["ar.wh"], t["ar.bh"])
        return out[:, :, 0], softplus(out[:, :, 1])

    def ar_params_at(self, s: np.ndarray, y: int, x: int):
        """AR LL parameters at (y, x) from the causal neighbourhood only."""
        t = self.t
        H, W = s.shape
        f = t["ar.b5"].copy()
        for dy in range(5):
            for dx in range(5):
                if dy > 2 or (dy == 2 and dx >= 2):
                    continue
                yy, xx = y + dy - 2, x + dx - 2
                if 0 <= yy < H and 0 <= xx < W:
                    f = f + t["ar.w5"][:, 0, dy, dx] * s[yy, xx]
        f = lrelu(f)
        f = lrelu(t["ar.w1"] @ f + t["ar.b1"])
        out = t["ar.wh"] @ f + t["ar.bh"]
        return out[0], float(softplus(np.array(out[1])))


def depthwise3x3(x, w, b):
    """Depthwise 3x3 conv (one filter per channel), zero padding."""
    H, W, C = x.shape
    xp = np.zeros((H + 2, W + 2, C))
    xp[1:H + 1, 1:W + 1] = x
    out = np.empty((H, W, C))
    out[...] = b
    for dy in range(3):
        for dx in range(3):
            out += xp[dy:dy + H, dx:dx + W, :] * w[:, dy, dx]
    return out
