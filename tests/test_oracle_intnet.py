"""Pins of the oracle's integer-network context model (oracle/intnet.py).

The scalar definitions (requantisation, LeakyReLU, hard sigmoid / tanh,
weight scaling) are checked on hand-worked values at their rounding and
clamping boundaries; the vectorised model is checked against a separate
brute-force evaluation with explicit loops over positions, channels and
taps on tiny subbands (a transposed weight, a mirrored tap, a wrong group
scale or a misplaced clamp fails it); and the codec round-trips streams of
the integer model, which say so in the header.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle import intnet as I
from oracle.context import step_map


def test_requantisation_rounds_half_up_and_shifts_left():
    assert list(I.rq([5, -5, 7, -7, 6, -6], 1)) == [3, -2, 4, -3, 3, -3]
    assert list(I.rq([7, -7, 6, -6, 2, -2], 2)) == [2, -2, 2, -1, 1, 0]
    assert list(I.rq([3, -3], 0)) == [3, -3]
    assert list(I.rq([3, -3], -2)) == [12, -12]


def test_activations():
    assert list(I.lrelu_i([100, 0, -1, -100, -128, -129, -256])) == [100, 0, -1, -1, -1, -2, -2]
    assert list(I.hsig([0, 32, -32, 40, -40, 1])) == [64, 128, 0, 128, 0, 66]
    assert list(I.htanh([16, -16, 100, -3, 0])) == [128, -128, 128, -24, 0]
    assert list(I.clampa([200, -200, 5])) == [127, -127, 5]


def test_weight_scaling():
    assert I.max_shift(0.3) == 7            # 0.3 * 128 = 38.4 <= 56 < 76.8
    assert I.max_shift(7.0) == 3            # 7 * 8 = 56 exactly
    assert I.max_shift(56.0) == 0 and I.max_shift(56.0001) == -1
    assert I.max_shift(100.0, I.BMAX) == 11  # 100 * 2048 <= 2^18 < 100 * 4096
    w = np.array([[0.3, -0.1], [0.25, 0.05]])
    b = np.array([0.5, -0.25])
    wq, bq, S = I.quantise_conv(w, b, [(0, 1, 4), (1, 1, 7)])
    # group 0: k = 7, + 4 = 11; group 1: max 0.1, k = 9, + 7 = 16; S = 11
    assert S == 11
    assert wq.tolist() == [[38, -2], [32, 1]]   # rint(w * 2^7), rint(w * 2^(11 - 7))
    assert bq.tolist() == [1024, -512]
    # a large bias lowers the scale so that it fits in 2^18
    _, bq2, S2 = I.quantise_conv(w, np.array([1000.0, 0.0]), [(0, 2, 4)])
    assert S2 == 8 and bq2.tolist() == [256000, 0]


def test_cell_saturated_gates_closed_form():
    # hs(f) = hs(i) = 128 (1.0), ht(g) = +-128: c = c_prev +- 1.0, and
    # h = hs(o) clamp(c) / 128
    c_prev = np.array([-300, -5, 0, 77, 3000])
    for g in (128, -128):
        c = I.clampa(I.rq(128 * c_prev + 128 * g, I.FH), I.CMAX)
        assert list(c) == list(c_prev + g)
    c = np.array([-200, -128, -64, 0, 64, 127, 500])
    h = I.clampa(I.rq(64 * np.clip(c, -128, 128), I.FH))   # hs(o) = 64 (one half)
    assert list(h) == [-64, -64, -32, 0, 32, 64, 64]


# --------------------------------------------------------------------------
# brute force: explicit loops, Python integers
def _rq(v, n):
    return (v + (1 << (n - 1))) >> n if n > 0 else v << (-n)


def _cl(v, lim=127):
    return max(-lim, min(lim, v))


def _conv_px(x, wq, bq, y, xx, co):
    """One output of a KxK (or 1x1) conv with zero padding; x [H][W][Cin]."""
    H, W, Cin = x.shape
    acc = int(bq[co])
    if wq.ndim == 2:
        for ci in range(Cin):
            acc += int(wq[co, ci]) * int(x[y, xx, ci])
        return acc
    k = wq.shape[2]
    r = k // 2
    for ci in range(Cin):
        for dy in range(k):
            for dx in range(k):
                yy, xs = y + dy - r, xx + dx - r
                if 0 <= yy < H and 0 <= xs < W:
                    acc += int(wq[co, ci, dy, dx]) * int(x[yy, xs, ci])
    return acc


def _layer(x, cv, fa_out=I.FA, act=False, cout=None):
    H, W, _ = x.shape
    cout = cv.wq.shape[0] if cout is None else cout
    out = np.zeros((H, W, cout), dtype=np.int64)
    for y in range(H):
        for xx in range(W):
            for co in range(cout):
                v = _conv_px(x, cv.wq, cv.bq, y, xx, co)
                if act and v < 0:
                    v = v >> 7
                out[y, xx, co] = _cl(_rq(v, cv.S - fa_out))
    return out


def _brute_lstm(m, s_prev, h, c, up):
    C = m.C
    x = np.clip(np.asarray(s_prev, dtype=np.int64), -127, 127)
    if up:
        x = np.repeat(np.repeat(x, 2, 0), 2, 1)
    H, W = x.shape
    if h is None:
        h = np.zeros((H, W, C), dtype=np.int64)
        c = np.zeros((H, W, C), dtype=np.int64)
    elif up:
        h = np.repeat(np.repeat(h, 2, 0), 2, 1)
        c = np.repeat(np.repeat(c, 2, 0), 2, 1)
    e = _layer(x[:, :, None], m.we)
    xin = np.concatenate([e, h], axis=2)
    hn = np.zeros_like(h)
    cn = np.zeros_like(c)
    for y in range(H):
        for xx in range(W):
            for ch in range(C):
                g = [_cl(_rq(_conv_px(xin, m.wg.wq, m.wg.bq, y, xx, q * C + ch), m.wg.S - I.FA))
                     for q in range(4)]
                hs = [max(0, min(128, 2 * v + 64)) for v in g]
                tg = max(-128, min(128, 8 * g[3]))
                cv = _cl(_rq(hs[1] * int(c[y, xx, ch]) + hs[0] * tg, 7), 32767)
                cn[y, xx, ch] = cv
                hn[y, xx, ch] = _cl(_rq(hs[2] * max(-128, min(128, cv)), 7))
    return hn, cn


def _brute_step(m, k, s, l, ns):
    n = m.nets[ns][k]
    H, W = s.shape
    if k == 0:
        z = _layer(l, n["win"])
        u = _layer(z, n["w1"], act=True)
        dq, dbq, dS = n["dw"]
        v = np.zeros_like(u)
        for y in range(H):
            for xx in range(W):
                for ch in range(m.C):
                    acc = int(dbq[ch])
                    for dy in range(3):
                        for dx in range(3):
                            yy, xs = y + dy - 1, xx + dx - 1
                            if 0 <= yy < H and 0 <= xs < W:
                                acc += int(dq[ch, dy, dx]) * int(u[yy, xs, ch])
                    v[y, xx, ch] = _cl(_rq(acc, dS - I.FA))
        z = np.clip(z + _layer(v, n["w2"]), -127, 127)
        u2 = _layer(z, n["w3"], act=True)
        z = np.clip(z + _layer(u2, n["w4"]), -127, 127)
    else:
        sm = step_map(H, W)
        sc = np.where(sm < k, np.clip(s, -127, 127), 0).astype(np.int64)
        a = _layer(sc[:, :, None], n["wa"])
        z = _layer(np.concatenate([a, l], axis=2), n["wz"])
        u = _layer(z, n["w1"], act=True)
        z = np.clip(z + _layer(u, n["w2"]), -127, 127)
    t = np.zeros((H, W), dtype=np.int64)
    j = np.zeros((H, W), dtype=np.int64)
    hd = n["wh"]
    for y in range(H):
        for xx in range(W):
            t[y, xx] = max(-(1 << 23), min(1 << 23, _rq(_conv_px(z, hd.wq, hd.bq, y, xx, 0),
                                                        hd.S - 4)))
            j[y, xx] = max(0, min(127, _rq(_conv_px(z, hd.wq, hd.bq, y, xx, 1), hd.S - 3) + 24))
    return t, j


@pytest.fixture(scope="module")
def tiny():
    cfg = S.ModelConfig(levels=2, C=4)
    t = S.random_model(cfg, 3)
    # larger weights than the init so that clamps and LeakyReLU branches occur
    for name in list(t):
        if name.startswith(("lstm.", "sb.", "ll.")) and not name.endswith(".bh"):
            t[name] = t[name] * 4.0
    blob = S.pack_blob(cfg, t)
    return I.IntContextModel(K.Model(blob).tensors, 4)


def test_integer_model_equals_brute_force(tiny):
    rng = np.random.default_rng(0)
    s_prev = rng.integers(-200, 200, (3, 4))
    s = rng.integers(-40, 40, (6, 8))
    h, c = tiny.lstm(s_prev, None, None, True)
    hb, cb = _brute_lstm(tiny, s_prev, None, None, True)
    assert np.array_equal(h, hb) and np.array_equal(c, cb)
    assert np.any(np.abs(c) > 0) and np.any(h != 0)
    s2 = rng.integers(-40, 40, (6, 8))
    h2, c2 = tiny.lstm(s, h, c, False)
    hb2, cb2 = _brute_lstm(tiny, s, hb, cb, False)
    assert np.array_equal(h2, hb2) and np.array_equal(c2, cb2)
    for ns, l in (("sb", h2), ("ll", np.zeros_like(h2))):
        for k in range(4):
            t, j = tiny.step_tj(k, s2, l, ns)
            tb, jb = _brute_step(tiny, k, s2, l, ns)
            assert np.array_equal(t, tb), (ns, k)
            assert np.array_equal(j, jb), (ns, k)


def test_integer_steps_are_causal(tiny):
    rng = np.random.default_rng(1)
    s = rng.integers(-40, 40, (6, 8))
    l = rng.integers(-127, 128, (6, 8, 4))
    sm = step_map(6, 8)
    for k in range(4):
        t, j = tiny.step_tj(k, s, l, "sb")
        s2 = np.where(sm >= k, rng.integers(-40, 40, s.shape), s)   # change steps >= k
        t2, j2 = tiny.step_tj(k, s2, l, "sb")
        assert np.array_equal(t, t2) and np.array_equal(j, j2)


def test_integer_model_streams_round_trip():
    cfg = S.ModelConfig(levels=4, C=8)
    blob = S.pack_blob(cfg, S.random_model(cfg, 0))
    img = S.rgb_natural(48, 64, seed=2)
    bs = K.encode_image(blob, img, q=8.0, integer=True)
    hd = K.parse_header(bs)
    assert hd["integer"] and (bs[6] >> 2) & 3 == 3
    out = K.decode_image(blob, bs)
    # the probability model changes only the rate
    assert np.array_equal(out, K.decode_image(blob, K.encode_image(blob, img, q=8.0)))
    model = K.Model(blob, integer=True)
    planes, colour = K.colour_forward(img, False, 8)
    bs2, qenc = K.encode_planes(model, planes, width=64, height=48, bitdepth=8,
                                colour=colour, q=8.0, chunk=100)
    _, qdec = K.decode_symbols(K.Model(blob), bs2)     # decoding follows the stream
    for qa, qb in zip(qenc, qdec):
        for a, b in zip(qa, qb):
            assert np.array_equal(a, b)


def test_integer_autoregressive_ll_sequential_equals_parallel():
    """The integer AR LL model evaluated position by position from the
    causal neighbourhood (explicit tap loops) equals its masked-convolution
    evaluation over the whole plane, and ignores every non-causal symbol."""
    cfg = S.ModelConfig(levels=2, C=8, ll_mode=1)
    t = S.random_model(cfg, 5)
    for name in ("ar.w5", "ar.w1", "ar.wh"):
        t[name] = t[name] * 4.0
    m = I.IntContextModel(K.Model(S.pack_blob(cfg, t)).tensors, 8, ll_mode=1)
    rng = np.random.default_rng(2)
    s = rng.integers(-150, 150, (5, 7))
    ta, ja = m.ar_tj_all(s)
    assert len(np.unique(ta)) > 5 and len(np.unique(ja)) > 3
    for y in range(5):
        for x in range(7):
            assert m.ar_tj_at(s, y, x) == (ta[y, x], ja[y, x])
            s2 = s.copy()
            s2.reshape(-1)[y * 7 + x:] = rng.integers(-150, 150, s2.size - (y * 7 + x))
            assert m.ar_tj_at(s2, y, x) == (ta[y, x], ja[y, x])


def test_integer_autoregressive_ll_streams_round_trip():
    cfg = S.ModelConfig(levels=4, C=8, ll_mode=1)
    blob = S.pack_blob(cfg, S.random_model(cfg, 1))
    img = S.gray_sinusoids(48, 64, seed=9)
    bs = K.encode_image(blob, img, q=8.0, integer=True)
    hd = K.parse_header(bs)
    assert hd["integer"] and hd["ll_ar"]
    assert np.array_equal(K.decode_image(blob, bs),
                          K.decode_image(blob, K.encode_image(blob, img, q=8.0)))
