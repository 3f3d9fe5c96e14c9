"""Pins of the oracle's lifting transform (Section 3.1, Fig. 2, Section 3.4).

Each test checks the oracle against something other than itself: the
perfect-reconstruction property the lifting structure guarantees for any
P/U, the JPEG 2000 reversible 5/3 transform written out from its textbook
definition, the LeGall 5/3 synthesis filters, the closed-form 2-D Haar basis
functions (the subband impulse responses of Section 3.4 for a Haar linear
part), and scipy's 2-D correlation for the CNN convolutions.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

import synthetic as S
from oracle import lifting as LF
from tests._lib import golden


def _model(levels=4, seed=0):
    cfg = S.ModelConfig(levels=levels, C=8)
    return S.random_model(cfg, seed)


def test_conv2d_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(9, 13, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    out = LF.conv2d(x, w, b)
    for o in range(2):
        ref = b[o] + sum(correlate2d(x[:, :, i], w[o, i], mode="same",
                                     boundary="fill") for i in range(3))
        np.testing.assert_allclose(out[:, :, o], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("levels,shape", [(4, (64, 48)), (5, (96, 64)), (1, (6, 10))])
def test_float_perfect_reconstruction_any_weights(levels, shape):
    t = _model(levels, seed=3)
    lift = LF.Lifting(t)
    x = np.random.default_rng(1).uniform(-128, 127, shape)
    sb = lift.forward(x, levels, lossless=False)
    y = lift.inverse(sb, levels, lossless=False)
    assert np.max(np.abs(y - x)) < 1e-9


def test_integer_lifting_exact_roundtrip_12bit_5_levels():
    t = _model(5, seed=4)
    lift = LF.Lifting(t)
    x = np.random.default_rng(2).integers(0, 4096, (64, 96)).astype(np.float64) - 2048
    sb = lift.forward(x, 5, lossless=True)
    for s in sb:
        assert np.all(s == np.round(s))
    y = lift.inverse(sb, 5, lossless=True)
    assert np.array_equal(y, x)


def _jpeg2000_53_rows(x):
    """Reversible 5/3 of ITU-T T.800 along axis 1, from its definition:
    d[n] = x[2n+1] - floor((x[2n] + x[2n+2]) / 2),
    s[n] = x[2n] + floor((d[n-1] + d[n] + 2) / 4), symmetric extension."""
    H, W = x.shape
    N = W // 2
    xi = x.astype(np.int64)
    d = np.zeros((H, N), dtype=np.int64)
    s = np.zeros((H, N), dtype=np.int64)
    for n in range(N):
        right = xi[:, 2 * n + 2] if 2 * n + 2 < W else xi[:, 2 * n]   # x[W] = x[W-2]
        d[:, n] = xi[:, 2 * n + 1] - np.floor_divide(xi[:, 2 * n] + right, 2)
    for n in range(N):
        left = d[:, n - 1] if n > 0 else d[:, 0]                     # d[-1] = d[0]
        s[:, n] = xi[:, 2 * n] + np.floor_divide(left + d[:, n] + 2, 4)
    return s, d


def test_integer_mode_without_cnn_is_jpeg2000_reversible_53():
    x = np.random.default_rng(5).integers(-2048, 2048, (6, 20)).astype(np.float64)
    lp, hp = LF.lift_fwd(x, 1, None, None, lossless=True)
    s, d = _jpeg2000_53_rows(x)
    assert np.array_equal(lp, s)
    assert np.array_equal(hp, d)
    lp0, hp0 = LF.lift_fwd(x.T, 0, None, None, lossless=True)
    assert np.array_equal(lp0.T, s) and np.array_equal(hp0.T, d)


def test_float_53_synthesis_filters():
    """Inverse 1-D step without CNN: the LeGall 5/3 synthesis filters
    g0 = [1/2, 1, 1/2] and g1 = [-1/8, -1/4, 3/4, -1/4, -1/8]."""
    N = 8
    lp = np.zeros((1, N)); hp = np.zeros((1, N))
    lp[0, 3] = 1.0
    x = LF.lift_inv(lp, hp, 1, None, None, lossless=False)[0]
    ref = np.zeros(2 * N); ref[5:8] = [0.5, 1.0, 0.5]
    np.testing.assert_allclose(x, ref, atol=0)
    lp[:] = 0; hp[0, 3] = 1.0
    x = LF.lift_inv(lp, hp, 1, None, None, lossless=False)[0]
    ref = np.zeros(2 * N); ref[5:10] = [-0.125, -0.25, 0.75, -0.25, -0.125]
    np.testing.assert_allclose(x, ref, atol=0)


def _haar_1d(kind, level, n):
    """Closed-form 1-D Haar synthesis function of the lifting pair
    L = (e + o) / 2, H = o - e at `level` (support 2^level)."""
    f = np.zeros(n)
    s = 1 << level
    if kind == "L":
        f[:s] = 1.0
    else:
        f[:s // 2] = -0.5
        f[s // 2:s] = 0.5
    return f


def test_subband_impulse_responses_are_haar_basis_functions():
    """Section 3.4: an impulse placed in each of the 13 subbands of an
    all-zero 16x16 latent (4 levels, level-4 subbands 1x1) and inverse
    transformed; with a Haar linear part and no CNN residual the responses
    are the 2-D Haar basis functions (outer product of the column and row
    synthesis functions)."""
    levels = 4
    lift = LF.Lifting(None, linear="haar")
    shapes = LF.subband_shapes(16, 16, levels)
    assert len(shapes) == 13 and shapes[0][:2] == (1, 1)
    names = ["LL"] + ["HL", "LH", "HH"] * levels
    for i, (h, w, lv) in enumerate(shapes):
        sb = [np.zeros((hh, ww)) for hh, ww, _ in shapes]
        sb[i][0, 0] = 7.0
        x = lift.inverse(sb, levels, lossless=False)
        nm = names[i]
        row_kind = "H" if nm in ("HL", "HH") else "L"   # HL: row highpass
        col_kind = "H" if nm in ("LH", "HH") else "L"
        ref = 7.0 * np.outer(_haar_1d(col_kind, lv, 16), _haar_1d(row_kind, lv, 16))
        np.testing.assert_allclose(x, ref, atol=1e-12, err_msg=f"subband {i} {nm}{lv}")


def test_subband_layout_matches_the_paper():
    # tests/golden/subband_layout.txt: Secs. 3.1, 3.2 and 3.4
    g = golden("subband_layout.txt")
    shapes = LF.subband_shapes(16, 16, 4)
    assert len(shapes) == g["subbands"][0][0]
    for lv, count, h, w in g["level"]:
        at = [s for s in shapes if s[2] == lv]
        assert len(at) == count and all(s[:2] == (h, w) for s in at), (lv, at)
    d = g["ll_divisor"][0][0]
    for H, W in [(512, 768), (64, 32), (1024, 2048)]:
        assert LF.subband_shapes(H, W, 4)[0][:2] == (H // d, W // d)


def test_subband_geometry():
    shapes = LF.subband_shapes(512, 768, 4)
    assert len(shapes) == 13
    assert shapes[0] == (32, 48, 4)
    assert [s[2] for s in shapes] == [4, 4, 4, 4, 3, 3, 3, 2, 2, 2, 1, 1, 1]
    assert sum(h * w for h, w, _ in shapes) == 512 * 768
    shapes5 = LF.subband_shapes(2176, 3840, 5)
    assert len(shapes5) == 16 and shapes5[0][:2] == (68, 120)


def test_forward_coefficient_count_and_order():
    t = _model(4, seed=6)
    lift = LF.Lifting(t)
    x = np.random.default_rng(7).uniform(-100, 100, (32, 48))
    sb = lift.forward(x, 4, lossless=False)
    assert [s.shape for s in sb] == [(h, w) for h, w, _ in LF.subband_shapes(32, 48, 4)]


def test_temporal_lifting_gop_closed_form_without_cnn():
    # GOP size of the paper's video experiments (tests/golden/gop.txt). With
    # the predict and update CNNs zeroed, the temporal lifting is the Haar
    # transform along time: the last lowpass band is the mean of the GOP and
    # the level-1 highpass bands (the last n/2, in frame order) are the
    # differences of the frame pairs.
    n = golden("gop.txt")["gop_size"][0][0]
    T = int(round(np.log2(n)))
    assert 2 ** T == n
    t = {k: (np.zeros_like(v) if k.startswith("tlift.") else v)
         for k, v in _model(4, seed=8).items()}
    rng = np.random.default_rng(10)
    frames = [rng.uniform(-128, 127, (8, 12)) for _ in range(n)]
    bands = LF.temporal_forward(frames, t, T)
    assert len(bands) == n
    np.testing.assert_allclose(bands[0], np.mean(frames, axis=0), atol=1e-12)
    for m, h in enumerate(bands[n - n // 2:]):
        np.testing.assert_allclose(h, frames[2 * m + 1] - frames[2 * m], atol=1e-12)


def test_temporal_lifting_perfect_reconstruction():
    t = _model(4, seed=8)
    rng = np.random.default_rng(9)
    frames = [rng.uniform(-128, 127, (16, 24)) for _ in range(8)]
    bands = LF.temporal_forward(frames, t, 3)
    assert len(bands) == 8
    back = LF.temporal_inverse(bands, t, 3)
    for a, b in zip(frames, back):
        assert np.max(np.abs(a - b)) < 1e-9


# ---------------------------------------------------------------------------
# The integer-mode FP32 operation sequence (tanh32, conv3x3_fp32)
def test_tanh32_within_a_few_ulps_of_tanh():
    from oracle.lifting import tanh32
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.uniform(-12, 12, 200000), rng.normal(0, 0.1, 100000),
                        np.linspace(-0.2, 0.2, 20001), [0.0, -0.0, 1e-30, 40.0, -90.0,
                                                       0.171875, -0.171875]])
    x32 = x.astype(np.float32)
    got = tanh32(x32).astype(np.float64)
    ref = np.tanh(x32.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(got - ref) / ulp
    assert err.max() <= 5.0, float(err.max())   # measured 4.2
    assert np.all(np.sign(got) == np.sign(ref))
    assert np.signbit(tanh32(np.float32(-0.0))) and tanh32(np.float32(90.0)) == 1.0


def test_tanh32_coefficients_are_the_nearest_floats():
    import math
    from oracle.lifting import _INV_FACT32
    for n, c in _INV_FACT32.items():
        exact = 1.0 / math.factorial(n)
        assert c == np.float32(exact)
        assert abs(float(c) - exact) <= np.spacing(np.float32(exact)) / 2


def test_conv3x3_fp32_matches_fp64_conv_within_rounding():
    from oracle.lifting import conv2d, conv3x3_fp32
    rng = np.random.default_rng(22)
    x = rng.integers(-2048, 2048, (9, 11, 3)).astype(np.float64)
    w = rng.uniform(-0.2, 0.2, (5, 3, 3, 3)).astype(np.float32).astype(np.float64)
    b = rng.uniform(-1, 1, 5).astype(np.float32).astype(np.float64)
    got = conv3x3_fp32(x, w, b).astype(np.float64)
    ref = conv2d(x, w, b)
    # 28 rounded terms of magnitude <= 0.2 * 2048 each
    bound = 28 * 2 * np.finfo(np.float32).eps * (np.abs(w).max() * 2048 * 27 + 1)
    assert np.max(np.abs(got - ref)) <= bound


def test_integer_lifting_uses_the_fp32_sequence_and_stays_exact():
    """Integer mode rounds P_lin + CNN evaluated by lift_cnn_fp32; the
    round trip stays exact and the P values equal floor of that FP32 sum."""
    from oracle.lifting import lift_cnn_fp32, predict
    cfg = S.ModelConfig(levels=3, C=8)
    t = {k: v.astype(np.float64) for k, v in S.random_model(cfg, 5).items()}
    net = LF.net_of(t, "lift.row.P.")
    e = np.random.default_rng(23).integers(-3000, 3000, (12, 10)).astype(np.float64)
    p = predict(e, 1, net, True)
    lin = 0.5 * (e + np.concatenate([e[:, 1:], e[:, -1:]], axis=1))
    want = np.floor((lin.astype(np.float32) + lift_cnn_fp32(e, net)).astype(np.float32))
    assert np.array_equal(p, want.astype(np.float64))
    lift = LF.Lifting(t)
    x = np.random.default_rng(24).integers(-2048, 2048, (32, 48)).astype(np.float64)
    sb = lift.forward(x, 3, True)
    assert all(np.array_equal(s, np.round(s)) for s in sb)
    assert np.array_equal(lift.inverse(sb, 3, True), x)


# ---------------------------------------------------------------------------
# Motion-compensated temporal lifting (Section 3.3)
def _tlift_tensors(seed=3, zero=False):
    cfg = S.ModelConfig(levels=4, C=8)
    t = {k: v.astype(np.float64) for k, v in S.random_model(cfg, seed).items()}
    if zero:
        for k in t:
            if k.startswith("tlift."):
                t[k] = np.zeros_like(t[k])
    return t


def test_zero_motion_is_the_identity_motion_transform():
    t = _tlift_tensors()
    rng = np.random.default_rng(30)
    frames = [rng.uniform(-128, 127, (32, 48)) for _ in range(8)]
    zero = [np.zeros((2, 3, 2), dtype=np.int64) for _ in range(7)]
    a = LF.temporal_forward(frames, t, 3)
    b = LF.temporal_forward(frames, t, 3, zero)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert all(np.array_equal(x, y) for x, y in
               zip(LF.temporal_inverse(a, t, 3), LF.temporal_inverse(b, t, 3, zero)))


def test_mc_lifting_reconstructs_perfectly_for_any_vectors():
    t = _tlift_tensors(seed=4)
    rng = np.random.default_rng(31)
    frames = [rng.uniform(-128, 127, (48, 64)) for _ in range(8)]
    mvs = [rng.integers(-16, 17, (3, 4, 2)) for _ in range(7)]
    bands = LF.temporal_forward(frames, t, 3, mvs)
    back = LF.temporal_inverse(bands, t, 3, mvs)
    assert max(np.max(np.abs(a - b)) for a, b in zip(back, frames)) < 1e-9


def test_mc_warp_reads_the_block_vector_with_clamping():
    f = np.arange(32 * 32, dtype=np.float64).reshape(32, 32)
    mv = np.zeros((2, 2, 2), dtype=np.int64)
    mv[0, 1] = (2, -3)           # block rows 0..15, columns 16..31
    mv[1, 0] = (-20, 5)
    w = LF.mc_warp(f, mv, +1)
    assert w[4, 20] == f[6, 17] and w[4, 4] == f[4, 4]
    assert w[17, 3] == f[0, 8]                         # row 17 - 20 clamped to 0
    v = LF.mc_warp(f, mv, -1)
    assert v[4, 20] == f[2, 23] and v[17, 3] == f[31, 0]


def test_motion_search_matches_brute_force_definition():
    rng = np.random.default_rng(32)
    ref = rng.integers(0, 256, (32, 40))
    cur = np.roll(ref, (1, -2), axis=(0, 1)) + rng.integers(-3, 4, (32, 40))
    R = 4
    got = LF.motion_search(cur, ref, 16, R)
    H, W = cur.shape
    for by in range(2):
        for bx in range(3):
            best = None
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    sad = 0
                    for y in range(by * 16, min(by * 16 + 16, H)):
                        for x in range(bx * 16, min(bx * 16 + 16, W)):
                            yy = min(max(y + dy, 0), H - 1)
                            xx = min(max(x + dx, 0), W - 1)
                            sad += abs(int(cur[y, x]) - int(ref[yy, xx]))
                    key = (sad, abs(dy) + abs(dx), dy, dx)
                    if best is None or key < best:
                        best = key
            assert tuple(got[by, bx]) == best[2:], (by, bx, got[by, bx], best)
    flat = LF.motion_search(np.full((32, 32), 7), np.full((32, 32), 7), 16, 3)
    assert np.all(flat == 0)                           # all ties -> (0, 0)


def test_translated_gop_highpass_vanishes_with_motion():
    """Frames of one canvas moving by (2, -3) pixels per frame: the search
    finds the motion, and with zero CNN residuals (Haar predict) the
    level-1 highpass bands are exactly zero wherever the prediction reads
    inside the frame."""
    t = _tlift_tensors(zero=True)
    canvas = np.random.default_rng(33).integers(0, 256, (120, 140)).astype(np.float64)
    frames = [canvas[40 + 2 * k:40 + 2 * k + 48, 40 - 3 * k:40 - 3 * k + 64] for k in range(8)]
    mvs = LF.gop_motion(frames, 3)
    assert np.all(mvs[0] == (2, -3))
    bands = LF.temporal_forward(frames, t, 3, mvs)
    for h in bands[4:8]:                               # level-1 highpass bands
        assert np.all(h[:46, 3:] == 0.0)
    zero = LF.temporal_forward(frames, t, 3)
    # only the border strips the motion uncovers (2 rows, 3 columns) remain
    assert np.sum(np.abs(bands[4])) < 0.15 * np.sum(np.abs(zero[4]))
