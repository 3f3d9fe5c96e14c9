"""Closed-form pins of the oracle's layer composition, colour transforms and
padding (Sections 3.1 and 3.2).

Each test sets the context-fusion weights of Section 3.2 to special values
(zeros, identities, single taps) for which the step's output has a closed
form that is written out here by hand, position by position, without the
oracle's convolution helpers. The weight choices are made so that a
plausible slip in the oracle fails at least one of them: a missing skip
connection of the DepthConvBlock or the residual block, the [a, l] channel
blocks of the steps 2-4 fusion swapped, a wrong LeakyReLU slope, a flipped
or transposed spatial tap, the head's two outputs exchanged, or softplus
evaluated inaccurately at large or very negative arguments.

The colour transforms are checked against the published matrices: BT.601
full-range YCbCr as JPEG File Interchange Format writes it (coefficients
printed to six decimals) and the reversible colour transform of JPEG 2000
(Part 1, Annex G). Padding is checked against an explicit whole-sample
mirror index table.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle.context import ContextModel, softplus, step_map

C = 4


def _zero_model(C=C, ll_mode=0):
    cfg = S.ModelConfig(levels=4, C=C, ll_mode=ll_mode)
    t = {name: np.zeros(shape) for name, shape in S.tensor_specs(cfg)}
    return ContextModel(t, C, ll_mode), t


def _lrelu(v):
    return v if v >= 0 else 0.01 * v


def _head_select(t, p, mu_ch, rho_ch, rho_bias=0.0):
    """Head 1x1 that copies channel mu_ch to mu and channel rho_ch to rho."""
    t[p + "wh"][:] = 0.0
    t[p + "wh"][0, mu_ch] = 1.0
    t[p + "wh"][1, rho_ch] = 1.0
    t[p + "bh"][:] = [0.0, rho_bias]


# --------------------------------------------------------------------------
# step 1: 1x1 -> DepthConvBlock (two residual parts) -> head
@pytest.mark.parametrize("ns", ["sb", "ll"])
def test_step1_skip_paths_add_their_biases(ns):
    """All block weights zero: part 1 adds W2 b_dw + b2 (the depthwise conv
    of a zero input is its bias), part 2 adds b4. mu = l0 + bin0 + bdw0 +
    b2_0 + b4_0 with W2 = identity."""
    cm, t = _zero_model()
    p = f"{ns}.s0."
    rng = np.random.default_rng(0)
    l = rng.normal(size=(6, 8, C))
    t[p + "win"][:] = np.eye(C)
    t[p + "bin"][:] = [0.25, -0.5, 1.0, 2.0]
    t[p + "b1"][:] = [3.0, -3.0, 1.0, 1.0]      # lrelu(b1) is killed by wdw = 0
    t[p + "bdw"][:] = [0.125, 0.5, -0.75, 1.5]
    t[p + "w2"][:] = np.eye(C)
    t[p + "b2"][:] = [1.0, 0.0, 0.0, -1.0]
    t[p + "b3"][:] = 5.0                         # killed by w4 = 0
    t[p + "b4"][:] = [0.0, 0.375, 0.0, 0.0]
    _head_select(t, p, 0, 1)
    mu, sg = cm.step_params(0, np.zeros((6, 8)), l, ns)
    for y in range(6):
        for x in range(8):
            e_mu = l[y, x, 0] + 0.25 + 0.125 + 1.0 + 0.0
            e_rho = l[y, x, 1] - 0.5 + 0.5 + 0.0 + 0.375
            assert abs(mu[y, x] - e_mu) < 1e-12
            assert abs(sg[y, x] - math.log1p(math.exp(e_rho))) < 1e-12


def test_step1_depthwise_tap_orientation_and_leaky_slope():
    """Identity 1x1s and a depthwise kernel with one off-centre tap:
    z = l + lrelu(l)[y + dy - 1, x + dx - 1] (zero outside the plane);
    negative l makes the 0.01 slope visible."""
    cm, t = _zero_model()
    p = "sb.s0."
    rng = np.random.default_rng(1)
    H, W = 5, 7
    l = rng.normal(size=(H, W, C)) * 3.0
    t[p + "win"][:] = np.eye(C)
    t[p + "w1"][:] = np.eye(C)
    dy, dx = 0, 2                                # the up-right neighbour
    t[p + "wdw"][:, dy, dx] = 1.0
    t[p + "w2"][:] = np.eye(C)
    _head_select(t, p, 2, 3)
    mu, sg = cm.step_params(0, np.zeros((H, W)), l, "sb")
    for y in range(H):
        for x in range(W):
            yy, xx = y + dy - 1, x + dx - 1
            nb = [_lrelu(l[yy, xx, c]) if 0 <= yy < H and 0 <= xx < W else 0.0
                  for c in range(C)]
            assert abs(mu[y, x] - (l[y, x, 2] + nb[2])) < 1e-12
            rho = l[y, x, 3] + nb[3]
            assert abs(sg[y, x] - math.log1p(math.exp(rho))) < 1e-12


def test_step1_feed_forward_part():
    """Part 2 with W3 = [I; -I] and W4 = [I, -I]: W4 lrelu(W3 z) =
    lrelu(z) - lrelu(-z) = 1.01 z, so z -> 2.01 z (the slope enters
    through both halves)."""
    cm, t = _zero_model()
    p = "sb.s0."
    l = np.linspace(-4.0, 4.0, 3 * 5 * C).reshape(3, 5, C)
    t[p + "win"][:] = np.eye(C)
    t[p + "w3"][:] = np.concatenate([np.eye(C), -np.eye(C)], axis=0)
    t[p + "w4"][:] = np.concatenate([np.eye(C), -np.eye(C)], axis=1)
    _head_select(t, p, 1, 0, rho_bias=-1.0)
    mu, sg = cm.step_params(0, np.zeros((3, 5)), l, "sb")
    np.testing.assert_allclose(mu, 2.01 * l[:, :, 1], rtol=0, atol=1e-12)
    want = np.vectorize(lambda r: math.log1p(math.exp(r)))(2.01 * l[:, :, 0] - 1.0)
    np.testing.assert_allclose(sg, want, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# steps 2-4: masked 3x3 input conv -> 1x1 over [a, l] -> residual block -> head
def _masked(s, k, y, x):
    """s[y, x] if (y, x) is inside and coded before step k, else 0."""
    H, W = s.shape
    if not (0 <= y < H and 0 <= x < W):
        return 0.0
    return s[y, x] if step_map(H, W)[y, x] < k else 0.0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_steps234_fusion_reads_a_block_first(k):
    """wz = [I, 0] selects the masked-symbol block a; a single tap of the
    input conv at (dy, dx) = (1, 0) gives a0[y, x] = (m_<k s)[y, x - 1]."""
    cm, t = _zero_model()
    p = f"sb.s{k}."
    rng = np.random.default_rng(2 + k)
    H, W = 6, 8
    s = rng.integers(-9, 10, (H, W)).astype(np.float64)
    l = rng.normal(size=(H, W, C)) + 100.0       # must not leak into mu
    t[p + "wa"][0, 0, 1, 0] = 1.0
    t[p + "ba"][:] = [0.0, 0.5, 0.0, 0.0]
    t[p + "wz"][:, :C] = np.eye(C)
    t[p + "bz"][:] = [0.0, 0.0, 0.0, 0.0]
    _head_select(t, p, 0, 1)
    mu, sg = cm.step_params(k, s, l, "sb")
    for y in range(H):
        for x in range(W):
            assert abs(mu[y, x] - _masked(s, k, y, x - 1)) < 1e-12
            assert abs(sg[y, x] - math.log1p(math.exp(0.5))) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_steps234_fusion_reads_l_block_second(k):
    """wz = [0, I] selects the long-term context l."""
    cm, t = _zero_model()
    p = f"sb.s{k}."
    rng = np.random.default_rng(5 + k)
    H, W = 4, 8
    s = rng.integers(-9, 10, (H, W)).astype(np.float64)
    l = rng.normal(size=(H, W, C))
    t[p + "wa"][:, 0, 1, 1] = 1000.0             # would dominate if selected
    t[p + "wz"][:, C:] = np.eye(C)
    t[p + "bz"][:] = [0.0, 0.0, 0.0, 0.25]
    _head_select(t, p, 2, 3)
    mu, sg = cm.step_params(k, s, l, "sb")
    np.testing.assert_allclose(mu, l[:, :, 2], rtol=0, atol=1e-12)
    want = np.vectorize(lambda r: math.log1p(math.exp(r)))(l[:, :, 3] + 0.25)
    np.testing.assert_allclose(sg, want, rtol=0, atol=1e-12)


def test_steps234_residual_block_skip_and_taps():
    """Residual block z + w2 * lrelu(w1 * z + b1) + b2:
    (a) w2 = 0: z + b2;
    (b) w1 = single tap at (0, 1) (the row above), w2 = centre tap:
        z + lrelu(z[y - 1, x] + b1), zero above the plane."""
    cm, t = _zero_model()
    p = "sb.s2."
    rng = np.random.default_rng(9)
    H, W = 5, 6
    l = rng.normal(size=(H, W, C)) * 2.0
    t[p + "wz"][:, C:] = np.eye(C)
    t[p + "w1"][:] = rng.normal(size=(C, C, 3, 3))
    t[p + "b1"][:] = 3.0
    t[p + "b2"][:] = [0.5, -0.5, 0.0, 0.0]
    _head_select(t, p, 0, 1)
    mu, _ = cm.step_params(2, np.zeros((H, W)), l, "sb")
    np.testing.assert_allclose(mu, l[:, :, 0] + 0.5, rtol=0, atol=1e-12)

    t[p + "w1"][:] = 0.0
    t[p + "b2"][:] = 0.0
    for c in range(C):
        t[p + "w1"][c, c, 0, 1] = 1.0
        t[p + "w2"][c, c, 1, 1] = 1.0
    t[p + "b1"][:] = [0.0, -0.25, 0.0, 0.0]
    _head_select(t, p, 1, 0)
    mu, sg = cm.step_params(2, np.zeros((H, W)), l, "sb")
    for y in range(H):
        for x in range(W):
            above = l[y - 1, x, 1] if y >= 1 else 0.0
            assert abs(mu[y, x] - (l[y, x, 1] + _lrelu(above - 0.25))) < 1e-12
            above0 = l[y - 1, x, 0] if y >= 1 else 0.0
            rho = l[y, x, 0] + _lrelu(above0)
            assert abs(sg[y, x] - math.log1p(math.exp(rho))) < 1e-12


# --------------------------------------------------------------------------
# head and softplus
@pytest.mark.parametrize("rho,want", [
    (-30.0, 9.357622968839737e-14),   # log(1 + e^-30) = e^-30 - e^-60/2 + ...
    (0.0, 0.6931471805599453),        # log 2
    (20.0, 20.000000002061153),       # 20 + log(1 + e^-20)
    (40.0, 40.0),                     # 40 + 4.2e-18
])
def test_head_softplus_on_constant_input(rho, want):
    cm, t = _zero_model()
    p = "sb.s1."
    t[p + "bz"][:] = [7.0, rho, 0.0, 0.0]
    _head_select(t, p, 0, 1)
    t[p + "bh"][:] = [0.5, 0.0]
    mu, sg = cm.step_params(1, np.zeros((2, 4)), np.zeros((2, 4, C)), "sb")
    np.testing.assert_allclose(mu, 7.5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(sg, want, rtol=1e-14, atol=0)
    np.testing.assert_allclose(softplus(np.array([rho])), [want], rtol=1e-14, atol=0)


def test_autoregressive_ll_single_tap_closed_form():
    """Autoregressive LL model with one 5x5 tap at the position above
    (dy, dx) = (1, 2) and identity 1x1: mu = lrelu(lrelu(s[y - 1, x]))."""
    cm, t = _zero_model(C=2, ll_mode=1)
    t["ar.w5"][0, 0, 1, 2] = 1.0
    t["ar.w1"][:] = np.eye(2)
    t["ar.wh"][0, 0] = 1.0
    s = np.array([[3.0, -2.0, 5.0], [-7.0, 1.0, 0.0], [4.0, -4.0, 2.0]])
    mu, _ = cm.ar_params_all(s)
    for y in range(3):
        for x in range(3):
            v = s[y - 1, x] if y >= 1 else 0.0
            assert abs(mu[y, x] - _lrelu(_lrelu(v))) < 1e-12
            m1, _ = cm.ar_params_at(s, y, x)
            assert abs(m1 - _lrelu(_lrelu(v))) < 1e-12


# --------------------------------------------------------------------------
# colour (Section 3.1: YCbCr; lossless: the JPEG 2000 RCT)
# BT.601 full range as printed in JFIF 1.02 (level shift 128 on Y here)
JFIF_FWD = np.array([[0.299, 0.587, 0.114],
                     [-0.168736, -0.331264, 0.5],
                     [0.5, -0.418688, -0.081312]])
JFIF_INV = np.array([[1.0, 0.0, 1.402],
                     [1.0, -0.344136, -0.714136],
                     [1.0, 1.772, 0.0]])
COLOURS = np.array([[255, 0, 0], [0, 255, 0], [0, 0, 255], [128, 128, 128],
                    [255, 255, 255], [0, 0, 0], [17, 200, 93]], dtype=np.uint8)


def test_ycbcr_forward_matches_bt601_full_range():
    img = COLOURS.reshape(1, -1, 3)
    planes, colour = K.colour_forward(img, False, 8)
    assert colour == 1
    got = np.stack([planes[0][0] + 128.0, planes[1][0], planes[2][0]], axis=1)
    want = COLOURS.astype(np.float64) @ JFIF_FWD.T
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-4)
    # pure red: Cr at its maximum 127.5, Cb negative; pure blue the reverse
    assert abs(got[0, 2] - 127.5) < 1e-9 and got[0, 1] < -40
    assert abs(got[2, 1] - 127.5) < 1e-9 and got[2, 2] < -20


def test_ycbcr_inverse_matches_bt601_full_range():
    rng = np.random.default_rng(4)
    ycc = np.stack([rng.uniform(0, 255, 50), rng.uniform(-128, 127, 50),
                    rng.uniform(-128, 127, 50)], axis=1)
    planes = [ycc[None, :, 0] - 128.0, ycc[None, :, 1], ycc[None, :, 2]]
    got = K.colour_inverse(planes, 1, 8)[0]
    want = ycc @ JFIF_INV.T
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-3)


def test_rct_matches_jpeg2000_definition():
    """JPEG 2000 RCT: Y = floor((R + 2G + B) / 4), U = B - G, V = R - G;
    inverse G = Y - floor((U + V) / 4), R = V + G, B = U + G."""
    rng = np.random.default_rng(5)
    rgb = rng.integers(0, 4096, (40, 3))
    img = rgb.reshape(1, 40, 3).astype(np.uint16)
    planes, colour = K.colour_forward(img, True, 12)
    assert colour == 2
    R, G, B = rgb[:, 0], rgb[:, 1], rgb[:, 2]
    assert np.array_equal(planes[0][0], (R + 2 * G + B) // 4 - 2048)
    assert np.array_equal(planes[1][0], B - G)
    assert np.array_equal(planes[2][0], R - G)
    back = K.colour_inverse(planes, 2, 12)[0]
    assert np.array_equal(back, rgb.astype(np.float64))


# --------------------------------------------------------------------------
# padding (sizes that are not multiples of 2^levels)
def test_pad_plane_whole_sample_mirror_table():
    """Whole-sample symmetric extension repeats no edge sample:
    5 -> 8 reads indices 0 1 2 3 4 3 2 1."""
    x = np.arange(5, dtype=np.float64)[None, :] * np.ones((5, 1))
    y = np.arange(5, dtype=np.float64)[:, None] * np.ones((1, 5)) * 10
    p = K.pad_plane(x + y, 8)
    table = [0, 1, 2, 3, 4, 3, 2, 1]
    assert p.shape == (8, 8)
    for i in range(8):
        for j in range(8):
            assert p[i, j] == 10 * table[i] + table[j]


def test_pad_plane_beyond_one_reflection_clamps():
    """Pads longer than the plane minus one sample reflect once and then
    clamp to the first sample (3 -> 8: 0 1 2 1 0 0 0 0); the library uses
    the same reading."""
    x = np.arange(3, dtype=np.float64)[None, :] * np.ones((8, 1))
    p = K.pad_plane(x, 8)
    assert list(p[0]) == [0, 1, 2, 1, 0, 0, 0, 0]
    assert np.array_equal(K.pad_plane(np.ones((8, 8)) * 3, 8), np.ones((8, 8)) * 3)
