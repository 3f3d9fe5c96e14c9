"""Tensor-core (tcgen05, BF16) path against the oracle.

* One convolution on the tensor cores vs the oracle's FP64 convolution of the
  same BF16-rounded inputs and weights: within BF16 output rounding
  (2^-8 relative) plus 1e-3 absolute.
* The BF16 codec: encode -> decode reproduces the encoder's quantised
  coefficients exactly; batch invariance; reconstruction PSNR within 0.01 dB
  of the oracle's (the lifting stays FP32); entropy parameters against the
  FP64 oracle are reported and bounded loosely (BF16 errors are reported,
  not gated at 1e-3).
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle.lifting import conv2d
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


@pytest.fixture(scope="module")
def tc(pw):
    c = pw.Codec(0, "bf16")
    yield c
    c.close()


@pytest.mark.parametrize("P,H,W,cin,cout,ks,act", [
    (1, 16, 8, 64, 64, 1, 0),
    (2, 37, 45, 64, 64, 3, 1),
    (1, 50, 23, 128, 256, 3, 0),
    (3, 5, 3, 32, 64, 3, 0),
    (2, 19, 30, 128, 64, 1, 0),
    (1, 40, 40, 64, 128, 1, 1),
    (1, 33, 70, 32, 32, 3, 0),
    (2, 160, 96, 64, 64, 3, 0),
])
def test_conv_bf16_matches_oracle(tc, P, H, W, cin, cout, ks, act):
    rng = np.random.default_rng(P * 1000 + H + W + cin + cout + ks)
    x = rng.normal(size=(P, H, W, cin)).astype(np.float32)
    w = (rng.normal(size=(cout, cin, ks, ks)) / np.sqrt(cin * ks * ks)).astype(np.float32)
    b = rng.normal(size=cout).astype(np.float32)
    y = tc.conv_bf16(x, w, b, act=bool(act))
    xb, wb = bf16(x).astype(np.float64), bf16(w).astype(np.float64)
    for p in range(P):
        ref = conv2d(xb[p], wb, b.astype(np.float64))
        if act:
            ref = np.where(ref >= 0, ref, 0.01 * ref)
        err = np.abs(y[p] - ref)
        assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-3), float(err.max())


def _blob(C, levels=4, seed=0):
    cfg = S.ModelConfig(levels=levels, C=C, ll_mode=0)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


@pytest.mark.parametrize("C", [32, 64])
@pytest.mark.parametrize("rgb", [False, True])
def test_bf16_roundtrip_symbols_exact(tc, C, rgb):
    gm = tc.load_model(_blob(C))
    img = S.rgb_natural(72, 104, seed=7) if rgb else S.gray_sinusoids(72, 104, seed=7)
    bs = tc.encode_image(gm, img, q=8.0, chunk=300)
    assert np.array_equal(tc.decode_symbols(gm, bs), tc.analyse(gm, img, q=8.0))


def test_bf16_batch_invariance(tc):
    gm = tc.load_model(_blob(64))
    imgs = [S.rgb_natural(48, 80, seed=s) for s in (20, 21, 22)]
    single = [tc.encode_image(gm, im, q=8.0) for im in imgs]
    assert tc.encode_batch(gm, imgs, q=8.0) == single
    dec = tc.decode_batch(gm, single)
    for i, bs in enumerate(single):
        assert np.array_equal(dec[i], tc.decode_image(gm, bs))


def test_bf16_psnr_matches_oracle(tc):
    blob = _blob(32)
    gm = tc.load_model(blob)
    img = S.rgb_natural(64, 96, seed=9)
    out = tc.decode_image(gm, tc.encode_image(gm, img, q=8.0))
    ref = K.decode_image(blob, K.encode_image(blob, img, q=8.0))

    def psnr(a):
        return 10 * np.log10(255.0 ** 2 / np.mean((a.astype(float) - img) ** 2))
    assert abs(psnr(out) - psnr(ref)) < 0.01


def test_bf16_entropy_params_error_vs_oracle(tc):
    blob = _blob(32)
    gm = tc.load_model(blob)
    om = K.Model(blob)
    img = S.gray_sinusoids(80, 112, seed=5)
    planes, _ = K.colour_forward(img, False, 8)
    qsb = [K.quantise(s, np.float32(1 / 8.0)) for s in om.lift.forward(K.pad_plane(planes[0], 16), 4, False)]
    mu, sg = tc.context_params(gm, 80, 112, np.concatenate([q.reshape(-1) for q in qsb]))
    ref = K.context_params_all(om, qsb)
    mu_o = np.concatenate([r[0].reshape(-1) for r in ref])
    sg_o = np.concatenate([r[1].reshape(-1) for r in ref])
    e_mu = np.abs(mu - mu_o) / np.maximum(np.abs(mu_o), 1.0)
    e_sg = np.abs(sg - sg_o) / sg_o
    print(f"BF16 vs FP64 oracle: mu rel err mean {e_mu.mean():.2e} max {e_mu.max():.2e}; "
          f"sigma rel err mean {e_sg.mean():.2e} max {e_sg.max():.2e}")
    assert e_mu.max() < 0.25 and e_sg.max() < 0.25
    assert e_mu.mean() < 0.02 and e_sg.mean() < 0.02


def test_bf16_lift_inverse_matches_oracle(tc):
    """Inverse lifting with the CNNs' middle layer on the tensor cores (BF16
    operands, FP32 accumulation) against the FP64 oracle's exact inverse.

    The layer-2 inputs lie in (-1, 1) (tanh) and enter in BF16 (2^-9
    relative) like the weights; with the lifting nets' residual outputs of
    order 1 this perturbs each lifting step by ~1e-3, and 16 steps over four
    levels keep the reconstruction within 0.1 of the signal (range +-128)
    and its RMS error below 0.01.
    """
    blob = _blob(32)
    gm = tc.load_model(blob)
    om = K.Model(blob)
    H, W = 80, 112        # level-1 subbands 40 x 56: ragged 16 x 16 tiles
    x = np.random.default_rng(3).uniform(-128, 127, (H, W))
    sb = om.lift.forward(x, 4, lossless=False)
    flat = np.concatenate([s.reshape(-1) for s in sb])
    got = tc.lift_inverse(gm, flat.astype(np.float32), H, W)
    err = got - x
    print(f"BF16 tensor-core inverse lifting vs FP64 oracle: max {np.abs(err).max():.2e} "
          f"rms {np.sqrt(np.mean(err ** 2)):.2e}")
    assert np.abs(err).max() < 0.1
    assert np.sqrt(np.mean(err ** 2)) < 0.01


def test_precision_class_recorded_in_stream(tc, pw):
    blob = _blob(32)
    fp = pw.Codec(0, "fp32")
    bs = fp.encode_image(fp.load_model(blob), S.gray_sinusoids(32, 48, seed=3), q=8.0)
    with pytest.raises(pw.PwError) as e:
        tc.decode_image(tc.load_model(blob), bs)
    assert e.value.code == pw.PW_EINVAL
    fp.close()


def test_bf16_ar_ll_roundtrip(tc):
    cfg = S.ModelConfig(levels=4, C=64, ll_mode=1)
    gm = tc.load_model(S.pack_blob(cfg, S.random_model(cfg, 5)))
    for im in (S.gray_sinusoids(64, 96, seed=15), S.rgb_natural(48, 80, seed=16)):
        bs = tc.encode_image(gm, im, q=8.0)
        assert np.array_equal(tc.decode_symbols(gm, bs), tc.analyse(gm, im, q=8.0))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_compact_head_ragged_subbands_vs_oracle(pw, prec):
    """The head convolution of steps 2-4 runs on the step's own positions
    only (a quarter of the plane). Subbands whose width is not a multiple of
    4 (18 and 9 columns here) and whose height is odd (7 rows) exercise its
    border handling; the entropy parameters stay within the precision's
    error against the FP64 oracle everywhere, including the last columns."""
    codec = pw.Codec(0, prec)
    blob = _blob(64)
    gm = codec.load_model(blob)
    om = K.Model(blob)
    H, W = 112, 144       # subbands 56x72, 28x36, 14x18, 7x9
    img = S.gray_sinusoids(H, W, seed=21)
    planes, _ = K.colour_forward(img, False, 8)
    qsb = [K.quantise(s, np.float32(1 / 8.0)) for s in om.lift.forward(K.pad_plane(planes[0], 16), 4, False)]
    mu, sg = codec.context_params(gm, H, W, np.concatenate([q.reshape(-1) for q in qsb]))
    ref = K.context_params_all(om, qsb)
    o = 0
    worst = 0.0
    for q, (mo, so) in zip(qsb, ref):
        n = q.size
        m_g = mu[o:o + n].reshape(q.shape)
        s_g = sg[o:o + n].reshape(q.shape)
        o += n
        e_mu = np.abs(m_g - mo) / np.maximum(np.abs(mo), 1.0)
        e_sg = np.abs(s_g - so) / so
        assert np.all(np.isfinite(m_g)) and np.all(np.isfinite(s_g))
        worst = max(worst, float(e_mu[:, -2:].max()), float(e_sg[:, -2:].max()))
        assert e_mu.mean() < 0.02 and e_sg.mean() < 0.02, (q.shape, e_mu.mean(), e_sg.mean())
        assert e_mu.max() < 0.25 and e_sg.max() < 0.25, (q.shape, e_mu.max(), e_sg.max())
    print(f"{prec}: worst relative error in the last two columns {worst:.2e}")
    bs = codec.encode_image(gm, img, q=8.0)
    assert np.array_equal(codec.decode_symbols(gm, bs), codec.analyse(gm, img, q=8.0))
    gm.close()
    codec.close()
