"""GPU parity of the integer-network context model (precision class INT8)
against the oracle's integer model (oracle/intnet.py).

The class's arithmetic is exact integer arithmetic, so the bar is equality
everywhere, with no near-tie certificate: the entropy parameters (t = 16 mu
and the scale bin j) at every position, and the streams themselves - the
GPU encoder writes the oracle encoder's stream byte for byte, header
included, and each decodes the other's streams to the same symbols. The
inverse transform stays FP32, so images agree with the oracle's to one
grey level.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle import intnet as I
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


@pytest.fixture(scope="module")
def codec(pw):
    c = pw.Codec(0, "int8")
    yield c
    c.close()


def _blob(C=32, seed=0, ll_mode=0, gain=1.0):
    """gain > 1 scales the context model's weights (not the heads' biases)
    so that clamps, the LeakyReLU's negative branch and the saturating
    hard sigmoid / tanh are exercised."""
    cfg = S.ModelConfig(levels=4, C=C, ll_mode=ll_mode)
    t = S.random_model(cfg, seed)
    if gain != 1.0:
        for name in list(t):
            if name.startswith(("lstm.", "sb.", "ll.")) and not name.endswith(".bh"):
                t[name] = (t[name] * gain).astype(np.float32)
    return S.pack_blob(cfg, t)


def _latent(om, img):
    planes, _ = K.colour_forward(img, False, 8)
    planes = [K.pad_plane(p, 1 << om.levels) for p in planes]
    d32 = np.float32(1.0 / 8.0)
    return [[K.quantise(s, d32) for s in om.lift.forward(p, om.levels, False)] for p in planes]


def _flat(qsb_list):
    nsb = len(qsb_list[0])
    return np.concatenate([np.stack([qc[i] for qc in qsb_list]).reshape(-1)
                           for i in range(nsb)]).astype(np.int64)


@pytest.mark.parametrize("C,H,W,gain", [(32, 80, 112, 1.0), (32, 80, 112, 4.0),
                                        (64, 512, 768, 1.0)])
def test_integer_parameters_equal_the_oracle_everywhere(codec, C, H, W, gain):
    blob = _blob(C=C, seed=1, gain=gain)
    gm = codec.load_model(blob)
    om = K.Model(blob, integer=True)
    img = S.gray_sinusoids(H, W, seed=5)
    qsb = _latent(om, img)[0]
    mu_g, sg_g = codec.context_params(gm, H, W, _flat([qsb]))
    tj = I.context_tj_all(om.int_context(), qsb)
    t_o = np.concatenate([t.reshape(-1) for t, _ in tj])
    j_o = np.concatenate([j.reshape(-1) for _, j in tj])
    t_g = np.rint(mu_g.astype(np.float64) * 16).astype(np.int64)
    j_g = ((sg_g.view(np.uint32).astype(np.int64) - 0x3E000000) >> 20)
    assert np.array_equal(t_g, t_o), int(np.sum(t_g != t_o))
    assert np.array_equal(j_g, j_o), int(np.sum(j_g != j_o))
    print(f"\nINT8 C={C} {H}x{W} gain {gain:g}: {t_o.size} positions, t and j identical; "
          f"t range [{t_o.min()}, {t_o.max()}], j range [{j_o.min()}, {j_o.max()}]")
    gm.close()


@pytest.mark.parametrize("kind,gain", [("gray", 1.0), ("rgb", 1.0), ("rgb", 4.0)])
def test_gpu_stream_equals_oracle_stream(codec, kind, gain):
    blob = _blob(seed=2, gain=gain)
    gm = codec.load_model(blob)
    img = S.gray_sinusoids(96, 128, seed=6) if kind == "gray" else S.rgb_natural(64, 96, seed=6)
    bs_g = codec.encode_image(gm, img, q=8.0, chunk=500)
    bs_o = K.encode_image(blob, img, q=8.0, chunk=500, integer=True)
    assert bs_g == bs_o, "the integer class's stream differs from the oracle's"
    # each side decodes the other's stream
    om = K.Model(blob)
    _, q_o = K.decode_symbols(om, bs_g)
    assert np.array_equal(codec.decode_symbols(gm, bs_o), _flat(q_o))
    out = codec.decode_image(gm, bs_o)
    ref = K.decode_image(blob, bs_o)
    assert np.max(np.abs(out.astype(int) - ref.astype(int))) <= 1
    gm.close()


def test_gpu_stream_equals_oracle_stream_fullsize(codec):
    """768 x 512 gray, C = 64: the GPU encoder's stream is the oracle
    encoder's, byte for byte."""
    blob = _blob(C=64, seed=0)
    gm = codec.load_model(blob)
    img = S.gray_sinusoids(512, 768, seed=3)
    bs_g = codec.encode_image(gm, img, q=8.0)
    bs_o = K.encode_image(blob, img, q=8.0, integer=True)
    assert len(bs_g) == len(bs_o) and bs_g == bs_o
    assert np.array_equal(codec.decode_symbols(gm, bs_o), codec.analyse(gm, img, q=8.0))
    print(f"\nINT8 768x512 gray: {len(bs_g)} bytes identical to the oracle's")
    gm.close()


@pytest.mark.parametrize("gain", [1.0, 4.0])
def test_integer_autoregressive_ll_equals_the_oracle(codec, gain):
    """pWave++'s default LL model (autoregressive) in integer form: the
    parameters at every position and the streams equal the oracle's."""
    blob = _blob(seed=4, ll_mode=1, gain=gain)
    gm = codec.load_model(blob)
    om = K.Model(blob, integer=True)
    img = S.gray_sinusoids(96, 128, seed=8)
    qsb = _latent(om, img)[0]
    mu_g, sg_g = codec.context_params(gm, 96, 128, _flat([qsb]))
    tj = I.context_tj_all(om.int_context(), qsb)
    t_o = np.concatenate([t.reshape(-1) for t, _ in tj])
    j_o = np.concatenate([j.reshape(-1) for _, j in tj])
    assert np.array_equal(np.rint(mu_g.astype(np.float64) * 16).astype(np.int64), t_o)
    assert np.array_equal((sg_g.view(np.uint32).astype(np.int64) - 0x3E000000) >> 20, j_o)
    bs_g = codec.encode_image(gm, img, q=8.0)
    assert bs_g == K.encode_image(blob, img, q=8.0, integer=True)
    assert np.array_equal(codec.decode_symbols(gm, bs_g), _flat([qsb]))
    gm.close()


def test_integer_class_limits(pw, codec):
    cfg = S.ModelConfig(levels=4, C=32, prob=1)
    with pytest.raises(pw.PwError) as e:            # mixture heads: no integer model
        codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 0)))
    assert e.value.code == pw.PW_EUNSUPPORTED
    blob = _blob(seed=3)
    gm = codec.load_model(blob)
    img = S.gray_sinusoids(64, 64, seed=7)
    bs = codec.encode_image(gm, img, q=8.0)
    f32 = pw.Codec(0, "fp32")
    m32 = f32.load_model(blob)
    with pytest.raises(pw.PwError) as e:            # another class's decoder refuses it
        f32.decode_image(m32, bs)
    assert e.value.code == pw.PW_EINVAL
    # the same images through the float class reconstruct identically
    # (the probability model changes only the rate)
    assert np.array_equal(f32.decode_image(m32, f32.encode_image(m32, img, q=8.0)),
                          codec.decode_image(gm, bs))
    m32.close()
    f32.close()
    gm.close()


def test_integer_class_escapes_and_lossless_equal_the_oracle(codec):
    """Large symbols: a fine quantiser (residuals beyond +-62 take the
    escape path) and a 12-bit lossless RGB image (context inputs clamped at
    +-127): the GPU's streams equal the oracle's byte for byte and the
    lossless image decodes exactly."""
    blob = _blob(seed=6)
    gm = codec.load_model(blob)
    img = S.rgb_natural(48, 80, seed=10)
    bs_g = codec.encode_image(gm, img, q=1.0 / 8.0)
    bs_o = K.encode_image(blob, img, q=1.0 / 8.0, integer=True)
    assert bs_g == bs_o
    q = codec.analyse(gm, img, q=1.0 / 8.0)
    assert np.max(np.abs(q)) > 62                     # escapes were coded
    assert np.array_equal(codec.decode_symbols(gm, bs_g), q)
    img12 = S.lossless_blobs(48, 64, seed=11)
    bs_g = codec.encode_image(gm, img12, lossless=True, bitdepth=12)
    bs_o = K.encode_image(blob, img12, lossless=True, bitdepth=12, integer=True)
    assert bs_g == bs_o
    assert np.array_equal(codec.decode_image(gm, bs_g), img12)
    gm.close()


def test_integer_class_gop_reconstructs_like_the_float_class(pw, codec):
    """A motion-compensated GOP through the INT8 class: the temporal and
    spatial transforms are the FP32 ones, so the frames decode exactly as the
    FP32 class decodes its own stream of the same GOP (the context model
    changes only the rate)."""
    bl, bh = _blob(seed=7), _blob(seed=8)
    frames = S.video_gop(48, 64, 8, seed=13)
    ml, mh = codec.load_model(bl), codec.load_model(bh)
    gs = codec.encode_gop(ml, mh, frames, q=8.0)
    out = codec.decode_gop(ml, mh, gs, 8, frames.shape[1:])
    f32 = pw.Codec(0, "fp32")
    fl, fh = f32.load_model(bl), f32.load_model(bh)
    gs32 = f32.encode_gop(fl, fh, frames, q=8.0)
    assert gs != gs32
    assert np.array_equal(out, f32.decode_gop(fl, fh, gs32, 8, frames.shape[1:]))
    for m in (ml, mh, fl, fh):
        m.close()
    f32.close()
