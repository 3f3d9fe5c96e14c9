"""Ragged batches: streams of one format whose image sizes differ, decoded in
one pw_decode_batch call on a canvas of the largest padded size (every
convolution, coder pass and lifting step covers all of them in one launch).

Bar: bit-identical to decoding every stream alone, in every precision class,
for both LL models, lossless 12-bit streams (also equal to the input), a
post-processing model, and the logistic-mixture model (decoded one batch per
size); a corrupt stream in a ragged batch is reported and streams of
different formats are refused.
"""
import numpy as np
import pytest

import synthetic as S
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

# (H, W): multiples of 16 and not, taller and wider than the rest, and one
# whose level-4 subbands are smaller than the canvas's compact-head minimum
SIZES = [(64, 96), (48, 80), (96, 64), (37, 53), (112, 128), (64, 96)]


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


def _blob(C=32, seed=0, ll_mode=0, prob=0, post=0, levels=4):
    cfg = S.ModelConfig(levels=levels, C=C, ll_mode=ll_mode, prob=prob, post=post)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


def _imgs(rgb, sizes=SIZES, seed=0):
    if rgb:
        return [S.rgb_natural(h, w, seed=seed + i) for i, (h, w) in enumerate(sizes)]
    return [S.gray_sinusoids(h, w, seed=seed + i) for i, (h, w) in enumerate(sizes)]


def _check(codec, model, streams):
    alone = [codec.decode_image(model, bs) for bs in streams]
    got = codec.decode_ragged(model, streams)
    for i, (a, g) in enumerate(zip(alone, got)):
        assert g.shape == a.shape, i
        assert np.array_equal(a, g), f"stream {i} ({a.shape}) differs from its single decode"
    # twice: the plan's tables are rebuilt per call
    got2 = codec.decode_ragged(model, streams[::-1])
    for a, g in zip(alone[::-1], got2):
        assert np.array_equal(a, g)
    return alone


@pytest.mark.parametrize("prec,C", [("fp32", 32), ("int8", 32), ("bf16", 32), ("fp8", 32),
                                    ("fp8", 64)])
@pytest.mark.parametrize("rgb", [False, True])
def test_ragged_batch_equals_single_decodes(pw, prec, C, rgb):
    codec = pw.Codec(0, prec)
    model = codec.load_model(_blob(C=C, seed=1))
    qs = [4.0, 8.0, 16.0, 32.0, 8.0, 2.0]
    streams = [codec.encode_image(model, im, q=q) for im, q in zip(_imgs(rgb, seed=3), qs)]
    _check(codec, model, streams)
    model.close()
    codec.close()


@pytest.mark.parametrize("prec", ["fp32", "fp8", "int8"])
def test_ragged_autoregressive_ll(pw, prec):
    codec = pw.Codec(0, prec)
    model = codec.load_model(_blob(seed=2, ll_mode=1))
    streams = [codec.encode_image(model, im, q=8.0) for im in _imgs(True, seed=5)]
    _check(codec, model, streams)
    model.close()
    codec.close()


def test_ragged_lossless_12bit_exact(pw):
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(seed=4, levels=5))
    sizes = [(96, 160), (64, 64), (130, 100), (32, 200)]
    imgs = [S.lossless_blobs(h, w, seed=20 + i) for i, (h, w) in enumerate(sizes)]
    streams = [codec.encode_image(model, im, lossless=True, bitdepth=12) for im in imgs]
    got = codec.decode_ragged(model, streams)
    for im, g in zip(imgs, got):
        assert np.array_equal(im, g)
    _check(codec, model, streams)
    model.close()
    codec.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ragged_post_processing_model(pw, prec):
    codec = pw.Codec(0, prec)
    model = codec.load_model(_blob(seed=6, post=1))
    streams = [codec.encode_image(model, im, q=8.0) for im in _imgs(True, seed=9)]
    _check(codec, model, streams)
    model.close()
    codec.close()


def test_ragged_mixture_model_one_batch_per_size(pw):
    codec = pw.Codec(0, "fp32")
    model = codec.load_model(_blob(seed=7, prob=1))
    streams = [codec.encode_image(model, im, q=8.0) for im in _imgs(False, seed=11)]
    _check(codec, model, streams)
    model.close()
    codec.close()


def test_ragged_larger_sizes_fp8(pw):
    """Several tiles per plane in every convolution and lifting step."""
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(C=64, seed=8))
    sizes = [(256, 384), (200, 300), (320, 240), (512, 512)]
    streams = [codec.encode_image(model, im, q=8.0) for im in _imgs(True, sizes, seed=13)]
    _check(codec, model, streams)
    model.close()
    codec.close()


def test_ragged_corrupt_stream_and_mixed_formats(pw):
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(seed=9))
    streams = [codec.encode_image(model, im, q=8.0) for im in _imgs(True, seed=15)]
    bad = bytearray(streams[2])
    bad[len(bad) - 40] ^= 0x5A                      # a payload byte
    with pytest.raises(pw.PwError) as e:
        codec.decode_ragged(model, streams[:2] + [bytes(bad)] + streams[3:])
    assert e.value.code == pw.PW_ECORRUPT
    gray = codec.encode_image(model, S.gray_sinusoids(48, 64, seed=1), q=8.0)
    with pytest.raises(pw.PwError) as e:
        codec.decode_ragged(model, streams[:2] + [gray])
    assert e.value.code == pw.PW_EINVAL
    # the context still decodes afterwards
    _check(codec, model, streams)
    model.close()
    codec.close()


def test_decode_image_allocates_when_no_buffer(pw):
    """pw_decode_image with out->data == NULL allocates the image itself."""
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(seed=10))
    for img in (S.rgb_natural(40, 72, seed=2), S.gray_sinusoids(33, 50, seed=3)):
        bs = codec.encode_image(model, img, q=8.0)
        got = codec.decode_image_alloc(model, bs)
        assert got.shape == img.shape and got.dtype == img.dtype
        assert np.array_equal(got, codec.decode_image(model, bs))
    img12 = S.lossless_blobs(48, 64, seed=4)
    bs = codec.encode_image(model, img12, lossless=True, bitdepth=12)
    assert np.array_equal(codec.decode_image_alloc(model, bs), img12)
    model.close()
    codec.close()


def test_batch_plane_limit(pw):
    """More than 65535 planes (images x components) in one call are refused
    before any device work."""
    codec = pw.Codec(0, "fp32")
    model = codec.load_model(_blob(seed=11))
    bs = codec.encode_image(model, S.rgb_natural(16, 16, seed=1), q=8.0)
    n = 65535 // 3 + 1
    with pytest.raises(pw.PwError) as e:
        codec.decode_batch(model, [bs] * n)
    assert e.value.code == pw.PW_EUNSUPPORTED
    assert np.array_equal(codec.decode_batch(model, [bs] * 4)[3], codec.decode_image(model, bs))
    model.close()
    codec.close()


@pytest.mark.parametrize("prec", ["fp8", "fp32"])
def test_ragged_device_streams_and_images(pw, prec):
    """Device-resident streams of different sizes into device images in one
    call; equal sizes still take the plain batch path."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    codec = pw.Codec(0, prec)
    model = codec.load_model(_blob(seed=12))
    imgs = _imgs(True, seed=21)
    streams = [codec.encode_image(model, im, q=8.0) for im in imgs]
    d_bs = [torch.from_numpy(np.frombuffer(b, dtype=np.uint8).copy()).to(dev) for b in streams]
    outs = [torch.zeros(im.shape, dtype=torch.uint8, device=dev) for im in imgs]
    for _ in range(2):
        codec.decode_ragged_device(model, [t.data_ptr() for t in d_bs], [len(b) for b in streams],
                                   [o.data_ptr() for o in outs], [im.shape for im in imgs])
        for o, bs in zip(outs, streams):
            assert np.array_equal(o.cpu().numpy(), codec.decode_image(model, bs))
    same = [streams[0], streams[5]]                    # both 64 x 96
    o2 = torch.zeros((2,) + imgs[0].shape, dtype=torch.uint8, device=dev)
    codec.decode_batch_device(model, [d_bs[0].data_ptr(), d_bs[5].data_ptr()],
                              [len(b) for b in same], o2.data_ptr(), imgs[0].shape)
    assert np.array_equal(o2[1].cpu().numpy(), codec.decode_image(model, streams[5]))
    model.close()
    codec.close()


def test_ragged_fast_coder_format(pw):
    """Streams in the coder's fast format (one rANS state per 32 symbols,
    6144-symbol chunks, recorded in their headers) form ragged batches too."""
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(C=64, seed=13))
    codec.set_lane_rule(5)
    sizes = [(96, 128), (80, 144), (112, 96), (64, 64)]
    streams = [codec.encode_image(model, im, q=8.0, chunk=6144)
               for im in _imgs(True, sizes, seed=31)]
    _check(codec, model, streams)
    model.close()
    codec.close()
