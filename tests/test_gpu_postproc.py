"""Post-processing after the inverse transform (Section 3.1) against the
oracle: a model whose weight blob carries a post-processing CNN decodes, in
the FP32 class, to within one grey level of the oracle's decode (PSNR within
0.01 dB); in the BF16 class (its middle layers on the tensor cores) to
within one grey level at under 2 % of the samples; lossless streams skip it
and stay exact."""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


def _psnr(a, b):
    return 10 * np.log10(255.0 ** 2 / np.mean((a.astype(float) - b.astype(float)) ** 2))


def _blob(levels=4, seed=6):
    cfg = S.ModelConfig(levels=levels, C=32, post=1)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_post_processed_decode_matches_oracle(pw, prec):
    blob = _blob()
    codec = pw.Codec(0, prec)
    gm = codec.load_model(blob)
    img = S.rgb_natural(64, 96, seed=21)
    bs = codec.encode_image(gm, img, q=8.0)
    out = codec.decode_image(gm, bs)
    om = K.Model(blob)
    hd = K.parse_header(bs)
    sym = codec.decode_symbols(gm, bs)
    from oracle.lifting import subband_shapes
    qcomp, o = [[], [], []], 0
    for h, w, _ in subband_shapes(64, 96, 4):
        blk = sym[o:o + 3 * h * w].reshape(3, h, w).astype(np.int64)
        o += 3 * h * w
        for c in range(3):
            qcomp[c].append(blk[c])
    planes = K.post_process(om, hd, K.reconstruct_planes(om, hd, qcomp))
    ref = K.to_samples(K.colour_inverse(planes, hd["colour"], 8), 8)
    d = np.abs(out.astype(int) - ref.astype(int))
    if prec == "fp32":
        assert d.max() <= 1 and abs(_psnr(out, img) - _psnr(ref, img)) < 0.01
    else:
        assert d.max() <= 1 and np.mean(d > 0) < 0.02
    gm.close()
    codec.close()


def test_lossless_stream_of_a_post_model_stays_exact(pw):
    blob = _blob(levels=5, seed=7)
    codec = pw.Codec(0, "fp32")
    gm = codec.load_model(blob)
    img = S.lossless_blobs(64, 96, seed=22)
    out = codec.decode_image(gm, codec.encode_image(gm, img, lossless=True, bitdepth=12))
    assert np.array_equal(out, img)
    gm.close()
    codec.close()
