"""Motion-compensated temporal lifting (Section 3.3) against the oracle.

* Block motion search: the library's vectors equal the oracle's full-search
  definition exactly (integer SAD on the integer luma, same tie rule), on a
  GOP of the video workload's kind and on a panning GOP whose motion is
  known.
* MC temporal lifting with given vectors: forward bands and inverse frames
  within 2e-3 of the FP64 oracle (FP32 CNNs over samples of +-128), and
  perfect reconstruction.
* GOP codec: the library's version-2 container carries exactly the oracle's
  vectors for the same frames, its decode's PSNR is within 0.01 dB of the
  oracle's own round trip, and version-1 (zero-motion) containers written by
  the oracle still decode to within one grey level of the oracle's decode.
"""
import struct

import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle import lifting as LF
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


@pytest.fixture(scope="module")
def codec(pw):
    c = pw.Codec(0, "fp32")
    yield c
    c.close()


def _blob(seed, C=32):
    cfg = S.ModelConfig(levels=4, C=C, ll_mode=0)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


def _psnr(a, b):
    return 10 * np.log10(255.0 ** 2 / np.mean((a.astype(float) - b.astype(float)) ** 2))


@pytest.mark.parametrize("kind", ["video", "panning"])
def test_motion_search_equals_oracle(codec, kind):
    if kind == "video":
        frames = S.video_gop(64, 96, 8, seed=11)
    else:
        canvas = S.rgb_natural(160, 200, seed=12)
        frames = np.stack([canvas[40 + 3 * k:104 + 3 * k, 60 - 2 * k:156 - 2 * k]
                           for k in range(8)])
    luma = np.stack([K.pad_plane(LF.gop_luma(f), 16) for f in frames])
    want = LF.gop_motion(list(luma), 3)
    got = codec.motion_search(luma)
    for f in range(7):
        assert np.array_equal(got[f].astype(np.int64), want[f]), f
    if kind == "panning":
        assert np.all(got[0][1:-1, 1:-1] == (3, -2))
        assert np.all(got[6][1:-1, 1:-1] == (12, -8))   # level 3: frames 0 and 4


def test_mc_temporal_lifting_matches_oracle(codec):
    blob = _blob(2)
    gm, om = codec.load_model(blob), K.Model(blob)
    rng = np.random.default_rng(13)
    frames = rng.uniform(-128, 127, (8, 48, 80))
    mvs = [rng.integers(-16, 17, (3, 5, 2)) for _ in range(7)]
    mv8 = np.stack(mvs).astype(np.int8)
    bands = LF.temporal_forward(list(frames), om.tensors, 3, mvs)
    got = codec.temporal_lift_mc(gm, frames.astype(np.float32), mv8, forward=True)
    assert np.max(np.abs(got - np.stack(bands))) < 2e-3
    back = codec.temporal_lift_mc(gm, np.stack(bands).astype(np.float32), mv8, forward=False)
    ref = LF.temporal_inverse(bands, om.tensors, 3, mvs)
    assert np.max(np.abs(back - np.stack(ref))) < 2e-3
    assert np.max(np.abs(back - frames)) < 2e-3
    gm.close()


def test_gop_stream_vectors_and_psnr_match_oracle(codec):
    bl, bh = _blob(2), _blob(3)
    ml, mh = codec.load_model(bl), codec.load_model(bh)
    frames = S.video_gop(40, 56, 8, seed=7)
    gs = codec.encode_gop(ml, mh, frames, q=8.0)
    ver = struct.unpack_from("<H", gs, 4)[0]
    assert ver == 2
    luma = [K.pad_plane(LF.gop_luma(f), 16) for f in frames]
    want = b"".join(np.asarray(v, dtype=np.int8).tobytes() for v in LF.gop_motion(luma, 3))
    assert gs[36:36 + len(want)] == want
    out = codec.decode_gop(ml, mh, gs, 8, frames.shape[1:])
    ref = K.decode_gop(bl, bh, K.encode_gop(bl, bh, frames, q=8.0))
    assert abs(_psnr(out, frames) - _psnr(ref, frames)) < 0.01
    fine = codec.decode_gop(ml, mh, codec.encode_gop(ml, mh, frames, q=1 / 32.0), 8,
                            frames.shape[1:])
    assert np.max(np.abs(fine.astype(int) - frames.astype(int))) <= 1
    ml.close()
    mh.close()


def test_version1_zero_motion_gop_still_decodes(codec):
    bl, bh = _blob(2), _blob(3)
    ml, mh = codec.load_model(bl), codec.load_model(bh)
    frames = S.video_gop(32, 48, 8, seed=9)
    gs = K.encode_gop(bl, bh, frames, q=1 / 16.0, motion=False)
    out = codec.decode_gop(ml, mh, gs, 8, frames.shape[1:])
    ref = K.decode_gop(bl, bh, gs)
    assert np.max(np.abs(out.astype(int) - ref.astype(int))) <= 1
    ml.close()
    mh.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_gop_in_tensor_core_classes_close_to_fp32(pw, prec):
    """The tensor-core classes' GOP decode (their temporal inverse lifting
    runs the CNNs' middle layers on the tensor cores) reconstructs within
    0.05 dB of the FP32 class's PSNR on the same GOP."""
    frames = S.video_gop(48, 64, 8, seed=21)
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0)
    bl, bh = (S.pack_blob(cfg, S.random_model(cfg, s)) for s in (31, 32))
    ps = {}
    for p in ("fp32", prec):
        c = pw.Codec(0, p)
        ml, mh = c.load_model(bl), c.load_model(bh)
        gs = c.encode_gop(ml, mh, frames, q=8.0)
        ps[p] = _psnr(c.decode_gop(ml, mh, gs, 8, frames.shape[1:]), frames)
        ml.close()
        mh.close()
        c.close()
    assert abs(ps[prec] - ps["fp32"]) < 0.05, ps
