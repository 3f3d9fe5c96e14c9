"""pw_model_random_blob (host only, no GPU): the library's own random-init
model is a valid weight blob of the architecture. The oracle's blob reader
parses it; its tensors have the names and shapes of the architecture spec
(the seeded-input module's tensor_specs), lie inside their init bounds, are
deterministic in the seed, and the oracle codec round-trips an image with it.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import blob as OB
from oracle import codec as K
from tests._lib import ensure_built


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


@pytest.mark.parametrize("levels,C,ll_mode", [(4, 32, 0), (4, 64, 1), (5, 128, 0)])
def test_blob_has_the_architecture(pw, levels, C, ll_mode):
    blob = pw.random_model_blob(levels, C, 16, ll_mode, seed=7)
    assert len(blob) % 256 == 0
    cfg, tensors = OB.read_blob(blob)
    assert cfg == dict(levels=levels, C=C, F=16, ll_mode=ll_mode)
    mc = S.ModelConfig(levels=levels, C=C, F=16, ll_mode=ll_mode)
    specs = S.tensor_specs(mc)
    assert list(tensors) == [n for n, _ in specs]
    for name, shape in specs:
        t = tensors[name]
        assert t.shape == tuple(shape), name
        if name.endswith(".bh"):
            np.testing.assert_allclose(t, [0.0, np.log(np.expm1(1.5))], rtol=1e-6)
            continue
        b = S.weights._init_scale(name, shape, mc)
        assert np.all(np.abs(t) <= b * (1 + 1e-6)), name
        if t.size >= 64:
            # a uniform draw over +-b: spread over the range, mean near zero
            assert t.max() > 0.5 * b and t.min() < -0.5 * b, name
            assert abs(t.mean()) < 0.2 * b, name


def test_blob_is_deterministic_in_the_seed(pw):
    a = pw.random_model_blob(4, 32, 16, 0, seed=1)
    assert a == pw.random_model_blob(4, 32, 16, 0, seed=1)
    b = pw.random_model_blob(4, 32, 16, 0, seed=2)
    assert len(a) == len(b) and a != b
    assert OB.model_hash(a) != OB.model_hash(b)


def test_unsupported_configuration_is_refused(pw):
    for bad in [(0, 32, 16, 0), (4, 48, 16, 0), (4, 32, 8, 0), (4, 32, 16, 2)]:
        with pytest.raises(pw.PwError):
            pw.random_model_blob(*bad, seed=0)


def test_oracle_codec_round_trips_with_the_blob(pw):
    blob = pw.random_model_blob(4, 32, 16, 0, seed=5)
    img = S.rgb_natural(32, 48, seed=3)
    # a fine quantiser step (q = 1/64): the lossy round trip is nearly exact
    bs = K.encode_image(blob, img, q=1.0 / 64.0)
    out = K.decode_image(blob, bs)
    assert out.shape == img.shape
    assert np.max(np.abs(out.astype(int) - img.astype(int))) <= 1
    # the stream is bound to this blob (the model hash in its header)
    hd = K.parse_header(bs)
    assert hd["model_hash"] == OB.model_hash(blob)


@pytest.mark.gpu
def test_init_random_model_is_the_blob_model(pw):
    """pw_model_init_random loads the model of pw_model_random_blob (same
    hash), and a GPU round trip with it returns the encoder's symbols."""
    codec = pw.Codec(0, "fp32")
    m = codec.init_random_model(4, 32, 16, 0, seed=5)
    assert m.hash == OB.model_hash(pw.random_model_blob(4, 32, 16, 0, seed=5))
    img = S.rgb_natural(32, 48, seed=3)
    bs = codec.encode_image(m, img, q=8.0)
    assert np.array_equal(codec.decode_symbols(m, bs), codec.analyse(m, img, q=8.0))
    m.close()
    codec.close()
