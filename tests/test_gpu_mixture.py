"""GPU parity of the logistic-mixture (K = 3) probability model against the
oracle (FP32 precision class, four-step LL).

Bars:
* tables are integer results of a fixed FP32 operation sequence: the
  library's tables of any key are byte-identical to the oracle's;
* the mixture parameters (w, mu, sigma) of the FP32 context model are within
  1e-3 relative of the oracle's FP64 ones (absolute floor 1e-3), and the
  decisions taken on them agree except at certified near-ties (an oracle
  value within 1e-5 relative of a decision boundary), counted and printed;
* what the coder does with the decisions is exact: fed the GPU's own
  parameters (index injection), the oracle's encoder writes the GPU's stream
  byte for byte and its decoder returns the GPU's symbols, at the
  single-image size of the benchmark (768 x 512 gray, C = 64);
* round trips are exact and the GPU decodes the oracle's streams.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle import entropy as E
from oracle.lifting import subband_shapes
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

TIE_EPS = 1e-5


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


def _blob(C=32, levels=4, seed=0, prob=1):
    cfg = S.ModelConfig(levels=levels, C=C, prob=prob)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


@pytest.fixture(scope="module")
def mix32(codec):
    blob = _blob()
    gm = codec.load_model(blob)
    yield blob, gm, K.Model(blob)
    gm.close()


def _latent(om, img):
    planes, _ = K.colour_forward(img, False, 8)
    planes = [K.pad_plane(p, 1 << om.levels) for p in planes]
    d32 = np.float32(1.0 / 8.0)
    return [[K.quantise(s, d32) for s in om.lift.forward(p, om.levels, False)] for p in planes]


def _flat(qsb_list):
    nsb = len(qsb_list[0])
    return np.concatenate([np.stack([qc[i] for qc in qsb_list]).reshape(-1)
                           for i in range(nsb)]).astype(np.int64)


def _decisions(par):
    ctr, q, j, g = E.mix_decision(par)
    return np.concatenate([ctr[:, None], q, j, g], axis=1)


def test_mix_tables_bit_exact(codec):
    rng = np.random.default_rng(0)
    n = 3000
    keys = np.concatenate([rng.integers(-255, 256, (n, 3)), rng.integers(0, 128, (n, 3)),
                           rng.integers(-31, 1, (n, 3))], axis=1)
    # extremes: narrowest / widest scales, far offsets, negligible weights
    ext = np.array([[0, 0, 0, 0, 0, 0, 0, 0, 0],
                    [255, -255, 0, 127, 127, 127, 0, -31, -31],
                    [-255, -255, -255, 0, 127, 64, -31, -31, 0],
                    [8, 16, 24, 0, 0, 0, 0, 0, 0],
                    [1, -1, 0, 127, 0, 1, -1, -2, 0]])
    keys = np.concatenate([keys, ext])
    got = codec.mix_tables(keys)
    ref = E.mix_tables(keys[:, 0:3], keys[:, 3:6], keys[:, 6:9])
    assert got.shape == ref.shape
    assert np.array_equal(got.astype(np.int64), ref.astype(np.int64)), \
        int(np.sum(np.any(got.astype(np.int64) != ref, axis=1)))


def test_mixture_params_match_oracle(codec, mix32):
    blob, gm, om = mix32
    assert gm.mixture
    img = S.gray_sinusoids(80, 112, seed=5)
    qsb = _latent(om, img)[0]
    par_g = codec.context_mixture(gm, 80, 112, _flat([qsb])).astype(np.float64)
    par_o = np.concatenate([p.reshape(-1, 9) for p in K.context_params_all(om, qsb)])
    assert np.all(np.abs(par_g - par_o) <= 1e-3 * np.maximum(np.abs(par_o), 1.0))
    diff = np.any(_decisions(par_g) != _decisions(par_o), axis=1)
    ties = E.mix_near_tie(par_o, TIE_EPS)
    print(f"\nmixture decisions differing from the oracle: {int(diff.sum())} of {diff.size}; "
          f"near-ties at {TIE_EPS:g}: {int(ties.sum())}")
    assert not np.any(diff & ~ties), int(np.sum(diff & ~ties))


@pytest.mark.parametrize("rgb", [False, True])
def test_mixture_roundtrip_symbols_exact(codec, mix32, rgb):
    blob, gm, om = mix32
    img = S.rgb_natural(72, 104, seed=7) if rgb else S.gray_sinusoids(72, 104, seed=7)
    bs = codec.encode_image(gm, img, q=8.0, chunk=200)
    assert K.parse_header(bs)["mixture"]
    assert np.array_equal(codec.decode_symbols(gm, bs), codec.analyse(gm, img, q=8.0))


def test_mixture_changes_only_the_rate(codec, mix32):
    """Laplace and mixture models with the same lifting weights (drawn first,
    equal for the same seed) reconstruct the same image; the streams differ."""
    blob, gm, om = mix32
    lap = codec.load_model(_blob(prob=0))
    img = S.rgb_natural(64, 96, seed=9)
    bm, bl = codec.encode_image(gm, img, q=8.0), codec.encode_image(lap, img, q=8.0)
    assert bm != bl
    assert np.array_equal(codec.decode_image(gm, bm), codec.decode_image(lap, bl))
    lap.close()


def test_mixture_decodes_oracle_stream(codec, mix32):
    """A stream of the oracle encoder decodes exactly on the GPU whenever the
    GPU's decisions on the oracle's latent equal the oracle's (differences
    may sit only at certified near-ties)."""
    blob, gm, om = mix32
    img = S.gray_sinusoids(48, 64, seed=8)
    bs = K.encode_image(blob, img, q=8.0, chunk=256)
    qsb = _latent(om, img)[0]
    par_o = np.concatenate([p.reshape(-1, 9) for p in K.context_params_all(om, qsb)])
    par_g = codec.context_mixture(gm, 48, 64, _flat([qsb])).astype(np.float64)
    diff = np.any(_decisions(par_g) != _decisions(par_o), axis=1)
    assert not np.any(diff & ~E.mix_near_tie(par_o, TIE_EPS))
    if np.any(diff):
        pytest.skip(f"{int(diff.sum())} certified near-tie decision differences in this input")
    assert np.array_equal(codec.decode_symbols(gm, bs), _flat([qsb]))
    out = codec.decode_image(gm, bs)
    ref = K.decode_image(blob, bs)
    assert np.max(np.abs(out.astype(int) - ref.astype(int))) <= 1


def test_mixture_index_injection_stream_identical_fullsize(codec):
    """768 x 512 gray, C = 64 (the single-image workload's model size): the
    oracle's coder, given the GPU's mixture parameters, writes the GPU's
    stream byte for byte and decodes it to the GPU's symbols."""
    H, W = 512, 768
    blob = _blob(C=64, seed=2)
    gm = codec.load_model(blob)
    img = S.gray_sinusoids(H, W, seed=3)
    bs = codec.encode_image(gm, img, q=8.0)
    sym = codec.decode_symbols(gm, bs)
    assert np.array_equal(sym, codec.analyse(gm, img, q=8.0))
    par = codec.context_mixture(gm, H, W, sym).astype(np.float64)
    gm.close()
    shapes = subband_shapes(H, W, 4)
    qsb, params, o = [], [], 0
    for h, w, _ in shapes:
        qsb.append(sym[o:o + h * w].reshape(h, w).astype(np.int64))
        params.append(par[o:o + h * w].reshape(h, w, 9))
        o += h * w
    om = K.Model(blob)
    hd = K.parse_header(bs)
    ref = K.encode_symbols_with_params(om, [qsb], [params], width=W, height=H, bitdepth=8,
                                       colour=hd["colour"], q=8.0, chunk=hd["chunk"])
    assert len(ref) == len(bs)
    head_gpu = bytearray(bs[:64])
    head_gpu[6] &= ~0x0C & 0xFF                       # precision-class bits (2-3)
    assert bytes(head_gpu) == ref[:64]
    assert bs[64:] == ref[64:], "payload or offset table differs"
    _, dec = K.decode_symbols(om, bs, params=[params])
    for i in range(len(shapes)):
        assert np.array_equal(dec[0][i], qsb[i]), i
    print(f"\nmixture 768x512 gray: {len(bs)} bytes, {hd['n_chunks']} chunks, "
          f"byte-identical to the oracle coder")


def test_mixture_model_limits(codec, pw, mix32):
    blob, gm, om = mix32
    with pytest.raises(pw.PwError) as e:                # Laplace parameters only
        codec.context_params(gm, 48, 64, np.zeros(48 * 64, dtype=np.int32))
    assert e.value.code == pw.PW_EUNSUPPORTED
    c16 = pw.Codec(0, "bf16")
    with pytest.raises(pw.PwError) as e:                # FP32 precision class only
        c16.load_model(blob)
    assert e.value.code == pw.PW_EUNSUPPORTED
    c16.close()


def test_mixture_escapes_round_trip_and_decode_oracle_stream(codec, mix32):
    """A fine quantiser: residuals beyond +-62 are coded through the mixture
    tables' escape symbols; GPU round trip exact, and the oracle's stream
    decodes on the GPU whenever the decisions match."""
    blob, gm, om = mix32
    img = S.rgb_natural(40, 64, seed=12)
    bs = codec.encode_image(gm, img, q=1.0 / 8.0)
    q = codec.analyse(gm, img, q=1.0 / 8.0)
    assert np.max(np.abs(q)) > 62
    assert np.array_equal(codec.decode_symbols(gm, bs), q)
    bs_o = K.encode_image(blob, img, q=1.0 / 8.0)
    planes, _ = K.colour_forward(img, False, 8)
    d32 = np.float32(8.0)
    qo = [[K.quantise(s, d32) for s in om.lift.forward(K.pad_plane(p, 16), om.levels, False)]
          for p in planes]
    diff = False
    for c in range(3):
        par_o = np.concatenate([p.reshape(-1, 9) for p in K.context_params_all(om, qo[c])])
        par_g = codec.context_mixture(gm, 48, 64, _flat([qo[c]])).astype(np.float64)
        d = np.any(_decisions(par_g) != _decisions(par_o), axis=1)
        assert not np.any(d & ~E.mix_near_tie(par_o, TIE_EPS))
        diff = diff or bool(np.any(d))
    if diff:
        pytest.skip("certified near-tie decision differences in this input")
    assert np.array_equal(codec.decode_symbols(gm, bs_o), _flat(qo))
