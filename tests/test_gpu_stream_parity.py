"""Stream-level parity of the tensor-core precision classes with the oracle's
coder, by index injection, at the benchmark's full image size (768x512,
C = 64 four-step context model).

The BF16 and FP8 classes compute the entropy parameters (mu, sigma) of
Section 3.2 with reduced-precision convolutions, so their table indices can
differ from the FP64 oracle's wherever a value lies near a decision boundary;
what the coder then does with the indices is integer work and must be exact.
So the GPU's own parameters are handed to the oracle (pw_context_params on
the GPU-decoded latent, the same kernels and class as the encoder), and:

* the oracle's encoder, coding the GPU's quantised latent with those
  parameters, writes a stream identical byte for byte to the GPU's
  (offset table and payload; header equal except the precision-class bits
  that only the library records);
* the oracle's decoder, given the same parameters, decodes the GPU's stream
  to exactly the GPU's symbols.

Cases cover both classes, gray and RGB, and the four quantiser steps of the
batched workload (4, 8, 16, 32).
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle.lifting import subband_shapes
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu

H, W = 512, 768


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


@pytest.fixture(scope="module")
def blob():
    cfg = S.ModelConfig(levels=4, C=64, F=16, ll_mode=0)
    return S.pack_blob(cfg, S.random_model(cfg, 0))


def _qcomp(flat, nc, shapes):
    """Library latent (subband-major, components stacked) -> per-component
    subband lists."""
    out, o = [[] for _ in range(nc)], 0
    for h, w, _ in shapes:
        blk = flat[o:o + nc * h * w].reshape(nc, h, w)
        o += nc * h * w
        for c in range(nc):
            out[c].append(blk[c].astype(np.int64))
    assert o == flat.size
    return out


def _gpu_params(codec, model, qsb, shapes):
    """(mu, sigma) per subband of one component from pw_context_params."""
    flat = np.concatenate([q.reshape(-1) for q in qsb]).astype(np.int32)
    mu, sg = codec.context_params(model, H, W, flat)
    out, o = [], 0
    for h, w, _ in shapes:
        out.append((mu[o:o + h * w].reshape(h, w).astype(np.float64),
                    sg[o:o + h * w].reshape(h, w).astype(np.float64)))
        o += h * w
    return out


@pytest.mark.parametrize("prec,kind,q,ls", [("fp8", "rgb", 4.0, 7), ("bf16", "rgb", 8.0, 7),
                                            ("fp8", "gray", 16.0, 7), ("bf16", "gray", 32.0, 7),
                                            ("fp8", "rgb", 8.0, 5)])
def test_index_injection_stream_identical(pw, blob, prec, kind, q, ls):
    """ls: log2 of the symbols per interleaved rANS state (7 = default)."""
    img = (S.rgb_natural(H, W, seed=1) if kind == "rgb" else
           S.gray_sinusoids(H, W, seed=3))
    nc = 3 if kind == "rgb" else 1
    codec = pw.Codec(0, prec)
    codec.set_lane_rule(ls)
    model = codec.load_model(blob)
    bs = codec.encode_image(model, img, q=q)
    shapes = subband_shapes(H, W, 4)
    sym = codec.decode_symbols(model, bs)
    assert np.array_equal(sym, codec.analyse(model, img, q=q))
    qcomp = _qcomp(sym, nc, shapes)
    params = [_gpu_params(codec, model, qcomp[c], shapes) for c in range(nc)]
    model.close()
    codec.close()

    om = K.Model(blob)
    hd = K.parse_header(bs)
    assert hd["lane_shift"] == ls
    ref = K.encode_symbols_with_params(om, qcomp, params, width=W, height=H, bitdepth=8,
                                       colour=hd["colour"], q=q, chunk=hd["chunk"],
                                       lane_shift=ls)
    assert len(ref) == len(bs), (len(ref), len(bs))
    head_gpu = bytearray(bs[:64])
    head_gpu[6] &= ~0x0C & 0xFF                       # precision-class bits (2-3)
    assert bytes(head_gpu) == ref[:64]
    assert bs[64:] == ref[64:], "payload or offset table differs"

    _, dec = K.decode_symbols(om, bs, params=params)
    for c in range(nc):
        for i in range(len(shapes)):
            assert np.array_equal(dec[c][i], qcomp[c][i]), (c, i)
    print(f"\n{prec} {kind} q={q:g} lane shift {ls}: {len(bs)} bytes, {hd['n_chunks']} chunks, "
          f"byte-identical to the oracle coder")
