"""Graph replay of image decodes: after one direct run of a plan (and once
the autotuner has settled), decodes replay a captured CUDA graph of the
plan's whole device chain. The replayed chain must give exactly the
direct chain's results for every stream of the plan - each replay reads the
new streams through the plan's stream table - in every precision class, for
host and device outputs, and must still report a corrupt stream."""
import numpy as np
import pytest

import synthetic as S
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


def _blob(C=32, seed=0, prob=0):
    cfg = S.ModelConfig(levels=4, C=C, prob=prob)
    return S.pack_blob(cfg, S.random_model(cfg, seed))


def _decode_until_replayed(codec, model, streams, shape, dtype, limit=40):
    """Decode repeatedly (the autotuner may need a few runs to settle) until
    a decode came from a replayed graph; returns that decode's output."""
    start = codec.graph_replays
    for _ in range(limit):
        out = codec.decode_batch(model, streams, shape, dtype)
        if codec.graph_replays > start:
            return out
    pytest.fail("no decode was replayed from a graph")


@pytest.mark.parametrize("prec,prob", [("fp32", 0), ("bf16", 0), ("fp8", 0), ("fp32", 1)])
def test_replayed_decodes_equal_direct_decodes(pw, prec, prob):
    codec = pw.Codec(0, prec)
    model = codec.load_model(_blob(prob=prob))
    imgs = [S.rgb_natural(64, 96, seed=s) for s in (1, 2, 3, 4)]
    streams = [codec.encode_image(model, im, q=8.0, chunk=300) for im in imgs]
    shape, dtype = (64, 96, 3), np.uint8
    assert codec.set_graphs(False)                    # on by default
    ref_a = codec.decode_batch(model, streams[:2], shape, dtype)
    ref_b = codec.decode_batch(model, streams[2:], shape, dtype)
    codec.set_graphs(True)
    got_a = _decode_until_replayed(codec, model, streams[:2], shape, dtype)
    assert np.array_equal(got_a, ref_a)
    # other streams of the same plan through the same graph
    n0 = codec.graph_replays
    got_b = codec.decode_batch(model, streams[2:], shape, dtype)
    assert codec.graph_replays == n0 + 1
    assert np.array_equal(got_b, ref_b)
    assert np.array_equal(codec.decode_batch(model, streams[:2], shape, dtype), ref_a)
    model.close()
    codec.close()


def test_replayed_single_image_device_output_and_corrupt_stream(pw):
    torch = pytest.importorskip("torch")
    codec = pw.Codec(0, "fp32")
    model = codec.load_model(_blob())
    img = S.gray_sinusoids(256, 256, seed=0)
    bs = codec.encode_image(model, img, q=8.0)
    ref = codec.decode_image(model, bs)
    dev = torch.device("cuda", 0)
    d_bs = torch.from_numpy(np.frombuffer(bs, dtype=np.uint8).copy()).to(dev)
    out = torch.empty((256, 256), dtype=torch.uint8, device=dev)
    start = codec.graph_replays
    for _ in range(5):
        out.zero_()
        codec.decode_batch_device(model, [d_bs.data_ptr()], [len(bs)], out.data_ptr(), (256, 256))
        assert np.array_equal(out.cpu().numpy(), ref)
    assert codec.graph_replays > start
    bad = bytearray(bs)
    bad[len(bs) // 2] ^= 0x5A                         # payload byte
    with pytest.raises(pw.PwError) as e:
        codec.decode_image(model, bytes(bad))
    assert e.value.code == pw.PW_ECORRUPT
    assert np.array_equal(codec.decode_image(model, bs), ref)
    model.close()
    codec.close()


def test_page_locked_host_buffers_decode_like_pageable(pw):
    """Streams and images in page-locked host memory take the direct copy
    path; the results equal the pageable path's."""
    torch = pytest.importorskip("torch")
    codec = pw.Codec(0, "fp8")
    model = codec.load_model(_blob(C=64))
    imgs = [S.rgb_natural(64, 96, seed=s) for s in (5, 6, 7)]
    streams = [codec.encode_image(model, im, q=8.0) for im in imgs]
    ref = codec.decode_batch(model, streams, (64, 96, 3), np.uint8)
    offs = np.cumsum([0] + [(len(b) + 255) // 256 * 256 for b in streams])
    host = np.zeros(int(offs[-1]), dtype=np.uint8)
    for i, b in enumerate(streams):
        host[offs[i]:offs[i] + len(b)] = np.frombuffer(b, dtype=np.uint8)
    h_in = torch.from_numpy(host).pin_memory()
    h_out = torch.zeros((3, 64, 96, 3), dtype=torch.uint8).pin_memory()
    ptrs = [h_in.data_ptr() + int(offs[i]) for i in range(3)]
    for _ in range(3):                               # direct, then graph replays
        h_out.zero_()
        codec.decode_batch_host_ptrs(model, ptrs, [len(b) for b in streams], h_out.data_ptr(),
                                     (64, 96, 3))
        assert np.array_equal(h_out.numpy(), ref)
    model.close()
    codec.close()
