"""Decode server (pw_server_*): every served result is bit-identical to the
same stream decoded alone with pw_decode_image, for a mix of sizes, colour
formats and quantiser steps decoded concurrently on several lanes, with and
without a tight device-memory budget; admission errors and statistics.
"""
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


def _requests(n, seed):
    """A small mixed request set: sizes, gray/RGB and q like the serving
    workload (Poisson stream), scaled down so the test stays short."""
    reqs = S.request_stream(n=n, rate=200.0, seed=seed, lo=48, hi=224)
    imgs = []
    for r in reqs:
        if r["c"] == 1:
            imgs.append(S.gray_sinusoids(r["h"], r["w"], seed=r["seed"] % 1000))
        else:
            imgs.append(S.rgb_natural(r["h"], r["w"], seed=r["seed"] % 1000))
    return reqs, imgs


@pytest.mark.parametrize("prec,prob", [("fp32", 0), ("bf16", 0), ("fp8", 0), ("int8", 0),
                                       ("fp32", 1)])
def test_server_results_identical_to_single_decode(pw, prec, prob):
    """prob = 1: the logistic-mixture model (FP32); int8: the integer-network
    class."""
    codec = pw.Codec(0, prec)
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0, prob=prob)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 11)))
    reqs, imgs = _requests(14, seed=3)
    # two requests repeated so that same-geometry batches form
    reqs += reqs[:2]
    imgs += imgs[:2]
    streams = [codec.encode_image(model, im, q=r["q"]) for r, im in zip(reqs, imgs)]
    alone = [codec.decode_image(model, bs) for bs in streams]
    # a roomy budget, then one that holds the largest request but not two
    big = max(codec.decode_footprint(model, bs) for bs in streams)
    for budget, lanes in [(8 << 30, 3), (big + big // 2, 3)]:
        srv = pw.Server(codec, model, hbm_budget=budget, lanes=lanes, max_batch=4)
        tickets = [srv.submit(bs) for bs in streams]
        got = [srv.poll(t, timeout_ms=120000) for t in tickets]
        st = srv.stats()
        srv.close()
        for i, (a, g) in enumerate(zip(alone, got)):
            assert g is not None, f"request {i} not served"
            assert g.shape == a.shape and np.array_equal(a, g), f"request {i} differs"
        assert st["submitted"] == len(streams) and st["completed"] == len(streams)
        assert st["failed"] == 0 and st["queued"] == 0
        assert 1 <= st["batches"] <= len(streams)
        assert st["p99_ms"] >= st["p50_ms"] > 0 and st["mpix_per_s"] > 0
    model.close()
    codec.close()


def test_server_admission_and_errors(pw):
    codec = pw.Codec(0, "bf16")
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 11)))
    bs = codec.encode_image(model, S.gray_sinusoids(96, 128, seed=1), q=8)
    # a budget below one request's workspace: rejected at submission
    srv = pw.Server(codec, model, hbm_budget=1 << 20, lanes=1, max_batch=2)
    with pytest.raises(pw.PwError) as e:
        srv.submit(bs)
    assert e.value.code == pw.PW_EAGAIN
    assert srv.stats()["rejected"] == 1
    srv.close()
    srv = pw.Server(codec, model, hbm_budget=1 << 30, lanes=1, max_batch=2)
    # not a stream, and a stream of another model
    with pytest.raises(pw.PwError) as e:
        srv.submit(b"\0" * 80)
    assert e.value.code == pw.PW_ECORRUPT
    other = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 12)))
    with pytest.raises(pw.PwError) as e:
        srv.submit(codec.encode_image(other, S.gray_sinusoids(96, 128, seed=1), q=8))
    assert e.value.code == pw.PW_EINVAL
    # a truncated payload fails in the lane and is reported by poll
    t_bad = srv.submit(bs[: len(bs) - 40])
    t_ok = srv.submit(bs)
    with pytest.raises(pw.PwError):
        srv.poll(t_bad, timeout_ms=120000)
    assert np.array_equal(srv.poll(t_ok, timeout_ms=120000), codec.decode_image(model, bs))
    st = srv.stats()
    assert st["failed"] >= 1 and st["completed"] >= 1
    srv.close()
    other.close()
    model.close()
    codec.close()


@pytest.mark.parametrize("prec", ["fp8", "fp32"])
def test_server_forms_ragged_batches_of_similar_sizes(pw, prec):
    """A burst of requests of one format and similar (not equal) sizes, on
    one lane: the server batches them across sizes (fewer batches than
    requests) and every result equals the stream's single decode."""
    codec = pw.Codec(0, prec)
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 13)))
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(100, 129)), int(rng.integers(140, 161))) for _ in range(12)]
    imgs = [S.rgb_natural(h, w, seed=40 + i) for i, (h, w) in enumerate(sizes)]
    streams = [codec.encode_image(model, im, q=8.0) for im in imgs]
    alone = [codec.decode_image(model, bs) for bs in streams]
    srv = pw.Server(codec, model, hbm_budget=8 << 30, lanes=1, max_batch=6)
    tickets = [srv.submit(bs) for bs in streams]
    got = [srv.poll(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    srv.close()
    for i, (a, g) in enumerate(zip(alone, got)):
        assert np.array_equal(a, g), f"request {i} differs"
    print(f"\n{prec}: {len(streams)} requests of sizes {sizes[:3]}... in {st['batches']} batches")
    assert st["completed"] == len(streams)
    assert st["batches"] < len(streams)
    model.close()
    codec.close()


def test_server_ragged_batch_with_a_corrupt_stream(pw):
    """A corrupt stream inside a ragged batch fails only its own ticket: the
    batch is re-decoded one request at a time and the others are exact."""
    codec = pw.Codec(0, "fp8")
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 14)))
    sizes = [(112, 144), (120, 150), (104, 160), (116, 148), (110, 152)]
    streams = [codec.encode_image(model, S.rgb_natural(h, w, seed=60 + i), q=8.0)
               for i, (h, w) in enumerate(sizes)]
    bad = bytearray(streams[2])
    bad[len(bad) - 40] ^= 0x5A
    streams[2] = bytes(bad)
    srv = pw.Server(codec, model, hbm_budget=8 << 30, lanes=1, max_batch=5)
    tickets = [srv.submit(bs) for bs in streams]
    for i, t in enumerate(tickets):
        if i == 2:
            with pytest.raises(pw.PwError) as e:
                srv.poll(t, timeout_ms=120000)
            assert e.value.code == pw.PW_ECORRUPT
        else:
            assert np.array_equal(srv.poll(t, timeout_ms=120000),
                                  codec.decode_image(model, streams[i]))
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1 and st["completed"] == len(streams) - 1
    model.close()
    codec.close()
