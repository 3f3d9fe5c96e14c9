"""Autotuner of the tensor-core convolutions: encoding and decoding with
tuning disabled (default schedules) and enabled (candidate schedules sampled
on the real launches: one or two tiles per MMA round, default or
alternative pipeline shape) give bit-identical streams and images, and
every tuned class keeps the fastest of its sampled candidates."""
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


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_autotune_does_not_change_results(pw, prec):
    codec = pw.Codec(0, prec)
    cfg = S.ModelConfig(levels=4, C=64, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 4)))
    img = S.rgb_natural(200, 296, seed=13)
    old = pw.pw_autotune(0)
    bs0 = codec.encode_image(model, img, q=8.0)
    out0 = codec.decode_image(model, bs0)
    pw.pw_autotune(1)
    # the tuning samples run on real launches: repeat until classes converge
    bs1 = [codec.encode_image(model, img, q=8.0) for _ in range(4)]
    outs = [codec.decode_image(model, bs0) for _ in range(4)]
    pw.pw_autotune(old)
    assert all(b == bs0 for b in bs1)
    assert all(np.array_equal(out0, o) for o in outs)
    rep = pw.autotune_report()
    assert rep, "no convolution class was tuned"
    for e in rep:
        sampled = [v for v in e["us"] if v >= 0]
        if len(sampled) >= 2:
            assert e["us"][e["choice"]] == min(sampled)
    print("\n" + "\n".join(f"{e['ks']}x{e['ks']} epi {e['epi']} fp8 {e['fp8']} 2^{e['log2tiles']} "
                             f"tiles: choice {e['choice']} us {e['us']}" for e in rep))
    model.close()
    codec.close()


def test_autotune_settles(pw):
    """Repeated decodes of one plan finish every class's sampling, after
    which pw_autotune_settled reports it (what a service waits for)."""
    codec = pw.Codec(0, "fp8")
    cfg = S.ModelConfig(levels=4, C=64, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 5)))
    bs = codec.encode_image(model, S.rgb_natural(136, 200, seed=14), q=8.0)
    ref = codec.decode_image(model, bs)
    n = 0
    while not pw.pw_autotune_settled() and n < 40:
        assert np.array_equal(codec.decode_image(model, bs), ref)
        n += 1
    assert pw.pw_autotune_settled() == 1, n
    model.close()
    codec.close()
