"""Per-kernel-class timing (pw_ctx_profile, pw_ctx_profile_classes,
pw_kernel_class): every class is recorded when profiling is on; with a class
mask only the selected class is, with the same launch count as in the full
recording; profiling never changes the decoded image."""
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


def _stats(pw, codec):
    st = (pw.pw_kernel_stat * 32)()
    n = pw.pw_ctx_kernel_stats(codec.ctx, st, 32)
    assert n >= 0
    return {st[i].name.decode(): (int(st[i].launches), float(st[i].ms)) for i in range(n)}


def test_class_mask_records_only_the_selected_class(pw):
    codec = pw.Codec(0, "fp8")
    cfg = S.ModelConfig(levels=4, C=32, ll_mode=0)
    model = codec.load_model(S.pack_blob(cfg, S.random_model(cfg, 5)))
    bs = codec.encode_image(model, S.rgb_natural(64, 96, seed=2), q=8.0)
    ref = codec.decode_image(model, bs)
    pw.pw_ctx_profile(codec.ctx, 1)
    out_all = codec.decode_image(model, bs)
    every = _stats(pw, codec)
    pw.pw_ctx_profile(codec.ctx, 0)
    assert {"rans_decode", "ctx_lstm_gates_conv3x3", "lift_step"} <= set(every)
    assert all(ms >= 0.0 and n > 0 for n, ms in every.values())
    k = pw.pw_kernel_class(b"rans_decode")
    assert k >= 0 and pw.pw_kernel_class(b"no such class") == -1
    pw.pw_ctx_profile_classes(codec.ctx, 1 << k)
    out_one = codec.decode_image(model, bs)
    one = _stats(pw, codec)
    pw.pw_ctx_profile(codec.ctx, 0)
    assert set(one) == {"rans_decode"}
    assert one["rans_decode"][0] == every["rans_decode"][0]
    assert np.array_equal(ref, out_all) and np.array_equal(ref, out_one)
    model.close()
    codec.close()
