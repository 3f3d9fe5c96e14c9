"""Host-only parts of the binding and the library (no GPU, no CUDA call):
the stream-header parser against the oracle's on an oracle-encoded stream,
the padded plane size, status strings, the kernel-class names the benchmark
uses, and the autotuner's report before anything was tuned.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import codec as K
from oracle.lifting import subband_shapes
from tests._lib import ensure_built


@pytest.fixture(scope="module")
def pw():
    ensure_built()
    import paper_2405_12631_gb300 as m
    return m


def test_stream_header_parser_agrees_with_the_oracle(pw):
    cfg = S.ModelConfig(levels=4, C=32, F=16, ll_mode=0)
    blob = S.pack_blob(cfg, S.random_model(cfg, 0))
    img = S.rgb_natural(40, 56, seed=2)           # not a multiple of 16: padded
    bs = K.encode_image(blob, img, q=16.0)
    mine, ref = pw.parse_stream_header(bs), K.parse_header(bs)
    for k in ("version", "width", "height", "ncomp", "levels", "bitdepth", "colour", "chunk",
              "n_chunks", "model_hash", "payload_bytes"):
        assert mine[k] == ref[k], k
    assert np.float32(mine["delta_l"]) == ref["delta_l"]
    assert np.float32(mine["delta_h"]) == ref["delta_h"]
    # padded plane = the sum of the subband sizes of the padded plane
    n = pw.padded_elems(mine)
    assert n == sum(h * w for h, w, _ in subband_shapes(48, 64, 4)) == 48 * 64
    with pytest.raises(ValueError):
        pw.parse_stream_header(b"XXXX" + bs[4:])


def test_status_strings(pw):
    assert pw.pw_strerror(pw.PW_OK) == b"ok"
    for code in (2, 3, 5, 6):   # ENOMEM, ECORRUPT, ETIMEOUT, EAGAIN: fixed strings
        s = pw.pw_strerror(code)
        assert s and s != b"unknown error"
    assert pw.pw_strerror(12345) == b"unknown error"


def test_kernel_class_names_round_trip(pw):
    names = ["ctx_lstm_gates_conv3x3", "ctx_conv3x3", "ctx_conv1x1", "ctx_small",
             "rans_decode", "rans_encode", "cdf_bank", "lift_step", "colour", "parse", "quant",
             "ctx_head_conv3x3", "mix_head"]
    assert [pw.pw_kernel_class(n.encode()) for n in names] == list(range(len(names)))
    assert pw.pw_kernel_class(b"no_such_class") == -1


def test_autotune_report_empty_before_tuning(pw):
    assert pw.autotune_report() == []
