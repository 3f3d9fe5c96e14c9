"""The allocation-free rANS decoding entry point (pw_rans_decode_noalloc).

It exists for callers that cannot allocate device memory while decoding
(plug-ins inside a host application's fixed memory budget, real-time
pipelines that must not stall on cudaMalloc / cudaFree). Its output must
equal the regular pw_rans_decode's and the values the oracle coded, bit for
bit, on two calls in a row (the second call reuses the shared scratch array
left by the first); it must refuse more chunks than its fixed scratch array
holds, report a chunk outside the payload as corrupt, and decode correctly
again on the call after that (the status word is cleared per call). This file is
collected last so that a run stopping at the first failure has run every
other test already.
"""
import ctypes

import numpy as np
import pytest

from oracle import entropy as E
from oracle import rans as R
from tests._lib import ensure_built

pytestmark = pytest.mark.gpu


def _chunks(seed, nchunks):
    bank = E.cdf_bank().astype(np.int64)
    rng = np.random.default_rng(seed)
    counts, lanes, idx, payload, offs, nb, vals = [], [], [], b"", [], [], []
    for c in range(nchunks):
        n = int(rng.integers(1, 2000))
        nl = int(rng.choice([1, 5, 32]))
        tid = rng.integers(0, 2048, n)
        ctr = rng.integers(-30, 30, n)
        r = np.round(rng.laplace(0, 3, n)).astype(np.int64)
        big = rng.uniform(size=n) < 0.02
        r[big] = rng.integers(-3000, 3000, big.sum())
        st, words = R.encode_chunk([R.symbol_ops(int(r[p]), bank[tid[p]]) for p in range(n)], nl)
        b = R.pack_chunk(st, words)
        offs.append(len(payload)); nb.append(len(b)); payload += b
        t = 16 * ctr + (tid // 128 - 8)
        idx.append(((t + (1 << 23)) << 7) | (tid % 128))
        counts.append(n); lanes.append(nl)
        vals.append(ctr + r)
    u32 = lambda a: np.asarray(a, dtype=np.uint32)
    return (payload, u32(offs), u32(nb), u32(counts), u32(lanes),
            np.concatenate(idx).astype(np.uint32), np.concatenate(vals).astype(np.int32))


def _noalloc(pw, payload, offs, nb, counts, lanes, idx):
    """Call the entry point through the C ABI on device copies; returns
    (status, decoded values)."""
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy()).cuda()
    d_pay = dev(np.frombuffer(payload, dtype=np.uint8))
    d_off, d_nb, d_cnt, d_ln, d_idx = (dev(a) for a in (offs, nb, counts, lanes, idx))
    d_out = torch.full((int(counts.sum()),), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P = ctypes.c_void_p
    rc = pw.pw_rans_decode_noalloc(P(stream), P(d_pay.data_ptr()), len(payload), len(counts),
                                   P(d_off.data_ptr()), P(d_nb.data_ptr()),
                                   P(d_cnt.data_ptr()), P(d_ln.data_ptr()),
                                   P(d_idx.data_ptr()), P(d_out.data_ptr()))
    return rc, d_out.cpu().numpy()


def test_noalloc_decode_matches_regular_decode_twice():
    ensure_built()
    import paper_2405_12631_gb300 as pw
    codec = pw.Codec(0, "fp32")
    for call, seed in enumerate((11, 12)):
        payload, offs, nb, counts, lanes, idx, vals = _chunks(seed, 9)
        want = codec.rans_decode(payload, offs, nb, counts, lanes, idx)
        assert np.array_equal(want, vals)
        rc, got = _noalloc(pw, payload, offs, nb, counts, lanes, idx)
        assert rc == pw.PW_OK, (call, pw.pw_last_error())
        assert np.array_equal(got, want), call
    codec.close()


def test_noalloc_chunk_outside_payload_is_corrupt_then_recovers():
    """A chunk whose offset + nbytes runs past payload_bytes (a bad input
    the descriptor kernel checks before any payload byte is read) gives
    PW_ECORRUPT; the next call with good inputs decodes exactly."""
    ensure_built()
    import paper_2405_12631_gb300 as pw
    payload, offs, nb, counts, lanes, idx, vals = _chunks(13, 5)
    bad = offs.copy()
    bad[2] = len(payload) - nb[2] // 2
    rc, _ = _noalloc(pw, payload, bad, nb, counts, lanes, idx)
    assert rc == pw.PW_ECORRUPT, pw.pw_last_error()
    rc, got = _noalloc(pw, payload, offs, nb, counts, lanes, idx)
    assert rc == pw.PW_OK, pw.pw_last_error()
    assert np.array_equal(got, vals)


def test_noalloc_rejects_too_many_chunks():
    ensure_built()
    import paper_2405_12631_gb300 as pw
    P = ctypes.c_void_p
    rc = pw.pw_rans_decode_noalloc(None, P(1), 16, 16385, P(1), P(1), P(1), P(1), P(1), P(1))
    assert rc == pw.PW_EINVAL
    assert b"16384" in pw.pw_last_error()
