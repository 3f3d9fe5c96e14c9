"""Pins of the oracle's interleaved rANS coder.

Round trips (random tables, escapes, lane counts), an exhaustive round trip
over every short sequence of a small alphabet, and brute-force code lengths
on 8x8 inputs compared with the ideal information content sum(-log2 f/M).
"""
import itertools

import numpy as np
import pytest

from oracle import entropy as E
from oracle import rans as R


@pytest.fixture(scope="module")
def bank():
    return E.cdf_bank().astype(np.int64)


def _roundtrip(bank, r, tid, nl):
    ops = [R.symbol_ops(int(r[p]), bank[tid[p]]) for p in range(len(r))]
    st, words = R.encode_chunk(ops, nl)
    out, used, xf = R.decode_chunk(st, words, len(r), nl, lambda p: bank[tid[p]])
    assert out == [int(v) for v in r]
    assert used == len(words)
    assert all(v == R.L for v in xf)
    return st, words


@pytest.mark.parametrize("nl", [1, 3, 32])
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 700])
def test_roundtrip_random_with_escapes(bank, nl, n):
    rng = np.random.default_rng(n * 100 + nl)
    tid = rng.integers(0, 2048, n)
    r = np.round(rng.laplace(0, 5, n)).astype(np.int64)
    big = rng.uniform(size=n) < 0.07
    r[big] = rng.integers(-200000, 200000, big.sum())
    _roundtrip(bank, r, tid, nl)


def test_escape_extremes(bank):
    r = np.array([63, -63, 64, -64, 62, -62, (1 << 30), -(1 << 30), 0])
    tid = np.full(len(r), 8 * 128 + 20)
    for nl in (1, 2, 9):
        _roundtrip(bank, r, tid, nl)


def test_exhaustive_small_alphabet(bank):
    vals = [-2, -1, 0, 1, 70]            # 70 escapes (ESC_R)
    tid = np.array([8 * 128 + 5, 3 * 128 + 40, 12 * 128 + 90, 8 * 128 + 0])
    for nl in (1, 2):
        for seq in itertools.product(vals, repeat=4):
            _roundtrip(bank, np.array(seq), tid, nl)


@pytest.mark.parametrize("nl", [1, 4, 32])
def test_code_length_8x8_against_ideal(bank, nl):
    """Stored bits B = 16 * words + 32 * lanes. Each lane's final decoder
    state is the known constant 2^16, so B - 16 * lanes carries the symbols;
    it must lie within 0.05 bit per symbol of the ideal information content
    below, and above by at most that plus 16 bits of flush per lane."""
    rng = np.random.default_rng(nl)
    for trial in range(40):
        n = 64
        tid = rng.integers(0, 2048, n)
        j = tid % 128
        r = np.array([int(np.round(rng.laplace(0, float(E.sigma_of_bin(jj))))) for jj in j])
        r = np.clip(r, -E.T, E.T)
        _, words = _roundtrip(bank, r, tid, nl)
        s = r + E.T + 1
        f = np.array([bank[t][k + 1] - bank[t][k] for t, k in zip(tid, s)])
        ideal = float(np.sum(-np.log2(f / E.M)))
        B = 16 * len(words) + 32 * nl
        assert B - 16 * nl >= ideal - 0.05 * n
        assert B - 16 * nl <= ideal + 0.05 * n + 16 * nl
