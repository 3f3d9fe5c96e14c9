"""Interleaved rANS coder, plain Python (test infrastructure only).

The paper codes the quantised subbands with adaptive arithmetic coding
(Section 3.1) but does not specify the coder. This module defines the
replacement used throughout: range-variant asymmetric numeral systems
(Duda 2013) with `nl` interleaved states sharing one stream of 16-bit words
(Giesen 2014 interleaving), so one GPU warp can decode 32 symbols at a time.

Parameters: total frequency M = 2^15, state interval [2^16, 2^32), 16-bit
renormalisation words. A chunk holds n symbols; symbol p belongs to lane
p mod nl and iteration p div nl. For every iteration the decoder runs
"rounds": round 0 decodes each active lane's main symbol, later rounds decode
one bypass bit (a symbol of frequency M/2) for each lane that still has
escape bits pending. After every round the lanes whose state fell below 2^16
read one word each, in ascending lane order. The encoder runs everything in
reverse (iterations, rounds and lanes descending), pushing words on a stack;
the stream is the reversed stack. A chunk is stored as nl u32 initial decoder
states followed by the u16 words (little endian).

Escapes: symbol 0 (ESC_L) and 126 (ESC_R) mean r < -T or r > T; the excess
e = |r| - T - 1 follows as an order-0 Exp-Golomb code in bypass bits: k ones,
a zero, then the k low bits of e + 1, most significant first.

Pins (tests/test_oracle_rans.py): decode(encode(s)) = s for random tables,
lane counts and escapes; exhaustive round trips over small alphabets; brute
force code lengths on 8x8 inputs lie between the ideal information content
and that plus the state-flush overhead.
"""
from __future__ import annotations

import numpy as np

M = 1 << 15
L = 1 << 16
HALF = M >> 1
T = 62
ESC_L = 0
ESC_R = 2 * T + 2


def symbol_ops(r: int, cdf: np.ndarray):
    """Coding operations (start, freq) for residual r with table `cdf`."""
    if -T <= r <= T:
        s = r + T + 1
        return [(int(cdf[s]), int(cdf[s + 1]) - int(cdf[s]))]
    s = ESC_L if r < -T else ESC_R
    e = (-r if r < -T else r) - T - 1
    ops = [(int(cdf[s]), int(cdf[s + 1]) - int(cdf[s]))]
    v = e + 1
    k = v.bit_length() - 1
    bits = [1] * k + [0] + [(v >> (k - 1 - i)) & 1 for i in range(k)]
    ops += [(b * HALF, HALF) for b in bits]
    return ops


def encode_chunk(ops: list, nl: int):
    """Encode a chunk given per-symbol operation lists.

    Returns (states, words): the nl initial decoder states and the u16 word
    stream in decoder read order.
    """
    n = len(ops)
    x = [L] * nl
    stack = []
    niter = (n + nl - 1) // nl
    for it in range(niter - 1, -1, -1):
        base = it * nl
        rounds = max(len(ops[p]) for p in range(base, min(base + nl, n)))
        for rnd in range(rounds - 1, -1, -1):
            for lane in range(nl - 1, -1, -1):
                p = base + lane
                if p >= n or rnd >= len(ops[p]):
                    continue
                c, f = ops[p][rnd]
                xl = x[lane]
                if xl >= (f << 17):
                    stack.append(xl & 0xFFFF)
                    xl >>= 16
                x[lane] = (xl // f) * M + (xl % f) + c
    return x, stack[::-1]


def _word(words, ptr: int) -> int:
    if ptr >= len(words):
        raise ValueError("corrupt chunk: word stream exhausted")
    return int(words[ptr])


def _find(cdf: np.ndarray, slot: int) -> int:
    return int(np.searchsorted(cdf, slot, side="right")) - 1


def decode_chunk(states, words, n: int, nl: int, table_of, on_symbol=None):
    """Decode n residuals. table_of(p) returns the CDF of symbol p; it is
    called for every symbol of an iteration before that iteration decodes.
    on_symbol(p, r), if given, is called once symbol p is complete (before
    the next iteration asks for its tables), which lets a single-lane chunk
    drive an autoregressive context model.

    Returns (residuals, words consumed, final states).
    """
    x = list(states)
    ptr = 0
    out = [0] * n
    niter = (n + nl - 1) // nl
    for it in range(niter):
        base = it * nl
        lanes = [l for l in range(nl) if base + l < n]
        sym = {}
        for l in lanes:
            cdf = table_of(base + l)
            slot = x[l] & (M - 1)
            s = _find(cdf, slot)
            f = int(cdf[s + 1]) - int(cdf[s])
            x[l] = f * (x[l] >> 15) + slot - int(cdf[s])
            sym[l] = s
        for l in lanes:
            if x[l] < L:
                x[l] = (x[l] << 16) | _word(words, ptr)
                ptr += 1
        # escape state machines: phase 0 counts ones, phase 1 reads k bits
        pend = {l: [0, 0, 0] for l in lanes if sym[l] in (ESC_L, ESC_R)}
        while pend:
            for l in sorted(pend):
                slot = x[l] & (M - 1)
                b = slot >> 14
                x[l] = HALF * (x[l] >> 15) + (slot & (HALF - 1))
                st = pend[l]
                if st[0] == 0:
                    if b == 1:
                        st[1] += 1
                    else:
                        st[0] = 1
                        st[2] = 1
                else:
                    st[2] = (st[2] << 1) | b
                    st[1] -= 1
            done = []
            for l in sorted(pend):
                if x[l] < L:
                    x[l] = (x[l] << 16) | _word(words, ptr)
                    ptr += 1
                st = pend[l]
                if st[0] == 1 and st[1] == 0:
                    done.append(l)
            for l in done:
                e = pend.pop(l)[2] - 1
                sym[l] = (ESC_L, e) if sym[l] == ESC_L else (ESC_R, e)
        for l in lanes:
            s = sym[l]
            if isinstance(s, tuple):
                r = -(s[1] + T + 1) if s[0] == ESC_L else s[1] + T + 1
            else:
                r = s - T - 1
            out[base + l] = r
            if on_symbol is not None:
                on_symbol(base + l, r)
    return out, ptr, x


def pack_chunk(states, words) -> bytes:
    return (np.asarray(states, dtype="<u4").tobytes() +
            np.asarray(words, dtype="<u2").tobytes())


def unpack_chunk(buf: bytes, nl: int):
    states = np.frombuffer(buf[:4 * nl], dtype="<u4").astype(np.int64).tolist()
    words = np.frombuffer(buf[4 * nl:], dtype="<u2")
    return states, words
