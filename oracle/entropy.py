"""Entropy parameters -> table indices, and the Laplace CDF table bank.

Test infrastructure only. The paper codes each quantised coefficient with a
Laplace distribution whose mean and scale come from the context model
(Section 3.1) and uses adaptive arithmetic coding. Encoder and decoder must
pick the same integer frequency table for every symbol, so the mapping from
(mu, sigma) to a table and the tables themselves are fixed-point by
definition. This module states that definition:

Index decision (FP32, exact IEEE operations only):
  t   = rint(16 * mu)              (round half to even; |t| clamped to 2^23)
  ctr = (t + 8) >> 4               (floor division by 16)
  phi = t - 16 * ctr               in [-8, 7]: mean offset in 1/16 steps
  j   = clamp((bits(sigma) - bits(0.125)) >> 20, 0, 127)
        (8 bins per octave from the float32 bit pattern, 16 octaves above
        0.125)
Table (phi, j) models r = y - ctr for r in [-T, T] plus two escape symbols
(ESC_L for r < -T, ESC_R for r > T), 127 symbols in all, with
  mean  mu' = phi / 16,  scale b_j = float32 with bits
  bits(0.125) + (j << 20) + (1 << 19)  (the middle of bin j),
  F(u)  = exp(u / b) / 2 for u < 0, 1 - exp(-u / b) / 2 otherwise,
  p_s   = F(upper edge of s) - F(lower edge of s), edges at r +- 1/2 - mu',
  f_s   = 1 + floor(max(p_s, 0) * (M - 127)),  M = 2^15,
and the signed remainder M - sum(f) added to the first largest f. The
exponential is the project's own FP32 routine (Cody-Waite reduction by ln 2,
degree-6 Taylor polynomial, Horner order), so both sides evaluate the same
sequence of correctly rounded FP32 operations. numpy float32 array
arithmetic performs exactly those single operations (no fused multiply-add).

Pins (tests/test_oracle_entropy.py): every table is strictly increasing,
starts at 0, ends at M, has every frequency >= 1, and is within (127+1)/M of
the FP64 Laplace probabilities; the FP32 exponential is within 2 ulp of
numpy's FP64 exp; the index decision matches its definition on hand-picked
boundary values.
"""
from __future__ import annotations

import numpy as np

M = 1 << 15
LOG2M = 15
T = 62
NSYM = 2 * T + 3          # ESC_L, r = -T..T, ESC_R
NPHI = 16
NJ = 128
SIG_BITS0 = 0x3E000000    # float32 bits of 0.125
f32 = np.float32

# FP32 constants of the exponential (each the float32 nearest the value)
LOG2E = f32(1.4426950408889634)
LN2_HI = f32(0.693145751953125)           # 0x3F317200, 16 significant bits
LN2_LO = f32(0.6931471805599453 - 0.693145751953125)
EXP_C = [f32(1.0), f32(1.0), f32(0.5), f32(1.0 / 6.0), f32(1.0 / 24.0),
         f32(1.0 / 120.0), f32(1.0 / 720.0)]


def exp32(z: np.ndarray) -> np.ndarray:
    """exp(z) for float32 z <= 0 with a fixed sequence of FP32 operations.

    z < -80 returns 0. Otherwise k = rint(z * log2 e), r = (z - k ln2_hi) -
    k ln2_lo, p = Horner(1/0!, ..., 1/6!)(r), result p * 2^k (2^k built from
    its bit pattern, exact).
    """
    z = np.asarray(z, dtype=f32)
    small = z < f32(-80.0)
    zz = np.where(small, f32(0.0), z).astype(f32)
    k = np.rint(zz * LOG2E).astype(f32)
    r = (zz - k * LN2_HI).astype(f32)
    r = (r - k * LN2_LO).astype(f32)
    p = EXP_C[6]
    for c in (EXP_C[5], EXP_C[4], EXP_C[3], EXP_C[2], EXP_C[1], EXP_C[0]):
        p = (p * r).astype(f32)
        p = (p + c).astype(f32)
    ki = k.astype(np.int32)
    scale = ((ki + 127).astype(np.uint32) << np.uint32(23)).view(f32)
    out = (p * scale).astype(f32)
    return np.where(small, f32(0.0), out).astype(f32)


def sigma_of_bin(j) -> np.ndarray:
    """Representative scale of bin j (float32, middle of the bin)."""
    j = np.asarray(j, dtype=np.uint32)
    return (np.uint32(SIG_BITS0) + (j << np.uint32(20)) +
            np.uint32(1 << 19)).view(f32)


def sigma_bin(sigma32: np.ndarray) -> np.ndarray:
    """Bin index j of float32 scales (bit-pattern quantiser, clamped)."""
    b = np.asarray(sigma32, dtype=f32).view(np.uint32).astype(np.int64)
    j = (b - SIG_BITS0) >> 20
    return np.clip(j, 0, NJ - 1)


def index_decision(mu, sigma):
    """(ctr, phi, j) from entropy parameters; decision taken in FP32.

    mu and sigma may be FP64 (oracle) or FP32; they are first rounded to
    float32, the precision in which the decision is defined.
    """
    m32 = np.asarray(mu, dtype=np.float64).astype(f32)
    s32 = np.asarray(sigma, dtype=np.float64).astype(f32)
    t = np.rint((m32 * f32(16.0)).astype(f32)).astype(np.float64)
    t = np.clip(t, -(1 << 23), 1 << 23).astype(np.int64)
    ctr = (t + 8) >> 4
    phi = t - 16 * ctr
    j = sigma_bin(s32)
    return ctr, phi, j


def _edge(j):
    """Lower edge of sigma bin j (float32 bit pattern bits(0.125) + j << 20)."""
    j = np.asarray(j, dtype=np.int64)
    return (np.uint32(SIG_BITS0) + (np.clip(j, 0, NJ).astype(np.uint32)
                                    << np.uint32(20))).view(f32).astype(np.float64)


def near_tie(mu, sigma, eps: float):
    """True where an FP64 (mu, sigma) lies within relative eps of a decision
    boundary: 16 mu near a half-integer, or sigma near an inner bin edge."""
    mu = np.asarray(mu, dtype=np.float64)
    sg = np.asarray(sigma, dtype=np.float64)
    v = 16.0 * mu
    d = np.abs(v - (np.floor(v) + 0.5))
    tie_mu = d <= eps * np.maximum(np.abs(v), 1.0)
    j = sigma_bin(sg.astype(f32))
    lo, hi = _edge(j), _edge(j + 1)
    tie_lo = (j >= 1) & (np.abs(sg - lo) <= eps * sg)
    tie_hi = (j + 1 <= NJ - 1) & (np.abs(sg - hi) <= eps * sg)
    return tie_mu | tie_lo | tie_hi


def cdf_table(phi: int, j: int) -> np.ndarray:
    """Cumulative frequencies (NSYM + 1 entries, uint32) of table (phi, j)."""
    mup = f32(f32(phi) / f32(16.0))
    b = sigma_of_bin(j)
    inv_b = f32(f32(1.0) / b)
    k = np.arange(NSYM - 1, dtype=f32)           # edges between symbols
    u = (k - f32(T + 0.5)).astype(f32)
    u = (u - mup).astype(f32)
    z = (u * inv_b).astype(f32)
    neg = u < f32(0.0)
    e_neg = exp32(np.where(neg, z, f32(0.0)).astype(f32))
    e_pos = exp32(np.where(neg, f32(0.0), -z).astype(f32))
    Fn = (f32(0.5) * e_neg).astype(f32)
    Fp = (f32(1.0) - (f32(0.5) * e_pos).astype(f32)).astype(f32)
    F = np.where(neg, Fn, Fp).astype(f32)
    p = np.empty(NSYM, dtype=f32)
    p[0] = F[0]
    p[1:NSYM - 1] = (F[1:] - F[:-1]).astype(f32)
    p[NSYM - 1] = f32(f32(1.0) - F[-1])
    p = np.maximum(p, f32(0.0))
    q = np.floor((p * f32(M - NSYM)).astype(f32)).astype(np.int64)
    f = 1 + q
    rem = M - int(f.sum())
    f[int(np.argmax(f))] += rem
    cdf = np.zeros(NSYM + 1, dtype=np.int64)
    cdf[1:] = np.cumsum(f)
    assert cdf[-1] == M
    return cdf.astype(np.uint32)


def cdf_bank() -> np.ndarray:
    """All 16 x 128 tables: array [NPHI * NJ, NSYM + 1] (uint16).

    Table id = (phi + 8) * 128 + j.
    """
    bank = np.zeros((NPHI * NJ, NSYM + 1), dtype=np.uint32)
    for phi in range(-8, 8):
        for j in range(NJ):
            bank[(phi + 8) * NJ + j] = cdf_table(phi, j)
    return bank.astype(np.uint16)


def table_id(phi, j):
    return (np.asarray(phi) + 8) * NJ + np.asarray(j)


def laplace_probs64(phi: int, j: int) -> np.ndarray:
    """FP64 symbol probabilities of table (phi, j) (for the pins)."""
    mup = phi / 16.0
    b = float(sigma_of_bin(j))
    edges = np.arange(NSYM - 1) - (T + 0.5) - mup
    F = np.where(edges < 0, 0.5 * np.exp(np.minimum(edges, 0) / b),
                 1.0 - 0.5 * np.exp(-np.maximum(edges, 0) / b))
    p = np.empty(NSYM)
    p[0] = F[0]
    p[1:-1] = np.diff(F)
    p[-1] = 1.0 - F[-1]
    return p
