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

Logistic mixture (K = 3), the alternative probability model that Section
4 compares with the Laplace one (the paper gives no layer or coding details;
this is the reading). The head has 9 outputs per position: weight logits
w_k, means mu_k and scale pre-activations rho_k, sigma_k = softplus(rho_k).
Decision (FP32, from (w, mu, sigma) rounded to float32): a = the first k of largest w_k;
ctr = rint(mu_a) (|ctr| <= 2^23); q_k = clamp(rint(8 (mu_k - ctr)),
-255, 255) (eighth-step mean offsets); g_k = clamp(rint(4 (w_k - w_a)),
-31, 0) (quarter-step log-weights, 0 for the reference component);
j_k = the scale bin of sigma_k as above. Table of a key (q, j, g)
for r = y - ctr, edges u_e = e - 62.5 (e = 0..125): m_k = q_k / 8,
inv_k = 1 / b_{j_k}, om_k = exp32(g_k / 4), W = (om_0 + om_1) + om_2,
z = (u_e - m_k) inv_k, S(z) = 1 / (1 + exp32(-z)) for z >= 0 and
e / (1 + e), e = exp32(z), otherwise, F(u_e) = ((om_0 S_0 + om_1 S_1) +
om_2 S_2) / W, then p, f and the remainder exactly as for the Laplace
tables (same escapes, M and minimum frequency). Every operation is one
correctly rounded FP32 operation, so encoder and decoder build the same
table for every symbol.

Pins (tests/test_oracle_entropy.py): every table is strictly increasing,
starts at 0, ends at M, has every frequency >= 1, and is within (127+1)/M of
the FP64 Laplace probabilities; the FP32 exponential is within 2 ulp of
numpy's FP64 exp; the index decision matches its definition on hand-picked
boundary values. Mixture pins (tests/test_oracle_mixture.py): valid CDFs
within (127+1)/M of the FP64 mixture; three equal components give the
closed-form logistic; a component of weight e^(-31/4) barely moves the
table and one of full weight moves it by the FP64 amount; hand-worked
decisions at the rounding, argmax and clamping boundaries.
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


# ---------------------------------------------------------------------------
# Logistic mixture with K = 3 components (the probability model the batched
# single-image configuration names; the paper's own model is the Laplace
# above). The head gives per position 9 values: weight logits w_k, means
# mu_k and scale pre-activations rho_k (scale softplus(rho_k)). As for the
# Laplace model, the parameters are first reduced to integers by an FP32
# decision, and the symbol's table is a function of those integers alone:
#   a    = the first k with the largest w_k, ctr = rint(mu_a) (|t| <= 2^23),
#   q_k  = clamp(rint(8 (mu_k - ctr)), -255, 255)   mean offset in 1/8,
#   j_k  = the scale bin of softplus(rho_k)          (as sigma_bin),
#   g_k  = clamp(rint(4 (w_k - w_a)), -31, 0)       log-weight in 1/4.
# Table (FP32, exact IEEE operations in this order): m_k = q_k / 8,
# 1/b_k with b_k = sigma_of_bin(j_k), weights om_k = exp32(g_k / 4),
# W = (om_0 + om_1) + om_2; at the 126 symbol edges u (as for the Laplace
# tables) F(u) = ((om_0 s_0 + om_1 s_1) + om_2 s_2) / W with
# s_k = sigmoid((u - m_k) / b_k) = 1 / (1 + exp32(-z)) for z >= 0 and
# exp32(z) / (1 + exp32(z)) for z < 0; then the probabilities, frequencies
# and remainder exactly as cdf_table does.
MIX_K = 3


def mix_params(head):
    """Raw head outputs [..., 9] (w, mu, rho) -> entropy parameters
    (w, mu, sigma), sigma = softplus(rho) (FP64)."""
    h = np.array(head, dtype=np.float64)
    rho = h[..., 6:9]
    h[..., 6:9] = np.where(rho > 20.0, rho, np.log1p(np.exp(np.minimum(rho, 20.0))))
    return h


def mix_decision(par):
    """(ctr, q, j, g) from mixture parameters [..., 9] (weight logits w,
    means mu, scales sigma): ctr [...] int, q, j, g [..., 3] int; decided in
    FP32 (parameters rounded to float32 first)."""
    h32 = np.asarray(par, dtype=np.float64).astype(f32)
    w, mu, sg = h32[..., 0:3], h32[..., 3:6], h32[..., 6:9]
    a = np.argmax(w, axis=-1)
    wa = np.take_along_axis(w, a[..., None], -1)
    mua = np.take_along_axis(mu, a[..., None], -1)[..., 0]
    t = np.rint(mua).astype(np.float64)
    ctr = np.clip(t, -(1 << 23), 1 << 23).astype(np.int64)
    d = (mu - ctr.astype(f32)[..., None]).astype(f32)
    q = np.clip(np.rint((d * f32(8.0)).astype(f32)), -255, 255).astype(np.int64)
    dw = (w - wa).astype(f32)
    g = np.clip(np.rint((dw * f32(4.0)).astype(f32)), -31, 0).astype(np.int64)
    j = sigma_bin(sg)
    return ctr, q, j, g


def _sigmoid32(z):
    z = np.asarray(z, dtype=f32)
    e_pos = exp32(np.where(z >= 0, -z, f32(0.0)).astype(f32))
    e_neg = exp32(np.where(z < 0, z, f32(0.0)).astype(f32))
    s_pos = (f32(1.0) / (f32(1.0) + e_pos).astype(f32)).astype(f32)
    s_neg = (e_neg / (f32(1.0) + e_neg).astype(f32)).astype(f32)
    return np.where(z >= 0, s_pos, s_neg).astype(f32)


def mix_tables(q, j, g) -> np.ndarray:
    """Cumulative frequencies [N, NSYM + 1] (uint32) of N mixture keys
    (q, j, g: [N, 3] ints), each built as the header describes."""
    q = np.asarray(q, dtype=np.int64).reshape(-1, MIX_K)
    j = np.asarray(j, dtype=np.int64).reshape(-1, MIX_K)
    g = np.asarray(g, dtype=np.int64).reshape(-1, MIX_K)
    N = q.shape[0]
    m = (q.astype(f32) / f32(8.0)).astype(f32)                       # [N, K]
    inv_b = (f32(1.0) / sigma_of_bin(j)).astype(f32)                 # [N, K]
    om = exp32((g.astype(f32) * f32(0.25)).astype(f32))              # [N, K]
    W = ((om[:, 0] + om[:, 1]).astype(f32) + om[:, 2]).astype(f32)  # [N]
    u = (np.arange(NSYM - 1, dtype=f32) - f32(T + 0.5)).astype(f32)  # [E]
    acc = None
    for k in range(MIX_K):
        z = ((u[None, :] - m[:, k:k + 1]).astype(f32) * inv_b[:, k:k + 1]).astype(f32)
        term = (om[:, k:k + 1] * _sigmoid32(z)).astype(f32)
        acc = term if acc is None else (acc + term).astype(f32)
    F = (acc / W[:, None]).astype(f32)                               # [N, E]
    p = np.empty((N, NSYM), dtype=f32)
    p[:, 0] = F[:, 0]
    p[:, 1:NSYM - 1] = (F[:, 1:] - F[:, :-1]).astype(f32)
    p[:, NSYM - 1] = (f32(1.0) - F[:, -1]).astype(f32)
    p = np.maximum(p, f32(0.0))
    f = 1 + np.floor((p * f32(M - NSYM)).astype(f32)).astype(np.int64)
    rem = M - f.sum(axis=1)
    f[np.arange(N), np.argmax(f, axis=1)] += rem
    cdf = np.zeros((N, NSYM + 1), dtype=np.int64)
    cdf[:, 1:] = np.cumsum(f, axis=1)
    assert np.all(cdf[:, -1] == M)
    return cdf.astype(np.uint32)


def mix_table(q, j, g) -> np.ndarray:
    """The table of one key (three ints each)."""
    return mix_tables([q], [j], [g])[0]


def mix_probs64(q, j, g) -> np.ndarray:
    """FP64 symbol probabilities of one mixture key (for the pins)."""
    om = np.exp(np.asarray(g, dtype=np.float64) / 4.0)
    om = om / om.sum()
    edges = np.arange(NSYM - 1) - (T + 0.5)
    F = np.zeros(NSYM - 1)
    for k in range(MIX_K):
        b = float(sigma_of_bin(int(j[k])))
        F += om[k] / (1.0 + np.exp(-(edges - q[k] / 8.0) / b))
    p = np.empty(NSYM)
    p[0] = F[0]
    p[1:-1] = np.diff(F)
    p[-1] = 1.0 - F[-1]
    return p


def mix_near_tie(par, eps: float):
    """True where an FP64 mixture parameter (w, mu, sigma) lies within
    relative eps of one of the decision's boundaries (the argmax, rint of
    mu_a, of 8 (mu_k - ctr) and of 4 (w_k - w_a), or a scale-bin edge)."""
    h = np.asarray(par, dtype=np.float64)
    w, mu, sg = h[..., 0:3], h[..., 3:6], h[..., 6:9]
    srt = np.sort(w, axis=-1)
    tie = np.abs(srt[..., 2] - srt[..., 1]) <= eps * np.maximum(np.abs(srt[..., 2]), 1.0)
    a = np.argmax(w, axis=-1)
    mua = np.take_along_axis(mu, a[..., None], -1)[..., 0]
    wa = np.take_along_axis(w, a[..., None], -1)
    half = lambda v: np.abs(v - (np.floor(v) + 0.5)) <= eps * np.maximum(np.abs(v), 1.0)
    tie |= half(mua)
    ctr = np.rint(mua)
    tie |= np.any(half(8.0 * (mu - ctr[..., None])), axis=-1)
    tie |= np.any(half(4.0 * (w - wa)), axis=-1)
    tie |= np.any(near_tie(np.zeros_like(sg), sg, eps), axis=-1)   # scale-bin edges
    return tie
