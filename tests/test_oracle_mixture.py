"""Pins of the oracle's logistic-mixture probability model (K = 3).

The tables are checked against the mathematics they approximate: every
table is a valid CDF (strictly increasing, 0 .. M, frequencies >= 1) within
the quantisation bound (127 + 1) / M of the FP64 mixture probabilities; three
identical components are one logistic distribution, written out here from
its closed form 1 / (1 + exp(-(x - m) / b)); a component with weight
exp(-31 / 4) relative to the others barely moves the table; and the FP32
decision gives hand-worked keys at its rounding and clamping boundaries.
"""
import numpy as np

from oracle import entropy as E

M = E.M


def _logistic_probs(m, b):
    edges = np.arange(E.NSYM - 1) - (E.T + 0.5)
    F = 1.0 / (1.0 + np.exp(-(edges - m) / b))
    p = np.empty(E.NSYM)
    p[0] = F[0]
    p[1:-1] = np.diff(F)
    p[-1] = 1.0 - F[-1]
    return p


def test_mixture_tables_are_valid_cdfs_near_the_fp64_mixture():
    rng = np.random.default_rng(0)
    N = 400
    q = rng.integers(-255, 256, (N, 3))
    j = rng.integers(0, 128, (N, 3))
    g = rng.integers(-31, 1, (N, 3))
    g[:, rng.integers(0, 3, N) * 0] = 0
    tabs = E.mix_tables(q, j, g)
    for i in range(N):
        c = tabs[i].astype(np.int64)
        f = np.diff(c)
        assert c[0] == 0 and c[-1] == M and np.all(f >= 1)
        p64 = E.mix_probs64(q[i], j[i], g[i])
        assert np.max(np.abs(f / M - p64)) <= (E.NSYM + 1) / M


def test_identical_components_are_one_logistic():
    for q0, j0 in ((0, 40), (-37, 64), (100, 10), (5, 127)):
        c = E.mix_table([q0] * 3, [j0] * 3, [0, 0, 0]).astype(np.int64)
        p = _logistic_probs(q0 / 8.0, float(E.sigma_of_bin(j0)))
        assert np.max(np.abs(np.diff(c) / M - p)) <= (E.NSYM + 1) / M
        # and the table does not depend on the components' weights then
        c2 = E.mix_table([q0] * 3, [j0] * 3, [0, -13, -31]).astype(np.int64)
        assert np.max(np.abs(c2 - c)) <= 2


def test_negligible_component_barely_changes_the_table():
    base = E.mix_table([12, 12, 12], [50, 50, 50], [0, 0, 0]).astype(np.int64)
    far = E.mix_table([12, 12, -200], [50, 50, 50], [0, 0, -31]).astype(np.int64)
    w = np.exp(-31 / 4.0) / (2.0 + np.exp(-31 / 4.0))      # weight of the far component
    assert np.max(np.abs(far - base)) / M <= w + (E.NSYM + 1) / M
    near = E.mix_table([12, 12, -200], [50, 50, 50], [0, 0, 0]).astype(np.int64)
    # a full-weight one moves the CDF by a third of the difference of the two
    # logistics (FP64), up to the tables' quantisation
    d64 = np.max(np.abs(np.cumsum(E.mix_probs64([12, 12, -200], [50, 50, 50], [0, 0, 0]))
                        - np.cumsum(E.mix_probs64([12] * 3, [50] * 3, [0] * 3))))
    assert d64 > 0.15
    assert abs(np.max(np.abs(near - base)) / M - d64) <= 2 * (E.NSYM + 1) / M


def test_mixture_decision_hand_worked_values():
    # w: components 1 and 2 tie at the maximum -> the first (1) is the reference
    head = np.array([0.1, 0.3, 0.3,  # w
                     -4.0, 2.5, 7.9,  # mu
                     0.0, 30.0, -30.0])  # rho
    ctr, q, j, g = E.mix_decision(E.mix_params(head))
    assert ctr == 2                              # rint(2.5) = 2 (half to even)
    assert list(q) == [-48, 4, 47]               # rint(8 (mu - 2)): -48, 4, 47.2 -> 47
    assert list(g) == [-1, 0, 0]                 # rint(4 (w - 0.3)) = rint(-0.8) = -1
    assert j[0] == E.sigma_bin(np.float32(np.log(2.0)))
    # scale 30: log2(30 / 0.125) = 7.9 octaves of 8 bins -> bin 63; ~1e-13 -> bin 0
    assert j[1] == 63 == E.sigma_bin(np.float32(30.0)) and j[2] == 0
    # reference component 2 (largest w): ctr = -400; offsets and log-weights clamp
    far = np.array([0.0, -20.0, 1.0, 0.0, 400.0, -400.0, 1.0, 1.0, 1.0])
    ctr, q, j, g = E.mix_decision(E.mix_params(far))
    assert ctr == -400 and list(q) == [255, 255, 0] and list(g) == [-4, -31, 0]


def test_mixture_params_softplus():
    p = E.mix_params([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 0.0, 25.0, -40.0])
    assert list(p[:6]) == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    assert p[6] == np.log(2.0) and p[7] == 25.0
    assert abs(p[8] / np.exp(-40.0) - 1.0) < 1e-12


def test_mixture_near_tie_flags_boundaries():
    # parameters (w, mu, sigma); sigma 1.3 lies inside a scale bin
    h = np.array([0.0, 0.0, -1.0, 0.0, 0.0, 0.0, 1.3, 1.3, 1.3])
    assert E.mix_near_tie(h, 1e-6)                     # argmax tie
    h = np.array([1.0, 0.0, -1.0, 0.5 + 1e-9, 0.0, 0.0, 1.3, 1.3, 1.3])
    assert E.mix_near_tie(h, 1e-6)                     # mu_a at a half
    h = np.array([1.0, 0.0, -1.0, 0.3, 0.0, 0.0, 1.3, 1.3, 1.3])
    assert not E.mix_near_tie(h, 1e-6)
    h = np.array([1.0, 0.0, -1.0, 0.3, 0.0, 0.0, 1.3, 1.0, 1.3])
    assert E.mix_near_tie(h, 1e-6)                     # sigma 1.0 on a bin edge
    h = np.array([1.0, 0.0, -1.0, 0.3, 0.0625 * (1 + 1e-9), 0.0, 1.3, 1.3, 1.3])
    assert E.mix_near_tie(h, 1e-6)                     # 8 (mu_1 - ctr) at a half
