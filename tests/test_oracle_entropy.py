"""Pins of the oracle's index decision and CDF table bank.

The tables are checked against the invariants an integer rANS table must
have (strictly increasing, 0 .. M, every frequency >= 1) and against the
FP64 Laplace probabilities of the scale and mean they stand for; the FP32
exponential against numpy's FP64 exp; the index decision against values
worked out by hand from its definition.
"""
import numpy as np
import pytest

from oracle import entropy as E


@pytest.fixture(scope="module")
def bank():
    return E.cdf_bank().astype(np.int64)


def test_bank_shape_and_integer_invariants(bank):
    assert bank.shape == (2048, 128)
    assert np.all(bank[:, 0] == 0)
    assert np.all(bank[:, -1] == E.M)
    f = np.diff(bank, axis=1)
    assert f.min() >= 1


def test_bank_close_to_fp64_laplace(bank):
    worst = 0.0
    for phi in range(-8, 8):
        for j in range(0, 128, 3):
            p = E.laplace_probs64(phi, j)
            f = np.diff(bank[(phi + 8) * 128 + j]) / E.M
            worst = max(worst, float(np.max(np.abs(f - p))))
    assert worst <= (E.NSYM + 1) / E.M


def test_bank_centre_symbol_dominates_for_small_scale(bank):
    # phi = 0, j = 0 (sigma ~ 0.133): almost all mass on r = 0
    f = np.diff(bank[8 * 128 + 0])
    assert np.argmax(f) == E.T + 1
    assert f[E.T + 1] > 0.95 * E.M


def test_exp32_accuracy():
    z = np.linspace(-80.0, 0.0, 200001).astype(np.float32)
    e = E.exp32(z).astype(np.float64)
    r = np.exp(z.astype(np.float64))
    rel = np.abs(e - r) / r
    assert rel.max() < 2.5 * 2.0 ** -23
    assert E.exp32(np.float32(0.0)) == np.float32(1.0)
    assert E.exp32(np.float32(-100.0)) == 0.0


def test_index_decision_hand_values():
    mu = np.array([0.0, 1 / 32, 3 / 32, -0.5, 15 / 32, 17 / 32, 2.0, -3.0 - 1 / 16])
    sg = np.full(mu.shape, 1.0)
    ctr, phi, j = E.index_decision(mu, sg)
    # t = rint(16 mu): 0, 0 (half to even), 2, -8, 8 (7.5 -> 8), 8 (8.5 -> 8), 32, -49
    t = 16 * ctr + phi
    assert list(t) == [0, 0, 2, -8, 8, 8, 32, -49]
    assert list(ctr) == [0, 0, 0, 0, 1, 1, 2, -3]
    assert list(phi) == [0, 0, 2, -8, -8, -8, 0, -1]
    assert np.all((phi >= -8) & (phi <= 7))
    # sigma bins: 8 per octave from 0.125
    s = np.array([1e-3, 0.125, 0.1406249, 0.140625, 0.25, 1.0, 8192.0, 1e9])
    _, _, j = E.index_decision(np.zeros_like(s), s)
    assert list(j) == [0, 0, 0, 1, 8, 24, 127, 127]


def test_bin_representative_inside_its_bin():
    j = np.arange(128)
    rep = E.sigma_of_bin(j)
    assert np.array_equal(E.sigma_bin(rep), j)


def test_near_tie_flags_boundaries():
    assert E.near_tie(np.array([1 / 32 + 1e-9]), np.array([1.03]), 1e-6)[0]
    assert not E.near_tie(np.array([0.01]), np.array([1.03]), 1e-6)[0]
    assert E.near_tie(np.array([0.01]), np.array([1.0]), 1e-6)[0]   # 1.0 is a bin edge
    assert E.near_tie(np.array([0.0]), np.array([0.140625 * (1 + 1e-8)]), 1e-6)[0]
    assert not E.near_tie(np.array([0.0]), np.array([0.13]), 1e-6)[0]
