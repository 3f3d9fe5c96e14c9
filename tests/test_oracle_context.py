"""Pins of the oracle's context model (Section 3.2, Figs. 3-5).

The four-step partition is checked against the properties the text states
(a quarter of the positions per step, 0/2/6/8 available neighbours in a 3x3
window); causality is checked by brute force; the ConvLSTM cell against the
closed forms its defining equations give for saturated gates; the
autoregressive LL model's sequential evaluation against its masked-conv
evaluation.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import context as CX
from oracle.context import ContextModel, step_map
from tests._lib import golden


def test_steps_tile_every_position_once_with_quarter_density():
    for h, w in [(8, 8), (16, 24), (7, 13), (1, 1), (2, 5)]:
        sm = step_map(h, w)
        assert sm.shape == (h, w) and set(np.unique(sm)) <= {0, 1, 2, 3}
        if h % 2 == 0 and w % 4 == 0:
            counts = [np.count_nonzero(sm == k) for k in range(4)]
            assert counts == [h * w // 4] * 4
    sm = step_map(8, 8)
    # steps 1 and 2 together are the even columns (half available before step 3)
    assert np.all((sm < 2) == (np.arange(8)[None, :] % 2 == 0))


def test_neighbour_counts_match_the_paper():
    # tests/golden/four_step_neighbours.txt: the counts Sec. 3.2 prints
    g = golden("four_step_neighbours.txt")
    per_step = g["available_per_step"][0]
    assert per_step == [0, 2, 6, 8]
    sm = step_map(16, 16)
    seen = []
    for k, expect in enumerate(per_step):
        ys, xs = np.nonzero(sm == k)
        assert ys.size * g["positions_per_step_fraction_inverse"][0][0] == sm.size
        for y, x in zip(ys, xs):
            if 1 <= y < 15 and 1 <= x < 15:
                win = sm[y - 1:y + 2, x - 1:x + 2]
                avail = np.count_nonzero(win < k)
                assert avail == expect, (k, y, x, avail)
                seen.append(avail)
    assert np.mean(seen) == g["mean_available"][0][0]


def _cm(C=8, ll_mode=0, seed=0):
    cfg = S.ModelConfig(levels=4, C=C, ll_mode=ll_mode)
    t = {k: v.astype(np.float64) for k, v in S.random_model(cfg, seed).items()}
    return ContextModel(t, C, ll_mode)


@pytest.mark.parametrize("ns", ["sb", "ll"])
def test_step_params_are_causal_brute_force(ns):
    cm = _cm(C=4)
    rng = np.random.default_rng(0)
    H, W = 8, 8
    s = rng.integers(-5, 6, (H, W)).astype(np.float64)
    l = rng.normal(size=(H, W, 4)) if ns == "sb" else np.zeros((H, W, 4))
    sm = step_map(H, W)
    for k in range(4):
        mu0, sg0 = cm.step_params(k, s, l, ns)
        for y in range(H):
            for x in range(W):
                if sm[y, x] < k:
                    continue
                s2 = s.copy()
                s2[y, x] += 17.0
                mu1, sg1 = cm.step_params(k, s2, l, ns)
                sel = sm == k
                assert np.array_equal(mu0[sel], mu1[sel])
                assert np.array_equal(sg0[sel], sg1[sel])
    # and positions of earlier steps do matter (the mask is not all zero)
    mu0, _ = cm.step_params(3, s, l, ns)
    s2 = s.copy(); s2[sm == 0] += 9.0
    mu1, _ = cm.step_params(3, s2, l, ns)
    assert not np.array_equal(mu0[sm == 3], mu1[sm == 3])


def _lstm_zero_weights(C):
    t = {"lstm.we": np.zeros((C, 1, 3, 3)), "lstm.be": np.zeros(C),
         "lstm.wg": np.zeros((4 * C, 2 * C, 3, 3)), "lstm.bg": np.zeros(4 * C)}
    return ContextModel(t, C, 0)


def test_lstm_cell_closed_forms_for_saturated_gates():
    """ConvLSTM (Shi et al. 2015): c' = f c + i g, h' = o tanh(c').
    Gate order i, f, o, g. With weights zero the gates are the biases:
    (a) i = 0, f = 1 keeps the cell; (b) i = 1, f = 0 replaces it by
    tanh(b_g); the output gate scales tanh(c')."""
    C = 3
    cm = _lstm_zero_weights(C)
    big = 60.0
    s_prev = np.zeros((2, 2))
    c0 = np.arange(12, dtype=np.float64).reshape(2, 2, 3) / 10.0 - 0.5
    h0 = np.zeros((2, 2, C))
    bg = cm.t["lstm.bg"]
    bg[0:C] = -big; bg[C:2 * C] = big; bg[2 * C:3 * C] = big; bg[3 * C:] = 0.3
    h, c = cm.lstm(s_prev, h0, c0, up=False)
    np.testing.assert_allclose(c, c0, atol=1e-15)
    np.testing.assert_allclose(h, np.tanh(c0), atol=1e-15)
    bg[0:C] = big; bg[C:2 * C] = -big; bg[2 * C:3 * C] = 0.0; bg[3 * C:] = 0.7
    h, c = cm.lstm(s_prev, h0, c0, up=False)
    np.testing.assert_allclose(c, np.full_like(c0, np.tanh(0.7)), atol=1e-15)
    np.testing.assert_allclose(h, 0.5 * np.tanh(np.tanh(0.7)), atol=1e-15)


def test_lstm_upsamples_previous_state_nearest():
    C = 2
    cm = _lstm_zero_weights(C)
    big = 60.0
    bg = cm.t["lstm.bg"]
    bg[0:C] = -big; bg[C:2 * C] = big; bg[2 * C:3 * C] = big
    c0 = np.random.default_rng(1).normal(size=(2, 3, C))
    h, c = cm.lstm(np.zeros((2, 3)), np.zeros((2, 3, C)), c0, up=True)
    assert c.shape == (4, 6, C)
    for y in range(4):
        for x in range(6):
            np.testing.assert_allclose(c[y, x], c0[y // 2, x // 2], atol=1e-15)


def test_lstm_input_conv_reads_previous_subband():
    """A 3x3 input filter that is an impulse at the centre makes e equal the
    previous subband; with i = 1, f = 0, o = 1 and the g-gate weight on e
    equal to 1, c' = tanh(s_prev)."""
    C = 1
    cm = _lstm_zero_weights(C)
    big = 60.0
    cm.t["lstm.we"][0, 0, 1, 1] = 1.0
    cm.t["lstm.wg"][3 * C, 0, 1, 1] = 1.0      # g gate <- e (centre tap)
    bg = cm.t["lstm.bg"]
    bg[0:C] = big; bg[C:2 * C] = -big; bg[2 * C:3 * C] = big
    s_prev = np.array([[0.5, -1.0], [2.0, 0.0]])
    h, c = cm.lstm(s_prev, None, None, up=False)
    np.testing.assert_allclose(c[:, :, 0], np.tanh(s_prev), atol=1e-15)
    np.testing.assert_allclose(h[:, :, 0], np.tanh(np.tanh(s_prev)), atol=1e-15)


def test_ar_ll_sequential_equals_masked_conv_and_is_causal():
    cm = _cm(C=6, ll_mode=1)
    rng = np.random.default_rng(2)
    s = rng.integers(-20, 21, (5, 7)).astype(np.float64)
    mu_all, sg_all = cm.ar_params_all(s)
    for y in range(5):
        for x in range(7):
            mu, sg = cm.ar_params_at(s, y, x)
            assert abs(mu - mu_all[y, x]) < 1e-12
            assert abs(sg - sg_all[y, x]) < 1e-12
            s2 = s.copy()
            flat = s2.reshape(-1)
            flat[y * 7 + x:] += 11.0      # current and later positions
            mu2, sg2 = cm.ar_params_at(s2, y, x)
            assert mu2 == mu and sg2 == sg


def test_depthwise_matches_per_channel_scipy():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(3)
    x = rng.normal(size=(6, 5, 4)); w = rng.normal(size=(4, 3, 3)); b = rng.normal(size=4)
    out = CX.depthwise3x3(x, w, b)
    for c in range(4):
        ref = b[c] + correlate2d(x[:, :, c], w[c], mode="same")
        np.testing.assert_allclose(out[:, :, c], ref, atol=1e-12)
