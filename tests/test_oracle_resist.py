"""Pins of the oracle's resist model, loss and metrics (Sec. II-B, II-C, III-A):
closed forms on constant images and hand-counted metric cases."""
import math

import numpy as np

from oracle import resist


def test_constant_image_closed_form():
    n = 8
    c = 0.23
    I = np.full((n, n), c)
    Zt = np.zeros((n, n), np.uint8)
    Zt[:, :3] = 1
    p = resist.ResistParams(sigma_z=50.0, I_th=0.225, alpha=1.0, beta=7.5)
    out = resist.resist(I, Zt, p)
    loss = 0.0
    R1 = 0.0
    R0 = 0.0
    for d, coef in ((1.0, 1.0), (0.98, 7.5), (1.02, 7.5)):
        z = 1.0 / (1.0 + math.exp(-50.0 * (d * d * c - 0.225)))
        loss += coef * (24 * (z - 1.0) ** 2 + 40 * z ** 2)
        R1 += coef * 2 * (z - 1.0) * 50.0 * z * (1 - z) * d * d
        R0 += coef * 2 * z * 50.0 * z * (1 - z) * d * d
    assert abs(out.loss - loss) <= 1e-14 * loss
    assert np.allclose(out.R[:, :3], R1, rtol=1e-14, atol=0)
    assert np.allclose(out.R[:, 3:], R0, rtol=1e-14, atol=0)
    # c >= I_th prints everywhere at nominal: L2 counts the 40 non-target pixels
    assert out.l2 == 40
    # 0.98^2 * 0.23 = 0.2209 < 0.225 <= 1.02^2 * 0.23 = 0.2393: every pixel is in the band
    assert out.pvb == 64


def test_threshold_tie_prints():
    I = np.array([[0.225, 0.2249999]])
    Zt = np.array([[1, 1]], np.uint8)
    out = resist.resist(I, Zt, resist.ResistParams())
    assert out.l2 == 1  # only the pixel below threshold misses


def test_pvband_hand_count():
    th = 0.225
    # pixel intensities chosen on either side of th/1.02^2 and th/0.98^2
    lo_edge, hi_edge = th / 1.02 ** 2, th / 0.98 ** 2
    vals = np.array([[lo_edge - 1e-4, lo_edge + 1e-4, 0.5 * (lo_edge + hi_edge), hi_edge - 1e-4, hi_edge + 1e-4, 1.0]])
    out = resist.resist(vals, np.zeros_like(vals, np.uint8), resist.ResistParams())
    # printed at the outer corner (1.02^2 I >= th) but not at the inner one
    # (0.98^2 I < th): entries 2, 3 and 4 of the six
    assert out.pvb == 3


def test_beta_zero_drops_corner_terms():
    rng = np.random.default_rng(0)
    I = rng.uniform(0, 0.5, (16, 16))
    Zt = (rng.random((16, 16)) < 0.5).astype(np.uint8)
    a = resist.resist(I, Zt, resist.ResistParams(beta=0.0))
    b = resist.resist(I, Zt, resist.ResistParams(beta=7.5))
    assert abs(a.loss - a.loss_terms[0]) == 0.0
    assert abs(b.loss - (b.loss_terms[0] + 7.5 * (b.loss_terms[1] + b.loss_terms[2]))) <= 1e-13 * b.loss


def test_sigmoid_midpoint_symmetry_and_limits():
    """The sigmoid resist prints half at the threshold, is point-symmetric about it,
    saturates to 0 / 1 within exp(-sigma_z) one unit away, and its slope at the
    threshold is sigma_z / 4 (central difference)."""
    th, sz = 0.225, 50.0
    assert resist.sigmoid_resist(np.array(th), sz, th) == 0.5
    x = np.linspace(-0.3, 0.3, 61)
    s = resist.sigmoid_resist(th + x, sz, th) + resist.sigmoid_resist(th - x, sz, th)
    assert np.allclose(s, 1.0, rtol=0, atol=1e-15)
    assert 1.0 - resist.sigmoid_resist(np.array(th + 1.0), sz, th) <= 1e-21
    assert resist.sigmoid_resist(np.array(th - 1.0), sz, th) < 1e-21
    h = 1e-6
    slope = (resist.sigmoid_resist(np.array(th + h), sz, th) - resist.sigmoid_resist(np.array(th - h), sz, th)) / (2 * h)
    assert abs(slope - sz / 4) <= 1e-6 * sz


def test_saturated_loss_counts_misprinted_pixels():
    """Far above (below) the threshold every corner prints (does not print), so the
    loss is the count of target pixels that disagree, weighted alpha + 2 beta, and
    dL/dI vanishes; the metrics count the same pixels."""
    n = 12
    rng = np.random.default_rng(3)
    Zt = (rng.random((n, n)) < 0.4).astype(np.uint8)
    for level, printed in ((5.0, 1), (-5.0, 0)):
        I = np.full((n, n), level)
        out = resist.resist(I, Zt, resist.ResistParams(alpha=1.0, beta=7.5))
        wrong = int(np.count_nonzero(Zt != printed))
        assert abs(out.loss - (1.0 + 2 * 7.5) * wrong) <= 1e-12 * max(wrong, 1)
        assert np.abs(out.R).max() <= 1e-60
        assert out.l2 == wrong and out.pvb == 0
