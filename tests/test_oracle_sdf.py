"""Pins of the oracle's exact distance transform and TSDF (Eqs. sdf, tsdf):
O(n^4) brute force on small masks (bit-exact integers), hand-worked values,
the clamp, the mask invariant and the unit-gradient property."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import sdf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _masks():
    rng = np.random.default_rng(0)
    out = {
        "random": (rng.random((40, 56)) < 0.3).astype(np.uint8),
        "sparse": (rng.random((64, 64)) < 0.01).astype(np.uint8),
        "empty": np.zeros((17, 23), np.uint8),
        "full": np.ones((19, 13), np.uint8),
        "single": np.zeros((33, 31), np.uint8),
        "checker": (np.add.outer(np.arange(24), np.arange(24)) % 2).astype(np.uint8),
        "rects": synth.rect_clip(3, n=64, nrect=(2, 4), short=(4, 10), long=(4, 30), gap=4, border=2),
    }
    out["single"][20, 7] = 1
    return out


@pytest.mark.parametrize("name", list(_masks().keys()))
@pytest.mark.parametrize("value", [0, 1])
def test_edt_matches_bruteforce_bit_exact(name, value):
    m = _masks()[name]
    assert np.array_equal(sdf.edt_sq(m, value), sdf.edt_sq_bruteforce(m, value))


def test_edt_sampled_rows_match_bruteforce():
    m = synth.random_mask(9, 128, p=0.05)
    rows = [0, 1, 63, 100, 127]
    bf = sdf.edt_sq_bruteforce(m, 1)[rows]
    assert np.array_equal(sdf.edt_sq_rows(m, 1, rows), bf)


def test_tsdf_hand_values():
    with open(os.path.join(GOLDEN, "tsdf_hand.json")) as f:
        g = json.load(f)
    m = np.array(g["mask"], np.uint8)
    phi = sdf.tsdf(m, g["d_lo"], g["d_hi"])
    assert np.allclose(phi, np.array(g["phi"]), rtol=0, atol=1e-15)


def test_tsdf_clamps_and_degenerate_masks():
    assert np.all(sdf.tsdf(np.zeros((9, 9), np.uint8)) == sdf.D_HI)
    assert np.all(sdf.tsdf(np.ones((9, 9), np.uint8)) == sdf.D_LO)
    m = np.zeros((8, 300), np.uint8)
    m[:, 0] = 1
    phi = sdf.tsdf(m, -3.0, 100.0)
    assert phi[0, 299] == 100.0 and phi[0, 0] == -0.5
    assert phi[0, 50] == 49.5


def test_mask_invariant_and_unit_gradient():
    m = synth.rect_clip(5, n=128, border=8)
    phi = sdf.tsdf(m)
    assert np.array_equal((phi <= 0).astype(np.uint8), m)
    d = sdf.opposite_class_d2(m)
    assert np.all(d[m == 0] >= 1) and np.all(d[m == 1] >= 1)
    # away from the medial axis the distance field has |grad| ~ 1
    gy, gx = np.gradient(phi)
    g = np.hypot(gx, gy)
    band = (phi > 2) & (phi < 6)
    assert abs(np.median(g[band]) - 1.0) <= 1e-2
