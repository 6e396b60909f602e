"""Pins of the oracle's modulation-branch supervision (Sec. III-B): the candidate
maps, the label search and the approximated-Heaviside loss, checked against what the
definitions fix: limits and monotonicity of H(phi + dh), the all-ones candidate
reducing to the unmodulated solve, atan identities of H_eps, and the loss gradient
against finite differences."""
import numpy as np
import pytest

import synth
from oracle import modulation, resist, sdf, solve


def test_candidates_limits_and_monotonicity():
    Zt = synth.rect_clip(2, n=64, border=4)
    phi = sdf.tsdf(Zt, -20.0, 40.0)
    c = modulation.candidates(phi, [-100.0, -5.0, 0.0, 5.0, 100.0])
    assert not c[0].any()                       # far below: no pixel reaches zero
    assert c[-1].all()                          # far above: every pixel
    assert np.all(np.diff(c, axis=0) >= 0)      # grows with dh
    # dh = 0: the pixels with phi >= 0, i.e. the outside of the mask plus its zero set
    assert np.array_equal(c[2], (phi >= 0).astype(float))


def test_all_ones_candidate_is_the_unmodulated_solve():
    n, K, k = 64, 4, 7
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(3, n=n, border=4)
    p = solve.SolveParams(iters=3, resist=resist.ResistParams(beta=1.0))
    plain = solve.ilt_solve(Zt, o.H, o.w, p)
    best, losses, cands = modulation.search(Zt, o.H, o.w, p, plain.phi, [1e6, -1e6])
    assert cands[0].all() and losses[0] == plain.loss[-1]
    # m = 0 switches the curvature term off: the same as lambda = 0
    nolam = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=3, lam=0.0, resist=resist.ResistParams(beta=1.0)))
    assert losses[1] == nolam.loss[-1]
    assert best == int(np.argmin(losses))


def test_ahf_identities():
    eps = 0.03
    phi = np.linspace(-1.0, 1.0, 201)
    h = modulation.ahf(phi, eps)
    assert modulation.ahf(0.0, eps) == 0.5
    assert np.allclose(h + modulation.ahf(-phi, eps), 1.0, rtol=0, atol=1e-15)   # odd part of atan
    assert modulation.ahf(eps, eps) == pytest.approx(0.75)                       # atan(1) = pi/4
    assert np.all(np.diff(h) > 0) and h.min() > 0 and h.max() < 1
    # eps -> 0 tends to the Heaviside step away from zero
    assert np.allclose(modulation.ahf(phi[np.abs(phi) > 0.1], 1e-9), (phi[np.abs(phi) > 0.1] > 0), atol=1e-8)


def test_ahf_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    phi = rng.uniform(-0.2, 0.2, (6, 6))
    m = (rng.random((6, 6)) < 0.5).astype(float)
    L, g = modulation.ahf_loss(phi, m, 0.03)
    h = 1e-7
    for (i, j) in [(0, 0), (2, 3), (5, 1)]:
        e = np.zeros_like(phi)
        e[i, j] = h
        fd = (modulation.ahf_loss(phi + e, m, 0.03)[0] - modulation.ahf_loss(phi - e, m, 0.03)[0]) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # zero exactly when every pixel's H_eps equals its label (m = H_eps(phi))
    assert modulation.ahf_loss(phi, modulation.ahf(phi, 0.03), 0.03)[0] == 0.0
