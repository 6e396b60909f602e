"""Pins of the oracle's level-set update (Eqs. numerical-settings, curva_numer,
dso_evolution): exact derivatives of quadratics, circle curvature, a flat
front's transport distance, and mean-curvature shrinkage of a circle."""
import json
import os

import numpy as np

from oracle import levelset, sdf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_quadratic_derivatives_and_curvature_hand_values():
    """Central differences are exact on quadratics, so at the centre of
    phi = a x + b y + c x^2 + d y^2 + e x y the curvature term is the closed
    form (2c b^2 - 2 a b e + 2d a^2) / (a^2 + b^2); values in the fixture are
    worked by hand from Eq. (curva_numer)."""
    with open(os.path.join(GOLDEN, "curvature_quadratic.json")) as f:
        cases = json.load(f)["cases"]
    y, x = np.mgrid[-3:4, -3:4].astype(np.float64)
    for c in cases:
        a, b, cc, d, e = c["a"], c["b"], c["c"], c["d"], c["e"]
        phi = a * x + b * y + cc * x * x + d * y * y + e * x * y
        px, py, pxx, pyy, pxy = levelset.central_differences(phi)
        assert px[3, 3] == a and py[3, 3] == b
        assert pxx[3, 3] == 2 * cc and pyy[3, 3] == 2 * d and pxy[3, 3] == e
        kc = levelset.curvature_term(phi)[3, 3]
        assert abs(kc - c["Kc"]) <= 1e-12 * max(1.0, abs(c["Kc"]))


def test_circle_distance_curvature_is_inverse_radius():
    n = 160
    cy, cx, R0 = 80.3, 79.6, 12.0
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    rho = np.hypot(y - cy, x - cx)
    phi = rho - R0
    kc = levelset.curvature_term(phi)
    # second-order stencil: |Kc - 1/rho| <= C / rho^3 with C ~ 0.23 (measured
    # bound 0.25), i.e. <= 1e-3 relative from rho = 16 on
    sel = (rho >= 4) & (rho <= 70)
    err = np.abs(kc[sel] - 1.0 / rho[sel])
    assert np.max(err * rho[sel] ** 3) <= 0.25
    far = rho[sel] >= 16
    assert np.max(err[far] * rho[sel][far]) <= 1e-3


def test_straight_edge_has_zero_curvature():
    y, x = np.mgrid[0:32, 0:32].astype(np.float64)
    phi = 0.6 * x - 0.8 * y + 3.0
    kc = levelset.curvature_term(phi)
    assert np.abs(kc[1:-1, 1:-1]).max() <= 1e-14


def test_flat_front_moves_exactly_dt():
    n = 40
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    x0 = 17.25
    phi = x - x0  # inside (phi <= 0) is x <= x0
    V = np.full((n, n), 3.0)  # dL/dM > 0 everywhere: the mask must shrink
    dt = 0.5
    for s in range(1, 5):
        phi, M = levelset.step(phi, V, 3.0, None, dt, 0.0)
        # the zero crossing sits exactly dt*s further inside; the replicated
        # right border holds still and its influence spreads one column per step
        assert np.allclose(phi[:, :n - 1 - s], (x - (x0 - dt * s))[:, :n - 1 - s], atol=1e-12)
    # the other sign grows the mask by the same amount
    phi = x - x0
    phi, _ = levelset.step(phi, -V, 3.0, None, dt, 0.0)
    assert np.allclose(phi[:, 1:n - 1], (x - (x0 + dt))[:, 1:n - 1], atol=1e-12)


def test_zero_velocity_skips_transport():
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((16, 16))
    out, M = levelset.step(phi, np.zeros((16, 16)), 0.0, None, 0.5, 0.0)
    assert np.array_equal(out, phi)
    assert np.array_equal(M, (phi <= 0).astype(np.uint8))


def _radius(phi, cy, cx):
    """Mean sub-pixel zero crossing along the four axis rays from the centre."""
    rs = []
    iy, ix = int(round(cy)), int(round(cx))
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        prof = [phi[iy + dy * t, ix + dx * t] for t in range(0, 60)]
        for t in range(len(prof) - 1):
            if prof[t] <= 0 < prof[t + 1]:
                rs.append(t + prof[t] / (prof[t] - prof[t + 1]))
                break
    return float(np.mean(rs))


def test_circle_shrinks_at_mean_curvature_rate():
    """With V = 0, phi_t = lambda |grad phi| div(grad phi/|grad phi|) is mean
    curvature flow: a circle's radius follows rho(t)^2 = rho0^2 - 2 lambda t."""
    n = 128
    cy = cx = 64.0
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    rho0 = 20.0
    phi = np.hypot(y - cy, x - cx) - rho0
    lam, dt, steps = 1.0, 0.2, 250
    r_start = _radius(phi, cy, cx)
    zeros = np.zeros((n, n))
    for _ in range(steps):
        phi, _ = levelset.step(phi, zeros, 0.0, None, dt, lam)
    r_end = _radius(phi, cy, cx)
    t = dt * steps
    expect_drop = rho0 - np.sqrt(rho0 ** 2 - 2 * lam * t)
    assert abs((r_start - r_end) - expect_drop) <= 0.02 * expect_drop


def test_mask_extraction_ties_inside():
    phi = np.array([[-1.0, 0.0, 1e-30, 2.0]])
    assert levelset.mask_from_phi(phi).tolist() == [[1, 1, 0, 0]]


def test_upwind_kink_follows_hopf_lax_solution():
    """For phi_t + F |grad phi| = 0 with F > 0 the viscosity solution is
    phi(x, t) = min over |y - x| <= F t of phi0(y) (Hopf-Lax): at the bottom of
    the V-shaped phi0 = |x - c| - 5 nothing moves, elsewhere phi drops by F t.
    A downwind (swapped) gradient would lower the bottom by sqrt(2) F t."""
    n = 32
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    c = 15
    phi0 = np.abs(x - c) - 5.0
    dt = 0.5
    V = np.full((n, n), -2.0)  # dL/dM < 0: the mask grows, outward speed F = dt
    phi, _ = levelset.step(phi0, V, 2.0, None, dt, 0.0)
    expect = np.maximum(np.abs(x - c) - dt, 0.0) - 5.0
    assert np.allclose(phi[:, 1:-1], expect[:, 1:-1], atol=1e-12)
