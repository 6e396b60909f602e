"""Pins of the oracle's WENO5 upwind derivatives (the optional scheme for
|grad phi| of Sec. III-C): exactness on quadratics (every ENO candidate is
exact, whatever the weights), fifth-order convergence on a smooth profile (the
nonlinear weights reach the ideal ones), no overshoot at a kink, and the flat
front moving exactly dt like the first-order scheme."""
import numpy as np

from oracle import levelset


def test_weno_derivatives_exact_on_quadratics():
    n = 32
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    phi = 0.3 * x * x - 0.2 * y * y + 0.1 * x * y + 2 * x - y + 5
    dmx, dpx, dmy, dpy = levelset.weno5_derivatives(phi)
    ex = 0.6 * x + 0.1 * y + 2
    ey = -0.4 * y + 0.1 * x - 1
    inner = (slice(4, -4), slice(4, -4))  # away from the replicated border
    for d, e in ((dmx, ex), (dpx, ex), (dmy, ey), (dpy, ey)):
        assert np.abs(d - e)[inner].max() <= 1e-12


def _err(n, period, axis):
    t = np.arange(n, dtype=np.float64)
    w = 2 * np.pi / period
    prof = np.sin(w * t)
    phi = np.tile(prof, (8, 1)) if axis == 1 else np.tile(prof[:, None], (1, 8))
    dmx, dpx, dmy, dpy = levelset.weno5_derivatives(phi)
    exact = w * np.cos(w * t)
    if axis == 1:
        d1, d2, ex = dmx[:, 4:-4], dpx[:, 4:-4], np.tile(exact, (8, 1))[:, 4:-4]
    else:
        d1, d2, ex = dmy[4:-4, :], dpy[4:-4, :], np.tile(exact[:, None], (1, 8))[4:-4, :]
    return max(np.abs(d1 - ex).max(), np.abs(d2 - ex).max()) / w


def test_weno_fifth_order_convergence():
    """Halving the grid spacing (per period) divides the error by about 2^5."""
    for axis in (0, 1):
        e1, e2, e3 = _err(64, 16, axis), _err(128, 32, axis), _err(256, 64, axis)
        assert e1 / e2 > 24 and e2 / e3 > 24, (e1, e2, e3)


def test_weno_no_overshoot_at_a_kink():
    n = 40
    x = np.arange(n, dtype=np.float64)
    phi = np.tile(np.abs(x - 17.3), (4, 1))
    dmx, dpx, _, _ = levelset.weno5_derivatives(phi)
    for d in (dmx, dpx):
        assert d.min() >= -1 - 1e-9 and d.max() <= 1 + 1e-9


def test_weno_flat_front_moves_exactly_dt():
    n = 24
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    phi = x - 11.5
    V = -np.ones((n, n))  # V < 0: the mask grows, the front moves towards +x
    out, _ = levelset.step(phi, V, 1.0, None, 0.5, 0.0, weno=True)
    inner = (slice(None), slice(4, -4))
    assert np.abs(out - (phi - 0.5))[inner].max() <= 1e-12
