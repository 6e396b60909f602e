"""Level-set update, FP64 (test infrastructure only).

* Mask from the level-set function, Eq. (phi2mask): M = 1 where phi <= 0.
* Central differences of Eq. (numerical-settings) (compact 3-point second
  derivatives, 4-point mixed derivative), x along image columns (axis 1) and
  y along rows (axis 0); borders replicate the edge pixel.
* Curvature term of Eq. (curva_numer) without its lambda m prefactor:
      Kc = (phi_xx phi_y^2 - 2 phi_x phi_y phi_xy + phi_yy phi_x^2) / (phi_x^2 + phi_y^2),
  which equals |grad phi| div(grad phi / |grad phi|); Kc = 0 where
  phi_x^2 + phi_y^2 < 1e-12 (the paper leaves that case open).
* Update, Eqs. (levelset_evolution), (dso_evolution) with the descent sign:
  the mask grows where dL/dM < 0, so the transport speed along the outward
  normal is F = -dt V / max|V| (Sec. III-C sets the step from max|v|), and
      phi <- phi - [max(F, 0) |grad phi|^+ + min(F, 0) |grad phi|^-]
                 + dt lambda m Kc,
  with Godunov's first-order upwind gradient magnitudes
      |grad|^+ = sqrt(max(D-x,0)^2 + min(D+x,0)^2 + max(D-y,0)^2 + min(D+y,0)^2)
      |grad|^- = sqrt(min(D-x,0)^2 + max(D+x,0)^2 + min(D-y,0)^2 + max(D+y,0)^2).
  When max|V| = 0 the transport term is skipped.
* Optional fifth-order WENO one-sided derivatives in place of D-/D+ (Sec.
  III-C names WENO for |grad phi| without giving the scheme): the
  Hamilton-Jacobi WENO of Jiang & Shu / Jiang & Peng, three third-order ENO
  candidates on the one-sided differences v1..v5 combined with the weights
  0.1, 0.6, 0.3 modulated by the smoothness indicators, eps = 1e-6 max v_k^2
  + 1e-99. Borders replicate the edge pixel (three ghost cells).
"""
from __future__ import annotations

import numpy as np

KC_EPS = 1e-12


def mask_from_phi(phi: np.ndarray) -> np.ndarray:
    """Eq. (phi2mask): 1 where phi <= 0 (ties are inside)."""
    return (np.asarray(phi) <= 0).astype(np.uint8)


def _pad(phi):
    """Replicate-edge ghost pixels for the stencils (Neumann borders; the paper states no border rule)."""
    return np.pad(np.asarray(phi, dtype=np.float64), 1, mode="edge")


def central_differences(phi: np.ndarray):
    """(phi_x, phi_y, phi_xx, phi_yy, phi_xy) of Eq. (numerical-settings)."""
    P = _pad(phi)
    c = P[1:-1, 1:-1]
    xp, xm = P[1:-1, 2:], P[1:-1, :-2]
    yp, ym = P[2:, 1:-1], P[:-2, 1:-1]
    px = 0.5 * (xp - xm)
    py = 0.5 * (yp - ym)
    pxx = xp + xm - 2.0 * c
    pyy = yp + ym - 2.0 * c
    pxy = 0.25 * ((P[2:, 2:] - P[2:, :-2]) - (P[:-2, 2:] - P[:-2, :-2]))
    return px, py, pxx, pyy, pxy


def curvature_term(phi: np.ndarray) -> np.ndarray:
    """|grad phi| div(grad phi / |grad phi|) per Eq. (curva_numer)."""
    px, py, pxx, pyy, pxy = central_differences(phi)
    den = px * px + py * py
    num = pxx * py * py - 2.0 * px * py * pxy + pyy * px * px
    out = np.zeros_like(den)
    ok = den >= KC_EPS
    out[ok] = num[ok] / den[ok]
    return out


def upwind_gradients(phi: np.ndarray):
    """Godunov upwind |grad phi|^+ and |grad phi|^- (one-sided differences)."""
    P = _pad(phi)
    c = P[1:-1, 1:-1]
    dmx = c - P[1:-1, :-2]
    dpx = P[1:-1, 2:] - c
    dmy = c - P[:-2, 1:-1]
    dpy = P[2:, 1:-1] - c
    gp = np.sqrt(np.maximum(dmx, 0) ** 2 + np.minimum(dpx, 0) ** 2
                 + np.maximum(dmy, 0) ** 2 + np.minimum(dpy, 0) ** 2)
    gm = np.sqrt(np.minimum(dmx, 0) ** 2 + np.maximum(dpx, 0) ** 2
                 + np.minimum(dmy, 0) ** 2 + np.maximum(dpy, 0) ** 2)
    return gp, gm


def weno5_combine(v1, v2, v3, v4, v5):
    """WENO5 derivative from the five one-sided differences (v3 nearest the node on
    the upwind side): the three ENO candidates and their nonlinear weights."""
    p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
    p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
    p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
    s1 = 13.0 / 12.0 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - 4 * v2 + 3 * v3) ** 2
    s2 = 13.0 / 12.0 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    s3 = 13.0 / 12.0 * (v3 - 2 * v4 + v5) ** 2 + 0.25 * (3 * v3 - 4 * v4 + v5) ** 2
    eps = 1e-6 * np.maximum.reduce([v1 * v1, v2 * v2, v3 * v3, v4 * v4, v5 * v5]) + 1e-99
    a1 = 0.1 / (s1 + eps) ** 2
    a2 = 0.6 / (s2 + eps) ** 2
    a3 = 0.3 / (s3 + eps) ** 2
    return (a1 * p1 + a2 * p2 + a3 * p3) / (a1 + a2 + a3)


def weno5_derivatives(phi: np.ndarray):
    """(D-x, D+x, D-y, D+y) by WENO5; x along columns, y along rows."""
    P = np.pad(np.asarray(phi, dtype=np.float64), 3, mode="edge")
    n0, n1 = np.asarray(phi).shape

    def sl(dy, dx):
        return P[3 + dy:3 + dy + n0, 3 + dx:3 + dx + n1]

    def axis_pair(shift):
        # d(k) = phi(k) - phi(k - 1) along the axis, k relative to the node
        d = {k: shift(k) - shift(k - 1) for k in range(-2, 4)}
        minus = weno5_combine(d[-2], d[-1], d[0], d[1], d[2])
        plus = weno5_combine(d[3], d[2], d[1], d[0], d[-1])
        return minus, plus

    dmx, dpx = axis_pair(lambda k: sl(0, k))
    dmy, dpy = axis_pair(lambda k: sl(k, 0))
    return dmx, dpx, dmy, dpy


def upwind_gradients_weno5(phi: np.ndarray):
    """Godunov |grad phi|^+ and |grad phi|^- with WENO5 one-sided derivatives."""
    dmx, dpx, dmy, dpy = weno5_derivatives(phi)
    gp = np.sqrt(np.maximum(dmx, 0) ** 2 + np.minimum(dpx, 0) ** 2
                 + np.maximum(dmy, 0) ** 2 + np.minimum(dpy, 0) ** 2)
    gm = np.sqrt(np.minimum(dmx, 0) ** 2 + np.maximum(dpx, 0) ** 2
                 + np.minimum(dmy, 0) ** 2 + np.maximum(dpy, 0) ** 2)
    return gp, gm


def step(phi: np.ndarray, V: np.ndarray, vmax: float, m, dt: float, lam: float, weno: bool = False):
    """One explicit level-set update (first-order Godunov, or WENO5 derivatives in the
    Godunov flux). Returns (phi_next, mask_next)."""
    phi = np.asarray(phi, dtype=np.float64)
    out = phi.copy()
    if vmax > 0:
        F = -dt * np.asarray(V, dtype=np.float64) / vmax
        gp, gm = upwind_gradients_weno5(phi) if weno else upwind_gradients(phi)
        out -= np.maximum(F, 0.0) * gp + np.minimum(F, 0.0) * gm
    if lam != 0.0:
        mm = 1.0 if m is None else np.asarray(m, dtype=np.float64)
        out += dt * lam * mm * curvature_term(phi)
    return out, mask_from_phi(out)
