"""Supervision of the modulation branch, FP64 (test infrastructure only).

Sec. III-B (modulation branch supervision): the curvature modulation m_theta of
Eq. (dso_evolution) is learned from a label found by search. The converged level set
phi_gt of a clip is shifted by distances dh drawn uniformly from [-20, 20]; each shift
gives a candidate map m~ = H(phi_gt + dh) with the Heaviside H(z) = 1 for z >= 0, else 0
(Eq. heaviside); the label m_gt is the candidate whose DSO run gives the smallest
L_DSO. The branch is trained through the approximated Heaviside
H_eps(phi) = (1 + (2 / pi) atan(phi / eps)) / 2 with the loss
L_m = sum over pixels of (H_eps(phi_m) - m_gt)^2 (Sec. III-B; eps = 0.03 in Sec. IV).

Readings: each candidate's DSO run starts from the TSDF of the target with the
solver's parameters and m = m~; "smallest L_DSO" compares the loss of the final
mask (the last history entry); ties go to the first candidate.
"""
from __future__ import annotations

import numpy as np

from . import solve


def candidates(phi_gt: np.ndarray, dh) -> np.ndarray:
    """[len(dh), n, n] candidate maps H(phi_gt + dh_j) as 0.0 / 1.0."""
    phi = np.asarray(phi_gt, dtype=np.float64)
    return np.stack([(phi + float(d) >= 0.0).astype(np.float64) for d in dh])


def search(Zt, H, w, p: solve.SolveParams, phi_gt, dh, defocus=None):
    """Returns (index of m_gt, the candidates' final L_DSO, the candidates)."""
    cands = candidates(phi_gt, dh)
    losses = [solve.ilt_solve(Zt, H, w, p, m=c, defocus=defocus).loss[-1] for c in cands]
    return int(np.argmin(losses)), losses, cands


def ahf(phi, eps: float) -> np.ndarray:
    """Approximated Heaviside H_eps(phi) = (1 + (2/pi) atan(phi/eps)) / 2."""
    return 0.5 * (1.0 + (2.0 / np.pi) * np.arctan(np.asarray(phi, dtype=np.float64) / eps))


def ahf_loss(phi_m, m_gt, eps: float):
    """L_m = sum (H_eps(phi_m) - m_gt)^2 and dL_m/dphi_m."""
    phi = np.asarray(phi_m, dtype=np.float64)
    r = ahf(phi, eps) - np.asarray(m_gt, dtype=np.float64)
    dH = (1.0 / np.pi) * eps / (eps * eps + phi * phi)   # d/dphi of H_eps
    return float(np.sum(r * r)), 2.0 * r * dH
