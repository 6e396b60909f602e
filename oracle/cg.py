"""Conjugate-gradient direction for the level-set velocity, FP64 (test infrastructure only).

Sec. III-C: DSO optimises with the conjugate-gradient method of its cited level-set
ILT work and sets the time step by the CFL condition dt = eta / max|v| (Sec. IV:
eta = 0.85). The paper prints no CG update. Reading: nonlinear CG on the velocity
field V_i = dL/dM of iteration i, with the Polak-Ribiere coefficient clipped at zero
(PR+),

    beta_i = max(0, <V_i, V_i - V_{i-1}> / <V_{i-1}, V_{i-1}>)   (0 if <V_{i-1}, V_{i-1}> = 0)
    D_i    = V_i + beta_i D_{i-1},

restarted (beta = 0, D_i = V_i) at the first iteration of a solve and at every
iteration that follows a re-initialisation (the TSDF reshapes phi, so the previous
direction no longer matches it). The level-set step then moves the front with D_i in
place of V_i, normalised by max|D_i|, so the CFL number is the step's dt.
<.,.> is the sum over all pixels.
"""
from __future__ import annotations

import numpy as np


def pr_plus_beta(V: np.ndarray, Vprev: np.ndarray) -> float:
    """Polak-Ribiere coefficient, clipped at zero (PR+)."""
    V = np.asarray(V, dtype=np.float64)
    Vp = np.asarray(Vprev, dtype=np.float64)
    den = float(np.sum(Vp * Vp))
    if den == 0.0:
        return 0.0
    return max(0.0, float(np.sum(V * (V - Vp))) / den)


def direction(V: np.ndarray, Vprev, Dprev, restart: bool):
    """The CG direction of this iteration. Returns (D, beta)."""
    V = np.asarray(V, dtype=np.float64)
    if restart or Vprev is None or Dprev is None:
        return V.copy(), 0.0
    beta = pr_plus_beta(V, Vprev)
    return V + beta * np.asarray(Dprev, dtype=np.float64), beta


def restarts_at(gi: int, reinit_every: int, first: bool) -> bool:
    """Whether global iteration gi restarts CG: the first iteration of a solve, or
    the iteration right after a re-initialisation (gi a multiple of reinit_every)."""
    return first or (reinit_every > 0 and gi % reinit_every == 0)
