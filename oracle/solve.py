"""The DevelSet-Optimizer loop, FP64 (test infrastructure only).

Sec. III-A / III-C: starting from phi_0 (the TSDF of the target, or a given
level set), each iteration i
  1. extracts the mask M = [phi <= 0]                        Eq. (phi2mask)
  2. images it, I = sum_j w_j |M (*) h_j|^2                    Sec. II-B
  3. evaluates L_DSO and R = dL/dI at the three dose corners  Sec. III-A
  4. back-propagates V = dL/dM                                 Eqs. (ilt_gradient), (pvb_gradient), (vel)
  5. updates phi by upwind transport + curvature               Eq. (dso_evolution)
     (with ``optimizer="cg"`` the front moves with the conjugate-gradient
     direction D of V instead, Sec. III-C; see ``cg``)
  6. re-initialises phi to the TSDF of its mask when (i + 1) is a multiple
     of ``reinit_every`` (global iteration index, so a split run resumes
     exactly; with CG, when it starts at a multiple of ``reinit_every``).
History entry i holds (L_DSO, L2, PVB) of the mask that iteration i imaged;
entry ``iters`` holds the final mask's.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cg, litho, resist as _resist, levelset, sdf


@dataclass
class SolveParams:
    """Parameters of the DSO loop (Sec. III-C, Sec. IV): resist, dt, lambda, iterations, re-initialisation period, start index, clamp, options."""
    resist: _resist.ResistParams = field(default_factory=_resist.ResistParams)
    dt: float = 0.5
    lam: float = 0.1
    iters: int = 20
    reinit_every: int = 5
    start_iter: int = 0
    d_lo: float = sdf.D_LO
    d_hi: float = sdf.D_HI
    weno: bool = False  # WENO5 one-sided derivatives in the upwind |grad phi|
    optimizer: str = "steepest"  # or "cg": PR+ conjugate-gradient direction (oracle/cg.py)


@dataclass
class SolveResult:
    """Final phi and mask, and per-iteration L_DSO, L2 and PVBand (entry iters: the final mask)."""
    phi: np.ndarray
    mask: np.ndarray
    loss: list
    l2: list
    pvb: list


def iterate(phi, Zt, H, w, p: SolveParams, i: int, m=None, defocus=None, cg_state=None):
    """One DSO iteration at global index i. Returns (phi_next, ResistResult).
    defocus = (H_def, w_def): the inner process corner images through that system.
    cg_state: dict {"V", "D", "first"} carried between iterations when
    p.optimizer == "cg" (updated in place)."""
    M = levelset.mask_from_phi(phi)
    I = litho.aerial(M, H, w)
    if defocus is None:
        res = _resist.resist(I, Zt, p.resist)
        V = litho.aerial_gradient(M, res.R, H, w)
    else:
        Hd, wd = defocus
        res = _resist.resist(I, Zt, p.resist, litho.aerial(M, Hd, wd))
        V = litho.aerial_gradient(M, res.R, H, w) + litho.aerial_gradient(M, res.R_def, Hd, wd)
    if p.optimizer == "cg":
        restart = cg.restarts_at(i, p.reinit_every, cg_state["first"])
        D, _ = cg.direction(V, cg_state["V"], cg_state["D"], restart)
        cg_state.update(V=V, D=D, first=False)
        V = D
    elif p.optimizer != "steepest":
        raise ValueError(f"unknown optimizer {p.optimizer!r}")
    vmax = float(np.abs(V).max())
    phi, M = levelset.step(phi, V, vmax, m, p.dt, p.lam, weno=p.weno)
    if p.reinit_every > 0 and (i + 1) % p.reinit_every == 0:
        phi = sdf.tsdf(M, p.d_lo, p.d_hi)
    return phi, res


def ilt_solve(Zt, H, w, p: SolveParams, phi0=None, m=None, defocus=None) -> SolveResult:
    """The DSO loop of Sec. III-A / III-C from phi0 (default: the TSDF of the target, Eq. tsdf), m the optional modulation map."""
    Zt = (np.asarray(Zt) != 0).astype(np.uint8)
    phi = sdf.tsdf(Zt, p.d_lo, p.d_hi) if phi0 is None else np.asarray(phi0, dtype=np.float64).copy()
    loss, l2, pvb = [], [], []
    cg_state = {"V": None, "D": None, "first": True}
    for t in range(p.iters):
        phi, res = iterate(phi, Zt, H, w, p, p.start_iter + t, m, defocus, cg_state)
        loss.append(res.loss)
        l2.append(res.l2)
        pvb.append(res.pvb)
    M = levelset.mask_from_phi(phi)
    Idef = None if defocus is None else litho.aerial(M, defocus[0], defocus[1])
    res = _resist.resist(litho.aerial(M, H, w), Zt, p.resist, Idef)
    loss.append(res.loss)
    l2.append(res.l2)
    pvb.append(res.pvb)
    return SolveResult(phi=phi, mask=M, loss=loss, l2=l2, pvb=pvb)
