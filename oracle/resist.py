"""Resist models, DSO loss and printability metrics, FP64 (test infrastructure only).

* Constant-threshold resist, Eq. (binary_intensity): Z = [I >= I_th]  (ties print).
* Sigmoid resist, Sec. III-A: Z = 1 / (1 + exp(-sigma_z (I - I_th))).
* L_DSO = alpha L_ilt + beta L_pvb (Sec. III-A), with
      L_ilt = sum (Z_nom - Z_t)^2,
      L_pvb = sum (Z_in - Z_t)^2 + sum (Z_out - Z_t)^2   (summed over pixels).
* Process corners: a dose change d scales the mask amplitude, so the corner
  image is d^2 I; inner corner d_in = 0.98, outer d_out = 1.02 (Sec. II-C
  uses +/-2% dose). With a defocused optical system given (Sec. II-C: the
  inner corner is defocus at -2% dose, the outer nominal focus at +2% dose),
  the inner corner images through it: Z_in = Z(d_in^2 I_def), and
  dL/dI splits into R (for I: nominal and outer terms) and R_def (for I_def).
* R = dL_DSO/dI = sum_c coef_c 2 (Z_c - Z_t) sigma_z Z_c (1 - Z_c) d_c^2,
  the chain factor of Eqs. (ilt_gradient), (pvb_gradient).
* Squared L2 error (Sec. II-C.1): #{ [I >= I_th] != Z_t } (pixels = nm^2 at 1 nm/px).
* PVBand (Sec. II-C.2): #{ [d_in^2 I >= I_th] xor [d_out^2 I >= I_th] }.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ResistParams:
    """Resist and loss constants: sigma_z, I_th (Sec. IV values), loss weights alpha / beta (Sec. III-A), dose corners (Sec. II-C)."""
    sigma_z: float = 50.0     # Sec. IV hyper-parameters
    I_th: float = 0.225
    alpha: float = 1.0
    beta: float = 0.0
    dose_in: float = 0.98
    dose_out: float = 1.02


@dataclass
class ResistResult:
    """L_DSO, its three squared-error terms, dL/dI (and dL/dI_def), and the binary L2 and PVBand counts."""
    loss: float
    loss_terms: tuple  # (sum (Z_nom-Zt)^2, sum (Z_in-Zt)^2, sum (Z_out-Zt)^2)
    R: np.ndarray      # dL/dI
    l2: int
    pvb: int
    R_def: np.ndarray | None = None  # dL/dI_def when a defocused system images the inner corner


def sigmoid_resist(I: np.ndarray, sigma_z: float, I_th: float) -> np.ndarray:
    """Sigmoid resist of Sec. III-A: Z = 1 / (1 + exp(-sigma_z (I - I_th)))."""
    return 1.0 / (1.0 + np.exp(-sigma_z * (I - I_th)))


def threshold_resist(I: np.ndarray, I_th: float) -> np.ndarray:
    """Constant-threshold resist of Sec. II-B: Z = [I >= I_th] (a tie prints)."""
    return (I >= I_th).astype(np.uint8)


def resist(I: np.ndarray, Zt: np.ndarray, p: ResistParams, I_def: np.ndarray | None = None) -> ResistResult:
    """Loss, dL/dI and metrics. With I_def (the defocused system's image) the
    inner corner images through it, and the result carries R_def = dL/dI_def."""
    I = np.asarray(I, dtype=np.float64)
    Id = I if I_def is None else np.asarray(I_def, dtype=np.float64)
    Zt = np.asarray(Zt, dtype=np.float64)
    conds = ((1.0, p.alpha, I, 0), (p.dose_in, p.beta, Id, 1), (p.dose_out, p.beta, I, 0))
    R = [np.zeros_like(I), np.zeros_like(I)]
    terms = []
    loss = 0.0
    for d, coef, img, which in conds:
        Z = sigmoid_resist(d * d * img, p.sigma_z, p.I_th)
        e = Z - Zt
        s = float(np.sum(e * e))
        terms.append(s)
        loss += coef * s
        R[which] += coef * 2.0 * e * p.sigma_z * Z * (1.0 - Z) * d * d
    l2 = int(np.count_nonzero(threshold_resist(I, p.I_th) != Zt.astype(np.uint8)))
    zin = threshold_resist(p.dose_in ** 2 * Id, p.I_th)
    zout = threshold_resist(p.dose_out ** 2 * I, p.I_th)
    pvb = int(np.count_nonzero(zin != zout))
    if I_def is None:
        return ResistResult(loss=loss, loss_terms=tuple(terms), R=R[0] + R[1], l2=l2, pvb=pvb)
    return ResistResult(loss=loss, loss_terms=tuple(terms), R=R[0], l2=l2, pvb=pvb, R_def=R[1])
