"""Exact squared Euclidean distance transform and the TSDF, FP64 / int64
(test infrastructure only).

Eq. (sdf) defines phi as minus/plus the distance to the boundary curve, and
Eq. (tsdf) clamps it to [D_l, D_u] = [-100, 900]. On a pixel grid the boundary
lies between pixels of opposite class, so the distance is measured between
pixel centres and shifted by half a pixel:

    phi(p) = +(sqrt(d2_1(p)) - 1/2)   where M(p) = 0 (outside),
    phi(p) = -(sqrt(d2_0(p)) - 1/2)   where M(p) = 1 (inside),

where d2_v(p) = min over pixels q with M(q) = v of |p - q|^2 (an exact
integer). A class that is empty gives an infinite distance, hence the clamp
value. This keeps the mask unchanged: [phi <= 0] == M.

The exact transform is computed from its definition, using that the squared
distance separates over the axes:
    d2(y, x) = min_{x'} [ (x - x')^2 + g(y, x')^2 ],
    g(y, x') = min { |y - y'| : M(y', x') = v }.
The brute-force O(n^4) form is kept for pins on small images.
"""
from __future__ import annotations

import numpy as np

INF = np.iinfo(np.int64).max // 4
D_LO, D_HI = -100.0, 900.0  # Eq. (tsdf) bounds from Sec. III-A


def edt_sq_bruteforce(mask: np.ndarray, value: int) -> np.ndarray:
    """d2_v by the definition, O(n^4). INF where no pixel has class ``value``."""
    mask = np.asarray(mask)
    ys, xs = np.nonzero(mask == value)
    h, w = mask.shape
    if ys.size == 0:
        return np.full((h, w), INF, dtype=np.int64)
    yy, xx = np.mgrid[0:h, 0:w]
    d = (yy.ravel()[:, None] - ys[None, :]) ** 2 + (xx.ravel()[:, None] - xs[None, :]) ** 2
    return d.min(axis=1).reshape(h, w).astype(np.int64)


def column_distance(mask: np.ndarray, value: int) -> np.ndarray:
    """g(y, x) = min |y - y'| over M(y', x) = value; INF if the column has none."""
    mask = np.asarray(mask)
    h, w = mask.shape
    g = np.full((h, w), INF, dtype=np.int64)
    ys = np.arange(h)
    for x in range(w):
        pos = np.nonzero(mask[:, x] == value)[0]
        if pos.size == 0:
            continue
        i = np.searchsorted(pos, ys)
        below = pos[np.minimum(i, pos.size - 1)]
        above = pos[np.maximum(i - 1, 0)]
        g[:, x] = np.minimum(np.abs(below - ys), np.abs(ys - above))
    return g


def edt_sq_rows(mask: np.ndarray, value: int, rows=None, g=None) -> np.ndarray:
    """Exact d2_v for the given rows (all rows if None), int64 [len(rows), w]."""
    mask = np.asarray(mask)
    h, w = mask.shape
    if g is None:
        g = column_distance(mask, value)
    rows = np.arange(h) if rows is None else np.asarray(rows)
    x = np.arange(w)
    dx2 = (x[:, None] - x[None, :]) ** 2  # [x, x']
    out = np.empty((rows.size, w), dtype=np.int64)
    for i, y in enumerate(rows):
        gy = g[y]
        fin = gy < INF
        if not fin.any():
            out[i] = INF
            continue
        cand = dx2[:, fin] + (gy[fin] ** 2)[None, :]
        out[i] = cand.min(axis=1)
    return out


def edt_sq(mask: np.ndarray, value: int) -> np.ndarray:
    """Exact squared distance of every pixel to the nearest pixel equal to value (Eq. sdf), all rows."""
    return edt_sq_rows(mask, value)


def opposite_class_d2(mask: np.ndarray, rows=None) -> np.ndarray:
    """Per pixel: squared distance to the nearest pixel of the other class;
    -1 where the other class is empty (the convention of the CUDA scratch)."""
    mask = (np.asarray(mask) != 0).astype(np.uint8)
    d1 = edt_sq_rows(mask, 1, rows)
    d0 = edt_sq_rows(mask, 0, rows)
    m = mask if rows is None else mask[np.asarray(rows)]
    d = np.where(m == 0, d1, d0)
    return np.where(d >= INF, -1, d)


def tsdf(mask: np.ndarray, d_lo: float = D_LO, d_hi: float = D_HI, rows=None) -> np.ndarray:
    """Truncated signed distance, Eqs. (sdf), (tsdf), float64."""
    mask = (np.asarray(mask) != 0).astype(np.uint8)
    d = opposite_class_d2(mask, rows)
    m = mask if rows is None else mask[np.asarray(rows)]
    dist = np.where(d < 0, np.inf, np.sqrt(np.where(d < 0, 0, d).astype(np.float64)) - 0.5)
    phi = np.where(m == 0, dist, -dist)
    return np.clip(phi, d_lo, d_hi)
