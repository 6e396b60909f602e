"""Seeded synthetic inputs for the level-set ILT hot path.

This module only *draws inputs*: binary target clips and the optical kernel
set (H_k, w_k) of a synthetic Hopkins imaging system. It contains none of the
method's arithmetic (no imaging, no loss, no level-set update, no distance
transform), so both the FP64 oracle and the CUDA path may use it.

Workloads (all at 1 nm per pixel):

* ``rect_clip``      -- 256^2 clips of 3-6 axis-aligned rectangles (short side
  8-24 px, long side 8-96 px, Euclidean gap >= 8 px, >= 16 px from the border).
* ``manhattan_clip`` -- 2048^2 metal-layer clips: horizontal preferred-direction
  wires 60-120 nm wide and 200-1500 nm long, occasional vertical stubs, spacing
  >= 70 nm between distinct shapes, pattern density drawn from U[20%, 40%].
  They stand in for the ten ICCAD-2013 M1 clips the paper evaluates on
  (Sec. IV), which are not reproduced here.
* ``optics``         -- the top-K eigenpairs of a transmission cross
  coefficient (TCC) built from a circular pupil and an annular source
  (sigma 0.6-0.9); the paper uses K = 24 SOCS kernels (Sec. II-B).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rect_clip",
    "manhattan_clip",
    "optics",
    "Optics",
    "window_radius_for",
    "random_kernels",
]


# --------------------------------------------------------------------------
# target clips
# --------------------------------------------------------------------------

def _rect_gap(a, b):
    """Euclidean distance between two pixel rectangles (y0, y1, x0, x1) that
    cover the half-open pixel ranges [y0, y1) x [x0, x1), taken as continuous
    sets (pixel i spans [i, i + 1]): along an axis it is the number of empty
    pixels between them."""
    dy = max(0, max(a[0], b[0]) - min(a[1], b[1]))
    dx = max(0, max(a[2], b[2]) - min(a[3], b[3]))
    return math.hypot(dy, dx)


def rect_clip(seed: int, n: int = 256, nrect=(3, 6), short=(8, 24), long=(8, 96),
              gap: float = 8.0, border: int = 16, max_tries: int = 10000) -> np.ndarray:
    """A binary clip of ``nrect`` random axis-aligned rectangles.

    Returns ``uint8[n, n]`` (1 = pattern). Rectangles keep a Euclidean gap of
    at least ``gap`` pixels between each other and stay ``border`` pixels
    away from the clip edge.
    """
    rng = np.random.default_rng(seed)
    count = int(rng.integers(nrect[0], nrect[1] + 1))
    rects = []
    tries = 0
    while len(rects) < count and tries < max_tries:
        tries += 1
        s = int(rng.integers(short[0], short[1] + 1))
        l = int(rng.integers(max(long[0], 1), long[1] + 1))
        h, wdt = (s, l) if rng.random() < 0.5 else (l, s)
        if h > n - 2 * border or wdt > n - 2 * border:
            continue
        y0 = int(rng.integers(border, n - border - h + 1))
        x0 = int(rng.integers(border, n - border - wdt + 1))
        r = (y0, y0 + h, x0, x0 + wdt)
        if all(_rect_gap(r, q) >= gap for q in rects):
            rects.append(r)
    z = np.zeros((n, n), np.uint8)
    for (y0, y1, x0, x1) in rects:
        z[y0:y1, x0:x1] = 1
    return z


def manhattan_clip(seed: int, n: int = 2048, width=(60, 120), length=(200, 1500),
                   space: int = 70, density=(0.20, 0.40), margin: int = 64,
                   stub_prob: float = 0.25, max_attempts: int = 40) -> np.ndarray:
    """A seed-generated Manhattan metal-layer clip, ``uint8[n, n]``.

    Horizontal wires are laid on tracks; each track holds wire segments of
    width U{width} and length U{length} separated by end-to-end gaps of at
    least ``space``. Track pitch is chosen so that the drawn density target
    (U[density]) is met; some wires get a vertical stub (width U{width}) into
    the free space above or below. Every pair of distinct shapes keeps a
    Euclidean spacing >= ``space`` (checked rectangle to rectangle). The
    clip is regenerated from the same stream until its density is within
    0.02 of the target (the closest attempt is kept otherwise).
    """
    rng = np.random.default_rng(seed)
    target = float(rng.uniform(density[0], density[1]))
    best, best_err = None, 1e9
    for _ in range(max_attempts):
        z = _manhattan_attempt(rng, n, width, length, space, target, margin, stub_prob)
        err = abs(z.mean() - target)
        if err < best_err:
            best, best_err = z, err
        if err <= 0.02:
            break
    return best


def _manhattan_attempt(rng, n, width, length, space, target, margin, stub_prob):
    lo, hi = margin, n - margin
    shapes = []  # list of lists of rects (y0, y1, x0, x1); a shape = wire + optional stub
    fill = 0.72  # expected fraction of a track covered by wire
    y = lo
    tracks = []
    while True:
        w = int(rng.integers(width[0], width[1] + 1))
        if y + w > hi:
            break
        tracks.append((y, w))
        pitch = w * fill / max(target, 1e-3)
        gap_y = max(space, int(round(pitch - w + rng.uniform(-0.25, 0.25) * w)))
        y = y + w + gap_y
    for (ty, w) in tracks:
        x = lo + int(rng.integers(0, 200))
        while True:
            L = int(rng.integers(length[0], length[1] + 1))
            if x + L > hi:
                L = hi - x
                if L < length[0]:
                    break
            shapes.append([(ty, ty + w, x, x + L)])
            x = x + L + space + int(rng.integers(0, 300))
            if x >= hi - length[0]:
                break
    # vertical stubs (jogs) into the free space next to a wire
    all_rects = [(si, r) for si, s in enumerate(shapes) for r in s]
    for si in range(len(shapes)):
        if rng.random() >= stub_prob:
            continue
        wy0, wy1, wx0, wx1 = shapes[si][0]
        sw = int(rng.integers(width[0], width[1] + 1))
        if wx1 - wx0 < sw:
            continue
        sx0 = int(rng.integers(wx0, wx1 - sw + 1))
        sl = int(rng.integers(60, 400))
        if rng.random() < 0.5:
            stub = (max(lo, wy0 - sl), wy0, sx0, sx0 + sw)
        else:
            stub = (wy1, min(hi, wy1 + sl), sx0, sx0 + sw)
        if stub[1] - stub[0] < 20:
            continue
        ok = True
        for (sj, r) in all_rects:
            if sj == si:
                continue
            if _rect_gap(stub, r) < space:
                ok = False
                break
        if ok:
            shapes[si].append(stub)
            all_rects.append((si, stub))
    z = np.zeros((n, n), np.uint8)
    for s in shapes:
        for (y0, y1, x0, x1) in s:
            z[y0:y1, x0:x1] = 1
    return z


# --------------------------------------------------------------------------
# optics: synthetic Hopkins TCC -> SOCS kernels
# --------------------------------------------------------------------------

@dataclass
class Optics:
    """A SOCS kernel set on a k x k low-frequency window.

    ``H[j, a, b]`` is the spectrum of kernel j at frequency (u, v) =
    (a - r, b - r), r = (k - 1) / 2, where u runs along image rows (axis 0)
    and v along columns (axis 1), in units of 1/n cycles per pixel.
    ``w[j]`` are the non-negative SOCS weights (TCC eigenvalues), sorted in
    decreasing order. ``tcc`` is the full k^2 x k^2 TCC the kernels came from
    (row/column index a * k + b).
    """
    n: int
    k: int
    H: np.ndarray  # complex128 [K, k, k]
    w: np.ndarray  # float64 [K]
    tcc: np.ndarray  # complex128 [k*k, k*k]
    f_cut: float  # pupil cutoff in frequency bins

    @property
    def K(self):
        return self.H.shape[0]

    @property
    def r(self):
        return (self.k - 1) // 2


def window_radius_for(n: int, r_ref: int = 17, n_ref: int = 2048) -> int:
    """Window radius at a fixed 1 nm pixel pitch: r scales with the clip side
    (r = ceil(r_ref * n / n_ref)), so that k_n is 11, 19, 27, 35 for n = 512,
    1024, 1536, 2048."""
    return int(math.ceil(r_ref * n / n_ref))


def _tcc(k: int, f_cut: float, sigma_in: float, sigma_out: float, sub: int, defocus: float = 0.0):
    r = (k - 1) // 2
    step = 1.0 / sub
    smax = sigma_out * f_cut
    g = np.arange(-math.ceil(smax / step), math.ceil(smax / step) + 1) * step
    sy, sx = np.meshgrid(g, g, indexing="ij")
    rad = np.hypot(sy, sx)
    sel = (rad >= sigma_in * f_cut - 1e-12) & (rad <= sigma_out * f_cut + 1e-12)
    sy, sx = sy[sel], sx[sel]
    J = np.full(sy.shape, 1.0 / sy.size)
    fu, fv = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    fu, fv = fu.ravel().astype(np.float64), fv.ravel().astype(np.float64)
    # P[s, f] = pupil(f + s): circular, cutoff f_cut, inclusive; optional defocus phase
    # exp(2 pi i W rho^2), rho = |f + s| / f_cut, W in waves at the pupil edge
    rho = np.hypot(fu[None, :] + sy[:, None], fv[None, :] + sx[:, None])
    P = (rho <= f_cut + 1e-12).astype(np.complex128)
    if defocus != 0.0:
        P = P * np.exp(2j * np.pi * defocus * (rho / f_cut) ** 2)
    # TCC(f1, f2) = sum_s J(s) P(f1 + s) conj(P(f2 + s)), Hermitian PSD
    tcc = P.T @ (J[:, None] * np.conj(P))
    return tcc if defocus != 0.0 else tcc.real


def manhattan_clip_bits(seed: int) -> np.ndarray:
    """``manhattan_clip(seed)`` packed eight pixels per byte (``np.packbits``, row-major),
    for handing many clips between processes."""
    return np.packbits(manhattan_clip(seed))


def optics(n: int, K: int, k: int, sigma_in: float = 0.6, sigma_out: float = 0.9,
           sub: int = 4, phase_seed: int | None = 12345, defocus: float = 0.0) -> Optics:
    """SOCS kernels of a synthetic annular-source Hopkins system.

    The pupil is the disc |f| <= f_cut with f_cut = r / (1 + sigma_out), so
    that the TCC support fills the k x k window. The source is uniform on
    sigma_in f_cut <= |s| <= sigma_out f_cut, sampled on a sub-grid of step
    1/``sub`` bin and normalised to unit total power, so a clear field images
    to TCC(0, 0) = 1. Kernels are the top-K eigenvectors (unit norm) times a
    seeded random unit phase each: eigenvector phase is arbitrary, and a
    non-trivial phase keeps the complex arithmetic of every consumer honest.
    ``defocus`` (waves at the pupil edge) adds the phase exp(2 pi i W rho^2) to
    the pupil: the optical system of a defocused process corner.
    """
    if k % 2 != 1:
        raise ValueError("window side k must be odd")
    r = (k - 1) // 2
    f_cut = r / (1.0 + sigma_out)
    tcc = _tcc(k, f_cut, sigma_in, sigma_out, sub, defocus)
    evals, evecs = np.linalg.eigh(tcc)
    order = np.argsort(evals)[::-1][:K]
    w = np.clip(evals[order], 0.0, None)
    H = evecs[:, order].T.reshape(K, k, k).astype(np.complex128)
    if phase_seed is not None:
        rng = np.random.default_rng(phase_seed)
        H = H * np.exp(2j * np.pi * rng.random(K))[:, None, None]
    return Optics(n=n, k=k, H=H, w=w, tcc=tcc.astype(np.complex128), f_cut=f_cut)


def random_kernels(seed: int, K: int, k: int):
    """Arbitrary complex kernel spectra and positive weights (for tests of the
    imaging algebra that must hold for any kernel set)."""
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((K, k, k)) + 1j * rng.standard_normal((K, k, k))
    H /= np.sqrt((np.abs(H) ** 2).sum(axis=(1, 2), keepdims=True))
    w = np.sort(rng.uniform(0.05, 1.0, K))[::-1]
    return H, w


def random_mask(seed: int, n: int, p: float = 0.3) -> np.ndarray:
    """i.i.d. Bernoulli(p) binary mask, uint8[n, n]."""
    rng = np.random.default_rng(seed)
    return (rng.random((n, n)) < p).astype(np.uint8)


def random_field(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, m: int | None = None) -> np.ndarray:
    """Uniform real field float64[n, m or n]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, m if m is not None else n))
