"""SOCS lithography imaging and its adjoint, FP64 (test infrastructure only).

Definitions follow Sec. II-B (SOCS approximation of Hopkins imaging) and
Sec. III-A Eq. (ilt_gradient):

* Kernel j lives in the frequency domain on a k x k window W centred on DC:
  ``H[j, a, b]`` is the value at frequency (u, v) = (a - r, b - r).
  Its spatial kernel is h_j = IDFT_n(zero-pad(H_j)) on the n x n torus.
* Coherent field   A_j = M (*) h_j           (circular 2-D convolution)
* Aerial image     I   = sum_j w_j |A_j|^2   (Sec. II-B, N_k terms)
* Gradient of a loss L(I) with R = dL/dI, following Eq. (ilt_gradient):
      dL/dM = sum_j w_j { h'_j (*) [R . (M (*) h*_j)] + (h'_j)* (*) [R . (M (*) h_j)] }
  where h' is the 180-degree rotation of h and h* its conjugate. (The paper
  writes the sigmoid chain factor 2 sigma_z (Z - Z_t) Z (1 - Z) where R
  appears here and leaves the weights and the sum over kernels implicit.)

The convolution is computed with a full-size FFT (numpy.fft), which is exact
for any kernel; the CUDA library uses a different algorithm.
"""
from __future__ import annotations

import numpy as np


def pad_window(Hj: np.ndarray, n: int) -> np.ndarray:
    """Place a k x k centred spectrum into an n x n DFT array (negative
    frequencies wrap to the end, as numpy.fft orders them)."""
    k = Hj.shape[-1]
    r = (k - 1) // 2
    if k > n:
        raise ValueError("window larger than the image")
    out = np.zeros(Hj.shape[:-2] + (n, n), dtype=np.complex128)
    idx = np.arange(-r, r + 1) % n
    out[..., idx[:, None], idx[None, :]] = Hj
    return out


def spatial_kernel(Hj: np.ndarray, n: int) -> np.ndarray:
    """h_j = IDFT_n(zero-padded H_j), complex [n, n] (numpy's 1/n^2 inverse)."""
    return np.fft.ifft2(pad_window(Hj, n))


def conv(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Circular 2-D convolution (x (*) h)(p) = sum_q x(q) h(p - q) on the torus."""
    return np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(h))


def rot180(h: np.ndarray) -> np.ndarray:
    """h'(m) = h(-m) on the torus: the 180-degree rotation of a kernel."""
    return np.roll(np.flip(h, axis=(-2, -1)), shift=(1, 1), axis=(-2, -1))


def coherent_field(M: np.ndarray, Hj: np.ndarray) -> np.ndarray:
    """A_j = M (*) h_j, complex [n, n]."""
    n = M.shape[0]
    return np.fft.ifft2(np.fft.fft2(M) * pad_window(Hj, n))


def aerial(M: np.ndarray, H: np.ndarray, w: np.ndarray) -> np.ndarray:
    """I = sum_j w_j |M (*) h_j|^2  (Sec. II-B), float64 [n, n]."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    Mf = np.fft.fft2(M)
    I = np.zeros((n, n))
    for j in range(H.shape[0]):
        A = np.fft.ifft2(Mf * pad_window(H[j], n))
        I += w[j] * (A.real ** 2 + A.imag ** 2)
    return I


def aerial_gradient(M: np.ndarray, R: np.ndarray, H: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dL/dM for a loss with dL/dI = R, in the two-term form of Eq. (ilt_gradient).

    Returns float64 [n, n]. The two terms are complex conjugates of each other
    for a real mask; their sum is real and the (rounding-level) imaginary part
    is dropped.
    """
    M = np.asarray(M, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    n = M.shape[0]
    V = np.zeros((n, n))
    for j in range(H.shape[0]):
        h = spatial_kernel(H[j], n)
        hr = rot180(h)
        t1 = conv(hr, R * conv(M, np.conj(h)))
        t2 = conv(np.conj(hr), R * conv(M, h))
        V += w[j] * (t1 + t2).real
    return V


def conv_adjoint(y: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Adjoint of x -> x (*) h under <a, b> = sum conj(a) b: y -> y (*) conj(h'),
    with h' the 180-degree rotation."""
    return conv(y, np.conj(rot180(h)))
