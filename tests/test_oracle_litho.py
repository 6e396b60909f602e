"""Pins of the oracle's SOCS imaging and gradient (Sec. II-B, Eq. ilt_gradient).

Each test checks the oracle against something it does not compute itself:
a brute-force spatial convolution, a closed form (clear field, pinhole,
Parseval), the Hopkins bilinear form built from the TCC, or an exact identity
of a quadratic map.
"""
import numpy as np
import pytest

import synth
from oracle import litho, resist


def brute_conv(x, h):
    """(x (*) h)(p) = sum_q x(q) h(p - q) on the torus, by the definition."""
    n = x.shape[0]
    out = np.zeros((n, n), dtype=np.complex128)
    for qy in range(n):
        for qx in range(n):
            if x[qy, qx] != 0:
                out += x[qy, qx] * np.roll(h, (qy, qx), axis=(0, 1))
    return out


def test_fft_convolution_equals_spatial_bruteforce_64():
    n, K, k = 64, 3, 7
    H, w = synth.random_kernels(1, K, k)
    M = synth.random_field(2, n, 0.0, 1.0)
    I_ref = np.zeros((n, n))
    for j in range(K):
        # spatial kernel from its own definition: h(x) = n^-2 sum_f H(f) e^{+2 pi i f.x / n}
        r = (k - 1) // 2
        y = np.arange(n)
        h = np.zeros((n, n), dtype=np.complex128)
        for a in range(k):
            for b in range(k):
                u, v = a - r, b - r
                h += H[j, a, b] * np.exp(2j * np.pi * (u * y[:, None] + v * y[None, :]) / n)
        h /= n * n
        A = brute_conv(M, h)
        I_ref += w[j] * np.abs(A) ** 2
    I = litho.aerial(M, H, w)
    assert np.max(np.abs(I - I_ref)) <= 1e-12 * np.max(np.abs(I_ref))


def test_clear_field_is_dc_response():
    o = synth.optics(64, 6, 9)
    M = np.ones((64, 64))
    I = litho.aerial(M, o.H, o.w)
    r = o.r
    expect = float(np.sum(o.w * np.abs(o.H[:, r, r]) ** 2))
    assert np.allclose(I, expect, rtol=1e-12, atol=0)
    # with every eigenpair the clear field reproduces TCC(0,0) = total source power = 1
    full = synth.optics(64, 81, 9)
    I_full = litho.aerial(M, full.H, full.w)
    assert np.allclose(I_full, 1.0, rtol=1e-10)


def test_pinhole_images_kernel_intensity():
    n = 48
    o = synth.optics(n, 5, 9)
    y0, x0 = 7, 30
    M = np.zeros((n, n))
    M[y0, x0] = 1.0
    I = litho.aerial(M, o.H, o.w)
    expect = np.zeros((n, n))
    yy, xx = np.mgrid[0:n, 0:n]
    r = o.r
    for j in range(o.K):
        # h_j(x - x0) evaluated directly from the spectrum
        h = np.zeros((n, n), dtype=np.complex128)
        for a in range(o.k):
            for b in range(o.k):
                h += o.H[j, a, b] * np.exp(2j * np.pi * ((a - r) * (yy - y0) + (b - r) * (xx - x0)) / n)
        h /= n * n
        expect += o.w[j] * np.abs(h) ** 2
    assert np.max(np.abs(I - expect)) <= 1e-12 * np.max(expect)


def test_parseval_per_kernel():
    n, k = 64, 9
    H, _ = synth.random_kernels(3, 2, k)
    M = synth.random_mask(4, n).astype(np.float64)
    for j in range(2):
        A = litho.coherent_field(M, H[j])
        # direct DFT of M on the window, by the definition
        r = (k - 1) // 2
        y = np.arange(n)
        lhs = np.sum(np.abs(A) ** 2)
        rhs = 0.0
        for a in range(k):
            eu = np.exp(-2j * np.pi * (a - r) * y / n)
            for b in range(k):
                ev = np.exp(-2j * np.pi * (b - r) * y / n)
                Mhat = eu @ M @ ev
                rhs += abs(Mhat * H[j, a, b]) ** 2
        rhs /= n * n
        assert abs(lhs - rhs) <= 1e-12 * rhs


def test_socs_with_all_kernels_equals_hopkins_bilinear_form():
    n, k = 16, 7
    o = synth.optics(n, k * k, k)
    M = synth.random_mask(5, n).astype(np.float64)
    I = litho.aerial(M, o.H, o.w)
    r = (k - 1) // 2
    y = np.arange(n)
    f = np.array([(a - r, b - r) for a in range(k) for b in range(k)])
    Mhat = np.array([np.exp(-2j * np.pi * u * y / n) @ M @ np.exp(-2j * np.pi * v * y / n) for u, v in f])
    yy, xx = np.mgrid[0:n, 0:n]
    I_ref = np.zeros((n, n))
    for i1 in range(k * k):
        for i2 in range(k * k):
            t = o.tcc[i1, i2] * Mhat[i1] * np.conj(Mhat[i2])
            if t == 0:
                continue
            du, dv = f[i1] - f[i2]
            I_ref += (t * np.exp(2j * np.pi * (du * yy + dv * xx) / n)).real
    I_ref /= n ** 4
    assert np.max(np.abs(I - I_ref)) <= 1e-10 * np.max(np.abs(I_ref))


def test_convolution_adjoint_dot_product():
    n = 32
    rng = np.random.default_rng(7)
    H, _ = synth.random_kernels(8, 1, 9)
    h = litho.spatial_kernel(H[0], n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lhs = np.vdot(litho.conv(x, h), y)
    rhs = np.vdot(x, litho.conv_adjoint(y, h))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the rotation helper is the torus reflection m -> -m
    g = rng.standard_normal((n, n))
    gr = litho.rot180(g)
    for (a, b) in [(0, 0), (1, 2), (5, 31), (17, 0)]:
        assert gr[a, b] == g[(-a) % n, (-b) % n]


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_exact_for_quadratic_image(seed):
    """I(M) is quadratic in M, so <R, I(M+d) - I(M-d)> = 2 <dL/dM, d> exactly
    for every direction d (the adjoint/dot-product identity of the gradient)."""
    n = 32
    H, w = synth.random_kernels(10 + seed, 4, 7)
    rng = np.random.default_rng(seed)
    M = rng.uniform(0, 1, (n, n))
    R = rng.standard_normal((n, n))
    d = rng.standard_normal((n, n))
    V = litho.aerial_gradient(M, R, H, w)
    lhs = np.sum(R * (litho.aerial(M + d, H, w) - litho.aerial(M - d, H, w)))
    rhs = 2.0 * np.sum(V * d)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sum(np.abs(R * litho.aerial(d, H, w))))


@pytest.mark.parametrize("beta", [0.0, 7.5])
def test_loss_gradient_matches_finite_differences(beta):
    n = 32
    o = synth.optics(n, 6, 9)
    rng = np.random.default_rng(3)
    Zt = synth.rect_clip(11, n=n, nrect=(2, 3), short=(4, 8), long=(4, 16), gap=4, border=4)
    M = np.clip(Zt + 0.3 * rng.standard_normal((n, n)), 0, 1)
    p = resist.ResistParams(beta=beta)

    def L(Mx):
        return resist.resist(litho.aerial(Mx, o.H, o.w), Zt, p).loss

    R = resist.resist(litho.aerial(M, o.H, o.w), Zt, p).R
    V = litho.aerial_gradient(M, R, o.H, o.w)
    eps = 1e-6
    for (y, x) in [(3, 4), (10, 17), (16, 16), (25, 2), (31, 31)]:
        E = np.zeros((n, n))
        E[y, x] = eps
        fd = (L(M + E) - L(M - E)) / (2 * eps)
        assert abs(fd - V[y, x]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(V).max())
