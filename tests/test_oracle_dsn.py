"""Pins of the oracle's level-set network (Sec. III-B, DSN level-set branch): the
convolution against scipy's 2-D correlation, the pooling / upsampling adjoint pairs,
every gradient against finite differences, Adam's first step in closed form, and the
residual start (zero head = the target's own band-limited TSDF)."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import dsn


def test_layer_list_follows_the_reading():
    L = dsn.layer_shapes(32)
    assert len(L) == 15
    assert [o for _, o, _ in L[:8]] == [32, 32, 64, 64, 128, 128, 256, 256]
    assert L[8] == (256 + 128, 128, 3) and L[10] == (128 + 64, 64, 3) and L[12] == (64 + 32, 32, 3)
    assert L[-1] == (32, 1, 1)


@pytest.mark.parametrize("k", [1, 3])
def test_conv_is_zero_padded_correlation(k):
    rng = np.random.default_rng(k)
    x = rng.standard_normal((2, 3, 7, 9))
    W = rng.standard_normal((4, 3, k, k))
    b = rng.standard_normal(4)
    y = dsn.conv(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[n, c], W[o, c], mode="same") for c in range(3)) + b[o]
            assert np.allclose(y[n, o], ref, rtol=0, atol=1e-12)


def test_pool_and_upsample_adjoint_pairs():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 8, 6))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(dsn.avgpool(x) * y), np.sum(x * dsn.avgpool_backward(y)), rtol=1e-13)
    z = rng.standard_normal((2, 3, 16, 12))
    assert np.isclose(np.sum(dsn.upsample(y) * z[:, :, :8, :6]), np.sum(y * dsn.upsample_backward(z[:, :, :8, :6])),
                      rtol=1e-13)


def test_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 2, 5, 5))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((1, 3, 5, 5))
    dx, dW, db = dsn.conv_backward(x, W, dy)
    f = lambda xx, WW, bb: float(np.sum(dsn.conv(xx, WW, bb) * dy))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 3), (0, 1, 4, 4)]:
        e = np.zeros_like(x); e[idx] = h
        assert dx[idx] == pytest.approx((f(x + e, W, b) - f(x - e, W, b)) / (2 * h), rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0, 0), (2, 1, 1, 2), (1, 0, 2, 1)]:
        e = np.zeros_like(W); e[idx] = h
        assert dW[idx] == pytest.approx((f(x, W + e, b) - f(x, W - e, b)) / (2 * h), rel=1e-6, abs=1e-8)
    assert np.allclose(db, dy.sum(axis=(0, 2, 3)))


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    c, S = 2, 16
    P = dsn.init_params(c, 11)
    P = [p + 0.01 * rng.standard_normal(p.shape) for p in P]   # non-zero biases too
    x = dsn.band(rng.uniform(-30, 30, (2, 1, S, S)))
    label = dsn.band(rng.uniform(-30, 30, (2, 1, S, S)))
    y, cache = dsn.forward(P, x)
    L, dy = dsn.mse(y, label)
    G = dsn.backward(P, x, cache, dy)
    h = 1e-6
    for li in [0, 1, 5, 9, 12, 16, 23, 28, 29]:
        flat = P[li].reshape(-1)
        for j in [0, flat.size // 2, flat.size - 1]:
            old = flat[j]
            flat[j] = old + h
            Lp = dsn.mse(dsn.forward(P, x)[0], label)[0]
            flat[j] = old - h
            Lm = dsn.mse(dsn.forward(P, x)[0], label)[0]
            flat[j] = old
            fd = (Lp - Lm) / (2 * h)
            assert G[li].reshape(-1)[j] == pytest.approx(fd, rel=2e-4, abs=1e-9), (li, j)


def test_adam_first_step_closed_form():
    """From zero moments: m^ = g, v^ = g^2, so p moves by lr g / (|g| + eps)."""
    P = [np.array([1.0, -2.0, 3.0])]
    G = [np.array([0.5, -4.0, 0.0])]
    opt, state = dsn.Adam(lr=0.1), []
    opt.step(P, G, state)
    assert np.allclose(P[0], [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 4.0 / (4.0 + 1e-8), 3.0], rtol=0, atol=1e-15)


def test_zero_head_returns_the_input_level_set():
    P = dsn.init_params(2, 1)
    P[-2][...] = 0.0
    P[-1][...] = 0.0
    x = dsn.band(np.random.default_rng(2).uniform(-30, 30, (1, 1, 16, 16)))
    assert np.array_equal(dsn.forward(P, x)[0], x)


def test_modulation_loss_gradient_and_limits():
    """The modulation branch's loss: gradient against finite differences; zero when
    the labels equal H_eps of the output; its H_eps is the one of the modulation
    supervision (oracle/modulation.py)."""
    from oracle import modulation
    rng = np.random.default_rng(9)
    y = rng.uniform(-0.2, 0.2, (1, 1, 5, 5))
    m = (rng.random((1, 1, 5, 5)) < 0.5).astype(float)
    L, g = dsn.ahf_mean(y, m, 0.03)
    h = 1e-7
    for idx in [(0, 0, 0, 0), (0, 0, 2, 3), (0, 0, 4, 4)]:
        e = np.zeros_like(y); e[idx] = h
        fd = (dsn.ahf_mean(y + e, m, 0.03)[0] - dsn.ahf_mean(y - e, m, 0.03)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    assert dsn.ahf_mean(y, modulation.ahf(y, 0.03), 0.03)[0] == 0.0
    assert L * y.size == pytest.approx(modulation.ahf_loss(y, m, 0.03)[0], rel=1e-12)


# Resampling between a clip's grid and the DSN's coarser grid (the learned start of a
# clip larger than the network's side).

def _affine(a, b, c, rows, cols, f=1):
    """a x + b y + c at pixel indices (x = column, y = row), shape [rows, cols]."""
    y, x = np.mgrid[0:rows, 0:cols].astype(np.float64)
    return a * x + b * y + c


@pytest.mark.parametrize("f", [1, 2, 3, 4])
def test_phi_downsample_of_an_affine_field_is_its_centre_value_in_coarse_pixels(f):
    m = 5
    fine = _affine(0.7, -1.9, 3.25, m * f, m * f)
    I, J = np.mgrid[0:m, 0:m].astype(np.float64)
    want = (0.7 * (f * J + (f - 1) / 2) - 1.9 * (f * I + (f - 1) / 2) + 3.25) / f
    assert np.allclose(dsn.phi_downsample(fine, f), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("f", [1, 2, 3, 4])
def test_phi_upsample_matches_scipy_linear_zoom(f):
    from scipy.ndimage import zoom
    c = np.random.default_rng(f).standard_normal((2, 7, 7))
    got = dsn.phi_upsample(c, f)
    for b in range(2):
        ref = f * zoom(c[b], f, order=1, mode="nearest", grid_mode=True)
        assert np.allclose(got[b], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("f", [2, 4])
def test_phi_upsample_reproduces_an_affine_field_between_the_outer_centres(f):
    m = 6
    c = _affine(0.3, 1.7, -2.0, m, m)
    fine = dsn.phi_upsample(c, f)
    pos = (np.arange(m * f) + 0.5) / f - 0.5
    inside = (pos >= 0) & (pos <= m - 1)
    Y, X = np.meshgrid(pos, pos, indexing="ij")
    want = f * (0.3 * X + 1.7 * Y - 2.0)
    sel = inside[:, None] & inside[None, :]
    assert np.allclose(fine[sel], want[sel], rtol=0, atol=1e-12)
    # beyond the outer centres the field is held at its value there (edge clamp)
    top, right = fine[pos < 0], fine[:, pos > m - 1]
    assert len(top) == f // 2 and np.allclose(top, top[0], rtol=0, atol=1e-12)
    assert np.allclose(top[0][inside], f * (0.3 * pos[inside] - 2.0), rtol=0, atol=1e-12)
    assert right.shape[1] == f // 2 and np.allclose(right, right[:, :1], rtol=0, atol=1e-12)
    assert np.allclose(right[inside, 0], f * (0.3 * (m - 1) + 1.7 * pos[inside] - 2.0), rtol=0, atol=1e-12)


def test_phi_resampling_round_trips_and_keeps_the_zero_level_of_a_half_plane():
    f, m = 4, 8
    k = np.full((m, m), -3.5)
    assert np.allclose(dsn.phi_downsample(dsn.phi_upsample(k, f), f), k, rtol=0, atol=1e-12)
    # signed distance to the vertical line x = 13.5 - 1/2 (between fine columns 12 and 13):
    # a distance field in fine pixels becomes one in coarse pixels, with the same zero set
    fine = np.arange(m * f)[None, :].repeat(m * f, axis=0) - 12.5
    coarse = dsn.phi_downsample(fine, f)
    assert np.allclose(coarse, (np.arange(m)[None, :] * f + 1.5 - 12.5) / f * np.ones((m, 1)), atol=1e-12)
    back = dsn.phi_upsample(coarse, f)
    inner = slice(f, m * f - f)
    assert np.allclose(back[:, inner], fine[:, inner], rtol=0, atol=1e-12)
