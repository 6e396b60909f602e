"""Planted mistakes: each test swaps one piece of the oracle for a plausible
wrong version (on the CPU, through monkeypatch) and checks that the pin meant
to catch it fails. A pin that passed with the mistake in place would not pin
anything."""
import numpy as np
import pytest

from oracle import levelset, litho
import test_oracle_levelset as tl
import test_oracle_litho as tli


def _fails(fn, *a):
    with pytest.raises(AssertionError):
        fn(*a)


def test_missing_rotation_in_gradient_is_caught(monkeypatch):
    monkeypatch.setattr(litho, "rot180", lambda h: h)
    _fails(tli.test_gradient_exact_for_quadratic_image, 0)


def test_missing_conjugate_in_gradient_is_caught(monkeypatch):
    orig = litho.conv

    def aerial_gradient_noconj(M, R, H, w):
        n = M.shape[0]
        V = np.zeros((n, n))
        for j in range(H.shape[0]):
            h = litho.spatial_kernel(H[j], n)
            hr = litho.rot180(h)
            t1 = orig(hr, R * orig(M, h))        # conj dropped on h
            t2 = orig(np.conj(hr), R * orig(M, h))
            V += w[j] * (t1 + t2).real
        return V
    monkeypatch.setattr(litho, "aerial_gradient", aerial_gradient_noconj)
    _fails(tli.test_gradient_exact_for_quadratic_image, 1)


def test_transposed_window_is_caught(monkeypatch):
    orig = litho.pad_window
    monkeypatch.setattr(litho, "pad_window", lambda Hj, n: orig(np.swapaxes(Hj, -1, -2), n))
    _fails(tli.test_fft_convolution_equals_spatial_bruteforce_64)


def test_mixed_derivative_sign_is_caught(monkeypatch):
    orig = levelset.central_differences

    def bad(phi):
        px, py, pxx, pyy, pxy = orig(phi)
        return px, py, pxx, pyy, -pxy
    monkeypatch.setattr(levelset, "central_differences", bad)
    _fails(tl.test_quadratic_derivatives_and_curvature_hand_values)


def test_swapped_upwind_is_caught(monkeypatch):
    orig = levelset.upwind_gradients
    monkeypatch.setattr(levelset, "upwind_gradients", lambda phi: orig(phi)[::-1])
    _fails(tl.test_upwind_kink_follows_hopf_lax_solution)
