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


def test_wrong_weno_weights_are_caught(monkeypatch):
    def swapped(v1, v2, v3, v4, v5):  # the ideal weights 0.1 and 0.3 exchanged
        p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
        p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
        p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
        s1 = 13.0 / 12.0 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - 4 * v2 + 3 * v3) ** 2
        s2 = 13.0 / 12.0 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
        s3 = 13.0 / 12.0 * (v3 - 2 * v4 + v5) ** 2 + 0.25 * (3 * v3 - 4 * v4 + v5) ** 2
        eps = 1e-6 * np.maximum.reduce([v1 * v1, v2 * v2, v3 * v3, v4 * v4, v5 * v5]) + 1e-99
        a1, a2, a3 = 0.3 / (s1 + eps) ** 2, 0.6 / (s2 + eps) ** 2, 0.1 / (s3 + eps) ** 2
        return (a1 * p1 + a2 * p2 + a3 * p3) / (a1 + a2 + a3)
    monkeypatch.setattr(levelset, "weno5_combine", swapped)
    import test_oracle_weno as tw
    _fails(tw.test_weno_fifth_order_convergence)


def test_fletcher_reeves_in_place_of_polak_ribiere_is_caught(monkeypatch):
    from oracle import cg
    import test_oracle_cg as tc

    def fr(V, Vprev):
        den = float(np.sum(Vprev * Vprev))
        return 0.0 if den == 0.0 else float(np.sum(V * V)) / den
    monkeypatch.setattr(cg, "pr_plus_beta", fr)
    _fails(tc.test_polak_ribiere_is_zero_for_a_repeated_gradient)


def test_dropped_previous_direction_in_cg_is_caught(monkeypatch):
    from oracle import cg
    import test_oracle_cg as tc
    monkeypatch.setattr(cg, "direction", lambda V, Vp, Dp, restart: (np.asarray(V, float).copy(), 0.0))
    _fails(tc.test_cg_finite_termination_on_a_quadratic, 0)


def test_wrong_sign_of_beta_in_cg_is_caught(monkeypatch):
    from oracle import cg
    import test_oracle_cg as tc
    orig = cg.direction

    def minus(V, Vp, Dp, restart):
        D, beta = orig(V, Vp, Dp, restart)
        if restart or Vp is None:
            return D, beta
        return np.asarray(V, float) - beta * np.asarray(Dp, float), -beta
    monkeypatch.setattr(cg, "direction", minus)
    _fails(tc.test_cg_finite_termination_on_a_quadratic, 0)


def test_shift_with_the_wrong_sign_is_caught(monkeypatch):
    from oracle import modulation
    import test_oracle_modulation as tm
    monkeypatch.setattr(modulation, "candidates",
                        lambda phi, dh: np.stack([(np.asarray(phi, float) - float(d) >= 0).astype(float) for d in dh]))
    _fails(tm.test_candidates_limits_and_monotonicity)


def test_ahf_with_eps_on_the_wrong_side_is_caught(monkeypatch):
    from oracle import modulation
    import test_oracle_modulation as tm
    monkeypatch.setattr(modulation, "ahf",
                        lambda phi, eps: 0.5 * (1.0 + (2.0 / np.pi) * np.arctan(np.asarray(phi, float) * eps)))
    _fails(tm.test_ahf_identities)


def test_avgpool_backward_without_the_quarter_is_caught(monkeypatch):
    from oracle import dsn
    import test_oracle_dsn as td
    monkeypatch.setattr(dsn, "avgpool_backward", lambda dy: np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3))
    _fails(td.test_pool_and_upsample_adjoint_pairs)
    _fails(td.test_network_gradient_matches_finite_differences)


def test_conv_backward_with_the_taps_mirrored_is_caught(monkeypatch):
    from oracle import dsn
    import test_oracle_dsn as td
    orig = dsn.conv_backward

    def mirrored(x, W, dy):
        dx, dW, db = orig(x, W[:, :, ::-1, ::-1], dy)
        return dx, dW, db
    monkeypatch.setattr(dsn, "conv_backward", mirrored)
    _fails(td.test_conv_backward_matches_finite_differences)


def test_resampling_without_centre_alignment_or_unit_change_is_caught(monkeypatch):
    from oracle import dsn
    import test_oracle_dsn as td
    orig_up, orig_down = dsn.phi_upsample, dsn.phi_downsample

    def up_corner_aligned(c, f):                 # fine pixel p read at coarse p / f
        c = np.asarray(c, dtype=np.float64)
        m = c.shape[-1]
        pos = np.arange(m * f) / f
        i0 = np.floor(pos).astype(np.int64)
        t = pos - i0
        ia, ib = np.clip(i0, 0, m - 1), np.clip(i0 + 1, 0, m - 1)
        rows = (1.0 - t)[:, None] * c[..., ia, :] + t[:, None] * c[..., ib, :]
        return f * ((1.0 - t)[None, :] * rows[..., :, ia] + t[None, :] * rows[..., :, ib])
    monkeypatch.setattr(dsn, "phi_upsample", up_corner_aligned)
    _fails(td.test_phi_upsample_matches_scipy_linear_zoom, 2)
    _fails(td.test_phi_upsample_reproduces_an_affine_field_between_the_outer_centres, 4)
    monkeypatch.setattr(dsn, "phi_upsample", lambda c, f: orig_up(c, f) / f)     # units not converted
    _fails(td.test_phi_upsample_matches_scipy_linear_zoom, 2)
    monkeypatch.setattr(dsn, "phi_upsample", lambda c, f: orig_up(np.swapaxes(c, -1, -2), f))  # transposed
    _fails(td.test_phi_upsample_reproduces_an_affine_field_between_the_outer_centres, 2)
    monkeypatch.setattr(dsn, "phi_upsample", orig_up)
    monkeypatch.setattr(dsn, "phi_downsample", lambda a, f: orig_down(a, f) * f)  # mean kept in fine pixels
    _fails(td.test_phi_downsample_of_an_affine_field_is_its_centre_value_in_coarse_pixels, 4)
    monkeypatch.setattr(dsn, "phi_downsample",                                     # block's first pixel only
                        lambda a, f: np.asarray(a, dtype=np.float64)[..., ::f, ::f] / f)
    _fails(td.test_phi_downsample_of_an_affine_field_is_its_centre_value_in_coarse_pixels, 4)


def test_sigmoid_with_the_wrong_sign_is_caught(monkeypatch):
    from oracle import resist
    import test_oracle_resist as tr
    monkeypatch.setattr(resist, "sigmoid_resist", lambda I, sz, th: 1.0 / (1.0 + np.exp(sz * (I - th))))
    _fails(tr.test_sigmoid_midpoint_symmetry_and_limits)
    _fails(tr.test_saturated_loss_counts_misprinted_pixels)


def test_tsdf_without_the_half_pixel_or_with_city_block_distance_is_caught(monkeypatch):
    from oracle import sdf
    import test_oracle_sdf as ts
    orig = sdf.opposite_class_d2

    def tsdf_no_half(mask, d_lo=sdf.D_LO, d_hi=sdf.D_HI, rows=None):
        mask = (np.asarray(mask) != 0).astype(np.uint8)
        d = orig(mask, rows)
        m = mask if rows is None else mask[np.asarray(rows)]
        dist = np.where(d < 0, np.inf, np.sqrt(np.where(d < 0, 0, d).astype(np.float64)))
        return np.clip(np.where(m == 0, dist, -dist), d_lo, d_hi)
    monkeypatch.setattr(sdf, "tsdf", tsdf_no_half)
    _fails(ts.test_tsdf_hand_values)
    _fails(ts.test_tsdf_clamps_and_degenerate_masks)
    monkeypatch.undo()

    def city_block(mask, value):                 # |dy| + |dx| instead of dy^2 + dx^2
        M = np.asarray(mask) != 0
        src = np.argwhere(M == bool(value))
        H, W = M.shape
        out = np.full((H, W), sdf.INF, dtype=np.int64)
        for y in range(H):
            for x in range(W):
                if len(src):
                    d = np.abs(src[:, 0] - y) + np.abs(src[:, 1] - x)
                    out[y, x] = int((d.min()) ** 2)
        return out
    monkeypatch.setattr(sdf, "edt_sq_rows", lambda mask, value, rows=None, g=None:
                        city_block(mask, value) if rows is None else city_block(mask, value)[np.asarray(rows)])
    _fails(ts.test_edt_sampled_rows_match_bruteforce)


def test_reinitialisation_one_iteration_early_is_caught(monkeypatch):
    from oracle import levelset as ls, litho as lt, resist as rs, sdf, solve
    import test_oracle_solve as tso

    def iterate_early(phi, Zt, H, w, p, i, m=None, defocus=None, cg_state=None):
        M = ls.mask_from_phi(phi)
        res = rs.resist(lt.aerial(M, H, w), Zt, p.resist)
        V = lt.aerial_gradient(M, res.R, H, w)
        phi, M = ls.step(phi, V, float(np.abs(V).max()), m, p.dt, p.lam, weno=p.weno)
        if p.reinit_every > 0 and i % p.reinit_every == 0:       # i instead of i + 1
            phi = sdf.tsdf(M, p.d_lo, p.d_hi)
        return phi, res
    monkeypatch.setattr(solve, "iterate", iterate_early)
    _fails(tso.test_reinitialisation_schedule)


def test_aerial_image_without_the_socs_weights_is_caught(monkeypatch):
    monkeypatch.setattr(litho, "aerial", lambda M, H, w: sum(np.abs(litho.coherent_field(M, H[j])) ** 2
                                                             for j in range(H.shape[0])))
    _fails(tli.test_clear_field_is_dc_response)
    _fails(tli.test_pinhole_images_kernel_intensity)


def test_pvband_as_union_or_with_linear_dose_is_caught(monkeypatch):
    import dataclasses
    from oracle import resist
    import test_oracle_resist as tr
    orig = resist.resist

    def with_pvb(rule):
        def f(I, Zt, p, I_def=None):
            r = orig(I, Zt, p, I_def)
            return dataclasses.replace(r, pvb=rule(np.asarray(I, dtype=np.float64), p))
        return f
    union = lambda I, p: int(np.count_nonzero(resist.threshold_resist(p.dose_in ** 2 * I, p.I_th)
                                              | resist.threshold_resist(p.dose_out ** 2 * I, p.I_th)))
    linear = lambda I, p: int(np.count_nonzero(resist.threshold_resist(p.dose_in * I, p.I_th)
                                               != resist.threshold_resist(p.dose_out * I, p.I_th)))
    for rule in (union, linear):
        monkeypatch.setattr(resist, "resist", with_pvb(rule))
        _fails(tr.test_pvband_hand_count)
