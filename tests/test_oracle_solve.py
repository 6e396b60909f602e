"""Pins of the oracle's DSO loop (Sec. III-A, III-C): the descent sign of the
velocity, exact split-run resume, and that the loop improves printability."""
import numpy as np

import synth
from oracle import levelset, litho, resist, sdf, solve


def _setup(n=64, K=6, k=9, seed=2):
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(seed, n=n, nrect=(2, 3), short=(8, 14), long=(10, 30), gap=6, border=8)
    return o, Zt


def _smooth_loss(phi, Zt, o, p):
    M = levelset.mask_from_phi(phi)
    return resist.resist(litho.aerial(M, o.H, o.w), Zt, p).loss


def test_velocity_sign_descends():
    """Reading of Eq. (phi_v_grad): with V = +dL/dM, phi += dt (V/max|V|) |grad phi|
    lowers the smooth loss for a small step; the opposite sign raises it."""
    o, Zt = _setup()
    p = resist.ResistParams(I_th=0.225)
    phi = sdf.tsdf(Zt)
    M = levelset.mask_from_phi(phi)
    res = resist.resist(litho.aerial(M, o.H, o.w), Zt, p)
    V = litho.aerial_gradient(M, res.R, o.H, o.w)
    vmax = np.abs(V).max()
    down, _ = levelset.step(phi, V, vmax, None, 1.0, 0.0)
    up, _ = levelset.step(phi, -V, vmax, None, 1.0, 0.0)
    L0 = res.loss
    assert _smooth_loss(down, Zt, o, p) < L0 < _smooth_loss(up, Zt, o, p)


def test_split_run_resumes_exactly():
    o, Zt = _setup()
    p = solve.SolveParams(iters=7, reinit_every=3)
    full = solve.ilt_solve(Zt, o.H, o.w, p)
    a = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=4, reinit_every=3))
    b = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=3, reinit_every=3, start_iter=4), phi0=a.phi)
    assert np.array_equal(full.phi, b.phi)
    assert full.loss[:4] == a.loss[:4] and full.loss[4:] == b.loss


def test_loop_improves_printability():
    o, Zt = _setup(n=64, K=6, k=9, seed=4)
    p = solve.SolveParams(iters=15, dt=0.5, lam=0.1)
    out = solve.ilt_solve(Zt, o.H, o.w, p)
    assert out.loss[-1] < 0.8 * out.loss[0]
    assert out.l2[-1] < out.l2[0]


def test_reinitialisation_schedule():
    """Reading of the re-initialisation period: phi becomes the TSDF of its mask right
    after the update of every iteration i with (i + 1) a multiple of reinit_every
    (global index), and only then."""
    o, Zt = _setup()
    for iters, start, reinit in ((5, 0, True), (4, 0, False), (6, 0, False), (2, 3, True), (2, 4, False)):
        out = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=iters, reinit_every=5, start_iter=start))
        is_tsdf = np.array_equal(out.phi, sdf.tsdf(out.mask))
        assert is_tsdf == reinit, (iters, start)
