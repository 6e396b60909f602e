"""Pins of the oracle's defocused process corner (Sec. II-C: inner corner at
defocus and -2% dose, outer at nominal focus and +2% dose): the defocus phase
enters the TCC as exp(2 pi i W rho^2), so +W and -W image a real mask alike;
with the defocused system equal to the nominal one the two-image loss reduces to
the dose-only loss; and the two-system gradient matches finite differences."""
import numpy as np
import pytest

import synth
from oracle import litho, resist, solve


def test_defocus_sign_symmetry_for_real_masks():
    """TCC(-W) = conj TCC(W) and the pupil and source are symmetric, so with all k^2
    kernels (the exact Hopkins image) +W and -W give the same image of a real mask;
    a missing conjugate in the TCC breaks this."""
    n, k = 32, 7
    M = synth.rect_clip(5, n=n, nrect=(2, 3), short=(3, 6), long=(4, 12), gap=3, border=3).astype(np.float64)
    Ip = litho.aerial(M, *_hw(synth.optics(n, k * k, k, defocus=0.3)))
    Im = litho.aerial(M, *_hw(synth.optics(n, k * k, k, defocus=-0.3)))
    I0 = litho.aerial(M, *_hw(synth.optics(n, k * k, k)))
    assert np.abs(Ip - Im).max() <= 1e-12 * np.abs(Ip).max()
    assert np.abs(Ip - I0).max() > 1e-3 * np.abs(I0).max()  # defocus does change the image


def _hw(o):
    return o.H, o.w


def test_zero_defocus_matches_the_real_pupil():
    a = synth.optics(32, 6, 9)
    b = synth.optics(32, 6, 9, defocus=0.0)
    assert np.array_equal(a.tcc, b.tcc)


@pytest.mark.parametrize("beta", [0.0, 7.5])
def test_same_system_reduces_to_dose_only_loss(beta):
    n = 32
    o = synth.optics(n, 6, 9)
    Zt = synth.rect_clip(11, n=n, nrect=(2, 3), short=(4, 8), long=(4, 16), gap=4, border=4)
    M = synth.random_field(2, n, 0.0, 1.0)
    I = litho.aerial(M, o.H, o.w)
    p = resist.ResistParams(beta=beta)
    one = resist.resist(I, Zt, p)
    two = resist.resist(I, Zt, p, I_def=I)
    assert abs(two.loss - one.loss) <= 1e-12 * max(one.loss, 1.0)
    assert np.abs((two.R + two.R_def) - one.R).max() <= 1e-12 * max(np.abs(one.R).max(), 1e-30)
    assert (two.l2, two.pvb) == (one.l2, one.pvb)


def test_two_system_gradient_matches_finite_differences():
    n = 32
    o = synth.optics(n, 6, 9)
    od = synth.optics(n, 6, 9, defocus=0.25)
    rng = np.random.default_rng(4)
    Zt = synth.rect_clip(12, n=n, nrect=(2, 3), short=(4, 8), long=(4, 16), gap=4, border=4)
    M = np.clip(Zt + 0.3 * rng.standard_normal((n, n)), 0, 1)
    p = resist.ResistParams(beta=7.5)

    def L(Mx):
        return resist.resist(litho.aerial(Mx, o.H, o.w), Zt, p, litho.aerial(Mx, od.H, od.w)).loss

    r = resist.resist(litho.aerial(M, o.H, o.w), Zt, p, litho.aerial(M, od.H, od.w))
    V = litho.aerial_gradient(M, r.R, o.H, o.w) + litho.aerial_gradient(M, r.R_def, od.H, od.w)
    eps = 1e-6
    for (y, x) in [(3, 4), (10, 17), (16, 16), (25, 2), (31, 31)]:
        E = np.zeros((n, n))
        E[y, x] = eps
        fd = (L(M + E) - L(M - E)) / (2 * eps)
        assert abs(fd - V[y, x]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(V).max())


def test_defocus_solve_runs_and_lowers_the_loss():
    n = 64
    o = synth.optics(n, 4, 9)
    od = synth.optics(n, 4, 9, defocus=0.25)
    Zt = synth.rect_clip(13, n=n, nrect=(2, 3), short=(6, 10), long=(8, 20), gap=6, border=6)
    r = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=6, resist=resist.ResistParams(beta=7.5)),
                        defocus=(od.H, od.w))
    assert r.loss[-1] < r.loss[0]
