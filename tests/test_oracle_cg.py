"""Pins of the oracle's conjugate-gradient direction (Sec. III-C: DSO optimises with
CG; the update is the PR+ reading in oracle/cg.py). The direction rule is checked
where the mathematics fixes the result: on a strictly convex quadratic with exact
line searches, nonlinear CG is linear CG and reaches the minimiser in at most n
steps; Polak-Ribiere differs from Fletcher-Reeves when the gradient repeats; the
clip and the restarts; and a CG solve that restarts every iteration is the plain
solve."""
import numpy as np
import pytest

import synth
from oracle import cg, resist, solve


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cg_finite_termination_on_a_quadratic(seed):
    """f(x) = x^T A x / 2 - b^T x, A SPD: with the exact step along -D, CG hits
    A^-1 b within n iterations (a wrong sign, index or missing D term does not)."""
    rng = np.random.default_rng(seed)
    n = 6
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    x = np.zeros(n)
    gp = Dp = None
    for k in range(n):
        g = A @ x - b
        D, _ = cg.direction(g, gp, Dp, restart=k == 0)
        alpha = float(g @ D) / float(D @ A @ D)
        x = x - alpha * D
        gp, Dp = g, D
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9)
    # steepest descent (D = V) does not terminate in n steps on the same problem
    xs = np.zeros(n)
    for k in range(n):
        g = A @ xs - b
        xs = xs - float(g @ g) / float(g @ A @ g) * g
    assert not np.allclose(xs, np.linalg.solve(A, b), rtol=0, atol=1e-6)


def test_cg_conjugacy_on_a_quadratic():
    """The directions of linear CG are A-conjugate: D_i^T A D_j = 0 for i != j."""
    rng = np.random.default_rng(5)
    n = 5
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + np.eye(n)
    b = rng.standard_normal(n)
    x = np.zeros(n)
    gp = Dp = None
    Ds = []
    for k in range(n):
        g = A @ x - b
        D, _ = cg.direction(g, gp, Dp, restart=k == 0)
        Ds.append(D)
        x = x - float(g @ D) / float(D @ A @ D) * D
        gp, Dp = g, D
    G = np.array([[Di @ A @ Dj for Dj in Ds] for Di in Ds])
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) <= 1e-9 * np.max(np.abs(np.diag(G)))


def test_polak_ribiere_is_zero_for_a_repeated_gradient():
    """PR: <g, g - g> = 0, so beta = 0 and D = V (Fletcher-Reeves would give 1)."""
    g = np.array([1.0, -2.0, 3.0])
    D, beta = cg.direction(g, g.copy(), np.array([5.0, 5.0, 5.0]), restart=False)
    assert beta == 0.0 and np.array_equal(D, g)


def test_pr_plus_clips_negative_beta_and_zero_previous_gradient():
    V, Vp = np.array([1.0, 0.0]), np.array([2.0, 0.0])  # <V, V - Vp> = -1 < 0
    assert cg.pr_plus_beta(V, Vp) == 0.0
    assert cg.pr_plus_beta(V, np.zeros(2)) == 0.0
    # orthogonal successive gradients (as under exact line search): beta = |V|^2 / |Vp|^2
    assert cg.pr_plus_beta(np.array([0.0, 3.0]), np.array([2.0, 0.0])) == pytest.approx(9.0 / 4.0)


def test_restart_schedule():
    assert cg.restarts_at(7, 5, first=True)
    assert cg.restarts_at(10, 5, first=False)
    assert not cg.restarts_at(11, 5, first=False)
    assert not cg.restarts_at(3, 0, first=False)


def test_cg_solve_restarting_every_iteration_is_the_plain_solve():
    n, K, k = 64, 4, 7
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(3, n=n, border=4)
    base = dict(iters=4, reinit_every=1, resist=resist.ResistParams(beta=1.0))
    a = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(**base))
    b = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(optimizer="cg", **base))
    assert np.array_equal(a.phi, b.phi) and a.loss == b.loss


def test_cg_solve_differs_from_plain_between_restarts():
    n, K, k = 64, 4, 7
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(3, n=n, border=4)
    base = dict(iters=4, reinit_every=5, resist=resist.ResistParams(beta=1.0))
    a = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(**base))
    b = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(optimizer="cg", **base))
    assert a.loss[0] == b.loss[0]          # the first step is a restart
    assert not np.array_equal(a.phi, b.phi)
