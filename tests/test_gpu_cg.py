"""GPU parity of the conjugate-gradient option (Sec. III-C: DSO optimises with CG;
the PR+ reading of oracle/cg.py): devel_cg_direction against the oracle's direction,
and whole solves with DEVEL_OPT_CG against the oracle's CG loop."""
import numpy as np
import pytest

import synth
from oracle import cg, resist, solve
from gpu_util import need_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


def _direction(dv, opt, V, Vp, D, restart):
    n = opt.n
    tV, tVp, tD = dev(V.astype(np.float32)), dev(Vp.astype(np.float32)), dev(D.astype(np.float32))
    beta = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    vmax = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dv.devel_cg_direction(opt, tV, tVp, tD, restart, vmax, beta=beta, status=st)
    torch.cuda.synchronize()
    return host(tD, n), host(tVp, n), float(host(beta)[0]), float(host(vmax)[0]), int(host(st)[0])


@pytest.mark.parametrize("n", [64, 129, 256])
def test_cg_direction_matches_oracle(n):
    dv = need_gpu()
    o = synth.optics(n, 2, 5)
    opt = dv.devel_optics_create(n, o.H, o.w)
    rng = np.random.default_rng(n)
    V = rng.standard_normal((n, n)).astype(np.float32)
    Vp = (0.8 * V + 0.3 * rng.standard_normal((n, n))).astype(np.float32)
    D = rng.standard_normal((n, n)).astype(np.float32)
    Dg, Vpg, beta, vmax, st = _direction(dv, opt, V, Vp, D, False)
    Dref, bref = cg.direction(V.astype(np.float64), Vp.astype(np.float64), D.astype(np.float64), False)
    assert st == 0
    # FP32 sums (a few ulps per block, pairwise across blocks) and an FP32 quotient
    assert bref > 0 and abs(beta - bref) <= 5e-5 * bref
    assert rel_err(Dg, Dref) <= 1e-5
    assert np.array_equal(Vpg, V)                          # Vprev <- V
    assert vmax == float(np.abs(Dg).max())                 # max of the stored D
    # restart: D = V exactly, beta 0
    Dg, Vpg, beta, vmax, st = _direction(dv, opt, V, Vp, D, True)
    assert st == 0 and beta == 0.0 and np.array_equal(Dg, V) and np.array_equal(Vpg, V)
    assert vmax == float(np.abs(V).max())


def test_cg_direction_clips_negative_beta_and_zero_history():
    dv = need_gpu()
    n = 64
    o = synth.optics(n, 2, 5)
    opt = dv.devel_optics_create(n, o.H, o.w)
    V = np.ones((n, n), np.float32)
    D = np.full((n, n), 7.0, np.float32)
    Dg, _, beta, _, _ = _direction(dv, opt, V, 2 * V, D, False)  # <V, V - 2V> < 0
    assert beta == 0.0 and np.array_equal(Dg, V)
    Dg, _, beta, _, _ = _direction(dv, opt, V, 0 * V, D, False)  # <Vp, Vp> = 0
    assert beta == 0.0 and np.array_equal(Dg, V)


def test_cg_direction_reports_non_finite():
    dv = need_gpu()
    n = 64
    o = synth.optics(n, 2, 5)
    opt = dv.devel_optics_create(n, o.H, o.w)
    V = np.ones((n, n), np.float32)
    V[3, 7] = np.nan
    _, _, _, _, st = _direction(dv, opt, V, V + 1, V, False)
    assert st == dv.DEVEL_ENAN


def _solve(dv, opt, Zt, iters, start=0, phi0=None, reinit_every=5, beta=7.5, optimizer=1):
    n = opt.n
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda") if phi0 is None else dev(phi0.astype(np.float32))
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = dv.ilt_params(dv.resist_params(beta=beta), iters=iters, start_iter=start, reinit_every=reinit_every,
                      optimizer=optimizer)
    dv.devel_ilt_solve(p, [dv.Clip(opt, dev(Zt), phi, phi_given=phi0 is not None, mask_out=M, loss_hist=L,
                                   l2_hist=l2, pvb_hist=pvb)], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    return host(phi, n), host(M, n), host(L), host(l2), host(pvb)


@pytest.mark.parametrize("prec", [0, 1])
def test_cg_solve_matches_oracle(prec):
    dv = need_gpu()
    n, K, k, iters = 256, 8, 15, 20
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(1)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    phi, M, L, l2, pvb = _solve(dv, opt, Zt, iters)
    ref = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=iters, resist=resist.ResistParams(beta=7.5),
                                                         optimizer="cg"))
    mism = np.count_nonzero(M != ref.mask) / M.size
    assert mism <= 1e-3, mism
    assert abs(int(l2[-1]) - ref.l2[-1]) <= 0.01 * max(ref.l2[-1], 1)
    assert abs(int(pvb[-1]) - ref.pvb[-1]) <= 0.01 * max(ref.pvb[-1], 100)
    # CG differs from the plain solve on this workload (the option does something)
    plain = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=iters, resist=resist.ResistParams(beta=7.5)))
    assert not np.array_equal(ref.mask, plain.mask)


def test_cg_solve_resumed_at_a_restart_is_exact():
    """10 iterations in one call equal 5 + 5 (the split at a multiple of
    reinit_every, where the direction restarts) bit for bit."""
    dv = need_gpu()
    n = 128
    o = synth.optics(n, 6, 11)
    Zt = synth.rect_clip(4, n=n, border=8)
    opt = dv.devel_optics_create(n, o.H, o.w, 1)
    full = _solve(dv, opt, Zt, 10)
    a = _solve(dv, opt, Zt, 5)
    b = _solve(dv, opt, Zt, 5, start=5, phi0=a[0])
    assert np.array_equal(full[0], b[0]) and np.array_equal(full[1], b[1])
    assert np.array_equal(full[2][5:], b[2])
