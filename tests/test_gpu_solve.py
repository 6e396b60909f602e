"""GPU parity of devel_ilt_solve against the oracle's DSO loop (Sec. III-A,
III-C): ILT results within 0.1% thresholded-pixel mismatch, L2 and PVB within
1%, on the 256^2 rectangle workload (K = 8, k = 15, 20 iterations)."""
import numpy as np
import pytest

import synth
from oracle import levelset, litho, sdf, solve
from oracle import resist
from gpu_util import need_gpu, dev, host, loss_bound, torch

pytestmark = pytest.mark.gpu


def run_gpu(dv, Zt, o, iters, beta=0.0, phi0=None, start=0, reinit_every=5, prec=0):
    n = Zt.shape[0]
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda") if phi0 is None else dev(phi0.astype(np.float32))
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = dv.ilt_params(dv.resist_params(beta=beta), iters=iters, start_iter=start, reinit_every=reinit_every)
    clip = dv.Clip(opt, dev(Zt), phi, phi_given=phi0 is not None, mask_out=M, loss_hist=L, l2_hist=l2, pvb_hist=pvb)
    dv.devel_ilt_solve(p, [clip], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    return host(phi, n), host(M, n), host(L), host(l2), host(pvb)


# normwise aerial-image tolerance of each precision path (the litho parity tests' bars)
IMAGE_TOL = {0: 1e-5, 1: 2e-4}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed,beta", [(0, 0.0), (1, 0.0), (2, 0.0), (0, 7.5), (3, 7.5)])
def test_solve_matches_oracle_rect_workload(seed, beta, prec):
    """The steepest-descent solve on the 256^2 workload, without (beta = 0) and with the
    process-window term (beta = 7.5, Sec. III-A L_pvb). The first loss, of the target's
    own mask, differs from the oracle's only through the image error: within the bound
    that the precision's image tolerance implies (gpu_util.loss_bound)."""
    dv = need_gpu()
    o = synth.optics(256, 8, 15)
    Zt = synth.rect_clip(seed)
    phi, M, L, l2, pvb = run_gpu(dv, Zt, o, 20, beta=beta, prec=prec)
    rp = resist.ResistParams(beta=beta)
    ref = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=20, resist=rp))
    mismatch = np.count_nonzero(M != ref.mask) / M.size
    assert mismatch <= 1e-3, mismatch
    assert abs(l2[-1] - ref.l2[-1]) <= 0.01 * max(ref.l2[-1], 1)
    assert abs(pvb[-1] - ref.pvb[-1]) <= 0.01 * max(ref.pvb[-1], 100)
    M0 = levelset.mask_from_phi(sdf.tsdf(Zt))
    I0 = litho.aerial(M0, o.H, o.w)
    R0 = resist.resist(I0, Zt, rp).R
    assert abs(L[0] - ref.loss[0]) <= loss_bound(I0, R0, ref.loss[0], IMAGE_TOL[prec]), (L[0], ref.loss[0])


def test_solve_resume_is_exact():
    """A 4 + 3 split run is bit-identical to a 7-iteration run (reinit keyed on
    the global iteration index)."""
    dv = need_gpu()
    o = synth.optics(128, 6, 11)
    Zt = synth.rect_clip(7, n=128, border=8)
    phiA, MA, LA, _, _ = run_gpu(dv, Zt, o, 7, reinit_every=3)
    phi4, _, L4, _, _ = run_gpu(dv, Zt, o, 4, reinit_every=3)
    phiB, MB, LB, _, _ = run_gpu(dv, Zt, o, 3, phi0=phi4, start=4, reinit_every=3)
    assert np.array_equal(phiA, phiB) and np.array_equal(MA, MB)
    assert np.array_equal(LA[:4], L4[:4]) and np.array_equal(LA[4:], LB)


def test_bf16x3_aerial_error_per_iteration():
    """Compensated-BF16 precision on the 256^2 rectangle workload: along the
    oracle's own 20-iteration trajectory, the aerial image of every iterate's
    mask, imaged by the tensor-core path, stays within 2e-4 (normwise relative)
    of the FP64 oracle's image of the same mask."""
    dv = need_gpu()
    o = synth.optics(256, 8, 15)
    Zt = synth.rect_clip(0)
    opt = dv.devel_optics_create(256, o.H, o.w, dv.DEVEL_PREC_BF16X3)
    p = solve.SolveParams(iters=20)
    phi = sdf.tsdf(Zt)
    out = torch.empty(256 * 256, dtype=torch.float32, device="cuda")
    Hc = o.H.astype(np.complex64).astype(np.complex128)
    wc = o.w.astype(np.float32).astype(np.float64)
    errs = []
    for t in range(p.iters):
        M = levelset.mask_from_phi(phi)
        dv.devel_litho_forward(opt, dev(M.astype(np.float32)), out)
        torch.cuda.synchronize()
        ref = litho.aerial(M.astype(np.float64), Hc, wc)
        errs.append(float(np.abs(host(out, 256) - ref).max() / np.abs(ref).max()))
        phi, _ = solve.iterate(phi, Zt, o.H, o.w, p, t)
    assert max(errs) <= 2e-4, errs


def _clip_job(dv, opt, Zt, iters):
    n = Zt.shape[0]
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    return dv.Clip(opt, dev(Zt), phi, mask_out=M, loss_hist=L, l2_hist=l2)


@pytest.mark.parametrize("optimizer", [0, 1])
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("prec", [0, 1])
def test_batched_uneven_clips_equal_single_solves(prec, use_graph, optimizer):
    """One devel_ilt_solve over clips of uneven sides (each side with its own window,
    two clips sharing one handle) gives, clip for clip, bit-identical phi, masks and
    loss histories to solving each clip alone: the concurrent branches change the
    schedule, never a clip's arithmetic."""
    dv = need_gpu()
    iters = 6
    sides = [(128, 9), (192, 11), (256, 15)]
    opts = {n: dv.devel_optics_create(n, *_optics_arrays(n, k), prec) for n, k in sides}
    targets = [synth.rect_clip(40 + i, n=n, border=8) for i, (n, _) in enumerate(sides)]
    targets.append(synth.rect_clip(50, n=128, border=8))  # shares the 128 handle
    handles = [opts[128], opts[192], opts[256], opts[128]]
    p = dv.ilt_params(dv.resist_params(beta=2.0), iters=iters, reinit_every=3, use_graph=use_graph,
                      optimizer=optimizer)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch = [_clip_job(dv, h, Zt, iters) for h, Zt in zip(handles, targets)]
    dv.devel_ilt_solve(p, batch, st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    for h, Zt, b in zip(handles, targets, batch):
        one = _clip_job(dv, h, Zt, iters)
        dv.devel_ilt_solve(p, [one], st)
        torch.cuda.synchronize()
        assert int(host(st)[0]) == 0
        for name in ("phi", "mask_out", "loss_hist", "l2_hist"):
            assert torch.equal(getattr(b, name), getattr(one, name)), name


_OPTICS_CACHE = {}


def _optics_arrays(n, k):
    if (n, k) not in _OPTICS_CACHE:
        o = synth.optics(n, 6, k)
        _OPTICS_CACHE[(n, k)] = (o.H, o.w)
    return _OPTICS_CACHE[(n, k)]
