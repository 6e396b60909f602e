"""GPU parity of the defocused inner process corner (Sec. II-C): solves with a
second, defocused optical system against the oracle's two-system loop, on both
precision paths."""
import numpy as np
import pytest

import synth
from oracle import levelset, litho, resist, sdf, solve
from gpu_util import need_gpu, dev, host, loss_bound, torch

IMAGE_TOL = {0: 1e-5, 1: 2e-4}  # normwise aerial-image tolerance of each precision path

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_defocus_solve_matches_oracle(prec):
    dv = need_gpu()
    n, K, k, iters = 256, 8, 15, 20
    o = synth.optics(n, K, k)
    od = synth.optics(n, K, k, defocus=0.25)
    Zt = synth.rect_clip(2)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    optd = dv.devel_optics_create(n, od.H, od.w, prec)
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = dv.ilt_params(dv.resist_params(beta=7.5), iters=iters)
    dv.devel_ilt_solve(p, [dv.Clip(opt, dev(Zt), phi, mask_out=M, loss_hist=L, l2_hist=l2, pvb_hist=pvb,
                                   optics_defocus=optd)], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    ref = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=iters, resist=resist.ResistParams(beta=7.5)),
                          defocus=(od.H, od.w))
    mism = np.count_nonzero(host(M, n) != ref.mask) / (n * n)
    assert mism <= 1e-3, mism
    assert abs(int(host(l2)[-1]) - ref.l2[-1]) <= 0.01 * max(ref.l2[-1], 1)
    assert abs(int(host(pvb)[-1]) - ref.pvb[-1]) <= 0.01 * max(ref.pvb[-1], 100)
    # the first loss differs from the oracle's only through the two images' errors
    M0 = levelset.mask_from_phi(sdf.tsdf(Zt))
    I0, Id0 = litho.aerial(M0, o.H, o.w), litho.aerial(M0, od.H, od.w)
    r0 = resist.resist(I0, Zt, resist.ResistParams(beta=7.5), Id0)
    tol = IMAGE_TOL[prec]
    bound = loss_bound(I0, r0.R, ref.loss[0], tol) + loss_bound(Id0, r0.R_def, 0.0, tol)
    assert abs(host(L)[0] - ref.loss[0]) <= bound, (host(L)[0], ref.loss[0])


def test_defocus_handle_checks():
    dv = need_gpu()
    n = 64
    o = synth.optics(n, 4, 7)
    o2 = synth.optics(n, 4, 9)
    a = dv.devel_optics_create(n, o.H, o.w, 0)
    b = dv.devel_optics_create(n, o2.H, o2.w, 0)  # another window: refused
    Zt = synth.rect_clip(3, n=n, border=4)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    with pytest.raises(dv.DevelError):
        dv.devel_ilt_solve(dv.ilt_params(iters=2), [dv.Clip(a, dev(Zt), phi, optics_defocus=b)], st)
    with pytest.raises(dv.DevelError):
        dv.devel_ilt_solve(dv.ilt_params(iters=2), [dv.Clip(a, dev(Zt), phi, optics_defocus=a)], st)
