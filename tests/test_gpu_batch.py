"""GPU tests of devel_ilt_solve_batch: the DSO loop (Sec. III-A, III-C) with every stage
launched once over a batch of clips. Each clip's arithmetic is that of a single solve
(the reduction's slices, the resist's partials, the exact max |V| and the EDT are
per clip and in the same order), so the batch must give, clip for clip, bit-identical
phi, masks and loss histories to devel_ilt_solve on each clip alone, and the single
solve is the one held to the oracle. Cases: a ragged side (n = 200: image rows past n in
a 128-row tile must read as zeros per clip, not as the next clip's rows), the WENO5 step
and the curvature modulation m, a partial batch (nclips < capacity), graph capture and
replay, and the full-size workload (2048^2, K = 24, k = 35, beta = 7.5) across a
re-initialisation."""
import numpy as np
import pytest

import synth
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu


def _single(dv, opt, Zt, iters, p, m=None):
    n = Zt.shape[0]
    N = n * n
    phi = torch.zeros(N, dtype=torch.float32, device="cuda")
    M = torch.empty(N, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    clip = dv.Clip(opt, dev(Zt), phi, m=m, mask_out=M, loss_hist=L, l2_hist=l2, pvb_hist=pvb)
    dv.devel_ilt_solve(p, [clip], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    return phi, M, L, l2, pvb


def _batch(dv, bt, targets, iters, p, m=None, ldh=None):
    B = len(targets)
    n = targets[0].shape[0]
    N = n * n
    ldh = ldh or iters + 1
    tg = torch.stack([dev(Zt) for Zt in targets])
    phi = torch.zeros(B, N, dtype=torch.float32, device="cuda")
    M = torch.empty(B, N, dtype=torch.uint8, device="cuda")
    L = torch.zeros(B, ldh, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(B, ldh, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(B, ldh, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run():
        dv.devel_ilt_solve_batch(p, bt, tg, phi, st, m=m, mask_out=M, loss_hist=L, l2_hist=l2, pvb_hist=pvb)
        torch.cuda.synchronize()
        assert int(host(st)[0]) == 0
        return [t.clone() for t in (phi, M, L[:, :iters + 1], l2[:, :iters + 1], pvb[:, :iters + 1])]

    return run


def _check_equal(batch_out, singles):
    for c, one in enumerate(singles):
        for name, a, b in zip(("phi", "mask", "loss", "l2", "pvb"), [x[c] for x in batch_out], one):
            assert torch.equal(a, b), (c, name)


@pytest.mark.parametrize("n,k,upwind,use_graph,with_m", [
    (200, 11, 0, True, False),    # ragged side, graph replay
    (256, 15, 1, False, True),    # WENO5 step, curvature modulation, direct launches
    (256, 15, 0, True, True),
])
def test_batch_equals_single_solves(n, k, upwind, use_graph, with_m):
    dv = need_gpu()
    iters = 6
    o = synth.optics(n, 6, k)
    opt = dv.devel_optics_create(n, o.H, o.w, dv.DEVEL_PREC_BF16X3)
    bt = dv.Batch(opt, 4)
    targets = [synth.rect_clip(60 + i, n=n, border=8) for i in range(3)]  # 3 of capacity 4
    m = None
    if with_m:
        g = torch.Generator(device="cpu").manual_seed(5)
        m = (0.5 + torch.rand(3, n * n, generator=g)).cuda()
    p = dv.ilt_params(dv.resist_params(beta=2.0), iters=iters, reinit_every=3, use_graph=use_graph, upwind=upwind)
    run = _batch(dv, bt, targets, iters, p, m=m, ldh=iters + 3)
    out = run()
    if use_graph:  # the same arguments again: a replay of the captured graph, same results
        for a, b in zip(out, run()):
            assert torch.equal(a, b)
    singles = [_single(dv, opt, Zt, iters, p, m=None if m is None else m[c].contiguous())
               for c, Zt in enumerate(targets)]
    _check_equal(out, singles)
    bt.close()


def test_batch_full_size_equals_single_solves():
    """The full-size workload, two clips, six iterations across the re-initialisation after
    iteration 5."""
    dv = need_gpu()
    n, iters = 2048, 6
    o = synth.optics(n, 24, 35)
    opt = dv.devel_optics_create(n, o.H, o.w, dv.DEVEL_PREC_BF16X3)
    bt = dv.Batch(opt, 2)
    targets = [synth.manhattan_clip(1000), synth.manhattan_clip(1001)]
    p = dv.ilt_params(dv.resist_params(beta=7.5), iters=iters, reinit_every=5)
    out = _batch(dv, bt, targets, iters, p)()
    singles = [_single(dv, opt, Zt, iters, p) for Zt in targets]
    _check_equal(out, singles)
    bt.close()


def test_batch_refuses_what_it_does_not_batch():
    dv = need_gpu()
    o = synth.optics(128, 6, 11)
    opt32 = dv.devel_optics_create(128, o.H, o.w, dv.DEVEL_PREC_FP32)
    with pytest.raises(dv.DevelError):
        dv.Batch(opt32, 2)  # the batch is the compensated-BF16 path
    opt = dv.devel_optics_create(128, o.H, o.w, dv.DEVEL_PREC_BF16X3)
    bt = dv.Batch(opt, 2)
    tg = torch.zeros(3, 128 * 128, dtype=torch.uint8, device="cuda")
    phi = torch.zeros(3, 128 * 128, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dv.DevelError):  # more clips than the capacity
        dv.devel_ilt_solve_batch(dv.ilt_params(iters=2), bt, tg, phi, st)
    with pytest.raises(dv.DevelError):  # conjugate gradients are not batched
        dv.devel_ilt_solve_batch(dv.ilt_params(iters=2, optimizer=1), bt, tg[:2], phi[:2], st)
    hist = torch.zeros(2, 2, dtype=torch.int64, device="cuda")
    with pytest.raises(dv.DevelError):  # history rows shorter than iters + 1
        dv.devel_ilt_solve_batch(dv.ilt_params(iters=2), bt, tg[:2], phi[:2], st, l2_hist=hist)
    bt.close()
