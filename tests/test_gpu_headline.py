"""GPU parity of devel_ilt_solve at the full-size workload, the configuration the
throughput is quoted on (Sec. III-A loss with the PVB terms, Sec. III-C loop): the
2048^2 Manhattan clip of seed 1000, K = 24 SOCS kernels of 35 x 35, dose corners
+/-2%, alpha = 1, beta = 7.5, dt = 0.5, lambda = 0.1, 6 iterations with
re-initialisation every 5, on both precision paths, against the FP64 oracle's solve
of the same clip stored by tests/golden/make_oracle_manhattan2048.py (which calls only
oracle/ and the input generators, and stores the optics it used: the solve here is
given the same arrays).

Bars: <= 0.1% thresholded-pixel mismatch of the final mask, L2 and PVBand within 1% at
every iteration, the per-iteration loss within 1%, and the first loss (the target's own
mask) within the bound its image tolerance implies (gpu_util.loss_bound)."""
import os

import numpy as np
import pytest

import synth
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_solve_manhattan2048.npz")
IMAGE_TOL = {0: 1e-5, 1: 2e-4}  # normwise aerial-image tolerance of each precision path


@pytest.fixture(scope="module")
def record():
    rec = np.load(GOLDEN)
    n = 2048
    Zt = np.unpackbits(rec["target_bits"])[: n * n].reshape(n, n)
    # the input generator is deterministic across machines: the stored target is its output
    assert np.array_equal(Zt, synth.manhattan_clip(1000))
    return rec, Zt


@pytest.mark.parametrize("prec", [0, 1])
def test_headline_solve_matches_oracle(record, prec):
    dv = need_gpu()
    rec, Zt = record
    n, iters = 2048, 6
    opt = dv.devel_optics_create(n, rec["H"], rec["w"], prec)
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    pvb = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = dv.ilt_params(dv.resist_params(beta=7.5), dt=0.5, lam=0.1, iters=iters, reinit_every=5)
    dv.devel_ilt_solve(p, [dv.Clip(opt, dev(Zt), phi, mask_out=M, loss_hist=L, l2_hist=l2, pvb_hist=pvb)], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    dv.devel_optics_check(opt)
    ref_mask = np.unpackbits(rec["mask_bits"])[: n * n].reshape(n, n)
    mism = np.count_nonzero(host(M, n) != ref_mask) / (n * n)
    assert mism <= 1e-3, mism
    L, l2, pvb = host(L), host(l2), host(pvb)
    for t in range(iters + 1):
        assert abs(int(l2[t]) - int(rec["l2"][t])) <= 0.01 * max(int(rec["l2"][t]), 1), (t, l2, rec["l2"])
        assert abs(int(pvb[t]) - int(rec["pvb"][t])) <= 0.01 * max(int(rec["pvb"][t]), 100), (t, pvb, rec["pvb"])
        assert abs(L[t] - rec["loss"][t]) <= 0.01 * rec["loss"][t], (t, L, rec["loss"])
    # first iteration: the same mask on both sides, so only the image error moves the loss
    bound = 1.1 * IMAGE_TOL[prec] * float(rec["I0_max"]) * float(rec["R0_abs_sum"]) + 1e-5 * rec["loss"][0]
    assert abs(L[0] - rec["loss"][0]) <= bound, (L[0], rec["loss"][0], bound)
    dv.devel_optics_destroy(opt)
