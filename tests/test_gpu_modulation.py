"""GPU parity of the modulation-branch supervision (Sec. III-B): candidate maps
H(phi_gt + dh), the label search over DSO solves, and the approximated-Heaviside
loss, against the oracle."""
import numpy as np
import pytest

import synth
from oracle import modulation, resist, sdf, solve
from gpu_util import need_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [64, 129])
def test_candidates_match_oracle(n):
    dv = need_gpu()
    Zt = synth.rect_clip(5, n=n, border=4, long=(8, min(96, n - 8)))
    phi = sdf.tsdf(Zt, -20.0, 40.0).astype(np.float32)
    phi += np.random.default_rng(n).uniform(-0.5, 0.5, phi.shape).astype(np.float32)
    dh = np.random.default_rng(1).uniform(-20, 20, 7).astype(np.float32)
    out = torch.empty(len(dh) * n * n, dtype=torch.float32, device="cuda")
    dv.devel_modulation_candidates(n, dev(phi), dh, out)
    torch.cuda.synchronize()
    got = host(out).reshape(len(dh), n, n)
    ref = modulation.candidates(phi.astype(np.float64), dh.astype(np.float64))
    # the decision is taken in FP32 on the GPU: away from phi + dh = 0 it is unique,
    # at the ties it must match the FP32 sum
    tie = np.abs(phi[None] + dh[:, None, None].astype(np.float64)) < 1e-5
    assert np.array_equal(got[~tie], ref[~tie])
    f32 = ((phi[None] + dh[:, None, None]) >= np.float32(0)).astype(np.float32)
    assert np.array_equal(got[tie], f32[tie])


@pytest.mark.parametrize("n", [64, 130])
def test_ahf_loss_matches_oracle(n):
    dv = need_gpu()
    o = synth.optics(n, 2, 5)
    opt = dv.devel_optics_create(n, o.H, o.w)
    rng = np.random.default_rng(n)
    phi = rng.uniform(-0.3, 0.3, (n, n)).astype(np.float32)
    m = (rng.random((n, n)) < 0.4).astype(np.float32)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty(n * n, dtype=torch.float32, device="cuda")
    dv.devel_ahf_loss(opt, dev(phi), dev(m), 0.03, L, g)
    torch.cuda.synchronize()
    Lref, gref = modulation.ahf_loss(phi.astype(np.float64), m.astype(np.float64), 0.03)
    assert abs(float(host(L)[0]) - Lref) <= 1e-5 * Lref
    assert rel_err(host(g, n), gref) <= 1e-5
    # NaN reaches the loss
    phi[1, 2] = np.nan
    dv.devel_ahf_loss(opt, dev(phi), dev(m), 0.03, L)
    torch.cuda.synchronize()
    assert np.isnan(float(host(L)[0]))


def test_label_search_matches_oracle():
    dv = need_gpu()
    n, K, k, iters = 128, 6, 11, 10
    o = synth.optics(n, K, k)
    Zt = synth.rect_clip(6, n=n, border=8)
    p_or = solve.SolveParams(iters=iters, resist=resist.ResistParams(beta=2.0))
    phi_gt = solve.ilt_solve(Zt, o.H, o.w, p_or).phi.astype(np.float32)
    dh = np.random.default_rng(7).uniform(-20, 20, 6).astype(np.float32)
    handles = [dv.devel_optics_create(n, o.H, o.w, 1) for _ in dh]
    p = dv.ilt_params(dv.resist_params(beta=2.0), iters=iters)
    best, final, cands = dv.modulation_search(handles, dev(Zt), dev(phi_gt), dh, p)
    rbest, rfinal, rcands = modulation.search(Zt, o.H, o.w, p_or, phi_gt.astype(np.float64), dh.astype(np.float64))
    # each candidate's final L_DSO within 1% of the oracle's; the chosen label is the
    # oracle's best or within 1% of it
    assert np.all(np.abs(final - rfinal) <= 0.01 * np.abs(rfinal))
    assert best == int(np.argmin(final))            # the device argmin (ties: the first)
    assert rfinal[best] <= 1.01 * min(rfinal)
    assert np.array_equal(host(cands).reshape(len(dh), n, n)[rbest], rcands[rbest].astype(np.float32)) or \
        np.count_nonzero(host(cands).reshape(len(dh), n, n)[rbest] != rcands[rbest]) <= 2
