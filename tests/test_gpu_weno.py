"""GPU parity of the WENO5 upwind option (Sec. III-C names WENO for |grad phi|):
devel_levelset_step_weno5 against the oracle's WENO5 step, and whole solves with
DEVEL_UPWIND_WENO5 against the oracle's loop."""
import numpy as np
import pytest

import synth
from oracle import levelset, sdf, solve
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [33, 64, 200, 257])
@pytest.mark.parametrize("use_m", [False, True])
def test_weno_step_matches_oracle(n, use_m):
    dv = need_gpu()
    rng = np.random.default_rng(100 + n)
    Zt = synth.rect_clip(n, n=n, border=2, long=(8, min(96, n - 8))) if n >= 64 else synth.random_mask(n, n, 0.3)
    phi = sdf.tsdf(Zt, -20.0, 40.0).astype(np.float32)
    phi += rng.uniform(-0.3, 0.3, phi.shape).astype(np.float32)
    V = rng.standard_normal((n, n)).astype(np.float32)
    m = rng.uniform(0, 1, (n, n)).astype(np.float32) if use_m else None
    vmax = float(np.abs(V).max())
    dt, lam = 0.5, 0.1
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    vm = torch.tensor([vmax], dtype=torch.float64, device="cuda")
    dv.devel_levelset_step(n, dev(phi), dev(V), vm, dev(m) if use_m else None, dt, lam, out, M, weno5=True)
    torch.cuda.synchronize()
    ref, Mref = levelset.step(phi.astype(np.float64), V.astype(np.float64), vmax,
                              None if m is None else m.astype(np.float64), dt, lam, weno=True)
    got = host(out, n)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 4e-6
    unsure = np.abs(ref) <= 1e-5
    assert np.array_equal(host(M, n)[~unsure], Mref[~unsure])


def test_weno_step_flat_regions_stay_finite():
    """Where phi is flat (all one-sided differences zero, e.g. a clamped TSDF plateau)
    the WENO weights must not divide by zero: the transport term vanishes there."""
    dv = need_gpu()
    n = 64
    phi = np.full((n, n), 40.0, dtype=np.float32)
    phi[20:30, 20:30] = -5.0
    V = np.ones((n, n), dtype=np.float32)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    vm = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    dv.devel_levelset_step(n, dev(phi), dev(V), vm, None, 0.5, 0.0, out, None, weno5=True)
    torch.cuda.synchronize()
    got = host(out, n)
    assert np.isfinite(got).all()
    assert np.array_equal(got[40:, 40:], phi[40:, 40:])


@pytest.mark.parametrize("prec", [0, 1])
def test_weno_solve_matches_oracle(prec):
    dv = need_gpu()
    n, iters = 256, 20
    o = synth.optics(n, 8, 15)
    Zt = synth.rect_clip(1)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    M = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    l2 = torch.zeros(iters + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = dv.ilt_params(dv.resist_params(), iters=iters, upwind=dv.DEVEL_UPWIND_WENO5)
    dv.devel_ilt_solve(p, [dv.Clip(opt, dev(Zt), phi, mask_out=M, l2_hist=l2)], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == 0
    ref = solve.ilt_solve(Zt, o.H, o.w, solve.SolveParams(iters=iters, weno=True))
    mism = np.count_nonzero(host(M, n) != ref.mask) / (n * n)
    assert mism <= 1e-3, mism
    assert abs(int(host(l2)[-1]) - ref.l2[-1]) <= 0.01 * max(ref.l2[-1], 1)
