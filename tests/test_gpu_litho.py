"""GPU parity of the lithography calls against the FP64 oracle (Sec. II-B,
Eq. ilt_gradient): devel_litho_forward, devel_resist_loss, devel_litho_adjoint.

Tolerance for the FP32 path: normwise relative error (max |gpu - oracle| /
max |oracle|) <= 1e-5 on the aerial image and on dL/dM. Sizes span several
tiles and ragged tails (n not a multiple of 16, 64 or 32).
"""
import numpy as np
import pytest

import synth
from oracle import litho, resist
from gpu_util import need_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16X3 = 2e-4
PRECISIONS = [(0, TOL_FP32), (1, TOL_BF16X3)]  # DEVEL_PREC_FP32, DEVEL_PREC_BF16X3

CASES = [
    # (n, K, k, kind)
    (64, 4, 7, "random_kernels"),
    (200, 6, 11, "optics"),       # ragged: 200 = 3*64 + 8
    (256, 8, 15, "optics"),       # the 256^2 rectangle workload's optics
    (130, 5, 9, "random_kernels"),
]


def _model(n, K, k, kind, seed=0):
    if kind == "optics":
        o = synth.optics(n, K, k)
        return o.H, o.w
    return synth.random_kernels(100 + seed, K, k)


def _masks(n):
    yield "binary_random", synth.random_mask(1, n, 0.3).astype(np.float64)
    yield "rects", synth.rect_clip(2, n=n, border=4).astype(np.float64)
    yield "real", synth.random_field(3, n, -0.5, 1.5)


@pytest.mark.parametrize("prec,tol", PRECISIONS)
@pytest.mark.parametrize("n,K,k,kind", CASES)
def test_forward_matches_oracle(n, K, k, kind, prec, tol):
    dv = need_gpu()
    H, w = _model(n, K, k, kind)
    opt = dv.devel_optics_create(n, H, w, prec)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    for name, M in _masks(n):
        Mf = M.astype(np.float32)
        dv.devel_litho_forward(opt, dev(Mf), out)
        torch.cuda.synchronize()
        ref = litho.aerial(Mf.astype(np.float64), H.astype(np.complex64).astype(np.complex128),
                           w.astype(np.float32).astype(np.float64))
        e = rel_err(host(out, n), ref)
        assert e <= tol, (name, e)
    dv.devel_optics_check(opt)


def test_forward_clear_field_and_empty_mask():
    dv = need_gpu()
    n = 96
    o = synth.optics(n, 6, 9)
    opt = dv.devel_optics_create(n, o.H, o.w)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    dv.devel_litho_forward(opt, torch.ones(n * n, device="cuda"), out)
    torch.cuda.synchronize()
    expect = float(np.sum(o.w * np.abs(o.H[:, o.r, o.r]) ** 2))
    assert np.max(np.abs(host(out) - expect)) <= 1e-5 * expect
    dv.devel_litho_forward(opt, torch.zeros(n * n, device="cuda"), out)
    torch.cuda.synchronize()
    assert np.all(host(out) == 0.0)


@pytest.mark.parametrize("beta", [0.0, 7.5])
def test_resist_loss_matches_oracle(beta):
    dv = need_gpu()
    n = 200
    o = synth.optics(n, 4, 9)
    opt = dv.devel_optics_create(n, o.H, o.w)
    rng = np.random.default_rng(5)
    I = rng.uniform(0.0, 0.5, (n, n)).astype(np.float32)
    I[:10, :10] = 0.225  # ties print
    Zt = (rng.random((n, n)) < 0.4).astype(np.uint8)
    p = dv.resist_params(beta=beta)
    R = torch.empty(n * n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(4, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    dv.devel_resist_loss(opt, dev(I), dev(Zt), p, R, loss, cnt)
    torch.cuda.synchronize()
    ref = resist.resist(I.astype(np.float64), Zt, resist.ResistParams(beta=beta))
    assert rel_err(host(R, n), ref.R) <= TOL_FP32
    lh = host(loss)
    assert abs(lh[0] - ref.loss) <= 1e-5 * ref.loss
    assert np.allclose(lh[1:], ref.loss_terms, rtol=1e-5)
    # integer metrics: thresholds decided in the kernel's precision (FP32) on both sides
    th = np.float32(0.225)
    d2i, d2o = np.float32(0.98) * np.float32(0.98), np.float32(1.02) * np.float32(1.02)
    l2 = int(np.count_nonzero((I >= th) != (Zt != 0)))
    pvb = int(np.count_nonzero(((d2i * I) >= th) != ((d2o * I) >= th)))
    assert host(cnt).tolist() == [l2, pvb]


@pytest.mark.parametrize("prec,tol", PRECISIONS)
@pytest.mark.parametrize("n,K,k,kind", CASES)
def test_adjoint_matches_oracle(n, K, k, kind, prec, tol):
    dv = need_gpu()
    H, w = _model(n, K, k, kind, seed=1)
    opt = dv.devel_optics_create(n, H, w, prec)
    rng = np.random.default_rng(n)
    V = torch.empty(n * n, dtype=torch.float32, device="cuda")
    vmax = torch.zeros(1, dtype=torch.float64, device="cuda")
    Hc = H.astype(np.complex64).astype(np.complex128)
    wc = w.astype(np.float32).astype(np.float64)
    for name, M in _masks(n):
        Mf = M.astype(np.float32)
        R = rng.standard_normal((n, n)).astype(np.float32)
        dv.devel_litho_adjoint(opt, dev(Mf), dev(R), V, vmax)
        torch.cuda.synchronize()
        ref = litho.aerial_gradient(Mf.astype(np.float64), R.astype(np.float64), Hc, wc)
        e = rel_err(host(V, n), ref)
        assert e <= tol, (name, e)
        vm = float(host(vmax)[0])
        assert abs(vm - np.abs(ref).max()) <= tol * np.abs(ref).max()
        assert vm == float(np.abs(host(V)).max())
    dv.devel_optics_check(opt)


@pytest.mark.parametrize("prec,tol", PRECISIONS)
def test_forward_full_size(prec, tol):
    """2048^2, K = 24, k = 35 (the full-size workload's model), Manhattan
    clip, against the oracle's full-size FFT image."""
    dv = need_gpu()
    n = 2048
    o = synth.optics(n, 24, 35)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    Zt = synth.manhattan_clip(1000)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    dv.devel_litho_forward(opt, dev(Zt.astype(np.float32)), out)
    torch.cuda.synchronize()
    ref = litho.aerial(Zt.astype(np.float64), o.H.astype(np.complex64).astype(np.complex128),
                       o.w.astype(np.float32).astype(np.float64))
    got = host(out, n)
    assert rel_err(got, ref) <= tol
    dv.devel_optics_check(opt)


@pytest.mark.parametrize("prec,tol", PRECISIONS)
def test_adjoint_full_size(prec, tol):
    dv = need_gpu()
    n = 2048
    o = synth.optics(n, 24, 35)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    Zt = synth.manhattan_clip(1001).astype(np.float32)
    R = synth.random_field(9, n, -1.0, 1.0).astype(np.float32)
    V = torch.empty(n * n, dtype=torch.float32, device="cuda")
    vmax = torch.zeros(1, dtype=torch.float64, device="cuda")
    dv.devel_litho_adjoint(opt, dev(Zt), dev(R), V, vmax)
    torch.cuda.synchronize()
    ref = litho.aerial_gradient(Zt.astype(np.float64), R.astype(np.float64),
                                o.H.astype(np.complex64).astype(np.complex128),
                                o.w.astype(np.float32).astype(np.float64))
    assert rel_err(host(V, n), ref) <= tol
    dv.devel_optics_check(opt)


@pytest.mark.parametrize("n,K,k,kind", [(512, 6, 11, "optics"), (200, 6, 11, "optics")])
def test_autotuned_tiles_keep_parity(n, K, k, kind):
    """devel_optics_autotune only changes tile shapes: afterwards the forward image and
    dL/dM still match the oracle within the compensated-BF16 tolerance, and the chosen
    shapes are among the tuner's candidates."""
    dv = need_gpu()
    H, w = _model(n, K, k, kind)
    opt = dv.devel_optics_create(n, H, w, dv.DEVEL_PREC_BF16X3)
    dv.devel_optics_autotune(opt)
    cfg = dv.devel_optics_config(opt)
    ldn = -(-n // 64) * 64
    assert cfg["expand_tile_n"] in (64, 128)
    assert cfg["reduce_split"] % 64 == 0 and 64 <= cfg["reduce_split"] <= max(512, ldn)
    Hc = H.astype(np.complex64).astype(np.complex128)
    wc = w.astype(np.float32).astype(np.float64)
    M = synth.rect_clip(2, n=n, border=4).astype(np.float32)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    dv.devel_litho_forward(opt, dev(M), out)
    R = synth.random_field(5, n, -1.0, 1.0).astype(np.float32)
    V = torch.empty(n * n, dtype=torch.float32, device="cuda")
    vm = torch.zeros(1, dtype=torch.float64, device="cuda")
    dv.devel_litho_adjoint(opt, dev(M), dev(R), V, vm)
    torch.cuda.synchronize()
    dv.devel_optics_check(opt)
    assert rel_err(host(out, n), litho.aerial(M.astype(np.float64), Hc, wc)) <= TOL_BF16X3
    refV = litho.aerial_gradient(M.astype(np.float64), R.astype(np.float64), Hc, wc)
    assert rel_err(host(V, n), refV) <= TOL_BF16X3
