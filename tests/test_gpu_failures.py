"""Failure detection on the GPU without a GPU fault: a bounded device wait that
runs out, and non-finite values reaching the solver's status word. Nothing here
faults, traps or hangs the GPU: the wait gives up after about one second and the
context stays usable; the non-finite values come from the host (a NaN in the
kernel spectra)."""
import time

import numpy as np
import pytest

import synth
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_bounded_wait_gives_up_and_context_survives(prec):
    dv = need_gpu()
    n, K, k = 64, 4, 7
    o = synth.optics(n, K, k)
    opt = dv.devel_optics_create(n, o.H, o.w, prec)
    t0 = time.perf_counter()
    dv.devel_selftest_bounded_wait(opt)
    with pytest.raises(dv.DevelError) as ei:
        dv.devel_optics_check(opt)
    assert ei.value.code == dv.DEVEL_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    dv.devel_optics_check(opt)  # the flag was cleared
    # the context still works: a forward call gives a finite image
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    dv.devel_litho_forward(opt, dev(synth.rect_clip(1, n=n, border=4).astype(np.float32)), out)
    torch.cuda.synchronize()
    dv.devel_optics_check(opt)
    assert np.isfinite(host(out)).all() and host(out).max() > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_nonfinite_spectra_set_enan(prec):
    """A NaN in one kernel spectrum makes the image, the loss and the velocity
    non-finite; the solve reports DEVEL_ENAN in its status word (from the FP64 loss
    reduction and from the max |V| reduction) instead of silently stepping."""
    dv = need_gpu()
    n, K, k, iters = 64, 4, 7, 2
    o = synth.optics(n, K, k)
    H = o.H.copy()
    H[0, k // 2, k // 2] = np.nan
    opt = dv.devel_optics_create(n, H, o.w, prec)
    Zt = synth.rect_clip(3, n=n, border=4)
    phi = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    clip = dv.Clip(opt, dev(Zt), phi, loss_hist=L)
    dv.devel_ilt_solve(dv.ilt_params(iters=iters), [clip], st)
    torch.cuda.synchronize()
    assert int(host(st)[0]) == dv.DEVEL_ENAN
    assert not np.isfinite(host(L)).all()
