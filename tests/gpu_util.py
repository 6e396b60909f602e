"""Helpers of the GPU parity tests: device setup and error measures."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_12529_gb300 as dv  # fails loudly if the library is missing
    return dv


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.reshape(-1).cuda()


def host(t, n=None):
    a = t.detach().cpu().numpy()
    return a.reshape(n, n) if n is not None else a


def rel_err(got, ref):
    """Normwise relative error: max |got - ref| / max |ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def loss_bound(I, R, L, image_tol):
    """How far a loss evaluated on an image with normwise error <= image_tol may sit from
    the oracle's L: to first order |dL| <= sum_p |dL/dI(p)| |dI(p)| <= image_tol max|I|
    sum_p |R(p)| (R = dL/dI of the oracle), plus 1e-5 |L| for the FP32 per-pixel resist
    (the resist test's tolerance given the same image), with 10% slack for the
    second-order term (|d2L/dI2| <= (2 sigma_z)^2 per pixel and image_tol^2 ~ 4e-8)."""
    return 1.1 * image_tol * float(np.abs(I).max()) * float(np.abs(R).sum()) + 1e-5 * abs(float(L))
