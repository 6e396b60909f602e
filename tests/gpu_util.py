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
