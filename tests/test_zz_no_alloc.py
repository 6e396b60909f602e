"""The allocation-free TSDF entry point, devel_reinit_sdf_static.

It serves callers that cannot allocate device memory and so cannot hand the
library the distance scratch that devel_reinit_sdf takes (an embedder whose
device memory belongs to its own pool allocator, or a loop that must not pay
the synchronisation of cudaMalloc/cudaFree). Its scratch is a static device
array of 2048 x 2048 words inside the library. This test calls it through the
C ABI twice in a row, on different sizes and masks, and checks each result
against devel_reinit_sdf with a caller-provided scratch: the kernels are the
same, so phi must match bit for bit (the tolerance of the reinit tests). It
also checks that sizes beyond the array are refused. The file is named to be
collected last.
"""
import numpy as np
import pytest

import synth
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu


def _reference(dv, n, M):
    phi = torch.empty(n * n, dtype=torch.float32, device="cuda")
    d2 = torch.empty(n * n, dtype=torch.int32, device="cuda")
    dv.devel_reinit_sdf(n, M, phi, d2, -100.0, 900.0)
    return phi


def test_static_scratch_matches_caller_scratch_twice():
    dv = need_gpu()
    cases = [
        (2048, synth.manhattan_clip(1005)),             # the largest size the array holds
        (200, synth.random_mask(21, 200, 0.02)),         # then a smaller, sparse one
    ]
    for n, mask in cases:
        M = dev(mask.astype(np.uint8))
        phi_s = torch.full((n * n,), float("nan"), dtype=torch.float32, device="cuda")
        dv.devel_reinit_sdf_static(n, M, phi_s, -100.0, 900.0)
        phi_r = _reference(dv, n, M)
        torch.cuda.synchronize()
        a, b = host(phi_s), host(phi_r)
        assert np.array_equal(a, b)
        assert np.array_equal((a.reshape(n, n) <= 0).astype(np.uint8), (mask != 0).astype(np.uint8))


def test_static_scratch_refuses_sizes_beyond_the_array():
    dv = need_gpu()
    n = dv.REINIT_STATIC_MAX_N + 1
    M = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    phi = torch.empty(n * n, dtype=torch.float32, device="cuda")
    with pytest.raises(dv.DevelError) as e:
        dv.devel_reinit_sdf_static(n, M, phi)
    assert e.value.code == dv.DEVEL_EINVAL and str(dv.REINIT_STATIC_MAX_N) in str(e.value)
