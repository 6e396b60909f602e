"""GPU parity of devel_levelset_step and devel_reinit_sdf against the oracle
(Eqs. dso_evolution, numerical-settings, curva_numer, sdf, tsdf)."""
import numpy as np
import pytest

import synth
from oracle import levelset, sdf
from gpu_util import need_gpu, dev, host, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [33, 64, 200, 257])
@pytest.mark.parametrize("use_m", [False, True])
def test_step_matches_oracle(n, use_m):
    dv = need_gpu()
    rng = np.random.default_rng(n)
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
    dv.devel_levelset_step(n, dev(phi), dev(V), vm, dev(m) if use_m else None, dt, lam, out, M)
    torch.cuda.synchronize()
    ref, Mref = levelset.step(phi.astype(np.float64), V.astype(np.float64), vmax,
                              None if m is None else m.astype(np.float64), dt, lam)
    got = host(out, n)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 2e-6
    Mg = host(M, n)
    unsure = np.abs(ref) <= 1e-5
    assert np.array_equal(Mg[~unsure], Mref[~unsure])
    assert np.array_equal(Mg, (got <= 0).astype(np.uint8))


def test_step_zero_vmax_and_no_curvature_is_identity():
    dv = need_gpu()
    n = 50
    phi = np.random.default_rng(1).standard_normal((n, n)).astype(np.float32)
    out = torch.empty(n * n, dtype=torch.float32, device="cuda")
    vm = torch.zeros(1, dtype=torch.float64, device="cuda")
    dv.devel_levelset_step(n, dev(phi), dev(np.ones((n, n), np.float32)), vm, None, 0.5, 0.0, out, None)
    torch.cuda.synchronize()
    assert np.array_equal(host(out, n), phi)


def _reinit(dv, M):
    n = M.shape[0]
    phi = torch.empty(n * n, dtype=torch.float32, device="cuda")
    d2 = torch.empty(n * n, dtype=torch.int32, device="cuda")
    dv.devel_reinit_sdf(n, dev(M.astype(np.uint8)), phi, d2, -100.0, 900.0)
    torch.cuda.synchronize()
    return host(phi, n), host(d2, n)


REINIT_MASKS = {
    "rects256": lambda: synth.rect_clip(0),
    "random200": lambda: synth.random_mask(3, 200, 0.3),
    "sparse130": lambda: synth.random_mask(4, 130, 0.002),
    "empty64": lambda: np.zeros((64, 64), np.uint8),
    "full64": lambda: np.ones((64, 64), np.uint8),
    "single65": lambda: np.pad(np.ones((1, 1), np.uint8), ((40, 24), (3, 61))),
    "checker48": lambda: (np.add.outer(np.arange(48), np.arange(48)) % 2).astype(np.uint8),
    "tiny5": lambda: np.eye(5, dtype=np.uint8),
}


@pytest.mark.parametrize("name", list(REINIT_MASKS))
def test_reinit_bit_exact_distances(name):
    dv = need_gpu()
    M = REINIT_MASKS[name]()
    phi, d2 = _reinit(dv, M)
    ref_d2 = sdf.opposite_class_d2(M)
    assert np.array_equal(d2, ref_d2)
    ref_phi = sdf.tsdf(M)
    # phi = fl(fl(sqrt(d2)) - 0.5): within one float32 ulp of the exact value
    assert np.all(np.abs(phi - ref_phi) <= np.spacing(np.abs(ref_phi).astype(np.float32)) + 1e-30)
    assert np.array_equal((phi <= 0).astype(np.uint8), (M != 0).astype(np.uint8))


@pytest.mark.parametrize("n,kinds", [(200, ("random200", "rects", "empty", "full")), (65, ("single65", "full", "empty"))])
def test_reinit_batch_matches_the_oracle_and_single_calls(n, kinds):
    """devel_reinit_sdf_batch on masks stored back to back (a ragged side, the degenerate
    empty and full masks among them): every clip's d2 equals the oracle's exact squared
    distances, and its phi and d2 are bit-identical to devel_reinit_sdf on that mask alone."""
    dv = need_gpu()
    masks = []
    for i, k in enumerate(kinds):
        if k == "random200":
            masks.append(synth.random_mask(3, n, 0.3))
        elif k == "rects":
            masks.append(synth.rect_clip(7, n=n, border=8))
        elif k == "empty":
            masks.append(np.zeros((n, n), np.uint8))
        elif k == "full":
            masks.append(np.ones((n, n), np.uint8))
        else:
            masks.append(REINIT_MASKS[k]())
    nb = len(masks)
    M = np.stack([m.astype(np.uint8) for m in masks])
    phi = torch.empty(nb * n * n, dtype=torch.float32, device="cuda")
    d2 = torch.empty(nb * n * n, dtype=torch.int32, device="cuda")
    dv.devel_reinit_sdf_batch(n, nb, dev(M), phi, d2, -100.0, 900.0)
    torch.cuda.synchronize()
    phi_b = host(phi).reshape(nb, n, n)
    d2_b = host(d2).reshape(nb, n, n)
    for c in range(nb):
        assert np.array_equal(d2_b[c], sdf.opposite_class_d2(M[c])), c
        phi1, d21 = _reinit(dv, M[c])
        assert np.array_equal(phi_b[c], phi1) and np.array_equal(d2_b[c], d21), c


def test_reinit_full_size_sampled_rows():
    dv = need_gpu()
    M = synth.manhattan_clip(1003)
    phi, d2 = _reinit(dv, M)
    rows = [0, 1, 500, 1023, 1024, 2047]
    ref = sdf.opposite_class_d2(M, rows)
    assert np.array_equal(d2[rows], ref)
    assert np.array_equal((phi <= 0).astype(np.uint8), M)
