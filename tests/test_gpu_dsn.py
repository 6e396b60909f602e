"""GPU parity of the DSN level-set branch (Sec. III-B): the network's forward pass, its
gradients and one Adam step against the FP64 oracle (oracle/dsn.py) on a small
configuration (side 32, width 2, batch 2), and the residual start."""
import numpy as np
import pytest

from oracle import dsn, sdf
from gpu_util import need_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu

SIDE, WIDTH, BATCH, B = 32, 2, 2, 16.0


def _unflatten(flat, width):
    P, off = [], 0
    for cin, cout, k in dsn.layer_shapes(width):
        n = cout * cin * k * k
        P.append(flat[off:off + n].astype(np.float64).reshape(cout, cin, k, k))
        off += n
        P.append(flat[off:off + cout].astype(np.float64))
        off += cout
    assert off == flat.size
    return P


def bf16(a):
    """Round to BF16 (round to nearest even), through FP32, as float64: the storage
    precision of the GPU network's activations and weights."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _batch(seed):
    tsdf, gt = [], []
    rng = np.random.default_rng(seed)
    for i in range(BATCH):
        Zt = np.zeros((SIDE, SIDE), np.uint8)
        Zt[6 + i:20 + i, 8:14 + 2 * i] = 1
        t = sdf.tsdf(Zt, -100.0, 900.0)
        tsdf.append(t)
        gt.append(t + rng.normal(0, 2.0, t.shape))     # a stand-in label near the TSDF
    return np.array(tsdf, np.float32), np.array(gt, np.float32)


def test_forward_matches_oracle():
    dv = need_gpu()
    net = dv.Dsn(SIDE, BATCH, WIDTH, seed=3)
    P = _unflatten(net.get_params(), WIDTH)
    P = [p if p.ndim > 1 else p + 0.05 for p in P]         # non-zero biases
    net.set_params(np.concatenate([p.reshape(-1) for p in P]).astype(np.float32))
    P = _unflatten(net.get_params(), WIDTH)
    tsdf, _ = _batch(1)
    phi0 = torch.empty(BATCH * SIDE * SIDE, dtype=torch.float32, device="cuda")
    net.forward(BATCH, dev(tsdf), phi0, B)
    torch.cuda.synchronize()
    x = dsn.band(tsdf[:, None].astype(np.float64), B)
    got = host(phi0).reshape(BATCH, 1, SIDE, SIDE) / B
    # against the plain FP64 network: BF16 storage moves the network's part (y - x) by
    # a few percent; against the oracle storing in BF16 where the GPU does: FP32 sums
    y, _ = dsn.forward(P, x)
    assert rel_err(got - x, y - x) <= 5e-2
    y16, _ = dsn.forward(P, x, store=bf16)
    assert rel_err(got - x, y16 - x) <= 1e-2


def test_zero_head_gives_the_band_limited_tsdf():
    dv = need_gpu()
    net = dv.Dsn(SIDE, BATCH, WIDTH, seed=4)
    p = net.get_params()
    nh = WIDTH + 1                                          # head weights and bias are last
    p[-nh:] = 0.0
    net.set_params(p)
    tsdf, _ = _batch(2)
    phi0 = torch.empty(BATCH * SIDE * SIDE, dtype=torch.float32, device="cuda")
    net.forward(BATCH, dev(tsdf), phi0, B)
    torch.cuda.synchronize()
    assert np.array_equal(host(phi0).reshape(tsdf.shape), np.clip(tsdf, -B, B))


def test_gradients_and_adam_step_match_oracle():
    dv = need_gpu()
    net = dv.Dsn(SIDE, BATCH, WIDTH, seed=5)
    flat0 = net.get_params()
    P = _unflatten(flat0, WIDTH)
    tsdf, gt = _batch(3)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lr = 1e-3
    net.train_step(BATCH, dev(tsdf), dev(gt), lr, loss, B)
    torch.cuda.synchronize()
    x = dsn.band(tsdf[:, None].astype(np.float64), B)
    label = dsn.band(gt[:, None].astype(np.float64), B)
    # the oracle stores activations and weights in BF16 where the GPU does, so that both
    # take the ReLU decisions on the same values
    y, cache = dsn.forward(P, x, store=bf16)
    L, dy = dsn.mse(y, label)
    G = dsn.backward(P, x, cache, dy)
    assert abs(float(host(loss)[0]) - L) <= 1e-3 * L
    Gg = _unflatten(net.grads(), WIDTH)
    for i, (a, b) in enumerate(zip(Gg, G)):
        assert rel_err(a, b) <= 2e-2, (i, rel_err(a, b))
    # Adam's first step moves each parameter by about lr sign(g): the same move as the
    # oracle's except where the gradient is too small for its sign to be certain
    Pr = [p.copy() for p in P]
    dsn.Adam(lr=lr).step(Pr, G, [])
    moved = net.get_params().astype(np.float64) - flat0
    ref = np.concatenate([(a - b).reshape(-1) for a, b in zip(Pr, P)])
    gflat = np.concatenate([g.reshape(-1) for g in G])
    sure = np.abs(gflat) > 0.05 * np.abs(gflat).max()
    assert np.allclose(moved[sure], ref[sure], rtol=0, atol=0.05 * lr)


def test_training_lowers_the_loss():
    dv = need_gpu()
    net = dv.Dsn(SIDE, BATCH, WIDTH, seed=6)
    tsdf, _ = _batch(4)
    gt = tsdf + 3.0            # a learnable label: the level set moved out by 3 px
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    for _ in range(30):
        net.train_step(BATCH, dev(tsdf), dev(gt), 3e-3, loss, B)
        torch.cuda.synchronize()
        hist.append(float(host(loss)[0]))
    assert np.isfinite(hist).all() and hist[-1] < 0.5 * hist[0]


def test_modulation_branch_step_matches_oracle():
    """The modulation branch (Sec. III-B): H_eps of the output, the averaged L_m, its
    gradients and the first Adam step, against the oracle storing in BF16 where the GPU
    does."""
    dv = need_gpu()
    net = dv.Dsn(SIDE, BATCH, WIDTH, seed=7)
    flat0 = net.get_params()
    P = _unflatten(flat0, WIDTH)
    tsdf, _ = _batch(5)
    m_gt = (tsdf > 1.5).astype(np.float32)           # a 0 / 1 label map
    x = dsn.band(tsdf[:, None].astype(np.float64), B)
    m = torch.empty(BATCH * SIDE * SIDE, dtype=torch.float32, device="cuda")
    net.forward_ahf(BATCH, dev(tsdf), m, 0.03, B)
    torch.cuda.synchronize()
    y16, cache = dsn.forward(P, x, store=bf16)
    from oracle import modulation
    assert rel_err(host(m).reshape(y16.shape), modulation.ahf(y16, 0.03)) <= 2e-2
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train_step_ahf(BATCH, dev(tsdf), dev(m_gt), 1e-3, loss, 0.03, B)
    torch.cuda.synchronize()
    L, dy = dsn.ahf_mean(y16, m_gt[:, None].astype(np.float64), 0.03)
    G = dsn.backward(P, x, cache, dy)
    assert abs(float(host(loss)[0]) - L) <= 1e-2 * L
    Gg = _unflatten(net.grads(), WIDTH)
    for i, (a, b) in enumerate(zip(Gg, G)):
        assert rel_err(a, b) <= 5e-2, (i, rel_err(a, b))
