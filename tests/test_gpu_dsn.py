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


# Resampling between a clip's grid and the network's coarser grid, against the oracle
# (oracle/dsn.py phi_downsample / phi_upsample). FP32 on the GPU: the block sum has
# f^2 - 1 roundings and the interpolation a handful, hence the bounds below.

U32 = 2.0 ** -24


@pytest.mark.parametrize("n,f,nb", [(64, 4, 3), (96, 3, 2), (30, 5, 1), (16, 1, 2)])
def test_phi_resampling_matches_oracle(n, f, nb):
    dv = need_gpu()
    rng = np.random.default_rng(n + f)
    m = n // f
    fine = (rng.standard_normal((nb, n, n)) * 40.0).astype(np.float32)
    coarse = (rng.standard_normal((nb, m, m)) * 10.0).astype(np.float32)
    c_gpu = torch.empty(nb * m * m, dtype=torch.float32, device="cuda")
    f_gpu = torch.empty(nb * n * n, dtype=torch.float32, device="cuda")
    dv.devel_phi_downsample(n, f, dev(fine), c_gpu)
    dv.devel_phi_upsample(n, f, dev(coarse), f_gpu)
    torch.cuda.synchronize()
    down, up = host(c_gpu).reshape(nb, m, m), host(f_gpu).reshape(nb, n, n)
    ref_down, ref_up = dsn.phi_downsample(fine, f), dsn.phi_upsample(coarse, f)
    if f == 1:                       # identity maps: bit-exact
        assert np.array_equal(down, fine) and np.array_equal(up, coarse)
    tol_down = (f * f + 1) * U32 * np.abs(fine).max() / f
    assert np.abs(down - ref_down).max() <= tol_down
    tol_up = f * np.abs(coarse).max() * (8 + 2 * m) * U32
    assert np.abs(up - ref_up).max() <= tol_up


def test_phi_resampling_at_full_clip_size():
    """The bench's sizes (2048^2 clips, a 512^2 network grid, f = 4): every coarse pixel
    of the upsampled-then-downsampled field, and sampled windows of each map against the
    oracle."""
    dv = need_gpu()
    n, f, nb = 2048, 4, 2
    m = n // f
    rng = np.random.default_rng(7)
    coarse = (rng.standard_normal((nb, m, m)) * 10.0).astype(np.float32)
    f_gpu = torch.empty(nb * n * n, dtype=torch.float32, device="cuda")
    c_gpu = torch.empty(nb * m * m, dtype=torch.float32, device="cuda")
    dv.devel_phi_upsample(n, f, dev(coarse), f_gpu)
    dv.devel_phi_downsample(n, f, f_gpu, c_gpu)
    torch.cuda.synchronize()
    up = host(f_gpu).reshape(nb, n, n)
    down = host(c_gpu).reshape(nb, m, m)
    ref_up = dsn.phi_upsample(coarse, f)
    assert np.abs(up - ref_up).max() <= f * np.abs(coarse).max() * 16 * U32   # power-of-two f: exact positions
    for b, I, J in [(0, 0, 0), (1, 496, 3), (0, 255, 256), (1, 496, 496)]:   # 16 x 16 windows inside 512^2
        win = up[b, I * f:I * f + 16 * f, J * f:J * f + 16 * f]
        ref = dsn.phi_downsample(win, f)
        got = down[b, I:I + 16, J:J + 16]
        assert np.abs(got - ref).max() <= (f * f + 1) * U32 * np.abs(win).max() / f


def test_network_on_the_full_clip_grid():
    """The network at the side the full-size learned start uses (512^2, width 32): a zero
    head returns the band-limited input exactly, and a training step gives a finite loss
    and finite outputs."""
    dv = need_gpu()
    S, nb = 512, 2
    net = dv.Dsn(S, nb, 32, seed=5)
    p = net.get_params()
    p[-33:] = 0.0
    net.set_params(p)
    yy, xx = np.mgrid[0:S, 0:S]
    tsdf = np.stack([np.hypot(yy - 200.0, xx - 260.0) - 90.0, 300.0 - np.abs(xx - 256.0) - 0.5]).astype(np.float32)
    out = torch.empty(nb * S * S, dtype=torch.float32, device="cuda")
    net.forward(nb, dev(tsdf), out, B)
    torch.cuda.synchronize()
    assert np.array_equal(host(out).reshape(tsdf.shape), np.clip(tsdf, -B, B))
    net = dv.Dsn(S, nb, 32, seed=6)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train_step(nb, dev(tsdf), dev(tsdf + 3.0), 1e-3, loss, B)
    net.forward(nb, dev(tsdf), out, B)
    torch.cuda.synchronize()
    assert np.isfinite(loss.item()) and loss.item() > 0
    assert np.all(np.isfinite(host(out)))


def test_training_step_in_a_fresh_process():
    """A process whose first and only network is the full-clip one (512^2, width 32), whose
    every forward layer runs on the tensor-core kernel: its training step launches the
    warp-level input-gradient kernel without any earlier forward use of that kernel (which
    once set its shared-memory limit as a side effect), so it is run in a new interpreter."""
    import os
    import subprocess
    import sys
    need_gpu()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, torch\n"
        "import paper_2303_12529_gb300 as dv\n"
        "S, nb = 512, 1\n"
        "net = dv.Dsn(S, nb, 32, seed=7)\n"
        "yy, xx = np.mgrid[0:S, 0:S]\n"
        "x = torch.from_numpy((np.hypot(yy - 200.0, xx - 260.0) - 90.0).astype(np.float32)).cuda()\n"
        "loss = torch.zeros(1, dtype=torch.float64, device='cuda')\n"
        "net.train_step(nb, x, x + 3.0, 1e-3, loss, 16.0)\n"
        "torch.cuda.synchronize()\n"
        "assert np.isfinite(loss.item()) and loss.item() > 0\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("S,nb,width", [(256, 2, 32), (512, 1, 16), (512, 1, 32)])
def test_tensor_core_convolutions_match_oracle(S, nb, width):
    """At side 256 and width 32 the layers with 32, 64 or 128 output channels on planes of
    side >= 128 run on the tcgen05 implicit-GEMM kernel (the layers of levels 0 and 1 and
    of the decoder's levels 1 and 0); at side 512 and width 16 so do those of levels 1 and 2
    and of the decoder's levels 2 and 1, among them 16 -> 32 (one 16-channel step per
    channel block, raw rows copied 8 planes per box) and 96 -> 32 (a 64- and a 32-channel
    block); at side 512 and width 32 (the network of the full-size learned start) every 3x3
    layer does, level 3's 128 -> 256 and 256 -> 256 on the 64^2 plane with the operands
    swapped (weights as A, 64-pixel halo rows as B). The forward pass matches the oracle storing in BF16
    where the GPU does, and the same network computed entirely with the warp-level MMA
    kernel (DEVEL_DSN_NO_TC=1 at creation). At this width the 15 layers store about 10^7
    BF16 activations, and FP32 sums (either kernel) against the oracle's FP64 sums flip some
    of their roundings: the warp-level path sits 1.6% from the BF16-storing oracle here (the
    plain FP64 oracle 1.9% from that one), so the new path is held to the same 2.5% as the
    established one, and the two paths to 2.5% of each other."""
    import os
    dv = need_gpu()
    net = dv.Dsn(S, nb, width, seed=11)
    P = _unflatten(net.get_params(), width)
    P = [p if p.ndim > 1 else p + 0.05 for p in P]      # non-zero biases
    flat = np.concatenate([p.reshape(-1) for p in P]).astype(np.float32)
    net.set_params(flat)
    P = _unflatten(net.get_params(), width)
    yy, xx = np.mgrid[0:S, 0:S]
    tsdf = np.stack([np.hypot(yy - 100.0, xx - 140.0) - 40.0,
                     np.minimum(np.abs(yy - 128.0) - 20.5, 60.0 - np.abs(xx - 90.0))])[:nb].astype(np.float32)
    out = torch.empty(nb * S * S, dtype=torch.float32, device="cuda")
    net.forward(nb, dev(tsdf), out, B)
    os.environ["DEVEL_DSN_NO_TC"] = "1"
    try:
        ref_net = dv.Dsn(S, nb, width, seed=11)
    finally:
        del os.environ["DEVEL_DSN_NO_TC"]
    ref_net.set_params(flat)
    out_mma = torch.empty_like(out)
    ref_net.forward(nb, dev(tsdf), out_mma, B)
    torch.cuda.synchronize()
    x = dsn.band(tsdf[:, None].astype(np.float64), B)
    got = host(out).reshape(nb, 1, S, S) / B
    mma = host(out_mma).reshape(nb, 1, S, S) / B
    assert np.all(np.isfinite(got))
    y16, _ = dsn.forward(P, x, store=bf16)
    e_tc, e_mma, e_pair = rel_err(got - x, y16 - x), rel_err(mma - x, y16 - x), rel_err(got - x, mma - x)
    assert e_tc <= 2.5e-2 and e_mma <= 2.5e-2 and e_pair <= 2.5e-2, (e_tc, e_mma, e_pair)
