"""Level-set branch of DevelSet-Net (DSN), FP64 (test infrastructure only).

Sec. III-B: a convolutional encoder-decoder maps the target image to an initial
level-set function phi_0 for DSO, trained with the mean squared error to the
level set that DSO converges to (phi_gt); DSO then refines it (Sec. III-C). The paper
gives no layer list. Reading: four
levels with widths c, 2c, 4c, 8c (c = 32: 32 .. 256 channels), two 3x3 convolutions
(zero padding 1, bias, ReLU) per level, 2x2 average pooling down, nearest-neighbour
2x upsampling up, the encoder's level output concatenated after the upsampled
decoder input (channels [up, skip]), and a 1x1 convolution to one channel.

Input and output are band-limited level sets: x = clip(TSDF(Z_t), -B, B) / B and the
network predicts y = x + head(...) (a residual on the target's own TSDF, so a
network with zero head weights returns the plain DSO start); phi_0 = B y. Labels are
clip(phi_gt, -B, B) / B with B = 16 pixels; the loss is the mean over pixels of
(y - label)^2.

Tensors are NCHW float64. Parameters are a flat list in layer order, each layer's
weight [cout][cin][k][k] then bias [cout]; Adam (Kingma & Ba) updates them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BAND = 16.0


def layer_shapes(c: int):
    """(cin, cout, k) of every convolution, in order."""
    L = []
    w = [c, 2 * c, 4 * c, 8 * c]
    cin = 1
    for lv in range(4):                       # encoder levels 1..3 and the bottleneck
        L += [(cin, w[lv], 3), (w[lv], w[lv], 3)]
        cin = w[lv]
    for lv in (2, 1, 0):                      # decoder: up(from level lv+1) ++ skip(level lv)
        L += [(w[lv + 1] + w[lv], w[lv], 3), (w[lv], w[lv], 3)]
    L.append((w[0], 1, 1))                    # head
    return L


def init_params(c: int, seed: int):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    P = []
    for cin, cout, k in layer_shapes(c):
        std = np.sqrt(2.0 / (cin * k * k))
        P.append(rng.standard_normal((cout, cin, k, k)) * std)
        P.append(np.zeros(cout))
    return P


def conv(x, W, b):
    """Cross-correlation with zero padding (k - 1) / 2: y[n,o,i,j] = b[o] +
    sum_{c,u,v} W[o,c,u,v] x[n,c,i+u-r,j+v-r]."""
    k = W.shape[2]
    r = (k - 1) // 2
    N, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    y = np.zeros((N, W.shape[0], H, Wd))
    for u in range(k):
        for v in range(k):
            y += np.einsum("oc,nchw->nohw", W[:, :, u, v], xp[:, :, u:u + H, v:v + Wd])
    return y + b[None, :, None, None]


def conv_backward(x, W, dy):
    """Gradients of conv: (dx, dW, db)."""
    k = W.shape[2]
    r = (k - 1) // 2
    N, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for u in range(k):
        for v in range(k):
            dW[:, :, u, v] = np.einsum("nohw,nchw->oc", dy, xp[:, :, u:u + H, v:v + Wd])
            dxp[:, :, u:u + H, v:v + Wd] += np.einsum("oc,nohw->nchw", W[:, :, u, v], dy)
    return dxp[:, :, r:r + H, r:r + Wd], dW, dy.sum(axis=(0, 2, 3))


def avgpool(x):
    """Down one level of the encoder (Sec. III-B reading): the mean of each 2 x 2 block."""
    N, C, H, W = x.shape
    return x.reshape(N, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def avgpool_backward(dy):
    """Adjoint of avgpool: each gradient spread over its 2 x 2 block, times 1/4."""
    return np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3) / 4.0


def upsample(x):
    """Up one level of the decoder (Sec. III-B reading): nearest-neighbour 2x."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def upsample_backward(dy):
    """Adjoint of upsample: the sum over each 2 x 2 block."""
    N, C, H, W = dy.shape
    return dy.reshape(N, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(P, x, store=None):
    """Returns (y, cache). x: [N, 1, S, S] band-limited input level set.

    store: optional rounding applied where a storage format is narrower than FP64
    (the stored activations, the weights a convolution uses, the first layer's input;
    e.g. BF16), so that decisions taken on stored values (the ReLU masks of the
    backward pass) can be reproduced in another precision. None: plain FP64."""
    rnd = store if store is not None else (lambda a: a)
    cache = []
    li = [0]

    def cv(h, relu=True):
        W, b = rnd(P[2 * li[0]]), P[2 * li[0] + 1]
        li[0] += 1
        z = conv(h, W, b)
        out = rnd(np.maximum(z, 0.0)) if relu else z
        cache.append((h, W, out, relu))
        return out

    h = rnd(x)
    skips = []
    for lv in range(4):
        if lv > 0:
            h = rnd(avgpool(h))
        h = cv(cv(h))
        skips.append(h)
    for lv in (2, 1, 0):
        h = np.concatenate([upsample(h), skips[lv]], axis=1)
        h = cv(cv(h))
    y = x + cv(h, relu=False)
    return y, (cache, skips)


def backward(P, x, cache, dy):
    """Gradients of the parameters (flat list in P's order) for dL/dy = dy."""
    convs, skips = cache
    G = [None] * len(P)
    ci = [len(convs)]

    def cvb(dout):
        ci[0] -= 1
        h, W, out, relu = convs[ci[0]]
        dz = dout * (out > 0) if relu else dout
        dh, dW, db = conv_backward(h, W, dz)
        G[2 * ci[0]], G[2 * ci[0] + 1] = dW, db
        return dh

    dh = cvb(dy)                                   # head
    dskip = [np.zeros_like(s) for s in skips]
    for lv in (0, 1, 2):                           # decoder in reverse
        dcat = cvb(cvb(dh))
        cu = dcat.shape[1] - skips[lv].shape[1]
        dskip[lv] += dcat[:, cu:]
        dh = upsample_backward(dcat[:, :cu])
    for lv in (3, 2, 1, 0):                        # encoder in reverse
        dh = dh + dskip[lv] if lv < 3 else dh
        dh = cvb(cvb(dh))
        if lv > 0:
            dh = avgpool_backward(dh)
    return G


def mse(y, label):
    """Training loss of the level-set branch (Sec. III-B): mean (y - label)^2 and its gradient in y."""
    d = y - label
    return float(np.mean(d * d)), 2.0 * d / d.size


def ahf_mean(y, m_gt, eps: float):
    """Loss of the modulation branch (Sec. III-B, L_m per pixel, averaged): the branch's
    output y is read as phi_m and passed through the approximated Heaviside
    H_eps(y) = (1 + (2/pi) atan(y/eps)) / 2; returns mean (H_eps(y) - m_gt)^2 and its
    gradient in y."""
    y = np.asarray(y, dtype=np.float64)
    h = 0.5 * (1.0 + (2.0 / np.pi) * np.arctan(y / eps))
    r = h - np.asarray(m_gt, dtype=np.float64)
    dh = (1.0 / np.pi) * eps / (eps * eps + y * y)
    return float(np.mean(r * r)), 2.0 * r * dh / r.size


@dataclass
class Adam:
    """Adam (Kingma and Ba) with bias correction, the optimiser of the network's training."""
    lr: float = 1e-3
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    t: int = 0

    def step(self, P, G, state):
        """One update of every parameter; state = list of (m, v), created on first use."""
        self.t += 1
        if not state:
            state.extend((np.zeros_like(p), np.zeros_like(p)) for p in P)
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for i, (p, g) in enumerate(zip(P, G)):
            m, v = state[i]
            m[...] = self.b1 * m + (1.0 - self.b1) * g
            v[...] = self.b2 * v + (1.0 - self.b2) * g * g
            p -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)


def phi_downsample(phi, f: int):
    """Level set on the coarse grid of a DSN that runs at 1/f of the clip's side (Sec.
    III-B/C: the network predicts phi_0, DSO refines it on the clip's own grid).
    Reading: each coarse pixel takes the mean of its f x f block, and distances are
    re-expressed in coarse pixels (divided by f). phi: [..., n, n], n a multiple of f."""
    a = np.asarray(phi, dtype=np.float64)
    n = a.shape[-1]
    m = n // f
    out = np.zeros(a.shape[:-2] + (m, m))
    for I in range(m):
        for J in range(m):
            out[..., I, J] = a[..., f * I:f * I + f, f * J:f * J + f].mean(axis=(-2, -1)) / f
    return out


def phi_upsample(c, f: int):
    """The coarse level set back on the fine grid: bilinear interpolation with the
    pixel centres aligned (fine centre p sits at coarse coordinate (p + 1/2) / f - 1/2),
    coarse indices clamped to the grid, distances back in fine pixels (times f)."""
    c = np.asarray(c, dtype=np.float64)
    m = c.shape[-1]
    n = m * f
    pos = (np.arange(n) + 0.5) / f - 0.5
    i0 = np.floor(pos).astype(np.int64)
    t = pos - i0
    ia, ib = np.clip(i0, 0, m - 1), np.clip(i0 + 1, 0, m - 1)
    rows = (1.0 - t)[:, None] * c[..., ia, :] + t[:, None] * c[..., ib, :]            # [..., n, m]
    out = (1.0 - t)[None, :] * rows[..., :, ia] + t[None, :] * rows[..., :, ib]       # [..., n, n]
    return f * out


def band(phi, B: float = BAND):
    """Band-limited level set in network units: clip(phi, -B, B) / B."""
    return np.clip(np.asarray(phi, dtype=np.float64), -B, B) / B
