"""FP64 CPU oracle of the learned preconditioner stage's U-Net.

TEST INFRASTRUCTURE ONLY (same rules as ib_oracle: used by tests/ and bench's
CPU leg, never by the library).  The network is not in the paper; its
definition is the one documented in include/ib.h:

  level 1 (N):   conv3x3 4->16, GELU, conv3x3 16->16, GELU          -> s1
  level 2 (N/2): avgpool(s1), conv 16->32, GELU, conv 32->32, GELU  -> s2
  level 3 (N/4): avgpool(s2), conv 32->64, GELU, conv 64->64, GELU
  up:            nearest-upsample, concat [up | s2], conv 96->32, GELU, conv 32->32, GELU
  up:            nearest-upsample, concat [up | s1], conv 48->16, GELU, conv 16->16, GELU
  head:          conv1x1 16->3

Convolutions use circular padding (the grid is periodic).  Parameters are one
vector [W_0 b_0 W_1 b_1 ...] with W_l in [c_out][c_in][k][k].  With bf16=True the
weights are rounded to bfloat16 (round to nearest even) before use, as the GPU
kernels do; biases stay as given.  The backward pass is written out by hand
(reverse-mode chain rule through every layer) and pinned against finite
differences in the tests.  The forward pass is pinned on its own: the
convolution against an FFT circular cross-correlation, GELU at tabulated values
of the normal CDF, pooling and upsampling on hand-worked arrays, and the skip
order along single-channel paths.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

LAYERS = [  # (c_in, c_out, k, level, gelu)
    (4, 16, 3, 0, True), (16, 16, 3, 0, True),
    (16, 32, 3, 1, True), (32, 32, 3, 1, True),
    (32, 64, 3, 2, True), (64, 64, 3, 2, True),
    (96, 32, 3, 1, True), (32, 32, 3, 1, True),
    (48, 16, 3, 0, True), (16, 16, 3, 0, True),
    (16, 3, 1, 0, False),
]


def param_count():
    return sum(co * ci * k * k + co for ci, co, k, _, _ in LAYERS)


def unpack(theta):
    out, off = [], 0
    for ci, co, k, _, _ in LAYERS:
        W = theta[off:off + co * ci * k * k].reshape(co, ci, k, k)
        off += co * ci * k * k
        b = theta[off:off + co]
        off += co
        out.append((W, b))
    return out


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _shifted(x, dy, dx, R):
    # value at (y, x) = x[y + dy - R, x + dx - R] (circular)
    return np.roll(np.roll(x, -(dy - R), axis=1), -(dx - R), axis=2)


def conv(x, W, b):
    co, ci, k, _ = W.shape
    R = k // 2
    out = np.broadcast_to(b[:, None, None], (co,) + x.shape[1:]).astype(np.float64).copy()
    for dy in range(k):
        for dx in range(k):
            out += np.einsum("oc,chw->ohw", W[:, :, dy, dx], _shifted(x, dy, dx, R))
    return out


def conv_backward(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) with respect to x, W and b."""
    co, ci, k, _ = W.shape
    R = k // 2
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for dy in range(k):
        for dxx in range(k):
            xs = _shifted(x, dy, dxx, R)
            dW[:, :, dy, dxx] = np.einsum("ohw,chw->oc", g, xs)
            contrib = np.einsum("oc,ohw->chw", W[:, :, dy, dxx], g)
            dx += np.roll(np.roll(contrib, dy - R, axis=1), dxx - R, axis=2)
    return dx, dW, g.sum(axis=(1, 2))


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def pool(x):
    C, H, _ = x.shape
    return x.reshape(C, H // 2, 2, H // 2, 2).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(g):
    C, H, _ = g.shape
    return g.reshape(C, H // 2, 2, H // 2, 2).sum(axis=(2, 4))


def forward(theta, x, bf16=True, keep=False):
    """y = net(x) for x [4, N, N]; with keep, also the intermediate values."""
    P = unpack(np.asarray(theta, dtype=np.float64))
    if bf16:
        P = [(bf16_round(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in P]
    x = np.asarray(x, dtype=np.float64)
    pre, act = [None] * 11, [None] * 11

    def layer(i, inp):
        pre[i] = conv(inp, *P[i])
        act[i] = gelu(pre[i]) if LAYERS[i][4] else pre[i]
        return act[i]

    a1 = layer(1, layer(0, x))
    p1 = pool(a1)
    a3 = layer(3, layer(2, p1))
    p2 = pool(a3)
    a5 = layer(5, layer(4, p2))
    c2 = np.concatenate([up(a5), a3], axis=0)
    a7 = layer(7, layer(6, c2))
    c1 = np.concatenate([up(a7), a1], axis=0)
    a9 = layer(9, layer(8, c1))
    y = layer(10, a9)
    if keep:
        return y, dict(P=P, pre=pre, act=act, p1=p1, p2=p2, c1=c1, c2=c2, x=x)
    return y


def loss(theta, x, t, bf16=True):
    y = forward(theta, x, bf16)
    t = np.asarray(t, dtype=np.float64)
    return float(((y - t) ** 2).sum() / (t ** 2).sum())


def loss_and_grad(theta, x, t, bf16=True):
    """Relative squared error and its gradient with respect to theta."""
    y, c = forward(theta, x, bf16, keep=True)
    t = np.asarray(t, dtype=np.float64)
    tn = (t ** 2).sum()
    L = float(((y - t) ** 2).sum() / tn)
    P, pre, act = c["P"], c["pre"], c["act"]
    grads = [None] * 11

    def back(i, inp, g_act):
        g = g_act * gelu_grad(pre[i]) if LAYERS[i][4] else g_act
        dx, dW, db = conv_backward(inp, P[i][0], g)
        grads[i] = (dW, db)
        return dx

    g = 2.0 * (y - t) / tn
    g9 = back(10, act[9], g)
    g8 = back(9, act[8], g9)
    gc1 = back(8, c["c1"], g8)
    g7 = up_backward(gc1[:32])
    g1_skip = gc1[32:]
    g6 = back(7, act[6], g7)
    gc2 = back(6, c["c2"], g6)
    g5 = up_backward(gc2[:64])
    g3_skip = gc2[64:]
    g4 = back(5, act[4], g5)
    gp2 = back(4, c["p2"], g4)
    g3 = pool_backward(gp2) + g3_skip
    g2 = back(3, act[2], g3)
    gp1 = back(2, c["p1"], g2)
    g1 = pool_backward(gp1) + g1_skip
    g0 = back(1, act[0], g1)
    back(0, c["x"], g0)
    flat = []
    for dW, db in grads:
        flat.append(dW.ravel())
        flat.append(db.ravel())
    return L, np.concatenate(flat)
