"""Pins of the U-Net oracle: finite differences, equivariance, closed forms."""
import numpy as np
import pytest

import ib_workloads as W
from oracle import unet_oracle as U


def test_param_count_and_shapes_agree():
    n = sum(co * ci * k * k + co for ci, co, k in W.UNET_SHAPES)
    assert U.param_count() == n == 118451  # worked by hand: 592+2320+4640+9248+18496+36928+27680+9248+6928+2320+51
    assert [(ci, co, k) for ci, co, k, _, _ in U.LAYERS] == W.UNET_SHAPES


def test_bf16_rounding_closed_forms():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7, -2.5, 3.0e-3])
    r = U.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # exact tie -> even mantissa
    assert r[2] == 1.0 + 2.0 ** -7          # above the tie -> up
    assert r[3] == 1.0 + 2.0 ** -7          # representable
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8


def _case(N=16, seed=3):
    th = W.unet_init_params(seed).astype(np.float64)
    th[1::97] += 0.05  # non-zero biases somewhere
    rng = np.random.default_rng(seed + 1)
    x = rng.standard_normal((4, N, N))
    t = rng.standard_normal((3, N, N))
    return th, x, t


def test_gradient_matches_finite_differences():
    th, x, t = _case()
    L, g = U.loss_and_grad(th, x, t, bf16=False)
    assert abs(L - U.loss(th, x, t, bf16=False)) < 1e-12
    rng = np.random.default_rng(7)
    eps = 1e-6
    for _ in range(3):
        d = rng.standard_normal(th.size)
        fd = (U.loss(th + eps * d, x, t, False) - U.loss(th - eps * d, x, t, False)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-5 * max(abs(fd), 1e-3), (fd, g @ d)
    # single coordinates of the first and last layers and of a middle bias
    offs = np.cumsum([0] + [co * ci * k * k + co for ci, co, k in W.UNET_SHAPES])
    for idx in (0, 17, int(offs[5]) + 3, int(offs[10]) + 5, int(offs[11]) - 1):
        e = np.zeros_like(th)
        e[idx] = 1.0
        fd = (U.loss(th + 1e-5 * e, x, t, False) - U.loss(th - 1e-5 * e, x, t, False)) / 2e-5
        assert abs(fd - g[idx]) <= 1e-5 + 1e-4 * abs(fd), (idx, fd, g[idx])


def test_translation_equivariance():
    th, x, _ = _case(N=32)
    y = U.forward(th, x)
    ys = U.forward(th, np.roll(np.roll(x, 4, axis=1), 8, axis=2))
    assert np.abs(np.roll(np.roll(y, 4, axis=1), 8, axis=2) - ys).max() < 1e-12


def test_zero_weights_give_the_head_bias():
    th = np.zeros(U.param_count())
    th[-3:] = [0.5, -1.0, 2.0]
    y = U.forward(th, np.random.default_rng(0).standard_normal((4, 16, 16)))
    assert np.allclose(y[0], 0.5) and np.allclose(y[1], -1.0) and np.allclose(y[2], 2.0)


# ---------------------------------------------------------------- forward values
# The pins above check the backward pass against the forward one; these fix the
# forward pass itself against independent routes and tabulated values.

def test_conv_equals_fft_circular_cross_correlation():
    """conv(x, W, b)[o] = b[o] + sum_c IFFT(FFT(x_c) conj(FFT(K_oc))), K_oc the 3x3
    kernel placed at offsets (dy - 1, dx - 1) mod N: circular cross-correlation
    computed by a different route (numpy's FFT)."""
    rng = np.random.default_rng(11)
    N, ci, co = 8, 3, 2
    x = rng.standard_normal((ci, N, N))
    Wt = rng.standard_normal((co, ci, 3, 3))
    b = rng.standard_normal(co)
    y = U.conv(x, Wt, b)
    X = np.fft.fft2(x)
    ref = np.empty((co, N, N))
    for o in range(co):
        acc = np.zeros((N, N), dtype=complex)
        for c in range(ci):
            K = np.zeros((N, N))
            for dy in range(3):
                for dx in range(3):
                    K[(dy - 1) % N, (dx - 1) % N] = Wt[o, c, dy, dx]
            acc += X[c] * np.conj(np.fft.fft2(K))
        ref[o] = np.fft.ifft2(acc).real + b[o]
    assert np.abs(y - ref).max() < 1e-12
    # one entry by hand: the (0, 0) output reads x at rows/cols -1, 0, 1 (wrapped)
    v = b[0] + sum(Wt[0, c, dy, dx] * x[c, (dy - 1) % N, (dx - 1) % N]
                   for c in range(ci) for dy in range(3) for dx in range(3))
    assert abs(y[0, 0, 0] - v) < 1e-12


def test_gelu_tabulated_values():
    """Exact (erf) GELU: gelu(x) = x Phi(x), Phi the standard normal CDF, whose
    tabulated values are Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208,
    Phi(0.5) = 0.6914624612740131.  The tanh approximation misses gelu(1) by 1.5e-4."""
    g = U.gelu(np.array([0.0, 1.0, -1.0, 2.0, 0.5, -3.0]))
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15
    assert abs(g[2] - (0.8413447460685429 - 1.0)) < 1e-15
    assert abs(g[3] - 2 * 0.9772498680518208) < 1e-15
    assert abs(g[4] - 0.5 * 0.6914624612740131) < 1e-15
    assert abs(g[5] - (-3.0) * (1.0 - 0.9986501019683699)) < 1e-15
    # derivative: Phi(x) + x phi(x); at 1: 0.8413447460685429 + 0.24197072451914337
    assert abs(U.gelu_grad(np.array([1.0]))[0] - (0.8413447460685429 + 0.24197072451914337)) < 1e-15


def test_pool_and_upsample_by_hand():
    x = np.arange(16, dtype=np.float64).reshape(1, 4, 4)
    # 2x2 average pooling: [[0,1,4,5] -> 2.5, [2,3,6,7] -> 4.5, [8,9,12,13] -> 10.5, [10,11,14,15] -> 12.5]
    assert np.array_equal(U.pool(x)[0], np.array([[2.5, 4.5], [10.5, 12.5]]))
    u = U.up(np.array([[[1.0, 2.0], [3.0, 4.0]]]))[0]
    assert np.array_equal(u, np.array([[1, 1, 2, 2], [1, 1, 2, 2], [3, 3, 4, 4], [3, 3, 4, 4]], dtype=float))


def _centre_taps(paths):
    """Parameters that are zero except centre taps W[o, c, 1, 1] = 1 (the 1x1 head:
    W[o, c, 0, 0] = 1) for the listed (layer, out, in) triples."""
    th = np.zeros(U.param_count())
    offs = np.cumsum([0] + [co * ci * k * k + co for ci, co, k in W.UNET_SHAPES])
    for layer, o, c in paths:
        ci, co, k = W.UNET_SHAPES[layer]
        r = k // 2
        th[offs[layer] + ((o * ci + c) * k + r) * k + r] = 1.0
    return th


def _g(a):
    import math
    return np.vectorize(lambda t: 0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0))))(a)


def test_skip_connections_and_levels_along_single_channel_paths():
    """Single-channel paths through the network with unit centre taps (exact in
    bfloat16).  The first skip path reads channel 32 of the last level-1
    concatenation, the second reads channel 64 of the level-2 one: with the
    documented order [upsampled | skip] those are the skips' first channels (a
    swapped order reads a zero channel).  The expected values are composed here
    from math.erf and explicit 2 x 2 block means."""
    N = 8
    rng = np.random.default_rng(5)
    x = rng.standard_normal((4, N, N))
    # path A: x0 -> l0 -> l1 -> (skip, channel 32 of [up(a7) | a1]) -> l8 -> l9 -> head
    thA = _centre_taps([(0, 0, 0), (1, 0, 0), (8, 0, 32), (9, 0, 0), (10, 0, 0)])
    yA = U.forward(thA, x)
    expA = _g(_g(_g(_g(x[0]))))
    assert np.abs(yA[0] - expA).max() < 1e-13 and np.abs(yA[1:]).max() == 0.0
    # path B: x0 -> l0 -> l1 -> pool -> l2 -> l3 -> (skip, channel 64 of [up(a5) | a3])
    #         -> l6 -> l7 -> up -> (channel 0 of [up(a7) | a1]) -> l8 -> l9 -> head
    thB = _centre_taps([(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0), (6, 0, 64), (7, 0, 0),
                        (8, 0, 0), (9, 0, 0), (10, 0, 0)])
    yB = U.forward(thB, x)
    a1 = _g(_g(x[0]))
    p1 = np.array([[a1[2 * J:2 * J + 2, 2 * I:2 * I + 2].mean() for I in range(N // 2)] for J in range(N // 2)])
    a7 = _g(_g(_g(_g(p1))))
    upa7 = np.array([[a7[j // 2, i // 2] for i in range(N)] for j in range(N)])
    expB = _g(_g(upa7))
    assert np.abs(yB[0] - expB).max() < 1e-13 and np.abs(yB[1:]).max() == 0.0
    # path C: the deepest level, x0 -> l0 l1 pool l2 l3 pool l4 l5 -> up -> channel 0 of
    #         [up(a5) | a3] -> l6 l7 -> up -> l8 l9 -> head
    thC = _centre_taps([(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0), (4, 0, 0), (5, 0, 0), (6, 0, 0),
                        (7, 0, 0), (8, 0, 0), (9, 0, 0), (10, 0, 0)])
    yC = U.forward(thC, x)
    a3 = _g(_g(p1))
    p2 = np.array([[a3[2 * J:2 * J + 2, 2 * I:2 * I + 2].mean() for I in range(N // 4)] for J in range(N // 4)])
    a5 = _g(_g(p2))
    upa5 = np.array([[a5[j // 2, i // 2] for i in range(N // 2)] for j in range(N // 2)])
    a7c = _g(_g(upa5))
    up7 = np.array([[a7c[j // 2, i // 2] for i in range(N)] for j in range(N)])
    expC = _g(_g(up7))
    assert np.abs(yC[0] - expC).max() < 1e-13 and np.abs(yC[1:]).max() == 0.0
