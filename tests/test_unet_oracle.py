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
