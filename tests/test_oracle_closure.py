"""Pins of the closure network's FP64 oracle (not GPU): convolution against
explicit loops, gradients against central finite differences, bf16 rounding
on hand-worked values, the skip connection and the column-mean centring of
the correction."""
import numpy as np
import pytest

from oracle import closure as C


def test_conv3x3_against_explicit_loops():
    """Same-size 3x3 convolution with zero padding, element by element."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 5, 2))
    W = rng.normal(size=(3, 3, 3, 2))
    b = rng.normal(size=3)
    got = C.conv3x3(x, W, b)
    for p in range(2):
        for y in range(4):
            for xx in range(5):
                for o in range(3):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            yy, xs = y + ky - 1, xx + kx - 1
                            if 0 <= yy < 4 and 0 <= xs < 5:
                                acc += np.dot(W[o, ky, kx], x[p, yy, xs])
                    assert abs(got[p, y, xx, o] - acc) < 1e-12


def test_bf16_rounding_hand_values():
    """Round to nearest, ties to even, on the 8-bit bfloat16 mantissa."""
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.0e-40])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 0.0])
    got = C.bf16(vals)
    assert np.array_equal(got[:5], want[:5])
    assert abs(got[5]) < 1e-38


def test_zero_head_gives_window_mean():
    """With the last layer zero the output is the mean of the 8 frames."""
    th = C.init_params(3)
    L = C.unpack(th)
    L[-1][0][:] = 0.0
    L[-1][1][:] = 0.0
    x = np.random.default_rng(4).normal(size=(2, 16, 16, 24))
    y, _ = C.forward(th, x)
    np.testing.assert_allclose(y, C.mean8(x), atol=1e-15)


def test_output_keeps_the_column_means_of_the_window_mean():
    """The correction is centred along y per patch column and channel:
    whatever the parameters, the mean over the 16 rows of every column of
    every output field is that of the 8-frame mean, and the head's bias (a
    uniform correction) has no effect."""
    rng = np.random.default_rng(11)
    th = C.init_params(2) + rng.normal(0, 0.05, size=C.n_params())
    x = rng.normal(size=(3, 16, 16, 24)) + np.array([0.3, -1.0, 2.0] * 8)
    y, _ = C.forward(th, x)
    m8 = C.mean8(x)
    np.testing.assert_allclose(y.mean(axis=1), m8.mean(axis=1), atol=1e-13)
    assert np.max(np.abs(y - m8)) > 1e-3                 # it does redistribute
    th2 = th.copy()
    th2[-3:] += np.array([0.5, -2.0, 7.0])               # head biases
    y2, _ = C.forward(th2, x)
    np.testing.assert_allclose(y2, y, atol=1e-13)


def test_uniform_correction_by_hand():
    """Head weights that copy one input channel: the output is the 8-frame
    mean plus that channel less its mean over the pixel's patch column
    (16 rows, same x), written out pixel by pixel."""
    rng = np.random.default_rng(12)
    th = C.init_params(1)
    L = C.unpack(th)
    for W, b in L[:3]:                                  # layers 1-3 pass frame 0 field 1 (shifted positive)
        W[:] = 0.0
        b[:] = 0.0
    L[0][0][0, 1, 1, 1] = 1.0                           # a = relu(x[..., 1])
    L[1][0][0, 1, 1, 0] = 1.0
    L[2][0][0, 1, 1, 0] = 1.0
    L[3][0][:] = 0.0
    L[3][1][:] = 0.0
    L[3][0][2, 1, 1, 0] = 1.0                           # head channel 2 = that activation
    x = rng.normal(size=(1, 16, 16, 24))
    x[..., 1] = np.abs(x[..., 1])
    y, _ = C.forward(th, x)
    for i in range(16):
        for j in range(16):
            m = sum(x[0, k, j, 1] for k in range(16)) / 16.0
            m8 = [sum(x[0, i, j, 3 * f + c] for f in range(8)) / 8.0 for c in range(3)]
            want = [m8[0], m8[1], m8[2] + x[0, i, j, 1] - m]
            assert np.max(np.abs(y[0, i, j] - want)) < 1e-13


def test_gradient_against_finite_differences():
    """dL/dtheta of backward() equals central differences of loss() on one
    patch (exact arithmetic; with bf16 emulation the loss is piecewise
    constant in the weights)."""
    rng = np.random.default_rng(7)
    th = C.init_params(5)
    th += rng.normal(0, 0.01, size=th.size)     # non-zero biases and head
    x = rng.normal(size=(1, 16, 16, 24))
    t = rng.normal(size=(1, 16, 16, 3))
    L, g = C.backward(th, x, t)
    assert abs(L - C.loss(th, x, t)) < 1e-14
    idx = rng.choice(th.size, size=16, replace=False)
    idx = np.concatenate([idx, [th.size - 1, th.size - 4, 13824 + 3]])   # biases of the head and layer 1
    for i in idx:
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (C.loss(tp, x, t) - C.loss(tm, x, t)) / (2 * h)
        # central differences carry ~eps L / h of rounding (the head bias's exact gradient is 0)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-8) + 4e-16 * max(1.0, L) / h, (i, fd, g[i])
    assert np.max(np.abs(g[-3:])) < 1e-14                # the centring removes the head bias
