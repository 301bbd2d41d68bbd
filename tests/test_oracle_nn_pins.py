"""Pins of the oracle's learned-initialiser network (FP64): the transposed convolution against
its definition written as plain loops, the adjoint (transpose) identity between forward and
backward-data, finite-difference gradients of the whole network, Adam's closed-form first step,
and BF16 rounding against exact bit patterns."""
import numpy as np
import pytest

from oracle import nn


def _convT_loops(x, w, b):
    B, Ci, D = x.shape[0], x.shape[1], x.shape[2]
    Co, K = w.shape[1], w.shape[2]
    Do = 2 * D
    y = np.zeros((B, Co, Do, Do, Do))
    for bb in range(B):
        for co in range(Co):
            y[bb, co] += b[co]
            for ci in range(Ci):
                for iz in range(D):
                    for iy in range(D):
                        for ix in range(D):
                            for kz in range(K):
                                for ky in range(K):
                                    for kx in range(K):
                                        oz, oy, ox = 2 * iz - 1 + kz, 2 * iy - 1 + ky, 2 * ix - 1 + kx
                                        if 0 <= oz < Do and 0 <= oy < Do and 0 <= ox < Do:
                                            y[bb, co, oz, oy, ox] += x[bb, ci, iz, iy, ix] * w[ci, co, kz, ky, kx]
    return y


def test_conv_transpose_matches_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 2, 2, 2))
    w = rng.normal(size=(3, 2, 4, 4, 4))
    b = rng.normal(size=2)
    np.testing.assert_allclose(nn.conv_transpose3d(x, w, b), _convT_loops(x, w, b), rtol=1e-12, atol=1e-12)


def test_conv_transpose_adjoint_identity_and_weight_gradient():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 3, 3, 3))
    w = rng.normal(size=(3, 4, 4, 4, 4))
    y = rng.normal(size=(2, 4, 6, 6, 6))
    zero = np.zeros(4)
    dx, dw, db = nn.conv_transpose3d_backward(x, w, y)
    # <convT(x), y> = <x, convT^T(y)>
    assert abs(np.sum(nn.conv_transpose3d(x, w, zero) * y) - np.sum(x * dx)) <= 1e-10 * np.abs(y).sum()
    # linear in w: <convT(x; w'), y> = <w', dw>
    w2 = rng.normal(size=w.shape)
    assert abs(np.sum(nn.conv_transpose3d(x, w2, zero) * y) - np.sum(w2 * dw)) <= 1e-10 * np.abs(y).sum()
    assert np.allclose(db, y.sum(axis=(0, 2, 3, 4)))


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    n_in = 16
    theta = rng.normal(size=nn.n_params(n_in)) * 0.05
    x = rng.normal(size=(3, n_in))
    t = rng.normal(size=(3, 2, 32, 32, 32)) * 0.1
    L, g = nn.loss_and_grad(theta, n_in, x, t)
    for k in range(3):
        d = rng.normal(size=theta.shape)
        h = 1e-7   # small enough that no ReLU pre-activation changes sign along the step
        fd = (nn.loss_and_grad(theta + h * d, n_in, x, t)[0] - nn.loss_and_grad(theta - h * d, n_in, x, t)[0]) / (2 * h)
        assert abs(fd - g @ d) <= 1e-5 * abs(fd), (fd, g @ d)


def test_adam_first_step_closed_form():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = nn.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-12)


def test_bf16_round_bit_patterns():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.140625, 1e-3])
    r = nn.bf16_round(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even mantissa (1.0); 1 + 3 2^-9 rounds up
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert r[3] == -2.5 and r[4] == 3.140625
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3


def test_grid_to_points_exact_for_linear_fields_and_at_centres():
    G = 8
    box = np.array([-1.0, -2.0, 0.0, 1.0, 2.0, 3.0])
    lo, hi = box[:3], box[3:]
    centres = [lo[d] + (np.arange(G) + 0.5) * (hi[d] - lo[d]) / G for d in range(3)]
    Z, Y, X = np.meshgrid(centres[2], centres[1], centres[0], indexing="ij")
    a = np.array([0.3, -1.2, 2.0])
    grid = np.stack([a[0] * X + a[1] * Y + a[2] * Z + 1.0, -X]).astype(np.float64)
    rng = np.random.default_rng(0)
    inner_lo = np.array([c[0] for c in centres])
    inner_hi = np.array([c[-1] for c in centres])
    pts = inner_lo + rng.uniform(size=(50, 3)) * (inner_hi - inner_lo)
    v = nn.grid_to_points(grid, box, pts)
    np.testing.assert_allclose(v[:, 0], pts @ a + 1.0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v[:, 1], -pts[:, 0], rtol=1e-12, atol=1e-12)
    cpt = np.array([[centres[0][3], centres[1][5], centres[2][1]]])
    assert abs(nn.grid_to_points(grid, box, cpt)[0, 1] - grid[1, 1, 5, 3]) < 1e-14
    assert np.all(nn.grid_to_points(grid, box, np.array([[5.0, 0.0, 1.0]])) == 0.0)
