"""FP64 forward and backward of the learned initialiser network (the paper has no
learned part).

Network: x [n_in] (normalised Delta S, real parts then imaginary parts)
  h1 = relu(W1 x + b1)            W1 [1024][n_in]
  h2 = relu(W2 h1 + b2)           W2 [1024][1024]
  g0 = reshape(h2, [16][4][4][4])
  g1 = relu(convT(g0; C1, c1))    16 -> 16 channels, 4^3 -> 8^3
  g2 = relu(convT(g1; C2, c2))    16 -> 8,           8^3 -> 16^3
  y  = convT(g2; C3, c3)          8 -> 2,            16^3 -> 32^3   (Re, Im of Delta eps)
convT is the 3D transposed convolution with kernel 4, stride 2, padding 1:
  out[co][o] = b[co] + sum_ci sum_k in[ci][i] w[ci][co][k],   o = 2 i - 1 + k (per axis).
Loss: mean squared error over all outputs of the batch.  W1 and W2 enter the products rounded
to BF16 (the caller passes the rounded values here); accumulation is FP64 in the oracle.
"""
from __future__ import annotations

import numpy as np

K, S, P = 4, 2, 1
HIDDEN = 1024
CH = (16, 16, 8, 2)
GRID0 = 4

# flat parameter layout: name, shape
def param_shapes(n_in: int):
    return [("W1", (HIDDEN, n_in)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
            ("C1", (CH[0], CH[1], K, K, K)), ("c1", (CH[1],)), ("C2", (CH[1], CH[2], K, K, K)), ("c2", (CH[2],)),
            ("C3", (CH[2], CH[3], K, K, K)), ("c3", (CH[3],))]


def n_params(n_in: int) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(n_in))


def unpack(theta: np.ndarray, n_in: int) -> dict:
    out, o = {}, 0
    for name, shp in param_shapes(n_in):
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(params: dict, n_in: int) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in param_shapes(n_in)])


def conv_transpose3d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [B][Ci][D][D][D], w [Ci][Co][K][K][K] -> [B][Co][2D][2D][2D] (stride 2, pad 1)."""
    B, Ci, D = x.shape[0], x.shape[1], x.shape[2]
    Co = w.shape[1]
    Do = (D - 1) * S - 2 * P + K
    full = np.zeros((B, Co, (D - 1) * S + K, (D - 1) * S + K, (D - 1) * S + K))
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                contrib = np.einsum("bizyx,io->bozyx", x, w[:, :, kz, ky, kx])
                full[:, :, kz:kz + S * D:S, ky:ky + S * D:S, kx:kx + S * D:S] += contrib
    return full[:, :, P:P + Do, P:P + Do, P:P + Do] + b[None, :, None, None, None]


def conv_transpose3d_backward(x, w, dy):
    """Gradients of sum(dy * convT(x; w, b)) w.r.t. x, w, b."""
    B, Ci, D = x.shape[0], x.shape[1], x.shape[2]
    Co = w.shape[1]
    full = np.zeros((B, Co, (D - 1) * S + K, (D - 1) * S + K, (D - 1) * S + K))
    Do = dy.shape[2]
    full[:, :, P:P + Do, P:P + Do, P:P + Do] = dy
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                sl = full[:, :, kz:kz + S * D:S, ky:ky + S * D:S, kx:kx + S * D:S]
                dx += np.einsum("bozyx,io->bizyx", sl, w[:, :, kz, ky, kx])
                dw[:, :, kz, ky, kx] = np.einsum("bizyx,bozyx->io", x, sl)
    db = dy.sum(axis=(0, 2, 3, 4))
    return dx, dw, db


def relu(z):
    return np.maximum(z, 0.0)


def forward(p: dict, x: np.ndarray):
    """x [B][n_in] -> (y [B][2][32][32][32], cache)."""
    z1 = x @ p["W1"].T + p["b1"]
    h1 = relu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = relu(z2)
    g0 = h2.reshape(-1, CH[0], GRID0, GRID0, GRID0)
    a1 = conv_transpose3d(g0, p["C1"], p["c1"])
    g1 = relu(a1)
    a2 = conv_transpose3d(g1, p["C2"], p["c2"])
    g2 = relu(a2)
    y = conv_transpose3d(g2, p["C3"], p["c3"])
    return y, (x, z1, h1, z2, h2, g0, a1, g1, a2, g2)


def backward(p: dict, cache, dy: np.ndarray) -> dict:
    x, z1, h1, z2, h2, g0, a1, g1, a2, g2 = cache
    g = {}
    dg2, g["C3"], g["c3"] = conv_transpose3d_backward(g2, p["C3"], dy)
    da2 = dg2 * (a2 > 0)
    dg1, g["C2"], g["c2"] = conv_transpose3d_backward(g1, p["C2"], da2)
    da1 = dg1 * (a1 > 0)
    dg0, g["C1"], g["c1"] = conv_transpose3d_backward(g0, p["C1"], da1)
    dh2 = dg0.reshape(h2.shape)
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g


def mse(y: np.ndarray, t: np.ndarray):
    """Loss and dLoss/dy for the mean squared error over all entries."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def loss_and_grad(theta: np.ndarray, n_in: int, x: np.ndarray, t: np.ndarray):
    p = unpack(theta, n_in)
    y, cache = forward(p, x)
    L, dy = mse(y, t)
    return L, pack(backward(p, cache, dy), n_in)


def adam_step(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; step counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def grid_to_points(grid: np.ndarray, box, pts: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of a cell-centred grid [2][G][G][G] (index order z, y, x) over the
    box (lo x, y, z, hi x, y, z) at points [n][3]; the two nearest cell centres per axis (clamped
    to the grid), zero for points outside the box."""
    G = grid.shape[-1]
    lo = np.asarray(box[:3], dtype=np.float64)
    hi = np.asarray(box[3:], dtype=np.float64)
    out = np.zeros((pts.shape[0], 2))
    inside = np.all((pts >= lo) & (pts <= hi), axis=1)
    u = (pts[inside] - lo) / (hi - lo) * G - 0.5
    i0 = np.clip(np.floor(u), 0, G - 2).astype(int)
    f = np.clip(u - i0, 0.0, 1.0)
    acc = np.zeros((u.shape[0], 2))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((f[:, 2] if dz else 1 - f[:, 2]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 0] if dx else 1 - f[:, 0]))
                acc += w[:, None] * grid[:, i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx].T
    out[inside] = acc
    return out


def grid_to_tets(grid: np.ndarray, box, xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Average of the grid over each tet: mean of grid_to_points over the 35 points of the
    order-4 barycentric lattice (i v0 + j v1 + k v2 + l v3) / 4, i + j + k + l = 4.  [T][2]."""
    P = xyz[np.asarray(tets)]
    acc = np.zeros((P.shape[0], 2))
    n = 0
    for i in range(5):
        for j in range(5 - i):
            for k in range(5 - i - j):
                l = 4 - i - j - k
                pts = (i * P[:, 0] + j * P[:, 1] + k * P[:, 2] + l * P[:, 3]) / 4.0
                acc += grid_to_points(grid, box, pts)
                n += 1
    assert n == 35
    return acc / 35.0
