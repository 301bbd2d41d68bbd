"""GPU parity of the learned-initialiser kernels against the FP64 oracle network.

Both sides use the same parameters with W1, W2 rounded to BF16 (the GPU rounds them itself);
the GPU accumulates in FP32, so outputs, loss and gradients agree to ~1e-5 relative.
"""
import numpy as np
import pytest

from oracle import nn
from phantom import kuhn_mesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_IN = 96


def _theta(seed, n_in=N_IN, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in nn.param_shapes(n_in):
        fan_in = {"W1": n_in, "W2": 1024, "C1": 16 * 8, "C2": 16 * 8, "C3": 8 * 8}.get(name, 0)
        if fan_in:
            parts.append(rng.normal(size=shp).ravel() * scale * np.sqrt(2.0 / fan_in))
        else:
            parts.append(rng.normal(size=shp).ravel() * 0.01)
    return np.concatenate(parts).astype(np.float32)


def _oracle_theta(th32, n_in=N_IN):
    th = th32.astype(np.float64)
    p = nn.unpack(th, n_in)
    p["W1"] = nn.bf16_round(p["W1"])
    p["W2"] = nn.bf16_round(p["W2"])
    return nn.pack(p, n_in)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05322_gb300 import mw
    c = mw.Context(0)
    yield c
    c.close()


def test_forward_loss_gradient(ctx):
    th = _theta(1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, N_IN)).astype(np.float32)
    t = (rng.normal(size=(3, 2, 32, 32, 32)) * 0.1).astype(np.float32)
    ctx.nn_init(N_IN, th)
    y = ctx.nn_infer(x)
    tho = _oracle_theta(th)
    yo, _ = nn.forward(nn.unpack(tho, N_IN), x.astype(np.float64))
    assert _rel(y, yo) <= 1e-5
    L, g = ctx.nn_loss_grad(x, t)
    Lo, go = nn.loss_and_grad(tho, N_IN, x.astype(np.float64), t.astype(np.float64))
    assert abs(L - Lo) <= 1e-5 * Lo
    # per block of parameters
    gp, gop = nn.unpack(g.astype(np.float64), N_IN), nn.unpack(go, N_IN)
    for name, _ in nn.param_shapes(N_IN):
        assert _rel(gp[name], gop[name]) <= 1e-4, name


def test_adam_step_matches_oracle(ctx):
    th = _theta(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(4, N_IN)).astype(np.float32)
    t = (rng.normal(size=(4, 2, 32, 32, 32)) * 0.1).astype(np.float32)
    ctx.nn_init(N_IN, th)
    _, g = ctx.nn_loss_grad(x, t)
    losses, secs = ctx.nn_train(x, t, batch=4, epochs=1, lr=1e-3, seed=9)
    th1 = ctx.nn_get_params()
    Lo, go = nn.loss_and_grad(_oracle_theta(th), N_IN, x.astype(np.float64), t.astype(np.float64))
    tho, _, _ = nn.adam_step(th.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1, lr=1e-3)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    d_gpu, d_ora = th1.astype(np.float64) - th, tho - th
    assert abs(losses[0] - Lo) <= 1e-5 * Lo
    assert _rel(d_gpu[big], d_ora[big]) <= 1e-3
    assert np.abs(d_gpu).max() <= 1.001e-3 * 1.0001          # first Adam step moves each entry by <= lr


def test_grid_to_tets(ctx):
    from phantom import EPS_MATCHING
    m = kuhn_mesh(6, 6, 5, lo=(-0.05, -0.04, -0.03), hi=(0.05, 0.04, 0.03))
    ctx.set_mesh(m.xyz, m.tets)
    rng = np.random.default_rng(5)
    grid = rng.normal(size=(2, 32, 32, 32)).astype(np.float32)
    box = np.array([-0.03, -0.02, -0.025, 0.02, 0.03, 0.02])
    got = ctx.nn_grid_to_tets(grid, box)
    ref = nn.grid_to_tets(grid.astype(np.float64), box, m.xyz, m.tets)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.count_nonzero(np.abs(ref).sum(1)) > 100


def test_forward_loss_gradient_full_size(ctx):
    """The configuration the network trains at: 8192 inputs (64 x 64 complex Delta S), batch 64.
    The long-K GEMMs (8192 x 1024 forward, dW1 = dz1^T x backward) are checked here."""
    n_in, B = 8192, 64
    th = _theta(11, n_in)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(B, n_in)).astype(np.float32)
    t = (rng.normal(size=(B, 2, 32, 32, 32)) * 0.1).astype(np.float32)
    ctx.nn_init(n_in, th)
    y = ctx.nn_infer(x)
    tho = _oracle_theta(th, n_in)
    yo, _ = nn.forward(nn.unpack(tho, n_in), x.astype(np.float64))
    assert _rel(y, yo) <= 1e-5
    L, g = ctx.nn_loss_grad(x, t)
    Lo, go = nn.loss_and_grad(tho, n_in, x.astype(np.float64), t.astype(np.float64))
    assert abs(L - Lo) <= 1e-5 * Lo
    gp, gop = nn.unpack(g.astype(np.float64), n_in), nn.unpack(go, n_in)
    for name, _ in nn.param_shapes(n_in):
        assert _rel(gp[name], gop[name]) <= 1e-4, name
