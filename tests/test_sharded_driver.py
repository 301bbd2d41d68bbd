"""The column-sharded evaluation driver (the bench's multi-GPU path) on CPU ranks.

paper_2311_05322_gb300.sharded splits one evaluation by transmitter columns: each rank solves
its window, the S columns are all-gathered, each rank solves its adjoints and the per-tet
gradient shares are all-reduced.  Here gloo ranks run that driver with the oracle's FP64 pieces
as the window solves (sparse direct solves), for 2 and 3 ranks (uneven windows of 5
transmitters) with a Tikhonov term; J, the gradient and S must equal the unsharded oracle.
"""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import assemble as asm
from oracle import constants, inverse, solve, sources
from paper_2311_05322_gb300.sharded import ColumnShardedEvaluation, column_window
from phantom import EPS_MATCHING, kuhn_mesh

FREQS = [0.9e9, 1.1e9]
N_SRC = 5
ALPHA = 3e-4


def _problem():
    m = kuhn_mesh(4, 3, 3, lo=(-0.03, -0.024, -0.018), hi=(0.03, 0.024, 0.018))
    rng = np.random.default_rng(21)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    ang = 2 * np.pi * np.arange(N_SRC) / N_SRC
    pos = np.stack([0.02 * np.cos(ang), 0.015 * np.sin(ang), np.full(N_SRC, 0.003)], 1)
    direc = np.tile([0.0, 0.0, 1.0], (N_SRC, 1))
    sysm = asm.build_system(m.xyz, m.tets)
    edges, signs = sources.dipole_edges(m.xyz, sysm.topo.edge_vert, pos, direc)
    return m, eps, sysm, edges, signs


class _OracleWindow:
    """The window solves of one rank with the oracle's pieces."""

    def __init__(self, sysm, eps, edges, signs):
        self.sysm, self.eps, self.edges, self.signs = sysm, eps, edges, signs
        self.lus = [solve.factor(sysm, asm.assemble(sysm, eps, f, EPS_MATCHING)) for f in FREQS]

    def forward_cols(self, j0, nl):
        E = self.sysm.topo.n_edge
        self.j0, self.nl = j0, nl
        self.X = [lu.solve(sources.rhs(E, self.edges, self.signs, f)[:, j0:j0 + nl]) for lu, f in zip(self.lus, FREQS)]
        return np.stack([solve.s_matrix(X, self.edges, self.signs) for X in self.X])

    def gradient_cols(self, S, S_obs, S_empty):
        E = self.sysm.topo.n_edge
        J = 0.0
        g = np.zeros((self.sysm.topo.n_tet, 2))
        for fi, f in enumerate(FREQS):
            J += inverse.data_cost(S[fi], S_obs[fi], S_empty[fi])
            C = inverse.adjoint_weights(S[fi], S_obs[fi], S_empty[fi])
            Lam = self.lus[fi].solve(inverse.adjoint_rhs(E, self.edges, self.signs, C[:, self.j0:self.j0 + self.nl]))
            G = inverse.tet_field_products(self.sysm, Lam, self.X[fi])
            k2 = constants.k0(f) ** 2
            g[:, 0] += k2 * G.real
            g[:, 1] -= k2 * G.imag
        return J, g


def _rank(rank, world, port, S_obs, S_empty, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, eps, sysm, edges, signs = _problem()
    win = _OracleWindow(sysm, eps, edges, signs)
    pairs, w = inverse.tikhonov_weights(sysm)
    drv = ColumnShardedEvaluation(dist, N_SRC, len(FREQS))
    J, g, S = drv.evaluate(win.forward_cols, win.gradient_cols, S_obs, S_empty, ALPHA,
                           lambda: inverse.tikhonov(pairs, w, np.stack([eps.real, eps.imag], 1)))
    q.put((rank, drv.j0, drv.nl, J, g, S))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_column_windows_cover_the_transmitters():
    for n in (1, 5, 32, 33):
        for world in range(1, min(n, 9) + 1):
            wins = [column_window(r, world, n) for r in range(world)]
            assert wins[0][0] == 0 and sum(nl for _, nl in wins) == n
            assert all(a[0] + a[1] == b[0] for a, b in zip(wins, wins[1:]))
            assert max(nl for _, nl in wins) - min(nl for _, nl in wins) <= 1


def _run(world):
    m, eps, sysm, edges, signs = _problem()
    truth = eps.copy()
    truth[: m.n_tet // 5] += 6 - 4j
    _, S_obs, _ = solve.forward(sysm, truth, FREQS, EPS_MATCHING, edges, signs)
    _, S_empty, _ = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING, dtype=complex), FREQS, EPS_MATCHING,
                                  edges, signs)
    J_ref, g_ref, _, _, S_ref = inverse.gradient(sysm, eps, FREQS, EPS_MATCHING, edges, signs, S_obs, S_empty)
    pairs, w = inverse.tikhonov_weights(sysm)
    R, gR = inverse.tikhonov(pairs, w, np.stack([eps.real, eps.imag], 1))
    J_ref += ALPHA * R
    g_ref = g_ref + ALPHA * gR
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, S_obs, S_empty, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(nl for _, _, nl, _, _, _ in out) == sorted(column_window(r, world, N_SRC)[1] for r in range(world))
    scale = np.abs(g_ref).max()
    for rank, j0, nl, J, g, S in out:
        assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
        assert np.abs(g - g_ref).max() <= 1e-10 * scale
        assert np.abs(S - S_ref).max() <= 1e-12 * np.abs(S_ref).max()


def test_sharded_driver_two_ranks():
    _run(2)


def test_sharded_driver_three_ranks_uneven_windows():
    _run(3)
