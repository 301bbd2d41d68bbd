"""The multi-GPU split of one inversion evaluation, checked on CPU ranks.

The transmitter columns are independent, so a multi-GPU run would shard them: each rank solves
its own forward columns, the S columns are all-gathered (every rank needs the whole S for the
cost and the adjoint weights), each rank solves the adjoints of its own columns and forms their
part of G_T = sum_j lambda_j^T M^T x_j, and one all-reduce sums the per-tet gradient.  Two gloo
ranks run exactly that with the oracle's FP64 pieces; the result must equal the unsharded
oracle gradient (Sec. IV-D's adjoint gradient), J included.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import assemble as asm
from oracle import constants, inverse, solve, sources
from phantom import EPS_MATCHING, kuhn_mesh

FREQS = [0.9e9, 1.1e9]
N_SRC = 4


def _problem():
    m = kuhn_mesh(4, 3, 3, lo=(-0.03, -0.024, -0.018), hi=(0.03, 0.024, 0.018))
    rng = np.random.default_rng(12)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    ang = 2 * np.pi * np.arange(N_SRC) / N_SRC
    pos = np.stack([0.02 * np.cos(ang), 0.015 * np.sin(ang), np.full(N_SRC, 0.003)], 1)
    direc = np.tile([0.0, 0.0, 1.0], (N_SRC, 1))
    sysm = asm.build_system(m.xyz, m.tets)
    edges, signs = sources.dipole_edges(m.xyz, sysm.topo.edge_vert, pos, direc)
    return m, eps, sysm, edges, signs


def _rank(rank, world, port, S_obs, S_empty, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, eps, sysm, edges, signs = _problem()
    E = sysm.topo.n_edge
    cols = np.arange(rank, N_SRC, world)                 # this rank's transmitters
    g = np.zeros((sysm.topo.n_tet, 2))
    J = 0.0
    for fi, f in enumerate(FREQS):
        lu = solve.factor(sysm, asm.assemble(sysm, eps, f, EPS_MATCHING))
        X = lu.solve(sources.rhs(E, edges, signs, f)[:, cols])          # own forward columns
        S_own = solve.s_matrix(X, edges, signs)                          # [n_src receivers, own]
        parts = [torch.zeros(N_SRC, len(cols), 2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(np.stack([S_own.real, S_own.imag], -1)))
        S = np.zeros((N_SRC, N_SRC), dtype=np.complex128)
        for r, p in enumerate(parts):
            S[:, np.arange(r, N_SRC, world)] = p[..., 0].numpy() + 1j * p[..., 1].numpy()
        J += inverse.data_cost(S, S_obs[fi], S_empty[fi])                # whole S on every rank
        C = inverse.adjoint_weights(S, S_obs[fi], S_empty[fi])
        Lam = lu.solve(inverse.adjoint_rhs(E, edges, signs, C[:, cols]))  # own adjoint columns
        G = inverse.tet_field_products(sysm, Lam, X)
        k2 = constants.k0(f) ** 2
        g[:, 0] += k2 * G.real
        g[:, 1] -= k2 * G.imag
    gt = torch.from_numpy(g)
    dist.all_reduce(gt, op=dist.ReduceOp.SUM)
    q.put((rank, J, gt.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_column_sharded_gradient_matches_unsharded():
    m, eps, sysm, edges, signs = _problem()
    truth = eps.copy()
    truth[: m.n_tet // 5] += 6 - 4j
    _, S_obs, _ = solve.forward(sysm, truth, FREQS, EPS_MATCHING, edges, signs)
    _, S_empty, _ = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING, dtype=complex), FREQS, EPS_MATCHING,
                                  edges, signs)
    J_ref, g_ref, *_ = inverse.gradient(sysm, eps, FREQS, EPS_MATCHING, edges, signs, S_obs, S_empty)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, S_obs, S_empty, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    scale = np.abs(g_ref).max()
    for rank, J, g in out:
        assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
        assert np.abs(g - g_ref).max() <= 1e-10 * scale
