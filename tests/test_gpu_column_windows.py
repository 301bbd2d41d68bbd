"""The column-window calls of the sharded evaluation on one GPU.

mw_forward_cols / mw_gradient_cols solve one window of transmitter columns; the S columns of
all windows make the whole S, and the windows' gradient shares sum to the whole data gradient.
Checked against mw_gradient on the same context (same solver, different column blocks, so equal
to the FP64 solve tolerance) and against the oracle's direct-solve S and adjoint gradient.
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import inverse, solve, sources
from phantom import EPS_MATCHING, box_partition, kuhn_mesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FREQS = [0.95e9, 1.15e9]


def test_windows_reproduce_whole_evaluation():
    from paper_2311_05322_gb300 import mw
    m = kuhn_mesh(6, 5, 4, lo=(-0.03, -0.025, -0.02), hi=(0.03, 0.025, 0.02))
    rng = np.random.default_rng(31)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    n_src = 5
    ang = 2 * np.pi * np.arange(n_src) / n_src
    pos = np.stack([0.02 * np.cos(ang), 0.018 * np.sin(ang), np.full(n_src, 0.0025)], 1)
    direc = np.tile([0.0, 0.0, 1.0], (n_src, 1))
    sysm = asm.build_system(m.xyz, m.tets)
    edges, signs = sources.dipole_edges(m.xyz, sysm.topo.edge_vert, pos, direc)
    truth = eps.copy()
    truth[: m.n_tet // 6] += 5 - 3j
    _, S_obs, _ = solve.forward(sysm, truth, FREQS, EPS_MATCHING, edges, signs)
    _, S_emp, _ = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING, dtype=complex), FREQS, EPS_MATCHING, edges,
                                signs)
    J_o, g_o, _, _, S_o = inverse.gradient(sysm, eps, FREQS, EPS_MATCHING, edges, signs, S_obs, S_emp)

    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble(FREQS, np.stack([eps.real, eps.imag], 1), EPS_MATCHING)
    c.set_sources(pos, direc)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1), seed=7), 1, mw.MW_PREC_FP64)
    opts = mw.solve_opts(mode=mw.MW_MODE_FP64, tol=1e-12)
    J_ref, g_ref, S_ref = c.gradient(S_obs, S_emp, 0.0, opts, want_S=True)
    windows = [(0, 2), (2, 3)]
    S = np.zeros_like(S_ref)
    for j0, nl in windows:
        S[:, :, j0:j0 + nl] = c.forward_cols(j0, nl, opts)
    assert np.abs(S - S_ref).max() <= 1e-9 * np.abs(S_ref).max()
    assert np.abs(S - S_o).max() <= 1e-9 * np.abs(S_o).max()
    g = np.zeros_like(g_ref)
    Js = []
    for j0, nl in windows:
        c.forward_cols(j0, nl, opts)
        J, gp = c.gradient_cols(S, S_obs, S_emp, opts)
        Js.append(J)
        g += gp
    c.close()
    for J in Js:                                   # every window sees the cost of the whole S
        assert abs(J - J_ref) <= 1e-9 * abs(J_ref) and abs(J - J_o) <= 1e-8 * abs(J_o)
    assert np.abs(g - g_ref).max() <= 1e-8 * np.abs(g_ref).max()
    assert np.linalg.norm(g - g_o) <= 1e-6 * np.linalg.norm(g_o)


def test_gradient_cols_needs_a_window():
    from paper_2311_05322_gb300 import mw
    m = kuhn_mesh(3, 3, 2)
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble([1e9], np.tile([44.0, -20.0], (m.n_tet, 1)), EPS_MATCHING)
    c.set_sources(np.array([[0.0, 0.0, 0.01]]), np.array([[0.0, 0.0, 1.0]]))
    S = np.ones((1, 1, 1), complex)
    with pytest.raises(mw.MWError) as ei:
        c.gradient_cols(S, S, S)
    assert ei.value.status == mw.MW_ESTATE
    with pytest.raises(mw.MWError) as ei:
        c.forward_cols(0, 2)
    assert ei.value.status == mw.MW_EINVAL
    c.close()
