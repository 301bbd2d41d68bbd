"""Sparse (multifrontal) subdomain solves of the ORAS preconditioner against the oracle's
exact sparse-LU subdomain solves (Sec. IV-C).

Bars: the apply against the oracle operator to the FP32 factorisation's accuracy (2e-5 on the
small case, 1e-4 on subdomains of several thousand unknowns with deep trees); solves through
GMRES-IR to the FP64 bar of the mixed path (1e-6 against the direct solve); bit-identical
repeated applies.
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import oras, ports, solve
from phantom import EPS_CERAMIC, EPS_MATCHING, box_partition, kuhn_mesh, port_chamber

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mw():
    from paper_2311_05322_gb300 import mw
    return mw


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(cells, lo, hi, seed):
    m = kuhn_mesh(*cells, lo=lo, hi=hi)
    rng = np.random.default_rng(seed)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    return m, eps, asm.build_system(m.xyz, m.tets)


def _ctx(m, eps, freqs):
    mw = _mw()
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble(freqs, np.stack([eps.real, eps.imag], 1), EPS_MATCHING)
    return c


def _apply(c, E, R, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(R, E)) + 1j * rng.normal(size=(R, E))
    rd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    zd = torch.empty_like(rd)
    c.apply_preconditioner(0, rd, zd, R)
    return X, zd.cpu().numpy()


# BF16 tiles (8-bit mantissas) of the factors and of the sweeps' inputs: a few 1e-3 per product,
# compounded over the tree's heights; a layout or plan error gives O(1) differences.
@pytest.mark.parametrize("cells,parts,overlap,R,tol,bf16", [((5, 4, 3), (2, 2, 1), 1, 3, 2e-5, False),
                                                            ((12, 10, 8), (2, 1, 1), 2, 32, 1e-4, False),
                                                            ((12, 10, 8), (2, 2, 2), 1, 40, 1e-4, False),
                                                            ((5, 4, 3), (2, 2, 1), 1, 3, 3e-2, True),
                                                            ((12, 10, 8), (2, 1, 1), 2, 32, 3e-2, True),
                                                            ((12, 10, 8), (2, 2, 2), 1, 40, 3e-2, True)])
def test_sparse_apply_matches_oracle(cells, parts, overlap, R, tol, bf16):
    mw = _mw()
    m, eps, sysm = _case(cells, (-0.06, -0.05, -0.04), (0.06, 0.05, 0.04), 11)
    part = box_partition(m, parts, seed=3)
    n_sub = int(np.prod(parts))
    c = _ctx(m, eps, [1e9])
    c.setup_preconditioner(n_sub, part, overlap, mw.MW_PREC_SPARSE_BF16 if bf16 else mw.MW_PREC_SPARSE)
    _, sizes = c.get_partition()
    P = oras.ORAS(sysm, part, n_sub, overlap, eps, 1e9, EPS_MATCHING)
    X, Z = _apply(c, sysm.topo.n_edge, R)
    ref = np.stack([P.apply(X[k]) for k in range(R)], 1)
    assert _relerr(Z, ref) <= tol, (sizes.max(), _relerr(Z, ref))
    # repeated applies are bit-identical
    _, Z2 = _apply(c, sysm.topo.n_edge, R)
    assert np.array_equal(Z, Z2)
    if bf16:
        # the tensor-core sweeps' two schedules (persistent CTAs, the default, and one CTA per
        # output tile) run the same products in the same order
        c.set_sweep_schedule(False)
        _, Z3 = _apply(c, sysm.topo.n_edge, R)
        c.set_sweep_schedule(True)
        assert np.array_equal(Z, Z3)
        assert c.lib.mw_set_sweep_schedule(c.h, 2) == mw.MW_EINVAL


def test_sparse_apply_with_ports_and_metal():
    mw = _mw()
    m = kuhn_mesh(14, 12, 6, lo=(-0.035, -0.03, -0.015), hi=(0.035, 0.03, 0.015))
    fv, lab, ps, guide = port_chamber(m, n_per_wall=1, a_cells=4, b_cells=2, depth=2)
    rng = np.random.default_rng(17)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    eps[guide] = EPS_CERAMIC
    sysm = asm.build_system(m.xyz, m.tets)
    bnd = ports.classify(sysm, ports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill), fv, lab)
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.set_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill, fv, lab)
    c.assemble([1e9], np.stack([eps.real, eps.imag], 1), EPS_MATCHING)
    part = box_partition(m, (2, 2, 1), seed=7)
    c.setup_preconditioner(4, part, 2, mw.MW_PREC_SPARSE)
    zf = ports.face_coefficients(1e9, EPS_MATCHING, bnd)
    P = oras.ORAS(sysm, part, 4, 2, eps, 1e9, EPS_MATCHING, zface=zf, metal=bnd.metal)
    X, Z = _apply(c, sysm.topo.n_edge, 8)
    ref = np.stack([P.apply(X[k]) for k in range(8)], 1)
    assert _relerr(Z, ref) <= 1e-4
    assert np.allclose(Z[bnd.metal], X.T[bnd.metal], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("ncols,bf16", [(5, False), (32, False), (5, True), (32, True)])
def test_sparse_preconditioned_solve_matches_direct(ncols, bf16):
    mw = _mw()
    m, eps, sysm = _case((12, 10, 8), (-0.06, -0.05, -0.04), (0.06, 0.05, 0.04), 5)
    freqs = [0.9e9, 1.1e9]
    c = _ctx(m, eps, freqs)
    c.setup_preconditioner(2, box_partition(m, (2, 1, 1), seed=3), 2,
                           mw.MW_PREC_SPARSE_BF16 if bf16 else mw.MW_PREC_SPARSE)
    E = sysm.topo.n_edge
    rng = np.random.default_rng(8)
    B = rng.normal(size=(ncols, E)) + 1j * rng.normal(size=(ncols, E))
    bd = torch.from_numpy(np.ascontiguousarray(np.stack([B, B]))).cuda()      # [n_freq][n_cols][E]
    x = torch.empty_like(bd)
    st = c.solve_rhs(ncols, bd, x, mw.solve_opts(mode=mw.MW_MODE_MIXED, tol=1e-10))
    assert st["n_converged"] == 2 * ncols and st["max_relres"] <= 1e-10
    for fi, f in enumerate(freqs):
        ref = solve.solve_direct(sysm, asm.assemble(sysm, eps, f, EPS_MATCHING), B.T)
        assert _relerr(x[fi].cpu().numpy().T, ref) <= 1e-6
