"""GPU parity of the waveguide-port path (Eq. m1-m2 boundary terms, Eq. s1) against the oracle.

Bars as in test_gpu_parity.py: port vectors, norms and matrix values to 1e-13 relative (FP64,
different quadrature orders on each side, both exact to rounding on these faces); metal rows
and columns bit-exact identity; FP64 fields to rel-L2 1e-8 against the oracle's reduced direct
solve, mixed precision to 1e-6; gradients to 1e-6.
"""
import numpy as np
import pytest

from oracle import assemble as asm
from oracle import oras, ports, solve, sources
from phantom import (EPS_CERAMIC, EPS_MATCHING, box_partition, faces_on_plane, kuhn_mesh, port_chamber,
                     waveguide_section)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mw():
    from paper_2311_05322_gb300 import mw
    return mw


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    def __init__(self, m, eps, fv, lab, ps):
        self.m, self.eps, self.fv, self.lab, self.ps = m, eps, fv, lab, ps
        self.sysm = asm.build_system(m.xyz, m.tets)
        P = ports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill)
        self.bnd = ports.classify(self.sysm, P, fv, lab)

    def ctx(self, freqs, eps=None):
        mw = _mw()
        e = self.eps if eps is None else eps
        c = mw.Context(0)
        c.set_mesh(self.m.xyz, self.m.tets)
        c.set_ports(self.ps.origin, self.ps.u, self.ps.v, self.ps.a, self.ps.eps_fill, self.fv, self.lab)
        c.assemble(freqs, np.stack([e.real, e.imag], 1), EPS_MATCHING)
        return c


@pytest.fixture(scope="module")
def guide():
    """Lossy straight guide 4 x 2 x 6 cells, inhomogeneous middle section."""
    m, fv, lab, ps = waveguide_section((4, 2, 6), 0.02, 0.01, 0.03, 59.0 - 1.0j)
    rng = np.random.default_rng(9)
    eps = np.full(m.n_tet, 59.0 - 1.0j)
    mid = (m.centroids()[:, 2] > 0.01) & (m.centroids()[:, 2] < 0.02)
    eps[mid] = 50.0 + rng.uniform(-5, 5, mid.sum()) - 1j * rng.uniform(2, 8, mid.sum())
    return Case(m, eps, fv, lab, ps)


@pytest.fixture(scope="module")
def chamber():
    """14 x 12 x 6 box, one ceramic-filled guide per side wall (interior metal sheets, metal side
    walls, open top and bottom), seeded heterogeneous matching medium."""
    m = kuhn_mesh(14, 12, 6, lo=(-0.035, -0.03, -0.015), hi=(0.035, 0.03, 0.015))
    fv, lab, ps, guide = port_chamber(m, n_per_wall=1, a_cells=4, b_cells=2, depth=2)
    rng = np.random.default_rng(17)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    eps[guide] = EPS_CERAMIC
    return Case(m, eps, fv, lab, ps)


def test_port_vectors_and_norms(guide, chamber):
    for case in (guide, chamber):
        c = case.ctx([1e9])
        W, n = c.get_port_vectors()
        Wr, nr = ports.port_vectors(case.sysm, case.bnd)
        assert np.abs(W - Wr).max() <= 1e-13 * np.abs(Wr).max()
        assert np.allclose(n, nr, rtol=1e-13, atol=0)
        assert np.all(W[case.bnd.metal] == 0)
    # closed form of the aperture integral of sin^2: a b / 2
    c = guide.ctx([1e9])
    _, n = c.get_port_vectors()
    assert np.allclose(n, 0.02 * 0.01 / 2, rtol=1e-13, atol=0)


@pytest.mark.parametrize("freq", [1.0e9, 1.6e9])
def test_port_matrix(chamber, freq):
    c = chamber.ctx([freq])
    A = c.get_matrix(0)
    ref = ports.assemble_values(chamber.sysm, chamber.eps, freq, EPS_MATCHING, chamber.bnd)
    t = chamber.sysm.topo
    rows = np.repeat(np.arange(t.n_edge), np.diff(t.row_ptr))
    cols = t.col_idx
    met = chamber.bnd.metal
    keep = ~met[rows] & ~met[cols]
    assert np.abs(A[keep] - ref[keep]).max() <= 1e-13 * np.abs(ref).max()
    ident = ~keep
    assert np.array_equal(A[ident], np.where(rows[ident] == cols[ident], 1.0 + 0j, 0j))


# FP64 inverses agree with the oracle's sparse-LU subdomain solves to rounding; BF16 to a few 1e-3.
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (2, 1e-2)])
def test_port_preconditioner_apply(chamber, prec, tol):
    part = box_partition(chamber.m, (2, 2, 1), seed=7)
    c = chamber.ctx([1e9])
    c.setup_preconditioner(4, part, 1, prec)
    zf = ports.face_coefficients(1e9, EPS_MATCHING, chamber.bnd)
    P = oras.ORAS(chamber.sysm, part, 4, 1, chamber.eps, 1e9, EPS_MATCHING, zface=zf, metal=chamber.bnd.metal)
    E = chamber.sysm.topo.n_edge
    rng = np.random.default_rng(3)
    R = rng.normal(size=(8, E)) + 1j * rng.normal(size=(8, E))
    ref = np.stack([P.apply(R[k]) for k in range(8)], 1)
    rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda()
    zd = torch.empty_like(rd)
    c.apply_preconditioner(0, rd, zd, 8)
    assert _relerr(zd.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("mode,prec", [(0, 0), (0, 3), (1, 1), (1, 2)])
def test_port_solve_matches_direct(chamber, mode, prec):
    mw = _mw()
    freqs = [1.0e9, 1.5e9]
    c = chamber.ctx(freqs)
    c.setup_preconditioner(4, box_partition(chamber.m, (2, 2, 1), seed=7), 1, prec)
    E = chamber.sysm.topo.n_edge
    P = len(chamber.ps.a)
    F = torch.empty((2 * P, E), dtype=torch.complex128, device="cuda")
    S, st = c.solve(mw.solve_opts(mode=mode, tol=1e-10), fields=F)
    X, Sref, _ = ports.forward(chamber.sysm, chamber.eps, freqs, EPS_MATCHING, chamber.bnd)
    Xg = F.cpu().numpy().reshape(2, P, E).transpose(0, 2, 1)
    bar = 1e-8 if mode == 0 else 1e-6
    assert st["n_converged"] == 2 * P and st["max_relres"] <= 1e-10
    assert np.all(Xg[:, chamber.bnd.metal, :] == 0)
    assert _relerr(Xg, X) <= bar
    assert _relerr(S, Sref) <= bar
    assert np.abs(S[0] - S[0].T).max() <= 1e-7 * np.abs(S[0]).max()


def test_port_gradient_matches_oracle(chamber):
    mw = _mw()
    freqs = [1.0e9, 1.5e9]
    m = chamber.m
    truth = chamber.eps.copy()
    inner = np.linalg.norm(m.centroids()[:, :2], axis=1) < 0.012
    truth[inner] += 8 - 5j
    empty = np.full(m.n_tet, EPS_MATCHING, dtype=complex)
    empty[chamber.eps == EPS_CERAMIC] = EPS_CERAMIC
    _, S_obs, _ = ports.forward(chamber.sysm, truth, freqs, EPS_MATCHING, chamber.bnd)
    _, S_emp, _ = ports.forward(chamber.sysm, empty, freqs, EPS_MATCHING, chamber.bnd)
    J_ref, g_ref, *_ = ports.gradient(chamber.sysm, chamber.eps, freqs, EPS_MATCHING, chamber.bnd, S_obs, S_emp)
    c = chamber.ctx(freqs)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1), seed=7), 1, mw.MW_PREC_FP64)
    J, g = c.gradient(S_obs, S_emp, alpha=0.0, opts=mw.solve_opts(tol=1e-11))
    assert abs(J - J_ref) <= 1e-8 * abs(J_ref)
    assert _relerr(g, g_ref) <= 1e-6
    # the ports receive what they transmit: adjoint fields by reciprocity, no adjoint solves
    c.set_adjoint_mode(True)
    J2, g2 = c.gradient(S_obs, S_emp, alpha=0.0, opts=mw.solve_opts(tol=1e-11))
    assert abs(J2 - J_ref) <= 1e-8 * abs(J_ref)
    assert _relerr(g2, g_ref) <= 1e-6 and _relerr(g2, g) <= 1e-8


def test_straight_guide_te10_on_gpu():
    """Independent of the oracle: a matched lossless guide carries E_0 e^{-i beta z}, so
    S_10 -> e^{-i beta L} and S_00 -> 1 (errors 0.017 / 0.009 at this mesh, second order)."""
    mw = _mw()
    m, fv, lab, ps = waveguide_section((8, 4, 12), 0.02, 0.01, 0.03, 59.0)
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.set_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill, fv, lab)
    eps = np.full(m.n_tet, 59.0 + 0j)
    c.assemble([1.5e9], np.stack([eps.real, eps.imag], 1), 59.0)
    c.setup_preconditioner(2, box_partition(m, (1, 1, 2), seed=1), 1, mw.MW_PREC_FP64)
    S, _ = c.solve(mw.solve_opts(tol=1e-11))
    beta = ports.beta(1.5e9, ports.Port(np.zeros(3), np.zeros(3), np.zeros(3), 0.02, 59.0))
    assert abs(S[0, 1, 0] - np.exp(-1j * beta * 0.03)) < 0.02
    assert abs(S[0, 0, 0] - 1.0) < 0.012


def test_dipoles_in_metal_box(chamber):
    """n_port = 0: metal faces only, dipole sources; oracle = reduced direct solve."""
    mw = _mw()
    m, case = chamber.m, chamber
    met = case.lab == -1
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.set_ports(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0, complex),
                case.fv[met], case.lab[met])
    c.assemble([1e9], np.stack([case.eps.real, case.eps.imag], 1), EPS_MATCHING)
    ang = 2 * np.pi * np.arange(3) / 3
    pos = np.stack([0.015 * np.cos(ang), 0.012 * np.sin(ang), np.full(3, 0.0025)], 1)
    direc = np.tile([0.0, 0.0, 1.0], (3, 1))
    e, s = c.set_sources(pos, direc)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1), seed=7), 1, mw.MW_PREC_FP64)
    S, _ = c.solve(mw.solve_opts(tol=1e-11))
    bnd = ports.classify(case.sysm, [], case.fv[met], case.lab[met])
    vals = ports.assemble_values(case.sysm, case.eps, 1e9, EPS_MATCHING, bnd)
    B = sources.rhs(case.sysm.topo.n_edge, e.astype(np.int64), s, 1e9)
    B[bnd.metal] = 0
    X, _ = ports.solve_free(case.sysm, vals, bnd, B)
    Sref = solve.s_matrix(X, e.astype(np.int64), s)
    assert _relerr(S[0], Sref) <= 1e-8


def test_port_errors(guide):
    mw = _mw()
    g = guide
    c = g.ctx([1e9])
    ps = g.ps
    inner = faces_on_plane(g.m, 2, 0.015, (0, 0), (0.02, 0.01))
    bad = [
        dict(face_vert=inner[:1], face_label=[0]),                          # port face inside the mesh
        dict(face_vert=np.array([[0, 1, 2]]), face_label=[-1]),            # not a face
        dict(face_vert=g.fv[:1], face_label=[5]),                           # label out of range
        dict(a=np.array([0.02, -1.0])),                                     # a <= 0
        dict(eps_fill=np.array([59.0 + 1.0j, 59.0])),                       # active filling
        dict(u=np.array([[1.0, 0, 0], [0, 1.0, 0]])),                       # u parallel to v
        dict(face_vert=np.concatenate([g.fv, g.fv[-1:]]), face_label=np.concatenate([g.lab, [-1]])),  # relabelled
    ]
    for kw in bad:
        args = dict(origin=ps.origin, u=ps.u, v=ps.v, a=ps.a, eps_fill=ps.eps_fill, face_vert=g.fv, face_label=g.lab)
        args.update(kw)
        with pytest.raises(mw.MWError) as ei:
            c.set_ports(**args)
        assert ei.value.status == mw.MW_EINVAL
    # a port listed without faces
    with pytest.raises(mw.MWError):
        c.set_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill, g.fv[g.lab != 1], g.lab[g.lab != 1])
    # setting the boundary drops the assembly: solving needs a new assemble
    c2 = g.ctx([1e9])
    c2.set_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill, g.fv, g.lab)
    with pytest.raises(mw.MWError) as ei:
        c2.solve(mw.solve_opts())
    assert ei.value.status == mw.MW_ESTATE
