"""Pins of the CPU oracle against facts fixed by the paper's equations and by mathematics.

Each test ties one oracle function to something other than itself: closed-form counts, exact
polynomial reproduction of Whitney elements, brute-force quadrature of single elements, the
manufactured plane-wave solution of Eq. (m1) and its first-order convergence, dense LAPACK
solves on tiny meshes, reciprocity, the reciprocal adjoint identity, finite differences of the
cost, and exact minimisers of quadratics.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as asm
from oracle import constants, inverse, oras, solve, sources
from oracle.elements import face_matrices, tet_matrices
from oracle.topology import LOCAL_EDGES, build_topology
from phantom import EPS_MATCHING, kuhn_mesh, sphere_box

# ---------------------------------------------------------------------------------------
# textbook quadrature rules (barycentric points, weights summing to 1)
# ---------------------------------------------------------------------------------------
_A, _B = 0.5854101966249685, 0.1381966011250105
TET_Q2 = (np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]]), np.full(4, 0.25))
_a, _b = 0.445948490915965, 0.091576213509771
TRI_Q4 = (np.array([[_a, _a, 1 - 2 * _a], [_a, 1 - 2 * _a, _a], [1 - 2 * _a, _a, _a],
                    [_b, _b, 1 - 2 * _b], [_b, 1 - 2 * _b, _b], [1 - 2 * _b, _b, _b]]),
          np.array([0.223381589678011] * 3 + [0.109951743655322] * 3))


def _closed_form_counts(nx, ny, nz):
    V = (nx + 1) * (ny + 1) * (nz + 1)
    T = 6 * nx * ny * nz
    Fb = 4 * (nx * ny + ny * nz + nx * nz)
    F = (4 * T + Fb) // 2
    E = V + F - T - 1            # Euler characteristic of a 3-ball
    nnz = E + 6 * F + 6 * T      # diagonal + two per edge pair sharing a face (3/face) or a tet (3/tet)
    return V, T, E, F, Fb, nnz


@pytest.mark.parametrize("dims", [(4, 3, 2), (12, 12, 12), (5, 2, 3)])
def test_topology_counts(dims):
    m = kuhn_mesh(*dims)
    tp = build_topology(m.n_vert, m.tets)
    V, T, E, F, Fb, nnz = _closed_form_counts(*dims)
    assert (m.n_vert, m.n_tet, tp.n_edge, tp.n_face, tp.bface.size, tp.nnz) == (V, T, E, F, Fb, nnz)
    if dims == (12, 12, 12):
        assert (tp.n_edge, tp.nnz) == (13428, 205236)
    if dims == (4, 3, 2):
        assert (tp.n_edge, tp.nnz) == (255, 3159)


def test_topology_canonical_rules():
    m = kuhn_mesh(3, 2, 2)
    tp = build_topology(m.n_vert, m.tets)
    ev = tp.edge_vert
    assert np.all(ev[:, 0] < ev[:, 1])
    keys = ev[:, 0] * m.n_vert + ev[:, 1]
    assert np.all(np.diff(keys) > 0)                          # lexicographic ids
    for t in range(m.n_tet):                                  # brute force per tet
        for l, (a, b) in enumerate(LOCAL_EDGES):
            va, vb = m.tets[t, a], m.tets[t, b]
            e = tp.tet_edge[t, l]
            assert (min(va, vb), max(va, vb)) == tuple(ev[e])
            assert tp.tet_sign[t, l] == (1 if va < vb else -1)
    for r in range(tp.n_edge):
        cols = tp.col_idx[tp.row_ptr[r]:tp.row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0)


def _whitney_at(P, bary, sign):
    """Brute-force Whitney functions and curls at barycentric points of one tet."""
    Jm = (P[1:] - P[0]).T
    G = np.linalg.inv(Jm)
    g = np.vstack([-G.sum(axis=0), G])                        # rows grad lambda_0..3
    N = np.zeros((bary.shape[0], 6, 3))
    C = np.zeros((6, 3))
    for m, (a, b) in enumerate(LOCAL_EDGES):
        N[:, m] = sign[m] * (bary[:, a:a + 1] * g[b] - bary[:, b:b + 1] * g[a])
        C[m] = sign[m] * 2.0 * np.cross(g[a], g[b])
    return N, C, abs(np.linalg.det(Jm)) / 6.0


def test_element_matrices_match_brute_force_quadrature():
    rng = np.random.default_rng(3)
    P = rng.normal(size=(4, 3))
    tets = np.array([[0, 1, 2, 3]])
    sign = np.array([1, -1, 1, -1, -1, 1], dtype=np.int8)
    K, M, vol = tet_matrices(P, tets, sign[None])
    bary, w = TET_Q2
    N, C, v = _whitney_at(P, bary, sign)
    Mq = v * np.einsum("q,qmi,qni->mn", w, N, N)
    Kq = v * C @ C.T
    np.testing.assert_allclose(M[0], Mq, rtol=1e-12, atol=1e-14 * np.abs(Mq).max())
    np.testing.assert_allclose(K[0], Kq, rtol=1e-12, atol=1e-14 * np.abs(Kq).max())
    assert abs(vol[0] - v) < 1e-15


def test_face_matrix_matches_brute_force_quadrature():
    rng = np.random.default_rng(5)
    Q = rng.normal(size=(3, 3))
    sign = np.array([1, -1, 1], dtype=np.int8)
    B, area = face_matrices(Q, np.array([[0, 1, 2]]), sign[None])
    # brute force: tangential trace of 3D Whitney functions of a tet built on the face
    P = np.vstack([Q, Q.mean(axis=0) + np.cross(Q[1] - Q[0], Q[2] - Q[0])])
    bary3, w = TRI_Q4
    bary = np.hstack([bary3, np.zeros((bary3.shape[0], 1))])
    n = np.cross(Q[1] - Q[0], Q[2] - Q[0])
    n /= np.linalg.norm(n)
    N, _, _ = _whitney_at(P, bary, np.array([sign[0], sign[1], 1, sign[2], 1, 1]))
    Nt = np.cross(N[:, [0, 1, 3]], n)                          # E x n for the face edges
    Bq = area[0] * np.einsum("q,qmi,qni->mn", w, Nt, Nt)
    np.testing.assert_allclose(B[0], Bq, rtol=1e-12, atol=1e-14 * np.abs(Bq).max())


@pytest.fixture(scope="module")
def box_system():
    m = kuhn_mesh(4, 3, 2, lo=(-0.02, -0.015, -0.01), hi=(0.02, 0.015, 0.01))
    return m, asm.build_system(m.xyz, m.tets)


def _grad_matrix(sysm):
    ev = sysm.topo.edge_vert
    E = ev.shape[0]
    return sp.csr_matrix((np.r_[-np.ones(E), np.ones(E)], (np.r_[np.arange(E), np.arange(E)], np.r_[ev[:, 0], ev[:, 1]])),
                         shape=(E, sysm.topo.n_vert))


def test_curl_of_gradient_is_zero(box_system):
    m, sysm = box_system
    K, Mm, B = asm.assemble_parts(sysm)
    phi = np.random.default_rng(0).normal(size=m.n_vert)
    u = _grad_matrix(sysm) @ phi
    assert np.linalg.norm(K @ u) <= 1e-12 * abs(K).sum() * np.abs(u).max()


def _interp(sysm, field):
    ev = sysm.topo.edge_vert
    a, b = sysm.xyz[ev[:, 0]], sysm.xyz[ev[:, 1]]
    return np.einsum("ei,ei->e", field(0.5 * (a + b)), b - a)     # exact for linear fields


def _box_gauss_integral(f, lo, hi, n=2):
    x, w = np.polynomial.legendre.leggauss(n)
    tot = 0.0
    for i, xi in enumerate(x):
        for j, yj in enumerate(x):
            for k, zk in enumerate(x):
                p = np.array([lo[d] + (hi[d] - lo[d]) * (c + 1) / 2 for d, c in enumerate((xi, yj, zk))])
                tot += w[i] * w[j] * w[k] * f(p[None])[0]
    return tot * np.prod([(hi[d] - lo[d]) / 2 for d in range(3)])


def test_whitney_reproduces_linear_fields(box_system):
    m, sysm = box_system
    K, Mm, B = asm.assemble_parts(sysm)
    vol = np.prod(np.subtract(m.hi, m.lo))
    assert abs(sysm.vol.sum() - vol) <= 1e-14 * vol
    rng = np.random.default_rng(11)
    for _ in range(3):
        a, bv = rng.normal(size=3), rng.normal(size=3) * 50
        field = lambda x: a[None] + np.cross(bv[None], x)
        u = _interp(sysm, field)
        exact_m = _box_gauss_integral(lambda x: np.sum(field(x) ** 2, axis=1), m.lo, m.hi)
        assert abs(u @ (Mm @ u) - exact_m) <= 1e-12 * exact_m
        assert abs(u @ (K @ u) - 4.0 * (bv @ bv) * vol) <= 1e-11 * 4.0 * (bv @ bv) * vol
        # boundary term for a constant field: sum over box faces of area * |n x a|^2
        uc = _interp(sysm, lambda x: np.broadcast_to(a, x.shape))
        L = np.subtract(m.hi, m.lo)
        exact_b = 2 * (L[1] * L[2] * (a[1] ** 2 + a[2] ** 2) + L[0] * L[2] * (a[0] ** 2 + a[2] ** 2)
                       + L[0] * L[1] * (a[0] ** 2 + a[1] ** 2))
        assert abs(uc @ (B @ uc) - exact_b) <= 1e-12 * exact_b


def test_elementwise_apply_equals_assembled_operator(box_system):
    m, sysm = box_system
    eps = np.full(m.n_tet, EPS_MATCHING) + np.random.default_rng(6).uniform(-3, 3, m.n_tet)
    X = np.random.default_rng(7).normal(size=(sysm.topo.n_edge, 3)) + 0j
    ref = sysm.csr(asm.assemble(sysm, eps, 1.1e9, EPS_MATCHING)) @ X
    topo = build_topology(m.n_vert, m.tets, with_pattern=False)
    Y = asm.apply_elementwise(m.xyz, m.tets, topo, eps, 1.1e9, EPS_MATCHING, X)
    assert np.linalg.norm(Y - ref) <= 1e-13 * np.linalg.norm(ref)


def test_matrix_complex_symmetric_and_matches_dense_solve(box_system):
    m, sysm = box_system
    eps = np.full(m.n_tet, EPS_MATCHING) + np.random.default_rng(2).uniform(-3, 3, m.n_tet)
    vals = asm.assemble(sysm, eps, 1.0e9, EPS_MATCHING)
    A = sysm.csr(vals)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    b = np.random.default_rng(4).normal(size=(sysm.topo.n_edge, 3)) + 0j
    x = solve.solve_direct(sysm, vals, b)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


# ---------------------------------------------------------------------------------------
# Manufactured plane wave E = x e^{-ikz}: Eq. (m1) with boundary data g on every outer face
# ---------------------------------------------------------------------------------------
def _planewave_error(n, L=0.04, f=1.0e9, eps=EPS_MATCHING):
    m = kuhn_mesh(n, n, n, lo=(-L / 2,) * 3, hi=(L / 2,) * 3)
    sysm = asm.build_system(m.xyz, m.tets)
    k = constants.k0(f) * np.sqrt(complex(eps))
    vals = asm.assemble(sysm, np.full(m.n_tet, eps, dtype=complex), f, eps)
    topo = sysm.topo
    Q = m.xyz[topo.faces[topo.bface]]
    cen = Q.mean(axis=1)
    nrm = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    nrm *= np.sign(np.einsum("fi,fi->f", nrm, cen))[:, None]          # outward (box centred at 0)
    area = 0.5 * np.linalg.norm(np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0]), axis=1)
    # surface gradients of the face barycentrics
    e = np.stack([Q[:, 2] - Q[:, 1], Q[:, 0] - Q[:, 2], Q[:, 1] - Q[:, 0]], axis=1)
    un = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0]) / (2 * area)[:, None]
    gl = np.cross(un[:, None, :], e) / (2 * area)[:, None, None]
    fe, _ = topo.face_edges(topo.bface)
    bary, w = TRI_Q4
    b = np.zeros(topo.n_edge, dtype=complex)
    for q in range(bary.shape[0]):
        x = np.einsum("p,fpi->fi", bary[q], Q)
        E = np.zeros_like(x, dtype=complex)
        E[:, 0] = np.exp(-1j * k * x[:, 2])
        curlE = np.zeros_like(E)
        curlE[:, 1] = -1j * k * E[:, 0]
        g = np.cross(curlE, nrm) + 1j * k * np.cross(nrm, np.cross(E, nrm))
        for le, (p, r) in enumerate(((0, 1), (0, 2), (1, 2))):
            Nq = bary[q, p] * gl[:, r] - bary[q, r] * gl[:, p]
            np.add.at(b, fe[:, le], w[q] * area * np.einsum("fi,fi->f", g, Nq))
    x = solve.solve_direct(sysm, vals, b[:, None])[:, 0]
    # L2 error of E_h - E with a degree-2 tet rule
    P = m.xyz[m.tets]
    err2 = 0.0
    nrm2 = 0.0
    for q in range(4):
        bq = TET_Q2[0][q]
        xq = np.einsum("p,tpi->ti", bq, P)
        Jm = P[:, 1:] - P[:, :1]
        G = np.linalg.inv(Jm)
        gr = np.concatenate([-G.sum(axis=2)[:, None, :], np.transpose(G, (0, 2, 1))], axis=1)
        Eh = np.zeros((m.n_tet, 3), dtype=complex)
        for le, (a, bb) in enumerate(LOCAL_EDGES):
            Nq = topo.tet_sign[:, le, None] * (bq[a] * gr[:, bb] - bq[bb] * gr[:, a])
            Eh += x[topo.tet_edge[:, le]][:, None] * Nq
        Ex = np.zeros_like(Eh)
        Ex[:, 0] = np.exp(-1j * k * xq[:, 2])
        err2 += 0.25 * np.sum(sysm.vol * np.sum(np.abs(Eh - Ex) ** 2, axis=1))
        nrm2 += 0.25 * np.sum(sysm.vol * np.sum(np.abs(Ex) ** 2, axis=1))
    return math.sqrt(err2 / nrm2)


@pytest.mark.slow
def test_planewave_first_order_convergence():
    errs = [_planewave_error(n) for n in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 0.15, errs
    assert rates[-1] >= 0.9, (errs, rates)


# ---------------------------------------------------------------------------------------
# Sources, S-matrix, adjoint, gradient
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_problem():
    m = kuhn_mesh(5, 5, 4, lo=(-0.03, -0.03, -0.024), hi=(0.03, 0.03, 0.024))
    sysm = asm.build_system(m.xyz, m.tets)
    n_src = 5
    ang = 2 * np.pi * np.arange(n_src) / n_src
    pos = np.stack([0.02 * np.cos(ang), 0.02 * np.sin(ang), np.full(n_src, 0.003)], 1)
    direc = np.tile([0.0, 0.0, 1.0], (n_src, 1))
    edges, signs = sources.dipole_edges(m.xyz, sysm.topo.edge_vert, pos, direc)
    rng = np.random.default_rng(9)
    eps = EPS_MATCHING + rng.uniform(-5, 5, m.n_tet) + 1j * rng.uniform(-3, 3, m.n_tet)
    return m, sysm, edges, signs, eps


def test_dipole_edge_brute_force(small_problem):
    m, sysm, edges, signs, _ = small_problem
    ev = sysm.topo.edge_vert
    ang = 2 * np.pi * np.arange(5) / 5
    pos = np.stack([0.02 * np.cos(ang), 0.02 * np.sin(ang), np.full(5, 0.003)], 1)
    for s in range(5):
        best, bd = -1, np.inf
        for e in range(ev.shape[0]):
            a, b = m.xyz[ev[e, 0]], m.xyz[ev[e, 1]]
            if a[0] != b[0] or a[1] != b[1]:
                continue
            d = np.sum((0.5 * (a + b) - pos[s]) ** 2)
            if d < bd:
                best, bd = e, d
        assert edges[s] == best
        assert signs[s] == 1   # lo -> hi is +z on a Kuhn grid


def test_reciprocity(small_problem):
    m, sysm, edges, signs, eps = small_problem
    X, S, _ = solve.forward(sysm, eps, (1.0e9, 1.2e9), EPS_MATCHING, edges, signs)
    for f in range(2):
        assert np.abs(S[f] - S[f].T).max() <= 1e-10 * np.abs(S[f]).max()


def test_adjoint_equals_reciprocal_combination(small_problem):
    m, sysm, edges, signs, eps = small_problem
    f = 1.0e9
    S_obs = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING + 2), (f,), EPS_MATCHING, edges, signs)[1]
    S_emp = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING, dtype=complex), (f,), EPS_MATCHING, edges, signs)[1]
    J, g, X, Lam, S = inverse.gradient(sysm, eps, (f,), EPS_MATCHING, edges, signs, S_obs, S_emp)
    C = inverse.adjoint_weights(S[0], S_obs[0], S_emp[0])
    lam_rec = X[0] @ C / (-1j * constants.omega(f) * constants.MU0)
    assert np.linalg.norm(Lam[0] - lam_rec) <= 1e-10 * np.linalg.norm(lam_rec)


def test_gradient_matches_central_differences(small_problem):
    m, sysm, edges, signs, eps = small_problem
    freqs = (0.9e9, 1.1e9)
    truth = eps.copy()
    truth[:20] += 6 - 4j
    S_obs = solve.forward(sysm, truth, freqs, EPS_MATCHING, edges, signs)[1]
    S_emp = solve.forward(sysm, np.full(m.n_tet, EPS_MATCHING, dtype=complex), freqs, EPS_MATCHING, edges, signs)[1]
    J, g, *_ = inverse.gradient(sysm, eps, freqs, EPS_MATCHING, edges, signs, S_obs, S_emp)

    def Jof(e):
        return inverse.data_cost(solve.forward(sysm, e, freqs, EPS_MATCHING, edges, signs)[1], S_obs, S_emp)

    rng = np.random.default_rng(1)
    dirs = [rng.normal(size=(m.n_tet, 2)) for _ in range(2)]
    for t in (0, 37):
        d = np.zeros((m.n_tet, 2))
        d[t, 0] = 1.0
        dirs.append(d)
        d = np.zeros((m.n_tet, 2))
        d[t, 1] = 1.0
        dirs.append(d)
    for d in dirs:
        h = 1e-6 * np.abs(eps).max()
        dc = d[:, 0] + 1j * d[:, 1]
        fd = (Jof(eps + h * dc) - Jof(eps - h * dc)) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-300), (fd, an)


def test_tikhonov_zero_constant_and_fd():
    m = kuhn_mesh(3, 3, 2)
    sysm = asm.build_system(m.xyz, m.tets)
    pairs, w = inverse.tikhonov_weights(sysm)
    assert pairs.shape[0] == sysm.topo.n_face - sysm.topo.bface.size
    R, g = inverse.tikhonov(pairs, w, np.tile([44.0, -20.0], (m.n_tet, 1)))
    assert R == 0.0 and np.all(g == 0)
    rng = np.random.default_rng(0)
    e2 = rng.normal(size=(m.n_tet, 2))
    R, g = inverse.tikhonov(pairs, w, e2)
    for _ in range(3):
        d = rng.normal(size=e2.shape)
        h = 1e-6
        fd = (inverse.tikhonov(pairs, w, e2 + h * d)[0] - inverse.tikhonov(pairs, w, e2 - h * d)[0]) / (2 * h)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    # two tets sharing one face: brute force
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.0]])
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    s2 = asm.build_system(xyz, tets)
    p2, w2 = inverse.tikhonov_weights(s2)
    area = 0.5 * np.linalg.norm(np.cross(xyz[2] - xyz[1], xyz[3] - xyz[1]))
    dist = np.linalg.norm(xyz[tets[0]].mean(0) - xyz[tets[1]].mean(0))
    assert p2.shape[0] == 1 and abs(w2[0] - area / dist) < 1e-15
    R2, _ = inverse.tikhonov(p2, w2, np.array([[1.0, 2.0], [4.0, -2.0]]))
    assert abs(R2 - 0.5 * area / dist * (9 + 16)) < 1e-14


# ---------------------------------------------------------------------------------------
# ORAS and GMRES
# ---------------------------------------------------------------------------------------
def test_oras_single_subdomain_is_exact_inverse(small_problem):
    m, sysm, edges, signs, eps = small_problem
    vals = asm.assemble(sysm, eps, 1e9, EPS_MATCHING)
    P = oras.ORAS(sysm, np.zeros(m.n_tet, dtype=np.int32), 1, 0, eps, 1e9, EPS_MATCHING)
    r = np.random.default_rng(0).normal(size=sysm.topo.n_edge) + 0j
    x = solve.solve_direct(sysm, vals, r[:, None])[:, 0]
    assert np.linalg.norm(P.apply(r) - x) <= 1e-11 * np.linalg.norm(x)
    A = sysm.csr(vals)
    xg, its, rel = oras.gmres(lambda v: A @ v, P.apply, r, tol=1e-12)
    assert its <= 2 and rel <= 1e-12


def test_oras_partition_of_unity_and_gmres_converges(small_problem):
    from phantom import box_partition
    m, sysm, edges, signs, eps = small_problem
    part = box_partition(m, (2, 2, 2), seed=7)
    P = oras.ORAS(sysm, part, 8, 1, eps, 1e9, EPS_MATCHING)
    cnt = np.zeros(sysm.topo.n_edge, dtype=int)
    for s in P.subs:
        cnt[s.dofs[s.owned]] += 1
    assert np.all(cnt == 1)                                 # sum_s R_s^T D_s R_s = I
    vals = asm.assemble(sysm, eps, 1e9, EPS_MATCHING)
    A = sysm.csr(vals)
    B = sources.rhs(sysm.topo.n_edge, edges, signs, 1e9)
    X = solve.solve_direct(sysm, vals, B)
    for j in range(2):
        x, its, rel = oras.gmres(lambda v: A @ v, P.apply, B[:, j], tol=1e-12, m=30)
        assert rel <= 1e-12
        assert np.linalg.norm(x - X[:, j]) <= 1e-9 * np.linalg.norm(X[:, j])


def _standalone_submesh(m, sub):
    """The overlapped tets of a subdomain as a mesh of their own, vertices renumbered in
    ascending global order (so edge orientation and lexicographic edge order are kept)."""
    verts = np.unique(m.tets[sub.tets])
    loc_tets = np.searchsorted(verts, m.tets[sub.tets])
    return verts, m.xyz[verts], loc_tets


@pytest.mark.parametrize("s", [0, 3, 6])
def test_oras_local_matrix_is_standalone_impedance_problem(small_problem, s):
    """With eps = eps_bg on every tet that carries an interface face, the ORAS local problem is
    the same boundary-value problem (Eq. m1-m2) posed on the overlapped subdomain as a mesh of
    its own, with the first-order impedance condition on its whole boundary.  The interior
    keeps a heterogeneous eps."""
    from phantom import box_partition
    m, sysm, _, _, eps0 = small_problem
    part = box_partition(m, (2, 2, 2), seed=7)
    subs, _ = oras.build_subdomains(sysm, part, 8, 1, which=[s])
    sub = subs[0]
    assert sub.iface.size > 0
    eps = eps0.copy()
    eps[sub.iface_tet] = EPS_MATCHING
    f = 1.05e9
    Bs = oras.local_matrix(sysm, sub, eps, f, EPS_MATCHING).toarray()
    verts, xyz, ltets = _standalone_submesh(m, sub)
    ss = asm.build_system(xyz, ltets)
    assert np.array_equal(verts[ss.topo.edge_vert], sysm.topo.edge_vert[sub.dofs])
    As = ss.csr(asm.assemble(ss, eps[sub.tets], f, EPS_MATCHING)).toarray()
    assert np.abs(Bs - As).max() <= 1e-14 * np.abs(As).max()
    # the interface faces carry a term of the same size as the volume terms: dropping it or
    # flipping its sign moves B_s far beyond rounding
    ref = oras.local_matrix(sysm, oras.Subdomain(sub.tets, sub.dofs, sub.owned, sub.iface[:0], sub.iface_tet[:0]),
                            eps, f, EPS_MATCHING).toarray()
    assert np.abs(ref - As).max() >= 1e-3 * np.abs(As).max()


def test_oras_local_matrix_brute_force_faces(small_problem):
    """Heterogeneous eps on the interface tets: B_s against a brute-force sum over the faces of
    the subdomain's tets.  A face whose three vertices belong to no other tet of the mesh is an
    outer face (i k0 sqrt(eps_bg)); one shared with a tet outside the subdomain is an interface
    face with i k0 sqrt(eps of the tet inside).  Face integrals by a degree-4 triangle rule of
    the tangential traces of the inside tet's own Whitney functions."""
    from phantom import box_partition
    m, sysm, _, _, eps = small_problem
    part = box_partition(m, (2, 2, 2), seed=7)
    subs, _ = oras.build_subdomains(sysm, part, 8, 1, which=[5])
    sub = subs[0]
    f = 0.95e9
    k0 = constants.k0(f)
    Bs = oras.local_matrix(sysm, sub, eps, f, EPS_MATCHING).toarray()
    n = sub.dofs.size
    ref = np.zeros((n, n), dtype=np.complex128)
    K, M, _ = tet_matrices(m.xyz, m.tets, sysm.topo.tet_sign)
    in_sub = set(int(t) for t in sub.tets)
    vsets = [frozenset(int(v) for v in tv) for tv in m.tets]
    bary3, w = TRI_Q4
    n_iface = n_outer = 0
    for t in sub.tets:
        loc = np.searchsorted(sub.dofs, sysm.topo.tet_edge[t])
        ref[np.ix_(loc, loc)] += K[t] - k0 * k0 * eps[t] * M[t]
        P = m.xyz[m.tets[t]]
        for k in range(4):
            fv = [q for q in range(4) if q != k]
            key = frozenset(int(m.tets[t, q]) for q in fv)
            others = [u for u in range(m.n_tet) if u != t and key <= vsets[u]]
            if others and others[0] in in_sub:
                continue
            z = 1j * k0 * np.sqrt(complex(EPS_MATCHING)) if not others else 1j * k0 * np.sqrt(complex(eps[t]))
            n_iface += bool(others)
            n_outer += not others
            bary = np.zeros((bary3.shape[0], 4))
            bary[:, fv] = bary3
            N, _, _ = _whitney_at(P, bary, sysm.topo.tet_sign[t])
            Q = P[fv]
            nrm = np.cross(Q[1] - Q[0], Q[2] - Q[0])
            area = 0.5 * np.linalg.norm(nrm)
            Nt = np.cross(N, nrm / (2 * area))
            ref[np.ix_(loc, loc)] += z * area * np.einsum("q,qmi,qni->mn", w, Nt, Nt)
    assert n_iface == sub.iface.size and n_iface > 0 and n_outer > 0
    assert np.abs(Bs - ref).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------------------
# L-BFGS
# ---------------------------------------------------------------------------------------
def test_lbfgs_quadratic_minimiser():
    rng = np.random.default_rng(0)
    n = 30
    Qh = rng.normal(size=(n, n))
    Q = Qh @ Qh.T / n + np.eye(n)
    c = rng.normal(size=n)
    fg = lambda x: (0.5 * x @ Q @ x - c @ x, Q @ x - c)
    x, hist, nfev = inverse.lbfgs(fg, np.zeros(n), m=8, max_it=200)
    assert np.linalg.norm(x - np.linalg.solve(Q, c)) <= 1e-8 * np.linalg.norm(np.linalg.solve(Q, c))
    assert all(b <= a for a, b in zip(hist, hist[1:]))


def _bfgs_inverse_explicit(S, Y, n):
    """Textbook BFGS inverse-Hessian update applied to the stored pairs, oldest first, from
    H0 = gamma I with gamma = s^T y / y^T y of the newest pair (Nocedal & Wright, Eq. 7.19):
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / y^T s."""
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    H = gamma * np.eye(n)
    I = np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / float(y @ s)
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("k", [1, 2, 5, 8])
def test_lbfgs_two_loop_equals_explicit_bfgs_inverse(k):
    rng = np.random.default_rng(40 + k)
    n = 12
    A = rng.normal(size=(n, n))
    Q = A @ A.T / n + 0.5 * np.eye(n)
    S = [rng.normal(size=n) for _ in range(k)]
    Y = [Q @ s + 0.05 * rng.normal(size=n) for s in S]
    assert all(float(s @ y) > 0 for s, y in zip(S, Y))
    g = rng.normal(size=n)
    H = _bfgs_inverse_explicit(S, Y, n)
    d = inverse.two_loop_direction(g, S, Y)
    assert np.linalg.norm(d + H @ g) <= 1e-12 * np.linalg.norm(H @ g)
    # secant condition of the newest pair, a property of every BFGS update order that ends on it
    Hy = -inverse.two_loop_direction(Y[-1], S, Y)
    assert np.linalg.norm(Hy - S[-1]) <= 1e-12 * np.linalg.norm(S[-1])


@pytest.mark.parametrize("n,m", [(6, 8), (20, 3)])
def test_lbfgs_iterates_follow_explicit_bfgs_directions(n, m):
    """Every accepted step of the driver is t d_k with t a power of 1/2 and d_k = -H_k g_k, H_k
    rebuilt here from the iterates' own pairs (skip rule, newest m kept); the first step is the
    steepest descent scaled to max |d| = 1.  With n <= m all pairs stay in memory."""
    rng = np.random.default_rng(n * 10 + m)
    A = rng.normal(size=(n, n))
    Q = A @ A.T / n + 0.3 * np.eye(n)
    c = rng.normal(size=n)
    fg = lambda x: (0.5 * x @ Q @ x - c @ x, Q @ x - c)
    xs = [np.zeros(n)]
    x, hist, nfev = inverse.lbfgs(fg, xs[0], m=m, max_it=12, callback=lambda it, x, f: xs.append(x.copy()))
    assert len(xs) == 13
    S, Y = [], []
    for k in range(len(xs) - 1):
        g = fg(xs[k])[1]
        if S:
            d = -_bfgs_inverse_explicit(S, Y, n) @ g
        else:
            d = -g / np.abs(g).max()
        step = xs[k + 1] - xs[k]
        t = float(step @ d) / float(d @ d)
        assert np.linalg.norm(step - t * d) <= 1e-10 * np.linalg.norm(step)
        assert abs(math.log2(t) - round(math.log2(t))) < 1e-9 and t <= 1.0 + 1e-12
        s, y = step, fg(xs[k + 1])[1] - g
        if float(s @ y) > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
    assert len(S) == min(m, len(xs) - 1)
