"""Pins of the waveguide-port oracle (Eq. m1-m2 boundary terms, Eq. s1) against closed forms,
the analytic TE10 solution of a straight guide, finite differences and exact special cases."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import assemble as asm
from oracle import constants, oras, ports
from oracle.elements import face_matrices
from phantom import box_partition, faces_on_plane, kuhn_mesh, waveguide_section

F_HZ = 1.5e9
A_W, B_W, LEN = 0.02, 0.01, 0.03


def _guide(cells, eps_fill=59.0 + 0.0j):
    m, fv, lab, ps = waveguide_section(cells, A_W, B_W, LEN, eps_fill)
    sysm = asm.build_system(m.xyz, m.tets)
    P = ports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill)
    return m, sysm, ports.classify(sysm, P, fv, lab)


def _plane_grads(Q):
    """Surface gradients of the face barycentrics from the pseudo-inverse of the edge matrix
    (independent of the cross-product form used by the oracle)."""
    J = np.stack([Q[1] - Q[0], Q[2] - Q[0]], axis=1)        # x = q0 + J xi
    Jp = np.linalg.pinv(J)                                   # rows = grad lambda_1, grad lambda_2
    return np.stack([-Jp[0] - Jp[1], Jp[0], Jp[1]]), Jp


def _random_faces(n, seed):
    rng = np.random.default_rng(seed)
    xyz = rng.normal(size=(3 * n, 3)) * 0.01
    return xyz, np.arange(3 * n).reshape(n, 3)


def test_mode_norm_closed_form():
    """int over the aperture of sin^2(pi x / a) = a b / 2, on coarse and fine port meshes."""
    for cells in [(2, 1, 2), (4, 2, 2), (7, 3, 2)]:
        _, sysm, bnd = _guide(cells)
        _, n = ports.port_vectors(sysm, bnd)
        assert np.allclose(n, A_W * B_W / 2, rtol=1e-13, atol=0)


def test_face_moments_constant_field_closed_form():
    """int_F (lambda_a grad lambda_b - lambda_b grad lambda_a) . c = |F|/3 (grad lambda_b - grad lambda_a) . c."""
    xyz, faces = _random_faces(20, 3)
    c = np.array([0.3, -1.1, 0.7])
    mom, nrm = ports.face_moments(xyz, faces, lambda x: np.broadcast_to(c, x.shape))
    for f in range(faces.shape[0]):
        Q = xyz[faces[f]]
        g, _ = _plane_grads(Q)
        area = 0.5 * np.linalg.norm(np.cross(Q[1] - Q[0], Q[2] - Q[0]))
        for m, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
            assert mom[f, m] == pytest.approx(area / 3 * (g[b] - g[a]) @ c, rel=1e-12, abs=1e-18)
        assert nrm[f] == pytest.approx(area * (c @ c), rel=1e-13)


def test_face_moments_whitney_field_is_face_mass_matrix():
    """Integrating N_m . N_k with the rule reproduces the closed-form face mass matrix B^F."""
    xyz, faces = _random_faces(12, 4)
    BF, _ = face_matrices(xyz, faces, np.ones((faces.shape[0], 3), dtype=np.int8))
    pairs = ((0, 1), (0, 2), (1, 2))
    for k, (a, b) in enumerate(pairs):
        def field(pts, a=a, b=b):
            out = np.empty(pts.shape)
            for f in range(faces.shape[0]):
                Q = xyz[faces[f]]
                g, Jp = _plane_grads(Q)
                xi = (pts[f] - Q[0]) @ Jp.T                     # [q, 2]
                lam = np.stack([1 - xi[:, 0] - xi[:, 1], xi[:, 0], xi[:, 1]], 1)
                out[f] = lam[:, a, None] * g[b] - lam[:, b, None] * g[a]
            return out
        mom, _ = ports.face_moments(xyz, faces, field)
        assert np.allclose(mom, BF[:, :, k], rtol=1e-12, atol=1e-14 * np.abs(BF).max())


def test_beta_branch():
    a = 0.02
    kc2 = (np.pi / a) ** 2
    for eps, f in [(59.0, 1.5e9), (59.0 - 3.0j, 1.5e9), (59.0, 0.8e9), (44.0 - 20.0j, 1.0e9), (1.0, 10e9)]:
        p = ports.Port(np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), a, eps)
        b = ports.beta(f, p)
        k2 = constants.k0(f) ** 2 * eps
        assert abs(b * b - (k2 - kc2)) <= 1e-12 * abs(k2)
        assert b.imag <= 0 and b.real >= 0
    above = ports.beta(1.5e9, ports.Port(np.zeros(3), np.zeros(3), np.zeros(3), a, 59.0))
    below = ports.beta(0.8e9, ports.Port(np.zeros(3), np.zeros(3), np.zeros(3), a, 59.0))
    assert above.imag == 0 and above.real > 0          # propagating, lossless
    assert below.real == 0 and below.imag < 0          # evanescent: decays along the guide


@pytest.fixture(scope="module")
def guides():
    return {c: _guide(c) for c in [(4, 2, 6), (8, 4, 12)]}


def test_straight_guide_converges_to_te10(guides):
    """Matched straight guide: the exact field is E_0(x) e^{-i beta z}, so S_10 = e^{-i beta L},
    S_00 = 1 (projection of the incident mode) and S is symmetric; second-order convergence."""
    errs = []
    for cells, (m, sysm, bnd) in guides.items():
        _, S, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 + 0j), [F_HZ], 59.0, bnd)
        S = S[0]
        b = ports.beta(F_HZ, bnd.ports[0])
        assert abs(S[0, 1] - S[1, 0]) <= 1e-12 * abs(S[1, 0])
        errs.append((abs(S[1, 0] - np.exp(-1j * b * LEN)), abs(S[0, 0] - 1.0), abs(abs(S[1, 0]) - 1.0)))
    (e10c, e00c, _), (e10f, e00f, magf) = errs
    assert e10f < 0.02 and e00f < 0.012 and magf < 0.02
    assert e10c / e10f > 3.5 and e00c / e00f > 3.5


def test_straight_guide_lossy_fill():
    eps_fill = 59.0 - 3.0j
    m, sysm, bnd = _guide((8, 4, 12), eps_fill)
    _, S, _ = ports.forward(sysm, np.full(m.n_tet, eps_fill), [F_HZ], 59.0, bnd)
    b = ports.beta(F_HZ, bnd.ports[0])
    exact = np.exp(-1j * b * LEN)
    assert abs(exact) < 0.8
    assert abs(S[0, 1, 0] - exact) < 0.02


def test_straight_guide_field_matches_edge_integrals(guides):
    """Away from the metal, the edge unknowns approach the line integrals of the exact field."""
    m, sysm, bnd = guides[(8, 4, 12)]
    X, _, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 + 0j), [F_HZ], 59.0, bnd)
    b = ports.beta(F_HZ, bnd.ports[0])
    ev = sysm.topo.edge_vert
    pa, pb = m.xyz[ev[:, 0]], m.xyz[ev[:, 1]]
    t, w = np.polynomial.legendre.leggauss(6)
    ref = np.zeros(ev.shape[0], dtype=complex)
    for ti, wi in zip(t, w):
        x = pa + 0.5 * (ti + 1) * (pb - pa)
        Ey = np.sin(np.pi * x[:, 0] / A_W) * np.exp(-1j * b * x[:, 2])
        ref += 0.5 * wi * Ey * (pb - pa)[:, 1]
    x0 = X[0][:, 0]
    assert np.all(x0[bnd.metal] == 0)
    free = ~bnd.metal
    rel = np.linalg.norm(x0[free] - ref[free]) / np.linalg.norm(ref[free])
    assert rel < 0.03


def test_classify_rejects_bad_faces():
    m, fv, lab, ps = waveguide_section((4, 2, 6), A_W, B_W, LEN)
    sysm = asm.build_system(m.xyz, m.tets)
    P = ports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill)
    inner = faces_on_plane(m, 2, LEN / 2, (0, 0), (A_W, B_W))
    with pytest.raises(ValueError):
        ports.classify(sysm, P, inner[:1], np.array([0]))           # a port face inside the mesh
    ports.classify(sysm, P, inner[:1], np.array([-1]))              # an inner metal sheet is fine
    with pytest.raises(ValueError):
        ports.classify(sysm, P, fv[:1], np.array([2]))              # no port 2
    with pytest.raises(ValueError):
        ports.classify(sysm, P, np.array([[0, 1, 2]]), np.array([-1]))  # not a face of the mesh


def _lossy_guide(seed=9):
    m, sysm, bnd = _guide((4, 2, 6), 59.0 - 1.0j)
    rng = np.random.default_rng(seed)
    eps = np.full(m.n_tet, 59.0 - 1.0j)
    mid = (m.centroids()[:, 2] > 0.01) & (m.centroids()[:, 2] < 0.02)
    eps[mid] = 50.0 + rng.uniform(-5, 5, mid.sum()) - 1j * rng.uniform(2, 8, mid.sum())
    return m, sysm, bnd, eps


def test_port_gradient_matches_central_differences():
    m, sysm, bnd, eps = _lossy_guide()
    freqs = [1.4e9, 1.6e9]
    truth = eps.copy()
    truth[::7] += 4.0 - 2.0j
    _, S_obs, _ = ports.forward(sysm, truth, freqs, 59.0, bnd)
    _, S_emp, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 - 1.0j), freqs, 59.0, bnd)
    J, g, *_ = ports.gradient(sysm, eps, freqs, 59.0, bnd, S_obs, S_emp)

    def Jof(e):
        _, S, _ = ports.forward(sysm, e, freqs, 59.0, bnd)
        return 0.5 * np.sum(np.abs(S - S_obs) ** 2 / np.abs(S_emp) ** 2)

    assert Jof(eps) == pytest.approx(J, rel=1e-13)
    mid = np.nonzero((m.centroids()[:, 2] > 0.01) & (m.centroids()[:, 2] < 0.02))[0]
    for t in mid[[0, 5, 17]]:
        for part, dz in ((0, 1.0), (1, 1.0j)):
            h = 1e-4
            ep, em = eps.copy(), eps.copy()
            ep[t] += h * dz
            em[t] -= h * dz
            fd = (Jof(ep) - Jof(em)) / (2 * h)
            assert g[t, part] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())


def _identity_form(sysm, vals, bnd):
    """The global matrix with the metal rows and columns replaced by those of the identity."""
    D = sp.diags((~bnd.metal).astype(float))
    return (D @ sysm.csr(vals) @ D + sp.diags(bnd.metal.astype(float))).tocsr()


def test_port_oras_single_subdomain_is_exact_inverse():
    m, sysm, bnd, eps = _lossy_guide()
    zf = ports.face_coefficients(F_HZ, 59.0, bnd)
    P = oras.ORAS(sysm, np.zeros(m.n_tet, dtype=np.int32), 1, 0, eps, F_HZ, 59.0, zface=zf, metal=bnd.metal)
    vals = ports.assemble_values(sysm, eps, F_HZ, 59.0, bnd)
    rng = np.random.default_rng(2)
    r = rng.normal(size=sysm.topo.n_edge) + 1j * rng.normal(size=sysm.topo.n_edge)
    z = P.apply(r)
    ref = spla.spsolve(_identity_form(sysm, vals, bnd).tocsc(), r)
    assert np.allclose(z, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert np.array_equal(z[bnd.metal], r[bnd.metal])


def test_port_oras_gmres_reaches_direct_solution():
    m, sysm, bnd, eps = _lossy_guide()
    zf = ports.face_coefficients(F_HZ, 59.0, bnd)
    part = box_partition(m, (1, 1, 3), seed=5)
    P = oras.ORAS(sysm, part, 3, 1, eps, F_HZ, 59.0, zface=zf, metal=bnd.metal)
    vals = ports.assemble_values(sysm, eps, F_HZ, 59.0, bnd)
    A = _identity_form(sysm, vals, bnd)
    W, n = ports.port_vectors(sysm, bnd)
    b = ports.rhs(F_HZ, bnd, W)[:, 0]
    x, its, rel = oras.gmres(lambda v: A @ v, P.apply, b, tol=1e-11, m=30)
    ref, _ = ports.solve_free(sysm, vals, bnd, b[:, None])
    assert rel <= 1e-11 and its < 60
    assert np.allclose(x, ref[:, 0], rtol=0, atol=1e-9 * np.abs(ref).max())


def test_open_box_without_ports_equals_dipole_assembly():
    """With no listed faces every boundary face is open: the port assembly reduces to Eq. (m2)
    with the first-order impedance condition everywhere (assemble.py)."""
    m = kuhn_mesh(3, 3, 2, lo=(-0.02, -0.02, -0.01), hi=(0.02, 0.02, 0.01))
    sysm = asm.build_system(m.xyz, m.tets)
    bnd = ports.classify(sysm, [], np.zeros((0, 3), dtype=np.int64), np.zeros(0, dtype=np.int64))
    rng = np.random.default_rng(1)
    eps = 44 + rng.uniform(-5, 5, m.n_tet) - 1j * rng.uniform(5, 20, m.n_tet)
    assert np.array_equal(ports.assemble_values(sysm, eps, 1e9, 44 - 20j, bnd), asm.assemble(sysm, eps, 1e9, 44 - 20j))


def _rotation(seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_rotated_guide_gives_the_same_s_matrix():
    """The discrete problem is invariant under a rigid rotation of mesh and port frames."""
    m, fv, lab, ps = waveguide_section((4, 2, 6), A_W, B_W, LEN, 59.0 - 1.0j)
    rng = np.random.default_rng(3)
    eps = 59.0 + rng.uniform(-3, 3, m.n_tet) - 1j * rng.uniform(0.5, 2, m.n_tet)
    sysm = asm.build_system(m.xyz, m.tets)
    P = ports.make_ports(ps.origin, ps.u, ps.v, ps.a, ps.eps_fill)
    _, S0, _ = ports.forward(sysm, eps, [F_HZ], 59.0, ports.classify(sysm, P, fv, lab))
    Q = _rotation(7)
    xyz = m.xyz @ Q.T + np.array([0.01, -0.02, 0.005])
    sysr = asm.build_system(xyz, m.tets)
    Pr = ports.make_ports(ps.origin @ Q.T + np.array([0.01, -0.02, 0.005]), ps.u @ Q.T, ps.v @ Q.T, ps.a, ps.eps_fill)
    _, S1, _ = ports.forward(sysr, eps, [F_HZ], 59.0, ports.classify(sysr, Pr, fv, lab))
    assert np.abs(S1 - S0).max() <= 1e-9 * np.abs(S0).max()


def test_mirrored_broad_side_axis_gives_the_same_s_matrix():
    """sin(pi s / a) is symmetric about the aperture's centre line: origin at the opposite corner
    with u reversed describes the same mode."""
    m, sysm, bnd = _guide((4, 2, 6), 59.0 - 1.0j)
    _, S0, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 - 1.0j), [F_HZ], 59.0, bnd)
    flipped = [ports.Port(p.origin + p.a * p.u, -p.u, p.v, p.a, p.eps_fill) for p in bnd.ports]
    b2 = ports.Boundary(flipped, bnd.fcls, bnd.metal)
    _, S1, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 - 1.0j), [F_HZ], 59.0, b2)
    assert np.abs(S1 - S0).max() <= 1e-12 * np.abs(S0).max()
    # the field direction matters: a mode along the broad side (v = u) couples to nothing TE10-like
    wrong = [ports.Port(p.origin, p.u, p.u, p.a, p.eps_fill) for p in bnd.ports]
    _, S2, _ = ports.forward(sysm, np.full(m.n_tet, 59.0 - 1.0j), [F_HZ], 59.0, ports.Boundary(wrong, bnd.fcls, bnd.metal))
    assert np.abs(S2[0, 1, 0]) < 0.5 * np.abs(S0[0, 1, 0])
