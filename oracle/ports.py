"""Waveguide-port excitation: the boundary terms of Eq. (m1)-(m2) and the S-matrix of Eq. (s1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Boundary classes (Sec. IV-B, the system of Eq. m1):
  * Gamma_o, open: first-order impedance i k B^F with k = k0 sqrt(eps_bg) (as in assemble.py);
  * Gamma_m, metal: E x n = 0, so the trial and test space V drops every edge of a metal face;
    the unknowns are the free edges only (reduced system);
  * port p (Gamma_t while p transmits, Gamma_r while it receives): modal impedance i beta_p B^F.
The faces of class Gamma_o and port carry B^F = int_F (N_m x n).(N_n x n), the same face matrix
as the open boundary, so
    A_f = K - k0^2 M_eps + sum_{F in Gamma_o} i k0 sqrt(eps_bg) B^F + sum_p sum_{F in port p} i beta_p B^F
restricted to the free edges.

TE10 mode of a rectangular port with corner o, unit broad-side direction u (width a) and unit
narrow-side direction v:  E_p(x) = sin(pi ((x - o).u) / a) v.  Propagation constant of the
dominant mode in the filling eps_p:  beta_p^2 = k0^2 eps_p - (pi / a)^2, taken on the branch
beta = -i sqrt(pi^2/a^2 - k0^2 eps_p) (principal root), so Im beta <= 0 (no growth along the
guide for e^{i omega t}) and beta > 0 above cut-off in a lossless filling.

Source (Eq. m2 right-hand side): g = 2 i beta_p E_p on the transmitting port, so the load of
transmitter p is b_p = 2 i beta_p w_p with w_p,e = int_{port p} E_p . N_e.
S-matrix (Eq. s1): S_ij = int_{port i} E_j . E_i / int_{port i} |E_i|^2 = w_i^T x_j / n_i,
n_i = int_{port i} |E_i|^2, E_j = sum_e x_j,e N_e the field of transmitter j.
The face integrals use a collapsed (Duffy) tensor Gauss-Legendre rule with nq points per
direction; at nq = 16 the rule is exact to rounding for the mode on faces up to a full port wide.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from . import assemble as asm
from . import constants, inverse
from .elements import face_gradients

OPEN, METAL = 0, 1       # face classes; port p has class 2 + p


@dataclass
class Port:
    origin: np.ndarray       # [3] corner of the aperture
    u: np.ndarray            # [3] unit broad-side direction (the mode varies along u)
    v: np.ndarray            # [3] unit narrow-side direction (the field points along v)
    a: float                 # broad-side width
    eps_fill: complex        # relative permittivity filling the guide


@dataclass
class Boundary:
    ports: list
    fcls: np.ndarray         # [F_b] class of each boundary face (topo.bface order)
    metal: np.ndarray        # [E] bool, edges of metal faces (tangential field fixed to zero)

    @property
    def free(self) -> np.ndarray:
        return np.nonzero(~self.metal)[0]


def make_ports(origin, u, v, a, eps_fill) -> list:
    return [Port(np.asarray(origin[p], float), np.asarray(u[p], float), np.asarray(v[p], float), float(a[p]),
                 complex(eps_fill[p])) for p in range(len(a))]


def classify(sysm: asm.System, ports: list, face_vert: np.ndarray, label: np.ndarray) -> Boundary:
    """Face classes from listed faces: label -1 = metal (any mesh face), p >= 0 = port p (boundary
    faces only).  Unlisted boundary faces are open."""
    topo = sysm.topo
    nv = topo.n_vert
    fv = np.sort(np.asarray(face_vert, dtype=np.int64), axis=1)
    keys_all = (topo.faces[:, 0] * nv + topo.faces[:, 1]) * nv + topo.faces[:, 2]
    keys = (fv[:, 0] * nv + fv[:, 1]) * nv + fv[:, 2]
    fid = np.searchsorted(keys_all, keys)
    if np.any(fid >= keys_all.size) or np.any(keys_all[np.minimum(fid, keys_all.size - 1)] != keys):
        raise ValueError("listed face is not a face of the mesh")
    label = np.asarray(label, dtype=np.int64)
    if np.any(label < -1) or np.any(label >= len(ports)):
        raise ValueError("face label out of range")
    bpos = np.full(topo.n_face, -1, dtype=np.int64)
    bpos[topo.bface] = np.arange(topo.bface.size)
    fcls = np.full(topo.bface.size, OPEN, dtype=np.int64)
    port_f = label >= 0
    if np.any(bpos[fid[port_f]] < 0):
        raise ValueError("a port face is not a boundary face")
    fcls[bpos[fid[port_f]]] = 2 + label[port_f]
    met = ~port_f
    on_b = bpos[fid[met]] >= 0
    fcls[bpos[fid[met]][on_b]] = METAL
    metal = np.zeros(topo.n_edge, dtype=bool)
    if np.any(met):
        fe, _ = topo.face_edges(fid[met])
        metal[fe.ravel()] = True
    return Boundary(list(ports), fcls, metal)


def beta(freq_hz: float, port: Port) -> complex:
    """TE10 propagation constant, beta = -i sqrt((pi/a)^2 - k0^2 eps_p) (principal root)."""
    k0 = constants.k0(freq_hz)
    z = (np.pi / port.a) ** 2 - k0 * k0 * complex(port.eps_fill)
    return -1j * np.sqrt(complex(z.real, z.imag if z.imag != 0 else 0.0))


def mode(port: Port, x: np.ndarray) -> np.ndarray:
    """E_p at points x [..., 3] -> [..., 3]."""
    s = (x - port.origin) @ port.u
    return np.sin(np.pi * s / port.a)[..., None] * port.v


def face_coefficients(freq_hz: float, eps_bg: complex, bnd: Boundary) -> np.ndarray:
    """z_F of every boundary face: i k0 sqrt(eps_bg) (open), 0 (metal), i beta_p (port p)."""
    k0 = constants.k0(freq_hz)
    table = np.array([1j * k0 * np.sqrt(complex(eps_bg)), 0.0]
                     + [1j * beta(freq_hz, p) for p in bnd.ports], dtype=np.complex128)
    return table[bnd.fcls]


def assemble_values(sysm: asm.System, eps: np.ndarray, freq_hz: float, eps_bg: complex, bnd: Boundary):
    """K - k0^2 M_eps + sum_F z_F B^F over the full edge pattern (before the metal edges go)."""
    k0 = constants.k0(freq_hz)
    vals = np.zeros(sysm.topo.nnz, dtype=np.complex128)
    elem = sysm.K.astype(np.complex128) - (k0 * k0) * eps[:, None, None] * sysm.M
    np.add.at(vals, sysm.pos_tet.ravel(), elem.reshape(-1))
    z = face_coefficients(freq_hz, eps_bg, bnd)
    np.add.at(vals, sysm.pos_face.ravel(), (z[:, None, None] * sysm.BF).reshape(-1))
    return vals


def reduced_matrix(sysm: asm.System, vals: np.ndarray, bnd: Boundary):
    """A_f on the free edges (CSC)."""
    free = bnd.free
    return sysm.csr(vals)[free][:, free].tocsc()


def _gauss01(nq: int):
    t, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (t + 1.0), 0.5 * w


def face_moments(xyz: np.ndarray, faces: np.ndarray, field, nq: int = 16):
    """int_F N_e . field for the edges (q0q1, q0q2, q1q2) of each face [F, 3] (sorted triples, so
    every face edge points from its lower to its higher vertex), and int_F |field|^2 [F].

    Collapsed rule: x = q0 + xi (q1 - q0) + eta (q2 - q0), eta = (1 - xi) t, dA = 2|F| (1 - xi) dxi dt.
    """
    Q = xyz[np.asarray(faces)]
    g, area = face_gradients(Q)                      # [F,3,3] surface gradients, [F]
    r, w = _gauss01(nq)
    xi = np.repeat(r, nq)
    eta = (1.0 - xi) * np.tile(r, nq)
    wt = np.repeat(w, nq) * np.tile(w, nq) * (1.0 - xi)            # [nq^2]
    lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)               # [nq^2, 3]
    pts = np.einsum("qk,fkd->fqd", lam, Q)                          # [F, nq^2, 3]
    E = field(pts)                                                  # [F, nq^2, 3]
    mom = np.empty((Q.shape[0], 3), dtype=E.dtype)
    for m, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        N = lam[None, :, a, None] * g[:, None, b, :] - lam[None, :, b, None] * g[:, None, a, :]
        mom[:, m] = 2.0 * area * np.einsum("q,fqd,fqd->f", wt, N, E)
    nrm = 2.0 * area * np.einsum("q,fqd,fqd->f", wt, E, E)
    return mom, nrm


def port_vectors(sysm: asm.System, bnd: Boundary, nq: int = 16):
    """W [E, P] with W[:, p] = w_p (zero on metal edges) and the norms n [P]."""
    topo = sysm.topo
    P = len(bnd.ports)
    W = np.zeros((topo.n_edge, P))
    n = np.zeros(P)
    for p, port in enumerate(bnd.ports):
        sel = np.nonzero(bnd.fcls == 2 + p)[0]
        if sel.size == 0:
            raise ValueError(f"port {p} has no faces")
        faces = topo.faces[topo.bface[sel]]
        mom, nrm = face_moments(sysm.xyz, faces, lambda x: mode(port, x), nq)
        np.add.at(W[:, p], sysm.bface_edges[sel].ravel(), mom.ravel())
        n[p] = nrm.sum()
    W[bnd.metal] = 0.0
    return W, n


def rhs(freq_hz: float, bnd: Boundary, W: np.ndarray) -> np.ndarray:
    """b_p = 2 i beta_p w_p for every port (columns)."""
    return W * np.array([2j * beta(freq_hz, p) for p in bnd.ports])[None, :]


def solve_free(sysm, vals, bnd, B):
    """Solution of the reduced system, zero on the metal edges; also returns the LU."""
    free = bnd.free
    lu = spla.splu(reduced_matrix(sysm, vals, bnd))
    X = np.zeros(B.shape, dtype=np.complex128)
    X[free] = lu.solve(np.ascontiguousarray(B[free]))
    return X, lu


def s_matrix(X: np.ndarray, W: np.ndarray, n: np.ndarray) -> np.ndarray:
    """S[i, j] = w_i^T x_j / n_i (Eq. s1)."""
    return (W.T @ X) / n[:, None]


def forward(sysm, eps, freqs, eps_bg, bnd, nq: int = 16):
    """Fields [n_f, E, P], S [n_f, P, P] and the reduced LUs, every port transmitting in turn."""
    W, n = port_vectors(sysm, bnd, nq)
    Xs, Ss, lus = [], [], []
    for f in freqs:
        X, lu = solve_free(sysm, assemble_values(sysm, eps, f, eps_bg, bnd), bnd, rhs(f, bnd, W))
        Xs.append(X)
        Ss.append(s_matrix(X, W, n))
        lus.append(lu)
    return np.stack(Xs), np.stack(Ss), lus


def gradient(sysm, eps, freqs, eps_bg, bnd, S_obs, S_empty, nq: int = 16):
    """Data cost and its gradient [T, 2] for port data (the adjoint of inverse.py with the
    receiver functionals q_i = w_i / n_i in place of the dipole edges): A lambda_j = sum_i c_ij q_i.
    The load b_j does not depend on eps, and metal edges carry no unknown, so G_T keeps its form."""
    W, n = port_vectors(sysm, bnd, nq)
    Qr = W / n[None, :]
    X, S, lus = forward(sysm, eps, freqs, eps_bg, bnd, nq)
    J = inverse.data_cost(S, S_obs, S_empty)
    free = bnd.free
    g = np.zeros((sysm.topo.n_tet, 2))
    Lams = []
    for fi, f in enumerate(freqs):
        C = inverse.adjoint_weights(S[fi], S_obs[fi], S_empty[fi])
        Lam = np.zeros_like(X[fi])
        Lam[free] = lus[fi].solve(np.ascontiguousarray((Qr @ C)[free]))
        Lams.append(Lam)
        G = inverse.tet_field_products(sysm, Lam, X[fi])
        k2 = constants.k0(f) ** 2
        g[:, 0] += k2 * G.real
        g[:, 1] -= k2 * G.imag
    return J, g, X, np.stack(Lams), S
