"""One-level Optimized Restricted Additive Schwarz (ORAS) preconditioner and GMRES (Sec. IV-C).

Readings of the paper's (silent) details, shared with the CUDA library as specification:
  * subdomain s starts from the tets with tet_part == s; each overlap layer adds every tet that
    shares at least one vertex with the current set;
  * the subdomain unknowns are the edges of its (overlapped) tets, sorted by global id;
  * the owner of an edge is the lowest subdomain id whose non-overlapping tet set touches it, so
    the restricted partition of unity D_s is boolean and sum_s R_s^T D_s R_s = I;
  * the local matrix is the same boundary-value problem on the overlapped subdomain with the
    first-order impedance condition of Eq. (m1) on its artificial boundary:
        B_s = sum_{T in s} (K^T - k0^2 eps_T M^T) + sum_{outer faces of s} i k0 sqrt(eps_bg) B^F
              + sum_{interface faces F of s} i k0 sqrt(eps_{T_in}) B^F,
    T_in the subdomain tet that owns the interface face;
  * M^{-1} r = sum_s R_s^T D_s B_s^{-1} R_s r.
Subdomain solves use a sparse LU (library primitive).
GMRES: right preconditioning, x0 = 0, Hermitian inner product, modified Gram-Schmidt Arnoldi,
Givens rotations, restart length m; convergence is tested on the true residual at each restart.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble as asm
from . import constants
from .elements import face_matrices


@dataclass
class Subdomain:
    tets: np.ndarray        # overlapped tet list, ascending
    dofs: np.ndarray        # global edge ids, ascending
    owned: np.ndarray       # local indices (into dofs) of owned edges
    iface: np.ndarray       # interface face ids (into topo.faces)
    iface_tet: np.ndarray   # the inside tet of each interface face


def build_subdomains(sysm: asm.System, tet_part: np.ndarray, n_sub: int, overlap: int, which=None):
    """Subdomains (all, or the ids in `which`) and the owner of every edge."""
    topo = sysm.topo
    tets = sysm.tets
    # owner of an edge = lowest subdomain id among the non-overlapping tets that touch it
    owner = np.full(topo.n_edge, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(owner, topo.tet_edge.ravel(), np.repeat(np.asarray(tet_part, dtype=np.int64), 6))
    subs = []
    ids = range(n_sub) if which is None else which
    ft = topo.face_tets
    has1 = ft[:, 1] >= 0
    for s in ids:
        cur = tet_part == s
        for _ in range(overlap):
            vmask = np.zeros(topo.n_vert, dtype=bool)
            vmask[tets[cur].ravel()] = True
            cur = vmask[tets].any(axis=1)
        tl = np.nonzero(cur)[0]
        dofs = np.unique(topo.tet_edge[tl])
        owned = np.nonzero(owner[dofs] == s)[0]
        in0 = cur[ft[:, 0]]
        in1 = np.where(has1, cur[np.maximum(ft[:, 1], 0)], False)
        iface = np.nonzero(has1 & (in0 != in1))[0]
        iface_tet = np.where(in0[iface], ft[iface, 0], ft[iface, 1])
        subs.append(Subdomain(tl, dofs, owned, iface, iface_tet))
    assert np.all(owner < n_sub)
    return subs, owner


def local_matrix(sysm: asm.System, sub: Subdomain, eps: np.ndarray, freq_hz: float, eps_bg: complex,
                 zface: np.ndarray | None = None):
    """B_s as a scipy CSC matrix over sub.dofs.  zface [F_b], when given, replaces the open-boundary
    coefficient i k0 sqrt(eps_bg) on each outer face (port and metal faces, ports.py)."""
    topo = sysm.topo
    k0 = constants.k0(freq_hz)
    n = sub.dofs.size
    loc = np.searchsorted(sub.dofs, topo.tet_edge[sub.tets])           # [t,6]
    elem = sysm.K[sub.tets] - (k0 * k0) * eps[sub.tets, None, None] * sysm.M[sub.tets]
    rows = [np.repeat(loc, 6, axis=1).ravel()]
    cols = [np.tile(loc, (1, 6)).ravel()]
    vals = [elem.reshape(-1)]
    # outer boundary faces belonging to the subdomain
    in_sub = np.zeros(topo.n_tet, dtype=bool)
    in_sub[sub.tets] = True
    bsel = in_sub[topo.face_tets[topo.bface, 0]]
    if np.any(bsel):
        fl = np.searchsorted(sub.dofs, sysm.bface_edges[bsel])
        zb = 1j * k0 * np.sqrt(complex(eps_bg)) if zface is None else zface[bsel][:, None, None]
        rows.append(np.repeat(fl, 3, axis=1).ravel())
        cols.append(np.tile(fl, (1, 3)).ravel())
        vals.append((zb * sysm.BF[bsel]).reshape(-1))
    if sub.iface.size:
        fe, fs = topo.face_edges(sub.iface)
        BF, _ = face_matrices(sysm.xyz, topo.faces[sub.iface], fs)
        fl = np.searchsorted(sub.dofs, fe)
        z = 1j * k0 * np.sqrt(eps[sub.iface_tet].astype(np.complex128))
        rows.append(np.repeat(fl, 3, axis=1).ravel())
        cols.append(np.tile(fl, (1, 3)).ravel())
        vals.append((z[:, None, None] * BF).reshape(-1))
    Bm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return Bm.tocsc()


class ORAS:
    """M^{-1} = sum_s R_s^T D_s B_s^{-1} R_s with sparse-LU subdomain solves.

    With metal edges (ports.py) each B_s keeps only its free edges, and the operator is extended
    by the identity on the metal edges (z = r there), matching a global matrix whose metal rows
    and columns are those of the identity."""

    def __init__(self, sysm, tet_part, n_sub, overlap, eps, freq_hz, eps_bg, zface=None, metal=None):
        self.subs, self.owner = build_subdomains(sysm, tet_part, n_sub, overlap)
        self.free = [np.ones(s.dofs.size, dtype=bool) if metal is None else ~metal[s.dofs] for s in self.subs]
        self.lus = []
        for s, fr in zip(self.subs, self.free):
            B = local_matrix(sysm, s, eps, freq_hz, eps_bg, zface)
            self.lus.append(spla.splu(B if metal is None else B[fr][:, fr].tocsc()))
        self.n = sysm.topo.n_edge

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r, dtype=np.complex128)
        for sub, lu, fr in zip(self.subs, self.lus, self.free):
            rs = np.ascontiguousarray(r[sub.dofs], dtype=np.complex128)
            y = rs.copy()
            y[fr] = lu.solve(np.ascontiguousarray(rs[fr]))
            z[sub.dofs[sub.owned]] = y[sub.owned]
        return z

    def dense_inverse_rows(self, s: int) -> np.ndarray:
        """Owned rows of B_s^{-1} (n_own x n_s), the operator the GPU applies as a GEMM."""
        sub = self.subs[s]
        n = sub.dofs.size
        fr = self.free[s]
        Binv = np.eye(n, dtype=np.complex128)
        Binv[np.ix_(fr, fr)] = self.lus[s].solve(np.eye(int(fr.sum()), dtype=np.complex128))
        return Binv[sub.owned, :]


def gmres(matvec, precond, b: np.ndarray, tol: float = 1e-12, m: int = 50, max_it: int = 5000):
    """Right-preconditioned restarted GMRES(m) for one column.  Returns (x, iterations, relres)."""
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        r = b - matvec(x)
        rel = np.linalg.norm(r) / bn
        if rel <= tol or its >= max_it:
            return x, its, rel
        beta = np.linalg.norm(r)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(precond(V[j]))
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = bb / den if den else 0.0
            # rotation [c s; -conj(s) conj(c)] maps (a, bb) to (den, 0) with c = a/den, s = bb/den
            cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) / bn <= tol * 0.5 or its >= max_it:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + precond(V[:k].T @ y)
