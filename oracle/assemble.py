"""Assembly of the edge-element system of Eq. (m2) for a volume source.

With k^2 = k0^2 eps_r (Sec. IV-B, below Eq. m1) and the first-order impedance condition with the
background wavenumber k_bg = k0 sqrt(eps_bg) on the whole outer boundary, Eq. (m2) becomes
    A_f = K - k0^2 M_eps + i k0 sqrt(eps_bg) B,
    K = sum_T K^T,  M_eps = sum_T eps_T M^T,  B = sum_{F on the outer boundary} B^F,
summed in tet-index order, then boundary-face order, into the canonical pattern of topology.py.
sqrt is the principal branch (Re > 0, Im < 0 for lossy media).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import constants
from .elements import face_matrices, tet_matrices
from .topology import Topology, build_topology


@dataclass
class System:
    topo: Topology
    xyz: np.ndarray
    tets: np.ndarray
    K: np.ndarray       # [T,6,6] element curl-curl matrices
    M: np.ndarray       # [T,6,6] element mass matrices
    vol: np.ndarray     # [T]
    pos_tet: np.ndarray  # [T,36] nnz position of each local (m,n) entry
    bface_edges: np.ndarray  # [F_b,3]
    BF: np.ndarray      # [F_b,3,3] boundary face matrices
    pos_face: np.ndarray  # [F_b,9]

    def csr(self, values: np.ndarray) -> sp.csr_matrix:
        E = self.topo.n_edge
        return sp.csr_matrix((values, self.topo.col_idx, self.topo.row_ptr), shape=(E, E))


def build_system(xyz: np.ndarray, tets: np.ndarray, with_pattern: bool = True) -> System:
    """Topology, element and boundary-face matrices; with_pattern=False skips the CSR pattern
    and the assembly positions (enough for element-wise operator applies and subdomains)."""
    topo = build_topology(xyz.shape[0], tets, with_pattern=with_pattern)
    K, M, vol = tet_matrices(xyz, tets, topo.tet_sign)
    te = topo.tet_edge
    fe, fs = topo.face_edges(topo.bface)
    BF, _ = face_matrices(xyz, topo.faces[topo.bface], fs)
    if with_pattern:
        rows = np.repeat(te, 6, axis=1)
        cols = np.tile(te, (1, 6))
        pos_tet = topo.nnz_position(rows.ravel(), cols.ravel()).reshape(-1, 36)
        pos_face = topo.nnz_position(np.repeat(fe, 3, axis=1).ravel(), np.tile(fe, (1, 3)).ravel()).reshape(-1, 9)
    else:
        pos_tet = pos_face = None
    return System(topo, xyz, np.asarray(tets), K, M, vol, pos_tet, fe, BF, pos_face)


def assemble(sysm: System, eps: np.ndarray, freq_hz: float, eps_bg: complex) -> np.ndarray:
    """Values of A_f in the canonical pattern (complex128 [nnz])."""
    k0 = constants.k0(freq_hz)
    vals = np.zeros(sysm.topo.nnz, dtype=np.complex128)
    elem = sysm.K.astype(np.complex128) - (k0 * k0) * eps[:, None, None] * sysm.M
    np.add.at(vals, sysm.pos_tet.ravel(), elem.reshape(-1))
    zb = 1j * k0 * np.sqrt(complex(eps_bg))
    np.add.at(vals, sysm.pos_face.ravel(), (zb * sysm.BF).reshape(-1))
    return vals


def assemble_parts(sysm: System):
    """K, the unweighted mass matrix sum_T M^T and B as separate real CSR matrices (for pins)."""
    out = []
    for elem, pos in ((sysm.K, sysm.pos_tet), (sysm.M, sysm.pos_tet), (sysm.BF, sysm.pos_face)):
        v = np.zeros(sysm.topo.nnz)
        np.add.at(v, pos.ravel(), elem.reshape(-1))
        out.append(sysm.csr(v))
    return out


def apply_system(sysm: System, eps: np.ndarray, freq_hz: float, eps_bg: complex, X: np.ndarray,
                 zface: np.ndarray | None = None) -> np.ndarray:
    """A_f X as the sum of element contributions (no assembled matrix): for each tet,
    (K^T - k0^2 eps_T M^T) acting on its 6 edge values, plus i k0 sqrt(eps_bg) B^F on each
    boundary face (or zface[F] B^F, the per-face coefficients of ports.py); scattered into the
    rows of the edges.  Same operator as assemble()."""
    k0 = constants.k0(freq_hz)
    te = sysm.topo.tet_edge
    Y = np.zeros(X.shape, dtype=np.complex128)
    for t0 in range(0, te.shape[0], 200000):
        sl = slice(t0, t0 + 200000)
        elem = sysm.K[sl].astype(np.complex128) - (k0 * k0) * eps[sl, None, None] * sysm.M[sl]
        yt = np.einsum("tmn,tnr->tmr", elem, X[te[sl]])
        np.add.at(Y, te[sl].ravel(), yt.reshape(-1, X.shape[1]))
    fe = sysm.bface_edges
    zb = 1j * k0 * np.sqrt(complex(eps_bg)) if zface is None else zface[:, None, None]
    yf = np.einsum("fmn,fnr->fmr", zb * sysm.BF, X[fe])
    np.add.at(Y, fe.ravel(), yf.reshape(-1, X.shape[1]))
    return Y


def apply_elementwise(xyz, tets, topo: Topology, eps: np.ndarray, freq_hz: float, eps_bg: complex,
                      X: np.ndarray) -> np.ndarray:
    """apply_system for a mesh given by its topology (element matrices computed here)."""
    K, M, vol = tet_matrices(xyz, tets, topo.tet_sign)
    fe, fs = topo.face_edges(topo.bface)
    BF, _ = face_matrices(xyz, topo.faces[topo.bface], fs)
    sysm = System(topo, xyz, np.asarray(tets), K, M, vol, None, fe, BF, None)
    return apply_system(sysm, eps, freq_hz, eps_bg, X)
