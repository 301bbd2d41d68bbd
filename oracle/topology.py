"""Mesh topology for lowest-order Nedelec (Whitney) elements, one unknown per edge (Sec. IV-D).

Canonical rules (a specification the CUDA library follows independently):
  * local edges of a tet, by local vertex pairs: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3);
  * a global edge is the vertex pair (lo, hi), lo < hi; its id is the rank of (lo, hi) in
    lexicographic order;
  * sign of a local edge = +1 when its local tail has the smaller global vertex id, else -1
    (the global edge points from lo to hi);
  * the matrix pattern holds every (row, col) pair of edges that share a tet, columns sorted
    ascending (structural zeros kept);
  * faces are sorted vertex triples; a face seen by one tet is a boundary face.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
# local faces of a tet, as local vertex triples; face k is opposite local vertex k (faces are
# canonicalised by sorting their global vertex ids)
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


@dataclass
class Topology:
    n_vert: int
    n_tet: int
    edge_vert: np.ndarray   # [E, 2] int64, lo < hi
    tet_edge: np.ndarray    # [T, 6] int64
    tet_sign: np.ndarray    # [T, 6] int8
    row_ptr: np.ndarray     # [E+1] int64
    col_idx: np.ndarray     # [nnz] int64
    faces: np.ndarray       # [F, 3] int64 sorted vertex triples, lexicographic order
    face_tets: np.ndarray   # [F, 2] int64 adjacent tets (second = -1 on the boundary)
    bface: np.ndarray       # [F_b] indices into faces of boundary faces (ascending)

    @property
    def n_edge(self) -> int:
        return self.edge_vert.shape[0]

    @property
    def nnz(self) -> int:
        return self.col_idx.shape[0]

    @property
    def n_face(self) -> int:
        return self.faces.shape[0]

    def face_edges(self, face_ids: np.ndarray):
        """Global edges of faces and their signs, in face-local order (q0,q1) (q0,q2) (q1,q2)
        of the sorted triple (signs are all +1 since q0 < q1 < q2)."""
        f = self.faces[face_ids]
        pairs = np.stack([f[:, [0, 1]], f[:, [0, 2]], f[:, [1, 2]]], axis=1)  # [n,3,2]
        keys = pairs[..., 0] * self.n_vert + pairs[..., 1]
        ekeys = self.edge_vert[:, 0] * self.n_vert + self.edge_vert[:, 1]
        eid = np.searchsorted(ekeys, keys)
        assert np.all(ekeys[eid] == keys)
        return eid, np.ones_like(eid, dtype=np.int8)

    def nnz_position(self, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
        """Index into col_idx of the (row, col) entries (must be in the pattern)."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        key_pat = np.repeat(np.arange(self.n_edge, dtype=np.int64), np.diff(self.row_ptr)) * self.n_edge + self.col_idx
        key = rows * self.n_edge + cols
        pos = np.searchsorted(key_pat, key)
        assert np.all(key_pat[pos] == key)
        return pos


def edge_numbering(n_vert: int, tets: np.ndarray):
    """Canonical edges (lexicographic (lo, hi)), tet -> 6 edges and their signs."""
    tets = np.asarray(tets, dtype=np.int64)
    T = tets.shape[0]
    a = tets[:, [p for p, _ in LOCAL_EDGES]]
    b = tets[:, [q for _, q in LOCAL_EDGES]]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    keys = lo * n_vert + hi
    uniq, inv = np.unique(keys.ravel(), return_inverse=True)
    edge_vert = np.stack([uniq // n_vert, uniq % n_vert], axis=1)
    tet_edge = inv.reshape(T, 6)
    tet_sign = np.where(a < b, 1, -1).astype(np.int8)
    return edge_vert, tet_edge, tet_sign


def face_list(n_vert: int, tets: np.ndarray):
    """Sorted vertex triples in lexicographic order, their adjacent tets, boundary face ids."""
    tets = np.asarray(tets, dtype=np.int64)
    fv = np.sort(tets[:, LOCAL_FACES], axis=2).reshape(-1, 3)      # [4T, 3]
    fkey = (fv[:, 0] * n_vert + fv[:, 1]) * n_vert + fv[:, 2]
    order = np.argsort(fkey, kind="stable")
    fk_sorted = fkey[order]
    ufk, start, cnt = np.unique(fk_sorted, return_index=True, return_counts=True)
    F = ufk.shape[0]
    faces = fv[order[start]]
    face_tets = np.full((F, 2), -1, dtype=np.int64)
    tet_of = order // 4
    face_tets[:, 0] = tet_of[start]
    two = cnt == 2
    face_tets[two, 1] = tet_of[start[two] + 1]
    assert cnt.max() <= 2, "non-manifold mesh"
    bface = np.nonzero(cnt == 1)[0]
    return faces, face_tets, bface


def matrix_pattern(n_edge: int, tet_edge: np.ndarray):
    """CSR pattern: all pairs of edges sharing a tet, columns ascending."""
    E = n_edge
    r = np.repeat(tet_edge, 6, axis=1).ravel()
    c = np.tile(tet_edge, (1, 6)).ravel()
    pk = np.unique(r * E + c)
    rows = pk // E
    col_idx = pk % E
    row_ptr = np.zeros(E + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=E), out=row_ptr[1:])
    return row_ptr, col_idx


def build_topology(n_vert: int, tets: np.ndarray, with_pattern: bool = True) -> Topology:
    tets = np.asarray(tets, dtype=np.int64)
    edge_vert, tet_edge, tet_sign = edge_numbering(n_vert, tets)
    if with_pattern:
        row_ptr, col_idx = matrix_pattern(edge_vert.shape[0], tet_edge)
    else:
        row_ptr, col_idx = np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int64)
    faces, face_tets, bface = face_list(n_vert, tets)
    return Topology(n_vert, tets.shape[0], edge_vert, tet_edge, tet_sign, row_ptr, col_idx, faces, face_tets, bface)
