"""Dipole excitation as an edge current (volume-source form of Eq. m1).

A z-directed dipole at x_s is a 1 A current on the z-directed edge (both endpoints share x and y)
whose midpoint is nearest x_s; ties go to the lowest edge id.  By the line-integral property of
Whitney functions (int_e' N_e . t = delta_ee'), the current density J = I t delta_e gives the
load int J . N_e' = I s delta_ee', s = +1 when the global edge (lo -> hi) points along the dipole.
With e^{i omega t}, curl curl E - k^2 E = -i omega mu0 J, so b_j = -i omega mu0 p_j, p_j = s e_edge.
"""
from __future__ import annotations

import numpy as np

from . import constants


def dipole_edges(xyz: np.ndarray, edge_vert: np.ndarray, pos: np.ndarray, direc: np.ndarray):
    a = xyz[edge_vert[:, 0]]
    b = xyz[edge_vert[:, 1]]
    d = b - a
    vert = (np.abs(d[:, 0]) <= 1e-9 * np.abs(d[:, 2])) & (np.abs(d[:, 1]) <= 1e-9 * np.abs(d[:, 2])) & (d[:, 2] != 0)
    cand = np.nonzero(vert)[0]
    mid = 0.5 * (a[cand] + b[cand])
    edges = np.empty(pos.shape[0], dtype=np.int64)
    signs = np.empty(pos.shape[0], dtype=np.int8)
    for s in range(pos.shape[0]):
        assert abs(direc[s, 0]) == 0 and abs(direc[s, 1]) == 0 and direc[s, 2] != 0, "z-directed dipoles only"
        dist2 = ((mid - pos[s]) ** 2).sum(axis=1)
        k = int(np.argmin(dist2))            # first minimum = lowest edge id
        e = cand[k]
        edges[s] = e
        signs[s] = 1 if d[e, 2] * direc[s, 2] > 0 else -1
    return edges, signs


def rhs(n_edge: int, edges: np.ndarray, signs: np.ndarray, freq_hz: float) -> np.ndarray:
    """Dense right-hand sides [E, n_src] complex128: b_j = -i omega mu0 p_j."""
    B = np.zeros((n_edge, edges.shape[0]), dtype=np.complex128)
    B[edges, np.arange(edges.shape[0])] = -1j * constants.omega(freq_hz) * constants.MU0 * signs
    return B


def p_matrix(n_edge: int, edges: np.ndarray, signs: np.ndarray) -> np.ndarray:
    P = np.zeros((n_edge, edges.shape[0]))
    P[edges, np.arange(edges.shape[0])] = signs
    return P
