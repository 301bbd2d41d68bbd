"""Whitney edge-element matrices for the bilinear form of Eq. (m2).

For a tet with barycentric coordinates lambda_p and local edge m = (a_m, b_m), the edge function
is N_m = s_m (lambda_a grad lambda_b - lambda_b grad lambda_a), s_m the canonical edge sign.  Then
  curl N_m = 2 s_m grad lambda_a x grad lambda_b,
  K_mn = int_T curl N_m . curl N_n,
  M_mn = int_T N_m . N_n, using int_T lambda_p lambda_q = |T| (1 + delta_pq) / 20.
On a boundary face the tangential trace of N_m is the 2D Whitney function of the face, so
  B_mn = int_F (N_m x n) . (N_n x n) uses surface gradients and int_F lambda_p lambda_q = |F|(1+delta_pq)/12.
"""
from __future__ import annotations

import numpy as np

from .topology import LOCAL_EDGES

FACE_EDGES = ((0, 1), (0, 2), (1, 2))


def tet_gradients(P: np.ndarray):
    """P: [T, 4, 3] vertex coordinates.  Returns (grad lambda [T, 4, 3], volume [T])."""
    Jm = P[:, 1:, :] - P[:, :1, :]               # rows v_i - v_0
    Ginv = np.linalg.inv(Jm)                      # columns are grad lambda_1..3
    g = np.empty((P.shape[0], 4, 3))
    g[:, 1:, :] = np.transpose(Ginv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    vol = np.abs(np.linalg.det(Jm)) / 6.0
    return g, vol


def _bracket(g, I, pairs, sign):
    """M-type matrix  s_m s_n [I_ac g_b.g_d - I_ad g_b.g_c - I_bc g_a.g_d + I_bd g_a.g_c]."""
    n = len(pairs)
    G = np.einsum("tpi,tqi->tpq", g, g)
    out = np.empty((g.shape[0], n, n))
    for m, (a, b) in enumerate(pairs):
        for k, (c, d) in enumerate(pairs):
            out[:, m, k] = (I[:, a, c] * G[:, b, d] - I[:, a, d] * G[:, b, c]
                            - I[:, b, c] * G[:, a, d] + I[:, b, d] * G[:, a, c])
    return out * sign[:, :, None] * sign[:, None, :]


def tet_matrices(xyz: np.ndarray, tets: np.ndarray, tet_sign: np.ndarray):
    """Element matrices K^T and M^T, each [T, 6, 6] float64, and volumes [T]."""
    P = xyz[np.asarray(tets)]
    g, vol = tet_gradients(P)
    s = tet_sign.astype(np.float64)
    cr = np.stack([np.cross(g[:, a], g[:, b]) for a, b in LOCAL_EDGES], axis=1)   # [T,6,3]
    K = 4.0 * vol[:, None, None] * np.einsum("tmi,tni->tmn", cr, cr) * s[:, :, None] * s[:, None, :]
    I = (vol / 20.0)[:, None, None] * (1.0 + np.eye(4))[None]
    M = _bracket(g, I, LOCAL_EDGES, s)
    return K, M, vol


def face_gradients(Q: np.ndarray):
    """Q: [F, 3, 3] face vertices.  Surface gradients of the face barycentrics and areas.

    grad lambda_i = n x e_i / (2|F|), e_i the edge opposite vertex i taken counter-clockwise
    about the unit normal n = (q1-q0) x (q2-q0) / (2|F|).
    """
    cr = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / (2.0 * area)[:, None]
    e = np.stack([Q[:, 2] - Q[:, 1], Q[:, 0] - Q[:, 2], Q[:, 1] - Q[:, 0]], axis=1)
    g = np.cross(n[:, None, :], e) / (2.0 * area)[:, None, None]
    return g, area


def face_matrices(xyz: np.ndarray, faces: np.ndarray, face_sign: np.ndarray):
    """Boundary mass matrices B^F [F, 3, 3] over the face edges (q0,q1) (q0,q2) (q1,q2)."""
    Q = xyz[np.asarray(faces)]
    g, area = face_gradients(Q)
    I = (area / 12.0)[:, None, None] * (1.0 + np.eye(3))[None]
    return _bracket(g, I, FACE_EDGES, face_sign.astype(np.float64)), area
