"""Direct solution of A_f x = b and the dipole S-matrix.

The discrete solution is unique: every material has Im eps < 0, so for x != 0 the imaginary part
of x^H A_f x is positive and A_f is nonsingular.  The oracle computes it by a sparse LU (library
primitive) and the iterative GPU solver must reach it.

S-matrix in dipole form (dipole reading of Eq. s1): S_f,ij = p_i^T x_f,j, the line integral of
the field of transmitter j along the edge of receiver i (unconjugated, like E . E^TE10).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import assemble as asm
from . import sources


def factor(sysm: asm.System, values: np.ndarray):
    return spla.splu(sysm.csr(values).tocsc())


def solve_direct(sysm: asm.System, values: np.ndarray, B: np.ndarray) -> np.ndarray:
    lu = factor(sysm, values)
    return lu.solve(np.ascontiguousarray(B))


def s_matrix(X: np.ndarray, edges: np.ndarray, signs: np.ndarray) -> np.ndarray:
    """S[i, j] = p_i^T x_j for receivers i and transmitters j (columns of X)."""
    return signs[:, None] * X[edges, :]


def forward(sysm: asm.System, eps: np.ndarray, freqs, eps_bg: complex, edges, signs):
    """Fields [n_f, E, n_src] and S [n_f, n_src, n_src] for every frequency by direct solves."""
    Xs, Ss, lus = [], [], []
    for f in freqs:
        vals = asm.assemble(sysm, eps, f, eps_bg)
        lu = factor(sysm, vals)
        X = lu.solve(sources.rhs(sysm.topo.n_edge, edges, signs, f))
        Xs.append(X)
        Ss.append(s_matrix(X, edges, signs))
        lus.append(lu)
    return np.stack(Xs), np.stack(Ss), lus
