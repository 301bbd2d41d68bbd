"""Cost functional, adjoint gradient, Tikhonov term and L-BFGS (Sec. IV-D, Eq. sahar:2).

Unknown: the per-tet relative permittivity eps_T (complex, piecewise constant), optimised as the
real vector [Re eps; Im eps].  Since kappa = k^2 = k0^2 eps_r, optimising eps differs from
optimising kappa only by the factor k0^2 per frequency.

Cost (Eq. sahar:2, summed over frequencies):
    J = 1/2 sum_f sum_ij w_f,ij |S_f,ij - S^obs_f,ij|^2 + alpha R,   w = 1 / |S^empty_f,ij|^2.
Adjoint: with dS = -p_i^T A^{-1} dA x_j, dA = -k0^2 M^T d eps_T and A^T = A,
    c_f,ij = w_f,ij conj(Delta S_f,ij),   A_f lambda_f,j = sum_i c_f,ij p_i,
    G_T,f = sum_j lambda_f,j^T M^T x_f,j,
    dJ/dRe eps_T = sum_f k0_f^2 Re G_T,f,   dJ/dIm eps_T = -sum_f k0_f^2 Im G_T,f.
Regularisation (the P0 reading of R = 1/2 int |grad kappa|^2): the face-jump form
    R = 1/2 sum_{interior F = T|T'} |F| / |c_T - c_T'| |eps_T - eps_T'|^2   (Re and Im parts).
"""
from __future__ import annotations

import numpy as np

from . import assemble as asm
from . import constants, solve, sources
from .elements import face_gradients


def data_cost(S: np.ndarray, S_obs: np.ndarray, S_empty: np.ndarray) -> float:
    w = 1.0 / np.abs(S_empty) ** 2
    return 0.5 * float(np.sum(w * np.abs(S - S_obs) ** 2))


def adjoint_weights(S, S_obs, S_empty):
    """c_f,ij = w_f,ij conj(S_f,ij - S^obs_f,ij)."""
    return (1.0 / np.abs(S_empty) ** 2) * np.conj(S - S_obs)


def adjoint_rhs(n_edge, edges, signs, C):
    """Right-hand sides sum_i c_ij p_i for each transmitter j: [E, n_src]."""
    R = np.zeros((n_edge, C.shape[1]), dtype=np.complex128)
    np.add.at(R, edges, signs[:, None] * C)
    return R


def tet_field_products(sysm: asm.System, Lam: np.ndarray, X: np.ndarray) -> np.ndarray:
    """G_T = sum_j lambda_j^T M^T x_j for all tets."""
    te = sysm.topo.tet_edge
    return np.einsum("tmr,tmn,tnr->t", Lam[te], sysm.M, X[te])


def gradient(sysm, eps, freqs, eps_bg, edges, signs, S_obs, S_empty):
    """Data cost, data gradient [T, 2], fields, adjoint states and S (direct solves)."""
    X, S, lus = solve.forward(sysm, eps, freqs, eps_bg, edges, signs)
    J = data_cost(S, S_obs, S_empty)
    g = np.zeros((sysm.topo.n_tet, 2))
    Lams = []
    for fi, f in enumerate(freqs):
        C = adjoint_weights(S[fi], S_obs[fi], S_empty[fi])
        Lam = lus[fi].solve(adjoint_rhs(sysm.topo.n_edge, edges, signs, C))
        Lams.append(Lam)
        G = tet_field_products(sysm, Lam, X[fi])
        k2 = constants.k0(f) ** 2
        g[:, 0] += k2 * G.real
        g[:, 1] -= k2 * G.imag
    return J, g, X, np.stack(Lams), S


# ----------------------------------------------------------------------------------------
# Tikhonov
# ----------------------------------------------------------------------------------------
def tikhonov_weights(sysm: asm.System):
    """Interior faces (tet pairs) and their weights |F| / |c_T - c_T'|."""
    topo = sysm.topo
    inner = np.nonzero(topo.face_tets[:, 1] >= 0)[0]
    pairs = topo.face_tets[inner]
    _, area = face_gradients(sysm.xyz[topo.faces[inner]])
    cen = sysm.xyz[sysm.tets].mean(axis=1)
    dist = np.linalg.norm(cen[pairs[:, 0]] - cen[pairs[:, 1]], axis=1)
    return pairs, area / dist


def tikhonov(pairs, w, eps2: np.ndarray):
    """R and dR/d[Re, Im] eps ([T, 2]) for eps2 = [T, 2]."""
    d = eps2[pairs[:, 0]] - eps2[pairs[:, 1]]
    R = 0.5 * float(np.sum(w[:, None] * d * d))
    g = np.zeros_like(eps2)
    np.add.at(g, pairs[:, 0], w[:, None] * d)
    np.add.at(g, pairs[:, 1], -w[:, None] * d)
    return R, g


# ----------------------------------------------------------------------------------------
# L-BFGS with Armijo backtracking
# ----------------------------------------------------------------------------------------
def two_loop_direction(g: np.ndarray, S: list, Y: list) -> np.ndarray:
    """d = -H g, H the limited-memory BFGS inverse Hessian of the stored pairs (oldest first in
    S, Y) started from H0 = gamma I, gamma = s^T y / y^T y of the newest pair.

    Two-loop recursion: the first loop runs newest to oldest and removes each pair's component,
    q <- q - a_i y_i with a_i = rho_i s_i^T q and rho_i = 1 / y_i^T s_i; after scaling by gamma
    the second loop runs oldest to newest and adds it back, r <- r + (a_i - rho_i y_i^T r) s_i."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        q -= a * y
        alphas.append((rho, a))
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    r = gamma * q
    for (s, y), (rho, a) in zip(zip(S, Y), reversed(alphas)):
        b = rho * float(y @ r)
        r += (a - b) * s
    return -r


def lbfgs(fg, x0: np.ndarray, m: int = 8, max_it: int = 20, c1: float = 1e-4, max_ls: int = 10,
          first_step_max: float = 1.0, callback=None):
    """Minimise fg(x) -> (f, g) from x0.

    Direction by the two-loop recursion with H0 = gamma I, gamma = s^T y / y^T y of the newest
    pair; while no pair is stored, the steepest-descent direction scaled so that
    max_k |d_k| = first_step_max.  A pair is kept only if s^T y > 1e-12 |s| |y|.  Step length 1,
    halved until f(x + t d) <= f(x) + c1 t g^T d (at most max_ls trials).  A non-descent
    direction is replaced by the scaled steepest-descent one.
    Returns x, the list of f values (one per accepted iterate, starting with f(x0)), and the
    number of function evaluations.
    """
    x = np.array(x0, dtype=np.float64)
    f, g = fg(x)
    hist = [f]
    S, Y = [], []
    nfev = 1
    for it in range(max_it):
        if S:
            d = two_loop_direction(g, S, Y)
        else:
            d = -g * (first_step_max / max(np.max(np.abs(g)), 1e-300))
        gd = float(g @ d)
        if not gd < 0.0:
            d = -g * (first_step_max / max(np.max(np.abs(g)), 1e-300))
            gd = float(g @ d)
        t = 1.0
        accepted = False
        for _ in range(max_ls):
            xn = x + t * d
            fn, gn = fg(xn)
            nfev += 1
            if fn <= f + c1 * t * gd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        s = xn - x
        y = gn - g
        sy = float(s @ y)
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn
        hist.append(f)
        if callback is not None:
            callback(it, x, f)
    return x, hist, nfev
