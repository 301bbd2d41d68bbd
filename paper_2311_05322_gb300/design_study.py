"""Antenna-count design study (Sec. V, Tables II-III) on the synthetic shoulder.

For N = 96, 64, 32 and 16 antennas in the layered design (two full rings and two half rings,
adjacent rings shifted by half a pitch, `phantom.antenna_layers`), data are computed on a fine
"data" mesh for the healthy shoulder and for a partial (about 1 mL) and a large (about 5 mL)
tear, and corrupted with complex Gaussian noise at 23, 15 and 10 dB (`phantom.add_noise`).
Each data set is inverted on a coarser "inverse" mesh (different meshes, Sec. IV-D) by the
library's L-BFGS, starting from the homogeneous matching medium, as in Sec. IV.  Reported per
configuration (Eq. saharerr and Eq. saharcont):
  err = ||Re eps_rec - Re eps_exact||_2 / ||Re eps_exact||_2  (and the same for Im), over every
        tet (total) and over the tets of the injury area, for the partial tear at 23 dB;
  ctr = mean over the injury area of (eps_rec(injured) - eps_rec(healthy)), real and imaginary,
        for both tears and every noise level;
plus the wall time of each reconstruction.  The exact permittivity on the inverse mesh is the
volume average of the true one over each tet (sampled on a barycentric lattice), the best a
piecewise-constant reconstruction can reach; the injury area is the set of tets the tear
touches (exact injured and healthy averages differ).  The 2-norms weight every tet equally
(the inverse mesh is uniform).

Everything numerical runs in libmw (solves, S, gradient, L-BFGS); this module generates the
seeded inputs, wires the calls and evaluates the two metrics above on the results.
Usage: python -m paper_2311_05322_gb300.design_study --scale reduced
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from phantom import (ARM_CENTER, EPS_MATCHING, SHOULDER_HI, SHOULDER_LO, add_noise, antenna_layers, box_partition,
                     kuhn_mesh, shoulder_eps, shoulder_eps_at, study_tear)

from . import mw

SCALES = {
    # data mesh, inverse mesh, partitions (data, inverse), L-BFGS iterations, antenna counts, noise levels
    "tiny": dict(data=(24, 24, 10), inv=(18, 18, 8), pdata=(4, 4, 2), pinv=(3, 3, 2), iters=6,
                 counts=(32, 16), snr_db=(23.0,), freq=1.0e9),
    "reduced": dict(data=(55, 55, 24), inv=(44, 44, 17), pdata=(11, 11, 5), pinv=(9, 9, 4), iters=15,
                    counts=(96, 64, 32, 16), snr_db=(23.0, 15.0, 10.0), freq=1.0e9),
}
TEARS = ("partial", "large")


def _mesh(cells):
    return kuhn_mesh(*cells, lo=SHOULDER_LO, hi=SHOULDER_HI)


def _pairs(e):
    return np.stack([e.real, e.imag], 1)


def lattice(m: int = 5) -> np.ndarray:
    """Barycentric points (i, j, k, l) / m with i + j + k + l = m: equal-weight samples of a tet."""
    pts = [(i, j, k, m - i - j - k) for i in range(m + 1) for j in range(m + 1 - i) for k in range(m + 1 - i - j)]
    return np.asarray(pts, dtype=np.float64) / m


def tet_average_eps(mesh, tear=None, matching=EPS_MATCHING, m: int = 5, chunk: int = 20000) -> np.ndarray:
    """Per-tet mean of the true permittivity over the lattice points of each tet."""
    lam = lattice(m)
    out = np.empty(mesh.n_tet, dtype=np.complex128)
    for t0 in range(0, mesh.n_tet, chunk):
        X = mesh.xyz[mesh.tets[t0:t0 + chunk]]                     # [t, 4, 3]
        pts = np.einsum("pk,tkd->tpd", lam, X).reshape(-1, 3)
        out[t0:t0 + chunk] = shoulder_eps_at(pts, tear, matching).reshape(X.shape[0], -1).mean(axis=1)
    return out


def err(rec: np.ndarray, exact: np.ndarray, mask: np.ndarray | None = None) -> tuple[float, float]:
    """Eq. (saharerr) for the real and the imaginary part, over the tets in mask (all if None)."""
    if mask is not None:
        rec, exact = rec[mask], exact[mask]
    d = rec - exact
    return (float(np.linalg.norm(d.real) / np.linalg.norm(exact.real)),
            float(np.linalg.norm(d.imag) / np.linalg.norm(exact.imag)))


def ctr(rec_injured: np.ndarray, rec_healthy: np.ndarray, mask: np.ndarray) -> tuple[float, float]:
    """Eq. (saharcont): mean of eps_rec(injured) - eps_rec(healthy) over the injury area."""
    d = (rec_injured - rec_healthy)[mask]
    return float(d.real.mean()), float(d.imag.mean())


class Forward:
    """A context on one mesh, its stale background preconditioner and the current antennas."""

    def __init__(self, cells, parts, freq, eps_ref):
        self.mesh = _mesh(cells)
        self.freq = freq
        c = mw.Context(0)
        c.set_mesh(self.mesh.xyz, self.mesh.tets)
        c.assemble([freq], _pairs(eps_ref), EPS_MATCHING)
        c.setup_preconditioner(int(np.prod(parts)), box_partition(self.mesh, parts, seed=7), 1, mw.MW_PREC_BF16)
        self.ctx = c
        self.opts = mw.solve_opts(mode=mw.MW_MODE_MIXED, tol=1e-8, inner_tol=1e-4)

    def antennas(self, n):
        pos, d = antenna_layers(n, 0.10, ARM_CENTER)
        self.ctx.set_sources(pos, d)

    def S(self, eps):
        self.ctx.assemble([self.freq], _pairs(eps), EPS_MATCHING)
        S, _ = self.ctx.solve(self.opts)
        return S


def run(scale: str = "reduced", seed: int = 5, verbose: bool = False) -> dict:
    cfg = SCALES[scale]
    t0 = time.time()
    data = Forward(cfg["data"], cfg["pdata"], cfg["freq"], shoulder_eps(_mesh(cfg["data"])))
    inv = Forward(cfg["inv"], cfg["pinv"], cfg["freq"], np.full(_mesh(cfg["inv"]).n_tet, EPS_MATCHING))
    hom = np.full(data.mesh.n_tet, EPS_MATCHING, dtype=complex)
    start = _pairs(np.full(inv.mesh.n_tet, EPS_MATCHING, dtype=complex))
    exact = {"healthy": tet_average_eps(inv.mesh)}
    masks = {}
    for k in TEARS:
        exact[k] = tet_average_eps(inv.mesh, study_tear(k))
        masks[k] = exact[k] != exact["healthy"]
    io = mw.inv_opts(m=8, max_it=cfg["iters"], alpha=0.0, first_step=1.0)
    hom_inv = np.full(inv.mesh.n_tet, EPS_MATCHING, dtype=complex)
    out = {"scale": scale, "config": dict(cfg), "inverse_tets": int(inv.mesh.n_tet),
           "injury_tets": {k: int(masks[k].sum()) for k in TEARS},
           "start_err_total_partial": err(hom_inv, exact["partial"]),
           "start_err_injury_partial": err(hom_inv, exact["partial"], masks["partial"]), "rows": []}
    for n in cfg["counts"]:
        data.antennas(n)
        inv.antennas(n)
        S_clean = {"healthy": data.S(shoulder_eps(data.mesh))}
        for k in TEARS:
            S_clean[k] = data.S(shoulder_eps(data.mesh, study_tear(k)))
        S_emp = data.S(hom)
        for si, snr in enumerate(cfg["snr_db"]):
            rec, secs, J = {}, {}, {}
            for ci, (case, S) in enumerate(S_clean.items()):
                S_obs = add_noise(S, snr, seed=seed * 100_000 + n * 1000 + si * 10 + ci)
                t = time.time()
                e, h = inv.ctx.invert(S_obs, S_emp, start, io, inv.opts)
                secs[case] = time.time() - t
                rec[case] = e[:, 0] + 1j * e[:, 1]
                J[case] = [float(h["J"][0]), float(h["J"][-1])]
            row = {"N": n, "snr_db": snr, "seconds": secs, "J_first_last": J,
                   "err_total_partial": err(rec["partial"], exact["partial"]),
                   "err_injury_partial": err(rec["partial"], exact["partial"], masks["partial"]),
                   "ctr": {k: ctr(rec[k], rec["healthy"], masks[k]) for k in TEARS}}
            out["rows"].append(row)
            if verbose:
                print(json.dumps(row), flush=True)
    out["total_s"] = time.time() - t0
    data.ctx.close()
    inv.ctx.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", default="reduced", choices=list(SCALES))
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps(run(a.scale, a.seed, verbose=True)), flush=True)
