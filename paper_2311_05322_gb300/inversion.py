"""Inversion time-to-misfit and the learned initialiser (Sec. IV-D).

Differential reading of the inversion: the healthy anatomy is known (a prior scan), the data are
the S-parameters of the injured shoulder computed on a finer "data" mesh with complex Gaussian
noise, and L-BFGS reconstructs eps on a coarser "inverse" mesh (different meshes, as Sec. IV-D
asks, to avoid the inverse crime) starting from the healthy permittivity.  The fit is to the
differential data (S_obs - S_healthy on the data mesh, plus S_healthy on the inverse mesh), so the
mesh-to-mesh modelling error of the healthy anatomy cancels to first order.  The learned
initialiser maps the normalised difference Delta S = S_injured - S_healthy to Delta eps on a
32^3 grid over the tendon band; its tet averages are added to the start.

Everything numerical runs in libmw (solves, S, gradient, L-BFGS, network training/inference,
grid-to-tet averaging); this module only wires the calls together and generates seeded inputs.
Usage: python -m paper_2311_05322_gb300.inversion --scale reduced
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass

import numpy as np

from phantom import (EPS_MATCHING, ROI_BOX, ROI_GRID, add_noise, box_partition, dipole_ring, kuhn_mesh, random_tear,
                     shoulder_eps, SHOULDER_HI, SHOULDER_LO, ARM_CENTER, tear_target_grid)

from . import mw

SCALES = {
    # data mesh, inverse mesh, transmitters, frequencies, partitions (data, inverse), samples, epochs, iterations
    "tiny": dict(data=(24, 24, 10), inv=(18, 18, 8), n_src=16, freqs=(1.0e9,), pdata=(4, 4, 2), pinv=(3, 3, 2),
                 samples=96, epochs=60, iters=6, alpha=0.0),
    "reduced": dict(data=(44, 44, 17), inv=(30, 30, 13), n_src=32, freqs=(1.0e9,), pdata=(9, 9, 4), pinv=(6, 6, 3),
                    samples=600, epochs=200, iters=10, alpha=0.0),
    # the reduced configuration with fewer samples and iterations (GPU test of the learned gain)
    "test": dict(data=(44, 44, 17), inv=(30, 30, 13), n_src=32, freqs=(1.0e9,), pdata=(9, 9, 4), pinv=(6, 6, 3),
                 samples=256, epochs=120, iters=5, alpha=0.0),
    "full": dict(data=(55, 55, 24), inv=(44, 44, 17), n_src=64, freqs=(0.8e9, 1.0e9, 1.2e9), pdata=(11, 11, 5),
                 pinv=(9, 9, 4), samples=2000, epochs=100, iters=20, alpha=0.0),
    # the reduced meshes with a smaller training set: the time-to-misfit leg of the default bench
    "bench": dict(data=(44, 44, 17), inv=(30, 30, 13), n_src=32, freqs=(1.0e9,), pdata=(9, 9, 4), pinv=(6, 6, 3),
                  samples=300, epochs=120, iters=10, alpha=0.0),
}
TARGET_SCALE = 20.0      # Delta eps is trained in units of 20
# inner-cycle reduction of the mixed solves (GMRES-IR; 1e-8 is decided by the outer FP64 residual):
# on the inverse meshes 1e-4 measured faster than 1e-2 (4.63 s against 4.79 s at full scale)
INNER_TOL = 1e-4
# An arm reaches the target misfit when its J is within this relative band of it.  The arms'
# J agree only to the forward solves' tolerance (relres 1e-8): the misfit is a small difference
# of S-matrices, so its relative error is far larger; measured between the plain FP64 and the
# mixed arm at the same eps (iteration 0) 5e-6, and 1.3e-5 after ten L-BFGS iterations.  The
# band is ten times that.
TARGET_REL_BAND = 1e-4
TARGET_BLUR_M = 0.003    # targets are blurred to about the resolution the inverse mesh can carry
FLUID_RANGE = ((60.0, 75.0), (25.0, 40.0))


def _mesh(cells):
    return kuhn_mesh(*cells, lo=SHOULDER_LO, hi=SHOULDER_HI)


def _sources(cells, n_src):
    hz = (SHOULDER_HI[2] - SHOULDER_LO[2]) / cells[2]
    return dipole_ring(n_src, 0.10, hz / 2 if cells[2] % 2 == 0 else 0.0, ARM_CENTER)


def _pairs(e):
    return np.stack([e.real, e.imag], 1)


@dataclass
class Forward:
    """A context on one mesh with a stale background preconditioner."""
    ctx: mw.Context
    mesh: object
    freqs: tuple
    opts: object

    @classmethod
    def build(cls, cells, n_src, freqs, parts, eps_ref, prec=mw.MW_PREC_BF16, mode=mw.MW_MODE_MIXED):
        m = _mesh(cells)
        c = mw.Context(0)
        c.set_mesh(m.xyz, m.tets)
        c.assemble(list(freqs), _pairs(eps_ref), EPS_MATCHING)
        c.setup_preconditioner(int(np.prod(parts)), box_partition(m, parts, seed=7), 1, prec)
        pos, d = _sources(cells, n_src)
        c.set_sources(pos, d)
        return cls(c, m, tuple(freqs), mw.solve_opts(mode=mode, tol=1e-8, inner_tol=INNER_TOL))

    def S(self, eps):
        self.ctx.assemble(list(self.freqs), _pairs(eps), EPS_MATCHING)
        S, _ = self.ctx.solve(self.opts)
        return S


def nn_input(dS: np.ndarray, S_empty: np.ndarray) -> np.ndarray:
    r = dS / np.abs(S_empty)
    return np.concatenate([r.real.ravel(), r.imag.ravel()]).astype(np.float32)


def he_init(n_in: int, seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the flat layout of mw_nn_init."""
    rng = np.random.default_rng(seed)
    hid, k3 = 1024, 64
    parts = [rng.normal(size=1024 * n_in) * np.sqrt(2.0 / n_in), np.zeros(hid),
             rng.normal(size=hid * hid) * np.sqrt(2.0 / hid), np.zeros(hid),
             rng.normal(size=16 * 16 * k3) * np.sqrt(2.0 / (16 * 8)), np.zeros(16),
             rng.normal(size=16 * 8 * k3) * np.sqrt(2.0 / (16 * 8)), np.zeros(8),
             rng.normal(size=8 * 2 * k3) * np.sqrt(1.0 / (8 * 8)), np.zeros(2)]
    return np.concatenate(parts).astype(np.float32)


def blurred_target(tear) -> np.ndarray:
    """Delta eps of the tear on the ROI grid, Gaussian-blurred (sigma TARGET_BLUR_M per axis)."""
    from scipy.ndimage import gaussian_filter
    g = tear_target_grid(tear)
    h = [(ROI_BOX[3 + d] - ROI_BOX[d]) / ROI_GRID for d in range(3)]
    sig = (TARGET_BLUR_M / h[2], TARGET_BLUR_M / h[1], TARGET_BLUR_M / h[0])     # grid axes z, y, x
    return np.stack([gaussian_filter(g[c], sig, mode="constant") for c in range(2)])


def make_dataset(fwd: Forward, S_healthy, S_empty, n: int, seed0: int, f_index: int, snr_db: float):
    """Noisy injured-minus-healthy S differences (inputs) and blurred Delta eps grids (targets)."""
    X, T, tears, rel = [], [], [], []
    for k in range(n):
        tear = random_tear(seed0 + k, eps_range=FLUID_RANGE)
        S = fwd.S(shoulder_eps(fwd.mesh, tear))
        dS = S[f_index] - S_healthy[f_index]
        rel.append(np.linalg.norm(dS) / np.linalg.norm(S_healthy[f_index]))
        Sn = add_noise(S[f_index], snr_db, seed=500_000 + seed0 + k)
        X.append(nn_input(Sn - S_healthy[f_index], S_empty[f_index]))
        T.append((blurred_target(tear) / TARGET_SCALE).astype(np.float32))
        tears.append(tear)
    return np.stack(X), np.stack(T), tears, float(np.median(rel))


def first_time_below(J, secs, target):
    for j, s in zip(J, secs):
        if j <= target:
            return float(s)
    return None


def held_out_tear(seed: int, k: int, n: int):
    """The k-th of n held-out tears: centre and fluid drawn from random_tear, semi-axes rescaled
    so that their mean is 2 + 8 (k + 1/2) / n mm (each clipped to 2-10 mm), which spreads the
    tears over the whole size range."""
    t = random_tear(99_000 + seed + 17 * k, eps_range=FLUID_RANGE)
    target = 0.002 + 0.008 * (k + 0.5) / n
    f = target / (sum(t.semi_axes) / 3.0)
    axes = tuple(min(0.010, max(0.002, a * f)) for a in t.semi_axes)
    return type(t)(t.center, axes, t.eps)


def _stats(v):
    v = [x for x in v if x is not None]
    if not v:
        return {"n": 0}
    return {"n": len(v), "mean": float(np.mean(v)), "std": float(np.std(v, ddof=1)) if len(v) > 1 else 0.0,
            "min": float(np.min(v)), "max": float(np.max(v))}


def run(scale: str = "reduced", seed: int = 3, plain: bool | None = None, snr_db: float = 40.0, tears: int = 1,
        alphas=(), verbose=False, reciprocal: bool = True, target_J: float | None = None, pinv=None):
    """Train the network once, then invert `tears` held-out tears from the healthy start and from
    the network's start (mixed solver; the plain FP64 inversion too on the first tear when
    `plain`).  Per tear: the target is the reference inversion's J after max_it (plain FP64 on the
    first tear when run, else the mixed inversion from the healthy start), and each variant's
    time to reach it.  `alphas`: Tikhonov sweep of the mixed inversion on the first tear.
    `pinv`: box partition of the inverse mesh, replacing the scale's.
    `reciprocal`: on the first tear, also the mixed inversions whose adjoint fields come from the
    forward fields by reciprocity (mw_set_adjoint_mode) instead of adjoint solves.
    `target_J`: the first tear's target when the plain FP64 inversion is not run here (its J
    after max_it from an earlier run with the same seeds: the inputs are deterministic)."""
    cfg = dict(SCALES[scale])
    if pinv is not None:
        cfg["pinv"] = tuple(int(v) for v in pinv)
    out = {"scale": scale, "config": {k: v for k, v in cfg.items()}}
    f_nn = len(cfg["freqs"]) // 2                       # network sees the middle frequency
    t0 = time.time()
    data_mesh = _mesh(cfg["data"])
    eps_h = shoulder_eps(data_mesh)
    hom = np.full(data_mesh.n_tet, EPS_MATCHING, dtype=complex)

    # --- training data on the data mesh, one frequency ------------------------------------------
    gen = Forward.build(cfg["data"], cfg["n_src"], (cfg["freqs"][f_nn],), cfg["pdata"], eps_h)
    S_h1 = gen.S(eps_h)
    S_e1 = gen.S(hom)
    n = cfg["samples"]
    X, T, _, rel = make_dataset(gen, S_h1, S_e1, n, 10_000 + 1000 * seed, 0, snr_db)
    n_tr = int(round(0.9 * n))
    mu, sd = X[:n_tr].mean(axis=0), X[:n_tr].std(axis=0) + 1e-12     # per-feature standardisation
    X = ((X - mu) / sd).astype(np.float32)
    out["data_generation_s"] = time.time() - t0
    # --- training ---------------------------------------------------------------------------------
    n_in = X.shape[1]
    gen.ctx.nn_init(n_in, he_init(n_in, seed))
    losses, train_s = gen.ctx.nn_train(X[:n_tr], T[:n_tr], batch=64, epochs=cfg["epochs"], lr=1e-3, seed=seed)
    Y = gen.ctx.nn_infer(X[n_tr:])
    mse_nn = float(np.mean((Y - T[n_tr:]) ** 2)) * TARGET_SCALE ** 2
    mse_zero = float(np.mean(T[n_tr:] ** 2)) * TARGET_SCALE ** 2
    out["network"] = {"median_rel_dS": rel, "n_in": n_in, "train": n_tr, "test": n - n_tr,
                      "epoch_loss_first_last": [losses[0], losses[-1]],
                      "train_s": train_s, "test_mse": mse_nn, "zero_predictor_mse": mse_zero,
                      "gain": 1.0 - mse_nn / mse_zero}
    theta = gen.ctx.nn_get_params()
    gen.ctx.close()

    # --- observed data: held-out tears on the data mesh, all frequencies, noise -------------------
    data = Forward.build(cfg["data"], cfg["n_src"], cfg["freqs"], cfg["pdata"], eps_h)
    S_emp = data.S(hom)
    S_hd = data.S(eps_h)
    w = 1.0 / np.abs(S_emp) ** 2                         # the cost's weights (Eq. sahar:2)
    obs = []
    for k in range(tears):
        tear = held_out_tear(seed, k, tears)
        S_inj = data.S(shoulder_eps(data_mesh, tear))
        S_obs = add_noise(S_inj, snr_db, seed=7_000 + seed + 31 * k)
        sig = float(np.sum(w * np.abs(S_inj - S_hd) ** 2))
        noise = float(np.sum(w * np.abs(S_obs - S_inj) ** 2))
        obs.append((tear, S_obs, {"tear_signal": sig, "noise": noise, "snr_db": 10.0 * np.log10(sig / noise)}))
    data.ctx.close()

    # --- inversions on the inverse mesh -------------------------------------------------------------
    inv_mesh = _mesh(cfg["inv"])
    eps0 = shoulder_eps(inv_mesh)
    inv = Forward.build(cfg["inv"], cfg["n_src"], cfg["freqs"], cfg["pinv"], eps0)
    inv.ctx.nn_init(n_in, theta)
    # differential data: fit S(eps) - S(eps_healthy) on the inverse mesh to S_obs - S_healthy on
    # the data mesh, i.e. S(eps) against S_obs - S_hd + S(eps_healthy, inverse mesh)
    S_hinv = inv.S(eps0)
    mixed = mw.solve_opts(mode=mw.MW_MODE_MIXED, tol=1e-8, inner_tol=INNER_TOL)
    if plain is None:
        plain = scale != "full"

    def invert(S_fit, start, sopts, alpha):
        io = mw.inv_opts(m=8, max_it=cfg["iters"], alpha=alpha, first_step=1.0)
        e, h = inv.ctx.invert(S_fit, S_emp, start, io, sopts)
        return {"J": h["J"].tolist(), "seconds": h["seconds"].tolist(), "evaluations": h["evaluations"]}

    cases = []
    for k, (tear, S_obs, snr) in enumerate(obs):
        S_fit = S_obs - S_hd + S_hinv
        x_obs = ((nn_input(S_obs[f_nn] - S_hd[f_nn], S_emp[f_nn]) - mu) / sd).astype(np.float32)
        grid = inv.ctx.nn_infer(x_obs[None])[0] * TARGET_SCALE
        learned0 = _pairs(eps0) + inv.ctx.nn_grid_to_tets(grid, np.asarray(ROI_BOX))
        res = {"mixed": invert(S_fit, _pairs(eps0), mixed, cfg["alpha"]),
               "mixed_learned": invert(S_fit, learned0, mixed, cfg["alpha"])}
        if k == 0 and reciprocal:
            # the same mixed inversions with the adjoint fields formed from the forward fields
            # by reciprocity instead of adjoint solves
            inv.ctx.set_adjoint_mode(True)
            res["mixed_reciprocal"] = invert(S_fit, _pairs(eps0), mixed, cfg["alpha"])
            res["mixed_learned_reciprocal"] = invert(S_fit, learned0, mixed, cfg["alpha"])
            inv.ctx.set_adjoint_mode(False)
        if plain and k == 0:
            inv.ctx.assemble(list(cfg["freqs"]), _pairs(eps0), EPS_MATCHING)
            # FP64 factorisation and FP64 apply: the plain path is FP64 throughout (its setup is
            # outside the inversion's clock, like the mixed path's)
            t_setup = time.time()
            inv.ctx.setup_preconditioner(int(np.prod(cfg["pinv"])), box_partition(inv.mesh, cfg["pinv"], seed=7), 1,
                                         mw.MW_PREC_FP64)
            out["plain_fp64_setup_s"] = time.time() - t_setup
            res["plain_fp64"] = invert(S_fit, _pairs(eps0), mw.solve_opts(mode=mw.MW_MODE_FP64, tol=1e-8),
                                       cfg["alpha"])
            inv.ctx.assemble(list(cfg["freqs"]), _pairs(eps0), EPS_MATCHING)
            inv.ctx.setup_preconditioner(int(np.prod(cfg["pinv"])), box_partition(inv.mesh, cfg["pinv"], seed=7), 1,
                                         mw.MW_PREC_BF16)
        ref = res["plain_fp64"] if "plain_fp64" in res else res["mixed"]
        target = ref["J"][-1]
        given = k == 0 and target_J is not None and "plain_fp64" not in res
        if given:
            target = target_J
        for v in res.values():
            v["time_to_target_s"] = first_time_below(v["J"], v["seconds"], target * (1.0 + TARGET_REL_BAND))
        cases.append({"tear": {"center": tear.center, "semi_axes": tear.semi_axes,
                               "eps": [tear.eps.real, tear.eps.imag]},
                      "inversion": res, "target_J": target, "target_rel_band": TARGET_REL_BAND,
                      "target_from": "plain_fp64 after max_it" if "plain_fp64" in res else
                      ("plain_fp64 after max_it, given" if given else "mixed after max_it"),
                      "learned_start_dJ0": res["mixed_learned"]["J"][0] - res["mixed"]["J"][0],
                      "learned_start_rel_dJ0": (res["mixed_learned"]["J"][0] - res["mixed"]["J"][0])
                      / res["mixed"]["J"][0], **snr})
        if verbose:
            print(json.dumps(cases[-1]), flush=True)
    # the first tear's record keeps the single-tear keys
    out.update({k: cases[0][k] for k in ("inversion", "target_J", "target_rel_band", "target_from", "tear",
                                         "learned_start_dJ0")})
    out["cases"] = cases
    out["summary"] = {
        "tears": len(cases),
        "snr_db": _stats([c["snr_db"] for c in cases]),
        "time_to_target_s": {v: _stats([c["inversion"][v]["time_to_target_s"] for c in cases])
                             for v in ("mixed", "mixed_learned")},
        "learned_start_rel_dJ0": _stats([c["learned_start_rel_dJ0"] for c in cases]),
        "learned_reaches_target_first": sum(
            1 for c in cases if c["inversion"]["mixed_learned"]["time_to_target_s"] is not None
            and (c["inversion"]["mixed"]["time_to_target_s"] is None
                 or c["inversion"]["mixed_learned"]["time_to_target_s"] < c["inversion"]["mixed"]["time_to_target_s"])),
    }
    sweep = []
    for a in alphas:
        tear, S_obs, _ = obs[0]
        r = invert(S_obs - S_hd + S_hinv, _pairs(eps0), mixed, a)
        # time until the run is within 5 % of its own final cost
        r["time_to_5pct_of_final_s"] = first_time_below(r["J"], r["seconds"], 1.05 * r["J"][-1])
        sweep.append({"alpha": a, **r})
    out["alpha_sweep"] = sweep
    out["total_s"] = time.time() - t0
    inv.ctx.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", default="reduced", choices=list(SCALES))
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain", action="store_true")
    ap.add_argument("--tears", type=int, default=1)
    ap.add_argument("--alphas", default="", help="comma-separated Tikhonov weights for the sweep")
    ap.add_argument("--pinv", default=None, help="box partition of the inverse mesh, e.g. 12x12x5")
    ap.add_argument("--target", type=float, default=None,
                    help="first tear's target J (the plain FP64 inversion's, from an earlier run)")
    a = ap.parse_args()
    plain = False if a.no_plain else (True if a.plain else None)
    alphas = [float(x) for x in a.alphas.split(",") if x]
    pinv = tuple(int(v) for v in a.pinv.split("x")) if a.pinv else None
    print(json.dumps(run(a.scale, a.seed, plain=plain, tears=a.tears, alphas=alphas, verbose=True, target_J=a.target,
                         pinv=pinv)),
          flush=True)
