"""Antenna-count study (Sec. V): the layered antenna design and the two metrics of Eq. (saharerr)
and Eq. (saharcont) on hand-made inputs (CPU), and a tiny run of the study on the GPU."""
import numpy as np
import pytest

from phantom import LAYER_FULL, LAYER_WEIGHTS, LAYER_Z, antenna_layers, layer_counts, study_tear


def _study():
    from paper_2311_05322_gb300 import design_study
    return design_study


def test_layer_counts_match_the_32_antenna_design_and_scale():
    assert layer_counts(32) == (5, 11, 10, 6)
    assert layer_counts(96) == (15, 33, 30, 18)
    assert layer_counts(64) == (10, 22, 20, 12)
    for n in range(4, 130):
        c = layer_counts(n)
        assert sum(c) == n
        q = n * np.asarray(LAYER_WEIGHTS) / sum(LAYER_WEIGHTS)
        assert np.all(np.abs(np.asarray(c) - q) < 1.0)


def test_antenna_layers_geometry():
    pos, d = antenna_layers(32, rho=0.1)
    assert pos.shape == (32, 3) and np.all(d == [0, 0, 1])
    assert np.allclose(np.hypot(pos[:, 0], pos[:, 1]), 0.1)
    k = 0
    prev = None
    for cnt, full, z in zip(layer_counts(32), LAYER_FULL, LAYER_Z):
        p = pos[k:k + cnt]
        k += cnt
        assert np.allclose(p[:, 2], z)
        ang = np.arctan2(p[:, 1], p[:, 0])
        if not full:
            assert np.all(p[:, 0] > 0)                     # half rings face away from the torso
        pitch = (2 * np.pi if full else np.pi) / cnt
        diff = np.diff(np.unwrap(ang))
        assert np.allclose(diff, pitch)
        # first antenna sits half a pitch (or a whole one, alternating) from the ring's start
        start = 0.0 if full else -0.5 * np.pi
        frac = ((ang[0] - start) / pitch) % 1.0
        assert np.isclose(frac, 0.5) or np.isclose(frac, 0.0) or np.isclose(frac, 1.0)
        if prev is not None:
            assert not np.isclose(frac, prev)                  # adjacent rings are shifted
        prev = frac


def test_study_tear_volumes():
    for kind, vol_ml in (("partial", 1.0), ("large", 5.0)):
        t = study_tear(kind)
        v = 4.0 / 3.0 * np.pi * np.prod(t.semi_axes) * 1e6
        assert abs(v - vol_ml) / vol_ml < 0.01


def test_err_and_ctr_on_hand_made_values():
    ds = _study()
    exact = np.array([3 + 4j, 0 + 0j, 4 + 3j])
    rec = np.array([3 + 4j, 3 + 4j, 4 + 3j])
    # real: ||(0,3,0)|| / ||(3,0,4)|| = 3/5; imag: ||(0,4,0)|| / ||(4,0,3)|| = 4/5
    assert ds.err(rec, exact) == pytest.approx((0.6, 0.8), rel=1e-15)
    mask = np.array([True, False, True])
    assert ds.err(rec, exact, mask) == (0.0, 0.0)
    inj = np.array([2 + 1j, 5 - 1j, 7 + 0j])
    hea = np.array([1 + 1j, 0 + 0j, 3 - 2j])
    # mean of (1+0j, 4+2j) over the mask's two entries
    assert ds.ctr(inj, hea, mask) == (2.5, 1.0)



def test_tet_average_is_the_volume_mean():
    """Lattice samples are an equal-weight rule exact for linear functions (mean of the lattice
    = centroid); on the phantom, tets away from interfaces get their tissue value exactly and
    tets the tear cuts get values between fluid and tissue."""
    ds = _study()
    lam = ds.lattice(5)
    assert lam.shape == (56, 4) and np.allclose(lam.sum(1), 1) and np.allclose(lam.mean(0), 0.25)
    from phantom import EPS_FLUID, EPS_MATCHING, EPS_TENDON, kuhn_mesh
    m = kuhn_mesh(12, 12, 8, lo=(-0.06, -0.02, -0.02), hi=(-0.02, 0.02, 0.02))
    t = study_tear("large")
    h = ds.tet_average_eps(m)
    inj = ds.tet_average_eps(m, t)
    touched = inj != h
    assert touched.sum() > 10
    # fluid replaces tendon or muscle only: a touched tet of one tissue lies on the segment
    # between that tissue and fluid (its fluid fraction), strictly inside or at the fluid end
    from phantom import EPS_MUSCLE
    pure = touched & (np.isclose(h, EPS_TENDON, rtol=1e-14, atol=0) | np.isclose(h, EPS_MUSCLE, rtol=1e-14, atol=0))
    assert pure.sum() > 10
    frac = (inj[pure] - h[pure]) / (EPS_FLUID - h[pure])
    assert np.all(frac.real > 0) and np.all(frac.real <= 1 + 1e-12) and np.allclose(frac.imag, 0, atol=1e-12)
    far = np.linalg.norm(m.centroids() - np.array([-0.055, 0.015, 0.015]), axis=1) < 0.004
    assert far.sum() > 0 and np.allclose(h[far], EPS_MATCHING, rtol=1e-14, atol=0)


@pytest.mark.gpu
def test_tiny_study_runs_and_fits():
    pytest.importorskip("torch")
    ds = _study()
    out = ds.run("tiny", seed=1)
    assert len(out["rows"]) == 2 and out["injury_tets"]["large"] > out["injury_tets"]["partial"] > 0
    for row in out["rows"]:
        for case, (j0, j1) in row["J_first_last"].items():
            assert np.isfinite(j1) and j1 < j0, (row["N"], case)
        assert all(np.isfinite(v) for v in row["err_total_partial"] + row["err_injury_partial"])
        assert all(np.isfinite(v) for k in row["ctr"] for v in row["ctr"][k])
