"""Launch-shape tuner: each choice is the fastest of its timed candidates, and no launch shape
changes a result bit (the same arithmetic runs in the same order)."""
import numpy as np
import pytest

from phantom import EPS_MATCHING, box_partition, kuhn_mesh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mw():
    from paper_2311_05322_gb300 import mw
    return mw


@pytest.fixture(scope="module")
def box():
    """10 x 8 x 6 Kuhn box (several 128-row and 64-K tiles per subdomain), seeded eps."""
    m = kuhn_mesh(10, 8, 6, lo=(-0.05, -0.04, -0.03), hi=(0.05, 0.04, 0.03))
    rng = np.random.default_rng(41)
    eps = EPS_MATCHING + rng.uniform(-6, 6, m.n_tet) + 1j * rng.uniform(-4, 4, m.n_tet)
    return m, eps


def _ctx(m, eps):
    mw = _mw()
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    c.assemble([1e9], np.stack([eps.real, eps.imag], 1), EPS_MATCHING)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1), seed=3), 1, mw.MW_PREC_BF16)
    return c


def test_autotune_report(box):
    mw = _mw()
    m, eps = box
    c = _ctx(m, eps)
    r = c.autotune(32, mw.MW_MODE_MIXED, 50)
    assert set(r["spmm_ms"]) == {1, 128, 256, 512}        # 1: the halo-tiled SpMM (32 columns: even)
    r5 = c.autotune(5, mw.MW_MODE_MIXED, 50)
    assert set(r5["spmm_ms"]) == {128, 256, 512}          # odd column counts take the row-per-warp kernel only
    assert set(r["dots_ms"]) == {2, 3, 4, 5, 6} and set(r["update_ms"]) == {2, 3, 4, 5, 6}
    assert min(r["tc_ms"]) == 2 and max(r["tc_ms"]) >= 4
    for chosen, table in (("spmm_threads", "spmm_ms"), ("dots_stages", "dots_ms"), ("update_stages", "update_ms"),
                          ("tc_stages", "tc_ms")):
        t = r[table]
        assert all(v > 0 for v in t.values())
        assert r[chosen] == min(t, key=t.get)
    # 5 columns: the streaming Gram-Schmidt kernels are not used, so they have no candidates
    r5 = c.autotune(5, mw.MW_MODE_MIXED, 50)
    assert r5["dots_stages"] == 0 and r5["dots_ms"] == {} and r5["update_ms"] == {} and r5["tc_stages"] >= 2
    # FP64 mode has no tensor-core apply
    r64 = c.autotune(32, mw.MW_MODE_FP64, 50)
    assert r64["tc_stages"] == 0 and r64["tc_ms"] == {}
    with pytest.raises(mw.MWError):
        c.set_launch_shapes(32, mw.MW_MODE_MIXED, 50, tc_stages=1)
    with pytest.raises(mw.MWError):
        c.set_launch_shapes(32, mw.MW_MODE_MIXED, 50, spmm_threads=300)


def test_launch_shapes_bit_identical(box):
    mw = _mw()
    m, eps = box
    c = _ctx(m, eps)
    tc_max = max(c.autotune(32, mw.MW_MODE_MIXED, 50)["tc_ms"])
    E = c.info.n_edge
    rng = np.random.default_rng(5)
    B = rng.normal(size=(32, E)) + 1j * rng.normal(size=(32, E))
    bd = torch.from_numpy(B).cuda()
    opts = mw.solve_opts(mode=mw.MW_MODE_MIXED, tol=1e-10)
    for z_bf16 in (True, False):                          # preconditioned vectors in BF16 or FP32
        c.set_z_storage(z_bf16)
        c.set_autotune(False)
        x_ref = torch.empty_like(bd)
        st_ref = c.solve_rhs(32, bd, x_ref, opts)
        assert st_ref["n_converged"] == 32
        c.set_autotune(True)
        for tc, dots, upd, spmm in [(2, 2, 6, 128), (tc_max, 6, 2, 512), (3, 5, 3, 256), (4, 4, 4, 1)]:
            c.set_launch_shapes(32, mw.MW_MODE_MIXED, 50, tc, dots, upd, spmm)
            x = torch.empty_like(bd)
            st = c.solve_rhs(32, bd, x, opts)
            assert torch.equal(x, x_ref), (z_bf16, tc, dots, upd, spmm)
            assert np.array_equal(st["iters"], st_ref["iters"])
