"""Failure detection without any GPU fault: invalid inputs, calls out of order, non-convergence,
the allocation cap, and the device-side bounded wait (a phase that never completes runs out
after a short limit and reports MW_ETIMEOUT; the context stays usable)."""
import numpy as np
import pytest

from phantom import EPS_MATCHING, box_partition, kuhn_mesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small():
    from paper_2311_05322_gb300 import mw
    m = kuhn_mesh(4, 4, 3, lo=(-0.024, -0.024, -0.018), hi=(0.024, 0.024, 0.018))
    c = mw.Context(0)
    c.set_mesh(m.xyz, m.tets)
    return mw, m, c


def test_invalid_inputs_and_order():
    mw, m, c = _small()
    with pytest.raises(mw.MWError) as e:
        c.solve()
    assert e.value.status == mw.MW_ESTATE
    bad = np.tile([44.0, -20.0], (m.n_tet, 1))
    bad[3, 0] = np.nan
    with pytest.raises(mw.MWError) as e:
        c.assemble([1e9], bad, EPS_MATCHING)
    assert e.value.status == mw.MW_EINVAL
    t = m.tets.copy()
    t[0, 1] = t[0, 0]
    with pytest.raises(mw.MWError) as e:
        c.set_mesh(m.xyz, t)
    assert e.value.status == mw.MW_EINVAL


def test_nonconvergence_keeps_last_iterate():
    mw, m, c = _small()
    c.assemble([1e9], np.tile([44.0, -20.0], (m.n_tet, 1)), EPS_MATCHING)
    c.set_sources(np.array([[0.0, 0.0, 0.003]]), np.array([[0.0, 0.0, 1.0]]))
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1)), 1, mw.MW_PREC_FP64)
    S, st = c.solve(mw.solve_opts(max_it=2, tol=1e-12), allow_noconv=True)
    assert st["status"] == mw.MW_ENOCONV and st["n_converged"] == 0
    assert 0 < st["max_relres"] < 1 and np.all(np.isfinite(S))


def test_memory_cap_gives_enomem_and_context_recovers():
    mw, m, c = _small()
    c.assemble([1e9], np.tile([44.0, -20.0], (m.n_tet, 1)), EPS_MATCHING)
    c.set_memory_cap(1)
    with pytest.raises(mw.MWError) as e:
        c.setup_preconditioner(4, box_partition(m, (2, 2, 1)), 1, mw.MW_PREC_FP64)
    assert e.value.status == mw.MW_ENOMEM
    c.set_memory_cap(0)
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1)), 1, mw.MW_PREC_FP64)


def test_bounded_wait_runs_out_and_context_stays_usable():
    mw, m, c = _small()
    assert c.selftest_bounded_wait(1 << 14) == mw.MW_ETIMEOUT
    c.assemble([1e9], np.tile([44.0, -20.0], (m.n_tet, 1)), EPS_MATCHING)
    c.set_sources(np.array([[0.0, 0.0, 0.003]]), np.array([[0.0, 0.0, 1.0]]))
    c.setup_preconditioner(4, box_partition(m, (2, 2, 1)), 1, mw.MW_PREC_FP64)
    S, st = c.solve(mw.solve_opts(tol=1e-10))
    assert st["n_converged"] == 1
