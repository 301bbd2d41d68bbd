"""Host-side plan of the halo-tiled SpMM (no GPU): rows in the Morton order of their edge
midpoints, cut into blocks whose column sets fit the shared-memory bound.  The invariants the
kernel relies on hold on several meshes and bounds, and the blocks cut the gathered rows of X
well below one per nonzero."""
import numpy as np
import pytest

from paper_2311_05322_gb300 import mw
from phantom import kuhn_mesh, shoulder


@pytest.mark.parametrize("cells,halo_max", [((4, 3, 2), 64), ((12, 12, 12), 480), ((9, 7, 5), 100),
                                            ((20, 6, 3), 480), ((5, 5, 5), 65535)])
def test_plan_invariants(cells, halo_max):
    m = kuhn_mesh(*cells)
    st = mw.spmm_plan_stats(m.xyz, m.tets, halo_max)
    assert 1 <= st["blocks"] and st["halo_max"] <= halo_max
    if halo_max == 65535:
        assert st["blocks"] == 1                              # one block holds every column


def test_plan_rejects_bound_out_of_range():
    m = kuhn_mesh(3, 3, 3)
    with pytest.raises(mw.MWError):
        mw.spmm_plan_stats(m.xyz, m.tets, 32)


def test_halo_rows_per_nonzero_on_the_shoulder_mesh():
    """On a shoulder mesh (1/2 of the bench's cells per axis), the staged X rows per nonzero
    (summed halos over nonzeros) stay below 1/2: the kernel gathers X at most half as often as
    a row-per-warp product, which reads one row of X per nonzero."""
    w = shoulder((40, 40, 17), n_src=4)
    st = mw.spmm_plan_stats(w.mesh.xyz, w.mesh.tets, 480)
    assert st["halo_max"] <= 480
    ratio = st["halo_total"] / st["nnz"]
    assert ratio < 0.5, ratio
    print(f"\nblocks {st['blocks']}, staged rows per nonzero {ratio:.3f}")
