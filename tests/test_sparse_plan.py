"""Host-side plan of the sparse subdomain solves (no GPU): nested dissection and multifrontal
structure pass their invariants on several meshes, partitions, overlaps and leaf sizes, and the
factor storage grows much more slowly than the dense inverses'."""
import numpy as np
import pytest

from paper_2311_05322_gb300 import mw
from phantom import box_partition, kuhn_mesh


@pytest.mark.parametrize("cells,parts,overlap,leaf", [((5, 4, 3), (2, 2, 1), 1, 64), ((5, 4, 3), (1, 1, 1), 0, 1),
                                                       ((12, 10, 8), (2, 1, 1), 2, 64), ((12, 10, 8), (2, 2, 2), 1, 256),
                                                       ((9, 7, 5), (3, 2, 1), 2, 17)])
def test_plan_invariants(cells, parts, overlap, leaf):
    m = kuhn_mesh(*cells)
    st = mw.sparse_plan_stats(m.xyz, m.tets, int(np.prod(parts)), box_partition(m, parts, seed=3), overlap, leaf)
    assert st["nodes"] >= 1 and st["max_front"] >= 1
    assert st["factor_entries"] <= 2 * st["dense_entries"]        # small cases: padding may dominate


def test_factor_storage_grows_like_n_four_thirds():
    """Nested dissection of a 3D mesh stores O(n^(4/3)) factor entries against n^2 dense ones."""
    c43, ratio = [], []
    for c in (12, 16, 24):
        m = kuhn_mesh(c, c, c // 2)
        st = mw.sparse_plan_stats(m.xyz, m.tets, 1, np.zeros(m.n_tet, np.int32), 0, 256)
        n = np.sqrt(st["dense_entries"])
        c43.append(st["factor_entries"] / n ** (4.0 / 3.0))
        ratio.append(st["factor_entries"] / st["dense_entries"])
    assert max(c43) / min(c43) < 1.2
    assert ratio[2] < ratio[0] / 3.5


def test_plan_rejects_bad_arguments():
    m = kuhn_mesh(3, 3, 2)
    with pytest.raises(mw.MWError):
        mw.sparse_plan_stats(m.xyz, m.tets, 1, np.zeros(m.n_tet, np.int32), 0, 0)   # leaf 0
    with pytest.raises(mw.MWError):
        mw.sparse_plan_stats(m.xyz, m.tets, 2, np.full(m.n_tet, 5, np.int32), 0, 64)  # part out of range
