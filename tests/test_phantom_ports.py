"""The waveguide geometry generators (inputs only): straight guide and waveguide-ring chamber."""
import numpy as np

from oracle.topology import build_topology
from phantom import faces_on_plane, kuhn_mesh, port_chamber, waveguide_section


def _boundary_keys(m):
    t = build_topology(m.n_vert, m.tets, with_pattern=False)
    return set(map(tuple, t.faces[t.bface].tolist())), set(map(tuple, t.faces.tolist()))


def test_waveguide_section_faces():
    m, fv, lab, ps = waveguide_section((4, 2, 6), 0.02, 0.01, 0.03)
    bkeys, _ = _boundary_keys(m)
    # every boundary face is listed exactly once: 4 metal walls and 2 ports, nothing open
    assert len(fv) == len(bkeys) == len(set(map(tuple, fv.tolist())))
    assert set(map(tuple, fv.tolist())) == bkeys
    assert (lab == 0).sum() == (lab == 1).sum() == 2 * 4 * 2
    assert (lab == -1).sum() == 2 * 2 * (4 * 6 + 2 * 6)
    assert np.allclose(ps.a, 0.02) and np.allclose(ps.v, [0, 1, 0]) and np.allclose(ps.u, [1, 0, 0])
    z = m.xyz[fv[lab == 1]][:, :, 2]
    assert np.allclose(z, 0.03)


def test_port_chamber_geometry():
    m = kuhn_mesh(20, 16, 8, lo=(-0.05, -0.04, -0.02), hi=(0.05, 0.04, 0.02))
    fv, lab, ps, guide = port_chamber(m, (0, 2, 3, 1), a_cells=3, b_cells=2, depth=2)
    bkeys, allkeys = _boundary_keys(m)
    listed = list(map(tuple, fv.tolist()))
    assert len(listed) == len(set(listed))                         # no face listed twice
    assert set(listed) <= allkeys                                   # all are mesh faces
    assert ps.n == 6 and np.array_equal(np.unique(lab[lab >= 0]), np.arange(6))
    for p in range(6):
        pf = fv[lab == p]
        assert len(pf) == 3 * 2 * 2                                  # a_cells x b_cells x 2 triangles
        assert set(map(tuple, pf.tolist())) <= bkeys                 # ports sit on the boundary
        P = m.xyz[pf].reshape(-1, 3)
        s = (P - ps.origin[p]) @ ps.u[p]
        assert s.min() > -1e-12 and s.max() < ps.a[p] + 1e-12       # inside the aperture
        assert np.allclose(ps.v[p], [0, 0, 1])
    # the x = lo wall has no guides and stays open; the other side walls are metal around the ports
    xlo = set(map(tuple, faces_on_plane(m, 0, -0.05, (-0.04, -0.02), (0.04, 0.02)).tolist()))
    assert not (xlo & set(listed))
    xhi = set(map(tuple, faces_on_plane(m, 0, 0.05, (-0.04, -0.02), (0.04, 0.02)).tolist()))
    assert xhi <= set(listed)
    # guide volume: ports x a_cells x b_cells x depth cells of 6 tets; interior metal sheets exist
    assert guide.sum() == 6 * 3 * 2 * 2 * 6
    interior_metal = set(map(tuple, fv[lab == -1].tolist())) - bkeys
    assert len(interior_metal) > 0
