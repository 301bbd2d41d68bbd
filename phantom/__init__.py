"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds input generation only: structured Kuhn tetrahedral meshes, the layered
cylindrical "shoulder" phantom and the 12^3 sphere phantom, z-directed dipole rings, seeded
box partitions for the Schwarz preconditioner and the counter-based random generator used for
tear placement and measurement noise.  None of the method's arithmetic (element matrices,
assembly, solves, S-parameters, gradients) lives here.

The paper's anatomical CAD shoulder (Sec. IV-A) and its waveguide array (Sec. III) are not
available, so the phantoms below stand in for them with the same tissue classes, a matching
medium around the body, and a ring of antennas around the arm; the tear is an ellipsoid of
synovial fluid inside the tendon band, as in Sec. IV-A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------
# Counter-based generator: splitmix64 (Steele, Lea, Flood 2014), uniform doubles from the top
# 53 bits, normals by the Box-Muller transform.
# ----------------------------------------------------------------------------------------
_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_open(self) -> float:
        """Uniform double in (0, 1]."""
        return ((self.next_u64() >> 11) + 1) * (1.0 / 9007199254740992.0)

    def normal_pair(self) -> tuple[float, float]:
        u1 = self.uniform_open()
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)

    def normals(self, n: int) -> np.ndarray:
        out = np.empty(n)
        for i in range(0, n, 2):
            a, b = self.normal_pair()
            out[i] = a
            if i + 1 < n:
                out[i + 1] = b
        return out


# ----------------------------------------------------------------------------------------
# Kuhn meshes
# ----------------------------------------------------------------------------------------
@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    lo: tuple
    hi: tuple
    xyz: np.ndarray  # [V, 3] float64, metres
    tets: np.ndarray  # [T, 4] int32, vertex ids in Kuhn path order (not sorted)

    @property
    def n_vert(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_tet(self) -> int:
        return self.tets.shape[0]

    def shape_n(self, d: int) -> int:
        return (self.nx, self.ny, self.nz)[d]

    @property
    def h(self) -> tuple:
        return tuple((self.hi[d] - self.lo[d]) / (self.nx, self.ny, self.nz)[d] for d in range(3))

    def centroids(self) -> np.ndarray:
        return self.xyz[self.tets].mean(axis=1)


# The six axis permutations; tet (p1, p2, p3) walks v000 -> +e_p1 -> +e_p2 -> v111.
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def kuhn_mesh(nx: int, ny: int, nz: int, lo=(-0.06, -0.06, -0.06), hi=(0.06, 0.06, 0.06)) -> Mesh:
    """Box [lo, hi] split into nx*ny*nz cells, each cut into 6 tets along its main diagonal.

    Vertex id = (k*(ny+1) + j)*(nx+1) + i.  Tets are ordered by cell (i fastest, then j, k) and
    within a cell by the permutation table above; each tet lists its vertices in path order.
    """
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel().astype(np.int64)
    j = j.ravel().astype(np.int64)
    k = k.ravel().astype(np.int64)

    def vid(di, dj, dk):
        return ((k + dk) * (ny + 1) + (j + dj)) * (nx + 1) + (i + di)

    tets = np.empty((i.size, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_PERMS):
        off = [0, 0, 0]
        tets[:, t, 0] = vid(*off)
        for s in range(3):
            off[perm[s]] += 1
            tets[:, t, s + 1] = vid(*off)
    return Mesh(nx, ny, nz, tuple(lo), tuple(hi), xyz, tets.reshape(-1, 4).astype(np.int32))


# ----------------------------------------------------------------------------------------
# Dielectric data (relative complex permittivity, e^{i omega t} convention: Im < 0 = loss)
# ----------------------------------------------------------------------------------------
EPS_MATCHING = 44.0 - 20.0j
EPS_SKIN = 41.0 - 16.0j
EPS_FAT = 5.5 - 1.0j
EPS_MUSCLE = 55.0 - 17.0j
EPS_BONE = 12.4 - 2.8j
EPS_TENDON = 45.8 - 13.0j
EPS_FLUID = 68.0 - 35.0j
EPS_SPHERE = 50.0 - 15.0j

# Tissue labels used by the shoulder phantom.
MATCHING, SKIN, FAT, MUSCLE, BONE, TENDON, FLUID = range(7)
LABEL_EPS = {MATCHING: EPS_MATCHING, SKIN: EPS_SKIN, FAT: EPS_FAT, MUSCLE: EPS_MUSCLE,
             BONE: EPS_BONE, TENDON: EPS_TENDON, FLUID: EPS_FLUID}


def eps_to_pairs(eps: np.ndarray) -> np.ndarray:
    """Complex per-tet permittivity -> [T, 2] float64 (re, im)."""
    return np.ascontiguousarray(np.stack([eps.real, eps.imag], axis=1).astype(np.float64))


# ----------------------------------------------------------------------------------------
# Antennas: z-directed dipoles on a ring
# ----------------------------------------------------------------------------------------
def dipole_ring(n: int, rho: float, z: float, center=(0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    ang = 2.0 * np.pi * np.arange(n) / n
    pos = np.stack([center[0] + rho * np.cos(ang), center[1] + rho * np.sin(ang), np.full(n, z)], 1)
    direc = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    return pos, direc


# Antenna-count study: four layers around the arm, two full rings and two half rings (on the
# +x side, away from the torso), split in the proportions 11 : 10 : 6 : 5 of the 32-antenna
# design; each ring starts half an angular pitch after the ring below it.
LAYER_WEIGHTS = (5, 11, 10, 6)                 # bottom to top: half, full, full, half
LAYER_FULL = (False, True, True, False)
LAYER_Z = (-0.03, -0.01, 0.01, 0.03)


def layer_counts(n: int) -> tuple:
    """Antennas per layer: n split in LAYER_WEIGHTS proportions, largest remainders first."""
    w = np.asarray(LAYER_WEIGHTS, dtype=np.float64)
    q = n * w / w.sum()
    c = np.floor(q).astype(int)
    for k in np.argsort(-(q - c), kind="stable")[: n - c.sum()]:
        c[k] += 1
    return tuple(int(v) for v in c)


def antenna_layers(n: int, rho: float = 0.10, center=(0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """z-dipole positions and directions of the n-antenna layered design."""
    pos = []
    shift = 0.0
    for cnt, full, z in zip(layer_counts(n), LAYER_FULL, LAYER_Z):
        span = 2.0 * np.pi if full else np.pi
        start = 0.0 if full else -0.5 * np.pi
        pitch = span / cnt
        ang = start + pitch * (np.arange(cnt) + 0.5 + shift)
        shift = 0.5 - shift
        pos.append(np.stack([center[0] + rho * np.cos(ang), center[1] + rho * np.sin(ang), np.full(cnt, z)], 1))
    pos = np.concatenate(pos)
    return pos, np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))


# ----------------------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------------------
def sphere_phantom(mesh: Mesh, seed: int = 1, radius: float = 0.015,
                   eps_bg: complex = EPS_MATCHING, eps_sph: complex = EPS_SPHERE):
    """Homogeneous box with one sphere; centre uniform in the disc rho <= 20 mm, |z| <= 20 mm."""
    g = SplitMix64(seed)
    r = 0.020 * math.sqrt(g.uniform())
    th = 2.0 * math.pi * g.uniform()
    zc = -0.020 + 0.040 * g.uniform()
    c = np.array([r * math.cos(th), r * math.sin(th), zc])
    cen = mesh.centroids()
    eps = np.full(mesh.n_tet, eps_bg, dtype=np.complex128)
    eps[np.linalg.norm(cen - c, axis=1) <= radius] = eps_sph
    return eps, c


ARM_CENTER = (0.0, 0.0)
ARM_R = 0.05
TORSO_CENTER = (-0.28, 0.0)
TORSO_R = 0.15
SKIN_T = 0.002
FAT_T = 0.003
BONE_R = 0.015
TENDON_RHO = (0.032, 0.042)
TENDON_THETA_DEG = (150.0, 210.0)
TENDON_HALF_Z = 0.030
SHOULDER_LO = (-0.18, -0.18, -0.0765)
SHOULDER_HI = (0.18, 0.18, 0.0765)


@dataclass
class Tear:
    center: tuple
    semi_axes: tuple
    eps: complex


def shoulder_labels(points: np.ndarray, tear: Tear | None = None) -> np.ndarray:
    """Tissue label of each point of the layered cylindrical shoulder phantom."""
    x, y, z = points[:, 0], points[:, 1], points[:, 2]
    rho_a = np.hypot(x - ARM_CENTER[0], y - ARM_CENTER[1])
    rho_t = np.hypot(x - TORSO_CENTER[0], y - TORSO_CENTER[1])
    depth = np.maximum(ARM_R - rho_a, TORSO_R - rho_t)
    lab = np.full(points.shape[0], MATCHING, dtype=np.int32)
    inside = depth > 0
    lab[inside] = MUSCLE
    lab[inside & (depth <= SKIN_T + FAT_T)] = FAT
    lab[inside & (depth <= SKIN_T)] = SKIN
    theta = np.degrees(np.arctan2(y - ARM_CENTER[1], x - ARM_CENTER[0])) % 360.0
    band = ((rho_a >= TENDON_RHO[0]) & (rho_a <= TENDON_RHO[1]) & (theta >= TENDON_THETA_DEG[0])
            & (theta <= TENDON_THETA_DEG[1]) & (np.abs(z) <= TENDON_HALF_Z))
    lab[band & (lab == MUSCLE)] = TENDON
    lab[rho_a <= BONE_R] = BONE
    if tear is not None:
        c, a = np.asarray(tear.center), np.asarray(tear.semi_axes)
        q = (((points - c) / a) ** 2).sum(axis=1) <= 1.0
        lab[q & ((lab == TENDON) | (lab == MUSCLE))] = FLUID
    return lab


def shoulder_eps(mesh: Mesh, tear: Tear | None = None, matching: complex = EPS_MATCHING) -> np.ndarray:
    return shoulder_eps_at(mesh.centroids(), tear, matching)


def study_tear(kind: str) -> Tear:
    """The two tears of the antenna-count study, centred in the tendon band at theta = 180 deg:
    partial (about 1 mL) and large (about 5 mL) ellipsoids of synovial fluid."""
    rho = 0.5 * (TENDON_RHO[0] + TENDON_RHO[1])
    axes = {"partial": (0.005, 0.005, 0.0095), "large": (0.005, 0.012, 0.020)}[kind]
    return Tear((ARM_CENTER[0] - rho, ARM_CENTER[1], 0.0), axes, EPS_FLUID)


def random_tear(seed: int, eps_range=None) -> Tear:
    """Tear centre uniform inside the tendon band, semi-axes uniform in 2-10 mm (volumes from
    about 0.03 to 4 mL, spanning the paper's 1 mL and 5 mL tears), axis aligned; fluid
    permittivity fixed, or uniform in the given (re, im) box."""
    g = SplitMix64(seed)
    rho = TENDON_RHO[0] + (TENDON_RHO[1] - TENDON_RHO[0]) * g.uniform()
    th = math.radians(TENDON_THETA_DEG[0] + (TENDON_THETA_DEG[1] - TENDON_THETA_DEG[0]) * g.uniform())
    zc = -TENDON_HALF_Z + 2.0 * TENDON_HALF_Z * g.uniform()
    axes = tuple(0.002 + 0.008 * g.uniform() for _ in range(3))
    if eps_range is None:
        eps = EPS_FLUID
    else:
        (r0, r1), (i0, i1) = eps_range
        eps = complex(r0 + (r1 - r0) * g.uniform(), -(i0 + (i1 - i0) * g.uniform()))
    return Tear((ARM_CENTER[0] + rho * math.cos(th), ARM_CENTER[1] + rho * math.sin(th), zc), axes, eps)


# ----------------------------------------------------------------------------------------
# Partitions for the overlapping Schwarz preconditioner
# ----------------------------------------------------------------------------------------
def box_partition(mesh: Mesh, parts: tuple, seed: int = 7, jitter: float = 0.25) -> np.ndarray:
    """Tet -> subdomain id from a px*py*pz box grid with seeded uneven cuts.

    Cut positions are the uniform cuts moved by up to +-jitter of a box width, snapped to cell
    boundaries; subdomain id = (bz*py + by)*px + bx.
    """
    g = SplitMix64(seed)
    n = (mesh.nx, mesh.ny, mesh.nz)
    cen = mesh.centroids()
    idx = []
    for d in range(3):
        p = parts[d]
        w = n[d] / p
        cuts = [0]
        for c in range(1, p):
            pos = c * w + jitter * w * (2.0 * g.uniform() - 1.0)
            cuts.append(int(round(min(max(pos, cuts[-1] + 1), n[d] - (p - c)))))
        cuts.append(n[d])
        cell = np.floor((cen[:, d] - mesh.lo[d]) / ((mesh.hi[d] - mesh.lo[d]) / n[d])).astype(np.int64)
        idx.append(np.searchsorted(np.asarray(cuts[1:-1]), cell, side="right"))
    return ((idx[2] * parts[1] + idx[1]) * parts[0] + idx[0]).astype(np.int32)


def add_noise(S: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """S + 10^(-snr/20) |S| (xi + i eta)/sqrt(2), xi, eta ~ N(0,1) from splitmix64/Box-Muller,
    drawn in row-major order of S (xi then eta per entry)."""
    g = SplitMix64(seed)
    flat = S.ravel()
    nrm = g.normals(2 * flat.size).reshape(-1, 2)
    amp = 10.0 ** (-snr_db / 20.0) * np.abs(flat)
    out = flat + amp * (nrm[:, 0] + 1j * nrm[:, 1]) / math.sqrt(2.0)
    return out.reshape(S.shape)


# ----------------------------------------------------------------------------------------
# Waveguide ports: faces of Kuhn meshes and rectangular port apertures
# ----------------------------------------------------------------------------------------
_TET_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


class _PlaneFaces:
    """The distinct tet faces of a Kuhn mesh that lie in a grid plane, grouped by (axis, vertex
    index of the plane), with the integer grid indices of their vertices."""

    def __init__(self, mesh: Mesh):
        V = np.int64(mesh.n_vert)
        fv = np.sort(mesh.tets[:, _TET_FACES].reshape(-1, 3).astype(np.int64), axis=1)
        key = np.unique((fv[:, 0] * V + fv[:, 1]) * V + fv[:, 2])
        fv = np.stack([key // (V * V), (key // V) % V, key % V], axis=1)
        nx1, ny1 = mesh.nx + 1, mesh.ny + 1
        grid = np.stack([fv % nx1, (fv // nx1) % ny1, fv // (nx1 * ny1)], axis=2)     # [F, 3 verts, 3 axes]
        self.groups = {}
        for d in range(3):
            on = (grid[:, 0, d] == grid[:, 1, d]) & (grid[:, 1, d] == grid[:, 2, d])
            idx = np.nonzero(on)[0]
            plane = grid[idx, 0, d]
            order = np.argsort(plane, kind="stable")
            idx, plane = idx[order], plane[order]
            cuts = np.searchsorted(plane, np.arange(mesh.shape_n(d) + 2))
            for q in range(mesh.shape_n(d) + 1):
                sel = idx[cuts[q]:cuts[q + 1]]
                self.groups[(d, q)] = (fv[sel], grid[sel])

    def query(self, axis: int, q: int, rng2) -> np.ndarray:
        """Faces in plane axis = q with all vertices inside the vertex-index ranges rng2 (two
        closed ranges over the other axes, increasing axis order)."""
        fv, g = self.groups.get((axis, q), (np.zeros((0, 3), np.int64), np.zeros((0, 3, 3), np.int64)))
        others = [d for d in range(3) if d != axis]
        ok = np.ones(fv.shape[0], dtype=bool)
        for k, d in enumerate(others):
            ok &= np.all((g[:, :, d] >= rng2[k][0]) & (g[:, :, d] <= rng2[k][1]), axis=1)
        return fv[ok]


def _plane_faces(mesh: Mesh) -> _PlaneFaces:
    pf = getattr(mesh, "_plane_faces", None)
    if pf is None:
        pf = _PlaneFaces(mesh)
        mesh._plane_faces = pf
    return pf


def faces_on_plane(mesh: Mesh, axis: int, value: float, lo2, hi2, tol: float = 1e-9) -> np.ndarray:
    """Sorted vertex triples of the tet faces lying in the plane x[axis] = value with every vertex
    inside the rectangle [lo2, hi2] of the two other axes (in increasing axis order)."""
    lo, hi = np.asarray(mesh.lo), np.asarray(mesh.hi)
    h = (hi - lo) / np.array([mesh.nx, mesh.ny, mesh.nz])
    q = int(round((value - lo[axis]) / h[axis]))
    if abs(lo[axis] + q * h[axis] - value) > tol or q < 0 or q > mesh.shape_n(axis):
        return np.zeros((0, 3), dtype=np.int64)
    others = [d for d in range(3) if d != axis]
    rng2 = [(int(np.ceil((lo2[k] - lo[d]) / h[d] - 1e-9)), int(np.floor((hi2[k] - lo[d]) / h[d] + 1e-9)))
            for k, d in enumerate(others)]
    return _plane_faces(mesh).query(axis, q, rng2)


@dataclass
class PortSet:
    """Rectangular apertures: corner, unit broad-side direction u (width a), unit narrow-side
    direction v, and the permittivity filling each guide."""
    origin: np.ndarray       # [P, 3]
    u: np.ndarray            # [P, 3]
    v: np.ndarray            # [P, 3]
    a: np.ndarray            # [P]
    eps_fill: np.ndarray     # [P] complex

    @property
    def n(self) -> int:
        return self.a.shape[0]


def waveguide_section(cells=(8, 4, 12), a: float = 0.02, b: float = 0.01, length: float = 0.03,
                      eps_fill: complex = 59.0 - 0.0j):
    """Straight rectangular guide [0, a] x [0, b] x [0, length] on a Kuhn mesh: metal side walls,
    port 0 at z = 0 and port 1 at z = length, broad side along x, field along y.
    Returns (mesh, face_vert [n, 3], label [n] (-1 metal, p port), PortSet)."""
    m = kuhn_mesh(*cells, lo=(0.0, 0.0, 0.0), hi=(a, b, length))
    walls = [faces_on_plane(m, 0, 0.0, (0, 0), (b, length)), faces_on_plane(m, 0, a, (0, 0), (b, length)),
             faces_on_plane(m, 1, 0.0, (0, 0), (a, length)), faces_on_plane(m, 1, b, (0, 0), (a, length))]
    p0 = faces_on_plane(m, 2, 0.0, (0, 0), (a, b))
    p1 = faces_on_plane(m, 2, length, (0, 0), (a, b))
    metal = np.concatenate(walls)
    fv = np.concatenate([metal, p0, p1])
    lab = np.concatenate([np.full(len(metal), -1), np.zeros(len(p0), np.int64), np.ones(len(p1), np.int64)])
    ports = PortSet(np.array([[0.0, 0.0, 0.0], [0.0, 0.0, length]]), np.tile([1.0, 0.0, 0.0], (2, 1)),
                    np.tile([0.0, 1.0, 0.0], (2, 1)), np.array([a, a]), np.array([eps_fill, eps_fill]))
    return m, fv, lab.astype(np.int32), ports


EPS_CERAMIC = 59.0 - 0.6j   # filling of the waveguide antennas


def _cell_range_faces(mesh: Mesh, axis: int, idx: int, rng2) -> np.ndarray:
    """Faces on the grid plane axis = idx (a vertex-index plane) covering the cell-index ranges
    rng2 = ((i0, i1), (j0, j1)) of the two other axes (increasing axis order): vertex indices
    i0..i1 and j0..j1."""
    return _plane_faces(mesh).query(axis, idx, rng2)


def _setdiff_rows(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    if b.size == 0:
        return a
    keep = ~(a[:, None, :] == b[None, :, :]).all(axis=2).any(axis=1)
    return a[keep]


def port_chamber(mesh: Mesh, n_per_wall=8, a_cells: int = 5, b_cells: int = 2, depth: int = 4,
                 eps_fill: complex = EPS_CERAMIC):
    """A ring of rectangular waveguide antennas on the side walls of a Kuhn box.

    Each guide is a stub of a_cells x b_cells cells (broad side horizontal along its wall,
    narrow side vertical, centred in z) reaching `depth` cells into the box from its wall, filled
    with eps_fill.  Its four side walls are metal sheets inside the mesh, its back face on the
    box wall is the port, and its front opening is open to the box.  The rest of a wall with
    guides is metal; a wall given 0 guides, the bottom and the top stay open.  Guides are evenly
    spaced along each wall.  n_per_wall: one count for every side wall, or four counts for the
    walls x = lo, x = hi, y = lo, y = hi (ports are numbered in that order).
    Returns (face_vert [n, 3], label [n] (-1 metal, p port), PortSet, guide tet mask [T]).
    """
    counts = (n_per_wall,) * 4 if np.isscalar(n_per_wall) else tuple(n_per_wall)
    n = (mesh.nx, mesh.ny, mesh.nz)
    lo, hi = np.asarray(mesh.lo), np.asarray(mesh.hi)
    h = (hi - lo) / np.array(n)
    z0 = (n[2] - b_cells) // 2
    z1 = z0 + b_cells
    cen = mesh.centroids()
    cell = np.floor((cen - lo) / h).astype(np.int64)
    guide = np.zeros(mesh.n_tet, dtype=bool)
    metal, port_faces, origin, u, width = [], [], [], [], []
    for wall, (ax, side) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        n_w = counts[wall]
        if n_w == 0:
            continue
        t = 1 - ax                                   # horizontal axis along this wall
        wall_idx = 0 if side == 0 else n[ax]
        d0, d1 = (0, depth) if side == 0 else (n[ax] - depth, n[ax])
        # full side wall (cell ranges over the two other axes, increasing axis order)
        full = _cell_range_faces(mesh, ax, wall_idx, ((0, n[t]), (0, n[2])))
        ap = []
        for k in range(n_w):
            c0 = int(round(n[t] * (k + 0.5) / n_w - a_cells / 2))
            c1 = c0 + a_cells
            r_t, r_z = (c0, c1), (z0, z1)
            pf = _cell_range_faces(mesh, ax, wall_idx, (r_t, r_z))
            ap.append(pf)
            port_faces.append(pf)
            # stub side walls (interior metal): t = c0, t = c1 over (depth, z); z = z0, z = z1 over (t, depth)
            for ti in (c0, c1):
                rr = ((d0, d1), r_z)                    # axes (ax, 2): ax < 2 always
                metal.append(_cell_range_faces(mesh, t, ti, rr))
            for zi in (z0, z1):
                rr = [None, None]
                rr[ax] = (d0, d1)
                rr[t] = r_t
                metal.append(_cell_range_faces(mesh, 2, zi, tuple(rr)))
            sel = (cell[:, ax] >= d0) & (cell[:, ax] < d1) & (cell[:, t] >= c0) & (cell[:, t] < c1) & \
                  (cell[:, 2] >= z0) & (cell[:, 2] < z1)
            guide |= sel
            o = lo.copy()
            o[ax] = lo[ax] + wall_idx * h[ax]
            o[t] = lo[t] + c0 * h[t]
            o[2] = lo[2] + z0 * h[2]
            origin.append(o)
            e = np.zeros(3)
            e[t] = 1.0
            u.append(e)
            width.append(a_cells * h[t])
        metal.append(_setdiff_rows(full, np.concatenate(ap)))
    metal = np.unique(np.concatenate(metal), axis=0)
    P = len(port_faces)
    fv = np.concatenate([metal] + port_faces)
    lab = np.concatenate([np.full(len(metal), -1)] + [np.full(len(pf), p) for p, pf in enumerate(port_faces)])
    ports = PortSet(np.array(origin), np.array(u), np.tile([0.0, 0.0, 1.0], (P, 1)), np.array(width),
                    np.full(P, eps_fill, dtype=complex))
    return fv, lab.astype(np.int32), ports, guide


# ----------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mesh: Mesh
    eps: np.ndarray          # complex [T]
    eps_bg: complex
    freqs: tuple
    src_pos: np.ndarray
    src_dir: np.ndarray
    parts: tuple | None = None
    overlap: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def n_src(self) -> int:
        return self.src_pos.shape[0]


def sphere_box(cells: int = 12, seed: int = 1, n_src: int = 8) -> Workload:
    """12^3 Kuhn cells on [-0.06, 0.06]^3 (h = 10 mm), one sphere, 8 dipoles at rho = 50 mm."""
    m = kuhn_mesh(cells, cells, cells)
    eps, c = sphere_phantom(m, seed)
    h = 0.12 / cells
    pos, d = dipole_ring(n_src, 0.05, h / 2 if cells % 2 == 0 else 0.0)
    return Workload(f"sphere_box_{cells}", m, eps, EPS_MATCHING, (1.0e9,), pos, d,
                    extra={"sphere_center": c})


def shoulder(cells=(80, 80, 34), n_src: int = 32, freqs=(1.0e9,), tear: Tear | None = None,
             parts=None, overlap: int = 1, name: str = "shoulder") -> Workload:
    m = kuhn_mesh(*cells, lo=SHOULDER_LO, hi=SHOULDER_HI)
    eps = shoulder_eps(m, tear)
    hz = (SHOULDER_HI[2] - SHOULDER_LO[2]) / cells[2]
    z = hz / 2 if cells[2] % 2 == 0 else 0.0
    pos, d = dipole_ring(n_src, 0.10, z, ARM_CENTER)
    return Workload(name, m, eps, EPS_MATCHING, tuple(freqs), pos, d, parts=parts, overlap=overlap,
                    extra={"tear": tear})


def shoulder_eps_at(points: np.ndarray, tear: Tear | None = None, matching: complex = EPS_MATCHING) -> np.ndarray:
    """Relative permittivity of the shoulder phantom at arbitrary points (complex); `matching`
    fills the medium around the body."""
    lab = shoulder_labels(points, tear)
    eps = np.empty(points.shape[0], dtype=np.complex128)
    for k, v in LABEL_EPS.items():
        eps[lab == k] = matching if k == MATCHING else v
    if tear is not None:
        eps[lab == FLUID] = tear.eps
    return eps


# Region of interest of the learned initialiser: a cell-centred 32^3 grid over the bounding box
# of the tendon band (x, y, z lo; x, y, z hi), where tears occur.
ROI_BOX = (-0.045, -0.025, -0.035, -0.025, 0.025, 0.035)
ROI_GRID = 32


def roi_centres(G: int = ROI_GRID, box=ROI_BOX) -> np.ndarray:
    """Cell centres [G^3][3] of the ROI grid, z slowest, x fastest."""
    lo, hi = np.asarray(box[:3]), np.asarray(box[3:])
    c = [lo[d] + (np.arange(G) + 0.5) * (hi[d] - lo[d]) / G for d in range(3)]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def tear_target_grid(tear: Tear, G: int = ROI_GRID, box=ROI_BOX) -> np.ndarray:
    """Delta eps = eps(injured) - eps(healthy) at the ROI cell centres: [2][G][G][G] (Re, Im)."""
    p = roi_centres(G, box)
    d = shoulder_eps_at(p, tear) - shoulder_eps_at(p, None)
    return np.stack([d.real, d.imag]).reshape(2, G, G, G)
