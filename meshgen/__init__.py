"""Seeded synthetic meshes and right-hand sides for the grid-overlay FD method.

This module holds the inputs only: simplicial meshes shaped like the paper's
test domains (Section 5: unit disk and ball, L-shaped domain, graded meshes)
and the right-hand sides used on them.  It contains none of the method's
arithmetic (no point location, no coefficients, no operator), so that both the
CUDA path and the FP64 oracle can consume the same inputs without sharing code.

Every generator is deterministic for a given seed (``numpy.random.default_rng``)
and returns ``(vertices[N_v, d] float64, simplices[N_e, d+1] int32)`` with every
simplex positively oriented (``flip_orientations`` makes mixed-orientation
copies).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2307_14437


def seed_for(config: int, instance: int = 0) -> int:
    """Seed of a workload: ``2307_14437 + 100*config + instance``."""
    return SEED_BASE + 100 * config + instance


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _signed_volumes(verts: np.ndarray, simp: np.ndarray) -> np.ndarray:
    d = verts.shape[1]
    e = verts[simp[:, 1:]] - verts[simp[:, :1]]          # (N_e, d, d)
    return np.linalg.det(e) / math.factorial(d)


def _orient_positive(verts: np.ndarray, simp: np.ndarray) -> np.ndarray:
    simp = np.array(simp, dtype=np.int64, copy=True)
    vol = _signed_volumes(verts, simp)
    neg = vol < 0
    simp[neg, 0], simp[neg, 1] = simp[neg, 1].copy(), simp[neg, 0].copy()
    return simp.astype(np.int32)


def _delaunay(points: np.ndarray) -> np.ndarray:
    from scipy.spatial import Delaunay
    tri = Delaunay(points)
    return np.asarray(tri.simplices, dtype=np.int64)


def _drop_unused(verts: np.ndarray, simp: np.ndarray):
    used = np.zeros(len(verts), dtype=bool)
    used[simp.ravel()] = True
    remap = -np.ones(len(verts), dtype=np.int64)
    remap[used] = np.arange(used.sum())
    return verts[used], remap[simp]


def flip_orientations(simp: np.ndarray, frac: float = 0.5, seed: int = SEED_BASE) -> np.ndarray:
    """A copy of ``simp`` in which a seeded random ``frac`` of the simplices
    have their first two local vertices swapped (negative orientation): the
    same mesh with mixed orientations and a different local vertex order."""
    simp = np.array(simp, dtype=np.int32, copy=True)
    rng = np.random.default_rng(seed)
    flip = rng.random(len(simp)) < frac
    simp[flip, 0], simp[flip, 1] = simp[flip, 1].copy(), simp[flip, 0].copy()
    return simp


def mesh_volume(verts: np.ndarray, simp: np.ndarray) -> float:
    return float(np.abs(_signed_volumes(verts, simp)).sum())


# ----------------------------------------------------------------------------
# 2D unit disk, ring construction (stand-in for the disk of Example 5.2)
# ----------------------------------------------------------------------------

def disk_ring_mesh(rings: int = 25, jitter: float = 0.2, seed: int = seed_for(1)):
    """Unit disk: a centre node plus rings k=1..rings of 6k nodes at r=k/rings.

    Interior ring nodes get seeded uniform noise of +-jitter*(1/rings) per
    coordinate; the outer ring stays on the unit circle.  Delaunay triangulated.
    rings=25 gives 1951 vertices and 3750 triangles.
    """
    rng = np.random.default_rng(seed)
    pts = [np.zeros((1, 2))]
    dr = 1.0 / rings
    for k in range(1, rings + 1):
        m = 6 * k
        th = 2.0 * np.pi * np.arange(m) / m
        ring = np.stack([k * dr * np.cos(th), k * dr * np.sin(th)], axis=1)
        if k < rings:
            ring = ring + rng.uniform(-jitter * dr, jitter * dr, size=ring.shape)
        pts.append(ring)
    verts = np.concatenate(pts, axis=0)
    simp = _orient_positive(verts, _delaunay(verts))
    return verts.astype(np.float64), simp


def graded_disk_mesh(h_fd: float, c: float = 0.195, floor: float = 1.25,
                     jitter: float = 0.2, seed: int = seed_for(4)):
    """Unit disk graded toward the boundary.

    Ring spacing is ``delta(r) = max(c (1-r)^1.5, floor*h_fd)``; ring k carries
    ``round(2 pi r_k / delta(r_k))`` nodes (at least 6); interior rings are
    jittered by +-jitter*delta.  With h_fd = 2/2047 this gives ~2.1e5 vertices.
    """
    rng = np.random.default_rng(seed)
    radii = [0.0]
    r = 0.0
    while True:
        dlt = max(c * (1.0 - r) ** 1.5, floor * h_fd)
        r = r + dlt
        if r >= 1.0 - 0.5 * floor * h_fd:
            break
        radii.append(r)
    radii.append(1.0)
    # rescale the last gap so that it is not thinner than half a spacing
    pts = [np.zeros((1, 2))]
    for i, rk in enumerate(radii[1:], start=1):
        dlt = max(c * (1.0 - rk) ** 1.5, floor * h_fd)
        dlt = min(dlt, radii[i] - radii[i - 1])
        m = max(6, int(round(2.0 * np.pi * rk / dlt)))
        th = 2.0 * np.pi * (np.arange(m) + 0.5 * (i % 2)) / m
        ring = np.stack([rk * np.cos(th), rk * np.sin(th)], axis=1)
        if i < len(radii) - 1:
            ring = ring + rng.uniform(-jitter * dlt, jitter * dlt, size=ring.shape)
        pts.append(ring)
    verts = np.concatenate(pts, axis=0)
    simp = _orient_positive(verts, _delaunay(verts))
    return verts.astype(np.float64), simp


# ----------------------------------------------------------------------------
# 2D L-shaped domain [-1,1]^2 minus [0,1]^2 (stand-in for Example 5.4)
# ----------------------------------------------------------------------------

_L_CORNERS = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 0.0], [0.0, 0.0],
                       [0.0, 1.0], [-1.0, 1.0]])


def _dist_to_polygon(p: np.ndarray, corners: np.ndarray) -> np.ndarray:
    d = np.full(len(p), np.inf)
    m = len(corners)
    for i in range(m):
        a = corners[i]
        b = corners[(i + 1) % m]
        ab = b - a
        t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
        q = a + t[:, None] * ab
        d = np.minimum(d, np.linalg.norm(p - q, axis=1))
    return d


def _in_L(p: np.ndarray) -> np.ndarray:
    inside_sq = (np.abs(p[:, 0]) < 1.0) & (np.abs(p[:, 1]) < 1.0)
    notch = (p[:, 0] > 0.0) & (p[:, 1] > 0.0)
    return inside_sq & ~notch


def lshape_mesh(spacing: float = 0.0076, jitter: float = 0.2, seed: int = seed_for(2)):
    """L-shaped domain, quasi-uniform jittered triangular lattice.

    Boundary nodes sit unjittered on the six edges; interior lattice nodes are
    jittered by +-jitter*spacing and kept at least 0.5*spacing from the
    boundary.  Delaunay triangulation, then triangles whose centroid lies in
    the notch are dropped.  spacing=0.0076 gives ~6.0e4 vertices.
    """
    rng = np.random.default_rng(seed)
    bnd = []
    m = len(_L_CORNERS)
    for i in range(m):
        a = _L_CORNERS[i]
        b = _L_CORNERS[(i + 1) % m]
        length = float(np.linalg.norm(b - a))
        k = max(1, int(round(length / spacing)))
        t = np.arange(k) / k
        bnd.append(a[None, :] + t[:, None] * (b - a)[None, :])
    bnd = np.concatenate(bnd, axis=0)
    dy = spacing * math.sqrt(3.0) / 2.0
    ny = int(math.ceil(2.0 / dy)) + 1
    nx = int(math.ceil(2.0 / spacing)) + 2
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = -1.0 + (ii + 0.5 * (jj % 2)) * spacing
    y = -1.0 + jj * dy
    lat = np.stack([x.ravel(), y.ravel()], axis=1)
    lat = lat + rng.uniform(-jitter * spacing, jitter * spacing, size=lat.shape)
    keep = _in_L(lat) & (_dist_to_polygon(lat, _L_CORNERS) >= 0.5 * spacing)
    verts = np.concatenate([bnd, lat[keep]], axis=0)
    simp = _delaunay(verts)
    cen = verts[simp].mean(axis=1)
    simp = simp[~((cen[:, 0] > 0.0) & (cen[:, 1] > 0.0))]
    verts, simp = _drop_unused(verts, simp)
    simp = _orient_positive(verts, simp)
    area = mesh_volume(verts, simp)
    if abs(area - 3.0) > 1e-9:
        raise RuntimeError(f"L-shape mesh does not conform: area {area}")
    return verts.astype(np.float64), simp


# ----------------------------------------------------------------------------
# 3D unit ball, Fibonacci shells (stand-in for Example 5.3)
# ----------------------------------------------------------------------------

def _fibonacci_sphere(m: int) -> np.ndarray:
    i = np.arange(m) + 0.5
    z = 1.0 - 2.0 * i / m
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - math.sqrt(5.0)) * np.arange(m)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def ball_shell_mesh(shells: int = 31, jitter: float = 0.2, seed: int = seed_for(3)):
    """Unit ball: centre plus shells k=1..shells of round(4 pi k^2) spiral points.

    Shell radius k/shells; every shell but the outer one is jittered by
    +-jitter/shells per coordinate.  Delaunay tetrahedralised.
    """
    rng = np.random.default_rng(seed)
    pts = [np.zeros((1, 3))]
    dr = 1.0 / shells
    for k in range(1, shells + 1):
        m = max(4, int(round(4.0 * np.pi * k * k)))
        sh = k * dr * _fibonacci_sphere(m)
        if k < shells:
            sh = sh + rng.uniform(-jitter * dr, jitter * dr, size=sh.shape)
        pts.append(sh)
    verts = np.concatenate(pts, axis=0)
    simp = _delaunay(verts)
    vol = np.abs(_signed_volumes(verts, simp))
    simp = simp[vol > 0.0]
    simp = _orient_positive(verts, simp)
    return verts.astype(np.float64), simp


# ----------------------------------------------------------------------------
# structured meshes (special cases used as pins)
# ----------------------------------------------------------------------------

def grid_aligned_mesh(d: int, lo: float, h: float, cells: int, origin_cells: int = 0):
    """The overlay grid itself, split into simplices.

    Vertices are the grid nodes ``lo + (origin_cells + i) h`` for
    i = 0..cells per axis (computed as one multiply and one add), so every mesh
    vertex coincides with an overlay node.  2D: each square split into two
    triangles along its main diagonal; 3D: each cube split into six
    tetrahedra around its main diagonal (Kuhn subdivision).
    """
    m = cells + 1
    idx = np.arange(m)
    coords = lo + (origin_cells + idx).astype(np.float64) * h
    if d == 1:
        verts = coords[:, None]
        simp = np.stack([idx[:-1], idx[1:]], axis=1)
        return verts, _orient_positive(verts, simp)
    if d == 2:
        y, x = np.meshgrid(coords, coords, indexing="ij")
        verts = np.stack([x.ravel(), y.ravel()], axis=1)
        t = []
        for j in range(cells):
            for i in range(cells):
                a = j * m + i
                b, c, e = a + 1, a + m, a + m + 1
                t.append((a, b, e))
                t.append((a, e, c))
        return verts, _orient_positive(verts, np.array(t))
    if d == 3:
        z, y, x = np.meshgrid(coords, coords, coords, indexing="ij")
        verts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
        t = []
        import itertools
        for k in range(cells):
            for j in range(cells):
                for i in range(cells):
                    def v(di, dj, dk):
                        return ((k + dk) * m + (j + dj)) * m + (i + di)
                    for perm in itertools.permutations(range(3)):
                        cur = [0, 0, 0]
                        path = [v(*cur)]
                        for ax in perm:
                            cur[ax] += 1
                            path.append(v(*cur))
                        t.append(path)
        return verts, _orient_positive(verts, np.array(t))
    raise ValueError("d must be 1, 2 or 3")


def interval_mesh(n_cells: int, jitter: float = 0.2, seed: int = SEED_BASE):
    """1D: the interval (-1,1) split into n_cells jittered cells."""
    rng = np.random.default_rng(seed)
    x = np.linspace(-1.0, 1.0, n_cells + 1)
    dx = 2.0 / n_cells
    x[1:-1] += rng.uniform(-jitter * dx, jitter * dx, size=n_cells - 1)
    verts = x[:, None]
    simp = np.stack([np.arange(n_cells), np.arange(1, n_cells + 1)], axis=1)
    return verts, _orient_positive(verts, simp)


# ----------------------------------------------------------------------------
# right-hand sides and random vectors
# ----------------------------------------------------------------------------

def gaussian_bump(points: np.ndarray, centre, width: float = 0.1) -> np.ndarray:
    """exp(-|x-c|^2 / (2 width^2))."""
    c = np.asarray(centre, dtype=np.float64)
    return np.exp(-np.sum((points - c) ** 2, axis=1) / (2.0 * width * width))


def target_bump(points: np.ndarray, centre=(0.3, 0.2), a: float = 20.0) -> np.ndarray:
    """exp(-a |x-c|^2)."""
    c = np.asarray(centre, dtype=np.float64)
    return np.exp(-a * np.sum((points - c) ** 2, axis=1))


def random_vector(n: int, seed: int) -> np.ndarray:
    """Uniform(-1, 1) float64 vector."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def grid_box(d: int, n: int, lo: float = -1.0, hi: float = 1.0):
    """Cube [lo,hi]^d with n nodes per axis: returns (box_lo, box_hi, h)."""
    h = (hi - lo) / (n - 1)
    return np.full(d, lo), np.full(d, hi), h


def grid_points(box_lo, h: float, n: int) -> np.ndarray:
    """Coordinates of all n^d nodes of the grid from box_lo with spacing h,
    in linear order (axis 0 fastest)."""
    lo = np.asarray(box_lo, dtype=np.float64).reshape(-1)
    axes = [lo[a] + h * np.arange(n) for a in range(len(lo))]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1, order="F") for m in mesh], axis=1)


def in_disk(c: np.ndarray) -> bool:
    return float(np.sum(c * c)) < 1.0


def in_lshape(c: np.ndarray) -> bool:
    return bool(_in_L(np.asarray(c, dtype=np.float64).reshape(1, -1))[0])


def rhs_family(points: np.ndarray, k: int, seed: int, width: float = 0.1, inside=None) -> np.ndarray:
    """k right-hand sides (k x len(points)): f = 1, then k-1 Gaussian bumps of
    the given width with seeded centres uniform in the domain (rejection
    sampling in [-1,1]^d against ``inside``; without it, in [-0.5,0.5]^d)."""
    rng = np.random.default_rng(seed)
    d = points.shape[1]
    out = np.empty((k, len(points)))
    out[0] = 1.0
    for j in range(1, k):
        if inside is None:
            c = rng.uniform(-0.5, 0.5, size=d)
        else:
            c = rng.uniform(-1.0, 1.0, size=d)
            while not inside(c):
                c = rng.uniform(-1.0, 1.0, size=d)
        out[j] = gaussian_bump(points, c, width)
    return out


# ----------------------------------------------------------------------------
# the batched workload: 32 meshes (16 disks, 16 L-shapes), 48 instances
# ----------------------------------------------------------------------------

BATCH_ALPHAS = (0.5, 1.0, 1.5)


def batch_instances(seed: int = seed_for(5)):
    """Instance list of the batched workload: 16 ring-disk and 16 L-shape
    meshes with vertex counts log-uniform in [5e3, 1.5e5]; mesh i of each kind
    runs at alpha = BATCH_ALPHAS[i % 3], and the first 8 of each kind also at
    the next alpha in the cycle (32 meshes, 48 instances).  Returns a list of
    dicts {kind, mesh, target_vertices, alpha, seed}."""
    rng = np.random.default_rng(seed)
    out = []
    for kind in ("disk", "lshape"):
        counts = np.exp(rng.uniform(np.log(5e3), np.log(1.5e5), size=16))
        for i, nv in enumerate(counts):
            ms = seed + 1000 * (kind == "lshape") + i
            for rep in ((0, 1) if i < 8 else (0,)):
                out.append({"kind": kind, "mesh": i, "target_vertices": int(nv),
                            "alpha": BATCH_ALPHAS[(i + rep) % 3], "seed": int(ms)})
    return out


def batch_mesh(spec):
    """The mesh of one batch instance (deterministic in spec's kind, target and seed)."""
    nv = spec["target_vertices"]
    if spec["kind"] == "disk":
        rings = max(2, int(round(math.sqrt(nv / 3.0))))
        return disk_ring_mesh(rings=rings, seed=spec["seed"])
    return lshape_mesh(spacing=0.0076 * math.sqrt(60503.0 / nv), seed=spec["seed"])
