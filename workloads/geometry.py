"""Seeded synthetic geometry for the immersed-boundary workloads.

This module only places points: icosphere tessellations (Sec. III.A of
arXiv:2401.04865), four-line fibers (Sec. IV.D), surface tessellations of
spherocylinders, cubes and ellipsoids, lattices and random ions.  It holds none
of the method's arithmetic (no Ewald sums, no solves) and serves both the
oracle-side tests and the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np


def icosphere(level: int, radius: float = 1.0) -> np.ndarray:
    """Icosphere bead centres (Sec. III.A): the 12 icosahedron vertices, then
    ``level`` rounds of edge bisection with the new points pushed radially onto
    the sphere.  Counts: 12, 42, 162, 642, 2562, 10242 for level 0..5."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    pts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = pts[i] + pts[j]
                pts.append(m / np.linalg.norm(m))
                cache[key] = len(pts) - 1
            return cache[key]

        new_faces = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    return np.array(pts) * radius


def min_spacing(p: np.ndarray) -> float:
    """Smallest centre-to-centre distance among the points (brute force)."""
    best = np.inf
    for i in range(len(p) - 1):
        d = np.sqrt(((p[i + 1:] - p[i]) ** 2).sum(axis=1)).min()
        best = min(best, d)
    return float(best)


def fiber(n_per_line: int, aspect: float, spacing: float) -> np.ndarray:
    """Four parallel lines of beads (Sec. IV.D), centred at the origin along z.
    The four lines sit at the corners of a square of side ``spacing``; the
    fiber length is ``aspect`` times the square's diagonal-ish width."""
    length = (n_per_line - 1) * spacing
    z = np.linspace(-length / 2.0, length / 2.0, n_per_line)
    h = spacing / 2.0
    out = [np.stack([np.full_like(z, sx * h), np.full_like(z, sy * h), z], axis=1)
           for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1))]
    return np.concatenate(out)


def fibonacci_sphere(n: int) -> np.ndarray:
    """n nearly uniform points on the unit sphere (golden-angle spiral)."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def ellipsoid(n: int, axes) -> np.ndarray:
    """~n surface points of an ellipsoid with semi-axes ``axes``, spaced by area:
    points of a dense spiral on the sphere are mapped to the ellipsoid and
    thinned so that the surface density is near uniform."""
    ax = np.asarray(axes, dtype=np.float64)
    # area element of the map sphere -> ellipsoid is proportional to |A^-1 n| det A
    m = 4 * n
    s = fibonacci_sphere(m)
    w = np.sqrt(((s / ax) ** 2).sum(axis=1)) * np.prod(ax)
    cdf = np.cumsum(w) / w.sum()
    pick = np.searchsorted(cdf, (np.arange(n) + 0.5) / n)
    return s[np.clip(pick, 0, m - 1)] * ax


def spherocylinder(n: int, aspect: float, radius: float = 1.0) -> np.ndarray:
    """~n surface points of a spherocylinder (cylinder of length
    2 radius (aspect - 1) with hemispherical caps) along z, near-uniform density."""
    length = 2.0 * radius * (aspect - 1.0)
    area_cyl = 2.0 * math.pi * radius * length
    area_caps = 4.0 * math.pi * radius * radius
    dA = (area_cyl + area_caps) / n
    ds = math.sqrt(dA)
    pts = []
    n_ring = max(3, int(round(2.0 * math.pi * radius / ds)))
    n_z = max(1, int(round(length / ds)))
    for k in range(n_z):
        z = -length / 2.0 + (k + 0.5) * length / n_z
        off = 0.5 * (k % 2)
        th = 2.0 * math.pi * (np.arange(n_ring) + off) / n_ring
        pts.append(np.stack([radius * np.cos(th), radius * np.sin(th), np.full(n_ring, z)], axis=1))
    n_cap = max(1, int(round(area_caps / dA)))
    cap = fibonacci_sphere(2 * (n_cap // 2) or 2) * radius
    top = cap[cap[:, 2] >= 0] + np.array([0.0, 0.0, length / 2.0])
    bot = cap[cap[:, 2] < 0] - np.array([0.0, 0.0, length / 2.0])
    pts += [top, bot]
    return np.concatenate(pts)


def cube(n: int, side: float = 2.0) -> np.ndarray:
    """~n surface points of a cube of the given side, a square grid on each face."""
    m = max(2, int(round(math.sqrt(n / 6.0))))
    g = (np.arange(m) + 0.5) / m * side - side / 2.0
    u, v = np.meshgrid(g, g, indexing="ij")
    u, v = u.ravel(), v.ravel()
    c = np.full_like(u, side / 2.0)
    faces = [np.stack([c, u, v], 1), np.stack([-c, u, v], 1),
             np.stack([u, c, v], 1), np.stack([u, -c, v], 1),
             np.stack([u, v, c], 1), np.stack([u, v, -c], 1)]
    return np.concatenate(faces)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly random rotation matrix (from a uniform unit quaternion)."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ions(rng: np.random.Generator, count: int, box, centres=(), exclusion: float = 0.0) -> np.ndarray:
    """Uniform random points in the box, rejected within ``exclusion`` of any
    centre (minimum image).  Overlaps between the points themselves are allowed."""
    box = np.asarray(box, dtype=np.float64)
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((0, 3))
    while out.shape[0] < count:
        cand = rng.uniform(0.0, 1.0, size=(2 * (count - out.shape[0]) + 16, 3)) * box
        if centres.shape[0]:
            ok = np.ones(cand.shape[0], dtype=bool)
            for c in centres:
                d = cand - c
                d -= box * np.floor(d / box + 0.5)
                ok &= (d * d).sum(axis=1) >= exclusion * exclusion
            cand = cand[ok]
        out = np.concatenate([out, cand])
    return out[:count]
