"""The five synthetic workloads (seeded; seed = 1000 + index) and small test systems.

Each builder returns a ``System``: bead positions, bodies as CSR offsets into
the bead list (bodies contiguous, ions are one-bead bodies), body reference
points (centroid of the bead centres), net body charges, external fields (one
row per right-hand side), the periodic box, the bead radius, the fluid
permittivity and the mesh/accuracy the library is asked to use.  Units: kT = 1,
gamma = 1, lengths in colloid radii, eps_f = 1/(4 pi l_B).

Only geometry and bookkeeping live here; nothing of the method's arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import geometry as geo


@dataclass
class System:
    name: str
    x: np.ndarray                 # [n,3] bead centres
    body_offsets: np.ndarray      # [n_b+1] int32 CSR offsets
    X: np.ndarray                 # [n_b,3] body reference points
    Q: np.ndarray                 # [n_b] net body charges
    E0: np.ndarray                # [R,3] external fields
    box: np.ndarray               # [3]
    a: float                      # bead radius
    eps: float                    # fluid permittivity eps_f
    mesh: tuple = (64, 64, 64)
    tol: float = 1e-6
    precision: str = "fp64"       # "fp64" or "mixed"
    q_guess: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_bodies(self) -> int:
        return int(self.body_offsets.shape[0] - 1)

    @property
    def nrhs(self) -> int:
        return int(self.E0.shape[0])


def eps_from_bjerrum(l_B: float) -> float:
    """eps_f = 1/(4 pi l_B) with kT = 1."""
    return 1.0 / (4.0 * math.pi * l_B)


def assemble(name, bodies, ions, ion_charges, body_charges, box, a, eps, E0, **kw) -> System:
    """Concatenate rigid bodies (lists of bead arrays) and ions into one System."""
    parts, offsets, X, Q = [], [0], [], []
    for b, qb in zip(bodies, body_charges):
        parts.append(b)
        offsets.append(offsets[-1] + b.shape[0])
        X.append(b.mean(axis=0))
        Q.append(qb)
    ions = np.asarray(ions, dtype=np.float64).reshape(-1, 3)
    ni = ions.shape[0]
    parts.append(ions)
    offsets = np.concatenate([np.asarray(offsets, dtype=np.int64), offsets[-1] + 1 + np.arange(ni)])
    X = np.concatenate([np.asarray(X, dtype=np.float64).reshape(-1, 3), ions])
    Q = np.concatenate([np.asarray(Q, dtype=np.float64), np.asarray(ion_charges, dtype=np.float64).reshape(ni)])
    x = np.concatenate(parts)
    return System(name=name, x=np.ascontiguousarray(x, dtype=np.float64),
                  body_offsets=np.asarray(offsets, dtype=np.int32),
                  X=np.ascontiguousarray(X),
                  Q=Q,
                  E0=np.asarray(E0, dtype=np.float64).reshape(-1, 3),
                  box=np.asarray(box, dtype=np.float64), a=float(a), eps=float(eps), **kw)


def config1(level: int = 2, a: float = 0.1) -> System:
    """Single polarizable sphere (radius 1, icosphere level 2 = 162 beads of radius
    0.1) at the centre of L = 20, E0 = z, no ions, FP64, mesh 64^3, tol 1e-8."""
    L = 20.0
    s = geo.icosphere(level) + L / 2.0
    return assemble("sphere162", [s], [], [], [0.0], [L] * 3, a, 1.0, [[0.0, 0.0, 1.0]],
                    mesh=(64, 64, 64), tol=1e-8, precision="fp64")


def config2(n_pairs: int = 1000, n_counter: int = 50, mesh=(128, 128, 128), seed: int = 1001) -> System:
    """One charged sphere (642 beads, Q = -50) with 2 n_pairs monovalent ions plus
    n_counter counterions, uniform outside r = 1.1 in L = 30; l_B = 0.7,
    bead radius 0.05, mesh 128^3, tol 1e-6, FP32 mesh (mixed)."""
    rng = np.random.default_rng(seed)
    L = 30.0
    c = np.array([L / 2.0] * 3)
    s = geo.icosphere(3) + c
    n_ions = 2 * n_pairs + n_counter
    ions = geo.random_ions(rng, n_ions, [L] * 3, [c], 1.1)
    qi = np.array([1.0] * n_pairs + [-1.0] * n_pairs + [1.0] * n_counter)
    Qb = -float(n_counter)
    sysm = assemble("sphere642_ions", [s], ions, qi, [Qb], [L] * 3, 0.05, eps_from_bjerrum(0.7),
                    [[0.0, 0.0, 0.0]], mesh=tuple(mesh), tol=1e-6, precision="mixed")
    sysm.q_guess = np.concatenate([np.full(s.shape[0], Qb / s.shape[0]), qi])
    return sysm


def config3(n_ions: int = 100_000, per_side: int = 4, mesh=(256, 256, 256), seed: int = 1002) -> System:
    """Simple cubic lattice of per_side^3 spheres (642 beads) at volume fraction 0.1
    with n_ions random monovalent ions (half +1, half -1), E0 = x, mesh 256^3,
    tol 1e-6, mixed precision."""
    rng = np.random.default_rng(seed)
    nb = per_side ** 3
    L = (nb * 4.0 * math.pi / 3.0 / 0.1) ** (1.0 / 3.0)
    sp = L / per_side
    centres = [np.array([(i + 0.5) * sp, (j + 0.5) * sp, (k + 0.5) * sp])
               for i in range(per_side) for j in range(per_side) for k in range(per_side)]
    base = geo.icosphere(3)
    bodies = [base + c for c in centres]
    ions = geo.random_ions(rng, n_ions, [L] * 3, centres, 1.1)
    qi = np.array([1.0] * (n_ions // 2) + [-1.0] * (n_ions - n_ions // 2))
    return assemble("sc64_ions", bodies, ions, qi, [0.0] * nb, [L] * 3, 0.05, eps_from_bjerrum(0.7),
                    [[1.0, 0.0, 0.0]], mesh=tuple(mesh), tol=1e-6, precision="mixed")


def _random_body(rng, beads=(500, 5000)):
    """One anisotropic body: spherocylinder rod (aspect 2-6), cube, or ellipsoid
    (semi-axis ratios in [1, 3]) with beads[0]-beads[1] beads (log-uniform)."""
    n = int(round(math.exp(rng.uniform(math.log(beads[0]), math.log(beads[1])))))
    kind = rng.integers(3)
    if kind == 0:
        p = geo.spherocylinder(n, rng.uniform(2.0, 6.0))
    elif kind == 1:
        p = geo.cube(n)
    else:
        p = geo.ellipsoid(n, [1.0, rng.uniform(1.0, 3.0), rng.uniform(1.0, 3.0)])
    return p @ geo.random_rotation(rng).T


def stack(systems: list[System], name: str = "batch") -> tuple[System, np.ndarray]:
    """Concatenate independent configurations that share box, bead radius,
    permittivity and fields into one bead list; returns the stacked System and
    cfg_bodies, the body offsets of the configurations ([n_configs + 1])."""
    s0 = systems[0]
    for s in systems[1:]:
        if not (np.array_equal(s.box, s0.box) and s.a == s0.a and s.eps == s0.eps
                and np.array_equal(s.E0, s0.E0)):
            raise ValueError("stacked configurations must share box, bead radius, eps and E0")
    x = np.concatenate([s.x for s in systems])
    offs, cfg, base = [0], [0], 0
    for s in systems:
        offs.extend((s.body_offsets[1:] + base).tolist())
        base += s.n
        cfg.append(cfg[-1] + s.n_bodies)
    out = System(name=name, x=np.ascontiguousarray(x), body_offsets=np.asarray(offs, dtype=np.int32),
                 X=np.concatenate([s.X for s in systems]), Q=np.concatenate([s.Q for s in systems]),
                 E0=s0.E0.copy(), box=s0.box.copy(), a=s0.a, eps=s0.eps, mesh=s0.mesh, tol=s0.tol,
                 precision=s0.precision)
    return out, np.asarray(cfg, dtype=np.int32)


def config4_batch(n_configs: int = 64, seed: int = 1003, max_bodies: int = 8,
                  common_radius: bool = False, beads=(500, 5000)) -> list[System]:
    """Independent configurations of 1-max_bodies anisotropic bodies in L = 40,
    random orientations, non-overlapping bounding spheres, Q = 0, three field
    directions; bead radius 0.45 x the configuration's minimum bead spacing, or,
    with common_radius, 0.45 x the smallest minimum spacing of the whole batch
    (one radius for configurations solved in one batched call)."""
    rng = np.random.default_rng(seed)
    L = 40.0
    out = []
    for c in range(n_configs):
        nb = int(rng.integers(1, max_bodies + 1))
        bodies, centres, radii = [], [], []
        for _ in range(nb):
            p = _random_body(rng, beads)
            rad = float(np.sqrt((p * p).sum(axis=1)).max())
            for _try in range(1000):
                cen = rng.uniform(rad, L - rad, size=3)
                if all(np.linalg.norm(cen - c2) > rad + r2 + 0.5 for c2, r2 in zip(centres, radii)):
                    break
            bodies.append(p + cen)
            centres.append(cen)
            radii.append(rad)
        spacing = min(geo.min_spacing(b) for b in bodies)
        out.append(assemble(f"polarizability_{c}", bodies, [], [], [0.0] * nb, [L] * 3,
                            0.45 * spacing, 1.0, np.eye(3), mesh=(128, 128, 128), tol=1e-6,
                            precision="mixed"))
        out[-1].extra["min_spacing"] = spacing
    if common_radius:
        a = 0.45 * min(s.extra["min_spacing"] for s in out)
        for s in out:
            s.a = a
    return out


def config5_trajectory(n_ions: int = 20_000, seed: int = 1004, mesh=(192, 192, 192)) -> System:
    """Eight polarizable spheres (642 beads) at random positions with centre
    separation >= 2.5 in L = 30 and n_ions ions (half +1, half -1), E0 = z,
    mesh 192^3, tol 1e-6, mixed precision."""
    rng = np.random.default_rng(seed)
    L = 30.0
    centres = []
    while len(centres) < 8:
        c = rng.uniform(1.5, L - 1.5, size=3)
        if all(np.linalg.norm(c - d) >= 2.5 for d in centres):
            centres.append(c)
    base = geo.icosphere(3)
    bodies = [base + c for c in centres]
    ions = geo.random_ions(rng, n_ions, [L] * 3, centres, 1.1)
    qi = np.array([1.0] * (n_ions // 2) + [-1.0] * (n_ions - n_ions // 2))
    return assemble("eight_spheres_ions", bodies, ions, qi, [0.0] * 8, [L] * 3, 0.05,
                    eps_from_bjerrum(0.7), [[0.0, 0.0, 1.0]], mesh=tuple(mesh), tol=1e-6,
                    precision="mixed")


def _segment_distance(p, c, axis, half, box):
    """Distance from points p to the segment c +- half axis (minimum image)."""
    d = p - c
    d -= box * np.floor(d / box + 0.5)
    t = np.clip(d @ axis, -half, half)
    return np.linalg.norm(d - t[:, None] * axis[None, :], axis=1)


_ICO3 = geo.icosphere(3)


def warm_start_training(seed: int, L: float = 30.0, mesh=(192, 192, 192), max_ions: int = 20_000) -> System:
    """One training configuration of the learned warm start: 2-8 bodies, each an
    icosphere of radius 1 (642 beads) or a spherocylinder rod (600-900 beads,
    aspect 2-4, radius 0.5-0.8), randomly oriented at random non-overlapping
    positions; a random number (0..max_ions) of +-1 ions at least 2a = 0.1 from every
    bead; a field of uniformly random direction and magnitude uniform in [0.1, 2];
    net body charges 0 (half of the bodies) or uniform in [-3, 3].  Bead radius
    0.05, l_B = 0.7, tol 1e-6, mixed precision: the physics of the eight-sphere
    trajectory."""
    rng = np.random.default_rng(seed)
    box = np.array([L, L, L])
    nb = int(rng.integers(2, 9))
    bodies, placed, Q = [], [], []
    while len(bodies) < nb:
        if rng.random() < 0.5:
            pts, half, rad = _ICO3.copy(), 0.0, 1.0
        else:
            rad, asp = rng.uniform(0.5, 0.8), rng.uniform(2.0, 4.0)
            pts, half = geo.spherocylinder(int(rng.integers(600, 901)), asp, rad), rad * (asp - 1.0)
        rot = geo.random_rotation(rng)
        pts = pts @ rot.T
        axis = rot @ np.array([0.0, 0.0, 1.0])
        for _ in range(500):
            c = rng.uniform(0.0, L, size=3)
            ok = True
            for (c2, _a2, h2, r2) in placed:
                d = c - c2
                d -= box * np.floor(d / box + 0.5)
                if np.linalg.norm(d) < half + rad + h2 + r2 + 0.3:
                    ok = False
                    break
            if ok:
                placed.append((c, axis, half, rad))
                bodies.append(pts + c)
                Q.append(0.0 if rng.random() < 0.5 else float(rng.uniform(-3.0, 3.0)))
                break
        else:
            break   # crowded: keep the bodies placed so far (at least two)
    n_ions = int(rng.integers(0, max_ions + 1))
    # ions anywhere at least 2a from every bead (the hard-sphere rule of the dynamics;
    # the bead shells are permeable, so a trajectory also puts ions inside bodies)
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(np.concatenate(bodies), L), boxsize=L)
    ions = np.zeros((0, 3))
    while ions.shape[0] < n_ions:
        cand = rng.uniform(0.0, L, size=(2 * (n_ions - ions.shape[0]) + 16, 3))
        near = np.zeros(len(cand), dtype=bool)
        for (c, _axis, half, rad) in placed:
            d = cand - c
            d -= box * np.floor(d / box + 0.5)
            near |= np.einsum("ij,ij->i", d, d) < (half + rad + 0.2) ** 2
        ok = np.ones(len(cand), dtype=bool)
        if near.any():
            dist, _ = tree.query(cand[near])
            ok[near] = dist >= 0.1
        ions = np.concatenate([ions, cand[ok]])
    ions = ions[:n_ions]
    qi = np.where(np.arange(n_ions) % 2 == 0, 1.0, -1.0)
    d = rng.normal(size=3)
    E0 = d / np.linalg.norm(d) * rng.uniform(0.1, 2.0)
    return assemble(f"warm_start_{seed}", bodies, ions, qi, Q, [L] * 3, 0.05, eps_from_bjerrum(0.7), [E0],
                    mesh=tuple(mesh), tol=1e-6, precision="mixed")


def small_system(seed: int = 7, n_bodies: int = 2, level: int = 1, n_ions: int = 6, L: float = 8.0,
                 a: float = 0.15, eps: float = 1.0, mesh=(32, 32, 32), tol=1e-8, charged=True,
                 nrhs: int = 1) -> System:
    """A tiny random system for brute-force checks: n_bodies icospheres (radius 1)
    at random non-overlapping centres plus n_ions +-1 ions, random E0."""
    rng = np.random.default_rng(seed)
    centres = []
    while len(centres) < n_bodies:
        c = rng.uniform(1.2, L - 1.2, size=3)
        if all(np.linalg.norm(c - d) >= 2.6 for d in centres):
            centres.append(c)
    base = geo.icosphere(level)
    bodies = [base @ geo.random_rotation(rng).T + c for c in centres]
    ions = geo.random_ions(rng, n_ions, [L] * 3, centres, 1.1) if n_ions else np.zeros((0, 3))
    qi = np.array([(1.0 if i % 2 == 0 else -1.0) for i in range(n_ions)])
    Qb = list(rng.uniform(-2.0, 2.0, size=n_bodies)) if charged else [0.0] * n_bodies
    E0 = rng.normal(size=(nrhs, 3))
    return assemble(f"small_{seed}", bodies, ions, qi, Qb, [L] * 3, a, eps, E0,
                    mesh=tuple(mesh), tol=tol, precision="fp64")


def rocksalt(m: int = 2, d: float = 1.0, a: float = 0.3, eps: float = 1.0) -> System:
    """Rock-salt lattice of (2m)^3 unit charges of alternating sign, spacing d,
    in a cubic periodic box of side 2 m d; every ion is its own body."""
    k = 2 * m
    pts, qs = [], []
    for i in range(k):
        for j in range(k):
            for l in range(k):
                pts.append([i * d, j * d, l * d])
                qs.append(1.0 if (i + j + l) % 2 == 0 else -1.0)
    pts = np.array(pts) + 0.25 * d
    return assemble("rocksalt", [], pts, qs, [], [k * d] * 3, a, eps, [[0.0, 0.0, 0.0]])
