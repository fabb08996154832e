"""Batched polarizability workload: configuration buckets, mesh autotuning and
sharding across processes.

Host orchestration around ``induced_charge_solve_batch``; every step of the
arithmetic runs in the library's kernels.  The polarizability tensor of a body
(Sec. II, the dipole S of Eq. rigid_dipole as a linear function of E0) needs
three right-hand sides, E0 = x, y, z; many independent configurations are
solved together so that one set of PME launches serves them all.

* Buckets.  Configurations are grouped by bead count (within a factor
  ``ratio``), and a bucket is cut where its mesh channels (3 x configurations)
  would exceed ``max_channels``.  Each bucket is one batched call on one mesh.
* Autotuner.  For a bucket the mesh is picked from candidate sizes by timing
  the batched solve itself: two short runs (p0 and p1 Krylov iterations) after a
  warm-up give the cost of one iteration and the set-up cost (near-field table,
  plans); the candidate with the least set-up + expected iterations x cost wins.
  Accuracy does not enter the choice: every candidate meets the same Ewald
  tolerance (Sec. III.D.2: xi follows the mesh, r_c and P follow tol).  Results
  are cached in a JSON file keyed by GPU, bucket shape, precision and tolerance.
* Sharding.  Configurations are independent, so processes take disjoint sets,
  assigned longest-processing-time first on the cost model N P^3 + G log G
  (spread/gather plus FFT); the only exchange is a host gather of the tensors.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

MESH_CANDIDATES = (64, 96, 128, 160, 192)


# ---------------------------------------------------------------- bucketing

def buckets(sizes, ratio: float = 2.0, max_channels: int = 192, nrhs: int = 3, classes=None) -> list[list[int]]:
    """Indices of configurations grouped by bead count: sorted ascending, a new
    bucket starts when the count exceeds ``ratio`` x the bucket's first, or when
    the bucket would hold more than max_channels / nrhs configurations.
    Configurations of different ``classes`` (e.g. whether the body-block
    preconditioner covers them, which sets how fast they converge) never share a
    bucket: a batched solve iterates until its slowest system converges."""
    cls = list(classes) if classes is not None else [0] * len(sizes)
    order = sorted(range(len(sizes)), key=lambda i: (cls[i], sizes[i], i))
    per = max(1, max_channels // max(1, nrhs))
    out: list[list[int]] = []
    for i in order:
        if (out and cls[i] == cls[out[-1][0]] and sizes[i] <= ratio * sizes[out[-1][0]]
                and len(out[-1]) < per):
            out[-1].append(i)
        else:
            out.append([i])
    return out


PRECOND_MAX_BEADS = 8192   # bodies the library's body-block preconditioner covers


def preconditioned(system) -> int:
    """1 if every multi-bead body of the configuration is small enough for the
    body-block preconditioner (the whole configuration is then preconditioned)."""
    sizes = np.diff(np.asarray(system.body_offsets))
    return int(np.all(sizes[sizes > 1] <= PRECOND_MAX_BEADS))


def cost_model(n_beads: int, mesh: int = 128, P: int = 9, nrhs: int = 3) -> float:
    """Relative cost of one PME evaluation: stencil work N P^3 plus FFT G log2 G, per field."""
    G = float(mesh) ** 3
    return nrhs * (n_beads * P ** 3 + G * math.log2(G))


def shard_lpt(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of independent items to `world`
    ranks: each item, largest first, goes to the least-loaded rank (ties: lower
    rank).  Deterministic, so every rank computes the same plan."""
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += costs[i]
    for o in out:
        o.sort()
    return out


# ---------------------------------------------------------------- solving

def _stack(systems):
    x = np.concatenate([s.x for s in systems])
    offs, cfg, base = [0], [0], 0
    for s in systems:
        offs.extend((np.asarray(s.body_offsets[1:]) + base).tolist())
        base += s.n
        cfg.append(cfg[-1] + s.n_bodies)
    X = np.concatenate([s.X for s in systems])
    Q = np.concatenate([s.Q for s in systems])
    return np.ascontiguousarray(x), np.asarray(offs, np.int32), X, Q, np.asarray(cfg, np.int32)


class Bucket:
    """Device-resident inputs and outputs of one batched call."""

    def __init__(self, ib, systems, E0):
        import torch
        self.ib = ib
        self.systems = systems
        x, offs, X, Q, cfg = _stack(systems)
        self.cfg = cfg
        self.n, self.nb = x.shape[0], X.shape[0]
        self.R = E0.shape[0]
        dev = "cuda"
        self.x = torch.as_tensor(x, device=dev)
        self.offs = torch.as_tensor(offs, device=dev)
        self.X = torch.as_tensor(X, device=dev)
        self.Q = torch.as_tensor(Q, device=dev)
        self.E0 = torch.as_tensor(np.ascontiguousarray(E0, dtype=np.float64), device=dev)
        self.bodies = ib.Bodies(self.offs, self.X, self.Q)
        self.q = torch.zeros((self.R, self.n), dtype=torch.float64, device=dev)
        self.S = torch.zeros((self.R, self.nb, 3), dtype=torch.float64, device=dev)

    def solve(self, ctx, opts):
        return self.ib.induced_charge_solve_batch(ctx, self.n, self.x, self.bodies, self.cfg, self.E0, self.R,
                                                  opts, self.q, None, self.S)

    def shifted_positions(self, rng):
        """(x, X) on the device with every configuration translated rigidly by its
        own uniform random vector in the box.  In a periodic box a translation
        changes no potential, charge or dipole, but every position-dependent table
        (cells, pair table, stencils) has to be built again."""
        import torch
        x, X = [], []
        for s in self.systems:
            d = rng.uniform(0.0, 1.0, size=3) * np.asarray(s.box, dtype=np.float64)
            x.append(np.mod(s.x + d, s.box))
            X.append(np.mod(s.X + d, s.box))
        return (torch.as_tensor(np.ascontiguousarray(np.concatenate(x)), device="cuda"),
                torch.as_tensor(np.ascontiguousarray(np.concatenate(X)), device="cuda"))

    def load_positions(self, x, X):
        self.x.copy_(x)
        self.X.copy_(X)


def context_for(ib, box, mesh, tol, a, eps, precision, nrhs):
    return ib.pme_setup(ib.make_params(box=box, mesh=[mesh] * 3, tol=tol, bead_radius=a, eps_f=eps,
                                       precision=precision, max_rhs=nrhs))


# ---------------------------------------------------------------- autotuner

def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:   # no CUDA: the key still works for a cache file read on the host
        return "unknown"


class Autotuner:
    """Mesh choice per bucket, measured on the device and cached in JSON."""

    def __init__(self, cache_path: str | None = None, candidates=MESH_CANDIDATES, probe=(3, 9),
                 expected_iters: int = 30):
        self.path = cache_path or os.environ.get("IBPME_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "ibpme", "autotune.json")
        self.candidates = tuple(candidates)
        self.probe = probe
        self.expected_iters = expected_iters
        self.cache = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def key(self, n_beads, n_configs, nrhs, precision, tol, box, a) -> str:
        nb = 1 << max(0, int(round(math.log2(max(1, n_beads)))))   # bead count to the nearest power of 2
        return json.dumps([_gpu_name(), nb, int(n_configs), int(nrhs), int(precision), float(tol),
                           [round(float(b), 6) for b in box], round(float(a), 6), list(self.candidates)])

    def save(self):
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1)
        os.replace(tmp, self.path)

    def measure(self, ib, bucket: Bucket, mesh, tol, a, eps, precision) -> dict | None:
        """Set-up and per-iteration cost of the batched solve on one mesh (None if
        the mesh cannot serve this tolerance in this box)."""
        box = bucket.systems[0].box
        try:
            ctx = context_for(ib, box, mesh, tol, a, eps, precision, bucket.R)
        except ib.IbpmeError:
            return None
        try:
            p0, p1 = self.probe
            t_first = time.perf_counter()
            bucket.solve(ctx, ib.make_opts(max_iter=p0))          # builds tables, plans, graphs
            t_first = time.perf_counter() - t_first
            runs = []
            for p in (p0, p1):
                t = time.perf_counter()
                _, st = bucket.solve(ctx, ib.make_opts(max_iter=p))
                runs.append((time.perf_counter() - t, st[0].iters))
            (ta, ia), (tb, ib_) = runs
            setup = max(0.0, t_first - ta)
            if ib_ > ia:
                # timing noise can make the longer probe no slower: then its own time per iteration
                per_iter = (tb - ta) / (ib_ - ia) if tb > ta else tb / ib_
                predicted = setup + ta + max(0, self.expected_iters - ia) * per_iter
            else:   # converged within the shorter probe: that run is the whole solve
                per_iter = ta / max(1, ia)
                predicted = setup + ta
            return dict(mesh=mesh, per_iter_ms=1e3 * per_iter, setup_ms=1e3 * setup, base_ms=1e3 * ta,
                        predicted_ms=1e3 * predicted)
        finally:
            ib.pme_destroy(ctx)

    def tune(self, ib, bucket: Bucket, tol, a, eps, precision) -> tuple[int, list[dict]]:
        key = self.key(bucket.n, len(bucket.systems), bucket.R, precision, tol, bucket.systems[0].box, a)
        if key in self.cache:
            return int(self.cache[key]["mesh"]), self.cache[key]["report"]
        report = [m for m in (self.measure(ib, bucket, N, tol, a, eps, precision) for N in self.candidates)
                  if m is not None]
        if not report:
            raise RuntimeError("no candidate mesh serves this tolerance in this box")
        best = min(report, key=lambda m: m["predicted_ms"])
        self.cache[key] = dict(mesh=best["mesh"], report=report)
        try:
            self.save()
        except OSError:
            pass   # a read-only cache location only costs re-tuning
        return best["mesh"], report


# ---------------------------------------------------------------- driver

def polarizability(ib, systems, precision=None, rtol=1e-6, tol=1e-6, tuner: Autotuner | None = None,
                   mesh: int | None = None, ratio=1.6, max_channels=192):
    """Polarizability tensors of every body of every configuration.

    systems: configurations sharing box, bead radius and permittivity (their E0
    is ignored: the fields are x, y, z).  Returns (tensors, report) with
    tensors[k] of shape [n_bodies_k, 3, 3], P[b, i, j] = S_i of body b for E0 = e_j,
    and report a list of per-bucket dicts (mesh, configurations, beads,
    iterations, residuals, time)."""
    import torch
    if precision is None:
        precision = ib.IBPME_MIXED
    E0 = np.eye(3)
    a, eps = systems[0].a, systems[0].eps
    out = [None] * len(systems)
    report = []
    for idx in buckets([s.n for s in systems], ratio=ratio, max_channels=max_channels, nrhs=3,
                       classes=[preconditioned(s) for s in systems]):
        bucket = Bucket(ib, [systems[i] for i in idx], E0)
        N = mesh
        tuned = None
        if N is None:
            tuner = tuner or Autotuner()
            N, tuned = tuner.tune(ib, bucket, tol, a, eps, precision)
        ctx = context_for(ib, systems[0].box, N, tol, a, eps, precision, 3)
        try:
            t = time.perf_counter()
            status, st = bucket.solve(ctx, ib.make_opts(rtol=rtol))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
        finally:
            ib.pme_destroy(ctx)
        S = bucket.S.cpu().numpy()                       # [3 fields][bodies][3 components]
        for k, i in enumerate(idx):
            lo, hi = bucket.cfg[k], bucket.cfg[k + 1]
            out[i] = np.transpose(S[:, lo:hi, :], (1, 2, 0)).copy()   # [body][component][field]
        report.append(dict(configs=idx, mesh=N, beads=bucket.n, status=status, iters=st[0].iters,
                           worst_residual=max(e.rel_residual for e in st), seconds=dt, tuning=tuned))
    return out, report


def polarizability_sharded(ib, systems, group=None, solve=None, **kw):
    """Polarizability tensors of one batch split across the ranks of a
    torch.distributed group: configurations are assigned longest processing time
    first on cost_model (shard_lpt), every rank solves its share with
    polarizability(ib, share, **kw) (bucketed and autotuned on its own GPU), and the
    tensors are gathered on rank 0 in configuration order over the host (no device
    collective).  solve(share) -> (tensors, report) replaces that call (tests).
    Returns (tensors, this rank's bucket report) on rank 0, (None, report) elsewhere."""
    solve = solve or (lambda part: polarizability(ib, part, **kw))
    report = []

    def solve_share(part):
        out, rep = solve(part)
        report.extend(rep)
        return out

    tensors = run_sharded(systems, [cost_model(s.n) for s in systems], solve_share, group=group)
    return tensors, report


def run_sharded(items, costs, solve_fn, group=None):
    """Solve independent items on every rank of a torch.distributed group and
    gather the results on rank 0 (host objects; no device collective).

    solve_fn(list of items) -> list of results, one per item.  Returns the
    results in item order on rank 0 and None elsewhere."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    plan = shard_lpt(costs, world)
    mine = plan[rank]
    res = list(solve_fn([items[i] for i in mine])) if mine else []
    if len(res) != len(mine):
        raise RuntimeError("solve_fn must return one result per item")
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((mine, res), gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = [None] * len(items)
    for idx, r in gathered:
        for i, v in zip(idx, r):
            out[i] = v
    return out
