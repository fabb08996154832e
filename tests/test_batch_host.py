"""Host logic of the batched polarizability workload (no GPU): bucketing,
longest-processing-time sharding, the sharded run over two gloo ranks, and the
autotuner's choice and cache."""
import os
import socket

import numpy as np
import pytest

from paper_2401_04865_gb300 import batch as B


def test_buckets_group_by_size_and_cap_channels():
    sizes = [500, 40000, 900, 1100, 20000, 700, 2100, 5000]
    out = B.buckets(sizes, ratio=2.0, max_channels=9, nrhs=3)     # at most 3 configurations per bucket
    assert sorted(i for b in out for i in b) == list(range(len(sizes)))
    for b in out:
        assert len(b) <= 3
        s = [sizes[i] for i in b]
        assert max(s) <= 2.0 * min(s)
    # sorted ascending: buckets do not interleave
    bounds = [(min(sizes[i] for i in b), max(sizes[i] for i in b)) for b in out]
    assert all(bounds[k][1] <= bounds[k + 1][0] for k in range(len(bounds) - 1))


def test_shard_lpt_covers_balances_and_is_deterministic():
    rng = np.random.default_rng(0)
    costs = list(np.exp(rng.uniform(np.log(500), np.log(40000), size=64)))
    for world in (1, 2, 3, 8):
        plan = B.shard_lpt(costs, world)
        assert sorted(i for p in plan for i in p) == list(range(64))
        loads = [sum(costs[i] for i in p) for p in plan]
        # LPT bound: makespan <= (4/3 - 1/(3 m)) OPT, and OPT >= max(mean load, largest item)
        opt_lb = max(sum(costs) / world, max(costs))
        assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * world)) * opt_lb + 1e-9
        assert plan == B.shard_lpt(costs, world)
    # a single huge item sits alone
    assert B.shard_lpt([100.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        items = list(range(10))
        costs = [float(1 + (i * 7) % 5) for i in items]
        # each rank records what it solved; the result of item i is (i, i^2, solving rank)
        res = B.run_sharded(items, costs, lambda xs: [(x, x * x, rank) for x in xs])
        if rank == 0:
            np.save(out_path, np.array(res))
        else:
            assert res is None
    finally:
        dist.destroy_process_group()


def test_run_sharded_gathers_every_item_in_order_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    assert res.shape == (10, 3)
    assert list(res[:, 0]) == list(range(10)) and list(res[:, 1]) == [i * i for i in range(10)]
    costs = [float(1 + (i * 7) % 5) for i in range(10)]
    plan = B.shard_lpt(costs, 2)
    for r in (0, 1):
        assert sorted(np.nonzero(res[:, 2] == r)[0].tolist()) == plan[r]


def _moment_tensors(systems):
    """A stand-in for the solve of each configuration: per body, the second moment
    sum_j r_j r_j^T of its beads about their centroid (geometry only)."""
    out = []
    for s in systems:
        off = s.body_offsets
        T = np.zeros((s.n_bodies, 3, 3))
        for b in range(s.n_bodies):
            r = s.x[off[b]:off[b + 1]] - s.X[b]
            T[b] = r.T @ r
        out.append(T)
    return out


def _pol_rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from workloads import configs as C
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        systems = C.config4_batch(n_configs=8, seed=1003, common_radius=True)
        solved = []

        def stub(part):
            solved.extend(s.name for s in part)
            return _moment_tensors(part), [dict(configs=len(part), beads=int(sum(s.n for s in part)))]

        tensors, report = B.polarizability_sharded(None, systems, solve=stub)
        names = [None] * world
        dist.all_gather_object(names, solved)
        if rank == 0:
            np.save(out_path, np.concatenate([t.ravel() for t in tensors]))
            np.save(out_path + ".plan.npy", np.array([len(n) for n in names]))
        else:
            assert tensors is None
        assert report and report[0]["configs"] == len(solved)
    finally:
        dist.destroy_process_group()


def test_polarizability_batch_sharded_over_two_gloo_ranks_equals_one_rank(tmp_path):
    """The 8-configuration prefix of the batched polarizability workload (real
    configurations of rods, cubes and ellipsoids) split over two gloo ranks with
    shard_lpt and gathered with run_sharded: rank 0 receives every configuration's
    tensors in configuration order, equal to one rank solving all of them, and the
    split follows the LPT plan of the cost model."""
    import torch.multiprocessing as mp
    from workloads import configs as C
    out = str(tmp_path / "pol.npy")
    mp.spawn(_pol_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    systems = C.config4_batch(n_configs=8, seed=1003, common_radius=True)
    want = np.concatenate([t.ravel() for t in _moment_tensors(systems)])
    assert np.array_equal(np.load(out), want)
    plan = B.shard_lpt([B.cost_model(s.n) for s in systems], 2)
    assert list(np.load(out + ".plan.npy")) == [len(p) for p in plan]


class _FakeBucket:
    def __init__(self, n, nconf):
        self.n = n
        self.R = 3
        box = np.array([40.0] * 3)
        self.systems = [type("S", (), {"box": box})() for _ in range(nconf)]


def test_autotuner_picks_the_cheapest_prediction_and_caches(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    t = B.Autotuner(cache_path=path, candidates=(64, 96, 128), expected_iters=30)
    calls = []

    def fake_measure(ib, bucket, mesh, tol, a, eps, precision):
        calls.append(mesh)
        if mesh == 64:
            return None                                  # cannot serve the tolerance
        per_iter = {96: 2.0, 128: 1.5}[mesh]
        setup = {96: 10.0, 128: 40.0}[mesh]
        return dict(mesh=mesh, per_iter_ms=per_iter, setup_ms=setup, base_ms=0.0,
                    predicted_ms=setup + 30 * per_iter)

    monkeypatch.setattr(t, "measure", fake_measure)
    mesh, report = t.tune(None, _FakeBucket(5000, 4), 1e-6, 0.02, 1.0, 1)
    assert mesh == 96 and [r["mesh"] for r in report] == [96, 128] and calls == [64, 96, 128]
    assert os.path.exists(path)
    # a fresh tuner reads the cache and measures nothing
    t2 = B.Autotuner(cache_path=path, candidates=(64, 96, 128))
    monkeypatch.setattr(t2, "measure", lambda *a, **k: pytest.fail("measured despite the cache"))
    assert t2.tune(None, _FakeBucket(5000, 4), 1e-6, 0.02, 1.0, 1)[0] == 96
    # another bucket shape is a different key
    calls.clear()
    monkeypatch.setattr(t2, "measure", fake_measure)
    t2.tune(None, _FakeBucket(40000, 4), 1e-6, 0.02, 1.0, 1)
    assert calls == [64, 96, 128]


def test_buckets_never_mix_classes_and_preconditioned_flag():
    sizes = [500, 600, 700, 800, 900, 1000]
    classes = [1, 0, 1, 0, 1, 0]
    out = B.buckets(sizes, ratio=1e9, max_channels=192, nrhs=3, classes=classes)
    assert sorted(i for b in out for i in b) == list(range(6))
    for b in out:
        assert len({classes[i] for i in b}) == 1
    assert len(out) == 2
    S = type("S", (), {})
    small, big = S(), S()
    small.body_offsets = np.array([0, 642, 643, 644])      # a sphere and two ions
    big.body_offsets = np.array([0, 642, 642 + 9000])      # a sphere and a 9,000-bead body
    assert B.preconditioned(small) == 1 and B.preconditioned(big) == 0
