"""Batched configurations: induced_charge_solve_batch against the FP64 oracle
solving each configuration on its own, against the library's single-system
solve, and against properties that hold at any size.

Independent configurations share the box, so their beads overlap in space:
any leak between them (a real-space pair, a shared mesh channel, a common
k = 0 sum) changes the answer far beyond the bars.
"""
import numpy as np
import pytest

import oracle as o
from workloads import configs as C

from helpers import FP64_RTOL, MIXED_RTOL, context, cuda, rel_err

pytestmark = pytest.mark.gpu


def _configs(E0):
    """Three uneven configurations in L = 9: charged bodies, ions, different sizes."""
    parts = [C.small_system(seed=31, n_bodies=2, level=2, n_ions=10, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7),
             C.small_system(seed=32, n_bodies=1, level=1, n_ions=0, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7),
             C.small_system(seed=33, n_bodies=3, level=1, n_ions=5, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7)]
    for s in parts:
        s.E0 = np.array(E0, dtype=np.float64).reshape(-1, 3)
    return parts


def _batch_solve(ib, ctx, s, cfg, prec=-1, rtol=1e-7, **kw):
    import torch
    R = s.nrhs
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    q = torch.zeros((R, s.n), dtype=torch.float64, device="cuda")
    psi = torch.zeros((R, s.n_bodies), dtype=torch.float64, device="cuda")
    S = torch.zeros((R, s.n_bodies, 3), dtype=torch.float64, device="cuda")
    status, st = ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, cfg, cuda(s.E0), R,
                                               ib.make_opts(rtol=rtol, precision=prec, **kw), q, psi, S)
    torch.cuda.synchronize()
    return status, st, q.cpu().numpy(), psi.cpu().numpy(), S.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle_per_configuration(cuda_lib, prec):
    ib = cuda_lib
    rng = np.random.default_rng(5)
    E0 = rng.normal(size=(3, 3))
    parts = _configs(E0)
    s, cfg = C.stack(parts)
    ctx = context(ib, s, precision=prec)
    try:
        status, st, q, psi, S = _batch_solve(ib, ctx, s, cfg, prec=ib.IBPME_FP64 if prec == "fp64" else -1)
        assert status == ib.IBPME_OK
        assert len(st) == 3 and all(e.rel_residual <= 1e-7 for e in st)
        bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
        b0 = 0
        for k, p in enumerate(parts):
            beads = slice(p.body_offsets[0] + b0, b0 + p.n)
            bods = slice(cfg[k], cfg[k + 1])
            qr, psr = o.solve_dense(p.x, p.body_offsets, p.X, p.Q, p.E0, p.box, p.a, p.eps)
            rel = o.relative_positions(p.x, p.X, p.body_offsets, p.box)
            for r in range(3):
                assert rel_err(q[r, beads], qr[r]) < bar, (k, r, rel_err(q[r, beads], qr[r]))
                pscale = max(np.abs(psr[r]).max(), np.abs(rel @ p.E0[r]).max())
                assert np.abs(psi[r, bods] - psr[r]).max() < bar * pscale, k
                Sr = o.dipoles(p.x, p.X, p.body_offsets, qr[r], p.box)
                assert rel_err(S[r, bods], Sr) < bar, (k, r)
            b0 += p.n
    finally:
        ib.pme_destroy(ctx)


def test_batch_equals_single_solves_and_copies_do_not_interact(cuda_lib):
    """A configuration stacked with an exact copy of itself (every bead on top of
    its twin) and with another configuration gives, per copy, the single-system
    solve's answer."""
    ib = cuda_lib
    E0 = np.eye(3)
    a, b, _ = _configs(E0)
    s, cfg = C.stack([a, b, a])
    ctx = context(ib, s, precision="fp64")
    try:
        status, st, q, psi, S = _batch_solve(ib, ctx, s, cfg, rtol=1e-9)
        assert status == ib.IBPME_OK
        import torch
        singles = []
        for p in (a, b):
            bodies = ib.Bodies(cuda(p.body_offsets.astype(np.int32)), cuda(p.X), cuda(p.Q))
            qs = torch.zeros((3, p.n), dtype=torch.float64, device="cuda")
            ps = torch.zeros((3, p.n_bodies), dtype=torch.float64, device="cuda")
            status1, _ = ib.induced_charge_solve(ctx, p.n, cuda(p.x), bodies, cuda(p.E0), 3,
                                                 ib.make_opts(rtol=1e-9), qs, ps)
            assert status1 == ib.IBPME_OK
            singles.append((qs.cpu().numpy(), ps.cpu().numpy()))
        n0, n1 = a.n, b.n
        for (lo, hi), (blo, bhi), (qs, ps) in [((0, n0), (cfg[0], cfg[1]), singles[0]),
                                               ((n0, n0 + n1), (cfg[1], cfg[2]), singles[1]),
                                               ((n0 + n1, s.n), (cfg[2], cfg[3]), singles[0])]:
            assert rel_err(q[:, lo:hi], qs) < 1e-7
            assert rel_err(psi[:, blo:bhi], ps) < 1e-7
        # the two copies of the same configuration agree with each other to rounding
        assert rel_err(q[:, :n0], q[:, n0 + n1:]) < 1e-9
    finally:
        ib.pme_destroy(ctx)


def test_batch_rejects_bad_configuration_ranges(cuda_lib):
    import torch
    ib = cuda_lib
    E0 = np.eye(3)
    s, cfg = C.stack(_configs(E0)[:2])
    ctx = context(ib, s, precision="fp64")
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    q = torch.zeros((3, s.n), dtype=torch.float64, device="cuda")
    try:
        for bad in ([0, 1], [0, 0, s.n_bodies], [1, s.n_bodies], [0, 2, 1, s.n_bodies]):
            with pytest.raises(ib.IbpmeError) as e:
                ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, bad, cuda(s.E0), 3, None, q)
            assert e.value.status == ib.IBPME_ERR_ARG
        m = ib.ibpme_mlp_create(seed=1)
        try:
            with pytest.raises(ib.IbpmeError) as e:
                ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, cfg, cuda(s.E0), 3,
                                              ib.make_opts(guess=ib.IBPME_GUESS_LEARNED, mlp=m), q)
            assert e.value.status == ib.IBPME_ERR_ARG
        finally:
            ib.ibpme_mlp_destroy(m)
        # the context still serves single solves afterwards
        p = _configs(E0)[1]
        bp = ib.Bodies(cuda(p.body_offsets.astype(np.int32)), cuda(p.X), cuda(p.Q))
        qs = torch.zeros((3, p.n), dtype=torch.float64, device="cuda")
        status, _ = ib.induced_charge_solve(ctx, p.n, cuda(p.x), bp, cuda(p.E0), 3, ib.make_opts(rtol=1e-7), qs)
        assert status == ib.IBPME_OK
    finally:
        ib.pme_destroy(ctx)


def test_polarizability_batch_is_symmetric_and_matches_oracle(cuda_lib):
    """Anisotropic bodies (rods, cubes, ellipsoids) as in the polarizability
    workload, scaled down: 6 configurations of 1-3 bodies with 60-200 beads in
    L = 40, three field directions, mixed precision.  The total polarizability of
    each configuration, P_ij = sum over bodies of S_i for E0 = e_j, is symmetric
    (Sec. II: the induced dipole is the gradient of a quadratic energy in E0), and
    the smallest configuration matches the FP64 oracle."""
    ib = cuda_lib
    parts = C.config4_batch(n_configs=6, seed=77, max_bodies=3, common_radius=True, beads=(60, 200))
    for p in parts:
        p.mesh = (96, 96, 96)
    s, cfg = C.stack(parts)
    ctx = context(ib, s, precision="mixed")
    try:
        status, st, q, psi, S = _batch_solve(ib, ctx, s, cfg, rtol=1e-7)
        assert status == ib.IBPME_OK
        for k in range(len(parts)):
            P = S[:, cfg[k]:cfg[k + 1], :].sum(axis=1).T     # P[i, j]: component i for field j
            assert np.abs(P - P.T).max() < 2e-3 * np.abs(P).max(), (k, P)
            assert np.all(np.linalg.eigvalsh(0.5 * (P + P.T)) > 0)
        k = int(np.argmin([p.n for p in parts]))
        p = parts[k]
        qr, _ = o.solve_dense(p.x, p.body_offsets, p.X, p.Q, p.E0, p.box, p.a, p.eps)
        lo = int(s.body_offsets[cfg[k]])
        for r in range(3):
            assert rel_err(q[r, lo:lo + p.n], qr[r]) < MIXED_RTOL, (r, rel_err(q[r, lo:lo + p.n], qr[r]))
    finally:
        ib.pme_destroy(ctx)


def test_polarizability_driver_autotunes_and_matches_oracle(cuda_lib, tmp_path):
    """The batched polarizability driver: buckets of at most three configurations,
    the mesh of each bucket picked by the autotuner from two candidates (both
    measured, the choice cached), and every body's 3x3 tensor of the smallest
    configuration against the FP64 oracle solving that configuration alone."""
    from paper_2401_04865_gb300 import batch as B
    ib = cuda_lib
    parts = C.config4_batch(n_configs=5, seed=78, max_bodies=2, common_radius=True, beads=(60, 150))
    tuner = B.Autotuner(cache_path=str(tmp_path / "tune.json"), candidates=(64, 96), probe=(2, 5))
    tensors, report = B.polarizability(ib, parts, tuner=tuner, rtol=1e-8, tol=1e-6, max_channels=9)
    assert len(tensors) == 5 and all(t.shape == (p.n_bodies, 3, 3) for t, p in zip(tensors, parts))
    assert sorted(i for rep in report for i in rep["configs"]) == list(range(5))
    for rep in report:
        assert len(rep["configs"]) <= 3 and rep["mesh"] in (64, 96) and rep["status"] == ib.IBPME_OK
        assert {m["mesh"] for m in rep["tuning"]} == {64, 96}
        assert all(m["per_iter_ms"] > 0 for m in rep["tuning"])
    import os
    assert os.path.exists(str(tmp_path / "tune.json"))
    k = int(np.argmin([p.n for p in parts]))
    p = parts[k]
    E0 = np.eye(3)
    qr, _ = o.solve_dense(p.x, p.body_offsets, p.X, p.Q, E0, p.box, p.a, p.eps)
    for j in range(3):
        Sr = o.dipoles(p.x, p.X, p.body_offsets, qr[j], p.box)    # [bodies][3] for E0 = e_j
        assert rel_err(tensors[k][:, :, j], Sr) < MIXED_RTOL, (j, rel_err(tensors[k][:, :, j], Sr))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_free_bead_operator_matches_full_operator(cuda_lib, prec, monkeypatch):
    """Batched configurations through the free-bead operator (each free bead carries
    its configuration) give the solves of the operator over every bead."""
    ib = cuda_lib
    rng = np.random.default_rng(8)
    parts = _configs(rng.normal(size=(2, 3)))
    s, cfg = C.stack(parts)
    res = {}
    for full in (True, False):
        if full:
            monkeypatch.setenv("IBPME_FULL_OPERATOR", "1")
        else:
            monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
        ctx = context(ib, s, precision=prec)
        try:
            status, st, q, psi, S = _batch_solve(ib, ctx, s, cfg, prec=ib.IBPME_FP64 if prec == "fp64" else -1,
                                                 rtol=1e-10)
            assert status == ib.IBPME_OK and all(e.rel_residual <= 1e-10 for e in st)
            res[full] = (q, psi, S)
        finally:
            ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
    assert rel_err(res[False][0], res[True][0]) < 1e-8
    assert rel_err(res[False][2], res[True][2]) < 1e-8
    assert np.abs(res[False][1] - res[True][1]).max() < 1e-8 * max(np.abs(res[True][1]).max(), 1.0)
