"""Failure paths of the C ABI, all made on the host side: an iteration limit too
small to converge, and body structures that break the CSR rules of the bodies
argument (empty body, offsets past n, not starting at 0, decreasing).

A solve that hits max_iter returns IBPME_ERR_NOT_CONVERGED with its last iterate
written (charges and body potentials) and its statistics filled; the residual the
statistics report is the residual of the written iterate, checked here with the
oracle's dense saddle matrix.  The fused BD step then writes the charges and leaves
forces and positions untouched.  Bad offsets are rejected with IBPME_ERR_ARG before
any kernel runs, and the context stays usable.
"""
import numpy as np
import pytest

import oracle as o
from helpers import context, cuda
from workloads import configs as C

pytestmark = pytest.mark.gpu


def _system():
    return C.small_system(seed=41, n_bodies=2, level=2, n_ions=12, L=8.0, a=0.14, mesh=(48, 48, 48), tol=1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_limit_returns_not_converged_with_the_last_iterate(cuda_lib, prec):
    import torch
    ib = cuda_lib
    s = _system()
    ctx = context(ib, s, precision=prec)
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        q = torch.full((1, s.n), 123.0, dtype=torch.float64, device="cuda")
        psi = torch.full((1, s.n_bodies), 123.0, dtype=torch.float64, device="cuda")
        opts = ib.make_opts(rtol=1e-12, max_iter=2, precond=ib.IBPME_PRECOND_NONE)
        status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0[:1]), 1, opts, q, psi)
        torch.cuda.synchronize()
        assert status == ib.IBPME_ERR_NOT_CONVERGED
        assert "not converged" in ib.last_error()
        assert st.iters == 2 and np.isfinite(st.rel_residual) and 1e-12 < st.rel_residual < 1.0
        assert st.matvecs_fp64 >= 1 and st.outer >= 1
        qh, ph = q.cpu().numpy()[0], psi.cpu().numpy()[0]
        assert not np.any(qh == 123.0) and not np.any(ph == 123.0)   # every output written
        # ions keep their charges; every body carries its net charge up to the iterate's error
        n_body = int(s.body_offsets[2])
        assert np.array_equal(qh[n_body:], s.Q[2:])
        # the reported residual is the written iterate's (oracle's dense saddle system)
        M = o.M_dense(s.x, s.box, s.a, s.eps)
        A = o.saddle_matrix(M, s.body_offsets)
        b = o.saddle_rhs(s.x, s.X, s.body_offsets, s.Q, s.E0[0], s.box)
        res = np.linalg.norm(b - A @ np.concatenate([qh, ph])) / np.linalg.norm(b)
        assert abs(res - st.rel_residual) < 1e-3 * st.rel_residual + 1e-7, (res, st.rel_residual)
    finally:
        ib.pme_destroy(ctx)


def test_bd_advance_not_converged_moves_nothing(cuda_lib):
    import torch
    ib = cuda_lib
    s = _system()
    n, nb = s.n, s.n_bodies
    ctx = context(ib, s, precision="mixed")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        full = lambda *shape: torch.full(shape, -7.0, dtype=torch.float64, device="cuda")
        q, F, L, xo, Xo = full(1, n), full(nb, 3), full(nb, 3), full(n, 3), full(nb, 3)
        opts = ib.make_opts(rtol=1e-12, max_iter=2, precond=ib.IBPME_PRECOND_NONE)
        status, st = ib.ibpme_bd_advance(ctx, n, cuda(s.x), bodies, cuda(s.E0[0]), opts, q[0], 1e-3, 1.0, 1.0, 3, 0,
                                         F, L, xo, Xo)
        torch.cuda.synchronize()
        assert status == ib.IBPME_ERR_NOT_CONVERGED and st.iters == 2
        assert not np.any(q.cpu().numpy() == -7.0)
        for t in (F, L, xo, Xo):
            assert np.all(t.cpu().numpy() == -7.0)
        # the context still solves the same system to convergence
        status, st = ib.ibpme_bd_advance(ctx, n, cuda(s.x), bodies, cuda(s.E0[0]), ib.make_opts(rtol=1e-8), q[0],
                                         1e-3, 1.0, 1.0, 3, 0, F, L, xo, Xo)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= 1e-8
        assert np.all(np.isfinite(xo.cpu().numpy()))
    finally:
        ib.pme_destroy(ctx)


def test_batch_reports_not_converged_when_one_configuration_misses(cuda_lib):
    import torch
    ib = cuda_lib
    parts = [C.small_system(seed=42, n_bodies=1, level=1, n_ions=0, L=8.0, a=0.14, mesh=(48, 48, 48), tol=1e-8),
             _system()]
    for p in parts:
        p.E0 = np.array([[0.3, -0.2, 1.0]])
    s, cfg = C.stack(parts)
    ctx = context(ib, s, precision="fp64")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        q = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
        opts = ib.make_opts(rtol=1e-12, max_iter=3, precond=ib.IBPME_PRECOND_NONE)
        status, st = ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, cfg, cuda(s.E0[:1]), 1, opts, q)
        torch.cuda.synchronize()
        assert status == ib.IBPME_ERR_NOT_CONVERGED and len(st) == 2
        assert max(e.rel_residual for e in st) > 1e-12 and all(np.isfinite(e.rel_residual) for e in st)
    finally:
        ib.pme_destroy(ctx)


@pytest.mark.parametrize("case", ["empty body", "past n", "not from zero", "decreasing"])
def test_bad_body_offsets_are_rejected(cuda_lib, case):
    import torch
    ib = cuda_lib
    s = _system()
    n = s.n
    off = s.body_offsets.astype(np.int32).copy()
    if case == "empty body":
        off = np.concatenate([off[:2], off[1:2], off[2:]]).astype(np.int32)   # body 1 has no bead
    elif case == "past n":
        off[-1] = n + 3
    elif case == "not from zero":
        off[0] = 1
    else:
        off[1], off[2] = off[2], off[1]
    nb = len(off) - 1
    X = np.zeros((nb, 3))
    Q = np.zeros(nb)
    ctx = context(ib, s, precision="fp64")
    try:
        q = torch.zeros((1, n), dtype=torch.float64, device="cuda")
        with pytest.raises(ib.IbpmeError) as e:
            ib.induced_charge_solve(ctx, n, cuda(s.x), ib.Bodies(cuda(off), cuda(X), cuda(Q)), cuda(s.E0[:1]), 1,
                                    None, q)
        assert e.value.status == ib.IBPME_ERR_ARG
        # the context is still good for a valid call
        good = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        status, st = ib.induced_charge_solve(ctx, n, cuda(s.x), good, cuda(s.E0[:1]), 1, ib.make_opts(rtol=1e-8), q)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK
    finally:
        ib.pme_destroy(ctx)
