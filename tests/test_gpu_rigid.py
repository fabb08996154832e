"""GPU parity of the rigid-body mobility problem (ibpme_rigid_mobility) through the C ABI.

Against the oracle's dense LU of the same saddle system on the periodic RPY mobility
(oracle/rpy_ref.py, pinned in test_oracle_rpy.py): a square of four beads, a twelve-bead
icosahedron and three free beads.  Bars: 1e-5 (FP64) and 1e-3 (mixed) of each output's
largest magnitude; the constraint forces add up to each body's force; single-bead
bodies do not rotate; the body-block preconditioner gives the same solution in fewer
iterations; an iteration limit returns IBPME_ERR_NOT_CONVERGED.
"""
import functools

import numpy as np
import pytest

from oracle import rpy_ref as R
from workloads import geometry as G

from helpers import FP64_RTOL, MIXED_RTOL, cuda, rel_err

pytestmark = pytest.mark.gpu

L, A, MU = 6.0, 0.2, 0.9


def _system():
    c1 = np.array([2.0, 2.2, 3.0])
    sq = np.array([[0.5, 0, 0], [0, 0.5, 0], [-0.5, 0, 0], [0, -0.5, 0]]) @ np.array(
        [[0.8, 0.6, 0.0], [-0.6, 0.8, 0.0], [0.0, 0.0, 1.0]]) + c1
    c2 = np.array([4.1, 3.9, 3.4])
    ico = G.icosphere(0) * 0.7 + c2
    ions = np.array([[0.7, 5.1, 1.0], [3.2, 0.6, 5.2], [5.3, 2.8, 0.9]])
    x = np.vstack([sq, ico, ions])
    off = np.array([0, 4, 16, 17, 18, 19], dtype=np.int32)
    X = np.vstack([c1, c2, ions])
    FL = np.random.default_rng(4).normal(size=(5, 6))
    return x, X, off, FL


@functools.lru_cache(maxsize=1)
def _reference():
    x, X, off, FL = _system()
    M = R.rpy_matrix(x, [L] * 3, A, MU)
    return R.rigid_mobility(x, X, off, [L] * 3, A, FL, MU, M=M)


def _ctx(ib, prec):
    p = {"fp64": ib.IBPME_FP64, "mixed": ib.IBPME_MIXED}[prec]
    return ib.pme_setup(ib.make_params(box=[L] * 3, mesh=(48, 48, 48), tol=1e-8 if prec == "fp64" else 1e-6,
                                       bead_radius=A, precision=p))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rigid_mobility_matches_dense_oracle(cuda_lib, prec):
    import torch
    ib = cuda_lib
    x, X, off, FL = _system()
    Wr, fr = _reference()
    # a mixed context's product (FP32 mesh and real space, atomic spreads) is exact to about
    # 1e-7 and varies at that level from call to call: its solves stop at 1e-6
    rtol = 1e-10 if prec == "fp64" else 1e-6
    ctx = _ctx(ib, prec)
    try:
        bodies = ib.Bodies(cuda(off), cuda(X), cuda(np.zeros(len(X))))
        W = torch.zeros((len(X), 6), dtype=torch.float64, device="cuda")
        f = torch.zeros((len(x), 3), dtype=torch.float64, device="cuda")
        status, st = ib.ibpme_rigid_mobility(ctx, len(x), cuda(x), bodies, cuda(FL), MU, ib.make_opts(rtol=rtol),
                                             W, f)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= rtol and st.iters > 0
        W, f = W.cpu().numpy(), f.cpu().numpy()
        # host buffers give the same answer
        Wh, fh = np.zeros((len(X), 6)), np.zeros((len(x), 3))
        status, _ = ib.ibpme_rigid_mobility(ctx, len(x), np.ascontiguousarray(x), ib.Bodies(off, X, np.zeros(len(X))),
                                            np.ascontiguousarray(FL), MU, ib.make_opts(rtol=rtol), Wh, fh)
        assert status == ib.IBPME_OK
    finally:
        ib.pme_destroy(ctx)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(W[:, :3], Wr[:, :3]) < bar, rel_err(W[:, :3], Wr[:, :3])
    assert rel_err(W[:2, 3:], Wr[:2, 3:]) < bar, rel_err(W[:2, 3:], Wr[:2, 3:])
    assert rel_err(f, fr) < bar, rel_err(f, fr)
    assert np.abs(W[2:, 3:]).max() == 0.0                      # single beads do not rotate
    same = 1e-9 if prec == "fp64" else 1e-4
    if prec == "fp64":   # the body-block preconditioner changes the iterations, not the solution
        ctx = _ctx(ib, prec)
        try:
            Wn = torch.zeros((len(X), 6), dtype=torch.float64, device="cuda")
            status, stn = ib.ibpme_rigid_mobility(ctx, len(x), cuda(x), ib.Bodies(cuda(off), cuda(X),
                                                  cuda(np.zeros(len(X)))), cuda(FL), MU,
                                                  ib.make_opts(rtol=rtol, precond=ib.IBPME_PRECOND_NONE), Wn)
            torch.cuda.synchronize()
            assert status == ib.IBPME_OK and st.iters < stn.iters, (st.iters, stn.iters)
            assert np.abs(Wn.cpu().numpy() - W).max() < 1e-8 * np.abs(W).max()
        finally:
            ib.pme_destroy(ctx)
    for b in range(len(X)):                                     # sum of the constraint forces = F
        assert np.abs(f[off[b]:off[b + 1]].sum(axis=0) - FL[b, :3]).max() < 10 * rtol * np.abs(FL).max()
    assert np.abs(Wh - W).max() < same * np.abs(W).max() and np.abs(fh - f).max() < same * np.abs(f).max()


def test_rigid_mobility_iteration_limit(cuda_lib):
    import torch
    ib = cuda_lib
    x, X, off, FL = _system()
    ctx = _ctx(ib, "fp64")
    try:
        bodies = ib.Bodies(cuda(off), cuda(X), cuda(np.zeros(len(X))))
        W = torch.zeros((len(X), 6), dtype=torch.float64, device="cuda")
        status, st = ib.ibpme_rigid_mobility(ctx, len(x), cuda(x), bodies, cuda(FL), MU,
                                             ib.make_opts(rtol=1e-14, max_iter=2), W)
        torch.cuda.synchronize()
        assert status == ib.IBPME_ERR_NOT_CONVERGED and st.iters == 2 and st.rel_residual > 1e-14
        assert np.isfinite(W.cpu().numpy()).all()
        with pytest.raises(ib.IbpmeError) as e:
            ib.ibpme_rigid_mobility(ctx, len(x), cuda(x), bodies, cuda(FL), 0.0, None, W)
        assert e.value.status == ib.IBPME_ERR_ARG
    finally:
        ib.pme_destroy(ctx)
