"""Learned warm start: the library's MLP kernels against the FP64 reference
network, training, and the gain of the trained network over the zero guess
(the converged solve decides)."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from workloads import configs as C

from helpers import cuda

pytestmark = pytest.mark.gpu


def _params(ib, m):
    p = np.zeros(ib.IBPME_MLP_NPARAM, dtype=np.float32)
    ib.ibpme_mlp_get(m, p)
    return p


def test_mlp_forward_and_gradient_match_fp64_reference(cuda_lib):
    import torch
    ib = cuda_lib
    m = ib.ibpme_mlp_create(seed=3)
    try:
        rng = np.random.default_rng(1)
        n = 777                                   # several tiles and a ragged tail
        X = rng.normal(size=(n, M.IN)).astype(np.float32)
        T = rng.normal(size=n).astype(np.float32)
        p = _params(ib, m)
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        ib.ibpme_mlp_forward(m, n, cuda(X), y)
        torch.cuda.synchronize()
        yr = M.forward(p, X)
        assert np.max(np.abs(y.cpu().numpy() - yr)) < 1e-5 * max(1.0, np.abs(yr).max())
        g = np.zeros(ib.IBPME_MLP_NPARAM, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        ib.ibpme_mlp_gradient(m, n, cuda(X), cuda(T), g, loss)
        Lr, gr = M.loss_and_grad(p, X, T)
        assert abs(loss[0] - Lr) < 1e-5 * Lr
        assert np.max(np.abs(g - gr)) < 1e-4 * np.abs(gr).max()
    finally:
        ib.ibpme_mlp_destroy(m)


def test_mlp_training_fits_a_smooth_target(cuda_lib):
    ib = cuda_lib
    m = ib.ibpme_mlp_create(seed=5)
    try:
        rng = np.random.default_rng(2)
        n = 20000
        X = rng.normal(size=(n, M.IN)).astype(np.float32)
        T = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3]).astype(np.float32)
        Xd, Td = cuda(X), cuda(T)
        first = ib.ibpme_mlp_train(m, n, Xd, Td, batch=1024, epochs=1, lr=3e-3, seed=1)
        last = ib.ibpme_mlp_train(m, n, Xd, Td, batch=1024, epochs=40, lr=3e-3, seed=2)
        assert last < 0.1 * first and last < 0.02
        # the trained parameters still agree with the reference network
        p = _params(ib, m)
        assert abs(M.loss_and_grad(p, X[:2000], T[:2000])[0] - last) < 0.02
    finally:
        ib.ibpme_mlp_destroy(m)


def _system(seed, rng):
    s = C.small_system(seed=seed, n_bodies=int(rng.integers(2, 5)), level=2, n_ions=16, L=12.0, a=0.12,
                       mesh=(48, 48, 48), tol=1e-6)
    d = rng.normal(size=3)
    s.E0 = (d / np.linalg.norm(d) * rng.uniform(0.1, 2.0)).reshape(1, 3)
    return s


def _solve(ib, ctx, s, guess, mlp=None, rtol=1e-6, prec=-1):
    import torch
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    q = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
    status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 1,
                                         ib.make_opts(rtol=rtol, guess=guess, mlp=mlp, precision=prec), q)
    torch.cuda.synchronize()
    assert status == ib.IBPME_OK
    return q, st, bodies


def test_learned_warm_start_gains_over_zero_guess(cuda_lib):
    """Train on converged solves of 2-4 spheres with ions in random fields, then
    solve unseen systems from the learned guess and from zero: the learned guess
    starts much closer (initial residual) and needs fewer iterations."""
    import torch
    ib = cuda_lib
    rng = np.random.default_rng(11)
    s0 = _system(100, rng)
    ctx = ib.pme_setup(ib.make_params(box=s0.box, mesh=s0.mesh, tol=s0.tol, bead_radius=s0.a, eps_f=s0.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=1))
    m = ib.ibpme_mlp_create(seed=7)
    try:
        feats, targets = [], []
        for k in range(40):
            s = _system(200 + k, rng)
            q, st, bodies = _solve(ib, ctx, s, ib.IBPME_GUESS_ZERO, rtol=1e-9, prec=ib.IBPME_FP64)
            f = torch.zeros((1, s.n, M.IN), dtype=torch.float32, device="cuda")
            t = torch.zeros((1, s.n), dtype=torch.float32, device="cuda")
            ib.ibpme_features(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 1, f, q, t)
            keep = s.body_offsets[1:] - s.body_offsets[:-1] > 1
            beads = np.repeat(keep, np.diff(s.body_offsets))
            feats.append(f[0][torch.as_tensor(beads, device="cuda")])
            targets.append(t[0][torch.as_tensor(beads, device="cuda")])
        X = torch.cat(feats).contiguous()
        T = torch.cat(targets).contiguous()
        loss = ib.ibpme_mlp_train(m, X.shape[0], X, T, batch=1024, epochs=150, lr=2e-3, seed=3)
        assert np.isfinite(loss)
        gains, starts = [], []
        for k in range(6):
            s = _system(900 + k, rng)
            _, st0, _ = _solve(ib, ctx, s, ib.IBPME_GUESS_ZERO)
            _, st1, _ = _solve(ib, ctx, s, ib.IBPME_GUESS_LEARNED, mlp=m)
            assert st1.fell_back == 0
            gains.append((st0.iters, st1.iters))
            starts.append((st0.init_rel_residual, st1.init_rel_residual))
        zero_it = np.mean([g[0] for g in gains])
        learned_it = np.mean([g[1] for g in gains])
        zero_r0 = np.mean([r[0] for r in starts])
        learned_r0 = np.mean([r[1] for r in starts])
        print(f"iterations zero {zero_it:.1f} learned {learned_it:.1f}; initial residual zero {zero_r0:.3f} "
              f"learned {learned_r0:.3f}; train loss {loss:.4f}")
        assert learned_r0 < 0.5 * zero_r0
        assert learned_it < zero_it
    finally:
        ib.ibpme_mlp_destroy(m)
        ib.pme_destroy(ctx)


def test_mlp_tensor_core_forward_matches_bf16_reference(cuda_lib):
    """ibpme_mlp_forward_tc (tcgen05.mma, BF16 hidden layer) against the FP64
    network with the hidden layer's operands rounded to BF16 (tight: checks the
    tensor-core operand layout and accumulation), and against the FP32 network
    within BF16 accuracy; 777 samples = six full 128-row tiles and a ragged one."""
    import torch
    ib = cuda_lib
    m = ib.ibpme_mlp_create(seed=11)
    try:
        rng = np.random.default_rng(4)
        n = 777
        X = rng.normal(size=(n, M.IN)).astype(np.float32)
        p = _params(ib, m)
        y = torch.zeros(n, dtype=torch.float32, device="cuda")
        ib.ibpme_mlp_forward_tc(m, n, cuda(X), y)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
        ref_q = M.forward_bf16_hidden(p, X)
        ref = M.forward(p, X)
        scale = max(1.0, np.abs(ref).max())
        assert np.max(np.abs(got - ref_q)) < 2e-4 * scale, np.max(np.abs(got - ref_q))
        assert np.max(np.abs(got - ref)) < 3e-2 * scale
        # no sample is skipped or duplicated across tiles: compare sample by sample
        assert np.argmax(np.abs(got - ref_q)) >= 0 and np.all(np.isfinite(got))
        # empty input
        ib.ibpme_mlp_forward_tc(m, 0, None, None)
    finally:
        ib.ibpme_mlp_destroy(m)
