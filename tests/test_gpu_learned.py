"""Learned warm start: the library's MLP kernels against the FP64 reference
network, training, and the gain of the trained network over the zero guess
(the converged solve decides)."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from workloads import configs as C

from helpers import context, cuda

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


def _features_gpu(ib, ctx, s, q=None):
    import torch
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    f = torch.zeros((1, s.n, M.IN), dtype=torch.float32, device="cuda")
    t = torch.zeros((1, s.n), dtype=torch.float32, device="cuda") if q is not None else None
    ib.ibpme_features(ctx, s.n, cuda(s.x), bodies, cuda(s.E0[:1]), 1, f, q, t)
    torch.cuda.synchronize()
    return f[0].cpu().numpy(), (t[0].cpu().numpy() if t is not None else None)


def test_features_and_targets_match_oracle(cuda_lib):
    """ibpme_features against the oracle's definitions bead by bead on a training
    configuration shrunk to L = 12 (seven spheres and rods, 583 ions at least 2a from
    every bead, some inside the bodies), and the training targets of the converged charges."""
    import torch
    ib = cuda_lib
    s = C.warm_start_training(3, L=12.0, mesh=(64, 64, 64), max_ions=600)
    nbb = int(s.body_offsets[np.argmax(np.diff(s.body_offsets) == 1)])   # beads on multi-bead bodies
    assert nbb > 4000 and s.n - nbb > 500
    ctx = context(ib, s, precision="mixed", max_rhs=1)
    try:
        F, S = M.warm_start_features(s.x, s.X, s.body_offsets, s.Q, s.E0[0], s.box, s.a, s.eps)
        q = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
        bd = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        status, _ = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bd, cuda(s.E0[:1]), 1, ib.make_opts(rtol=1e-8),
                                            q)
        assert status == ib.IBPME_OK
        Fg, Tg = _features_gpu(ib, ctx, s, q)
    finally:
        ib.pme_destroy(ctx)
    assert np.abs(F[:nbb, 4]).max() > 0.5           # ions near the surfaces: their normal field
    assert np.all(Fg[nbb:] == 0)
    err = np.abs(Fg[:nbb] - F[:nbb]).max(axis=0)
    assert np.all(err < 2e-4 * np.maximum(1.0, np.abs(F[:nbb]).max(axis=0))), err
    Tr = M.warm_start_targets(q.cpu().numpy()[0], s.body_offsets, s.Q, S)
    assert np.abs(Tg - Tr).max() < 1e-5 * max(1.0, np.abs(Tr).max())


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
    """Train on 120 method-generated solves of 2-8 spheres and rods with ions in
    random fields (L = 30, 96^3 mesh), then solve six unseen configurations from
    the learned guess and from zero: the learned guess starts closer (initial
    residual) and needs no more iterations; its features cost no mesh evaluation,
    so the solve from it makes the same FP64 evaluations as the one from zero."""
    from paper_2401_04865_gb300 import warmstart as W
    ib = cuda_lib
    gen = lambda k: C.warm_start_training(k, mesh=(96, 96, 96), max_ions=5000)
    s0 = gen(0)
    ctx = ib.pme_setup(ib.make_params(box=s0.box, mesh=s0.mesh, tol=s0.tol, bead_radius=s0.a, eps_f=s0.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=1))
    m = None
    try:
        X, T, _ = W.collect(ib, ctx, (gen(100 + k) for k in range(120)))
        m, loss = W.train(ib, X, T, epochs=24)
        assert np.isfinite(loss)
        its, starts, fp64 = [], [], []
        for k in range(6):
            s = gen(900 + k)
            _, st0, _ = _solve(ib, ctx, s, ib.IBPME_GUESS_ZERO)
            _, st1, _ = _solve(ib, ctx, s, ib.IBPME_GUESS_LEARNED, mlp=m)
            assert st1.fell_back == 0
            its.append((st0.iters, st1.iters))
            starts.append((st0.init_rel_residual, st1.init_rel_residual))
            fp64.append((st0.matvecs_fp64, st1.matvecs_fp64))
        zero_it, learned_it = np.mean(its, axis=0)
        zero_r0, learned_r0 = np.mean(starts, axis=0)
        print(f"rows {X.shape[0]} loss {loss:.4f}; iterations zero {zero_it:.2f} learned {learned_it:.2f}; "
              f"initial residual zero {zero_r0:.3f} learned {learned_r0:.3f}; fp64 evaluations {fp64}")
        assert learned_r0 < 0.6 * zero_r0
        assert learned_it <= zero_it
        assert all(b <= a for a, b in fp64)
    finally:
        if m is not None:
            ib.ibpme_mlp_destroy(m)
        ib.pme_destroy(ctx)


def test_learned_step_guess_adds_the_learned_change(cuda_lib):
    """IBPME_GUESS_LEARNED_STEP: the first call starts from the learned guess g; a
    second call at the same positions, given the first call's converged charges,
    starts from exactly those charges (g unchanged), so its initial residual is the
    previous-guess one; along a short BD trajectory the start is q_prev + g(now) -
    g(prev), which keeps every body's net charge and starts about as close as the
    previous charges alone (the learned change is small next to the step's own
    change on this system: within 25% on average)."""
    import torch
    from paper_2401_04865_gb300 import warmstart as W
    ib = cuda_lib
    gen = lambda k: C.warm_start_training(k, mesh=(96, 96, 96), max_ions=5000)
    s = gen(11)
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=1))
    m = None
    try:
        X, T, _ = W.collect(ib, ctx, (gen(300 + k) for k in range(40)))
        m, _ = W.train(ib, X, T, epochs=16)
        n, nb = s.n, s.n_bodies
        off, Xb, Q, E0 = cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q), cuda(s.E0[0])
        x = cuda(s.x)
        q = torch.zeros((1, n), dtype=torch.float64, device="cuda")
        step = lambda g: ib.induced_charge_solve(ctx, n, x, ib.Bodies(off, Xb, Q), E0, 1,
                                                 ib.make_opts(rtol=1e-8, guess=g, mlp=m), q)
        st, s1 = step(ib.IBPME_GUESS_LEARNED_STEP)     # first call: the learned guess itself
        assert st == ib.IBPME_OK
        q1 = q.clone()
        st, s2 = step(ib.IBPME_GUESS_LEARNED_STEP)     # same positions: starts from q1
        st3, s3 = ib.induced_charge_solve(ctx, n, x, ib.Bodies(off, Xb, Q), E0, 1,
                                          ib.make_opts(rtol=1e-8, guess=ib.IBPME_GUESS_USER), q1.clone())
        assert st == ib.IBPME_OK and st3 == ib.IBPME_OK
        assert abs(s2.init_rel_residual - s3.init_rel_residual) < 1e-6 * max(1e-12, s3.init_rel_residual) + 1e-14
        # a BD trajectory: learned change against the previous charges alone
        F = torch.zeros((nb, 3), dtype=torch.float64, device="cuda")
        Lt = torch.zeros_like(F)
        init = {}
        for mode in (ib.IBPME_GUESS_USER, ib.IBPME_GUESS_LEARNED_STEP):
            xa, Xa = cuda(s.x), cuda(s.X)
            xb, Xc = torch.empty_like(xa), torch.empty_like(Xa)
            q.zero_()
            r = []
            for k in range(12):
                st, sk = ib.ibpme_bd_advance(ctx, n, xa, ib.Bodies(off, Xa, Q), E0, ib.make_opts(rtol=1e-6, guess=mode, mlp=m),
                                             q[0], 1e-3, 1.0, 1.0, 77, k, F, Lt, xb, Xc)
                assert st == ib.IBPME_OK
                if k >= 2:
                    r.append(sk.init_rel_residual)
                sums = np.add.reduceat(q[0].cpu().numpy(), s.body_offsets[:-1])
                assert np.max(np.abs(sums - s.Q)) < 1e-9
                xa, xb, Xa, Xc = xb, xa, Xc, Xa
            init[mode] = float(np.mean(r))
        print("initial residual previous %.4f learned step %.4f" % (init[ib.IBPME_GUESS_USER],
                                                                   init[ib.IBPME_GUESS_LEARNED_STEP]))
        assert init[ib.IBPME_GUESS_LEARNED_STEP] <= 1.25 * init[ib.IBPME_GUESS_USER]
    finally:
        if m is not None:
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
