"""GPU parity for beads of unequal radii (radius classes) through the C ABI.

The pair kernel of two radii is j0(k a_alpha) j0(k a_beta)/k^2 (the shell of a bead
of radius a transforms as j0(ka), Eq. M00_Fourier); the oracle's two-radius sums are
pinned in test_oracle_radii.py.  Surface beads take one radius, the ions another, so
pairs of both classes overlap and one class's beads sit inside the other's shells.
Bars as in test_gpu_parity.py: 1e-5 (FP64) and 1e-3 (mixed) of each result's scale.
"""
import numpy as np
import pytest

import oracle as o
from workloads import configs as C

from helpers import FP64_RTOL, MIXED_RTOL, cuda, random_neutral_charges, rel_err

pytestmark = pytest.mark.gpu

A_SURF, A_ION = 0.12, 0.3


def _system(seed=71, n_bodies=3, level=2, n_ions=40, L=9.0, mesh=(48, 48, 48), tol=1e-7, nrhs=1):
    s = C.small_system(seed=seed, n_bodies=n_bodies, level=level, n_ions=n_ions, L=L, a=A_SURF, mesh=mesh, tol=tol,
                       nrhs=nrhs)
    ion = np.diff(s.body_offsets)[o.body_index(s.body_offsets)] == 1
    # two ions beside the first body's first bead: one whose shell holds the bead
    # (r = 0.1 < a_ion - a_surf), one overlapping it (a_ion - a_surf < r = 0.3 < a_ion + a_surf)
    i0 = int(np.flatnonzero(ion)[0])
    centre = s.X[0]
    u = o.min_image(s.x[0] - centre, s.box)
    u /= np.linalg.norm(u)
    for k, dist in enumerate((1.1, 1.3)):
        s.x[i0 + k] = centre + dist * u
        s.X[o.body_index(s.body_offsets)[i0 + k]] = s.x[i0 + k]
    cls = ion.astype(np.int32)
    rad = np.where(ion, A_ION, A_SURF)
    return s, cls, rad


def _context(ib, s, cls, prec, max_rhs=3):
    p = {"fp64": ib.IBPME_FP64, "mixed": ib.IBPME_MIXED}[prec]
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, eps_f=s.eps, precision=p, max_rhs=max_rhs,
                                      class_radius=(A_SURF, A_ION)))
    ib.ibpme_set_radius_classes(ctx, len(cls), cls)
    return ctx


def _field(ib, ctx, x, q, nrhs):
    import torch
    n = x.shape[0]
    psi = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda")
    E = torch.zeros((nrhs, n, 3), dtype=torch.float64, device="cuda")
    ib.pme_field(ctx, n, cuda(x), cuda(np.asarray(q).reshape(nrhs, n)), nrhs, psi, E)
    torch.cuda.synchronize()
    return psi.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pme_field_with_unequal_radii_matches_oracle(cuda_lib, prec):
    ib = cuda_lib
    s, cls, rad = _system()
    d = o.min_image(s.x[:, None, :] - s.x[None, :, :], s.box)
    r = np.sqrt((d * d).sum(axis=2)) + np.eye(s.n) * 1e9
    mixed_pair = cls[:, None] != cls[None, :]
    assert (mixed_pair & (r < A_SURF + A_ION)).sum() > 10   # overlapping pairs of the two classes
    q = np.stack([random_neutral_charges(s.n, 5), random_neutral_charges(s.n, 6) + 0.05])
    ctx = _context(ib, s, cls, prec)
    try:
        assert abs(ib.ibpme_get_params(ctx).bead_radius - A_ION) < 1e-15   # the largest class radius
        psi, E = _field(ib, ctx, s.x, q, 2)
    finally:
        ib.pme_destroy(ctx)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    for k in range(2):
        pr, Er = o.potential(s.x, q[k], s.box, rad, s.eps, field=True)
        assert rel_err(psi[k], pr) < bar, rel_err(psi[k], pr)
        assert rel_err(E[k], Er) < 10 * bar, rel_err(E[k], Er)
        # the classes matter: one radius for every bead misses by far more than the bar
        p1 = o.potential(s.x, q[k], s.box, A_SURF, s.eps)
        assert rel_err(p1, pr) > 30 * bar


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pme_field_with_unequal_radii_tiled_sampled(cuda_lib, prec):
    """8 spheres of 642 beads and 2,000 ions on 64^3 (tiled spread and gather, both
    classes binned into their own channels), at 150 sampled beads."""
    ib = cuda_lib
    s, cls, rad = _system(seed=72, n_bodies=8, level=3, n_ions=2000, L=14.0, mesh=(64, 64, 64), tol=1e-6)
    q = random_neutral_charges(s.n, 8)
    ctx = _context(ib, s, cls, prec)
    try:
        psi, E = _field(ib, ctx, s.x, q, 1)
    finally:
        ib.pme_destroy(ctx)
    idx = np.sort(np.random.default_rng(3).choice(s.n, 150, replace=False))
    pr, Er = o.potential(s.x, q, s.box, rad, s.eps, targets=idx, field=True)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(psi[0, idx], pr) < bar, rel_err(psi[0, idx], pr)
    assert rel_err(E[0, idx], Er) < 10 * bar, rel_err(E[0, idx], Er)


def test_equal_class_radii_give_the_one_radius_results(cuda_lib):
    """Two classes of the same radius go through the class channels, the mixing and the
    exact per-pair kernel, and reproduce the one-radius context (tabulated kernel)."""
    import torch
    ib = cuda_lib
    s, cls, _ = _system(seed=73)
    q = random_neutral_charges(s.n, 9)
    out = []
    for classes in (False, True):
        kw = dict(box=s.box, mesh=s.mesh, tol=s.tol, eps_f=s.eps, precision=ib.IBPME_FP64, bead_radius=A_SURF)
        if classes:
            kw["class_radius"] = (A_SURF, A_SURF)
        ctx = ib.pme_setup(ib.make_params(**kw))
        try:
            if classes:
                ib.ibpme_set_radius_classes(ctx, s.n, cls)
            out.append(_field(ib, ctx, s.x, q, 1))
        finally:
            ib.pme_destroy(ctx)
        torch.cuda.synchronize()
    assert rel_err(out[1][0], out[0][0]) < 1e-9
    assert rel_err(out[1][1], out[0][1]) < 1e-8


def _solve(ib, ctx, s, precond=None, rtol=1e-10):
    import torch
    R, n, nb = s.nrhs, s.n, s.n_bodies
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    q = torch.zeros((R, n), dtype=torch.float64, device="cuda")
    psi = torch.zeros((R, nb), dtype=torch.float64, device="cuda")
    S = torch.zeros((R, nb, 3), dtype=torch.float64, device="cuda")
    opts = ib.make_opts(rtol=rtol, precond=ib.IBPME_PRECOND_BODY if precond is None else precond)
    status, st = ib.induced_charge_solve(ctx, n, cuda(s.x), bodies, cuda(s.E0), R, opts, q, psi, S)
    torch.cuda.synchronize()
    return status, st, q.cpu().numpy(), psi.cpu().numpy(), S.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_with_unequal_radii_matches_dense_oracle(cuda_lib, prec, monkeypatch):
    """Two fields, three bodies of small beads, ions of a larger radius: the free-bead
    operator, the full operator and the unpreconditioned solve agree, and match the
    oracle's dense LU of the two-radius saddle system."""
    ib = cuda_lib
    s, cls, rad = _system(seed=74, nrhs=2)
    qr, psr = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0, s.box, rad, s.eps)
    out = {}
    for full, pre in ((False, None), (True, None), (False, ib.IBPME_PRECOND_NONE)):
        if full:
            monkeypatch.setenv("IBPME_FULL_OPERATOR", "1")
        else:
            monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
        ctx = _context(ib, s, cls, prec)
        try:
            status, st, q, psi, S = _solve(ib, ctx, s, precond=pre)
            assert status == ib.IBPME_OK and st.rel_residual <= 1e-10
            out[full, pre] = (st.iters, q, psi, S)
        finally:
            ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
    it_free, q, psi, S = out[False, None]
    for key in ((True, None), (False, ib.IBPME_PRECOND_NONE)):
        assert rel_err(out[key][1], q) < 1e-8
        assert rel_err(out[key][3], S) < 1e-8
    assert it_free < out[False, ib.IBPME_PRECOND_NONE][0]   # the two-radius body blocks still precondition
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    rel = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    for r in range(2):
        assert rel_err(q[r], qr[r]) < bar, rel_err(q[r], qr[r])
        pscale = max(np.abs(psr[r]).max(), np.abs(rel @ s.E0[r]).max())
        assert np.abs(psi[r] - psr[r]).max() < bar * pscale
        Sr = o.dipoles(s.x, s.X, s.body_offsets, qr[r], s.box)
        assert rel_err(S[r], Sr) < bar
    # the one-radius dense solution differs by far more than the bar
    q1, _ = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, A_SURF, s.eps)
    assert rel_err(q1, qr[0]) > 30 * bar


def test_bd_advance_with_unequal_radii_matches_oracle(cuda_lib):
    """Solve, forces and one BD step in one call with two radii: charges, bead and body
    forces, torques and energy against the dense FP64 oracle, and the step against the
    oracle's step with the hard-sphere contact at a_alpha + a_beta (two ions placed to
    overlap as large beads but not as small ones)."""
    import torch
    ib = cuda_lib
    s, cls, rad = _system(seed=75, n_bodies=2, n_ions=12, L=8.0, tol=1e-8)
    x = s.x.copy()
    X = s.X.copy()
    x[-1] = x[-2] + [0.45, 0.1, 0.0]   # r = 0.46: inside 2 a_ion = 0.6, outside 2 a_surf = 0.24
    X[-1] = x[-1]
    n, nb = s.n, s.n_bodies
    dt, gamma, kT, seed, step = 1e-3, 1.1, 0.8, 4242, 2
    qr, psr = o.solve_dense(x, s.body_offsets, X, s.Q, s.E0[0], s.box, rad, s.eps)
    f_ref = o.bead_forces(x, qr, s.E0[0], s.box, rad, s.eps)
    F_ref, L_ref = o.body_force_torque(x, X, s.body_offsets, f_ref, s.box)
    U_ref = o.energy(X, s.Q, psr, o.dipoles(x, X, s.body_offsets, qr, s.box), s.E0[0])
    hs = o.hard_sphere_forces(x, s.body_offsets, s.box, rad, gamma, dt)
    assert np.abs(hs[-1]).max() > 1.0
    xr, Xr = o.bd_step(x, X, s.body_offsets, f_ref + hs, s.box, rad, dt, gamma=gamma, kT=kT, seed=seed, step=step)
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device="cuda")
    ctx = _context(ib, s, cls, "fp64")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(X), cuda(s.Q))
        q, psi, f, F, L, U, xo, Xo = z(1, n), z(1, nb), z(n, 3), z(nb, 3), z(nb, 3), z(1), z(n, 3), z(nb, 3)
        status, st = ib.ibpme_bd_advance(ctx, n, cuda(x), bodies, cuda(s.E0[0]), ib.make_opts(rtol=1e-10), q, dt,
                                         gamma, kT, seed, step, F, L, xo, Xo, psi_out=psi, f_bead=f, U=U)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= 1e-10
        q, f, F, L, U, xo, Xo = (t.cpu().numpy() for t in (q, f, F, L, U, xo, Xo))
    finally:
        ib.pme_destroy(ctx)
    assert rel_err(q[0], qr) < FP64_RTOL
    assert rel_err(f, f_ref) < FP64_RTOL and rel_err(F, F_ref) < FP64_RTOL
    r = o.relative_positions(x, X, s.body_offsets, s.box)
    moment = np.add.reduceat(np.linalg.norm(r, axis=1) * np.linalg.norm(f_ref, axis=1), s.body_offsets[:-1])
    assert np.max(np.abs(L - L_ref)) < FP64_RTOL * moment.max()
    assert abs(U[0] - U_ref) < FP64_RTOL * abs(U_ref)
    disp_ref = o.min_image(xr - x, s.box)
    assert np.max(np.abs(o.min_image(xo - xr, s.box))) < FP64_RTOL * np.abs(disp_ref).max()
    assert np.max(np.abs(o.min_image(Xo - Xr, s.box))) < FP64_RTOL * np.abs(disp_ref).max()


def test_radius_class_arguments_are_checked(cuda_lib):
    import torch
    ib = cuda_lib
    s, cls, _ = _system(seed=76, n_bodies=2, n_ions=10)
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, eps_f=s.eps, precision=ib.IBPME_FP64,
                                      class_radius=(A_SURF, A_ION)))
    try:
        psi = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
        q = cuda(random_neutral_charges(s.n, 1).reshape(1, -1))
        with pytest.raises(ib.IbpmeError) as e:   # no binding
            ib.pme_field(ctx, s.n, cuda(s.x), q, 1, psi, None)
        assert e.value.status == ib.IBPME_ERR_ARG
        bad = cls.copy()
        bad[3] = 2
        with pytest.raises(ib.IbpmeError) as e:   # class out of range
            ib.ibpme_set_radius_classes(ctx, s.n, bad)
        assert e.value.status == ib.IBPME_ERR_ARG
        ib.ibpme_set_radius_classes(ctx, s.n - 1, cls[:-1])
        with pytest.raises(ib.IbpmeError) as e:   # bound for another bead count
            ib.pme_field(ctx, s.n, cuda(s.x), q, 1, psi, None)
        assert e.value.status == ib.IBPME_ERR_ARG
        ib.ibpme_set_radius_classes(ctx, s.n, cls)
        ib.pme_field(ctx, s.n, cuda(s.x), q, 1, psi, None)   # bound: runs
        torch.cuda.synchronize()
        assert np.isfinite(psi.cpu().numpy()).all()
        # the batched solve and the learned guess take one radius
        nb = s.n_bodies
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        qo = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
        with pytest.raises(ib.IbpmeError) as e:
            ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, [0, 1, nb], cuda(s.E0[:1]), 1, None, qo)
        assert e.value.status == ib.IBPME_ERR_UNEQUAL_RADII
        mlp = ib.ibpme_mlp_create(1)
        try:
            with pytest.raises(ib.IbpmeError) as e:
                ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0[:1]), 1,
                                        ib.make_opts(guess=ib.IBPME_GUESS_LEARNED, mlp=mlp), qo)
            assert e.value.status == ib.IBPME_ERR_UNEQUAL_RADII
        finally:
            ib.ibpme_mlp_destroy(mlp)
    finally:
        ib.pme_destroy(ctx)
    # a one-radius context takes no binding
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=A_SURF))
    try:
        with pytest.raises(ib.IbpmeError) as e:
            ib.ibpme_set_radius_classes(ctx, s.n, cls)
        assert e.value.status == ib.IBPME_ERR_ARG
    finally:
        ib.pme_destroy(ctx)
