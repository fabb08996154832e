"""GPU parity of the periodic RPY mobility (ibpme_rpy_mobility) through the C ABI.

Against oracle/rpy_ref.py (pinned in test_oracle_rpy.py): the FP64 path to 1e-5 and the
mixed path (FP32 mesh) to 1e-3 of the largest velocity, element by element; the tiled
mesh path at sampled beads; reciprocity and linearity; the electrostatics of the same
context unchanged by a mobility call; argument checks.
"""
import numpy as np
import pytest

from oracle import rpy_ref as R

from helpers import FP64_RTOL, MIXED_RTOL, cuda, rel_err

pytestmark = pytest.mark.gpu


def _cloud(n, L, seed):
    rng = np.random.default_rng(seed)
    box = np.array([L, 1.1 * L, 0.9 * L])
    x = rng.uniform(0, 1, size=(n, 3)) * box
    x[1] = x[0] + [0.2, 0.1, 0.0]      # overlapping (r < 2a)
    x[3] = x[2]                         # coincident
    return x, rng.normal(size=(n, 3)), box


def _ctx(ib, box, mesh, tol, a, prec):
    p = {"fp64": ib.IBPME_FP64, "mixed": ib.IBPME_MIXED}[prec]
    return ib.pme_setup(ib.make_params(box=box, mesh=mesh, tol=tol, bead_radius=a, eps_f=0.37, precision=p))


def _U(ib, ctx, x, F, mu):
    import torch
    U = torch.zeros((x.shape[0], 3), dtype=torch.float64, device="cuda")
    ib.ibpme_rpy_mobility(ctx, x.shape[0], cuda(x), cuda(F), mu, U)
    torch.cuda.synchronize()
    return U.cpu().numpy()


@pytest.mark.parametrize("prec,mesh,tol", [("fp64", (48, 48, 48), 1e-8), ("fp64", (40, 45, 36), 1e-8),
                                           ("mixed", (48, 48, 48), 1e-6)])
def test_rpy_mobility_matches_oracle(cuda_lib, prec, mesh, tol):
    """48^3 takes the double-float FP64 transforms, 40 x 45 x 36 cuFFT's FP64 ones."""
    ib = cuda_lib
    a, mu = 0.15, 0.8
    x, F, box = _cloud(40, 6.0, 3)
    ctx = _ctx(ib, box, mesh, tol, a, prec)
    try:
        U = _U(ib, ctx, x, F, mu)
    finally:
        ib.pme_destroy(ctx)
    Ur = R.rpy_mobility(x, F, box, a, mu)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(U, Ur) < bar, rel_err(U, Ur)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rpy_mobility_tiled_sampled(cuda_lib, prec):
    """7,000 beads on 64^3: tiled spread and gather of the three force channels, 30 sampled
    beads (the oracle's explicit k-sum over every source is the cost; its own xi balances it)."""
    ib = cuda_lib
    a, mu = 0.08, 1.3
    x, F, box = _cloud(7000, 8.0, 5)
    # Hasimoto's weight leaves (1 + ln(1/tol)) tol at the mesh's k_c: 1.5e-5 at tol 1e-6, so
    # the FP64 bar takes tol 1e-8 (P = 12)
    ctx = _ctx(ib, box, (64, 64, 64), 1e-8 if prec == "fp64" else 1e-6, a, prec)
    try:
        U = _U(ib, ctx, x, F, mu)
    finally:
        ib.pme_destroy(ctx)
    idx = np.sort(np.random.default_rng(1).choice(len(x), 30, replace=False))
    Ur = R.rpy_mobility(x, F, box, a, mu, targets=idx, xi=1.5, tol=1e-10)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(U[idx], Ur) < bar, rel_err(U[idx], Ur)


def test_rpy_reciprocity_linearity_and_shared_context(cuda_lib):
    import torch
    ib = cuda_lib
    a, mu = 0.15, 1.0
    x, F1, box = _cloud(60, 6.0, 8)
    F2 = np.random.default_rng(9).normal(size=F1.shape)
    ctx = _ctx(ib, box, (48, 48, 48), 1e-8, a, "fp64")
    try:
        q = np.random.default_rng(2).normal(size=len(x))
        q -= q.mean()
        psi0 = torch.zeros((1, len(x)), dtype=torch.float64, device="cuda")
        ib.pme_field(ctx, len(x), cuda(x), cuda(q.reshape(1, -1)), 1, psi0, None)
        U1, U2 = _U(ib, ctx, x, F1, mu), _U(ib, ctx, x, F2, mu)
        U12 = _U(ib, ctx, x, 2.0 * F1 - F2, mu)
        # host buffers
        Uh = np.zeros((len(x), 3))
        ib.ibpme_rpy_mobility(ctx, len(x), np.ascontiguousarray(x), np.ascontiguousarray(F1), mu, Uh)
        psi1 = torch.zeros_like(psi0)
        ib.pme_field(ctx, len(x), cuda(x), cuda(q.reshape(1, -1)), 1, psi1, None)
        torch.cuda.synchronize()
        # n = 0 is a no-op; mu <= 0 is rejected
        ib.ibpme_rpy_mobility(ctx, 0, None, None, mu, None)
        with pytest.raises(ib.IbpmeError) as e:
            ib.ibpme_rpy_mobility(ctx, len(x), cuda(x), cuda(F1), 0.0, torch.zeros((len(x), 3), dtype=torch.float64,
                                                                                    device="cuda"))
        assert e.value.status == ib.IBPME_ERR_ARG
    finally:
        ib.pme_destroy(ctx)
    s = np.abs(U1).max()
    assert abs(np.sum(F1 * U2) - np.sum(F2 * U1)) < 1e-9 * s * np.abs(F1).sum()   # M symmetric
    assert np.abs(U12 - (2 * U1 - U2)).max() < 1e-12 * s
    assert np.abs(Uh - U1).max() < 1e-13 * s
    assert np.abs(psi1.cpu().numpy() - psi0.cpu().numpy()).max() < 1e-13 * np.abs(psi0.cpu().numpy()).max()
    # a context with radius classes answers IBPME_ERR_UNEQUAL_RADII
    ctx = ib.pme_setup(ib.make_params(box=box, mesh=(48, 48, 48), tol=1e-8, class_radius=(0.1, 0.2)))
    try:
        ib.ibpme_set_radius_classes(ctx, len(x), np.zeros(len(x), dtype=np.int32))
        with pytest.raises(ib.IbpmeError) as e:
            ib.ibpme_rpy_mobility(ctx, len(x), cuda(x), cuda(F1), mu, torch.zeros((len(x), 3), dtype=torch.float64,
                                                                                  device="cuda"))
        assert e.value.status == ib.IBPME_ERR_UNEQUAL_RADII
    finally:
        ib.pme_destroy(ctx)
