"""Grand capacitance tensor (Sec. III.B, Eq. QS_capacitance) through ibpme_capacitance:
C = Sigma' M^{-1} Sigma'^T against the oracle's dense LU, in FP64 and mixed
precision, and for one sphere per cubic cell the lattice relations the oracle is
pinned to (the Wigner constant of the charge block, Clausius-Mossotti of the dipole
block, i.e. the effective permittivity of a dilute simple cubic lattice, Sec. IV.C)."""
import math
import numpy as np
import pytest

import oracle as o
from helpers import FP64_RTOL, MIXED_RTOL, context, cuda, rel_err
from workloads import configs as C
from workloads import geometry as G

pytestmark = pytest.mark.gpu


def _capacitance(ib, s, prec, rtol=1e-10, host=False, max_rhs=8):
    import torch
    ctx = context(ib, s, precision=prec, max_rhs=max_rhs)
    try:
        nb = s.n_bodies
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), None)
        if host:
            Cm = np.zeros((4 * nb, 4 * nb))
        else:
            Cm = torch.zeros((4 * nb, 4 * nb), dtype=torch.float64, device="cuda")
        status, st = ib.ibpme_capacitance(ctx, s.n, cuda(s.x), bodies, Cm, ib.make_opts(rtol=rtol))
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= rtol, (status, st.rel_residual)
        return Cm if host else Cm.cpu().numpy(), st
    finally:
        ib.pme_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_capacitance_matches_oracle(cuda_lib, prec):
    """Three charged-free bodies in a small box (4 x 3 = 12 columns: two groups of at
    most eight right-hand sides), element by element against Sigma' M^{-1} Sigma'^T."""
    ib = cuda_lib
    s = C.small_system(seed=71, n_bodies=3, level=2, n_ions=0, L=8.0, a=0.12, mesh=(48, 48, 48), tol=1e-8,
                       charged=False)
    Cg, st = _capacitance(ib, s, prec)
    Cr = o.grand_capacitance(s.x, s.X, s.body_offsets, s.box, s.a, s.eps)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(Cg, Cr) < bar, rel_err(Cg, Cr)
    assert np.abs(Cg - Cg.T).max() < bar * np.abs(Cr).max()
    assert st.iters > 0


def test_capacitance_host_output_and_preconditioner(cuda_lib):
    """The same tensor into a host array, with and without the body-block
    preconditioner (which in this problem inverts -M of each body block)."""
    ib = cuda_lib
    s = C.small_system(seed=72, n_bodies=2, level=2, n_ions=0, L=7.0, a=0.12, mesh=(48, 48, 48), tol=1e-8,
                       charged=False)
    Ch, st_pre = _capacitance(ib, s, "fp64", host=True)
    Cd, _ = _capacitance(ib, s, "fp64", max_rhs=3)   # groups of three columns
    assert rel_err(Ch, Cd) < 1e-8
    import torch
    ctx = context(ib, s, precision="fp64")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        Cn = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
        status, st_none = ib.ibpme_capacitance(ctx, s.n, cuda(s.x), bodies, Cn,
                                               ib.make_opts(rtol=1e-10, precond=ib.IBPME_PRECOND_NONE))
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK
    finally:
        ib.pme_destroy(ctx)
    assert rel_err(Cn.cpu().numpy(), Ch) < 1e-8
    assert st_pre.iters < st_none.iters


def test_lattice_capacitance_wigner_and_clausius_mossotti(cuda_lib):
    """One 162-bead sphere per cubic cell of side 6 and 16: the charge block follows
    1/C_QPsi(L) = 1/C_isolated - w/(4 pi eps L) + a_s^2/(3 eps L^3) (w = 2.837297, the
    simple-cubic Wigner constant) and the dipole block alpha / (1 - alpha/(3 eps V)),
    so eps_eff / eps = 1 + C_SE/(eps V) is Clausius-Mossotti's (1 + 2 phi)/(1 - phi)."""
    ib = cuda_lib
    eps = 0.9
    out = {}
    for L, mesh in ((6.0, 48), (16.0, 64)):
        x = G.icosphere(2) + L / 2
        s = C.assemble("sphere", [x], [], [], [0.0], [L] * 3, 0.1, eps, [[0.0, 0.0, 1.0]], mesh=(mesh,) * 3,
                       tol=1e-8)
        Cg, _ = _capacitance(ib, s, "fp64")
        assert np.abs(Cg[0, 1:]).max() < 1e-6 * Cg[0, 0]
        d = np.diag(Cg)[1:]
        assert np.ptp(d) < 1e-5 * d.mean()
        out[L] = (Cg[0, 0], d.mean())
        if L == 6.0:
            Cr = o.grand_capacitance(s.x, s.X, s.body_offsets, s.box, s.a, s.eps)
            assert rel_err(Cg, Cr) < FP64_RTOL
    w = 2.837297479
    want = -w / (4 * math.pi * eps) * (1 / 6.0 - 1 / 16.0) + (1 / (3 * eps)) * (1 / 6.0 ** 3 - 1 / 16.0 ** 3)
    got = 1 / out[6.0][0] - 1 / out[16.0][0]
    assert abs(got / want - 1) < 3e-3, (got, want)
    V6, V16 = 6.0 ** 3, 16.0 ** 3
    alpha = out[16.0][1] / (1 + out[16.0][1] / (3 * eps * V16))
    assert abs(out[6.0][1] / (alpha / (1 - alpha / (3 * eps * V6))) - 1) < 1e-4
    phi = alpha / (4 * math.pi * eps) * (4 * math.pi / 3) / V6
    eps_eff = 1 + out[6.0][1] / (eps * V6)
    assert abs(eps_eff / ((1 + 2 * phi) / (1 - phi)) - 1) < 1e-4


def test_capacitance_rejects_single_bead_bodies(cuda_lib):
    import torch
    ib = cuda_lib
    s = C.small_system(seed=73, n_bodies=1, level=1, n_ions=4, L=7.0, a=0.12, mesh=(48, 48, 48), tol=1e-8)
    ctx = context(ib, s, precision="fp64")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        Cm = torch.zeros((4 * s.n_bodies, 4 * s.n_bodies), dtype=torch.float64, device="cuda")
        with pytest.raises(ib.IbpmeError) as e:
            ib.ibpme_capacitance(ctx, s.n, cuda(s.x), bodies, Cm)
        assert e.value.status == ib.IBPME_ERR_ARG
    finally:
        ib.pme_destroy(ctx)
