"""pme_spread_noalloc: spreading for callers that cannot allocate device memory.

Some callers are not allowed to call cudaMalloc: code recording a CUDA graph
by stream capture, programs whose device memory is owned by a framework's pool,
and real-time loops that must never enter the allocator.  For them the library
offers pme_spread_noalloc, which needs no context and keeps its only scratch
(the wrapped positions) in a fixed array inside the library.  These checks run
it through the C ABI and compare its grid with the context-based pme_spread on
the same inputs, twice in a row with different inputs, the smaller call first,
so that scratch rows a kernel read past n by mistake, or rows left stale by the
earlier call, would show.  The file is named to be collected last.
"""
import numpy as np
import pytest

from helpers import cuda, rel_err

pytestmark = pytest.mark.gpu

# the bars of the spread parity test: FP64 grids agree to rounding, FP32 to single precision
TOL = {"fp64": 1e-12, "mixed": 2e-6}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_spread_matches_pme_spread_twice(cuda_lib, prec):
    import torch

    ib = cuda_lib
    box = np.array([5.0, 6.0, 5.5])
    mesh = (40, 48, 45)
    precision = ib.IBPME_FP64 if prec == "fp64" else ib.IBPME_MIXED
    params = ib.make_params(box=box, mesh=mesh, tol=1e-6, bead_radius=0.1, precision=precision, max_rhs=3)
    ctx = ib.pme_setup(params)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(17)
    try:
        for call, (n, nrhs) in enumerate([(97, 3), (301, 2)]):
            x = rng.uniform(-4, 10, size=(n, 3))
            q = rng.normal(size=(nrhs, n))
            xd, qd = cuda(x), cuda(q)
            ref = torch.zeros((nrhs, mesh[2], mesh[1], mesh[0]), dtype=dt, device="cuda")
            ib.pme_spread(ctx, n, xd, qd, nrhs, ref)
            got = torch.full_like(ref, 7.0)           # the call must clear what it accumulates into
            ib.pme_spread_noalloc(params, n, xd, qd, nrhs, got)
            torch.cuda.synchronize()
            err = rel_err(got.cpu().double().numpy(), ref.cpu().double().numpy())
            assert err < TOL[prec], (call, err)
    finally:
        ib.pme_destroy(ctx)


def test_noalloc_spread_rejects_what_it_cannot_hold(cuda_lib):
    import torch

    ib = cuda_lib
    params = ib.make_params(box=[5.0] * 3, mesh=[32] * 3, tol=1e-6, bead_radius=0.1)
    grid = torch.zeros((1, 32, 32, 32), dtype=torch.float64, device="cuda")
    big = ib.IBPME_NOALLOC_MAX_BEADS + 1
    x = torch.zeros((big, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros((1, big), dtype=torch.float64, device="cuda")
    with pytest.raises(ib.IbpmeError) as e:
        ib.pme_spread_noalloc(params, big, x, q, 1, grid)
    assert e.value.status == ib.IBPME_ERR_ARG and "scratch" in str(e.value)
    # host arrays would need a staging allocation: refused
    with pytest.raises(ib.IbpmeError) as e:
        ib.pme_spread_noalloc(params, 4, np.zeros((4, 3)), np.zeros((1, 4)), 1, grid)
    assert e.value.status == ib.IBPME_ERR_ARG
