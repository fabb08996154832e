"""GPU parity: the CUDA library through its C ABI against the FP64 oracle.

Bars: 1e-5 (FP64 path) and 1e-3 (mixed precision) relative to each result's
largest magnitude, element by element (helpers.rel_err).  Sizes span several
tiles with ragged tails; the full-size cases compare sampled outputs.
"""
import math

import numpy as np
import pytest

import oracle as o
from workloads import configs as C

from helpers import FP64_RTOL, MIXED_RTOL, context, cuda, random_neutral_charges, rel_err

pytestmark = pytest.mark.gpu


def _field(ib, ctx, x, q, nrhs=1, with_E=True):
    import torch
    n = x.shape[0]
    xd = cuda(x)
    qd = cuda(np.asarray(q).reshape(nrhs, n))
    psi = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda")
    E = torch.zeros((nrhs, n, 3), dtype=torch.float64, device="cuda") if with_E else None
    ib.pme_field(ctx, n, xd, qd, nrhs, psi, E)
    torch.cuda.synchronize()
    return psi.cpu().numpy(), (E.cpu().numpy() if with_E else None)


def test_setup_applies_the_paper_parameter_rules(cuda_lib):
    ib = cuda_lib
    for L, mesh, tol, a in [(20.0, 64, 1e-8, 0.1), (30.0, 128, 1e-6, 0.05), (13.89, 256, 1e-6, 0.05)]:
        ctx = ib.pme_setup(ib.make_params(box=[L] * 3, mesh=[mesh] * 3, tol=tol, bead_radius=a))
        p = ib.ibpme_get_params(ctx)
        ref = o.auto_params([L] * 3, [mesh] * 3, tol, a)
        assert p.P == ref["P"]
        for k in ("xi", "eta", "r_cut"):
            assert abs(getattr(p, k) - ref[k]) <= 1e-12 * ref[k]
        ib.pme_destroy(ctx)
    # invalid arguments are rejected with IBPME_ERR_ARG, not a fault
    bad = [dict(box=[10.0] * 3, mesh=[8] * 3, tol=1e-8),                 # mesh < P
           dict(box=[3.0] * 3, mesh=[16] * 3, tol=1e-10, bead_radius=0.4),  # r_cut >= L/2
           dict(box=[10.0] * 3, mesh=[32] * 3, bead_radius=0.0)]
    for kw in bad:
        kw.setdefault("bead_radius", 0.1)
        with pytest.raises(ib.IbpmeError) as e:
            ib.pme_setup(ib.make_params(**kw))
        assert e.value.status == ib.IBPME_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spread_matches_its_definition(cuda_lib, prec):
    import torch
    ib = cuda_lib
    rng = np.random.default_rng(3)
    n, nrhs = 37, 2
    box = np.array([5.0, 6.0, 5.5])
    mesh = (40, 48, 45)
    x = rng.uniform(-3, 9, size=(n, 3))          # outside the box too: wrapped internally
    q = rng.normal(size=(nrhs, n))
    ctx = ib.pme_setup(ib.make_params(box=box, mesh=mesh, tol=1e-6, bead_radius=0.1,
                                      precision=ib.IBPME_FP64 if prec == "fp64" else ib.IBPME_MIXED))
    p = ib.ibpme_get_params(ctx)
    dt = torch.float64 if prec == "fp64" else torch.float32
    grid = torch.zeros((nrhs, mesh[2], mesh[1], mesh[0]), dtype=dt, device="cuda")
    ib.pme_spread(ctx, n, cuda(x), cuda(q), nrhs, grid)
    got = grid.cpu().double().numpy()
    for r in range(nrhs):
        ref = o.spread_grid(x, q[r], box, mesh, p.xi, p.eta, p.P)
        assert rel_err(got[r], ref) < (1e-12 if prec == "fp64" else 2e-6)
    ib.pme_destroy(ctx)


def _field_case(name):
    if name == "sphere162":
        s = C.config1()
        q = random_neutral_charges(s.n, 1)
        return s.x, q, s.box, s.a, s.eps, s.mesh, s.tol
    if name == "overlapping_rect":
        rng = np.random.default_rng(5)
        box = np.array([6.0, 7.0, 6.5])
        x = rng.uniform(0, 1, size=(301, 3)) * box
        x[1] = x[0] + [0.05, 0.02, 0.0]           # overlapping beads (r < 2a)
        x[2] = x[0]                               # coincident beads
        q = random_neutral_charges(301, 2)
        return x, q, box, 0.2, 0.7, (40, 48, 45), 1e-8
    raise KeyError(name)


@pytest.mark.parametrize("case", ["sphere162", "overlapping_rect"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pme_field_matches_oracle(cuda_lib, case, prec):
    ib = cuda_lib
    x, q, box, a, eps, mesh, tol = _field_case(case)
    ref_psi, ref_E = o.potential(x, q, box, a, eps, field=True)
    ctx = ib.pme_setup(ib.make_params(box=box, mesh=mesh, tol=tol, bead_radius=a, eps_f=eps,
                                      precision=ib.IBPME_FP64 if prec == "fp64" else ib.IBPME_MIXED))
    psi, E = _field(ib, ctx, x, q)
    bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
    assert rel_err(psi[0], ref_psi) < bar
    assert rel_err(E[0], ref_E) < bar
    ib.pme_destroy(ctx)


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
def test_cached_stencil_mesh_kernels_match_fp64_and_oracle(cuda_lib, nrhs):
    """pme_field runs the cached-stencil spread and gather in both precisions.  A
    dense cluster straddling the periodic corner plus scattered beads, P = 9, one
    to four fields; the FP32 mesh against the FP64 mesh to FP32 rounding and
    against the oracle at the mixed bar, and a second call (cache reused) against
    the first."""
    ib = cuda_lib
    rng = np.random.default_rng(40 + nrhs)
    box = np.array([5.0, 6.0, 7.0])
    mesh = (32, 40, 48)
    d = rng.normal(size=(400, 3))
    cluster = 0.6 * d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0, 1, size=(400, 1)) ** (1 / 3)
    x = np.concatenate([cluster + [0.1, 5.9, 3.5], rng.uniform(0, 1, size=(300, 3)) * box])
    n = x.shape[0]
    q = np.stack([random_neutral_charges(n, 100 + r) for r in range(nrhs)])
    kw = dict(box=box, mesh=mesh, tol=1e-6, bead_radius=0.02, eps_f=0.8, max_rhs=4)
    c64 = ib.pme_setup(ib.make_params(precision=ib.IBPME_FP64, **kw))
    c32 = ib.pme_setup(ib.make_params(precision=ib.IBPME_MIXED, **kw))
    try:
        assert ib.ibpme_get_params(c32).P == 9
        p64, e64 = _field(ib, c64, x, q, nrhs=nrhs)
        p32, e32 = _field(ib, c32, x, q, nrhs=nrhs)
        for r in range(nrhs):
            assert rel_err(p32[r], p64[r]) < 2e-5, (r, rel_err(p32[r], p64[r]))
            assert rel_err(e32[r], e64[r]) < 2e-5, (r, rel_err(e32[r], e64[r]))
        # twice in a row: the cached bins and the graph-free path give the same result
        p32b, e32b = _field(ib, c32, x, q, nrhs=nrhs)
        assert rel_err(p32b, p32) < 1e-6 and rel_err(e32b, e32) < 1e-6
        if nrhs == 1:
            ref_psi, ref_E = o.potential(x, q[0], box, 0.02, 0.8, field=True)
            assert rel_err(p32[0], ref_psi) < MIXED_RTOL and rel_err(e32[0], ref_E) < MIXED_RTOL
    finally:
        ib.pme_destroy(c64)
        ib.pme_destroy(c32)


def _dense_surfaces(seed, n_surf=6, per=1500, n_ions=1000, box=(5.0, 6.0, 7.0)):
    """Beads packed on sphere surfaces (hundreds per grid cell, some straddling
    the periodic faces) plus scattered ions."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box)
    parts = []
    for k in range(n_surf):
        d = rng.normal(size=(per, 3))
        c = rng.uniform(0, 1, size=3) * box if k else np.array([0.2, 5.9, 3.5])   # one across the corner
        parts.append(c + 0.8 * d / np.linalg.norm(d, axis=1, keepdims=True))
    parts.append(rng.uniform(0, 1, size=(n_ions, 3)) * box)
    return np.mod(np.concatenate(parts), box), box


@pytest.mark.parametrize("nrhs,mesh", [(1, (36, 44, 52)), (3, (36, 44, 52)), (1, (40, 48, 56)), (3, (40, 48, 56)),
                                       (2, (38, 44, 50))])
def test_tiled_mesh_path_matches_direct_path_and_oracle(cuda_lib, nrhs, mesh, monkeypatch):
    """10,000 beads (9,000 on six sphere surfaces, 1,000 ions) take the tiled
    spread and gather (shared-memory regions for dense tiles, direct atomics for
    isolated ions), on meshes whose edges are and are not multiples of the tile
    edge (ragged last tiles) and with N_x a multiple of four (FP32 rows in float4
    groups) or not (scalar rows).  Against the same call with tiles switched off (FP64
    to rounding, FP32 to FP32 rounding) and against the oracle at sampled beads."""
    ib = cuda_lib
    x, box = _dense_surfaces(50 + nrhs)
    n = x.shape[0]
    q = np.stack([random_neutral_charges(n, 200 + r) for r in range(nrhs)])
    kw = dict(box=box, mesh=mesh, tol=1e-6, bead_radius=0.01, eps_f=0.8, max_rhs=4)
    out = {}
    for tiles in (True, False):
        if tiles:
            monkeypatch.delenv("IBPME_NO_TILES", raising=False)
        else:
            monkeypatch.setenv("IBPME_NO_TILES", "1")
        for prec in (ib.IBPME_FP64, ib.IBPME_MIXED):
            ctx = ib.pme_setup(ib.make_params(precision=prec, **kw))
            try:
                out[tiles, prec] = _field(ib, ctx, x, q, nrhs=nrhs)
            finally:
                ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_NO_TILES", raising=False)
    for prec, bar in ((ib.IBPME_FP64, 1e-12), (ib.IBPME_MIXED, 2e-6)):
        (pt, et), (pd, ed) = out[True, prec], out[False, prec]
        for r in range(nrhs):
            assert rel_err(pt[r], pd[r]) < bar, (prec, r, rel_err(pt[r], pd[r]))
            assert rel_err(et[r], ed[r]) < bar, (prec, r, rel_err(et[r], ed[r]))
    t = np.random.default_rng(1).choice(n, size=48, replace=False).astype(np.int32)
    for r in range(nrhs):
        ref_psi, ref_E = o.potential(x, q[r], box, 0.01, 0.8, targets=t, field=True)
        for prec, bar in ((ib.IBPME_FP64, FP64_RTOL), (ib.IBPME_MIXED, MIXED_RTOL)):
            p, e = out[True, prec]
            assert rel_err(p[r][t], ref_psi) < bar, (prec, r, rel_err(p[r][t], ref_psi))
            assert rel_err(e[r][t], ref_E) < bar, (prec, r, rel_err(e[r][t], ref_E))


@pytest.mark.parametrize("nrhs,mesh", [(1, (36, 44, 52)), (3, (40, 48, 56)), (2, (38, 44, 50))])
def test_tma_region_loads_equal_plain_loads(cuda_lib, nrhs, mesh, monkeypatch):
    """The tiled gathers stage the region of a tile that does not wrap around the box
    with cp.async.bulk.tensor copies (FP32 grid, and the double-float FP64 potential);
    the field and potential equal those of the same call with plain loads
    (IBPME_NO_TMA) to the rounding of the spread's atomics (their order differs from
    call to call), in both precisions, with tiles that wrap (a sphere across the corner)
    served by the plain loads in the same launch.  N_x = 38 has FP32 rows that are no
    multiple of 16 bytes: its FP32 gathers keep the plain loads.  A second call on each
    context reports any refused copy or expired wait of the first."""
    ib = cuda_lib
    x, box = _dense_surfaces(70 + nrhs)
    n = x.shape[0]
    q = np.stack([random_neutral_charges(n, 300 + r) for r in range(nrhs)])
    kw = dict(box=box, mesh=mesh, tol=1e-6, bead_radius=0.01, eps_f=0.8, max_rhs=4)
    out = {}
    for tma in (True, False):
        if tma:
            monkeypatch.delenv("IBPME_NO_TMA", raising=False)
        else:
            monkeypatch.setenv("IBPME_NO_TMA", "1")
        for prec in (ib.IBPME_FP64, ib.IBPME_MIXED):
            ctx = ib.pme_setup(ib.make_params(precision=prec, **kw))
            try:
                out[tma, prec] = _field(ib, ctx, x, q, nrhs=nrhs)
                # the next call reports a refused tensor copy or an expired wait of this one
                _field(ib, ctx, x, q, nrhs=nrhs)
            finally:
                ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_NO_TMA", raising=False)
    for prec, bar in ((ib.IBPME_FP64, 1e-12), (ib.IBPME_MIXED, 2e-6)):
        (pt, et), (pp, ep) = out[True, prec], out[False, prec]
        for r in range(nrhs):
            assert rel_err(pt[r], pp[r]) < bar and rel_err(et[r], ep[r]) < bar, (prec, r)


def test_spectral_error_decays_exponentially_with_the_stencil_width(cuda_lib):
    """Sec. III.D.2: with xi and the mesh fixed and eta = h^2 xi^2 P / pi, the window
    truncation and quadrature errors are both e^{-pi P / 2}.  The FP64 potential of a
    162-bead sphere with 40 ions against the oracle, P = 4 .. 10, at an Ewald tolerance
    of 1e-12 (every other error far below): the error falls at every step, by about
    e^{pi/2} per unit of P."""
    ib = cuda_lib
    rng = np.random.default_rng(12)
    from workloads import geometry as Gm
    sphere = Gm.icosphere(2) + 4.0
    ions = rng.uniform(0.0, 8.0, size=(40, 3))
    x = np.concatenate([sphere, ions])
    n = x.shape[0]
    q = random_neutral_charges(n, 13)
    box = np.array([8.0, 8.0, 8.0])
    ref = o.potential(x, q, box, 0.1, 1.0)
    errs = []
    for P in range(4, 11):
        ctx = ib.pme_setup(ib.make_params(box=box, mesh=(48, 48, 48), tol=1e-12, P=P, bead_radius=0.1, eps_f=1.0,
                                          precision=ib.IBPME_FP64))
        try:
            psi, _ = _field(ib, ctx, x, q, with_E=False)
        finally:
            ib.pme_destroy(ctx)
        errs.append(rel_err(psi[0], ref))
    for a, b in zip(errs, errs[1:]):
        assert b < a, errs
    rate = (math.log(errs[0]) - math.log(errs[-1])) / (len(errs) - 1)
    assert 1.1 < rate < 2.2, (rate, errs)   # pi / 2 = 1.57


def test_pme_field_multi_rhs_host_pointers_and_edge_cases(cuda_lib):
    ib = cuda_lib
    x, q0, box, a, eps, mesh, tol = _field_case("sphere162")
    n = x.shape[0]
    qs = np.stack([q0, random_neutral_charges(n, 7), random_neutral_charges(n, 8)])
    ctx = ib.pme_setup(ib.make_params(box=box, mesh=mesh, tol=tol, bead_radius=a, eps_f=eps))
    psi3, E3 = _field(ib, ctx, x, qs, nrhs=3)
    for r in range(3):
        psi1, E1 = _field(ib, ctx, x, qs[r])
        assert rel_err(psi3[r], psi1[0]) < 1e-12 and rel_err(E3[r], E1[0]) < 1e-12
    # host (numpy) arrays go through the library's staging
    psi_h = np.zeros((3, n))
    E_h = np.zeros((3, n, 3))
    ib.pme_field(ctx, n, np.ascontiguousarray(x), np.ascontiguousarray(qs), 3, psi_h, E_h)
    assert rel_err(psi_h, psi3) < 1e-12 and rel_err(E_h, E3) < 1e-12
    # empty input is a no-op
    ib.pme_field(ctx, 0, None, None, 1, None, None)
    # a single bead: only itself and its images
    one = np.array([[3.0, 4.0, 5.0]])
    psi1, _ = _field(ib, ctx, one, np.array([1.5]))
    assert rel_err(psi1[0], o.potential(one, [1.5], box, a, eps)) < FP64_RTOL
    # non-finite positions are reported, not propagated
    bad = x.copy()
    bad[5, 1] = np.nan
    with pytest.raises(ib.IbpmeError) as e:
        _field(ib, ctx, bad, q0)
    assert e.value.status == ib.IBPME_ERR_NONFINITE
    # nrhs beyond the context capacity
    with pytest.raises(ib.IbpmeError):
        _field(ib, ctx, x, np.zeros((4, n)), nrhs=4)
    ib.pme_destroy(ctx)


def _solve(ib, ctx, s, prec=-1, rtol=1e-6, guess=None, restart=50):
    import torch
    n, nb, R = s.n, s.n_bodies, s.nrhs
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    q = torch.zeros((R, n), dtype=torch.float64, device="cuda")
    mode = ib.IBPME_GUESS_ZERO
    if guess is not None:
        q.copy_(torch.as_tensor(np.array(np.broadcast_to(guess, (R, n)))))
        mode = ib.IBPME_GUESS_USER
    psi = torch.zeros((R, nb), dtype=torch.float64, device="cuda")
    S = torch.zeros((R, nb, 3), dtype=torch.float64, device="cuda")
    status, st = ib.induced_charge_solve(ctx, n, cuda(s.x), bodies, cuda(s.E0), R,
                                         ib.make_opts(rtol=rtol, guess=mode, precision=prec, restart=restart),
                                         q, psi, S)
    torch.cuda.synchronize()
    return status, st, q.cpu().numpy(), psi.cpu().numpy(), S.cpu().numpy()


def _check_solution(s, q, psi, S, bar, M=None):
    qr, psr = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0, s.box, s.a, s.eps, M=M)
    Sr = np.stack([o.dipoles(s.x, s.X, s.body_offsets, qr[r], s.box) for r in range(s.nrhs)])
    rel = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    for r in range(s.nrhs):
        assert rel_err(q[r], qr[r]) < bar, ("q", r, rel_err(q[r], qr[r]))
        # Psi - Psi_0 can vanish by symmetry (a neutral sphere): measure it on the scale of
        # the bead potentials it is balanced against, max(|Psi - Psi_0|, |r.E0|)
        pscale = max(np.abs(psr[r]).max(), np.abs(rel @ s.E0[r]).max())
        assert np.abs(psi[r] - psr[r]).max() < bar * pscale, ("psi", r, np.abs(psi[r] - psr[r]).max() / pscale)
        assert rel_err(S[r], Sr[r]) < bar, ("S", r, rel_err(S[r], Sr[r]))
    return qr, psr, Sr


@pytest.mark.parametrize("a", [0.12, 0.2])
def test_compact_bodies_match_the_table_path(cuda_lib, a, monkeypatch):
    """Intra-body pairs of compact bodies evaluated directly (FP32 for the inner
    operator, double-float for the FP64 operator and the field) against the same
    calls with every pair in the table: solves in both precisions, bead forces,
    body forces, torques and energy.  With a = 0.2 neighbouring beads of a body
    overlap (r < 2a), which takes the exact kernel."""
    import torch
    ib = cuda_lib
    s = C.small_system(seed=61, n_bodies=3, level=2, n_ions=40, L=9.0, a=a, mesh=(48, 48, 48), tol=1e-7, nrhs=2)
    out = {}
    q_common = None
    for compact in (False, True):
        if compact:
            monkeypatch.delenv("IBPME_NO_COMPACT", raising=False)
        else:
            monkeypatch.setenv("IBPME_NO_COMPACT", "1")
        for prec in ("fp64", "mixed"):
            ctx = context(ib, s, precision=prec)
            try:
                bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
                q = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
                psi = torch.zeros((2, s.n_bodies), dtype=torch.float64, device="cuda")
                S = torch.zeros((2, s.n_bodies, 3), dtype=torch.float64, device="cuda")
                status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 2,
                                                     ib.make_opts(rtol=1e-10), q, psi, S)
                torch.cuda.synchronize()
                assert status == ib.IBPME_OK and st.rel_residual <= 1e-10
                if q_common is None:
                    q_common = q[0:1].clone()
                f = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
                F = torch.zeros((s.n_bodies, 3), dtype=torch.float64, device="cuda")
                L = torch.zeros((s.n_bodies, 3), dtype=torch.float64, device="cuda")
                U = torch.zeros(1, dtype=torch.float64, device="cuda")
                ib.body_force_torque(ctx, s.n, cuda(s.x), q_common, bodies, cuda(s.E0[:1]), f, F, L, U)
                torch.cuda.synchronize()
                out[compact, prec] = [t.cpu().numpy() for t in (q, psi, S, f, F, L, U)]
            finally:
                ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_NO_COMPACT", raising=False)
    for prec in ("fp64", "mixed"):
        t, d = out[True, prec], out[False, prec]
        # forces only from the FP64 context: the mixed context's force pass runs its mesh
        # in FP32, whose atomic sums vary from run to run near 1e-7
        checks = (("q", 0, 1e-8), ("S", 2, 1e-8))
        if prec == "fp64":
            checks += (("f", 3, 1e-9), ("F", 4, 1e-9), ("L", 5, 1e-9), ("U", 6, 1e-10))
        for name, i, bar in checks:
            assert rel_err(t[i], d[i]) < bar, (prec, name, rel_err(t[i], d[i]))
        assert np.abs(t[1] - d[1]).max() < 1e-8 * max(np.abs(d[1]).max(), 1.0), (prec, "psi")
    q, psi, S = out[True, "fp64"][:3]
    _check_solution(s, q, psi, S, FP64_RTOL)


def test_solve_single_sphere_fp64(cuda_lib):
    ib = cuda_lib
    s = C.config1()
    ctx = context(ib, s)
    status, st, q, psi, S = _solve(ib, ctx, s)
    assert status == ib.IBPME_OK and st.rel_residual <= 1e-6
    _check_solution(s, q, psi, S, FP64_RTOL)
    # Sec. IV.A: dipole along E0, a little above 4 pi a^3 eps E0
    assert abs(S[0, 0, 0]) < 1e-8 * S[0, 0, 2] and abs(S[0, 0, 1]) < 1e-8 * S[0, 0, 2]
    assert 0.0 < S[0, 0, 2] / (4 * math.pi) - 1.0 < 0.3
    ib.pme_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_bodies_ions_three_fields(cuda_lib, prec):
    ib = cuda_lib
    s = C.small_system(seed=11, n_bodies=3, level=2, n_ions=25, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7,
                       nrhs=3)
    ctx = context(ib, s, precision=prec)
    status, st, q, psi, S = _solve(ib, ctx, s)
    assert status == ib.IBPME_OK and st.rel_residual <= 1e-6
    _check_solution(s, q, psi, S, FP64_RTOL if prec == "fp64" else MIXED_RTOL)
    # the constraint Sigma q = Q holds for every body to the solve's residual
    rel = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    for r in range(3):
        bnorm = np.sqrt(np.sum((rel @ s.E0[r]) ** 2) + np.sum(s.Q ** 2))
        assert np.max(np.abs(np.add.reduceat(q[r], s.body_offsets[:-1]) - s.Q)) <= 1e-6 * bnorm
    ib.pme_destroy(ctx)


def test_solve_charged_sphere_with_ions_full_size_mixed(cuda_lib):
    """The 642-bead sphere with 2,050 ions in L = 30 on 128^3 (mixed precision), solved
    from the uniform initial charge, against the dense FP64 oracle solve."""
    ib = cuda_lib
    s = C.config2()
    ctx = context(ib, s)
    status, st, q, psi, S = _solve(ib, ctx, s, guess=s.q_guess)
    assert status == ib.IBPME_OK and st.rel_residual <= 1e-6
    _check_solution(s, q, psi, S, MIXED_RTOL)
    ib.pme_destroy(ctx)


def test_mixed_warm_start_checks_once_in_fp64(cuda_lib):
    """A mixed solve from a nearby guess (the previous step's charges, perturbed):
    the first residual takes the FP32 mesh, one FP64 residual after the correction
    confirms convergence, and the charges still match the dense FP64 oracle.  A
    second context then solves the 2,050-ion system from the uniform guess, where
    the FP32 start is too coarse for the first FP64 check: the solve refines on and
    converges all the same."""
    ib = cuda_lib
    s = C.small_system(seed=13, n_bodies=3, level=2, n_ions=25, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7)
    ctx = context(ib, s, precision="mixed")
    try:
        status, st, q, psi, S = _solve(ib, ctx, s, rtol=1e-9)
        assert status == ib.IBPME_OK
        rng = np.random.default_rng(5)
        guess = q[0] * (1.0 + 1e-4 * rng.standard_normal(s.n))
        status, st, q, psi, S = _solve(ib, ctx, s, rtol=1e-6, guess=guess)
        assert status == ib.IBPME_OK and st.rel_residual <= 1e-6
        assert st.matvecs_fp64 == 1 and st.outer == 1, (st.matvecs_fp64, st.outer)
        _check_solution(s, q, psi, S, MIXED_RTOL)
    finally:
        ib.pme_destroy(ctx)
    s2 = C.config2()
    ctx = context(ib, s2)
    try:
        for _ in range(2):   # the second solve starts from the FP64 residual
            status, st, q, psi, S = _solve(ib, ctx, s2, guess=s2.q_guess)
            assert status == ib.IBPME_OK and st.rel_residual <= 1e-6
        _check_solution(s2, q, psi, S, MIXED_RTOL)
    finally:
        ib.pme_destroy(ctx)


def test_forces_torques_energy_fp64(cuda_lib):
    import torch
    ib = cuda_lib
    s = C.small_system(seed=21, n_bodies=2, level=2, n_ions=12, L=8.0, a=0.14, mesh=(48, 48, 48), tol=1e-8)
    M = o.M_dense(s.x, s.box, s.a, s.eps)
    qr, psr = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps, M=M)
    f_ref = o.bead_forces(s.x, qr, s.E0[0], s.box, s.a, s.eps)
    F_ref, L_ref = o.body_force_torque(s.x, s.X, s.body_offsets, f_ref, s.box)
    U_ref = o.energy(s.X, s.Q, psr, o.dipoles(s.x, s.X, s.body_offsets, qr, s.box), s.E0[0])
    ctx = context(ib, s)
    n, nb = s.n, s.n_bodies
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
    f = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    F = torch.zeros((nb, 3), dtype=torch.float64, device="cuda")
    L = torch.zeros((nb, 3), dtype=torch.float64, device="cuda")
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    ib.body_force_torque(ctx, n, cuda(s.x), cuda(qr), bodies, cuda(s.E0[0]), f, F, L, U)
    torch.cuda.synchronize()
    assert rel_err(f.cpu().numpy(), f_ref) < FP64_RTOL
    assert rel_err(F.cpu().numpy(), F_ref) < FP64_RTOL
    # a torque is a sum of cancelling moments: measure it on the scale sum_j |r_ij| |f_ij|
    r = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    moment = np.add.reduceat(np.linalg.norm(r, axis=1) * np.linalg.norm(f_ref, axis=1), s.body_offsets[:-1])
    assert np.max(np.abs(L.cpu().numpy() - L_ref)) < FP64_RTOL * moment.max()
    assert abs(U.item() - U_ref) < FP64_RTOL * abs(U_ref)
    ib.pme_destroy(ctx)


def test_bd_step_matches_oracle(cuda_lib):
    import torch
    ib = cuda_lib
    s = C.small_system(seed=4, n_bodies=2, level=1, n_ions=40, L=8.0, a=0.15, mesh=(32, 32, 32), tol=1e-6)
    x = s.x.copy()
    x[-1] = x[-2] + [0.1, 0.05, 0.0]     # two overlapping ions: hard-sphere push
    X = s.X.copy()
    X[-1] = x[-1]
    rng = np.random.default_rng(9)
    f = rng.normal(size=(s.n, 3))
    dt, gamma, kT, seed, step = 1e-3, 1.3, 0.9, 12345, 17
    f_tot = f + o.hard_sphere_forces(x, s.body_offsets, s.box, s.a, gamma, dt)
    xr, Xr = o.bd_step(x, X, s.body_offsets, f_tot, s.box, s.a, dt, gamma=gamma, kT=kT, seed=seed, step=step)
    ctx = context(ib, s)
    bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(X), cuda(s.Q))
    xo = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    Xo = torch.zeros((s.n_bodies, 3), dtype=torch.float64, device="cuda")
    ib.ibpme_bd_step(ctx, s.n, cuda(x), bodies, cuda(f), dt, gamma, kT, seed, step, xo, Xo)
    torch.cuda.synchronize()
    # positions are compared modulo the box (the library works with wrapped positions)
    dx = o.min_image(xo.cpu().numpy() - xr, s.box)
    dX = o.min_image(Xo.cpu().numpy() - Xr, s.box)
    assert np.max(np.abs(dx)) < 1e-12 and np.max(np.abs(dX)) < 1e-12
    ib.pme_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bd_advance_matches_oracle_and_the_three_calls(cuda_lib, prec):
    """ibpme_bd_advance (solve + forces + BD step in one call) against the dense FP64
    oracle (charges, bead forces, body forces, torques, energy; then the BD step of
    the oracle from the oracle's forces) and against induced_charge_solve,
    body_force_torque and ibpme_bd_step called in sequence.  Its forces gather the
    field from the FP64 mesh of the solve's final residual, so they meet the FP64
    bar also in a mixed context."""
    import torch
    ib = cuda_lib
    s = C.small_system(seed=23, n_bodies=2, level=2, n_ions=12, L=8.0, a=0.14, mesh=(48, 48, 48), tol=1e-8)
    n, nb = s.n, s.n_bodies
    dt, gamma, kT, seed, step = 1e-3, 1.1, 0.8, 777, 3
    qr, psr = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
    f_ref = o.bead_forces(s.x, qr, s.E0[0], s.box, s.a, s.eps)
    F_ref, L_ref = o.body_force_torque(s.x, s.X, s.body_offsets, f_ref, s.box)
    U_ref = o.energy(s.X, s.Q, psr, o.dipoles(s.x, s.X, s.body_offsets, qr, s.box), s.E0[0])
    f_tot = f_ref + o.hard_sphere_forces(s.x, s.body_offsets, s.box, s.a, gamma, dt)
    xr, Xr = o.bd_step(s.x, s.X, s.body_offsets, f_tot, s.box, s.a, dt, gamma=gamma, kT=kT, seed=seed, step=step)
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device="cuda")
    ctx = context(ib, s, precision=prec)
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        opts = ib.make_opts(rtol=1e-10)
        # one call
        q, psi, f, F, L, U, xo, Xo = z(1, n), z(1, nb), z(n, 3), z(nb, 3), z(nb, 3), z(1), z(n, 3), z(nb, 3)
        status, st = ib.ibpme_bd_advance(ctx, n, cuda(s.x), bodies, cuda(s.E0[0]), opts, q, dt, gamma, kT, seed,
                                         step, F, L, xo, Xo, psi_out=psi, f_bead=f, U=U)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= 1e-10
        one = [t.cpu().numpy() for t in (q, psi, f, F, L, U, xo, Xo)]
        # three calls
        q3, psi3, f3, F3, L3, U3, xo3, Xo3 = z(1, n), z(1, nb), z(n, 3), z(nb, 3), z(nb, 3), z(1), z(n, 3), z(nb, 3)
        status, st = ib.induced_charge_solve(ctx, n, cuda(s.x), bodies, cuda(s.E0[:1]), 1, opts, q3, psi3)
        assert status == ib.IBPME_OK
        ib.body_force_torque(ctx, n, cuda(s.x), q3[0], bodies, cuda(s.E0[0]), f3, F3, L3, U3)
        ib.ibpme_bd_step(ctx, n, cuda(s.x), bodies, f3, dt, gamma, kT, seed, step, xo3, Xo3)
        torch.cuda.synchronize()
        three = [t.cpu().numpy() for t in (q3, psi3, f3, F3, L3, U3, xo3, Xo3)]
    finally:
        ib.pme_destroy(ctx)
    q, psi, f, F, L, U, xo, Xo = one
    assert rel_err(q[0], qr) < FP64_RTOL
    assert rel_err(f, f_ref) < FP64_RTOL and rel_err(F, F_ref) < FP64_RTOL
    r = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    moment = np.add.reduceat(np.linalg.norm(r, axis=1) * np.linalg.norm(f_ref, axis=1), s.body_offsets[:-1])
    assert np.max(np.abs(L - L_ref)) < FP64_RTOL * moment.max()
    assert abs(U[0] - U_ref) < FP64_RTOL * abs(U_ref)
    # the step moves by F dt / gamma + noise: compare the displacement with the oracle's
    disp_ref = o.min_image(xr - s.x, s.box)
    assert np.max(np.abs(o.min_image(xo - xr, s.box))) < FP64_RTOL * np.abs(disp_ref).max()
    assert np.max(np.abs(o.min_image(Xo - Xr, s.box))) < FP64_RTOL * np.abs(disp_ref).max()
    # against the three calls: the same solve; the forces agree to the three-call
    # path's mesh precision
    bar = 1e-9 if prec == "fp64" else MIXED_RTOL
    assert rel_err(q[0], three[0][0]) < 1e-9 and rel_err(psi[0], three[1][0]) < 1e-7
    assert rel_err(f, three[2]) < bar and rel_err(F, three[3]) < bar
    assert abs(U[0] - three[5][0]) < bar * abs(U[0])
    assert np.max(np.abs(o.min_image(xo - three[6], s.box))) < bar * np.abs(disp_ref).max()


def test_full_size_lattice_field_sampled(cuda_lib):
    """64 spheres + 100,000 ions on 256^3 in mixed precision: the potential at a
    seeded sample of beads against the oracle's exact Ewald sum at those beads."""
    ib = cuda_lib
    s = C.config3()
    q = random_neutral_charges(s.n, 3)
    ctx = context(ib, s)
    psi, _ = _field(ib, ctx, s.x, q, with_E=False)
    t = np.random.default_rng(0).choice(s.n, size=64, replace=False).astype(np.int32)
    ref = o.potential(s.x, q, s.box, s.a, s.eps, targets=t, xi=0.5)   # small xi: few k-vectors
    assert rel_err(psi[0][t], ref) < MIXED_RTOL
    ib.pme_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_body_block_preconditioner_same_solution_fewer_iterations(cuda_lib, prec):
    """The body-block right preconditioner changes the Krylov iteration, not the
    answer: with and without it the solution matches the oracle at the same bar,
    and the preconditioned solve needs far fewer iterations (bodies of the same
    shape share one cached inverse)."""
    import torch
    ib = cuda_lib
    s = C.small_system(seed=21, n_bodies=3, level=2, n_ions=30, L=9.0, a=0.12, mesh=(48, 48, 48), tol=1e-7,
                       nrhs=2)
    ctx = context(ib, s, precision=prec)
    try:
        res = {}
        for mode in (ib.IBPME_PRECOND_NONE, ib.IBPME_PRECOND_BODY, ib.IBPME_PRECOND_BODY):
            bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
            q = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
            psi = torch.zeros((2, s.n_bodies), dtype=torch.float64, device="cuda")
            S = torch.zeros((2, s.n_bodies, 3), dtype=torch.float64, device="cuda")
            status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 2,
                                                 ib.make_opts(rtol=1e-8, precond=mode), q, psi, S)
            torch.cuda.synchronize()
            assert status == ib.IBPME_OK and st.rel_residual <= 1e-8
            res[mode] = (st.iters, q.cpu().numpy(), psi.cpu().numpy(), S.cpu().numpy())
        bar = FP64_RTOL if prec == "fp64" else MIXED_RTOL
        for mode in (ib.IBPME_PRECOND_NONE, ib.IBPME_PRECOND_BODY):
            _check_solution(s, res[mode][1], res[mode][2], res[mode][3], bar)
        it_none, it_body = res[ib.IBPME_PRECOND_NONE][0], res[ib.IBPME_PRECOND_BODY][0]
        assert it_body * 3 <= it_none, (it_none, it_body)
        # the two preconditioned solves agree (the second reuses the cached inverses)
        assert rel_err(res[ib.IBPME_PRECOND_BODY][1], res[ib.IBPME_PRECOND_NONE][1]) < (1e-6 if prec == "fp64" else 1e-4)
    finally:
        ib.pme_destroy(ctx)


def test_fp64_mesh_double_float_transforms_reach_tight_tolerance(cuda_lib):
    """On a power-of-two FP64 mesh the transforms run in double-float arithmetic
    (about 48 significant bits); with the Ewald tolerance at 1e-10 (P = 15,
    64^3; the truncation bounds of Sec. III.D.2 then leave a few 1e-9 over 400
    charges in the potential, and about k_c times more in the field) the
    potential matches the oracle below 1e-8 and the field below 1e-7, 1,000 and
    100 times under the 1e-5 FP64 bar: the transforms are not the accuracy limit."""
    ib = cuda_lib
    rng = np.random.default_rng(61)
    box = np.array([8.0, 8.0, 8.0])
    n = 400
    x = rng.uniform(0, 1, size=(n, 3)) * box
    q = random_neutral_charges(n, 62)
    ctx = ib.pme_setup(ib.make_params(box=box, mesh=(64, 64, 64), tol=1e-10, bead_radius=0.1, eps_f=0.9,
                                      precision=ib.IBPME_FP64))
    try:
        assert ib.ibpme_get_params(ctx).P == 15
        psi, E = _field(ib, ctx, x, q)
        ref_psi, ref_E = o.potential(x, q, box, 0.1, 0.9, field=True)
        assert rel_err(psi[0], ref_psi) < 1e-8, rel_err(psi[0], ref_psi)
        assert rel_err(E[0], ref_E) < 1e-7, rel_err(E[0], ref_E)
    finally:
        ib.pme_destroy(ctx)


def test_preconditioner_skips_configurations_with_large_bodies(cuda_lib):
    """In a batch, a configuration holding a body above the block limit (8,192
    beads) runs unpreconditioned while the others are preconditioned; every
    configuration still matches its single-system solve."""
    import torch
    from workloads import geometry as geo
    ib = cuda_lib
    L = 12.0
    big = geo.ellipsoid(8400, [1.0, 1.5, 2.0]) + L / 2
    small = geo.icosphere(2) * 0.8 + L / 2
    E0 = np.eye(3)
    a = 0.45 * min(geo.min_spacing(big), geo.min_spacing(small))
    parts = [C.assemble("big", [big], [], [], [0.0], [L] * 3, a, 1.0, E0, mesh=(64, 64, 64), tol=1e-6),
             C.assemble("small", [small], [], [], [0.0], [L] * 3, a, 1.0, E0, mesh=(64, 64, 64), tol=1e-6)]
    assert parts[0].n > 8192
    s, cfg = C.stack(parts)
    ctx = context(ib, s, precision="fp64")
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        q = torch.zeros((3, s.n), dtype=torch.float64, device="cuda")
        status, st = ib.induced_charge_solve_batch(ctx, s.n, cuda(s.x), bodies, cfg, cuda(s.E0), 3,
                                                   ib.make_opts(rtol=1e-8), q)
        assert status == ib.IBPME_OK
        got = q.cpu().numpy()
        lo = 0
        for p in parts:
            bp = ib.Bodies(cuda(p.body_offsets.astype(np.int32)), cuda(p.X), cuda(p.Q))
            qs = torch.zeros((3, p.n), dtype=torch.float64, device="cuda")
            status1, _ = ib.induced_charge_solve(ctx, p.n, cuda(p.x), bp, cuda(p.E0), 3,
                                                 ib.make_opts(rtol=1e-8, precond=ib.IBPME_PRECOND_NONE), qs)
            assert status1 == ib.IBPME_OK
            assert rel_err(got[:, lo:lo + p.n], qs.cpu().numpy()) < 1e-6
            lo += p.n
    finally:
        ib.pme_destroy(ctx)


def test_preconditioner_covers_bodies_of_thousands_of_beads(cuda_lib):
    """Bodies of 1,500 and 3,000 beads (an ellipsoid and a rod, above the former
    1,024-bead limit) get their block inverse from the blocked Gauss-Jordan kernel:
    the preconditioned solve matches the unpreconditioned one and needs at most a
    third of its iterations."""
    import torch
    from workloads import geometry as geo
    ib = cuda_lib
    L = 14.0
    ell = geo.ellipsoid(1500, [1.0, 1.5, 2.0]) + [4.0, 4.0, 7.0]
    rod = geo.spherocylinder(3000, 4.0, 0.8) + [10.0, 10.0, 7.0]
    a = 0.45 * min(geo.min_spacing(ell), geo.min_spacing(rod))
    s = C.assemble("large", [ell, rod], [], [], [0.5, -0.5], [L] * 3, a, 1.0, [[0.3, 0.2, 1.0]],
                   mesh=(64, 64, 64), tol=1e-6)
    ctx = context(ib, s, precision="mixed")
    try:
        out = {}
        for mode in (ib.IBPME_PRECOND_BODY, ib.IBPME_PRECOND_NONE):
            bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
            q = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
            status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 1,
                                                 ib.make_opts(rtol=1e-8, precond=mode), q)
            torch.cuda.synchronize()
            assert status == ib.IBPME_OK and st.rel_residual <= 1e-8
            out[mode] = (st.iters, q.cpu().numpy())
        it_body, it_none = out[ib.IBPME_PRECOND_BODY][0], out[ib.IBPME_PRECOND_NONE][0]
        assert it_body * 3 <= it_none, (it_body, it_none)
        assert rel_err(out[ib.IBPME_PRECOND_BODY][1], out[ib.IBPME_PRECOND_NONE][1]) < 1e-5
    finally:
        ib.pme_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_free_bead_operator_matches_full_operator(cuda_lib, prec, monkeypatch):
    """The Krylov operator evaluates the free beads (beads of multi-bead bodies) alone:
    their own stencils, the table's pairs between two free beads and the compact bodies.
    Against the same solves with every bead in every evaluation (ions at zero charge):
    bodies close enough for pairs between bodies inside r_c, ions, two fields, and the
    oracle's dense solution; iteration counts stay within one of each other."""
    import torch
    ib = cuda_lib
    s = C.small_system(seed=62, n_bodies=4, level=2, n_ions=40, L=8.0, a=0.12, mesh=(48, 48, 48), tol=1e-7, nrhs=2)
    # pairs of beads of different multi-bead bodies inside r_c exist (the free-free table is used)
    ctx = context(ib, s, precision=prec)
    rc = ib.ibpme_get_params(ctx).r_cut
    ib.pme_destroy(ctx)
    bid = o.body_index(s.body_offsets)
    body = np.diff(s.body_offsets)[bid] > 1
    xb, bb = s.x[body], bid[body]
    d = o.min_image(xb[:, None, :] - xb[None, :, :], s.box)
    inside = (np.sqrt((d * d).sum(axis=2)) < rc) & (bb[:, None] != bb[None, :])
    assert inside.sum() > 100
    out = {}
    for full in (True, False):
        if full:
            monkeypatch.setenv("IBPME_FULL_OPERATOR", "1")
        else:
            monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
        ctx = context(ib, s, precision=prec)
        try:
            bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
            q = torch.zeros((2, s.n), dtype=torch.float64, device="cuda")
            psi = torch.zeros((2, s.n_bodies), dtype=torch.float64, device="cuda")
            S = torch.zeros((2, s.n_bodies, 3), dtype=torch.float64, device="cuda")
            status, st = ib.induced_charge_solve(ctx, s.n, cuda(s.x), bodies, cuda(s.E0), 2,
                                                 ib.make_opts(rtol=1e-10, precond=ib.IBPME_PRECOND_NONE), q, psi, S)
            torch.cuda.synchronize()
            assert status == ib.IBPME_OK and st.rel_residual <= 1e-10
            out[full] = (st.iters, q.cpu().numpy(), psi.cpu().numpy(), S.cpu().numpy())
        finally:
            ib.pme_destroy(ctx)
    monkeypatch.delenv("IBPME_FULL_OPERATOR", raising=False)
    (it_f, qf, pf, Sf), (it_s, qs, ps, Ss) = out[True], out[False]
    assert abs(it_f - it_s) <= 1, (it_f, it_s)
    assert rel_err(qs, qf) < 1e-8 and rel_err(Ss, Sf) < 1e-8
    assert np.abs(ps - pf).max() < 1e-8 * max(np.abs(pf).max(), 1.0)
    _check_solution(s, qs, ps, Ss, FP64_RTOL)
