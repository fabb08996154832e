"""The 64-sphere lattice with 100,000 ions at full size (141,088 beads, 256^3 mesh,
mixed precision): one Brownian-dynamics step of the method (Sec. V.A) through
ibpme_bd_advance, checked against the FP64 oracle at a seeded sample of beads.

The oracle cannot solve a 41,152-unknown saddle system, so the solve is judged by
the equations it must satisfy: the oracle's exact Ewald sum of the GPU's charges
evaluated at the sampled beads fulfils the saddle rows of Eq. saddle
((M q)_alpha = (Psi - Psi_0)_i + r_alpha . E0 on body beads), every body carries
its net charge and every ion its own.  The bead forces of Eq. beadforce are the
oracle's q (E0 + E) at the sampled beads, and the step's new positions are the
oracle's Euler-Maruyama step (Eq. forward) from the GPU's bead forces at every
sampled bead that has no hard-sphere contact.
"""
import numpy as np
import pytest

import oracle as o
from helpers import MIXED_RTOL, context, cuda, rel_err
from workloads import configs as C

pytestmark = pytest.mark.gpu

DT, GAMMA, KT, SEED, STEP = 1e-3, 1.0, 1.0, 2024, 5


def _in_contact(s, bid):
    """Beads with a bead of another body closer than 2a (the only beads that feel the
    hard-sphere pair forces of Eq. hardsphereFD), from a periodic k-d tree."""
    from scipy.spatial import cKDTree

    xw = s.x - s.box * np.floor(s.x / s.box)
    xw = np.where(xw >= s.box, xw - s.box, xw)
    pairs = cKDTree(xw, boxsize=s.box).query_pairs(2 * s.a, output_type="ndarray")
    pairs = pairs[bid[pairs[:, 0]] != bid[pairs[:, 1]]]
    hit = np.zeros(s.n, dtype=bool)
    hit[pairs.ravel()] = True
    return hit


def test_full_size_lattice_bd_advance_sampled(cuda_lib):
    import torch

    ib = cuda_lib
    s = C.config3()
    n, nb = s.n, s.n_bodies
    n_body_beads = int(s.body_offsets[64])
    assert n == 141_088 and n_body_beads == 41_088 and nb == 64 + 100_000
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device="cuda")
    ctx = context(ib, s, precision="mixed", max_rhs=1)
    try:
        bodies = ib.Bodies(cuda(s.body_offsets.astype(np.int32)), cuda(s.X), cuda(s.Q))
        q, psi, f, F, L, U, xo, Xo = z(1, n), z(1, nb), z(n, 3), z(nb, 3), z(nb, 3), z(1), z(n, 3), z(nb, 3)
        status, st = ib.ibpme_bd_advance(ctx, n, cuda(s.x), bodies, cuda(s.E0[0]), ib.make_opts(rtol=1e-6), q[0],
                                         DT, GAMMA, KT, SEED, STEP, F, L, xo, Xo, psi_out=psi[0], f_bead=f, U=U)
        torch.cuda.synchronize()
        assert status == ib.IBPME_OK and st.rel_residual <= 1e-6, (status, st.rel_residual)
        q, psi, f, F, L, xo, Xo = (t.cpu().numpy() for t in (q[0], psi[0], f, F, L, xo, Xo))
    finally:
        ib.pme_destroy(ctx)

    # constraint rows of Eq. saddle: each body's charges sum to its net charge; ions keep theirs
    sums = np.add.reduceat(q, s.body_offsets[:-1])
    assert np.max(np.abs(sums - s.Q)) < 1e-9
    assert np.array_equal(q[n_body_beads:], s.Q[64:])

    rng = np.random.default_rng(77)
    tb = np.sort(rng.choice(n_body_beads, size=48, replace=False))
    ti = np.sort(rng.choice(np.arange(n_body_beads, n), size=48, replace=False))
    t = np.concatenate([tb, ti]).astype(np.int32)
    Mq, E = o.potential(s.x, q, s.box, s.a, s.eps, targets=t, field=True, xi=0.5)
    bid = o.body_index(s.body_offsets)
    r = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    # potential rows on the sampled body beads: (M q)_a - (Psi - Psi_0)_i - r_a . E0 = 0
    rows = Mq[:48] - psi[bid[tb]] - r[tb] @ s.E0[0]
    scale = max(np.abs(Mq[:48]).max(), np.abs(r[tb] @ s.E0[0]).max())
    assert np.abs(rows).max() < MIXED_RTOL * scale, np.abs(rows).max() / scale
    # ions: Psi - Psi_0 of a one-bead body is its own potential
    assert rel_err(psi[bid[ti]], Mq[48:]) < MIXED_RTOL

    # bead forces f = q (E0 + E) (Eq. beadforce) at every sampled bead; the lattice is a
    # mixed-precision workload at Ewald tolerance 1e-6, whose truncation bounds the field
    # near 1e-4 of its largest value (the FP64 bar holds at tolerance 1e-8), so the
    # mixed-precision bar applies
    f_ref = q[t][:, None] * (s.E0[0][None, :] + E)
    assert rel_err(f[t], f_ref) < MIXED_RTOL, rel_err(f[t], f_ref)
    # body forces and torques of the spheres from the GPU's own bead forces (Sec. III.C)
    F_ref, L_ref = o.body_force_torque(s.x[:n_body_beads], s.X[:64], s.body_offsets[:65], f[:n_body_beads], s.box)
    assert rel_err(F[:64], F_ref) < 1e-9 and rel_err(L[:64], L_ref) < 1e-9
    assert np.allclose(F[64:], f[n_body_beads:], rtol=1e-12, atol=0)

    # the BD step (Eq. forward) from the GPU's bead forces, at sampled beads without
    # hard-sphere contacts (for a body bead: none of its body's beads in contact)
    xr, Xr = o.bd_step(s.x, s.X, s.body_offsets, f, s.box, s.a, DT, gamma=GAMMA, kT=KT, seed=SEED, step=STEP)
    hit = _in_contact(s, bid)
    free = ~hit[ti]
    spheres = np.unique(bid[tb])
    sphere_hit = np.add.reduceat(hit[:n_body_beads].astype(int), s.body_offsets[:65][:-1]) > 0
    free_b = ~sphere_hit[bid[tb]]
    assert free.sum() >= 24 and free_b.sum() >= 24
    chk = np.concatenate([ti[free], tb[free_b]])
    disp = o.min_image(xr[chk] - s.x[chk], s.box)
    assert np.max(np.abs(o.min_image(xo[chk] - xr[chk], s.box))) < 1e-9 * np.abs(disp).max()
    sp = spheres[~sphere_hit[spheres]]
    assert np.max(np.abs(o.min_image(Xo[sp] - Xr[sp], s.box))) < 1e-9 * np.abs(disp).max()
