"""The oracle's warm-start features, targets and guess, pinned to geometry and
physics that fix them independently of their own code: the normals and curvature
of a sphere and of a cylinder, the twelve five-fold vertices of an icosphere, the
uniform-field response of an isolated conducting sphere (surface charge
3 eps E0 . n, so targets three times the normal-field feature), and the Coulomb
potential and field of the fixed charges near a body."""
import math

import numpy as np
import pytest

import oracle as o
from oracle import mlp_ref as M
from workloads import configs as C
from workloads import geometry as G


def _one_body(pts, L=30.0, a=0.05, eps=0.9, E0=(0.3, -0.4, 1.2), Q=0.0, mesh=96, tol=1e-6):
    s = C.assemble("one", [pts + L / 2], [], [], [Q], [L] * 3, a, eps, [list(E0)], mesh=(mesh,) * 3, tol=tol)
    return s


def _features(s):
    return M.warm_start_features(s.x, s.X, s.body_offsets, s.Q, s.E0[0], s.box, s.a, s.eps)


def test_sphere_features_follow_the_geometry():
    """An icosphere of radius 1 (642 beads) alone in a uniform field: normals
    radial to about a degree, curvature 1/R, f0 = cos of the angle to E0, f1 its sine, f2 = f0,
    no other charges, |r| = R everywhere, the twelve five-fold vertices singled out
    by the sixth-nearest distance, the smallest nearest distance the tessellation's
    minimum spacing."""
    pts = G.icosphere(3)
    s = _one_body(pts, Q=1.5)
    F, S = _features(s)
    N = len(pts)
    rhat = pts / np.linalg.norm(pts, axis=1)[:, None]
    E0 = s.E0[0]
    cos = rhat @ E0 / np.linalg.norm(E0)
    # normal: f0 = E0.n/|E0| and f1 = |E0 x n|/|E0| (no ions: S = eps A |E0|)
    A = 4 * math.pi / N
    assert abs(S[0] - s.eps * A * np.linalg.norm(E0)) < 1e-12 * S[0]
    assert np.max(np.abs(F[:, 0] - cos)) < 0.02 and np.median(np.abs(F[:, 0] - cos)) < 5e-3   # within ~1 degree
    assert np.max(np.abs(F[:, 0] ** 2 + F[:, 1] ** 2 - 1)) < 1e-12
    assert np.max(np.abs(F[:, 2] - cos)) < 1e-12          # r.E0 / (R |E0|) with <r.E0> = 0
    assert np.all(F[:, 3:6] == 0)                          # no other charges
    assert np.max(np.abs(F[:, 6] - 1.0)) < 0.03           # kappa R on a sphere
    assert np.max(np.abs(F[:, 7])) < 1e-12
    assert np.allclose(F[:, 8], 1.5 / (N * S[0])) and np.allclose(F[:, 9], 10 * s.a)
    h = math.sqrt(A)
    assert abs(F[:, 10].min() * h - G.min_spacing(pts)) < 1e-12
    five = np.sort(np.argsort(F[:, 11])[-12:])
    assert np.array_equal(five, np.arange(12))            # the icosahedron's vertices come first
    assert F[12:, 11].max() < 0.5 * F[:12, 11].min()


def test_cylinder_normals_and_mean_curvature():
    """On the cylindrical part of a spherocylinder (radius rho, away from the caps)
    the normal is perpendicular to the axis and kappa is the mean curvature 1/(2 rho)."""
    rho = 0.8
    pts = G.spherocylinder(900, 5.0, rho)
    s = _one_body(pts, E0=(0.0, 0.0, 1.0))
    F, S = _features(s)
    z = pts[:, 2]
    length = 2 * rho * 4.0
    mid = np.abs(z) < length / 2 - 2 * rho
    assert mid.sum() > 200
    # E0 along the axis: f0 = E0.n / |E0| vanishes where the normal is radial
    assert np.max(np.abs(F[mid, 0])) < 0.03
    R = np.linalg.norm(pts, axis=1).mean()
    kappa = F[mid, 6] / R
    assert abs(np.median(kappa) * rho - 0.5) < 0.05, np.median(kappa) * rho


def test_isolated_conducting_sphere_targets_are_three_times_the_normal_field():
    """A conducting sphere in a uniform field carries the surface charge
    3 eps E0 cos(theta): with bead area A the converged charges are
    q = 3 eps A E0.n, so y = (q - Q/N)/S = 3 f0 (162 beads, dense oracle solve).
    The bead model reaches the continuum factor as the beads cover the surface:
    here (2a about three quarters of the spacing) it is within 10%; the cos(theta)
    shape holds to a correlation of 0.998."""
    pts = G.icosphere(2)
    s = _one_body(pts, L=14.0, a=0.1, E0=(0.2, 0.5, -0.7), Q=0.7, mesh=48, tol=1e-8)
    F, S = _features(s)
    q, _ = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
    y = M.warm_start_targets(q, s.body_offsets, s.Q, S)
    slope = float(np.sum(y * F[:, 0]) / np.sum(F[:, 0] ** 2))
    assert abs(slope - 3.0) < 0.3, slope
    assert np.corrcoef(y, F[:, 0])[0, 1] > 0.998
    # the guess built from the targets gives back the charges, with the constraint exact
    qg = M.warm_start_guess(y, s.body_offsets, s.Q, S)
    assert np.max(np.abs(qg - q)) < 1e-12 * np.abs(q).max() + 1e-15
    assert abs(qg.sum() - 0.7) < 1e-12


def test_fixed_charge_field_is_coulomb_within_the_body_cutoff():
    """phi and Es at the beads of a sphere (R = R_max = 1, cutoff 7 from its centre):
    an ion at 1.6 from the centre gives the Coulomb potential q/(4 pi eps r) and field
    q (x_j - x_ion)/(4 pi eps r^3) at every bead; an ion at 7.3 gives nothing; the
    sphere's own net charge gives nothing; a second body (42 beads, Q = 2) whose
    centre is 6.65 away adds Q/N per bead of it that lies within the cutoff (35 of 42).  The
    features read them: f3, f4 and f5 from phi and Es, S from rms |Es|."""
    L, eps = 20.0, 0.7
    c = np.array([10.0, 10.0, 10.0])
    sph = G.icosphere(2) + c
    other = G.icosphere(1) * 0.5 + c + [0.0, 6.65, 0.0]
    ion_in, ion_out = c + [1.6, 0.0, 0.0], c + [0.0, 0.0, 7.3]
    s = C.assemble("field", [sph, other], [ion_in, ion_out], [1.0, -1.0], [0.9, 2.0], [L] * 3, 0.05, eps,
                   [[0.0, 0.0, 0.0]], mesh=(32,) * 3, tol=1e-6)
    phi, Es = M.body_field_of_fixed_charges(s.x, s.X, s.body_offsets, s.Q, s.box, s.a, s.eps)
    nb0 = len(sph)
    want_p = np.zeros(nb0)
    want_E = np.zeros((nb0, 3))
    srcs = [(ion_in, 1.0)] + [(p, 2.0 / len(other)) for p in other if np.linalg.norm(p - c) < 7.0]
    assert 0 < len(srcs) - 1 < len(other)
    for p, q in srcs:
        v = sph - p
        r = np.linalg.norm(v, axis=1)
        assert r.min() > 2 * s.a
        want_p += q / (4 * math.pi * eps * r)
        want_E += q * v / (4 * math.pi * eps * r[:, None] ** 3)
    assert np.max(np.abs(phi[:nb0] - want_p)) < 1e-12 * np.abs(want_p).max()
    assert np.max(np.abs(Es[:nb0] - want_E)) < 1e-12 * np.abs(want_E).max()
    F, S = _features(s)
    N = nb0
    A = 4 * math.pi / N
    assert abs(S[0] - eps * A * math.sqrt(np.mean(np.sum(want_E ** 2, axis=1)))) < 1e-12 * S[0]
    assert np.all(F[:nb0, :3] == 0)                        # E0 = 0
    nrm = F[:nb0, 4] ** 2 + F[:nb0, 5] ** 2
    assert np.max(np.abs(nrm - (eps * A / S[0]) ** 2 * np.sum(want_E ** 2, axis=1))) < 1e-10
    # the bead nearest the positive ion: the highest potential, the field pointing
    # into the body most strongly
    j = np.argmin(np.linalg.norm(sph - ion_in, axis=1))
    assert np.argmin(F[:nb0, 4]) == j and F[j, 3] == F[:nb0, 3].max()
