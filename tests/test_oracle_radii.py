"""Pins for the oracle's beads of unequal radii (pair kernel j0(k a) j0(k b)/k^2).

The paper fixes one bead radius (Sec. III.A); a bead of radius a is a charged
spherical shell whose transform is j0(ka) (Eq. M00_Fourier), so two radii
interact through j0(ka) j0(kb)/k^2.  These CPU tests tie the oracle's
closed forms to independent routes: quadrature of the inverse transform,
quadrature of the shell average, the one-radius kernel already pinned in
test_oracle.py, finite differences, xi independence, and the textbook
point-charge Ewald sum through an exact identity.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erfc

import oracle as o


def _phi2_by_quadrature(r, a, b, xi):
    """Inverse 3-D transform of j0(ka) j0(kb)(1 - e^{-k^2/4xi^2})/k^2 by oscillatory
    quadrature in 25-digit arithmetic (the integrand carries three frequencies, which
    a single-weight scipy rule resolves only to about 1e-8)."""
    mp = pytest.importorskip("mpmath")
    with mp.workdps(25):
        A, B, X, R = (mp.mpf(str(v)) for v in (a, b, xi, r))

        def f(k):
            return mp.sin(k * A) * mp.sin(k * B) / (k * A * k * B) * (1 - mp.exp(-k * k / (4 * X * X))) / k * mp.sin(k * R)

        v = mp.quadosc(f, [0, mp.inf], omega=min(float(a), float(b), float(r)))
        return float(v / (2 * mp.pi ** 2 * R))


def _shell_average_of_coulomb(r, a, b):
    """<1/(4 pi |x - y|)> for x uniform on a shell of radius a and y on one of radius b,
    centres r apart: the potential of shell a at distance s from its centre is
    1/(4 pi max(s, a)), and s is distributed as s/(2 b r) on [|r - b|, r + b]."""
    lo, hi = abs(r - b), r + b
    pts = [a] if lo < a < hi else None
    v, _ = quad(lambda s: s / (2 * b * r) / (4 * math.pi * max(s, a)), lo, hi, points=pts, epsabs=1e-15, epsrel=1e-13)
    return v


@pytest.mark.parametrize("a,b,xi,r", [
    (0.5, 0.2, 0.8, 0.1),      # shell b inside shell a
    (0.5, 0.2, 0.8, 0.45),     # overlapping shells
    (0.5, 0.2, 0.8, 1.2),      # apart
    (0.05, 0.11, 1.79, 0.03),
    (0.05, 0.11, 1.79, 0.12),
    (0.05, 0.11, 1.79, 0.4),
    (0.3, 0.1, 2.5, 0.35),
])
def test_pair_kernel_of_two_radii_matches_inverse_transform(a, b, xi, r):
    ref = _phi2_by_quadrature(r, a, b, xi)
    assert abs(o.phi_real2(r, a, b, xi) - ref) <= 1e-11 * max(abs(ref), 1e-3)
    assert abs(o.phi_real2(r, b, a, xi) - ref) <= 1e-11 * max(abs(ref), 1e-3)


@pytest.mark.parametrize("a,b", [(0.5, 0.2), (0.05, 0.11), (0.3, 0.3)])
def test_free_shell_potential_is_the_shell_average(a, b):
    for r in [0.2 * abs(a - b) + 1e-3, 0.9 * (a + b), 0.6 * (a + b), (a + b) * 1.5, 3.0]:
        if r <= 0:
            continue
        ref = _shell_average_of_coulomb(r, a, b)
        assert abs(o.M_free2(r, a, b) - ref) <= 1e-11 * abs(ref)
    # Newton: apart, the shells interact as points; one inside the other, the potential is constant
    assert abs(o.M_free2(2.5 * (a + b), a, b) - 1 / (4 * math.pi * 2.5 * (a + b))) < 1e-15
    if abs(a - b) > 0.01:
        for r in [0.0, 0.3 * abs(a - b), 0.9 * abs(a - b)]:
            assert abs(o.M_free2(r, a, b) - 1 / (4 * math.pi * max(a, b))) < 1e-13


@pytest.mark.parametrize("a,xi", [(0.5, 0.8), (0.05, 1.79), (0.1, 7.0)])
def test_equal_radii_give_the_one_radius_kernel(a, xi):
    """At a = b the two-radius forms are the pinned one-radius kernel, its derivative,
    M(r) of Sec. II and the self term of Sec. III.D.1 at r = 0."""
    for r in [0.3 * a, 1.3 * a, 2.5 * a, 5 * a, 1.0 / xi]:
        p1, p2 = o.phi_real(r, a, xi), o.phi_real2(r, a, a, xi)
        assert abs(p1 - p2) <= 1e-11 * max(abs(p1), 1.0)
        d1, d2 = o.dphi_real(r, a, xi), o.dphi_real2(r, a, a, xi)
        assert abs(d1 - d2) <= 1e-9 * max(abs(d1), 1.0)
        assert abs(o.M_free(r, a) - o.M_free2(r, a, a)) <= 1e-12 * o.M_free(r, a)
    assert abs(o.phi_real2(0.0, a, a, xi) - o.phi_self(a, xi)) <= 1e-12 * o.phi_self(a, xi)


@pytest.mark.parametrize("a,b,xi", [(0.5, 0.2, 0.8), (0.05, 0.11, 1.79)])
def test_two_radius_derivative_and_continuity(a, b, xi):
    # fourth-order central differences, points away from the kinks at |a - b| and a + b
    for r in [0.3 * abs(a - b), 1.3 * abs(a - b), 0.75 * (a + b), 1.3 * (a + b), 1.0 / xi]:
        h = 1e-3 * r
        f = [o.phi_real2(r + j * h, a, b, xi) for j in (-2, -1, 1, 2)]
        fd = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        assert abs(o.dphi_real2(r, a, b, xi) - fd) <= 1e-7 * max(abs(fd), 1e-2)
    for r0 in [abs(a - b), a + b]:
        lo, hi = o.phi_real2(r0 * (1 - 1e-9), a, b, xi), o.phi_real2(r0 * (1 + 1e-9), a, b, xi)
        assert abs(lo - hi) < 1e-8
    # the r -> 0 limit
    assert abs(o.phi_real2(1e-7, a, b, xi) - o.phi_real2(0.0, a, b, xi)) < 1e-6


def _mixed_system(n=36, L=5.0, seed=5):
    """Random neutral charges with two radii, including an overlapping pair of
    different radii and a small bead inside a large one."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, size=(n, 3))
    rad = np.where(np.arange(n) % 3 == 0, 0.35, 0.12)
    x[1] = x[0] + np.array([0.3, 0.1, 0.0])      # radii 0.12 and 0.35 overlapping
    x[2] = x[3] + np.array([0.05, 0.0, 0.1])     # 0.12 inside 0.35 (r < a - b)
    q = rng.normal(size=n)
    q -= q.mean()
    return x, q, np.array([L, L * 1.1, L * 0.9]), rad


def test_potential_with_radii_is_xi_independent():
    x, q, box, rad = _mixed_system()
    p1, E1 = o.potential(x, q, box, rad, 1.0, xi=0.9, field=True)
    p2, E2 = o.potential(x, q, box, rad, 1.0, xi=2.2, field=True)
    assert np.max(np.abs(p1 - p2)) < 1e-11 * np.max(np.abs(p1))
    assert np.max(np.abs(E1 - E2)) < 1e-10 * np.max(np.abs(E1))
    p3 = o.potential(x, q + 0.4, box, rad, 1.0, xi=0.9)
    p4 = o.potential(x, q + 0.4, box, rad, 1.0, xi=2.2)
    assert np.max(np.abs(p3 - p4)) < 1e-11 * np.max(np.abs(p3))


def test_one_radius_per_bead_equal_to_the_scalar_radius():
    x, q, box, rad = _mixed_system()
    same = np.full(len(q), 0.2)
    p1, E1 = o.potential(x, q, box, 0.2, 1.0, field=True)
    p2, E2 = o.potential(x, q, box, same, 1.0, field=True)
    assert np.max(np.abs(p1 - p2)) < 1e-12 * np.max(np.abs(p1))
    assert np.max(np.abs(E1 - E2)) < 1e-11 * np.max(np.abs(E1))


def _point_ewald_matrix(x, box, xi, nimg=3, mmax=14):
    """Textbook point-charge Ewald sum G(x_a - x_b) with k = 0 left out, without 1/eps:
    sum_n erfc(xi r_n)/(4 pi r_n) + (1/V) sum_{k != 0} e^{-k^2/4xi^2}/k^2 cos(k.r) - 1/(4 xi^2 V),
    the n = 0 term of the diagonal replaced by its regular part -xi/(2 pi^{3/2})."""
    n = x.shape[0]
    V = float(np.prod(box))
    d = x[:, None, :] - x[None, :, :]
    Mp = np.zeros((n, n))
    rng = range(-nimg, nimg + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                r = np.linalg.norm(d + np.array([i, j, k]) * box, axis=2)
                if i == j == k == 0:
                    np.fill_diagonal(r, 1.0)
                    t = erfc(xi * r) / (4 * math.pi * r)
                    np.fill_diagonal(t, -xi / (2 * math.pi ** 1.5))
                else:
                    t = erfc(xi * r) / (4 * math.pi * r)
                Mp += t
    m = np.arange(-mmax, mmax + 1)
    K = np.stack(np.meshgrid(*(2 * math.pi * m / L for L in box), indexing="ij"), axis=-1).reshape(-1, 3)
    k2 = np.sum(K * K, axis=1)
    K, k2 = K[k2 > 0], k2[k2 > 0]
    w = np.exp(-k2 / (4 * xi * xi)) / k2
    ph = x @ K.T
    C, S = np.cos(ph), np.sin(ph)
    Mp += ((C * w) @ C.T + (S * w) @ S.T) / V
    return Mp - 1.0 / (4 * xi * xi * V)


def test_shell_lattice_sum_is_point_ewald_plus_overlap_and_a_constant():
    """(1/V) sum_{k != 0} [j0(ka) j0(kb) - 1] e^{ik.r}/k^2 is, by Poisson summation, the
    image sum of the compactly supported W(r; a, b) - 1/(4 pi r) minus its k = 0 value
    -(a^2 + b^2)/6 over V.  So the shell matrix is the point-charge Ewald matrix plus
    the overlap correction of the nearest image plus (a^2 + b^2)/(6 V): apart,
    -(a + b - r)^2/(16 pi a b r) overlapping, 1/(4 pi max(a,b)) - 1/(4 pi r) nested,
    and 1/(4 pi a) at r = 0 of a bead with itself."""
    x, _, box, rad = _mixed_system(n=18)
    V = float(np.prod(box))
    M = o.M_dense(x, box, rad, 1.0)
    P = _point_ewald_matrix(x, box, xi=1.6)
    n = x.shape[0]
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.floor(d / box + 0.5)
    r = np.linalg.norm(d, axis=2)
    ref = P.copy()
    for i in range(n):
        for j in range(n):
            a, b = rad[i], rad[j]
            if i == j:
                ref[i, j] += 1 / (4 * math.pi * a)
            elif r[i, j] < abs(a - b):
                ref[i, j] += 1 / (4 * math.pi * max(a, b)) - 1 / (4 * math.pi * r[i, j])
            elif r[i, j] < a + b:
                ref[i, j] -= (a + b - r[i, j]) ** 2 / (16 * math.pi * a * b * r[i, j])
            ref[i, j] += (a * a + b * b) / (6 * V)
    assert r[0, 1] < rad[0] + rad[1] and r[2, 3] < abs(rad[2] - rad[3])
    assert np.max(np.abs(M - ref)) < 1e-10 * np.max(np.abs(M))


def test_dense_matrix_with_radii_matches_the_sums_and_is_spd():
    x, q, box, rad = _mixed_system(n=30)
    M = o.M_dense(x, box, rad, 0.7)
    assert np.max(np.abs(M - M.T)) < 1e-13 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(M).min() > 0
    p = o.potential(x, q, box, rad, 0.7)
    assert np.max(np.abs(M @ q - p)) < 1e-11 * np.max(np.abs(p))


def test_field_with_radii_is_minus_the_energy_gradient():
    """E_alpha = -d/dx_alpha of U = q^T M q / 2 divided by q_alpha (the self term does not
    depend on x_alpha): central differences of the oracle's own dense energy."""
    x, q, box, rad = _mixed_system(n=14, seed=9)
    _, E = o.potential(x, q, box, rad, 1.0, field=True)
    h = 1e-5
    for al in [0, 1, 2, 3, 7]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[al, c] += h
            xm[al, c] -= h
            Up = 0.5 * q @ o.M_dense(xp, box, rad, 1.0) @ q
            Um = 0.5 * q @ o.M_dense(xm, box, rad, 1.0) @ q
            fd = -(Up - Um) / (2 * h) / q[al]
            assert abs(E[al, c] - fd) <= 2e-6 * max(abs(fd), 1e-2)


def test_hard_sphere_force_with_radii_is_minus_gradient():
    """Eq. hardsphereFD with the contact distance a_alpha + a_beta of two radii:
    the forces are minus the gradient of sum gamma/(4 dt) (r - a_alpha - a_beta)^2
    over overlapping pairs of different bodies (central differences)."""
    rng = np.random.default_rng(2)
    L = 3.0
    x = rng.uniform(0, L, size=(10, 3))
    x[1] = x[0] + [0.3, 0.05, 0.0]
    x[4] = x[3] + [0.0, 0.2, 0.1]
    rad = np.array([0.35, 0.12, 0.12, 0.35, 0.12, 0.2, 0.2, 0.12, 0.35, 0.12])
    off = [0, 1, 2, 3, 5, 6, 7, 8, 9, 10]   # beads 3 and 4 share a body
    box = np.array([L, L, L])
    gamma, dt = 1.3, 0.01

    def U(y):
        bid = o.body_index(off)
        u = 0.0
        for i in range(len(y)):
            for j in range(i + 1, len(y)):
                if bid[i] == bid[j]:
                    continue
                r = np.linalg.norm(o.min_image(y[i] - y[j], box))
                c = rad[i] + rad[j]
                if r < c:
                    u += gamma / (4 * dt) * (r - c) ** 2
        return u

    f = o.hard_sphere_forces(x, off, box, rad, gamma, dt)
    assert np.abs(f[0]).max() > 1.0 and np.abs(f[3]).max() < 1e-12 and np.abs(f[4]).max() < 1e-12
    h = 1e-6
    for i in [0, 1, 2, 5]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = -(U(xp) - U(xm)) / (2 * h)
            assert abs(f[i, c] - fd) < 1e-5 * max(1.0, abs(fd))
