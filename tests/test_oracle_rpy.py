"""Pins for the periodic RPY mobility oracle (oracle/rpy_ref.py), CPU only.

Independent routes: 25-digit oscillatory quadrature of the inverse transform of
j0^2(ka)(I - k_hat k_hat)/k^2 for the free-space tensor (both regimes), adaptive
quadrature for the oracle's Gauss-Legendre wave integrals, xi independence of the
split, Hasimoto's periodic correction 2.837297 a/L of the self mobility, the
free-space pair tensor as the box grows, symmetry and positive definiteness.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import rpy_ref as R


def _free_by_quadrature(r, a):
    mp = pytest.importorskip("mpmath")
    with mp.workdps(25):
        A_, r_ = mp.mpf(str(a)), mp.mpf(str(r))

        def j0(x):
            return mp.sin(x) / x

        def j1x(x):
            return (mp.sin(x) - x * mp.cos(x)) / x ** 3

        fa = lambda k: j0(k * A_) ** 2 * (j0(k * r_) - j1x(k * r_))
        fb = lambda k: j0(k * A_) ** 2 * (3 * j1x(k * r_) - j0(k * r_))
        om = min(float(a), float(r))
        va = mp.quadosc(fa, [0, mp.inf], omega=om)
        vb = mp.quadosc(fb, [0, mp.inf], omega=om)
        return float(va / (2 * mp.pi ** 2)), float(vb / (2 * mp.pi ** 2))


@pytest.mark.parametrize("a,r", [(0.5, 0.3), (0.5, 0.9), (0.5, 1.7), (0.2, 1.0), (0.2, 0.05)])
def test_free_rpy_is_the_inverse_transform_of_its_kernel(a, r):
    """The closed form (Rotne-Prager apart, Yamakawa's form overlapping) equals the inverse
    transform of j0^2(ka)(I - k_hat k_hat)/(mu k^2), the Oseen tensor averaged over both shells."""
    A, B = R.rpy_free(r, a)
    Aq, Bq = _free_by_quadrature(r, a)
    assert abs(A - Aq) < 1e-10 * abs(Aq) and abs(B - Bq) < 1e-10 * max(abs(Bq), abs(Aq))


def test_free_rpy_limits_and_continuity():
    a = 0.3
    A0, B0 = R.rpy_free(0.0, a)
    assert abs(A0 - 1 / (6 * math.pi * a)) < 1e-15 and B0 == 0.0      # Stokes mobility
    lo, hi = R.rpy_free(2 * a * (1 - 1e-12), a), R.rpy_free(2 * a, a)
    assert abs(lo[0] - hi[0]) < 1e-10 and abs(lo[1] - hi[1]) < 1e-10
    A, B = R.rpy_free(500.0, a)                                       # far: the Oseen tensor
    assert abs(A - 1 / (8 * math.pi * 500)) < 1e-6 * A and abs(B - 1 / (8 * math.pi * 500)) < 1e-6 * B


@pytest.mark.parametrize("a,xi", [(0.3, 1.0), (0.1, 3.0)])
def test_wave_radial_quadrature(a, xi):
    """The oracle's Gauss-Legendre panels against scipy's adaptive rule."""
    r = np.array([0.0, 0.05, 0.4, 1.3, 2.9])
    A, B = R.rpy_wave_radial(r, a, xi)
    for i, rv in enumerate(r):
        w = lambda k: (math.sin(k * a) / (k * a)) ** 2 * (1 + k * k / (4 * xi * xi)) * math.exp(-k * k / (4 * xi * xi))

        def j0(x):
            return math.sin(x) / x if x else 1.0

        def j1x(x):
            return (math.sin(x) - x * math.cos(x)) / x ** 3 if x > 1e-3 else 1 / 3 - x * x / 30

        fa = lambda k: w(k) * (j0(k * rv) - j1x(k * rv))
        fb = lambda k: w(k) * (3 * j1x(k * rv) - j0(k * rv))
        qa, _ = quad(fa, 1e-14, 20 * xi, limit=800, epsabs=1e-16, epsrel=1e-14)
        qb, _ = quad(fb, 1e-14, 20 * xi, limit=800, epsabs=1e-16, epsrel=1e-14)
        c = 1 / (2 * math.pi ** 2)
        assert abs(A[i] - c * qa) < 1e-12 * abs(c * qa)
        assert abs(B[i] - c * qb) < 1e-12 * max(abs(c * qb), abs(c * qa))


def _cloud(n=14, L=5.0, seed=4):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, size=(n, 3))
    x[1] = x[0] + [0.25, 0.1, 0.0]     # an overlapping pair (r < 2a)
    return x, rng.normal(size=(n, 3)), np.array([L, 1.1 * L, 0.9 * L])


def test_rpy_mobility_is_xi_independent():
    x, F, box = _cloud()
    U1 = R.rpy_mobility(x, F, box, 0.2, mu=0.7, xi=1.1)
    U2 = R.rpy_mobility(x, F, box, 0.2, mu=0.7, xi=2.6)
    assert np.abs(U1 - U2).max() < 1e-11 * np.abs(U1).max()


def test_self_mobility_has_hasimoto_periodic_correction():
    """One bead in a cubic box: 6 pi mu a M_self = 1 - 2.837297 a/L + O((a/L)^3) (Hasimoto's
    periodic array of Stokeslets; the constant is that of the simple-cubic lattice sum)."""
    a = 0.5
    c = []
    for L in (8.0, 16.0, 32.0):
        M = R.rpy_matrix(np.array([[1.0, 2.0, 3.0]]), [L] * 3, a)
        assert np.abs(M - M[0, 0] * np.eye(3)).max() < 1e-12 * M[0, 0]   # isotropic
        c.append((1 - 6 * math.pi * a * M[0, 0]) * L / a)
    for L, v in zip((8.0, 16.0, 32.0), c):
        assert abs(v - 2.837297) < 5 * (a / L) ** 2
    assert abs(c[2] - 2.837297) < abs(c[0] - 2.837297)


def test_pair_tends_to_free_space_rpy():
    """A pair in a growing box: M_12 - M_11 tends to M_RPY(r) - I/(6 pi mu a) (the periodic
    correction common to both cancels up to O(r^2/L^3))."""
    a = 0.3
    d = np.array([0.5, 0.3, -0.2])
    r = np.linalg.norm(d)
    A, B = R.rpy_free(r, a)
    ref = A * np.eye(3) + B * np.outer(d, d) / r ** 2 - np.eye(3) / (6 * math.pi * a)
    errs = []
    for L in (6.0, 12.0, 24.0):
        x = np.array([[L / 2] * 3, np.array([L / 2] * 3) + d])
        M = R.rpy_matrix(x, [L] * 3, a)
        errs.append(np.abs((M[0:3, 3:6] - M[0:3, 0:3]) - ref).max())
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-4 * np.abs(ref).max()


def test_dense_mobility_symmetric_positive_definite():
    x, F, box = _cloud(n=9)
    M = R.rpy_matrix(x, box, 0.2)
    assert np.abs(M - M.T).max() < 1e-13 * np.abs(M).max()
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() > 0
    U = R.rpy_mobility(x, F, box, 0.2)
    assert np.abs(M @ F.reshape(-1) - U.reshape(-1)).max() < 1e-12 * np.abs(U).max()


def _square(L=6.0, R_=0.45, a=0.2, free=True):
    """Four beads on a square of half-diagonal R_ in the plane z = L/2, centred in a cubic box
    (the square's fourfold symmetry about z is then a symmetry of the periodic lattice), and
    optionally a free bead."""
    c = np.array([L / 2, L / 2, L / 2])
    sq = np.array([[R_, 0, 0], [0, R_, 0], [-R_, 0, 0], [0, -R_, 0]]) + c
    if not free:
        return sq, c[None, :], np.array([0, 4]), np.array([L, L, L]), a
    x = np.vstack([sq, [[0.6, 0.9, 1.3]]])
    return x, np.array([c, x[4]]), np.array([0, 4, 5]), np.array([L, L, L]), a


def test_rigid_square_translation_and_rotation_closed_forms():
    """A rigid square of four beads: pulled along its normal z each bead carries F/4 (symmetry),
    so U_z = sum_k (M_1k)_zz / 4; turned by a torque L about z each bead carries L/(4R) along its
    tangent, so Omega_z R = (sum_k M_1k t_k)_t L/(4R) (M the periodic pair tensors, t_k the
    tangents).  A collinear body would leave its spin about its own axis undetermined."""
    x, X, off, box, a = _square(free=False)
    M = R.rpy_matrix(x, box, a)
    R_ = 0.45
    W, f = R.rigid_mobility(x, X, off, box, a, [[0, 0, 1.0, 0, 0, 0]], M=M)
    assert np.abs(f - [0, 0, 0.25]).max() < 1e-12
    uz = sum(M[2, 3 * k + 2] for k in range(4)) * 0.25
    assert abs(W[0, 2] - uz) < 1e-12 * abs(uz) and np.abs(W[0, [0, 1, 3, 4, 5]]).max() < 1e-12 * abs(uz)
    W, f = R.rigid_mobility(x, X, off, box, a, [[0, 0, 0, 0, 0, 1.0]], M=M)
    t = np.array([[0, 1.0, 0], [-1.0, 0, 0], [0, -1.0, 0], [1.0, 0, 0]])     # tangents (counter-clockwise)
    assert np.abs(f - t / (4 * R_)).max() < 1e-10
    u1 = sum(M[0:3, 3 * k:3 * k + 3] @ t[k] for k in range(4)) / (4 * R_)
    assert abs(W[0, 5] * R_ - u1[1]) < 1e-10 * abs(u1[1])


def test_rigid_grand_mobility_symmetric_positive_definite():
    """The body mobility (U, Omega) = N (F, L) of rigid bodies is symmetric positive definite
    (reciprocal theorem): the square's 6 x 6 and the free bead's 3 x 3 blocks and their coupling;
    the free bead's rotation stays zero."""
    x, X, off, box, a = _square()
    M = R.rpy_matrix(x, box, a)
    cols = []
    dofs = [(0, k) for k in range(6)] + [(1, k) for k in range(3)]
    for b, k in dofs:
        FL = np.zeros((2, 6))
        FL[b, k] = 1.0
        W, _ = R.rigid_mobility(x, X, off, box, a, FL, M=M)
        assert np.abs(W[1, 3:]).max() == 0.0
        cols.append([W[bb, kk] for bb, kk in dofs])
    N = np.array(cols).T
    assert np.abs(N - N.T).max() < 1e-12 * np.abs(N).max()
    assert np.linalg.eigvalsh(0.5 * (N + N.T)).min() > 0
