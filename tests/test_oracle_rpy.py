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
