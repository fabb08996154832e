"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU only.  None of them compares the oracle with
itself: they use independent quadrature, analytic limits, lattice constants,
the paper's printed results, brute-force finite differences and invariances.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as o
from workloads import configs as C
from workloads import geometry as G

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _phi_by_quadrature(r, a, xi):
    """Inverse 3-D Fourier transform of j0^2(ka)(1 - e^{-k^2/4xi^2})/k^2 (the real-space
    share of Eq. splitting), computed by numerical quadrature."""
    def f(k):
        return (math.sin(k * a) / (k * a)) ** 2 * (1 - math.exp(-k * k / (4 * xi * xi))) / k

    K0 = 60.0
    i1, _ = quad(lambda k: f(k) * math.sin(k * r), 1e-12, K0, limit=4000, epsabs=1e-14, epsrel=1e-12)
    i2, _ = quad(f, K0, np.inf, weight="sin", wvar=r, limlst=400)
    return (i1 + i2) / (2 * math.pi ** 2 * r)


@pytest.mark.parametrize("a,xi,r", [(0.5, 0.8, 0.3), (0.5, 0.8, 0.7), (0.5, 0.8, 1.5), (0.5, 0.8, 2.5),
                                    (0.05, 1.79, 0.04), (0.05, 1.79, 0.3), (0.1, 1.153, 0.15)])
def test_real_kernel_matches_inverse_transform(a, xi, r):
    """Eq. psi_Re_1 (with the Heaviside sign read as -1/(4 pi r) + (4a-r)/(16 pi a^2))
    equals the inverse transform of its Fourier-space definition."""
    ref = _phi_by_quadrature(r, a, xi)
    assert abs(o.phi_real(r, a, xi) - ref) <= 1e-8 * max(abs(ref), 1e-3)


def test_printed_heaviside_sign_is_wrong():
    """The sign as printed, -(1/(4 pi r) + (4a-r)/(16 pi a^2)), misses the transform by
    2(4a-r)/(16 pi a^2): this is the reading recorded for Eq. psi_Re_1."""
    a, xi, r = 0.5, 0.8, 0.3
    printed = o.phi_real(r, a, xi) - 2 * (4 * a - r) / (16 * math.pi * a * a)
    assert abs(printed - _phi_by_quadrature(r, a, xi)) > 0.1


@pytest.mark.parametrize("a,xi", [(0.5, 0.8), (0.05, 1.79), (0.1, 7.0)])
def test_real_kernel_derivative(a, xi):
    for r in [0.3 * a, 1.3 * a, 2.5 * a, 5 * a, 1.0 / xi]:
        h = 1e-6 * max(r, 1e-3)
        fd = (o.phi_real(r + h, a, xi) - o.phi_real(r - h, a, xi)) / (2 * h)
        assert abs(o.dphi_real(r, a, xi) - fd) <= 1e-6 * max(abs(fd), 1e-2)


def test_real_kernel_limits():
    a = 0.4
    # xi -> 0: real-space kernel -> M(r) (Sec. II), error O(xi)
    for r in [0.2, 0.79, 0.81, 1.7, 3.0]:
        e1 = abs(o.phi_real(r, a, 1e-3) - o.M_free(r, a))
        e2 = abs(o.phi_real(r, a, 1e-4) - o.M_free(r, a))
        assert e2 < 0.2 * e1 + 1e-12 and e2 < 1e-4
    # a -> 0: point-charge Ewald erfc(xi r)/(4 pi r) (Eq. psi_Re_point)
    for r in [0.3, 1.0, 2.0]:
        pc = math.erfc(0.9 * r) / (4 * math.pi * r)
        assert abs(o.phi_real(r, 1e-4, 0.9) - pc) < 1e-8
    # r -> 0: self term (equation after psi_Re_1).  The wave share is smooth and
    # even in r, so the slope at 0 is that of M(r) = (4a - r)/(16 pi a^2): -1/(16 pi a^2)
    for xi in [0.5, 1.5]:
        for r in [1e-3, 1e-4]:
            slope = (o.phi_real(r, a, xi) - o.phi_self(a, xi)) / r
            assert abs(slope + 1 / (16 * math.pi * a * a)) < 50 * r
    # continuity at r = 2a
    assert abs(o.phi_real(2 * a * (1 + 1e-9), a, 1.0) - o.phi_real(2 * a * (1 - 1e-9), a, 1.0)) < 1e-8
    # M(r) continuous at 2a and 1/(4 pi a) at r = 0
    assert abs(o.M_free(0.0, a) - 1 / (4 * math.pi * a)) < 1e-15
    assert abs(o.M_free(2 * a - 1e-12, a) - o.M_free(2 * a, a)) < 1e-10


def test_madelung_rocksalt():
    """Rock salt with d > 2a: every pair interacts by plain Coulomb, so
    psi_alpha = q_alpha/(4 pi eps a) - M_NaCl q_alpha/(4 pi eps d)."""
    mad = GOLDEN["nacl_madelung_constant"]["value"]
    for m, xi in [(1, None), (2, 1.3), (2, 2.7)]:
        s = C.rocksalt(m=m, d=1.0, a=0.3)
        psi = o.potential(s.x, s.Q, s.box, s.a, s.eps, xi=xi)
        got = 1.0 / s.a - 4 * math.pi * psi / s.Q
        assert np.max(np.abs(got - mad)) < 1e-9


def _random_neutral(n=40, L=5.0, a=0.3, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, size=(n, 3))
    x[1] = x[0] + np.array([0.2, 0.1, 0.0])      # an overlapping pair (r < 2a)
    q = rng.normal(size=n)
    q -= q.mean()
    return x, q, np.array([L, L * 1.1, L * 0.9]), a


def test_xi_independence():
    x, q, box, a = _random_neutral()
    p1, E1 = o.potential(x, q, box, a, 1.0, xi=0.9, field=True)
    p2, E2 = o.potential(x, q, box, a, 1.0, xi=2.2, field=True)
    assert np.max(np.abs(p1 - p2)) < 1e-11 * np.max(np.abs(p1))
    assert np.max(np.abs(E1 - E2)) < 1e-10 * np.max(np.abs(E1))


def test_xi_independence_non_neutral():
    """With k = 0 excluded (Sec. II) the sums stay independent of xi for a net charge."""
    x, q, box, a = _random_neutral()
    q = q + 0.37
    p1 = o.potential(x, q, box, a, 1.0, xi=0.9)
    p2 = o.potential(x, q, box, a, 1.0, xi=2.2)
    assert np.max(np.abs(p1 - p2)) < 1e-11 * np.max(np.abs(p1))
    M1 = o.M_dense(x[:12], box, a, 1.0, xi=0.9)
    M2 = o.M_dense(x[:12], box, a, 1.0, xi=2.2)
    assert np.max(np.abs(M1 - M2)) < 1e-11 * np.max(np.abs(M1))


def test_single_charge_is_the_k_sum_of_its_images():
    """One unit charge: psi = (1/(eps V)) sum_{k != 0} j0^2(ka)/k^2 (Eq. M00_Fourier at r = 0),
    summed directly over a cube of wave vectors; the truncation error falls like 1/K,
    so two cubes are Richardson-extrapolated.  Without the k = 0 correction the
    oracle would be off by 1/(4 xi^2 V eps), about 10% here."""
    box = np.array([4.0, 4.0, 4.0])
    a = 0.3
    psi = o.potential(np.array([[1.0, 2.0, 3.0]]), [1.0], box, a, 1.0)[0]

    def cube_sum(M):
        m = np.arange(-M, M + 1)
        kx, ky, kz = np.meshgrid(*(2 * np.pi * m / 4.0,) * 3, indexing="ij")
        k2 = kx ** 2 + ky ** 2 + kz ** 2
        k2[M, M, M] = 1.0
        kk = np.sqrt(k2)
        t = (np.sin(kk * a) / (kk * a)) ** 2 / k2
        t[M, M, M] = 0.0
        return t.sum() / 64.0

    extrapolated = 2 * cube_sum(80) - cube_sum(40)
    assert abs(psi - extrapolated) < 2e-4 * abs(psi)
    assert abs(o.k0_term(box, 0.44, 1.0)) > 0.05 * abs(psi)


def test_translation_invariance():
    x, q, box, a = _random_neutral()
    p1 = o.potential(x, q, box, a, 1.0)
    p2 = o.potential(x + np.array([1.234, -7.1, 0.33]), q, box, a, 1.0)
    assert np.max(np.abs(p1 - p2)) < 1e-12 * np.max(np.abs(p1)) * 10


def test_dense_matrix_matches_sums_and_is_spd():
    x, q, box, a = _random_neutral(n=30)
    M = o.M_dense(x, box, a, 0.7)
    assert np.max(np.abs(M - M.T)) < 1e-13 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(M).min() > 0
    p = o.potential(x, q, box, a, 0.7)
    assert np.max(np.abs(M @ q - p)) < 1e-11 * np.max(np.abs(p))


def test_large_box_pair_tends_to_free_space():
    """A neutral pair in a growing box: the periodic M_12 tends to M(r) (Sec. II)
    up to the O(1/L) image/background correction."""
    a, r = 0.3, 0.45
    errs = []
    for L in [10.0, 20.0, 40.0]:
        x = np.array([[L / 2, L / 2, L / 2], [L / 2 + r, L / 2, L / 2]])
        M = o.M_dense(x, [L] * 3, a, 1.0)
        errs.append(abs((M[0, 0] - M[0, 1]) - (o.M_free(0, a) - o.M_free(r, a))))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-3


def test_saddle_constraint_linearity_and_gmres():
    s = C.small_system(seed=11, n_bodies=2, level=1, n_ions=5, nrhs=3)
    M = o.M_dense(s.x, s.box, s.a, s.eps)
    q, psi = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0, s.box, s.a, s.eps, M=M)
    off = s.body_offsets
    for r in range(3):
        sums = np.add.reduceat(q[r], off[:-1])
        assert np.max(np.abs(sums - s.Q)) < 1e-12 * max(1.0, np.abs(s.Q).max())
        # the solution satisfies Eq. saddle: bead potentials = body potential + r.E0
        rel = o.relative_positions(s.x, s.X, off, s.box)
        bid = o.body_index(off)
        assert np.max(np.abs(M @ q[r] - (psi[r][bid] + rel @ s.E0[r]))) < 1e-10
    # linearity in E0 (the Q part is common to all three right-hand sides)
    q0, _ = o.solve_dense(s.x, off, s.X, s.Q, np.zeros(3), s.box, s.a, s.eps, M=M)
    qz, _ = o.solve_dense(s.x, off, s.X, np.zeros_like(s.Q), s.E0, s.box, s.a, s.eps, M=M)
    comb = 2.0 * s.E0[0] - 0.5 * s.E0[1]
    qc, _ = o.solve_dense(s.x, off, s.X, s.Q, comb, s.box, s.a, s.eps, M=M)
    assert np.max(np.abs(qc - (q0 + 2.0 * qz[0] - 0.5 * qz[1]))) < 1e-10 * np.max(np.abs(qc))
    # restarted GMRES on the matrix-free operator converges to the dense solution
    qg, psig, it, res = o.solve_gmres(s.x, off, s.X, s.Q, s.E0[0], s.box, s.a, s.eps, rtol=1e-11, restart=20)
    assert res <= 1e-11
    assert np.max(np.abs(qg - q[0])) < 1e-8 * np.max(np.abs(q[0]))


def test_body_permutation_symmetry():
    s = C.small_system(seed=5, n_bodies=2, level=1, n_ions=0)
    q, psi = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
    n0 = s.body_offsets[1]
    xs = np.concatenate([s.x[n0:], s.x[:n0]])
    offs = np.array([0, s.n - n0, s.n], dtype=np.int32)
    q2, psi2 = o.solve_dense(xs, offs, s.X[::-1], s.Q[::-1], s.E0[0], s.box, s.a, s.eps)
    assert np.max(np.abs(np.concatenate([q2[s.n - n0:], q2[:s.n - n0]]) - q)) < 1e-10 * np.abs(q).max()
    assert np.max(np.abs(psi2[::-1] - psi)) < 1e-10 * np.abs(psi).max()


def test_single_sphere_dipole_against_paper():
    """Sec. IV.A: S -> 4 pi a^3 eps E0 from above (a_eff > a_b), error ~ N^-1/2,
    about 5% near N = 1000; the dipole is exactly along E0."""
    coef = GOLDEN["single_sphere_dipole_coefficient"]["value"]
    errs, ns = [], []
    for lev in [1, 2, 3]:
        a = G.min_spacing(G.icosphere(lev)) / 2.0    # beads as large as possible without overlap
        s = C.config1(level=lev, a=a)
        q, _ = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
        S = o.dipoles(s.x, s.X, s.body_offsets, q, s.box)[0]
        assert abs(S[0]) < 1e-10 * S[2] and abs(S[1]) < 1e-10 * S[2]
        errs.append(S[2] / coef - 1.0)
        ns.append(s.n)
    assert all(e > 0 for e in errs)                       # a_eff > a_b
    assert errs[0] > errs[1] > errs[2]
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -0.75 < slope < -0.4                           # ~ N^-1/2
    err_1000 = math.exp(np.polyval(np.polyfit(np.log(ns), np.log(errs), 1), math.log(1000.0)))
    assert 0.03 < err_1000 < 0.08                         # "about 5% at N ~ 1000"
    # config-1 sphere (162 beads of radius 0.1) as in the workload
    s = C.config1()
    q, _ = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
    S = o.dipoles(s.x, s.X, s.body_offsets, q, s.box)[0]
    assert 0.0 < S[2] / coef - 1.0 < 0.3


def _energy_of(x, s, M_fn):
    M = M_fn(x)
    q, psi = o.solve_dense(x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps, M=M)
    S = o.dipoles(x, s.X, s.body_offsets, q, s.box)
    return o.energy(s.X, s.Q, psi, S, s.E0[0]), q


def test_forces_are_energy_gradient():
    """Eq. beadforce against central differences of U (Eq. pot_syst) for bead-wise moves
    with the body reference points held fixed (Appendix derivation)."""
    s = C.small_system(seed=21, n_bodies=2, level=0, n_ions=3, L=6.0, a=0.2)

    def Mf(x):
        return o.M_dense(x, s.box, s.a, s.eps, xi=1.4)

    U0, q = _energy_of(s.x, s, Mf)
    f = o.bead_forces(s.x, q, s.E0[0], s.box, s.a, s.eps, xi=1.4)
    rng = np.random.default_rng(0)
    for al in rng.choice(s.n, size=5, replace=False):
        for d in range(3):
            h = 1e-5
            xp = s.x.copy(); xp[al, d] += h
            xm = s.x.copy(); xm[al, d] -= h
            fd = -(_energy_of(xp, s, Mf)[0] - _energy_of(xm, s, Mf)[0]) / (2 * h)
            assert abs(fd - f[al, d]) < 2e-6 * max(1.0, np.abs(f).max())


def test_newton_third_law_and_torque_identity():
    s = C.small_system(seed=9, n_bodies=2, level=1, n_ions=4)
    q, psi = o.solve_dense(s.x, s.body_offsets, s.X, s.Q, s.E0[0], s.box, s.a, s.eps)
    f = o.bead_forces(s.x, q, s.E0[0], s.box, s.a, s.eps)
    assert np.max(np.abs(f.sum(axis=0) - q.sum() * s.E0[0])) < 1e-9 * np.abs(f).max()
    # isolated neutral body in a big box: torque = S x E0 up to image terms
    s1 = C.config1(level=1, a=0.25)
    s1.E0 = np.array([[0.3, 0.0, 1.0]])
    q, psi = o.solve_dense(s1.x, s1.body_offsets, s1.X, s1.Q, s1.E0[0], s1.box, s1.a, s1.eps)
    f = o.bead_forces(s1.x, q, s1.E0[0], s1.box, s1.a, s1.eps)
    F, L = o.body_force_torque(s1.x, s1.X, s1.body_offsets, f, s1.box)
    S = o.dipoles(s1.x, s1.X, s1.body_offsets, q, s1.box)
    assert np.linalg.norm(L[0] - np.cross(S[0], s1.E0[0])) < 1e-2 * np.linalg.norm(S[0]) + 1e-9


def test_auto_params_balance_the_paper_error_bounds():
    """Sec. III.D.2: eta = h^2 xi^2 P / pi equalises the truncation bound
    e^{-h^2 P^2 xi^2/2 eta} and the quadrature bound e^{-pi^2 eta/2 xi^2 h^2}, both
    then e^{-pi P/2}; the wave-space bound e^{-k_c^2/4xi^2} and the real-space bound
    meet the tolerance; N_g = 1 + L k_c / pi."""
    for L, mesh, tol, a in [(20.0, 64, 1e-8, 0.1), (30.0, 128, 1e-6, 0.05), (13.89, 256, 1e-6, 0.05)]:
        p = o.auto_params([L] * 3, [mesh] * 3, tol, a)
        h, xi, P, eta = p["h"], p["xi"], p["P"], p["eta"]
        trunc = math.exp(-h * h * P * P * xi * xi / (2 * eta))
        quadr = math.exp(-math.pi ** 2 * eta / (2 * xi * xi * h * h))
        assert abs(trunc - quadr) <= 1e-12 * trunc
        assert abs(trunc - math.exp(-math.pi * P / 2)) <= 1e-12 * trunc
        assert math.exp(-math.pi * P / 2) <= tol < math.exp(-math.pi * (P - 1) / 2)
        assert math.exp(-p["k_c"] ** 2 / (4 * xi * xi)) <= tol * (1 + 1e-9)
        assert math.exp(-((p["r_cut"] - 2 * a) * xi) ** 2) <= tol * (1 + 1e-9)
        assert abs(1 + L * p["k_c"] / math.pi - mesh) < 1e-9


def test_philox_counter_based_generator():
    a = o.philox4x32_10((0, 0, 0, 0), (0, 0))
    b = o.philox4x32_10((1, 0, 0, 0), (0, 0))
    c = o.philox4x32_10((0, 0, 0, 0), (1, 0))
    assert a != b and a != c and all(0 <= v < 2 ** 32 for v in a + b + c)
    assert a == o.philox4x32_10((0, 0, 0, 0), (0, 0))
    z = np.array([o.normals(i, 3, 12345, 6) for i in range(20000)]).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # uniformity of the raw words (chi-square over 16 bins)
    w = np.array([o.philox4x32_10((i, 7, 0, 0), (99, 1))[2] for i in range(16000)]) >> 28
    cnt = np.bincount(w, minlength=16)
    chi2 = ((cnt - 1000) ** 2 / 1000).sum()
    assert chi2 < 45  # 15 dof, p ~ 1e-4


def test_hard_sphere_force_is_minus_gradient():
    box = np.array([5.0, 5.0, 5.0])
    x = np.array([[1.0, 1.0, 1.0], [1.07, 1.02, 0.99], [3.0, 3.0, 3.0]])
    off = np.array([0, 1, 2, 3])
    a, gamma, dt = 0.05, 1.0, 1e-3
    f = o.hard_sphere_forces(x, off, box, a, gamma, dt)

    def U(xx):
        d = np.linalg.norm(o.min_image(xx[0] - xx[1], box))
        return gamma / (4 * dt) * (d - 2 * a) ** 2 if d < 2 * a else 0.0

    for d in range(3):
        h = 1e-7
        xp = x.copy(); xp[0, d] += h
        xm = x.copy(); xm[0, d] -= h
        assert abs(-(U(xp) - U(xm)) / (2 * h) - f[0, d]) < 1e-4 * np.abs(f).max()
    assert np.allclose(f[0], -f[1]) and np.allclose(f[2], 0)


def test_bd_step_deterministic_limits():
    """kT = 0: ions move by F dt / gamma exactly (Eq. forward with M^H = I/gamma);
    a rigid body under a uniform force translates without rotating."""
    s = C.small_system(seed=4, n_bodies=1, level=1, n_ions=3)
    f = np.zeros((s.n, 3))
    f[:, 0] = 2.0
    xn, Xn = o.bd_step(s.x, s.X, s.body_offsets, f, s.box, s.a, dt=1e-3, kT=0.0)
    assert np.allclose(xn - s.x, np.array([2e-3, 0, 0]), atol=1e-15)
    # torque about the reference point rotates the body by Omega dt, rigidly
    f2 = np.zeros((s.n, 3))
    r = o.relative_positions(s.x, s.X, s.body_offsets, s.box)
    nb0 = s.body_offsets[1]
    f2[:nb0] = np.cross(np.array([0, 0, 1.0]), r[:nb0])
    xn, Xn = o.bd_step(s.x, s.X, s.body_offsets, f2, s.box, s.a, dt=1e-2, kT=0.0)
    d0 = np.linalg.norm(r[:nb0], axis=1)
    d1 = np.linalg.norm(xn[:nb0] - Xn[0], axis=1)
    assert np.allclose(d0, d1, atol=1e-12)


def test_bd_noise_variance():
    """Ion displacement variance 2 kT dt / gamma per axis (fluctuation-dissipation, Sec. V.A)."""
    n = 4000
    x = np.random.default_rng(1).uniform(0, 10, size=(n, 3))
    off = np.arange(n + 1, dtype=np.int32)
    xn, _ = o.bd_step(x, x.copy(), off, np.zeros((n, 3)), np.array([10.0] * 3), 0.05, dt=1e-3,
                      gamma=2.0, kT=1.5, seed=77, step=5)
    d = (xn - x).ravel()
    var = 2 * 1.5 * 1e-3 / 2.0
    assert abs(d.mean()) < 5 * math.sqrt(var / d.size)
    assert abs(d.var() / var - 1) < 5 * math.sqrt(2 / d.size)


def test_mlp_reference_gradient_by_finite_differences():
    """The oracle network's back-propagated gradient equals central differences of its loss."""
    from oracle import mlp_ref as M
    rng = np.random.default_rng(4)
    p = rng.normal(size=M.NPARAM) * 0.3
    X = rng.normal(size=(40, M.IN))
    T = rng.normal(size=40)
    L, g = M.loss_and_grad(p, X, T)
    assert abs(L - np.mean((M.forward(p, X) - T) ** 2)) < 1e-14
    for i in rng.choice(M.NPARAM, size=60, replace=False).tolist() + [M.NPARAM - 1, 0]:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (M.loss_and_grad(pp, X, T)[0] - M.loss_and_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_bf16_rounding_pins():
    """round_bf16: representable values are fixed, halfway cases go to the even
    neighbour, and every result is within half an ulp (2^-8 relative)."""
    from oracle import mlp_ref as M
    exact = np.array([1.0, -2.5, 1.0 + 2 ** -7, 3 * 2.0 ** -20], dtype=np.float32)
    assert np.array_equal(M.round_bf16(exact), exact.astype(np.float64))
    ties = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8], dtype=np.float32)
    assert np.array_equal(M.round_bf16(ties), [1.0, 1.0 + 2 ** -6])
    rng = np.random.default_rng(0)
    x = rng.normal(size=10000).astype(np.float32)
    r = M.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) + 1e-45)
    # the quantised network equals the exact one when the hidden operands are already BF16
    p = rng.normal(size=M.NPARAM) * 0.1
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    X = rng.normal(size=(50, M.IN))
    assert np.max(np.abs(M.forward_bf16_hidden(p, X) - M.forward(p, X))) < 2e-2


# ---------------------------------------------------------------------------
# Philox4x32-10 against its published known-answer vectors
# ---------------------------------------------------------------------------

def test_philox_known_answer_vectors():
    """Catches a wrong multiplier, Weyl constant, round count or word order in the
    generator: three published 128-bit outputs (all-zero, all-one and pi-digit inputs)."""
    kat = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")))
    for v in kat["vectors"]:
        ctr = tuple(int(w, 16) for w in v["ctr"])
        key = tuple(int(w, 16) for w in v["key"])
        assert o.philox4x32_10(ctr, key) == tuple(int(w, 16) for w in v["out"])


# ---------------------------------------------------------------------------
# Spread grid of Eq. H_hat: fixed by what the window must be, not by its formula
# ---------------------------------------------------------------------------

_ANISO_BOX = np.array([3.0, 4.0, 5.0])
_ANISO_MESH = (16, 20, 24)


def _grid_dft(H, box, m):
    """h_x h_y h_z sum_g H(x_g) e^{-i k.x_g} at k = 2 pi m / L (grid stored [z, y, x])."""
    Nz, Ny, Nx = H.shape
    h = box / np.array([Nx, Ny, Nz])
    k = 2 * math.pi * np.asarray(m, dtype=np.float64) / box
    ph = (np.exp(-1j * k[2] * h[2] * np.arange(Nz))[:, None, None]
          * np.exp(-1j * k[1] * h[1] * np.arange(Ny))[None, :, None]
          * np.exp(-1j * k[0] * h[0] * np.arange(Nx))[None, None, :])
    return (H * ph).sum() * np.prod(h), k


@pytest.mark.parametrize("P", [4, 5, 9])
def test_spread_stencil_is_the_P_nearest_nodes(P):
    """Catches a stencil shifted by a node or an axis mix-up: for one bead the nodes
    that receive charge are, per axis, the P nodes nearest to it in periodic distance
    (Sec. III.D.2), found here by sorting every node of the axis by its distance."""
    rng = np.random.default_rng(P)
    N = list(_ANISO_MESH)
    h = _ANISO_BOX / np.array(N)
    for _ in range(6):
        x = rng.uniform(-2.0, 7.0, size=3)
        H = o.spread_grid(x[None, :], np.array([1.0]), _ANISO_BOX, N, 1.5, 0.4, P)
        hit = np.nonzero(H)
        for d, axis in ((0, 2), (1, 1), (2, 0)):          # H is [z, y, x]
            nodes = np.arange(N[d])
            dist = np.abs((nodes * h[d] - x[d] + _ANISO_BOX[d] / 2) % _ANISO_BOX[d] - _ANISO_BOX[d] / 2)
            nearest = set(np.argsort(dist)[:P].tolist())
            assert set(hit[axis].tolist()) == nearest


@pytest.mark.parametrize("tol", [1e-8, 1e-10])
def test_spread_grid_carries_the_total_charge(tol):
    """Catches a wrong normalisation constant (the printed (2 xi / pi eta^2)^{3/2} included):
    the grid integrates to the total charge, sum_g H(x_g) h_x h_y h_z = sum q, to the
    window's truncation and quadrature error e^{-pi P/2} (Sec. III.D.2), bounded by tol."""
    p = o.auto_params(_ANISO_BOX, _ANISO_MESH, tol, 0.05)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.0, 6.0, size=(7, 3))
    q = rng.uniform(0.5, 1.5, size=7)
    H = o.spread_grid(x, q, _ANISO_BOX, _ANISO_MESH, p["xi"], p["eta"], p["P"])
    h = _ANISO_BOX / np.array(_ANISO_MESH)
    assert abs(H.sum() * np.prod(h) / q.sum() - 1.0) < 100 * tol


@pytest.mark.parametrize("tol", [1e-8, 1e-10])
def test_spread_grid_transform_is_the_filtered_structure_factor(tol):
    """Catches a wrong window width, a transposed grid axis or a wrong node position.
    By Poisson summation the grid's Fourier coefficients are the structure factor times
    the window's transform e^{-eta k^2/(8 xi^2)} (Sec. III.D.2, the transform pair stated
    with Eq. H_hat), summed over the aliases k' = k + 2 pi (m_x/h_x, m_y/h_y, m_z/h_z):
    h^3 sum_g H(x_g) e^{-i k.x_g} = sum_k' e^{-eta k'^2/(8 xi^2)} sum_b q_b e^{-i k'.x_b},
    to the window's truncation error e^{-pi P/2}, bounded by tol; checked at wave vectors
    along every axis and mixed ones up to k_c."""
    p = o.auto_params(_ANISO_BOX, _ANISO_MESH, tol, 0.05)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 6.0, size=(9, 3))
    q = rng.uniform(-1.0, 1.0, size=9)
    H = o.spread_grid(x, q, _ANISO_BOX, _ANISO_MESH, p["xi"], p["eta"], p["P"])
    two_pi_h = 2 * math.pi * np.array(_ANISO_MESH) / _ANISO_BOX
    aliases = np.array([(i, j, l) for i in range(-2, 3) for j in range(-2, 3) for l in range(-2, 3)])
    for m in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, -1, 1), (-3, 2, -2), (4, 3, -5), (6, 0, 0), (0, 0, -11)]:
        got, k = _grid_dft(H, _ANISO_BOX, m)
        assert np.linalg.norm(k) <= p["k_c"]
        want = 0.0
        for al in aliases:
            kp = k + al * two_pi_h
            want += math.exp(-p["eta"] * float(kp @ kp) / (8 * p["xi"] ** 2)) * np.sum(q * np.exp(-1j * (x @ kp)))
        assert abs(got - want) < 100 * tol * np.abs(q).sum()
        # the first alias matters near k_c (it is what a mesh too coarse for the window would show)
        direct = math.exp(-p["eta"] * float(k @ k) / (8 * p["xi"] ** 2)) * np.sum(q * np.exp(-1j * (x @ k)))
        if np.linalg.norm(k) > 0.85 * p["k_c"]:
            assert abs(direct - want) > 100 * tol * np.abs(q).sum()


# ---------------------------------------------------------------------------
# Rigid-body Brownian step (Sec. V.A): rotation and noise of multi-bead bodies
# ---------------------------------------------------------------------------

def _rotation_vectors(r, rn):
    """Rotation vectors of the rotations taking each body's r[b] onto rn[b]
    (least-squares rotation from the SVD of sum_j rn_j r_j^T, then its axis-angle)."""
    Hm = np.einsum("bji,bjk->bik", rn, r)
    U, _, Vt = np.linalg.svd(Hm)
    D = np.tile(np.eye(3), (len(r), 1, 1))
    D[:, 2, 2] = np.sign(np.linalg.det(U @ Vt))
    R = U @ D @ Vt
    ang = np.arccos(np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1))
    w = np.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0], R[:, 1, 0] - R[:, 0, 1]], axis=1)
    s = np.where(ang > 1e-12, ang / (2 * np.sin(np.maximum(ang, 1e-300))), 0.5)
    return w * s[:, None]


def _ring(n, radius):
    t = 2 * math.pi * np.arange(n) / n
    return np.stack([radius * np.cos(t), radius * np.sin(t), np.zeros(n)], axis=1)


def test_bd_rotation_under_torque_closed_form_inertia():
    """Catches a wrong rotational friction J (a transposed r r^T, |r|^2 dropped) or a
    missing 1/gamma: with kT = 0 the body turns by Omega dt, Omega = (gamma J)^{-1} L,
    where J has a closed form: a ring of n beads of radius R in the xy plane has
    J = n R^2 diag(1/2, 1/2, 1); a regular icosahedron of circumradius R has J = 8 R^2 I.
    The torque comes from two opposite forces on a pair of beads (no net force)."""
    box = np.array([12.0, 12.0, 12.0])
    Xc = np.array([6.0, 5.0, 7.0])
    gamma, dt, Fm = 1.7, 1e-3, 3.0
    ring = _ring(8, 1.3)                     # beads at 45 degree steps: +-y are beads 2 and 6
    ico = G.icosphere(0, 0.9)
    assert ico.shape == (12, 3)
    cases = []
    # ring: forces +-F z on the beads at +-y give L = 2 R F x; and +-F y on the beads at +-x give L = 2 R F z
    f = np.zeros((8, 3)); f[2, 2], f[6, 2] = Fm, -Fm
    f[0, 1], f[4, 1] = Fm, -Fm
    L = np.array([2 * 1.3 * Fm, 0.0, 2 * 1.3 * Fm])
    J = 8 * 1.3 ** 2 * np.diag([0.5, 0.5, 1.0])
    cases.append((ring, f, L, J))
    # icosahedron: +-F e on two opposite vertices n, -n give L = 2 R F (n x e)
    n_hat = ico[0] / np.linalg.norm(ico[0])
    opp = int(np.argmin(ico @ n_hat))
    e = np.cross(n_hat, [0.3, -0.5, 0.8]); e /= np.linalg.norm(e)
    f = np.zeros((12, 3)); f[0], f[opp] = Fm * e, -Fm * e
    cases.append((ico, f, 2 * 0.9 * Fm * np.cross(n_hat, e), 8 * 0.9 ** 2 * np.eye(3)))
    for shape, f, L, J in cases:
        x = Xc + shape
        off = np.array([0, len(shape)])
        xn, Xn = o.bd_step(x, Xc[None, :], off, f, box, 0.05, dt=dt, gamma=gamma, kT=0.0)
        assert np.allclose(Xn[0], Xc, atol=1e-15)              # no net force, no noise
        theta = _rotation_vectors(shape[None], (xn - Xn[0])[None])[0]
        want = np.linalg.solve(gamma * J, L) * dt
        assert np.linalg.norm(theta - want) < 1e-9 * np.linalg.norm(want)


def test_bd_rigid_drag_force_gives_back_its_angular_velocity():
    """Catches a torque or inertia of the wrong sign or handedness, for any body shape:
    bead forces equal to the free-draining drag of a rigid rotation, f_j = gamma w x r_j,
    make the body turn at Omega = w (L = gamma J w is an identity of the cross product)."""
    rng = np.random.default_rng(11)
    box = np.array([9.0, 9.0, 9.0])
    shape = rng.normal(size=(17, 3))
    shape -= shape.mean(axis=0)
    X = np.array([[4.0, 4.5, 5.0]])
    w = np.array([0.4, -1.1, 0.7])
    gamma, dt = 2.5, 1e-3
    f = gamma * np.cross(w, shape)
    xn, Xn = o.bd_step(X + shape, X, np.array([0, 17]), f, box, 0.05, dt=dt, gamma=gamma, kT=0.0)
    theta = _rotation_vectors(shape[None], (xn - Xn[0])[None])[0]
    assert np.linalg.norm(theta - w * dt) < 1e-9 * np.linalg.norm(w * dt)


def test_bd_body_noise_covariance():
    """Catches a wrong noise amplitude (a lost factor 2 or square root, the translational
    1/N_i, or the Cholesky factor of J in place of that of J^{-1}): over 10,000 draws of
    force-free 8-bead rings, the body displacement has variance 2 kT dt/(N_i gamma) per
    axis and the rotation vector has covariance 2 kT dt (gamma J)^{-1}, J = n R^2 diag(1/2, 1/2, 1)
    (fluctuation-dissipation with the free-draining mobility of Sec. V.A)."""
    box = np.array([10.0, 10.0, 10.0])
    n, R = 8, 1.0
    ring = _ring(n, R)
    nb = 2000
    X = np.tile([5.0, 5.0, 5.0], (nb, 1))
    x = (X[:, None, :] + ring[None]).reshape(-1, 3)
    off = np.arange(nb + 1) * n
    kT, dt, gamma = 1.3, 1e-3, 2.0
    th, dX = [], []
    for step in range(5):
        xn, Xn = o.bd_step(x, X, off, np.zeros_like(x), box, 0.05, dt=dt, gamma=gamma, kT=kT, seed=99, step=step)
        th.append(_rotation_vectors(np.repeat(ring[None], nb, 0), xn.reshape(nb, n, 3) - Xn[:, None, :]))
        dX.append(Xn - X)
    th = np.concatenate(th)
    dX = np.concatenate(dX)
    m = th.shape[0]
    sd = 5 * math.sqrt(2.0 / m)                     # five standard errors of a variance ratio
    var_t = 2 * kT * dt / (n * gamma)
    assert np.all(np.abs(dX.var(axis=0) / var_t - 1) < sd)
    assert np.all(np.abs(dX.mean(axis=0)) < 5 * math.sqrt(var_t / m))
    C = 2 * kT * dt * np.linalg.inv(gamma * n * R * R * np.diag([0.5, 0.5, 1.0]))
    cov = np.cov(th.T)
    d = np.sqrt(np.diag(C))
    corr = cov / np.outer(d, d)
    assert np.all(np.abs(np.diag(corr) - 1) < sd)
    assert np.all(np.abs(corr - np.diag(np.diag(corr))) < 5 / math.sqrt(m))


# ---------------------------------------------------------------------------
# Grand capacitance tensor, Eq. QS_capacitance
# ---------------------------------------------------------------------------

def _sphere_in_box(L, a=0.1, eps=1.0, level=2):
    x = G.icosphere(level) + L / 2
    return C.assemble("sphere", [x], [], [], [0.0], [L] * 3, a, eps, [[0.0, 0.0, 1.0]])


def test_grand_capacitance_reproduces_the_saddle_solution():
    """Catches a transposed Sigma', a wrong sign or a missing r_ij: by Eq. QS_capacitance the
    saddle solution of Eq. saddle for given Q and E0 has [Q; S] = C [Psi - Psi_0; E0] (the
    same field on every body), and C is symmetric positive definite."""
    s = C.small_system(seed=12, n_bodies=3, level=1, n_ions=0, L=7.0, a=0.2, charged=True)
    Cm = o.grand_capacitance(s.x, s.X, s.body_offsets, s.box, s.a, s.eps)
    nb = s.n_bodies
    assert Cm.shape == (4 * nb, 4 * nb)
    assert np.allclose(Cm, Cm.T, rtol=0, atol=1e-9 * np.abs(Cm).max())
    assert np.linalg.eigvalsh(0.5 * (Cm + Cm.T)).min() > 0
    rng = np.random.default_rng(3)
    for _ in range(3):
        E0 = rng.normal(size=3)
        Q = rng.normal(size=nb)
        q, psi = o.solve_dense(s.x, s.body_offsets, s.X, Q, E0, s.box, s.a, s.eps)
        S = o.dipoles(s.x, s.X, s.body_offsets, q, s.box)
        lhs = np.concatenate([Q, S.ravel()])
        rhs = Cm @ np.concatenate([psi, np.tile(E0, nb)])
        assert np.max(np.abs(lhs - rhs)) < 1e-8 * np.abs(lhs).max()


def test_sphere_charge_capacitance_in_a_periodic_box():
    """Catches a wrong k = 0 treatment or charge block: a charged conducting sphere in a
    cubic box with the uniform neutralizing background of Sec. II has
    1/C_QPsi(L) = 1/C_isolated - w/(4 pi eps L) + a_s^2/(3 eps L^3), w the simple-cubic
    Wigner constant (its images) and the last term the background inside the sphere
    (mean |r_i - r_j|^2 = 2 a_s^2 over its surface); differences between boxes cancel
    the tessellation's C_isolated."""
    w = GOLDEN["wigner_constant_simple_cubic"]["value"]
    eps = 1.0
    inv = {L: 1.0 / o.grand_capacitance(*(lambda s: (s.x, s.X, s.body_offsets, s.box, s.a, s.eps))(
        _sphere_in_box(L, eps=eps)))[0, 0] for L in (6.0, 8.0, 12.0, 16.0)}
    for L1, L2 in ((6.0, 12.0), (8.0, 16.0)):
        want = -w / (4 * math.pi * eps) * (1 / L1 - 1 / L2) + (1 / (3 * eps)) * (1 / L1 ** 3 - 1 / L2 ** 3)
        got = inv[L1] - inv[L2]
        assert abs(got / want - 1) < 2e-3, (L1, L2, got, want)
        # without the Wigner term the difference would be off by far more
        assert abs(inv[L1] - inv[L2]) > 10 * abs((1 / (3 * eps)) * (1 / L1 ** 3 - 1 / L2 ** 3))


def test_sphere_polarizability_in_a_cubic_lattice_is_clausius_mossotti():
    """Catches a wrong field block or lattice sum: one sphere per cubic cell (a simple
    cubic lattice) has the dipole response C_SE = alpha / (1 - alpha/(3 eps V)) with the
    isolated polarizability alpha (Lorentz local field), the charge-dipole blocks vanish
    by symmetry, and eps_eff = eps (1 + C_SE/(eps V)) is Clausius-Mossotti's
    (1 + 2 phi)/(1 - phi) with phi = alpha/(4 pi eps) (4 pi/3)/V (Sec. IV.C at low phi)."""
    eps = 1.3
    caps = {}
    for L in (6.0, 16.0):
        s = _sphere_in_box(L, eps=eps)
        Cm = o.grand_capacitance(s.x, s.X, s.body_offsets, s.box, s.a, s.eps)
        assert np.abs(Cm[0, 1:]).max() < 1e-10 * Cm[0, 0]
        d = np.diag(Cm)[1:]
        assert np.ptp(d) < 1e-8 * d.mean()                       # isotropic
        assert np.abs(Cm[1:, 1:] - np.diag(d)).max() < 1e-8 * d.mean()
        caps[L] = d.mean()
    V16, V6 = 16.0 ** 3, 6.0 ** 3
    alpha = caps[16.0] / (1 + caps[16.0] / (3 * eps * V16))      # invert the same relation at L = 16
    want = alpha / (1 - alpha / (3 * eps * V6))
    assert abs(caps[6.0] / want - 1) < 1e-4, (caps[6.0], want)
    phi = alpha / (4 * math.pi * eps) * (4 * math.pi / 3) / V6
    eps_eff = eps * (1 + caps[6.0] / (eps * V6))
    assert abs(eps_eff / (eps * (1 + 2 * phi) / (1 - phi)) - 1) < 1e-4
    # the lattice raises the dipole above the isolated sphere's by the factor 1/(1 - phi)
    assert caps[6.0] > alpha * (1 + 0.9 * phi)
