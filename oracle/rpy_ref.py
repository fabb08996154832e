"""Plain FP64 CPU oracle for the periodic Rotne-Prager-Yamakawa mobility (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and never calls it.

The paper leaves hydrodynamic interactions out and names the RPY tensor as the way
to add them (Sec. V.A, Eq. velocity): u_alpha = sum_beta M^H_alpha_beta . F_beta.
Here M^H is the RPY tensor of beads of radius a in a fluid of viscosity mu: the
Oseen tensor averaged over the surfaces of both beads, whose transform is
    M_hat(k) = j0^2(ka) (I - k_hat k_hat) / (mu k^2),
the same j0^2(ka) shape factor as the electrostatic kernel of Eq. M00_Fourier.  In a
periodic box the k = 0 mode is left out (the mean force is balanced by a pressure
gradient).  The sum is split with Hasimoto's weight H(k) = (1 + k^2/(4 xi^2)) e^{-k^2/(4 xi^2)}:
    wave space: (1/(mu V)) sum_{k != 0} j0^2(ka) H(k) (I - k_hat k_hat)/k^2 e^{i k.r}, explicitly per k;
    real space: sum over images of M_r(r) = M_RPY(r) - M_w(r) with M_w the inverse
    transform of the wave kernel over all k, a radial quadrature; M_r decays like
    e^{-xi^2 r^2} because (1 - H(k))/k^2 is smooth at k = 0 (no k = 0 correction).
The rigid-body mobility problem of the paper's last equation (constraint forces and body motions)
is solved densely on top of it (rigid_mobility).
An isotropic kernel f(k) (I - k_hat k_hat) has the real-space form A(r) I + B(r) r_hat r_hat with
    A = 1/(2 pi^2) int f k^2 [j0(kr) - j1(kr)/(kr)] dk,  B = 1/(2 pi^2) int f k^2 [3 j1(kr)/(kr) - j0(kr)] dk.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad


def rpy_free(r: float, a: float, mu: float = 1.0):
    """(A, B) of the free-space RPY tensor M = A I + B r_hat r_hat of two beads of radius a:
    r >= 2a: A = (1 + 2a^2/(3r^2))/(8 pi mu r), B = (1 - 2a^2/r^2)/(8 pi mu r);
    r < 2a:  A = (1 - 9r/(32a))/(6 pi mu a), B = 3r/(32a)/(6 pi mu a) (the overlapping form)."""
    if r >= 2.0 * a:
        return ((1.0 + 2.0 * a * a / (3.0 * r * r)) / (8.0 * math.pi * mu * r),
                (1.0 - 2.0 * a * a / (r * r)) / (8.0 * math.pi * mu * r))
    return ((1.0 - 9.0 * r / (32.0 * a)) / (6.0 * math.pi * mu * a), (3.0 * r / (32.0 * a)) / (6.0 * math.pi * mu * a))


def _wave_weight(k, a, xi):
    """j0^2(ka) H(k): the wave kernel's shape factor times Hasimoto's weight."""
    return (np.sin(k * a) / (k * a)) ** 2 * (1.0 + k * k / (4.0 * xi * xi)) * np.exp(-k * k / (4.0 * xi * xi))


def _j1_over_x(x):
    """j1(x)/x = (sin x - x cos x)/x^3, by its series below 1e-2."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-2
    xs = np.where(small, 1.0, x)
    x2 = x * x
    return np.where(small, 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0, (np.sin(xs) - xs * np.cos(xs)) / xs ** 3)


def _j0v(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))


def rpy_wave_radial(r, a: float, xi: float, mu: float = 1.0, panels: int = 96, order: int = 24):
    """(A_w, B_w) at the distances r (array): inverse transform over all k of the wave kernel
    j0^2(ka) H(k) (I - k_hat k_hat)/(mu k^2), by Gauss-Legendre quadrature on panels of
    [0, 14 xi] (the integrand falls like e^{-k^2/(4 xi^2)}: below 1e-19 of its size there)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    kmax = 14.0 * xi
    t, wt = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0.0, kmax, panels + 1)
    k = (0.5 * (edges[1:] - edges[:-1])[:, None] * (t[None, :] + 1.0) + edges[:-1, None]).reshape(-1)
    w = (0.5 * (edges[1:] - edges[:-1])[:, None] * wt[None, :]).reshape(-1) * _wave_weight(k, a, xi)
    x = r[:, None] * k[None, :]
    j0 = _j0v(x)
    jx = _j1_over_x(x)
    c = 1.0 / (2.0 * math.pi ** 2 * mu)
    return c * ((j0 - jx) @ w), c * ((3.0 * jx - j0) @ w)


def rpy_real_radial(r, a: float, xi: float, mu: float = 1.0):
    """(A_r, B_r) of the real-space kernel M_r = M_RPY - M_w at the distances r (array;
    r = 0: the self term, B = 0)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    Af = np.array([rpy_free(v, a, mu)[0] for v in r])
    Bf = np.array([rpy_free(v, a, mu)[1] for v in r])
    Aw, Bw = rpy_wave_radial(r, a, xi, mu)
    return Af - Aw, Bf - Bw


def rpy_split(box, a: float, tol: float = 1e-13, xi: float | None = None):
    """(xi, r_c, k_c) of the oracle's own Hasimoto split: both truncations ~ e^{-x^2} up to
    powers, so r_c = s/xi + 2a and k_c = 2 xi s with s = sqrt(ln(1/tol)) plus a margin."""
    box = np.asarray(box, dtype=np.float64)
    if xi is None:
        xi = 3.0 / float(np.min(box)) * 2.0
    s = math.sqrt(math.log(1.0 / tol)) + 1.0
    return float(xi), s / xi + 2.0 * a, 2.0 * xi * s


def rpy_mobility(x, F, box, a: float, mu: float = 1.0, targets=None, xi=None, tol=1e-13):
    """U_alpha = sum_beta M^H_alpha_beta . F_beta (periodic RPY, k = 0 left out) at the targets.

    x: [n,3]; F: [n,3]; box: [3]; returns U [nt,3]."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 3)
    box = np.asarray(box, dtype=np.float64).reshape(3)
    n = x.shape[0]
    targets = np.arange(n) if targets is None else np.asarray(targets)
    xi, rc, kc = rpy_split(box, a, tol, xi)
    V = float(np.prod(box))
    U = np.zeros((len(targets), 3))
    # real space: every source and image within r_c (the bead itself at n = 0 gives the self term)
    m = [int(math.ceil((rc + 0.5 * L) / L)) for L in box]
    shifts = np.array([[i, j, k] for i in range(-m[0], m[0] + 1) for j in range(-m[1], m[1] + 1)
                       for k in range(-m[2], m[2] + 1)], dtype=np.float64) * box
    for t, al in enumerate(targets):
        d0 = x[al] - x
        d0 -= box * np.floor(d0 / box + 0.5)
        d = (d0[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
        src = np.tile(np.arange(n), len(shifts))
        r = np.sqrt(np.sum(d * d, axis=1))
        sel = r < rc
        d, src, r = d[sel], src[sel], r[sel]
        A, B = rpy_real_radial(r, a, xi, mu)
        e = d / np.where(r > 0.0, r, 1.0)[:, None]
        Fs = F[src]
        U[t] = A @ Fs + (B * np.sum(e * Fs, axis=1)) @ e
    # wave space: explicit sum over k != 0, |k| <= k_c
    mk = [int(math.floor(kc * L / (2.0 * math.pi))) for L in box]
    g = [2.0 * math.pi * np.arange(-mm, mm + 1) / L for mm, L in zip(mk, box)]
    K = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)
    k2 = np.sum(K * K, axis=1)
    keep = (k2 > 0) & (k2 <= kc * kc)
    K, k2 = K[keep], k2[keep]
    kk = np.sqrt(k2)
    w = _wave_weight(kk, a, xi) / k2 / (mu * V)
    kh = K / kk[:, None]
    for s0 in range(0, K.shape[0], 2048):
        sl = slice(s0, s0 + 2048)
        ph = x @ K[sl].T                                  # [n, nk]
        Sre = np.cos(ph).T @ F                            # [nk, 3]: sum_beta F_beta cos(k.x_beta)
        Sim = -np.sin(ph).T @ F                           #           and -sin
        # project each k's force transform: (I - k_hat k_hat) S
        Pre = Sre - kh[sl] * np.sum(kh[sl] * Sre, axis=1)[:, None]
        Pim = Sim - kh[sl] * np.sum(kh[sl] * Sim, axis=1)[:, None]
        pt = x[targets] @ K[sl].T                         # [nt, nk]
        # Re(e^{i k.x_alpha} (Pre + i Pim)) weighted by w
        U += (np.cos(pt) * w[sl]) @ Pre - (np.sin(pt) * w[sl]) @ Pim
    return U


def rpy_matrix(x, box, a: float, mu: float = 1.0, xi=None, tol=1e-13):
    """Dense 3n x 3n periodic RPY mobility (bead-major, component-minor), column by column."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = x.shape[0]
    M = np.zeros((3 * n, 3 * n))
    for c in range(3 * n):
        F = np.zeros((n, 3))
        F[c // 3, c % 3] = 1.0
        M[:, c] = rpy_mobility(x, F, box, a, mu, xi=xi, tol=tol).reshape(-1)
    return M


def rigid_operator(x, X, body_offsets, box):
    """K (3n x 6 n_b): bead velocities K W = U_b + Omega_b x r_j of rigid-body motions W = (U, Omega)
    per body, r_j the bead's minimum-image position relative to its body's reference point.
    Single-bead bodies move by U alone (their Omega columns are zero)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    off = np.asarray(body_offsets, dtype=np.int64)
    n, nb = x.shape[0], len(off) - 1
    X = np.asarray(X, dtype=np.float64).reshape(nb, 3)
    box = np.asarray(box, dtype=np.float64)
    K = np.zeros((3 * n, 6 * nb))
    for b in range(nb):
        for j in range(off[b], off[b + 1]):
            K[3 * j:3 * j + 3, 6 * b:6 * b + 3] = np.eye(3)
            if off[b + 1] - off[b] > 1:
                r = x[j] - X[b]
                r -= box * np.floor(r / box + 0.5)
                # Omega x r = -[r]_x Omega
                K[3 * j:3 * j + 3, 6 * b + 3:6 * b + 6] = -np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]],
                                                                      [-r[1], r[0], 0.0]])
    return K


def rigid_mobility(x, X, body_offsets, box, a: float, FL, mu: float = 1.0, M=None):
    """Rigid-body mobility problem (the paper's last equation, physical sign): bead constraint
    forces f and body motions W = (U, Omega) with
        M f = K W          (the beads move rigidly with their bodies),
        K^T f = (F, L)     (the bead forces add up to each body's force and torque),
    M the periodic RPY mobility of the beads.  A single-bead body has no rotation: its Omega is
    set to zero and its torque is not an equation.  Dense LU.  FL: [n_b, 6] (F, L);
    returns W [n_b, 6] and f [n, 3]."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    off = np.asarray(body_offsets, dtype=np.int64)
    n, nb = x.shape[0], len(off) - 1
    if M is None:
        M = rpy_matrix(x, box, a, mu)
    K = rigid_operator(x, X, off, box)
    A = np.block([[M, -K], [K.T, np.zeros((6 * nb, 6 * nb))]])
    rhs = np.zeros(3 * n + 6 * nb)
    G = np.array(FL, dtype=np.float64).reshape(nb, 6).copy()
    for b in range(nb):
        if off[b + 1] - off[b] == 1:
            G[b, 3:] = 0.0
            for d in range(3):
                A[3 * n + 6 * b + 3 + d, 3 * n + 6 * b + 3 + d] = 1.0
    rhs[3 * n:] = G.reshape(-1)
    z = np.linalg.solve(A, rhs)
    return z[3 * n:].reshape(nb, 6), z[:3 * n].reshape(n, 3)


__all__ = ["rpy_free", "rpy_wave_radial", "rpy_real_radial", "rpy_split", "rpy_mobility", "rpy_matrix",
           "rigid_operator", "rigid_mobility"]
