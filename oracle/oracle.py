"""Plain FP64 CPU oracle for arXiv:2401.04865 (immersed-boundary electrostatics).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and never calls it.

What it computes, each function citing the passage it follows:

* Ewald sums of the regularized potential tensor M (Sec. II, Eq. M00_Fourier;
  Sec. III.D, Eq. splitting): real space directly over image shells, wave
  space as an explicit k-vector sum (both in ``ewald_ref.c``), self term.
  Beads of unequal radii (the paper fixes one, Sec. III.A): pass one radius
  per bead; pairs then interact through j0(k a_alpha) j0(k a_beta)/k^2, the
  real-space kernel being the average of erfc(xi s)/(4 pi s) over both shells.
* The dense matrix M for small systems (real part from ``ewald_ref.c``, wave
  part as C diag(G) C^T + S diag(G) S^T with C = cos(K x), S = sin(K x)).
* The saddle system of Eq. saddle, solved by dense LU (numpy.linalg.solve)
  or by textbook restarted GMRES (Saad) on the matrix-free operator.
* The grand capacitance tensor C = Sigma' M^{-1} Sigma'^T (Eq. QS_capacitance)
  by dense LU.
* Dipoles (Eq. rigid_dipole), energy (Eq. pot_syst), bead forces
  (Eq. beadforce: f = q (E0 + E) with E the field of all other charges),
  body forces and torques (Sec. III.C), the Brownian-dynamics step of
  Sec. V.A with the hard-sphere pair potential Eq. hardsphereFD.
* The parameter rules of Sec. III.D.2 (N_g, eta, P) as the library's
  automatic setup must apply them.
* Philox4x32-10 (Salmon et al., SC'11) and Box-Muller, for the Brownian noise.

Units: every potential is psi - psi_0 (Eq. pot_charge); eps is eps_f.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

_LIB = None


def lib():
    """Load (building on first use) the C part of the oracle."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.ibo_M_free.restype = d
        L.ibo_M_free.argtypes = [d, d]
        L.ibo_phi_self.restype = d
        L.ibo_phi_self.argtypes = [d, d]
        L.ibo_phi_real.restype = d
        L.ibo_phi_real.argtypes = [d, d, d]
        L.ibo_dphi_real.restype = d
        L.ibo_dphi_real.argtypes = [d, d, d]
        L.ibo_real_sum.restype = None
        L.ibo_real_sum.argtypes = [i, p, p, p, d, d, d, d, i, p, p, p]
        L.ibo_wave_sum.restype = None
        L.ibo_wave_sum.argtypes = [i, p, p, p, d, d, d, d, i, p, p, p]
        L.ibo_wave_vectors.restype = ctypes.c_long
        L.ibo_wave_vectors.argtypes = [p, d, d, d, ctypes.c_long, p]
        L.ibo_real_matrix.restype = None
        L.ibo_real_matrix.argtypes = [i, p, p, d, d, d, p]
        L.ibo_M_free2.restype = d
        L.ibo_M_free2.argtypes = [d, d, d]
        L.ibo_phi_real2.restype = d
        L.ibo_phi_real2.argtypes = [d, d, d, d]
        L.ibo_dphi_real2.restype = d
        L.ibo_dphi_real2.argtypes = [d, d, d, d]
        L.ibo_real_sum_radii.restype = None
        L.ibo_real_sum_radii.argtypes = [i, p, p, p, p, d, d, d, i, p, p, p]
        L.ibo_wave_sum_radii.restype = None
        L.ibo_wave_sum_radii.argtypes = [i, p, p, p, p, d, d, d, i, p, p, p]
        L.ibo_real_matrix_radii.restype = None
        L.ibo_real_matrix_radii.argtypes = [i, p, p, p, d, d, p]
        L.ibo_num_threads.restype = i
        _LIB = L
    return _LIB


def num_threads() -> int:
    """OpenMP threads the C part of the oracle uses."""
    return int(lib().ibo_num_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# Kernels (Sec. II and Sec. III.D.1)
# ---------------------------------------------------------------------------

def M_free(r: float, a: float) -> float:
    """Real-space regularized tensor (Sec. II), without 1/eps."""
    return lib().ibo_M_free(float(r), float(a))


def phi_real(r: float, a: float, xi: float) -> float:
    """Real-space Ewald kernel, Eq. psi_Re_1 (sign reading: see ewald_ref.c)."""
    return lib().ibo_phi_real(float(r), float(a), float(xi))


def dphi_real(r: float, a: float, xi: float) -> float:
    """d phi_real / dr."""
    return lib().ibo_dphi_real(float(r), float(a), float(xi))


def phi_self(a: float, xi: float) -> float:
    """Self term (Sec. III.D.1, the r -> 0 limit of Eq. psi_Re_1)."""
    return lib().ibo_phi_self(float(a), float(xi))


def M_free2(r: float, a: float, b: float) -> float:
    """Free-space potential between shells of radii a and b (real-space form of
    j0(ka) j0(kb)/k^2), without 1/eps."""
    return lib().ibo_M_free2(float(r), float(a), float(b))


def phi_real2(r: float, a: float, b: float, xi: float) -> float:
    """Real-space Ewald kernel of two beads of radii a and b (ewald_ref.c)."""
    return lib().ibo_phi_real2(float(r), float(a), float(b), float(xi))


def dphi_real2(r: float, a: float, b: float, xi: float) -> float:
    """d phi_real2 / dr."""
    return lib().ibo_dphi_real2(float(r), float(a), float(b), float(xi))


def _radii(a, n):
    """None for one radius (a scalar), else the per-bead radii as a C array."""
    if np.ndim(a) == 0:
        return None
    rad = _c(a).reshape(-1)
    if rad.shape[0] != n:
        raise ValueError("one radius per bead expected")
    return rad


def _amax(a) -> float:
    return float(np.max(a))


# ---------------------------------------------------------------------------
# Ewald sums
# ---------------------------------------------------------------------------

def ewald_split(box, a: float, n_src: int, tol: float = 1e-13, xi: float | None = None):
    """The oracle's own Ewald split (xi, r_c, k_c) for accuracy ``tol``.

    Real-space truncation ~ e^{-r_c^2 xi^2} (Eq. realspaceerror), wave-space
    truncation ~ e^{-k_c^2/(4 xi^2)} (Sec. III.D.2).  Unless given, xi balances
    the two sums with the classic sqrt(pi) (N/V^2)^{1/6}; the result does not
    depend on xi beyond ``tol`` (a test checks this).
    """
    box = np.asarray(box, dtype=np.float64)
    V = float(np.prod(box))
    if xi is None:
        xi = math.sqrt(math.pi) * (max(n_src, 1) / V ** 2) ** (1.0 / 6.0)
    s = math.sqrt(math.log(1.0 / tol))
    rc = s / xi + 2.0 * _amax(a)
    kc = 2.0 * xi * s
    return float(xi), float(rc), float(kc)


def k0_term(box, xi, eps):
    """k = 0 Fourier weight carried by the real-space image sum.

    By Poisson summation, sum_n phi_r(|r + n L|) = (1/V) sum_k phihat_r(k) e^{i k.r}
    over ALL k, and phihat_r(k) = j0^2(ka)(1 - e^{-k^2/4xi^2})/k^2 -> 1/(4 xi^2) at
    k = 0.  M of Eq. M00_Fourier has no k = 0 term (Sec. II: electroneutrality), so
    1/(4 xi^2 V eps) is subtracted from every element; for neutral charges it cancels."""
    V = float(np.prod(np.asarray(box, dtype=np.float64)))
    return 1.0 / (4.0 * xi * xi * V * eps)


def potential(x, q, box, a, eps, targets=None, field=False, xi=None, tol=1e-13):
    """psi_alpha - psi_0 (and E_alpha) at the targets, Eq. splitting + self term.

    x: [n,3]; q: [n]; box: [3]; a: the bead radius, or one radius per bead [n]
    (pair kernel j0(k a_alpha) j0(k a_beta)/k^2); returns psi [nt] (and E [nt,3]).
    """
    x = _c(x).reshape(-1, 3)
    q = _c(q).reshape(-1)
    box = _c(box).reshape(3)
    n = x.shape[0]
    if targets is None:
        targets = np.arange(n, dtype=np.int32)
    targets = _c(targets, np.int32)
    nt = targets.shape[0]
    xi, rc, kc = ewald_split(box, a, n, tol, xi)
    L = lib()
    pr = np.zeros(nt)
    pk = np.zeros(nt)
    Er = np.zeros((nt, 3)) if field else None
    Ek = np.zeros((nt, 3)) if field else None
    rad = _radii(a, n)
    if rad is None:
        L.ibo_real_sum(n, _ptr(x), _ptr(q), _ptr(box), a, xi, rc, eps, nt, _ptr(targets), _ptr(pr), _ptr(Er))
        L.ibo_wave_sum(n, _ptr(x), _ptr(q), _ptr(box), a, xi, kc, eps, nt, _ptr(targets), _ptr(pk), _ptr(Ek))
    else:
        L.ibo_real_sum_radii(n, _ptr(x), _ptr(q), _ptr(box), _ptr(rad), xi, rc, eps, nt, _ptr(targets), _ptr(pr),
                             _ptr(Er))
        L.ibo_wave_sum_radii(n, _ptr(x), _ptr(q), _ptr(box), _ptr(rad), xi, kc, eps, nt, _ptr(targets), _ptr(pk),
                             _ptr(Ek))
    # k = 0 is excluded from M (Sec. II); the real-space image sum carries it (see k0_term)
    pb = -k0_term(box, xi, eps) * float(np.sum(q))
    if field:
        return pr + pk + pb, Er + Ek
    return pr + pk + pb


def wave_vectors(box, a, xi, kc):
    """All k != 0 with |k| <= kc and their weights G(k) = j0^2(ka) e^{-k^2/4xi^2}/k^2."""
    box = _c(box).reshape(3)
    nk = lib().ibo_wave_vectors(_ptr(box), a, xi, kc, 0, None)
    out = np.zeros((max(nk, 1), 4))
    lib().ibo_wave_vectors(_ptr(box), a, xi, kc, nk, _ptr(out))
    return out[:nk, :3].copy(), out[:nk, 3].copy()


def M_dense(x, box, a, eps, xi=None, tol=1e-13, k_chunk=4096):
    """Dense potential tensor M (Eq. M00_Fourier) of the periodic system.

    M = (1/eps) [ real-space matrix (with self term) + (1/V) sum_k G(k) cos(k.(x_a - x_b)) ].
    The wave part uses cos(k.(x_a-x_b)) = cos(k.x_a)cos(k.x_b) + sin(k.x_a)sin(k.x_b),
    i.e. C diag(G) C^T + S diag(G) S^T, accumulated over chunks of k.  With one radius
    per bead the j0 factors move out of G onto the rows: C_ak = j0(k a_a) cos(k.x_a).
    """
    x = _c(x).reshape(-1, 3)
    box = _c(box).reshape(3)
    n = x.shape[0]
    xi, rc, kc = ewald_split(box, a, n, tol, xi)
    rad = _radii(a, n)
    Mr = np.zeros((n, n))
    if rad is None:
        lib().ibo_real_matrix(n, _ptr(x), _ptr(box), a, xi, rc, _ptr(Mr))
        K, G = wave_vectors(box, a, xi, kc)
    else:
        lib().ibo_real_matrix_radii(n, _ptr(x), _ptr(box), _ptr(rad), xi, rc, _ptr(Mr))
        K, _ = wave_vectors(box, 1.0, xi, kc)
        k2 = np.sum(K * K, axis=1)
        G = np.exp(-k2 / (4.0 * xi * xi)) / k2
    V = float(np.prod(box))
    Mw = np.zeros((n, n))
    for s in range(0, K.shape[0], k_chunk):
        ph = x @ K[s:s + k_chunk].T
        C = np.cos(ph)
        S = np.sin(ph)
        if rad is not None:
            kk = np.sqrt(np.sum(K[s:s + k_chunk] ** 2, axis=1))
            J = np.sin(rad[:, None] * kk[None, :]) / (rad[:, None] * kk[None, :])
            C = C * J
            S = S * J
        g = G[s:s + k_chunk]
        Mw += (C * g) @ C.T + (S * g) @ S.T
    return (Mr + Mw / V) / eps - k0_term(box, xi, eps)


def spread_grid(x, q, box, mesh, xi, eta, P):
    """The spread grid of Eq. H_hat, written out:
    H(x_g) = (2 xi^2/(pi eta))^{3/2} sum_beta q_beta exp(-2 xi^2 |x_g - x_beta|^2 / eta)
    on the nodes x_g = (i h_x, j h_y, k h_z), h_d = L_d / N_d, each bead restricted
    to the P closest nodes per axis (Sec. III.D.2), i.e. the nodes
    floor(x/h - P/2) + 1 ... floor(x/h - P/2) + P, taken periodically.
    Returns [N_z, N_y, N_x] (x fastest)."""
    x = _c(x).reshape(-1, 3)
    box = _c(box).reshape(3)
    N = [int(m) for m in mesh]
    h = box / np.array(N, dtype=np.float64)
    c = (2.0 * xi * xi / (math.pi * eta)) ** 1.5
    H = np.zeros((N[2], N[1], N[0]))
    for b in range(x.shape[0]):
        idx, w = [], []
        for d in range(3):
            xd = x[b, d] - box[d] * math.floor(x[b, d] / box[d])
            u = xd / h[d]
            s = math.floor(u - 0.5 * P) + 1
            nodes = s + np.arange(P)
            dist = nodes * h[d] - xd
            w.append(np.exp(-2.0 * xi * xi * dist * dist / eta))
            idx.append(np.mod(nodes, N[d]))
        blk = c * q[b] * w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :]
        np.add.at(H, np.ix_(idx[2], idx[1], idx[0]), blk)
    return H


# ---------------------------------------------------------------------------
# Bodies: summation tensor, relative positions (Sec. III.B and Appendix)
# ---------------------------------------------------------------------------

def min_image(d, box):
    box = np.asarray(box, dtype=np.float64)
    return d - box * np.floor(d / box + 0.5)


def body_index(body_offsets):
    """Body id of every bead from the CSR offsets (bodies are contiguous, Appendix)."""
    off = np.asarray(body_offsets, dtype=np.int64)
    counts = np.diff(off)
    return np.repeat(np.arange(len(counts)), counts)


def sigma_matrix(body_offsets, n):
    """Summation tensor Sigma (Appendix, Eq. Sigma1): N_b x N, ones on each body's beads."""
    off = np.asarray(body_offsets, dtype=np.int64)
    nb = len(off) - 1
    Sg = np.zeros((nb, n))
    for i in range(nb):
        Sg[i, off[i]:off[i + 1]] = 1.0
    return Sg


def relative_positions(x, X, body_offsets, box):
    """r_ij = x_ij - X_i (Sec. III.B), as the minimum periodic image."""
    bid = body_index(body_offsets)
    return min_image(np.asarray(x, dtype=np.float64) - np.asarray(X, dtype=np.float64)[bid], box)


# ---------------------------------------------------------------------------
# Saddle-point system, Eq. saddle
# ---------------------------------------------------------------------------

def saddle_rhs(x, X, body_offsets, Q, E0, box):
    """Right-hand side [-r.E0 ; Q] of Eq. saddle."""
    r = relative_positions(x, X, body_offsets, box)
    return np.concatenate([-(r @ np.asarray(E0, dtype=np.float64)), np.asarray(Q, dtype=np.float64)])


def saddle_matrix(M, body_offsets):
    """[[-M, Sigma^T], [Sigma, 0]] of Eq. saddle."""
    n = M.shape[0]
    Sg = sigma_matrix(body_offsets, n)
    nb = Sg.shape[0]
    A = np.zeros((n + nb, n + nb))
    A[:n, :n] = -M
    A[:n, n:] = Sg.T
    A[n:, :n] = Sg
    return A


def solve_dense(x, body_offsets, X, Q, E0, box, a, eps, M=None, xi=None):
    """Solve Eq. saddle by dense LU with partial pivoting (LAPACK gesv).

    Returns q [n] and Psi - Psi_0 [n_b].  E0 may be [3] or [R,3]; for R
    right-hand sides q is [R,n] and Psi - Psi_0 is [R,n_b].
    """
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    if M is None:
        M = M_dense(x, box, a, eps, xi=xi)
    A = saddle_matrix(M, body_offsets)
    E0 = np.asarray(E0, dtype=np.float64)
    many = E0.ndim == 2
    E0s = E0 if many else E0[None, :]
    B = np.stack([saddle_rhs(x, X, body_offsets, Q, e, box) for e in E0s], axis=1)
    U = np.linalg.solve(A, B)
    q, psi = U[:n].T, U[n:].T
    return (q, psi) if many else (q[0], psi[0])


def gmres(matvec, b, x0=None, rtol=1e-10, restart=50, max_iter=5000):
    """Restarted GMRES(m) (Saad & Schultz 1986; Saad, Iterative Methods, Alg. 6.9):
    Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
    matrix, stop when ||b - A x|| <= rtol ||b|| (true residual at each restart).
    Returns (x, iterations, relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * nb or it >= max_iter:
            return x, it, beta / nb
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_used = j + 1
            if abs(g[j + 1]) <= rtol * nb or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y


def saddle_operator(x, body_offsets, box, a, eps, xi=None, tol=1e-13):
    """Matrix-free operator of Eq. saddle using the oracle's Ewald sums."""
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    off = np.asarray(body_offsets, dtype=np.int64)
    bid = body_index(off)

    def matvec(v):
        q = v[:n]
        psi = v[n:]
        Mq = potential(x, q, box, a, eps, xi=xi, tol=tol)
        top = -Mq + psi[bid]
        bot = np.add.reduceat(q, off[:-1]) if n else np.zeros(len(off) - 1)
        return np.concatenate([top, bot])

    return matvec


def solve_gmres(x, body_offsets, X, Q, E0, box, a, eps, rtol=1e-10, restart=50, xi=None):
    """Solve Eq. saddle by restarted GMRES on the matrix-free oracle operator."""
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    A = saddle_operator(x, body_offsets, box, a, eps, xi=xi)
    b = saddle_rhs(x, X, body_offsets, Q, E0, box)
    u, it, res = gmres(A, b, rtol=rtol, restart=restart)
    return u[:n], u[n:], it, res


def sigma_prime(x, X, body_offsets, box):
    """Sigma' of Eq. QS_capacitance (Appendix): 4 N_b x N; rows 0..N_b-1 are Sigma,
    row N_b + 3 i + d holds r_ij,d on the beads of body i (body-major)."""
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    off = np.asarray(body_offsets, dtype=np.int64)
    nb = len(off) - 1
    r = relative_positions(x, X, off, box)
    Sp = np.zeros((4 * nb, n))
    for i in range(nb):
        Sp[i, off[i]:off[i + 1]] = 1.0
        for d in range(3):
            Sp[nb + 3 * i + d, off[i]:off[i + 1]] = r[off[i]:off[i + 1], d]
    return Sp


def grand_capacitance(x, X, body_offsets, box, a, eps, M=None, xi=None):
    """Grand capacitance tensor C = Sigma' M^{-1} Sigma'^T (Sec. III.B, Eq. QS_capacitance):
    [Q; S] = C [Psi - Psi_0; E0], with the 3 N_b field rows and columns body-major
    (the field E0 of each body's own bead rows).  M^{-1} Sigma'^T by dense LU."""
    x = _c(x).reshape(-1, 3)
    if M is None:
        M = M_dense(x, box, a, eps, xi=xi)
    Sp = sigma_prime(x, X, body_offsets, box)
    return Sp @ np.linalg.solve(M, Sp.T)


# ---------------------------------------------------------------------------
# Derived quantities: Eq. rigid_dipole, Eq. pot_syst, Eq. beadforce, Sec. III.C
# ---------------------------------------------------------------------------

def dipoles(x, X, body_offsets, q, box):
    """S_i = sum_j r_ij q_ij (Eq. rigid_dipole)."""
    r = relative_positions(x, X, body_offsets, box)
    off = np.asarray(body_offsets, dtype=np.int64)
    nb = len(off) - 1
    S = np.zeros((nb, 3))
    for i in range(nb):
        S[i] = (r[off[i]:off[i + 1]] * np.asarray(q)[off[i]:off[i + 1], None]).sum(axis=0)
    return S


def energy(X, Q, psi_rel, S, E0):
    """U = 1/2 sum_i (Q_i Psi_i - S_i . E0) (Eq. pot_syst), Psi_i = (Psi_i - Psi_0,i) + Psi_0,i,
    with the external potential Psi_0,i = -X_i . E0 (Sec. III.B)."""
    E0 = np.asarray(E0, dtype=np.float64)
    Psi = np.asarray(psi_rel) - np.asarray(X) @ E0
    return 0.5 * float(np.dot(Q, Psi) - np.sum(np.asarray(S) @ E0))


def bead_forces(x, q, E0, box, a, eps, xi=None):
    """f_alpha = q_alpha E0 - 1/2 (grad_alpha M):qq = q_alpha (E0 + E_alpha) (Eq. beadforce),
    where E_alpha = -sum_{beta != alpha} grad_alpha M_{alpha beta} q_beta is the Ewald field
    at alpha of all other charges (the self term of M does not depend on x_alpha)."""
    _, E = potential(x, q, box, a, eps, field=True, xi=xi)
    return np.asarray(q)[:, None] * (np.asarray(E0, dtype=np.float64)[None, :] + E)


def body_force_torque(x, X, body_offsets, f, box):
    """F_i = sum_j f_ij, L_i = sum_j r_ij x f_ij (Sec. III.C)."""
    r = relative_positions(x, X, body_offsets, box)
    off = np.asarray(body_offsets, dtype=np.int64)
    nb = len(off) - 1
    F = np.zeros((nb, 3))
    L = np.zeros((nb, 3))
    for i in range(nb):
        s = slice(off[i], off[i + 1])
        F[i] = f[s].sum(axis=0)
        L[i] = np.cross(r[s], f[s]).sum(axis=0)
    return F, L


# ---------------------------------------------------------------------------
# Parameter rules of Sec. III.D.2 (what the library's automatic setup must give)
# ---------------------------------------------------------------------------

def auto_params(box, mesh, tol, a):
    """Spectral-Ewald parameters for a given mesh and accuracy (Sec. III.D.2).

    k_c from N_g = 1 + L k_c / pi (smallest box axis); xi from the wave-space
    bound e^{-k_c^2/4xi^2} = tol; r_c from the real-space bound e^{-(r_c-2a)^2 xi^2} = tol
    (the kernel decays from the bead surface, 2a); P from e^{-pi P/2} <= tol;
    h = L / N_g; eta = h^2 xi^2 P / pi (largest axis spacing).
    """
    box = np.asarray(box, dtype=np.float64)
    mesh = np.asarray(mesh, dtype=np.int64)
    lnt = math.log(1.0 / tol)
    kc = min(math.pi * (mesh[d] - 1) / box[d] for d in range(3))
    xi = kc / (2.0 * math.sqrt(lnt))
    rc = math.sqrt(lnt) / xi + 2.0 * a
    P = int(math.ceil(2.0 * lnt / math.pi))
    h = max(box[d] / mesh[d] for d in range(3))
    eta = h * h * xi * xi * P / math.pi
    return dict(xi=xi, r_cut=rc, P=P, eta=eta, h=h, k_c=kc)


# ---------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC'11) and Box-Muller.
# ---------------------------------------------------------------------------

_PH_M0, _PH_M1 = 0xD2511F53, 0xCD9E8D57
_PH_W0, _PH_W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Ten Philox rounds on a 4x32-bit counter with a 2x32-bit key."""
    c0, c1, c2, c3 = (int(v) & _MASK for v in ctr)
    k0, k1 = (int(v) & _MASK for v in key)
    for r in range(10):
        p0 = _PH_M0 * c0
        p1 = _PH_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        if r < 9:
            k0 = (k0 + _PH_W0) & _MASK
            k1 = (k1 + _PH_W1) & _MASK
    return c0, c1, c2, c3


def normals(entity: int, step: int, seed: int, count: int = 6):
    """Standard normals for one body or ion at one step.

    Normal pair t (t = 0, 1, 2) comes from Philox on counter
    (entity, step, t, 0x1B5EED) and key (seed lo, seed hi): the first two words
    give u1, u2 = (w + 0.5) 2^-32 and Box-Muller gives
    sqrt(-2 ln u1) cos(2 pi u2), sqrt(-2 ln u1) sin(2 pi u2).
    """
    out = []
    key = (seed & _MASK, (seed >> 32) & _MASK)
    for t in range((count + 1) // 2):
        w = philox4x32_10((entity, step, t, 0x1B5EED), key)
        u1 = (w[0] + 0.5) * 2.0 ** -32
        u2 = (w[1] + 0.5) * 2.0 ** -32
        rad = math.sqrt(-2.0 * math.log(u1))
        out.append(rad * math.cos(2.0 * math.pi * u2))
        out.append(rad * math.sin(2.0 * math.pi * u2))
    return out[:count]


# ---------------------------------------------------------------------------
# Brownian dynamics step, Sec. V.A (free-draining, Heyes-Melrose hard spheres)
# ---------------------------------------------------------------------------

def hard_sphere_forces(x, body_offsets, box, a, gamma, dt):
    """Pair forces of U^hs = gamma/(4 dt) (r - 2a)^2 for r < 2a (Eq. hardsphereFD),
    between beads of different bodies (beads of one rigid body do not repel).
    With one radius per bead the contact distance 2a of a pair is a_alpha + a_beta."""
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    rad = np.full(n, float(a)) if np.ndim(a) == 0 else _c(a).reshape(-1)
    bid = body_index(body_offsets)
    f = np.zeros((n, 3))
    for al in range(n):
        d = min_image(x[al] - x, box)
        r = np.sqrt((d * d).sum(axis=1))
        contact = rad[al] + rad
        mask = (r < contact) & (bid != bid[al]) & (r > 0)
        # -dU/dr along (x_al - x_be)/r, with dU/dr = gamma/(2 dt) (r - contact)
        mag = gamma / (2.0 * dt) * (contact[mask] - r[mask])
        f[al] = (mag[:, None] * d[mask] / r[mask][:, None]).sum(axis=0)
    return f


def _rotation(theta):
    """Rotation matrix of the rotation vector theta (Rodrigues' formula)."""
    ang = float(np.linalg.norm(theta))
    if ang == 0.0:
        return np.eye(3)
    k = theta / ang
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * Kx + (1.0 - math.cos(ang)) * (Kx @ Kx)


def bd_step(x, X, body_offsets, f_bead, box, a, dt, gamma=1.0, kT=1.0, seed=0, step=0):
    """One Euler-Maruyama step (Eq. forward) of the overdamped Langevin equation
    with free-draining mobility M^H = I/gamma (Sec. V.A).

    Single-bead bodies (ions): dx = (F/gamma) dt + sqrt(2 kT dt/gamma) n.
    Rigid bodies of N_i beads: the constrained free-draining mobility gives
    U = F_i/(N_i gamma) and Omega = (gamma J_i)^{-1} L_i with
    J_i = sum_j (|r_ij|^2 I - r_ij r_ij^T); the Brownian displacement has
    covariance 2 kT dt times the same mobilities (Cholesky factor for the
    rotation); beads move rigidly: r_ij <- R(theta) r_ij with
    theta = Omega dt + noise, X_i <- X_i + U dt + noise, x_ij = X_i + r_ij.
    ``f_bead`` is the total bead force (electrostatic + hard sphere).
    Returns new bead positions and new body reference points.
    """
    x = _c(x).reshape(-1, 3)
    X = _c(X).reshape(-1, 3)
    off = np.asarray(body_offsets, dtype=np.int64)
    r = relative_positions(x, X, off, box)
    F, L = body_force_torque(x, X, off, f_bead, box)
    xn = x.copy()
    Xn = X.copy()
    for i in range(len(off) - 1):
        s = slice(off[i], off[i + 1])
        Ni = off[i + 1] - off[i]
        nrm = np.array(normals(i, step, seed, 6))
        dX = F[i] / (Ni * gamma) * dt + math.sqrt(2.0 * kT * dt / (Ni * gamma)) * nrm[:3]
        Xn[i] = X[i] + dX
        if Ni == 1:
            xn[s] = Xn[i] + r[s]
            continue
        J = np.zeros((3, 3))
        for rj in r[s]:
            J += np.dot(rj, rj) * np.eye(3) - np.outer(rj, rj)
        Mrot = np.linalg.inv(gamma * J)
        Om = Mrot @ L[i]
        Lc = np.linalg.cholesky(Mrot)
        theta = Om * dt + math.sqrt(2.0 * kT * dt) * (Lc @ nrm[3:])
        R = _rotation(theta)
        xn[s] = Xn[i] + r[s] @ R.T
    return xn, Xn


# ---------------------------------------------------------------------------
# Convenience: full per-configuration reference results
# ---------------------------------------------------------------------------

def reference_solution(x, body_offsets, X, Q, E0, box, a, eps, dense=None, xi=None):
    """q, Psi - Psi_0, S, U, bead forces, body F and L for one right-hand side."""
    x = _c(x).reshape(-1, 3)
    n = x.shape[0]
    if dense is None:
        dense = n <= 3000
    if dense:
        q, psi = solve_dense(x, body_offsets, X, Q, E0, box, a, eps, xi=xi)
    else:
        q, psi, _, _ = solve_gmres(x, body_offsets, X, Q, E0, box, a, eps, xi=xi)
    S = dipoles(x, X, body_offsets, q, box)
    U = energy(X, Q, psi, S, E0)
    f = bead_forces(x, q, E0, box, a, eps, xi=xi)
    F, L = body_force_torque(x, X, body_offsets, f, box)
    return dict(q=q, psi=psi, S=S, U=U, f=f, F=F, L=L)


__all__ = [
    "lib", "num_threads", "k0_term", "M_free", "phi_real", "dphi_real", "phi_self", "M_free2", "phi_real2", "dphi_real2", "ewald_split",
    "potential", "wave_vectors", "M_dense", "spread_grid", "min_image", "body_index", "sigma_matrix",
    "relative_positions", "saddle_rhs", "saddle_matrix", "solve_dense", "gmres", "sigma_prime",
    "grand_capacitance",
    "saddle_operator", "solve_gmres", "dipoles", "energy", "bead_forces",
    "body_force_torque", "auto_params", "philox4x32_10", "normals",
    "hard_sphere_forces", "bd_step", "reference_solution",
]
