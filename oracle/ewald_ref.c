/*
 * ewald_ref.c -- plain FP64 reference (oracle) for the regularized Ewald sums of
 * Krucker-Velasquez, Swan & Sherman, "Immersed boundary method for dynamic
 * simulation of polarizable colloids of arbitrary shape in explicit ion
 * electrolytes" (arXiv:2401.04865).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle that checks the
 * CUDA library.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code with the CUDA path and it
 * is deliberately slow: every sum is written out as the paper defines it.
 *
 *   - real-space sum: direct loop over every source bead and every periodic
 *     image shell within the cutoff (Sec. III.D.1, Eq. psi_Re_1), no cell list;
 *   - self term: Sec. III.D.1, the r -> 0 limit printed after Eq. psi_Re_1;
 *   - wave-space sum: explicit loop over every wave vector k != 0 with
 *     |k| <= k_c of the structure factor (Sec. III.D, Eq. splitting, first
 *     term), no grid, no FFT, no Gaussian spreading;
 *   - the free-space regularized tensor M(r) (Sec. II, real-space form of
 *     Eq. M00_Fourier);
 *   - the same sums for beads of unequal radii (the *2 and *_radii functions
 *     at the end), kernel j0(k a_alpha) j0(k a_beta)/k^2.
 *
 * Conventions: x is [n][3] row-major, q is [n], the box is orthorhombic with
 * side lengths L[3] and volume V = L0*L1*L2, eps is the fluid permittivity
 * eps_f.  All potentials are psi_alpha - psi_0(x_alpha) (Eq. pot_charge), all
 * fields are E = -grad psi.
 *
 * Reading of the paper used here (the printed Eq. psi_Re_1 is ambiguous in
 * sign): the Heaviside term is (-1/(4 pi r) + (4a - r)/(16 pi a^2)) H(2a - r).
 * With this sign the xi -> 0 limit reproduces the real-space M(r) of Sec. II
 * and the r -> 0 limit reproduces the printed self term; the test-suite pins
 * both limits and an independent quadrature of the inverse transform.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846264338327950288;

int ibo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Real-space form of the regularized potential tensor (Sec. II), without the
 * 1/eps factor: 1/(4 pi r) for r >= 2a, (4a - r)/(16 pi a^2) for r < 2a.
 * (The printed 1/(4 pi a eps r) carries a stray factor a; the form here is the
 * one that is continuous at r = 2a and is the inverse transform of
 * j0^2(ka)/k^2.) */
double ibo_M_free(double r, double a)
{
    if (r >= 2.0 * a)
        return 1.0 / (4.0 * PI * r);
    return (4.0 * a - r) / (16.0 * PI * a * a);
}

/* Self term (Sec. III.D.1, equation after psi_Re_1), without the 1/eps. */
double ibo_phi_self(double a, double xi)
{
    return (1.0 - exp(-4.0 * a * a * xi * xi)) / (8.0 * pow(PI, 1.5) * a * a * xi)
         + erfc(2.0 * a * xi) / (4.0 * PI * a);
}

/* Real-space pair kernel, Eq. psi_Re_1 written term by term (without 1/eps).
 * r > 0 is the pair distance, a the bead radius, xi the Ewald parameter. */
double ibo_phi_real(double r, double a, double xi)
{
    const double rp = r + 2.0 * a;     /* r_{alpha beta} + 2a */
    const double rm = r - 2.0 * a;     /* r_{alpha beta} - 2a */
    const double x2 = xi * xi;
    const double c_exp = 32.0 * pow(PI, 1.5) * a * a * xi;   /* 32 pi^{3/2} a^2 xi */
    double t = 0.0;
    t += -rp / (c_exp * r) * exp(-rp * rp * x2);
    t += -rm / (c_exp * r) * exp(-rm * rm * x2);
    t += 1.0 / (16.0 * pow(PI, 1.5) * a * a * xi) * exp(-r * r * x2);
    t += (2.0 * x2 * rp * rp + 1.0) / (64.0 * PI * a * a * x2 * r) * erfc(rp * xi);
    t += (2.0 * x2 * rm * rm + 1.0) / (64.0 * PI * a * a * x2 * r) * erfc(rm * xi);
    t += -(2.0 * x2 * r * r + 1.0) / (32.0 * PI * a * a * x2 * r) * erfc(r * xi);
    if (r < 2.0 * a)
        t += -1.0 / (4.0 * PI * r) + (4.0 * a - r) / (16.0 * PI * a * a);
    return t;
}

/* d/dr of ibo_phi_real, each printed term differentiated separately. */
double ibo_dphi_real(double r, double a, double xi)
{
    const double rp = r + 2.0 * a;
    const double rm = r - 2.0 * a;
    const double x2 = xi * xi;
    const double A = 1.0 / (32.0 * pow(PI, 1.5) * a * a * xi);
    const double B = 1.0 / (64.0 * PI * a * a * x2);
    const double two_over_sqrtpi = 2.0 / sqrt(PI);
    const double ep = exp(-rp * rp * x2), em = exp(-rm * rm * x2), e0 = exp(-r * r * x2);
    double d = 0.0;
    /* -A (u/r) e^{-u^2 xi^2} for u = r + 2a and u = r - 2a */
    d += -A * ep * (1.0 / r - rp / (r * r) - 2.0 * rp * rp * x2 / r);
    d += -A * em * (1.0 / r - rm / (r * r) - 2.0 * rm * rm * x2 / r);
    /* 2A e^{-r^2 xi^2} */
    d += -4.0 * A * x2 * r * e0;
    /* B (2 xi^2 u^2 + 1)/r erfc(u xi) for u = r + 2a and u = r - 2a */
    d += B * ((4.0 * x2 * rp / r - (2.0 * x2 * rp * rp + 1.0) / (r * r)) * erfc(rp * xi)
              - (2.0 * x2 * rp * rp + 1.0) / r * two_over_sqrtpi * xi * ep);
    d += B * ((4.0 * x2 * rm / r - (2.0 * x2 * rm * rm + 1.0) / (r * r)) * erfc(rm * xi)
              - (2.0 * x2 * rm * rm + 1.0) / r * two_over_sqrtpi * xi * em);
    /* -2B (2 xi^2 r^2 + 1)/r erfc(r xi) */
    d += -2.0 * B * ((4.0 * x2 - (2.0 * x2 * r * r + 1.0) / (r * r)) * erfc(r * xi)
                     - (2.0 * x2 * r * r + 1.0) / r * two_over_sqrtpi * xi * e0);
    /* Heaviside term */
    if (r < 2.0 * a)
        d += 1.0 / (4.0 * PI * r * r) - 1.0 / (16.0 * PI * a * a);
    return d;
}

/* Number of periodic images needed along one axis so that every image of a
 * displacement already reduced to [-L/2, L/2] within the cutoff is visited. */
static int image_range(double rc, double L)
{
    return (int)ceil((rc + 0.5 * L) / L);
}

/*
 * Real-space sum at the targets (Sec. III.D.1): for each target alpha,
 *   psi_alpha += (1/eps) sum_{beta, n} phi_r(|x_alpha - x_beta + n L|) q_beta
 * over all periodic images n with distance < rc, skipping beta == alpha at
 * n = 0, plus (1/eps) phi_self q_alpha.  If E != NULL the field
 *   E_alpha += (1/eps) sum -phi_r'(r) (x_alpha - x_beta + n L)/r q_beta
 * is accumulated as well.  Results are OVERWRITTEN (not accumulated).
 * A coincident pair (r == 0, beta != alpha) takes the r -> 0 limit, which is
 * the self value, and contributes no field.
 */
void ibo_real_sum(int n, const double *x, const double *q, const double *L,
                  double a, double xi, double rc, double eps,
                  int nt, const int *targets, double *psi, double *E)
{
    const int m0 = image_range(rc, L[0]), m1 = image_range(rc, L[1]), m2 = image_range(rc, L[2]);
    const double self = ibo_phi_self(a, xi);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nt; ++t) {
        const int al = targets[t];
        double p = self * q[al];
        double ex = 0.0, ey = 0.0, ez = 0.0;
        for (int be = 0; be < n; ++be) {
            double dx0 = x[3 * al + 0] - x[3 * be + 0];
            double dy0 = x[3 * al + 1] - x[3 * be + 1];
            double dz0 = x[3 * al + 2] - x[3 * be + 2];
            /* bring the displacement to the primary cell first */
            dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
            dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
            dz0 -= L[2] * floor(dz0 / L[2] + 0.5);
            for (int i = -m0; i <= m0; ++i)
                for (int j = -m1; j <= m1; ++j)
                    for (int k = -m2; k <= m2; ++k) {
                        if (be == al && i == 0 && j == 0 && k == 0)
                            continue;
                        const double dx = dx0 + i * L[0], dy = dy0 + j * L[1], dz = dz0 + k * L[2];
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= rc)
                            continue;
                        if (r == 0.0) {
                            p += self * q[be];
                            continue;
                        }
                        p += ibo_phi_real(r, a, xi) * q[be];
                        if (E) {
                            const double f = -ibo_dphi_real(r, a, xi) / r * q[be];
                            ex += f * dx; ey += f * dy; ez += f * dz;
                        }
                    }
        }
        psi[t] = p / eps;
        if (E) {
            E[3 * t + 0] = ex / eps;
            E[3 * t + 1] = ey / eps;
            E[3 * t + 2] = ez / eps;
        }
    }
}

/*
 * Wave-space sum at the targets (Sec. III.D, first term of Eq. splitting):
 *   psi_alpha = 1/(eps V) sum_{k != 0, |k| <= kc} j0^2(k a) e^{-k^2/(4 xi^2)}/k^2
 *               * Re( e^{i k.x_alpha} conj(S(k)) ),   S(k) = sum_beta q_beta e^{i k.x_beta}
 *   E_alpha   = 1/(eps V) sum_k G(k) k Im( e^{i k.x_alpha} conj(S(k)) )
 * with k = 2 pi (m0/L0, m1/L1, m2/L2) for integer m.  Each term is evaluated
 * directly; e^{i k.x} is formed as the product of the three axis factors
 * e^{i k_d x_d}, each taken from sin/cos of its own argument.
 * Results are OVERWRITTEN.
 */
void ibo_wave_sum(int n, const double *x, const double *q, const double *L,
                  double a, double xi, double kc, double eps,
                  int nt, const int *targets, double *psi, double *E)
{
    const int mx = (int)floor(kc * L[0] / (2.0 * PI));
    const int my = (int)floor(kc * L[1] / (2.0 * PI));
    const int mz = (int)floor(kc * L[2] / (2.0 * PI));
    const int wx = 2 * mx + 1, wy = 2 * my + 1, wz = 2 * mz + 1;
    const double V = L[0] * L[1] * L[2];

    /* per-bead axis phase factors: ph[b][d][m] = e^{i 2 pi m x_d / L_d}, m in [-M, M] */
    const int nall = n;
    double *cx = malloc(sizeof(double) * (size_t)nall * wx), *sx = malloc(sizeof(double) * (size_t)nall * wx);
    double *cy = malloc(sizeof(double) * (size_t)nall * wy), *sy = malloc(sizeof(double) * (size_t)nall * wy);
    double *cz = malloc(sizeof(double) * (size_t)nall * wz), *sz = malloc(sizeof(double) * (size_t)nall * wz);
#pragma omp parallel for
    for (int b = 0; b < nall; ++b) {
        for (int m = -mx; m <= mx; ++m) {
            const double th = 2.0 * PI * m * x[3 * b + 0] / L[0];
            cx[(size_t)b * wx + m + mx] = cos(th); sx[(size_t)b * wx + m + mx] = sin(th);
        }
        for (int m = -my; m <= my; ++m) {
            const double th = 2.0 * PI * m * x[3 * b + 1] / L[1];
            cy[(size_t)b * wy + m + my] = cos(th); sy[(size_t)b * wy + m + my] = sin(th);
        }
        for (int m = -mz; m <= mz; ++m) {
            const double th = 2.0 * PI * m * x[3 * b + 2] / L[2];
            cz[(size_t)b * wz + m + mz] = cos(th); sz[(size_t)b * wz + m + mz] = sin(th);
        }
    }

    /* list of wave vectors with 0 < |k| <= kc */
    size_t nk_max = (size_t)wx * wy * wz;
    int *km = malloc(sizeof(int) * 3 * nk_max);
    size_t nk = 0;
    for (int i = -mx; i <= mx; ++i)
        for (int j = -my; j <= my; ++j)
            for (int k = -mz; k <= mz; ++k) {
                if (i == 0 && j == 0 && k == 0)
                    continue;
                const double kx = 2.0 * PI * i / L[0], ky = 2.0 * PI * j / L[1], kz = 2.0 * PI * k / L[2];
                if (kx * kx + ky * ky + kz * kz > kc * kc)
                    continue;
                km[3 * nk + 0] = i; km[3 * nk + 1] = j; km[3 * nk + 2] = k;
                ++nk;
            }

    /* structure factor S(k) = sum_beta q_beta e^{i k.x_beta} and the weight G(k) */
    double *Sre = malloc(sizeof(double) * (nk ? nk : 1)), *Sim = malloc(sizeof(double) * (nk ? nk : 1));
    double *G = malloc(sizeof(double) * (nk ? nk : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (size_t t = 0; t < nk; ++t) {
        const int i = km[3 * t], j = km[3 * t + 1], k = km[3 * t + 2];
        const double kx = 2.0 * PI * i / L[0], ky = 2.0 * PI * j / L[1], kz = 2.0 * PI * k / L[2];
        const double kk = sqrt(kx * kx + ky * ky + kz * kz);
        const double j0 = sin(kk * a) / (kk * a);
        G[t] = j0 * j0 * exp(-kk * kk / (4.0 * xi * xi)) / (kk * kk);
        double sre = 0.0, sim = 0.0;
        for (int b = 0; b < n; ++b) {
            /* e^{i(kx x + ky y + kz z)} = product of the three axis factors */
            const double ax = cx[(size_t)b * wx + i + mx], bx = sx[(size_t)b * wx + i + mx];
            const double ay = cy[(size_t)b * wy + j + my], by = sy[(size_t)b * wy + j + my];
            const double az = cz[(size_t)b * wz + k + mz], bz = sz[(size_t)b * wz + k + mz];
            const double pre = ax * ay - bx * by, pim = ax * by + bx * ay;
            const double re = pre * az - pim * bz, im = pre * bz + pim * az;
            sre += q[b] * re;
            sim += q[b] * im;
        }
        Sre[t] = sre;
        Sim[t] = sim;
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int tt = 0; tt < nt; ++tt) {
        const int al = targets[tt];
        double p = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (size_t t = 0; t < nk; ++t) {
            const int i = km[3 * t], j = km[3 * t + 1], k = km[3 * t + 2];
            const double ax = cx[(size_t)al * wx + i + mx], bx = sx[(size_t)al * wx + i + mx];
            const double ay = cy[(size_t)al * wy + j + my], by = sy[(size_t)al * wy + j + my];
            const double az = cz[(size_t)al * wz + k + mz], bz = sz[(size_t)al * wz + k + mz];
            const double pre = ax * ay - bx * by, pim = ax * by + bx * ay;
            const double re = pre * az - pim * bz, im = pre * bz + pim * az;
            /* e^{i k.x_alpha} * conj(S) */
            const double zre = re * Sre[t] + im * Sim[t];
            const double zim = im * Sre[t] - re * Sim[t];
            p += G[t] * zre;
            if (E) {
                const double kx = 2.0 * PI * i / L[0], ky = 2.0 * PI * j / L[1], kz = 2.0 * PI * k / L[2];
                ex += G[t] * kx * zim;
                ey += G[t] * ky * zim;
                ez += G[t] * kz * zim;
            }
        }
        psi[tt] = p / (eps * V);
        if (E) {
            E[3 * tt + 0] = ex / (eps * V);
            E[3 * tt + 1] = ey / (eps * V);
            E[3 * tt + 2] = ez / (eps * V);
        }
    }
    free(cx); free(sx); free(cy); free(sy); free(cz); free(sz);
    free(km); free(Sre); free(Sim); free(G);
}

/* Wave vectors of the explicit sum, for callers that assemble the dense
 * wave-space matrix themselves: writes up to cap rows of (kx, ky, kz, G(k))
 * for k != 0, |k| <= kc, and returns the total count. */
long ibo_wave_vectors(const double *L, double a, double xi, double kc, long cap, double *out)
{
    const int mx = (int)floor(kc * L[0] / (2.0 * PI));
    const int my = (int)floor(kc * L[1] / (2.0 * PI));
    const int mz = (int)floor(kc * L[2] / (2.0 * PI));
    long nk = 0;
    for (int i = -mx; i <= mx; ++i)
        for (int j = -my; j <= my; ++j)
            for (int k = -mz; k <= mz; ++k) {
                if (i == 0 && j == 0 && k == 0)
                    continue;
                const double kx = 2.0 * PI * i / L[0], ky = 2.0 * PI * j / L[1], kz = 2.0 * PI * k / L[2];
                const double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kc * kc)
                    continue;
                if (nk < cap) {
                    const double kk = sqrt(k2);
                    const double j0 = sin(kk * a) / (kk * a);
                    out[4 * nk + 0] = kx; out[4 * nk + 1] = ky; out[4 * nk + 2] = kz;
                    out[4 * nk + 3] = j0 * j0 * exp(-k2 / (4.0 * xi * xi)) / k2;
                }
                ++nk;
            }
    return nk;
}

/*
 * Dense real-space part of M (Sec. III.D.1), including the self term on the
 * diagonal, without 1/eps: Mr[alpha][beta] = sum_n phi_r(|x_ab + nL|) over the
 * images within rc (n = 0 skipped on the diagonal) + delta_ab phi_self.
 */
void ibo_real_matrix(int n, const double *x, const double *L, double a, double xi, double rc, double *Mr)
{
    const int m0 = image_range(rc, L[0]), m1 = image_range(rc, L[1]), m2 = image_range(rc, L[2]);
    const double self = ibo_phi_self(a, xi);
#pragma omp parallel for schedule(dynamic, 4)
    for (int al = 0; al < n; ++al) {
        for (int be = 0; be < n; ++be) {
            double dx0 = x[3 * al + 0] - x[3 * be + 0];
            double dy0 = x[3 * al + 1] - x[3 * be + 1];
            double dz0 = x[3 * al + 2] - x[3 * be + 2];
            dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
            dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
            dz0 -= L[2] * floor(dz0 / L[2] + 0.5);
            double m = (al == be) ? self : 0.0;
            for (int i = -m0; i <= m0; ++i)
                for (int j = -m1; j <= m1; ++j)
                    for (int k = -m2; k <= m2; ++k) {
                        if (al == be && i == 0 && j == 0 && k == 0)
                            continue;
                        const double dx = dx0 + i * L[0], dy = dy0 + j * L[1], dz = dz0 + k * L[2];
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= rc)
                            continue;
                        m += (r == 0.0) ? self : ibo_phi_real(r, a, xi);
                    }
            Mr[(size_t)al * n + be] = m;
        }
    }
}

/* ------------------------------------------------------------------------
 * Beads of unequal radii.
 *
 * A bead of radius a carries its charge on a spherical shell of radius a;
 * the shell's Fourier transform is j0(ka), which is where the j0^2(ka) of
 * Eq. M00_Fourier comes from.  Two beads of radii a and b therefore interact
 * through j0(ka) j0(kb)/k^2 (the paper fixes one radius, Sec. III.A; this is
 * the same construction with two).  In real space the pair kernel is the
 * average of the point kernel over both shells.  For a radial kernel f with
 * s f(|s|) extended to an odd function of s and F any C^1 function with
 * F'' = s f(|s|), the average over shells of radii a and b with centres r
 * apart is
 *     [F(r+a+b) - F(r+a-b) - F(r-a+b) + F(r-a-b)] / (4 a b r),
 * because the distance from a fixed point to a uniform point of a shell of
 * radius b is distributed with density s/(2 b r) on [|r-b|, r+b].
 * ------------------------------------------------------------------------ */

/* F for the unscreened kernel 1/(4 pi s): F'' = sign(s)/(4 pi). */
static double F_coulomb(double s)
{
    return s * fabs(s) / (8.0 * PI);
}

/* F for the screened kernel erfc(xi s)/(4 pi s) (the real-space share of
 * Eq. splitting): F(s) = sign(s) f(|s|)/(4 pi) with
 * f(u) = (u^2/2 + 1/(4 xi^2)) erfc(xi u) - u e^{-xi^2 u^2}/(2 xi sqrt(pi)) - 1/(4 xi^2),
 * f(0) = 0, f'' = erfc(xi u). */
static double F_screened(double s, double xi)
{
    const double u = fabs(s);
    const double f = (0.5 * u * u + 0.25 / (xi * xi)) * erfc(xi * u)
                   - u * exp(-xi * xi * u * u) / (2.0 * xi * sqrt(PI)) - 0.25 / (xi * xi);
    return (s < 0.0 ? -f : f) / (4.0 * PI);
}

/* F' of the screened kernel (even in s): (u erfc(xi u) - e^{-xi^2 u^2}/(xi sqrt(pi)))/(4 pi). */
static double dF_screened(double s, double xi)
{
    const double u = fabs(s);
    return (u * erfc(xi * u) - exp(-xi * xi * u * u) / (xi * sqrt(PI))) / (4.0 * PI);
}

/* F' of the unscreened kernel: |s|/(4 pi). */
static double dF_coulomb(double s)
{
    return fabs(s) / (4.0 * PI);
}

/* Free-space shell-shell potential W(r; a, b) without 1/eps: the real-space
 * form of j0(ka) j0(kb)/k^2.  Equals M(r) above for a = b. */
double ibo_M_free2(double r, double a, double b)
{
    if (r == 0.0)   /* r -> 0 limit: [F'(a+b) - F'(|a-b|)] / (2ab) */
        return (dF_coulomb(a + b) - dF_coulomb(a - b)) / (2.0 * a * b);
    return (F_coulomb(r + a + b) - F_coulomb(r + a - b) - F_coulomb(r - a + b) + F_coulomb(r - a - b))
           / (4.0 * a * b * r);
}

/* Real-space Ewald kernel of a pair of radii a and b, without 1/eps: the
 * inverse transform of j0(ka) j0(kb)(1 - e^{-k^2/(4 xi^2)})/k^2.  At r = 0 it
 * takes the limit [F'(a+b) - F'(|a-b|)]/(2ab), which for a = b is the self
 * term of Sec. III.D.1. */
double ibo_phi_real2(double r, double a, double b, double xi)
{
    if (r == 0.0)
        return (dF_screened(a + b, xi) - dF_screened(a - b, xi)) / (2.0 * a * b);
    return (F_screened(r + a + b, xi) - F_screened(r + a - b, xi) - F_screened(r - a + b, xi)
            + F_screened(r - a - b, xi)) / (4.0 * a * b * r);
}

/* d/dr of ibo_phi_real2 for r > 0: N'(r)/(4abr) - phi/r with N the bracket. */
double ibo_dphi_real2(double r, double a, double b, double xi)
{
    const double dN = dF_screened(r + a + b, xi) - dF_screened(r + a - b, xi) - dF_screened(r - a + b, xi)
                    + dF_screened(r - a - b, xi);
    return dN / (4.0 * a * b * r) - ibo_phi_real2(r, a, b, xi) / r;
}

/* ibo_real_sum with a radius per bead (rad[n]): each pair takes
 * ibo_phi_real2 of its two radii, each target its own self term. */
void ibo_real_sum_radii(int n, const double *x, const double *q, const double *L,
                        const double *rad, double xi, double rc, double eps,
                        int nt, const int *targets, double *psi, double *E)
{
    const int m0 = image_range(rc, L[0]), m1 = image_range(rc, L[1]), m2 = image_range(rc, L[2]);
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nt; ++t) {
        const int al = targets[t];
        const double a = rad[al];
        double p = ibo_phi_real2(0.0, a, a, xi) * q[al];
        double ex = 0.0, ey = 0.0, ez = 0.0;
        for (int be = 0; be < n; ++be) {
            const double b = rad[be];
            double dx0 = x[3 * al + 0] - x[3 * be + 0];
            double dy0 = x[3 * al + 1] - x[3 * be + 1];
            double dz0 = x[3 * al + 2] - x[3 * be + 2];
            dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
            dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
            dz0 -= L[2] * floor(dz0 / L[2] + 0.5);
            for (int i = -m0; i <= m0; ++i)
                for (int j = -m1; j <= m1; ++j)
                    for (int k = -m2; k <= m2; ++k) {
                        if (be == al && i == 0 && j == 0 && k == 0)
                            continue;
                        const double dx = dx0 + i * L[0], dy = dy0 + j * L[1], dz = dz0 + k * L[2];
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= rc)
                            continue;
                        p += ibo_phi_real2(r, a, b, xi) * q[be];
                        if (E && r > 0.0) {
                            const double f = -ibo_dphi_real2(r, a, b, xi) / r * q[be];
                            ex += f * dx; ey += f * dy; ez += f * dz;
                        }
                    }
        }
        psi[t] = p / eps;
        if (E) {
            E[3 * t + 0] = ex / eps;
            E[3 * t + 1] = ey / eps;
            E[3 * t + 2] = ez / eps;
        }
    }
}

/* ibo_wave_sum with a radius per bead: the structure factor weighs each
 * source by j0(k a_beta), each target's sum by j0(k a_alpha), and the weight
 * is e^{-k^2/(4 xi^2)}/k^2 (no j0 in it).  Results are OVERWRITTEN. */
void ibo_wave_sum_radii(int n, const double *x, const double *q, const double *L,
                        const double *rad, double xi, double kc, double eps,
                        int nt, const int *targets, double *psi, double *E)
{
    const int mx = (int)floor(kc * L[0] / (2.0 * PI));
    const int my = (int)floor(kc * L[1] / (2.0 * PI));
    const int mz = (int)floor(kc * L[2] / (2.0 * PI));
    const double V = L[0] * L[1] * L[2];
    size_t nk = 0;
    int *km = malloc(sizeof(int) * 3 * (size_t)(2 * mx + 1) * (2 * my + 1) * (2 * mz + 1));
    for (int i = -mx; i <= mx; ++i)
        for (int j = -my; j <= my; ++j)
            for (int k = -mz; k <= mz; ++k) {
                if (i == 0 && j == 0 && k == 0)
                    continue;
                const double kx = 2.0 * PI * i / L[0], ky = 2.0 * PI * j / L[1], kz = 2.0 * PI * k / L[2];
                if (kx * kx + ky * ky + kz * kz > kc * kc)
                    continue;
                km[3 * nk + 0] = i; km[3 * nk + 1] = j; km[3 * nk + 2] = k;
                ++nk;
            }
    double *Sre = malloc(sizeof(double) * (nk ? nk : 1)), *Sim = malloc(sizeof(double) * (nk ? nk : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (size_t t = 0; t < nk; ++t) {
        const double kx = 2.0 * PI * km[3 * t] / L[0], ky = 2.0 * PI * km[3 * t + 1] / L[1],
                     kz = 2.0 * PI * km[3 * t + 2] / L[2];
        const double kk = sqrt(kx * kx + ky * ky + kz * kz);
        double sre = 0.0, sim = 0.0;
        for (int b = 0; b < n; ++b) {
            const double th = kx * x[3 * b] + ky * x[3 * b + 1] + kz * x[3 * b + 2];
            const double w = q[b] * sin(kk * rad[b]) / (kk * rad[b]);
            sre += w * cos(th);
            sim += w * sin(th);
        }
        Sre[t] = sre;
        Sim[t] = sim;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int tt = 0; tt < nt; ++tt) {
        const int al = targets[tt];
        double p = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (size_t t = 0; t < nk; ++t) {
            const double kx = 2.0 * PI * km[3 * t] / L[0], ky = 2.0 * PI * km[3 * t + 1] / L[1],
                         kz = 2.0 * PI * km[3 * t + 2] / L[2];
            const double k2 = kx * kx + ky * ky + kz * kz, kk = sqrt(k2);
            const double G = sin(kk * rad[al]) / (kk * rad[al]) * exp(-k2 / (4.0 * xi * xi)) / k2;
            const double th = kx * x[3 * al] + ky * x[3 * al + 1] + kz * x[3 * al + 2];
            const double re = cos(th), im = sin(th);
            p += G * (re * Sre[t] + im * Sim[t]);
            if (E) {
                const double zim = im * Sre[t] - re * Sim[t];
                ex += G * kx * zim;
                ey += G * ky * zim;
                ez += G * kz * zim;
            }
        }
        psi[tt] = p / (eps * V);
        if (E) {
            E[3 * tt + 0] = ex / (eps * V);
            E[3 * tt + 1] = ey / (eps * V);
            E[3 * tt + 2] = ez / (eps * V);
        }
    }
    free(km); free(Sre); free(Sim);
}

/* ibo_real_matrix with a radius per bead. */
void ibo_real_matrix_radii(int n, const double *x, const double *L, const double *rad, double xi, double rc,
                           double *Mr)
{
    const int m0 = image_range(rc, L[0]), m1 = image_range(rc, L[1]), m2 = image_range(rc, L[2]);
#pragma omp parallel for schedule(dynamic, 4)
    for (int al = 0; al < n; ++al) {
        for (int be = 0; be < n; ++be) {
            const double a = rad[al], b = rad[be];
            double dx0 = x[3 * al + 0] - x[3 * be + 0];
            double dy0 = x[3 * al + 1] - x[3 * be + 1];
            double dz0 = x[3 * al + 2] - x[3 * be + 2];
            dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
            dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
            dz0 -= L[2] * floor(dz0 / L[2] + 0.5);
            double m = (al == be) ? ibo_phi_real2(0.0, a, a, xi) : 0.0;
            for (int i = -m0; i <= m0; ++i)
                for (int j = -m1; j <= m1; ++j)
                    for (int k = -m2; k <= m2; ++k) {
                        if (al == be && i == 0 && j == 0 && k == 0)
                            continue;
                        const double dx = dx0 + i * L[0], dy = dy0 + j * L[1], dz = dz0 + k * L[2];
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= rc)
                            continue;
                        m += ibo_phi_real2(r, a, b, xi);
                    }
            Mr[(size_t)al * n + be] = m;
        }
    }
}
