// bodies.cu -- bead <-> body bookkeeping and segmented reductions over the
// contiguous bead ranges of the summation tensor Sigma (Appendix): dipoles
// (Eq. rigid_dipole), bead forces (Eq. beadforce), body forces and torques
// (Sec. III.C), the energy (Eq. pot_syst) and the Brownian-dynamics step of
// Sec. V.A (Eq. forward, Eq. hardsphereFD).  Ions one per thread, multi-bead bodies
// one per block (body_role).
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ibp {

namespace {

__global__ void bead_body_kernel(int nb, const int* __restrict__ off, int* __restrict__ bead_body) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    for (int j = off[b] + lane; j < off[b + 1]; j += 32) bead_body[j] = b;
}

__global__ void rel_kernel(int n, const double* __restrict__ xw, const int* __restrict__ bead_body,
                           const double* __restrict__ X, double L0, double L1, double L2, double iL0, double iL1,
                           double iL2, double* __restrict__ rel) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = bead_body[i];
    // minimum image with a multiplication by 1/L (the reference points need not be wrapped)
    const double d0 = xw[3 * i + 0] - X[3 * b + 0], d1 = xw[3 * i + 1] - X[3 * b + 1], d2 = xw[3 * i + 2] - X[3 * b + 2];
    rel[3 * i + 0] = d0 - L0 * floor(d0 * iL0 + 0.5);
    rel[3 * i + 1] = d1 - L1 * floor(d1 * iL1 + 0.5);
    rel[3 * i + 2] = d2 - L2 * floor(d2 * iL2 + 0.5);
}

// Block roles of the per-body kernels (kBodyThreads threads per block): the first
// body_ion_blocks(nb) blocks take one body per thread of their first kIonsPerBlock
// threads and handle the single-bead bodies (ions, most of the bodies of an
// electrolyte; few per block, so that the FP64 noise of the BD step spreads over
// many SMs); the others take one multi-bead body per block from the list mb_body
// (GB300 runs FP64 at a small fraction of its FP32 rate: a body's sums spread over
// the four schedulers of an SM instead of one warp).  Returns false for threads
// without work; a body block returns true for all its threads (block barriers).
constexpr int kBodyThreads = 256;
constexpr int kIonsPerBlock = 32;

__host__ __device__ __forceinline__ int body_ion_blocks(int nb) { return (nb + kIonsPerBlock - 1) / kIonsPerBlock; }

__device__ __forceinline__ bool body_role(int nb, int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                                          int& body, int& lane, bool& ion) {
    const int ib = body_ion_blocks(nb);
    if ((int)blockIdx.x < ib) {
        ion = true;
        lane = 0;
        body = (int)blockIdx.x * kIonsPerBlock + (int)threadIdx.x;
        return (int)threadIdx.x < kIonsPerBlock && body < nb && off[body + 1] - off[body] == 1;
    }
    ion = false;
    lane = threadIdx.x;
    body = mb_body[(int)blockIdx.x - ib];
    return true;
}

int body_grid(int nb, int nmb) { return body_ion_blocks(nb) + nmb; }

// Sums v[0..NV) over a body block (every thread takes part); thread 0 gets the totals.
template <int NV>
__device__ __forceinline__ void body_block_sum(double (&v)[NV], double (*sh)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();   // the previous sum's reads of sh are done
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[threadIdx.x >> 5][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = 0.0;
            for (int w = 0; w < kBodyThreads / 32; ++w) t += sh[w][i];
            v[i] = t;
        }
}

__global__ void dipole_kernel(int nb, int nmb, const int* __restrict__ mb_body, int n, int nrhs,
                              const int* __restrict__ off, const double* __restrict__ rel,
                              const double* __restrict__ q, double* __restrict__ S) {
    int b, lane;
    bool ion;
    if (!body_role(nb, nmb, mb_body, off, b, lane, ion)) return;
    if (ion) {
        const int j = off[b];
        for (int r = 0; r < nrhs; ++r) {
            const double qq = q[(size_t)r * n + j];
            double* o = S + ((size_t)r * nb + b) * 3;
            o[0] = rel[3 * j + 0] * qq;
            o[1] = rel[3 * j + 1] * qq;
            o[2] = rel[3 * j + 2] * qq;
        }
        return;
    }
    __shared__ double sh[kBodyThreads / 32][3];
    for (int r = 0; r < nrhs; ++r) {
        double v[3] = {0, 0, 0};
        for (int j = off[b] + lane; j < off[b + 1]; j += kBodyThreads) {
            const double qq = q[(size_t)r * n + j];
            v[0] += rel[3 * j + 0] * qq;
            v[1] += rel[3 * j + 1] * qq;
            v[2] += rel[3 * j + 2] * qq;
        }
        body_block_sum<3>(v, sh);
        if (lane == 0) {
            double* o = S + ((size_t)r * nb + b) * 3;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
    }
}

__global__ void force_kernel(int n, const double* __restrict__ q, const double* __restrict__ E0,
                             const double* __restrict__ E, double* __restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    f[i] = q[i / 3] * (E0[i % 3] + E[i]);
}

__global__ void force_torque_kernel(int nb, int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                                    const double* __restrict__ rel, const double* __restrict__ f,
                                    double* __restrict__ F, double* __restrict__ L) {
    int b, lane;
    bool ion;
    if (!body_role(nb, nmb, mb_body, off, b, lane, ion)) return;
    if (ion) {
        const int j = off[b];
        const double ax = f[3 * j], ay = f[3 * j + 1], az = f[3 * j + 2];
        const double rx = rel[3 * j], ry = rel[3 * j + 1], rz = rel[3 * j + 2];
        F[3 * b] = ax; F[3 * b + 1] = ay; F[3 * b + 2] = az;
        L[3 * b] = ry * az - rz * ay;
        L[3 * b + 1] = rz * ax - rx * az;
        L[3 * b + 2] = rx * ay - ry * ax;
        return;
    }
    __shared__ double sh[kBodyThreads / 32][6];
    double v[6] = {0, 0, 0, 0, 0, 0};   // F, then L
    for (int j = off[b] + lane; j < off[b + 1]; j += kBodyThreads) {
        const double ax = f[3 * j], ay = f[3 * j + 1], az = f[3 * j + 2];
        const double rx = rel[3 * j], ry = rel[3 * j + 1], rz = rel[3 * j + 2];
        v[0] += ax; v[1] += ay; v[2] += az;
        v[3] += ry * az - rz * ay;
        v[4] += rz * ax - rx * az;
        v[5] += rx * ay - ry * ax;
    }
    body_block_sum<6>(v, sh);
    if (lane == 0) {
        F[3 * b] = v[0]; F[3 * b + 1] = v[1]; F[3 * b + 2] = v[2];
        L[3 * b] = v[3]; L[3 * b + 1] = v[4]; L[3 * b + 2] = v[5];
    }
}

// Per-body energy contribution Q_i Psi_i - S_i . E0 with
// Psi_i - Psi_0,i = mean_j (psi_ij - r_ij . E0) (Eq. beadpot1) and Psi_0,i = -X_i . E0.
__global__ void energy_body_kernel(int nb, int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                                   const double* __restrict__ rel,
                                   const double* __restrict__ q, const double* __restrict__ psi,
                                   const double* __restrict__ E0, const double* __restrict__ X,
                                   const double* __restrict__ Q, double* __restrict__ contrib) {
    int b, lane;
    bool ion;
    if (!body_role(nb, nmb, mb_body, off, b, lane, ion)) return;
    const double e0 = E0[0], e1 = E0[1], e2 = E0[2];
    if (ion) {
        const int j = off[b];
        const double rE = rel[3 * j] * e0 + rel[3 * j + 1] * e1 + rel[3 * j + 2] * e2;
        const double Psi = (psi[j] - rE) / 1.0 - (X[3 * b] * e0 + X[3 * b + 1] * e1 + X[3 * b + 2] * e2);
        contrib[b] = Q[b] * Psi - q[j] * rE;
        return;
    }
    __shared__ double sh[kBodyThreads / 32][2];
    double v[2] = {0, 0};   // sum (psi - r.E0), sum q r.E0
    for (int j = off[b] + lane; j < off[b + 1]; j += kBodyThreads) {
        const double rE = rel[3 * j] * e0 + rel[3 * j + 1] * e1 + rel[3 * j + 2] * e2;
        v[0] += psi[j] - rE;
        v[1] += q[j] * rE;
    }
    body_block_sum<2>(v, sh);
    if (lane == 0) {
        const double cnt = (double)(off[b + 1] - off[b]);
        const double Psi = v[0] / cnt - (X[3 * b] * e0 + X[3 * b + 1] * e1 + X[3 * b + 2] * e2);
        contrib[b] = Q[b] * Psi - v[1];
    }
}

__global__ void half_sum_kernel(int m, const double* __restrict__ v, double* __restrict__ out) {
    __shared__ double s[32];
    double acc = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) acc += v[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) *out = 0.5 * t;
    }
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller ----
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const unsigned lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += W0;
            k.y += W1;
        }
    }
    return c;
}


// f_tot = f_bead + Heyes-Melrose forces gamma/(2 dt) (2a - r) (x_a - x_b)/r for
// r < 2a between beads of different bodies (Eq. hardsphereFD).
// The pair table's rows and columns are in the cell-sorted order: row t is
// bead order[t].
// Pairs are screened with the FP32 positions (a margin far above their rounding);
// the few that may overlap are decided in FP64.
// The same forces from the table's list of overlapping pairs (r < 2a, listed when the
// pair values were built), one thread per ordered pair adding the force on its row bead
// (the table holds both orders of a pair); f_out starts as a copy of f_bead.  A walk of
// every pair of the table to find the few overlapping ones was the cost of this pass.
__global__ void hard_sphere_list_kernel(const int* __restrict__ ov_count, const int* __restrict__ ov_list,
                                        const double* __restrict__ xw, double L0, double L1, double L2,
                                        const int* __restrict__ prow, const int* __restrict__ col,
                                        const int* __restrict__ order, const int* __restrict__ bead_body, double a,
                                        double coef, double* __restrict__ f_out) {
    const int m = *ov_count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const long long p = ov_list[t];
        const int al = order[prow[p]], be = order[col[p]];
        if (bead_body[al] == bead_body[be]) continue;
        const double dx = min_image_wrapped(xw[3 * al] - xw[3 * be], L0);
        const double dy = min_image_wrapped(xw[3 * al + 1] - xw[3 * be + 1], L1);
        const double dz = min_image_wrapped(xw[3 * al + 2] - xw[3 * be + 2], L2);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < 4.0 * a * a && r2 > 0.0) {
            const double r = sqrt(r2);
            const double mag = coef * (2.0 * a - r) / r;
            atomicAdd(f_out + 3 * al, mag * dx);
            atomicAdd(f_out + 3 * al + 1, mag * dy);
            atomicAdd(f_out + 3 * al + 2, mag * dz);
        }
    }
}

// Radii of the radius classes (beads of unequal radii: contact at a_alpha + a_beta).
struct HsRadii {
    double a[IBPME_MAX_RADIUS_CLASSES];
};

// cls: radius class of each bead, or NULL for one radius a (the FP32 screen then
// takes a as the largest radius).
__global__ void hard_sphere_kernel(int n, const double* __restrict__ xw, const float4* __restrict__ xf, double L0,
                                   double L1, double L2, const long long* __restrict__ rowptr,
                                   const int* __restrict__ col, const int* __restrict__ order,
                                   const int* __restrict__ bead_body, double a, const int* __restrict__ cls,
                                   HsRadii R, double coef, const double* __restrict__ f_in,
                                   double* __restrict__ f_out) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int al = order[t];
    const float4 pa = xf[al];
    const float Lx = (float)L0, Ly = (float)L1, Lz = (float)L2;
    const float lim = (float)(4.0 * a * a * (1.0 + 1e-3)) + 1e-5f;
    double fx = 0, fy = 0, fz = 0;
    for (long long p = rowptr[t] + lane; p < rowptr[t + 1]; p += 32) {
        const int be = order[col[p]];
        const float4 pb = xf[be];
        const float ex = min_image_wrapped(pa.x - pb.x, Lx), ey = min_image_wrapped(pa.y - pb.y, Ly);
        const float ez = min_image_wrapped(pa.z - pb.z, Lz);
        if (ex * ex + ey * ey + ez * ez >= lim) continue;
        if (bead_body[be] == bead_body[al]) continue;
        const double x0 = xw[3 * al], y0 = xw[3 * al + 1], z0 = xw[3 * al + 2];
        const double dx = min_image_wrapped(x0 - xw[3 * be], L0);
        const double dy = min_image_wrapped(y0 - xw[3 * be + 1], L1);
        const double dz = min_image_wrapped(z0 - xw[3 * be + 2], L2);
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double contact = cls ? R.a[cls[al]] + R.a[cls[be]] : 2.0 * a;
        if (r2 < contact * contact && r2 > 0.0) {   // overlap: the only pairs that need r
            const double r = sqrt(r2);
            const double m = coef * (contact - r) / r;
            fx += m * dx;
            fy += m * dy;
            fz += m * dz;
        }
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if (lane == 0) {
        f_out[3 * al] = f_in[3 * al] + fx;
        f_out[3 * al + 1] = f_in[3 * al + 1] + fy;
        f_out[3 * al + 2] = f_in[3 * al + 2] + fz;
    }
}

struct BdConst {
    double dt, gamma, kT;
    unsigned long long seed;
    unsigned step;
};

__device__ void rotation_matrix(const double* th, double* R) {
    const double ang = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    if (ang == 0.0) {
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
        return;
    }
    const double kx = th[0] / ang, ky = th[1] / ang, kz = th[2] / ang;
    const double K[9] = {0, -kz, ky, kz, 0, -kx, -ky, kx, 0};
    const double s = sin(ang), c1 = 1.0 - cos(ang);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = 0;
            for (int m = 0; m < 3; ++m) k2 += K[3 * i + m] * K[3 * m + j];
            R[3 * i + j] = (i == j ? 1.0 : 0.0) + s * K[3 * i + j] + c1 * k2;
        }
}

// One body per thread (ions) or per block: F, L, J summed over the body; threads 0-2
// draw the noise, thread 0 forms U, Omega, R.
// Box-Muller pair t of body b: Philox counter (body, step, t); (rad cos, rad sin).
__device__ __forceinline__ void bd_normals(int b, const BdConst& bc, unsigned t, double& rad, double& ang) {
    const uint2 key = make_uint2((unsigned)(bc.seed & 0xffffffffull), (unsigned)(bc.seed >> 32));
    const uint4 w = philox4x32_10(make_uint4((unsigned)b, bc.step, t, 0x1B5EEDu), key);
    const double u1 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
    rad = sqrt(-2.0 * log(u1));
    ang = 6.283185307179586476925286766559 * u2;
}

__global__ void bd_body_kernel(int nb, int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                               const double* __restrict__ rel,
                               const double* __restrict__ f, const double* __restrict__ X, BdConst bc,
                               double* __restrict__ X_out, double* __restrict__ Rm) {
    int b, lane;
    bool ion;
    if (!body_role(nb, nmb, mb_body, off, b, lane, ion)) return;
    if (ion) {   // translation only (r = 0, no rotation): z0, z1 from pair 0, z2 the cosine of pair 1
        double rad0, ang0, rad1, ang1, sn, cs;
        bd_normals(b, bc, 0u, rad0, ang0);
        bd_normals(b, bc, 1u, rad1, ang1);
        sincos(ang0, &sn, &cs);
        const double z[3] = {rad0 * cs, rad0 * sn, rad1 * cos(ang1)};
        const int j = off[b];
        const double mt = 1.0 / bc.gamma;
        const double st = sqrt(2.0 * bc.kT * bc.dt * mt);
        for (int i = 0; i < 3; ++i) X_out[3 * b + i] = X[3 * b + i] + f[3 * j + i] * mt * bc.dt + st * z[i];
        const double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        for (int i = 0; i < 9; ++i) Rm[9 * b + i] = R[i];
        return;
    }
    const int Ni = off[b + 1] - off[b];
    // noise: Box-Muller pair t from Philox counter (body, step, t) on lane t, in
    // parallel; an ion needs z0..z2 only (pairs 0 and 1, the cosine of pair 1)
    double za = 0.0, zb = 0.0;
    if (lane < 3) {   // pair t on lane t
        double rad, ang, sn, cs;
        bd_normals(b, bc, (unsigned)lane, rad, ang);
        sincos(ang, &sn, &cs);
        za = rad * cs;
        zb = rad * sn;
    }
    double z[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        z[2 * i] = __shfl_sync(0xffffffffu, za, i);
        z[2 * i + 1] = __shfl_sync(0xffffffffu, zb, i);
    }
    __shared__ double sh[kBodyThreads / 32][12];
    double v[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // F, L, J (upper triangle)
    for (int j = off[b] + lane; j < off[b + 1]; j += kBodyThreads) {
        const double rx = rel[3 * j], ry = rel[3 * j + 1], rz = rel[3 * j + 2];
        const double ax = f[3 * j], ay = f[3 * j + 1], az = f[3 * j + 2];
        v[0] += ax; v[1] += ay; v[2] += az;
        v[3] += ry * az - rz * ay;
        v[4] += rz * ax - rx * az;
        v[5] += rx * ay - ry * ax;
        const double rr = rx * rx + ry * ry + rz * rz;
        v[6] += rr - rx * rx; v[7] += -rx * ry; v[8] += -rx * rz;
        v[9] += rr - ry * ry; v[10] += -ry * rz; v[11] += rr - rz * rz;
    }
    body_block_sum<12>(v, sh);
    if (lane != 0) return;
    const double F[3] = {v[0], v[1], v[2]}, L[3] = {v[3], v[4], v[5]};
    const double J[6] = {v[6], v[7], v[8], v[9], v[10], v[11]};
    const double mt = 1.0 / (Ni * bc.gamma);
    const double st = sqrt(2.0 * bc.kT * bc.dt * mt);
    for (int i = 0; i < 3; ++i) X_out[3 * b + i] = X[3 * b + i] + F[i] * mt * bc.dt + st * z[i];
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (Ni > 1) {
        // symmetric 3x3 gamma J and its inverse (adjugate / determinant)
        const double a00 = bc.gamma * J[0], a01 = bc.gamma * J[1], a02 = bc.gamma * J[2];
        const double a11 = bc.gamma * J[3], a12 = bc.gamma * J[4], a22 = bc.gamma * J[5];
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        const double tr = a00 + a11 + a22;
        if (det > 1e-14 * tr * tr * tr) {
            const double id = 1.0 / det;
            const double m00 = c00 * id, m01 = c01 * id, m02 = c02 * id;
            const double m11 = (a00 * a22 - a02 * a02) * id, m12 = (a01 * a02 - a00 * a12) * id;
            const double m22 = (a00 * a11 - a01 * a01) * id;
            const double Om[3] = {m00 * L[0] + m01 * L[1] + m02 * L[2], m01 * L[0] + m11 * L[1] + m12 * L[2],
                                  m02 * L[0] + m12 * L[1] + m22 * L[2]};
            // Cholesky factor of the rotational mobility
            const double l00 = sqrt(m00);
            const double l10 = m01 / l00, l20 = m02 / l00;
            const double l11 = sqrt(m11 - l10 * l10);
            const double l21 = (m12 - l20 * l10) / l11;
            const double l22 = sqrt(m22 - l20 * l20 - l21 * l21);
            const double sr = sqrt(2.0 * bc.kT * bc.dt);
            const double th[3] = {Om[0] * bc.dt + sr * (l00 * z[3]),
                                  Om[1] * bc.dt + sr * (l10 * z[3] + l11 * z[4]),
                                  Om[2] * bc.dt + sr * (l20 * z[3] + l21 * z[4] + l22 * z[5])};
            rotation_matrix(th, R);
        }
    }
    for (int i = 0; i < 9; ++i) Rm[9 * b + i] = R[i];
}

__global__ void bd_bead_kernel(int n, const int* __restrict__ bead_body, const double* __restrict__ rel,
                               const double* __restrict__ X_out, const double* __restrict__ Rm,
                               double* __restrict__ x_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = bead_body[i];
    const double* R = Rm + 9 * b;
    const double rx = rel[3 * i], ry = rel[3 * i + 1], rz = rel[3 * i + 2];
    x_out[3 * i + 0] = X_out[3 * b + 0] + R[0] * rx + R[1] * ry + R[2] * rz;
    x_out[3 * i + 1] = X_out[3 * b + 1] + R[3] * rx + R[4] * ry + R[5] * rz;
    x_out[3 * i + 2] = X_out[3 * b + 2] + R[6] * rx + R[7] * ry + R[8] * rz;
}

}  // namespace

void bodies_upload(ibpme_ctx* c, int n, const ibpme_bodies* b, const double* xw, int ncfg, const int* cfg_beads,
                   const int* cfg_bodies, const unsigned long long* off_hash) {
    BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    const int nb = b->n_bodies;
    // the same offsets as the last (validated) upload, by their hash: no read-back
    const bool known = off_hash && bd.off_hash != 0 && *off_hash == bd.off_hash && bd.host_n == n &&
                       (int)bd.host_off.size() == nb + 1;
    std::vector<int> off;
    if (known) {
        off = bd.host_off;
    } else {
        off.resize(nb + 1);
        IBP_CUDA(cudaMemcpyAsync(off.data(), b->body_offsets, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost, s));
        IBP_CUDA(cudaStreamSynchronize(s));
        if (off[0] != 0 || off[nb] != n) fail(IBPME_ERR_ARG, "body_offsets must start at 0 and end at n = %d", n);
        for (int i = 0; i < nb; ++i)
            if (off[i + 1] <= off[i]) fail(IBPME_ERR_ARG, "body %d is empty or offsets decrease", i);
        bd.off_hash = 0;   // set below once the structure is recorded
    }
    // configurations: contiguous ranges of bodies (and hence of beads)
    std::vector<int> cb(ncfg + 1), cbe(ncfg + 1);
    if (ncfg == 1 && !cfg_bodies) {
        cb = {0, nb};
        cbe = {0, n};
    } else {
        for (int k = 0; k <= ncfg; ++k) cb[k] = cfg_bodies[k];
        if (cb[0] != 0 || cb[ncfg] != nb) fail(IBPME_ERR_ARG, "configuration body ranges must cover 0..n_bodies");
        for (int k = 0; k < ncfg; ++k)
            if (cb[k + 1] <= cb[k]) fail(IBPME_ERR_ARG, "configuration %d has no body", k);
        for (int k = 0; k <= ncfg; ++k) {
            cbe[k] = off[cb[k]];
            if (cfg_beads && cfg_beads[k] != cbe[k])
                fail(IBPME_ERR_ARG, "configuration %d: bead offset %d does not start body %d", k, cfg_beads[k], cb[k]);
        }
    }
    // unchanged structure (e.g. along a trajectory): keep the unknown lists
    const bool same = bd.host_n == n && bd.host_off == off && bd.host_cfg == cb;
    if (!same) {
        // unknowns of configuration k: its free beads (beads of multi-bead bodies), then its multi-bead bodies
        std::vector<int> free_idx, free_unk, mb_body, mb_unk, mb_first, mb_cnt, bead_unk(n, -1), body_unk(nb, -1),
            unk_cfg, bead_cfg(n), uo(ncfg + 1, 0), free_pos(n, -1), free_cfg;
        int u = 0;
        for (int k = 0; k < ncfg; ++k) {
            uo[k] = u;
            for (int i = cb[k]; i < cb[k + 1]; ++i) {
                for (int j = off[i]; j < off[i + 1]; ++j) bead_cfg[j] = k;
                if (off[i + 1] - off[i] < 2) continue;
                for (int j = off[i]; j < off[i + 1]; ++j) {
                    bead_unk[j] = u;
                    free_pos[j] = (int)free_idx.size();
                    free_cfg.push_back(k);
                    free_idx.push_back(j);
                    free_unk.push_back(u++);
                    unk_cfg.push_back(k);
                }
            }
            for (int i = cb[k]; i < cb[k + 1]; ++i) {
                if (off[i + 1] - off[i] < 2) continue;
                body_unk[i] = u;
                mb_body.push_back(i);
                mb_unk.push_back(u++);
                mb_first.push_back(bead_unk[off[i]]);
                mb_cnt.push_back(off[i + 1] - off[i]);
                unk_cfg.push_back(k);
            }
        }
        uo[ncfg] = u;
        bd.nb = nb;
        bd.nmb = (int)mb_body.size();
        bd.nfree = (int)free_idx.size();
        bd.nk = u;
        bd.ncfg = ncfg;
        bd.uo_h = uo;
        bd.cfg_beads_h = cbe;
        bd.cfg_bodies_h = cb;
        auto up = [&](DevBuf& dst, const std::vector<int>& v) {
            dst.ensure(sizeof(int) * (v.size() + 1));
            if (!v.empty())
                IBP_CUDA(cudaMemcpyAsync(dst.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
        };
        std::vector<int> iota(free_idx.size());
        for (size_t f = 0; f < iota.size(); ++f) iota[f] = (int)f;
        up(bd.free_idx, free_idx);
        up(bd.free_unk, free_unk);
        up(bd.free_pos, free_pos);
        up(bd.free_cfg, free_cfg);
        up(bd.iota, iota);
        bd.free_pos_h = free_pos;
        up(bd.mb_body, mb_body);
        up(bd.mb_unk, mb_unk);
        up(bd.mb_first, mb_first);
        up(bd.mb_cnt, mb_cnt);
        up(bd.bead_unk, bead_unk);
        up(bd.body_unk, body_unk);
        up(bd.unk_cfg, unk_cfg);
        up(bd.bead_cfg, bead_cfg);
        up(bd.uo, uo);
        up(bd.cfg_beads, cbe);
        up(bd.cfg_bodies, cb);
        up(bd.off, off);
        bd.bead_body.ensure(sizeof(int) * (n + 1));
        bead_body_kernel<<<div_up((long long)nb * 32, 128), 128, 0, s>>>(nb, bd.off.as<int>(), bd.bead_body.as<int>());
        IBP_CHECK_LAUNCH();
        IBP_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
        bd.host_off = off;
        bd.host_cfg = cb;
        bd.host_n = n;
        bd.max_beads = 0;
        for (int i = 0; i < nb; ++i) bd.max_beads = std::max(bd.max_beads, off[i + 1] - off[i]);
        ++bd.version;
    }
    bd.off_hash = off_hash ? *off_hash : 0;
    bd.X.ensure(sizeof(double) * 3 * nb);
    bd.Q.ensure(sizeof(double) * nb);
    IBP_CUDA(cudaMemcpyAsync(bd.X.p, b->X, sizeof(double) * 3 * nb, cudaMemcpyDeviceToDevice, s));
    IBP_CUDA(cudaMemcpyAsync(bd.Q.p, b->Q, sizeof(double) * nb, cudaMemcpyDeviceToDevice, s));
    bd.rel.ensure(sizeof(double) * 3 * n);
    rel_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, bd.bead_body.as<int>(), bd.X.as<double>(), c->p.box[0],
                                              c->p.box[1], c->p.box[2], 1.0 / c->p.box[0], 1.0 / c->p.box[1],
                                              1.0 / c->p.box[2], bd.rel.as<double>());
    IBP_CHECK_LAUNCH();
    c->bodies_current = true;
}

void body_dipoles(ibpme_ctx* c, int n, const double* q, int nrhs, double* S) {
    ProfScope ps(ST_BODIES, c->stream);
    BodyData& bd = c->bodies;
    dipole_kernel<<<body_grid(bd.nb, bd.nmb), kBodyThreads, 0, c->stream>>>(
        bd.nb, bd.nmb, bd.mb_body.as<int>(), n, nrhs, bd.off.as<int>(), bd.rel.as<double>(), q, S);
    IBP_CHECK_LAUNCH();
}

void bead_forces(ibpme_ctx* c, int n, const double* q, const double* E0, const double* E, double* f) {
    ProfScope ps(ST_BODIES, c->stream);
    force_kernel<<<div_up(3LL * n, 256), 256, 0, c->stream>>>(n, q, E0, E, f);
    IBP_CHECK_LAUNCH();
}

void body_reduce_force_torque(ibpme_ctx* c, int n, const double* f, double* F, double* L) {
    ProfScope ps(ST_BODIES, c->stream);
    (void)n;
    BodyData& bd = c->bodies;
    force_torque_kernel<<<body_grid(bd.nb, bd.nmb), kBodyThreads, 0, c->stream>>>(
        bd.nb, bd.nmb, bd.mb_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(), f, F, L);
    IBP_CHECK_LAUNCH();
}

void body_energy(ibpme_ctx* c, int n, const double* q, const double* psi, const double* E0, double* U) {
    ProfScope ps(ST_BODIES, c->stream);
    (void)n;
    BodyData& bd = c->bodies;
    double* contrib = static_cast<double*>(bd.scratch.ensure(sizeof(double) * (bd.nb + 1)));
    energy_body_kernel<<<body_grid(bd.nb, bd.nmb), kBodyThreads, 0, c->stream>>>(
        bd.nb, bd.nmb, bd.mb_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(), q, psi, E0, bd.X.as<double>(),
        bd.Q.as<double>(), contrib);
    IBP_CHECK_LAUNCH();
    half_sum_kernel<<<1, 1024, 0, c->stream>>>(bd.nb, contrib, U);
    IBP_CHECK_LAUNCH();
}

void bd_step(ibpme_ctx* c, int n, const double* xw, const double* f, const ibpme_bd_params* p, double* x_out,
             double* X_out) {
    BodyData& bd = c->bodies;
    NearList& nl = c->near;
    cudaStream_t s = c->stream;
    ProfScope ps(ST_BODIES, s);
    double* ftot = static_cast<double*>(bd.scratch.ensure(sizeof(double) * (3 * (size_t)n + 9 * (size_t)bd.nb)));
    double* Rm = ftot + 3 * (size_t)n;
    if (nl.ov_valid && c->ncls == 1) {
        IBP_CUDA(cudaMemcpyAsync(ftot, f, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToDevice, s));
        hard_sphere_list_kernel<<<152 * 4, 128, 0, s>>>(nl.ov_count.as<int>(), nl.ov_list.as<int>(), xw, c->p.box[0],
                                                        c->p.box[1], c->p.box[2], nl.prow.as<int>(), nl.col.as<int>(),
                                                        nl.cell_beads.as<int>(), bd.bead_body.as<int>(), c->a,
                                                        p->gamma / (2.0 * p->dt), ftot);
    } else {
        HsRadii R{};
        for (int k = 0; k < c->ncls; ++k) R.a[k] = c->cls_a[k];
        hard_sphere_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(
            n, xw, nl.xf.as<float4>(), c->p.box[0], c->p.box[1], c->p.box[2], nl.rowptr.as<long long>(),
            nl.col.as<int>(), nl.cell_beads.as<int>(), bd.bead_body.as<int>(), c->a,
            c->ncls > 1 ? c->cls.as<int>() : nullptr, R, p->gamma / (2.0 * p->dt), f, ftot);
    }
    IBP_CHECK_LAUNCH();
    BdConst bc{p->dt, p->gamma, p->kT, p->seed, (unsigned)(p->step & 0xffffffffLL)};
    bd_body_kernel<<<body_grid(bd.nb, bd.nmb), kBodyThreads, 0, s>>>(bd.nb, bd.nmb, bd.mb_body.as<int>(),
                                                                     bd.off.as<int>(), bd.rel.as<double>(), ftot,
                                                                     bd.X.as<double>(), bc, X_out, Rm);
    IBP_CHECK_LAUNCH();
    bd_bead_kernel<<<div_up(n, 256), 256, 0, s>>>(n, bd.bead_body.as<int>(), bd.rel.as<double>(), X_out, Rm, x_out);
    IBP_CHECK_LAUNCH();
}

}  // namespace ibp
