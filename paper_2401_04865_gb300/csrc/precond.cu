// precond.cu -- body-block right preconditioner of the reduced saddle system
// (Sec. III.B, Eq. saddle), a solver choice outside the paper.
//
// Within one rigid body the saddle operator is dominated by the body's own
// interactions.  For every multi-bead body of at most kPrecondMaxBeads (8,192) beads
// the preconditioner applies the exact inverse of that body's free-space block
//     P_b = [ -M_b  e ]      M_b(i, j) = M(|r_i - r_j|)   (Sec. II: 1/(4 pi eps r) for
//           [  e^T  0 ]                                   r >= 2a, (4a - r)/(16 pi a^2 eps) below)
// and the identity elsewhere.  With g = M_b^{-1} e and s = e^T g,
//     P_b^{-1} [v; psi] = [ -M_b^{-1} v + g t ; t ],   t = (g . v + psi) / s.
// M_b depends only on the distances between the body's beads, so it is the
// same for every position and orientation of a rigid body: inverses are kept
// per body shape (bead count and two rotation-invariant moments of the bead
// cloud) for the life of the context, and identical bodies share one.  GMRES
// then iterates on A P^{-1} (right preconditioning keeps the residual of the
// original system); only the inter-body coupling and the periodic images are
// left to the Krylov iteration.
#include "common.cuh"
#include "dfloat.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace ibp {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// moments of body b's bead cloud about its centroid: sum |d|^2, sum |d|^4 (rotation invariant)
__global__ void shape_moments_kernel(int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                                     const double* __restrict__ rel, double* __restrict__ out) {
    __shared__ double sh[3][32];
    const int b = blockIdx.x;
    if (b >= nmb) return;
    const int body = mb_body[b];
    const int j0 = off[body], j1 = off[body + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double c[3] = {0.0, 0.0, 0.0};
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
        for (int d = 0; d < 3; ++d) c[d] += rel[3 * j + d];
    for (int d = 0; d < 3; ++d) {
        double v = warp_sum(c[d]);
        if (lane == 0) sh[d][w] = v;
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[d][q];
        c[d] = t / (double)(j1 - j0);
    }
    __syncthreads();
    double m2 = 0.0, m4 = 0.0;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const double dx = rel[3 * j] - c[0], dy = rel[3 * j + 1] - c[1], dz = rel[3 * j + 2] - c[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        m2 += r2;
        m4 += r2 * r2;
    }
    m2 = warp_sum(m2);
    m4 = warp_sum(m4);
    if (lane == 0) {
        sh[0][w] = m2;
        sh[1][w] = m4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, bq = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += sh[0][q];
            bq += sh[1][q];
        }
        out[2 * b] = a;
        out[2 * b + 1] = bq;
    }
}

struct PrecondRadii {
    double a[IBPME_MAX_RADIUS_CLASSES];
};

// Free-space potential between shells of radii a and b, centres r apart (the real-space
// form of j0(ka) j0(kb)/k^2): 1/(4 pi r) apart, 1/(4 pi max(a, b)) one inside the
// other, (2(ab + ar + br) - a^2 - b^2 - r^2)/(16 pi a b r) overlapping; for a = b the
// (4a - r)/(16 pi a^2) of Sec. II.
__device__ __forceinline__ double shell_pair(double r, double a, double b) {
    if (r >= a + b) return 1.0 / (4.0 * kPi * r);
    if (r <= fabs(a - b)) return 1.0 / (4.0 * kPi * fmax(a, b));
    return (2.0 * (a * b + a * r + b * r) - a * a - b * b - r * r) / (16.0 * kPi * a * b * r);
}

// M_b of one body from its beads' relative positions (row-major nb x nb, FP32);
// cls: the beads' radius classes (NULL: every bead has radius a)
__global__ void block_matrix_kernel(int nb, const double* __restrict__ rel, double a, double eps,
                                    const int* __restrict__ cls, PrecondRadii R, float* __restrict__ A) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nb * nb) return;
    const int i = (int)(t / nb), j = (int)(t % nb);
    const double dx = rel[3 * i] - rel[3 * j], dy = rel[3 * i + 1] - rel[3 * j + 1],
                 dz = rel[3 * i + 2] - rel[3 * j + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (cls) {
        A[t] = (float)(shell_pair(r, R.a[cls[i]], R.a[cls[j]]) / eps);
        return;
    }
    A[t] = (float)(r >= 2.0 * a ? 1.0 / (4.0 * kPi * eps * r) : (4.0 * a - r) / (16.0 * kPi * a * a * eps));
}

// Blocked Gauss-Jordan inversion in place, FP32, one cooperative launch per shape.
// M_b is symmetric positive definite, so no pivoting.  For each panel p of kGjB
// columns (diagonal block P):
//   1. one block inverts P in shared memory (scalar Gauss-Jordan);
//   2. the column panel C = A[:, p] is saved and the row panel becomes
//      R = P^{-1} A[p, :] (R = P^{-1} on the panel's own columns);
//   3. every other row i: A[i, j] = (j in p ? 0 : A[i, j]) - C[i, :] R[:, j]; the
//      panel's rows take R.
// Grid-wide barriers separate the phases (the launch is cooperative, so every
// block is resident).  A non-positive pivot sets *bad and the result is unused.
constexpr int kGjB = 32;           // panel width
constexpr int kGjThreads = 256;
constexpr int kGjTile = 64;        // output tile of the rank-kGjB update (4 x 4 per thread)

__global__ void __launch_bounds__(kGjThreads) gj_blocked_kernel(int nb, float* __restrict__ A,
                                                                 float* __restrict__ Dinv,
                                                                 float* __restrict__ Cbuf,
                                                                 float* __restrict__ Rbuf, int* __restrict__ bad) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ float sD[kGjB][kGjB + 1];
    __shared__ float colk[kGjB], rowk[kGjB];
    __shared__ float sC[kGjTile][kGjB + 1];
    __shared__ float sR[kGjB][kGjTile + 1];
    const int tid = threadIdx.x;
    const int ntiles = (nb + kGjTile - 1) / kGjTile;
    for (int k0 = 0; k0 < nb; k0 += kGjB) {
        const int B = min(kGjB, nb - k0);
        // 1. the diagonal block's inverse (block 0)
        if (blockIdx.x == 0) {
            for (int e = tid; e < B * B; e += kGjThreads) sD[e / B][e % B] = A[(size_t)(k0 + e / B) * nb + k0 + e % B];
            __syncthreads();
            for (int k = 0; k < B; ++k) {
                if (tid < B) {
                    colk[tid] = sD[tid][k];
                    rowk[tid] = sD[k][tid];
                }
                __syncthreads();
                const float p = rowk[k];
                if (!(p > 0.f) && tid == 0) *bad = 1;
                const float ip = p > 0.f ? 1.0f / p : 0.f;
                for (int e = tid; e < B * B; e += kGjThreads) {
                    const int i = e / B, j = e % B;
                    float v;
                    if (i == k && j == k) v = ip;
                    else if (i == k) v = rowk[j] * ip;
                    else if (j == k) v = -colk[i] * ip;
                    else v = sD[i][j] - colk[i] * rowk[j] * ip;
                    sD[i][j] = v;
                }
                __syncthreads();
            }
            for (int e = tid; e < B * B; e += kGjThreads) Dinv[e] = sD[e / B][e % B];
        }
        grid.sync();
        // 2. C = A[:, panel]; R = P^{-1} A[panel, :] (R = P^{-1} on the panel columns)
        for (int e = tid; e < B * B; e += kGjThreads) sD[e / B][e % B] = Dinv[e];
        __syncthreads();
        for (long long e = blockIdx.x * (long long)kGjThreads + tid; e < (long long)nb * B;
             e += (long long)gridDim.x * kGjThreads) {
            const int i = (int)(e / B), c = (int)(e % B);
            Cbuf[e] = A[(size_t)i * nb + k0 + c];
        }
        for (int j = blockIdx.x * kGjThreads + tid; j < nb; j += gridDim.x * kGjThreads) {
            if (j >= k0 && j < k0 + B) {
                for (int r = 0; r < B; ++r) Rbuf[(size_t)r * nb + j] = sD[r][j - k0];
            } else {
                float col[kGjB];
                for (int c = 0; c < B; ++c) col[c] = A[(size_t)(k0 + c) * nb + j];
                for (int r = 0; r < B; ++r) {
                    float acc = 0.f;
                    for (int c = 0; c < B; ++c) acc += sD[r][c] * col[c];
                    Rbuf[(size_t)r * nb + j] = acc;
                }
            }
        }
        grid.sync();
        // 3. rank-B update by 64 x 64 tiles: thread (ty, tx) owns rows ty + 16 u, columns tx + 16 v
        const int ty = tid / 16, tx = tid % 16;
        for (int t = blockIdx.x; t < ntiles * ntiles; t += gridDim.x) {
            const int i0 = (t / ntiles) * kGjTile, j0 = (t % ntiles) * kGjTile;
            for (int e = tid; e < kGjTile * kGjB; e += kGjThreads) {
                const int r = e / kGjB, c = e % kGjB;
                sC[r][c] = (i0 + r < nb && c < B) ? Cbuf[(size_t)(i0 + r) * B + c] : 0.f;
                const int rr = e / kGjTile, cc = e % kGjTile;
                sR[rr][cc] = (rr < B && j0 + cc < nb) ? Rbuf[(size_t)rr * nb + j0 + cc] : 0.f;
            }
            __syncthreads();
            float acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
            for (int c = 0; c < B; ++c) {
                float cv[4], rv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) cv[u] = sC[ty + 16 * u][c];
#pragma unroll
                for (int v = 0; v < 4; ++v) rv[v] = sR[c][tx + 16 * v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += cv[u] * rv[v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + ty + 16 * u;
                if (i >= nb) continue;
                const bool prow = i >= k0 && i < k0 + B;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int j = j0 + tx + 16 * v;
                    if (j >= nb) continue;
                    float* a = A + (size_t)i * nb + j;
                    if (prow) *a = Rbuf[(size_t)(i - k0) * nb + j];
                    else *a = ((j >= k0 && j < k0 + B) ? 0.f : *a) - acc[u][v];
                }
            }
            __syncthreads();
        }
        grid.sync();
    }
}

// g = M^{-1} e (row sums of the FP32 inverse, summed in FP64)
__global__ void finish_shape_kernel(int nb, const float* __restrict__ minv, float* __restrict__ g) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) acc += (double)minv[(size_t)i * nb + j];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        g[i] = (float)t;
    }
}

__global__ void shape_s_kernel(int nb, const float* __restrict__ g, double* __restrict__ sinv) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += (double)g[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        *sinv = 1.0 / t;
    }
}

constexpr int kRowsPerBlock = 8;   // rows of M^{-1} per block: a body spreads over n_b / 8 SMs
constexpr int kApplyThreads = 256;

// out = P^{-1} u on the preconditioned bodies (grid: bodies x row chunks, R) and
// out = u on every other unknown (the trailing blocks of the grid).  With dir (the
// problem of prescribed bead potentials, whose operator is [-M 0; 0 I]) the block is
// [-M_b 0; 0 1] and its inverse -M_b^{-1} on the beads, the identity on the body row.
__global__ void __launch_bounds__(kApplyThreads)
precond_apply_kernel(bool dir, int npb, int chunks, int nk, long long ustride, const int* __restrict__ jdev,
                     const int* __restrict__ pb_shape, const int* __restrict__ pb_first,
                     const int* __restrict__ pb_psi, const int* __restrict__ pb_n,
                     const long long* __restrict__ shape_off, const long long* __restrict__ shape_goff,
                     const float* __restrict__ minv,
                     const float* __restrict__ gvec, const double* __restrict__ sinv, int nplain,
                     const int* __restrict__ plain, const double* __restrict__ u, double* __restrict__ out) {
    // u of the body as double-float: the FP32 inverse times it accumulates on the FP32
    // pipes (an FP64 multiply-add and a conversion per entry made this kernel wait on
    // GB300's FP64 rate), to about 2^-44 of each row's magnitude
    extern __shared__ float2 v[];   // the body's u as hi + lo floats (maxn entries)
    __shared__ df sh[32];
    __shared__ double tpsi;
    const int r = blockIdx.y;
    if (jdev) u += (size_t)(*jdev) * nk;
    const double* ur = u + (size_t)r * ustride;
    double* orow = out + (size_t)r * nk;
    const int body_blocks = npb * chunks;
    if ((int)blockIdx.x >= body_blocks) {   // identity on the unknowns no block covers
        const long long t = ((long long)blockIdx.x - body_blocks) * kApplyThreads + threadIdx.x;
        if (t < nplain) orow[plain[t]] = ur[plain[t]];
        return;
    }
    const int p = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
    const int nb = pb_n[p], first = pb_first[p], sh_id = pb_shape[p];
    const float* M = minv + shape_off[sh_id];
    const float* gv = gvec + shape_goff[sh_id];
    df acc = {0.0f, 0.0f};
    for (int j = threadIdx.x; j < nb; j += kApplyThreads) {
        const df d = df_split(ur[first + j]);
        v[j] = make_float2(d.hi, d.lo);
        acc = df_add(acc, df_mul_f(d, gv[j]));
    }
    acc = df_warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        df t = {0.0f, 0.0f};
        for (int q = 0; q < kApplyThreads / 32; ++q) t = df_add(t, sh[q]);
        tpsi = dir ? ur[pb_psi[p]] : (df_join(t) + ur[pb_psi[p]]) * sinv[sh_id];
    }
    __syncthreads();
    const double tp = tpsi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = chunk * kRowsPerBlock;
    for (int i = i0 + warp; i < min(nb, i0 + kRowsPerBlock); i += kApplyThreads / 32) {
        const float* Mi = M + (size_t)i * nb;
        df s = {0.0f, 0.0f};
        for (int j = lane; j < nb; j += 32) {
            const float2 vj = v[j];
            s = df_add(s, df_mul_f({vj.x, vj.y}, Mi[j]));
        }
        s = df_warp_sum(s);
        if (lane == 0) orow[first + i] = -df_join(s) + (dir ? 0.0 : (double)gv[i] * tp);
    }
    if (chunk == 0 && threadIdx.x == 0) orow[pb_psi[p]] = tp;
}

}  // namespace

// Shapes of the current bodies: reuse cached inverses, build the missing ones,
// and lay out the per-body tables of the apply kernel.  Returns false when no
// body qualifies (the solve then runs unpreconditioned).
namespace {

bool shape_matches(const Precond::Shape& sp, int nb, double m2, double m4) {
    return sp.nb == nb && std::fabs(sp.m2 - m2) <= 1e-9 * std::fabs(m2) + 1e-300 &&
           std::fabs(sp.m4 - m4) <= 1e-9 * std::fabs(m4) + 1e-300;
}

// Order-dependent hash of the radius classes of beads first .. first + nb - 1 (0: one radius).
unsigned long long class_hash(const ibpme_ctx* c, int first, int nb) {
    if (c->ncls < 2) return 0;
    unsigned long long h = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < nb; ++i) h = (h ^ (unsigned long long)(c->cls_h[first + i] + 1)) * 0x100000001B3ull;
    return h | 1ull;
}

// Moments of the current positions into pinned memory, without waiting (the
// solve synchronises before it returns, so the next call can read them).
void queue_moments(ibpme_ctx* c) {
    Precond& P = c->pre;
    const BodyData& bd = c->bodies;
    const size_t bytes = sizeof(double) * 2 * bd.nmb;
    if (P.hm_cap < bytes) {
        if (P.hm_pin) cudaFreeHost(P.hm_pin);
        P.hm_pin = nullptr;
        P.hm_cap = 0;
        IBP_CUDA(cudaMallocHost(&P.hm_pin, bytes));
        P.hm_cap = bytes;
    }
    double* mom = static_cast<double*>(P.moments.ensure(bytes));
    shape_moments_kernel<<<bd.nmb, 256, 0, c->stream>>>(bd.nmb, bd.mb_body.as<int>(), bd.off.as<int>(),
                                                        bd.rel.as<double>(), mom);
    IBP_CHECK_LAUNCH();
    IBP_CUDA(cudaMemcpyAsync(P.hm_pin, mom, bytes, cudaMemcpyDeviceToHost, c->stream));
}

}  // namespace

// A (nb x nb, FP32, symmetric positive definite) -> A^{-1} in place: one cooperative
// launch of the blocked Gauss-Jordan kernel, as many blocks as can be resident
// (at most one per 64 x 64 output tile).
void invert_spd(ibpme_ctx* c, int nb, float* A) {
    Precond& P = c->pre;
    cudaStream_t s = c->stream;
    float* Dinv = static_cast<float*>(P.gj_d.ensure(sizeof(float) * kGjB * kGjB));
    float* Cbuf = static_cast<float*>(P.gj_c.ensure(sizeof(float) * (size_t)nb * kGjB));
    float* Rbuf = static_cast<float*>(P.gj_r.ensure(sizeof(float) * (size_t)nb * kGjB));
    int* bad = static_cast<int*>(P.gj_bad.ensure(sizeof(int)));
    IBP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    int dev = 0, sms = 0, per_sm = 0;
    IBP_CUDA(cudaGetDevice(&dev));
    IBP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IBP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_blocked_kernel, kGjThreads, 0));
    const int tiles = div_up(nb, kGjTile) * div_up(nb, kGjTile);
    int blocks = std::max(1, std::min(per_sm * sms, std::max(tiles, div_up(nb, kGjThreads))));
    void* args[] = {&nb, &A, &Dinv, &Cbuf, &Rbuf, &bad};
    IBP_CUDA(cudaLaunchCooperativeKernel((const void*)gj_blocked_kernel, dim3(blocks), dim3(kGjThreads), args, 0, s));
    IBP_CHECK_LAUNCH();
    int hbad = 0;
    IBP_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    if (hbad) fail(IBPME_ERR_NONFINITE, "body block of %d beads is not positive definite", nb);
}

bool precond_prepare(ibpme_ctx* c) {
    Precond& P = c->pre;
    const BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    if (bd.nmb == 0) {
        P.npb = 0;
        return false;
    }
    // Steady state (a rigid-body trajectory): the same body structure as the last
    // preparation, and the moments of the previous call's positions still match
    // every assigned shape.  The tables stay; this call's moments are queued for
    // the next check.  A body that changed shape is caught one solve late, which
    // costs iterations, not accuracy (a right preconditioner does not change the
    // solution).
    if (P.prep_valid && P.prep_version == bd.version && P.prep_cls == cls_key(c) && P.hm_pin &&
        (int)P.assign.size() == bd.nmb) {
        bool same = true;
        for (int b = 0; b < bd.nmb && same; ++b) {
            const int id = P.assign[b];
            if (id >= 0) same = shape_matches(P.shapes[id], P.shapes[id].nb, P.hm_pin[2 * b], P.hm_pin[2 * b + 1]);
        }
        if (same) {
            queue_moments(c);
            return P.npb > 0;
        }
    }
    P.prep_valid = false;
    P.npb = 0;
    std::vector<int> mb_body(bd.nmb), mb_first(bd.nmb), mb_cnt(bd.nmb), mb_unk(bd.nmb);
    IBP_CUDA(cudaMemcpyAsync(mb_body.data(), bd.mb_body.p, sizeof(int) * bd.nmb, cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaMemcpyAsync(mb_first.data(), bd.mb_first.p, sizeof(int) * bd.nmb, cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaMemcpyAsync(mb_cnt.data(), bd.mb_cnt.p, sizeof(int) * bd.nmb, cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaMemcpyAsync(mb_unk.data(), bd.mb_unk.p, sizeof(int) * bd.nmb, cudaMemcpyDeviceToHost, s));
    double* mom = static_cast<double*>(P.moments.ensure(sizeof(double) * 2 * bd.nmb));
    shape_moments_kernel<<<bd.nmb, 256, 0, s>>>(bd.nmb, bd.mb_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(),
                                                mom);
    IBP_CHECK_LAUNCH();
    std::vector<double> hm(2 * (size_t)bd.nmb);
    IBP_CUDA(cudaMemcpyAsync(hm.data(), mom, sizeof(double) * 2 * bd.nmb, cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    const std::vector<int>& off = bd.host_off;

    // A configuration is preconditioned only if every one of its multi-bead bodies
    // qualifies: a system mixing P_b^{-1} blocks (eigenvalues near 1) with raw
    // blocks of M (eigenvalues near the self term) converges slower than either.
    const std::vector<int>& cb = bd.cfg_bodies_h;
    auto cfg_of = [&](int body) {
        return (int)(std::upper_bound(cb.begin(), cb.end(), body) - cb.begin()) - 1;
    };
    std::vector<char> cfg_ok(std::max(1, bd.ncfg), 1);
    for (int b = 0; b < bd.nmb; ++b)
        if (mb_cnt[b] > kPrecondMaxBeads) cfg_ok[cfg_of(mb_body[b])] = 0;
    std::vector<int> pb_shape, pb_first, pb_psi, pb_n;
    std::vector<char> covered(bd.nk, 0);
    std::vector<int> assign(bd.nmb, -1);
    for (int b = 0; b < bd.nmb; ++b) {
        const int nb = mb_cnt[b];
        if (nb > kPrecondMaxBeads || !cfg_ok[cfg_of(mb_body[b])]) continue;
        const double m2 = hm[2 * b], m4 = hm[2 * b + 1];
        const unsigned long long ck = class_hash(c, off[mb_body[b]], nb);
        int id = -1;
        for (size_t q = 0; q < P.shapes.size(); ++q) {
            if (P.shapes[q].ckey == ck && shape_matches(P.shapes[q], nb, m2, m4)) {
                id = (int)q;
                break;
            }
        }
        if (id < 0) {   // a new shape: build M_b from this body, invert, keep FP32 M^{-1}, g and 1/s
            const long long need = P.used + (long long)nb * nb;
            if (need * (long long)sizeof(float) > kPrecondCacheBytes) {   // cache full: start over
                P.shapes.clear();
                P.used = 0;
                P.gused = 0;
                pb_shape.clear();   // the bodies already listed refer to dropped shapes: redo them
                pb_first.clear();
                pb_psi.clear();
                pb_n.clear();
                std::fill(covered.begin(), covered.end(), 0);
                std::fill(assign.begin(), assign.end(), -1);
                b = -1;
                continue;
            }
            Precond::Shape sp;
            sp.nb = nb;
            sp.m2 = m2;
            sp.m4 = m4;
            sp.ckey = ck;
            sp.off = P.used;
            sp.goff = P.gused;
            P.used += (long long)nb * nb;
            P.gused += nb;
            P.minv.grow(sizeof(float) * (size_t)P.used, s);
            P.gvec.grow(sizeof(float) * (size_t)P.gused, s);
            P.sinv.grow(sizeof(double) * (P.shapes.size() + 1), s);
            float* A = P.minv.as<float>() + sp.off;   // inverted in place in the cache
            const double* rel = bd.rel.as<double>() + 3 * (size_t)off[mb_body[b]];
            const long long nn = (long long)nb * nb;
            PrecondRadii R{};
            for (int q = 0; q < c->ncls; ++q) R.a[q] = c->cls_a[q];
            const int* bcls = c->ncls > 1 ? c->cls.as<int>() + off[mb_body[b]] : nullptr;
            block_matrix_kernel<<<div_up(nn, 256), 256, 0, s>>>(nb, rel, c->a, c->eps, bcls, R, A);
            IBP_CHECK_LAUNCH();
            invert_spd(c, nb, A);
            finish_shape_kernel<<<nb, 128, 0, s>>>(nb, A, P.gvec.as<float>() + sp.goff);
            IBP_CHECK_LAUNCH();
            id = (int)P.shapes.size();
            shape_s_kernel<<<1, 256, 0, s>>>(nb, P.gvec.as<float>() + sp.goff, P.sinv.as<double>() + id);
            IBP_CHECK_LAUNCH();
            P.shapes.push_back(sp);
        }
        assign[b] = id;
        pb_shape.push_back(id);
        pb_first.push_back(mb_first[b]);
        pb_psi.push_back(mb_unk[b]);
        pb_n.push_back(nb);
        for (int i = 0; i < nb; ++i) covered[mb_first[b] + i] = 1;
        covered[mb_unk[b]] = 1;
    }
    P.assign = assign;
    P.prep_version = bd.version;
    P.prep_cls = cls_key(c);
    if (pb_shape.empty()) {
        P.prep_valid = true;   // the structure is known to leave every body unpreconditioned
        queue_moments(c);
        return false;
    }
    std::vector<int> plain;
    for (int u = 0; u < bd.nk; ++u)
        if (!covered[u]) plain.push_back(u);
    std::vector<long long> shape_off(P.shapes.size()), shape_goff(P.shapes.size());
    for (size_t q = 0; q < P.shapes.size(); ++q) {
        shape_off[q] = P.shapes[q].off;
        shape_goff[q] = P.shapes[q].goff;
    }
    auto up = [&](DevBuf& dst, const void* src, size_t bytes) {
        dst.ensure(bytes > 0 ? bytes : 4);
        if (bytes) IBP_CUDA(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyHostToDevice, s));
    };
    up(P.pb_shape, pb_shape.data(), sizeof(int) * pb_shape.size());
    up(P.pb_first, pb_first.data(), sizeof(int) * pb_first.size());
    up(P.pb_psi, pb_psi.data(), sizeof(int) * pb_psi.size());
    up(P.pb_n, pb_n.data(), sizeof(int) * pb_n.size());
    up(P.plain, plain.data(), sizeof(int) * plain.size());
    up(P.shape_off, shape_off.data(), sizeof(long long) * shape_off.size());
    up(P.shape_goff, shape_goff.data(), sizeof(long long) * shape_goff.size());
    IBP_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    P.npb = (int)pb_shape.size();
    P.nplain = (int)plain.size();
    int maxn = 0;
    for (int v : pb_n) maxn = std::max(maxn, v);
    P.chunks = div_up(maxn, kRowsPerBlock);
    P.maxn = maxn;
    P.prep_valid = true;
    queue_moments(c);
    return true;
}

void precond_apply(ibpme_ctx* c, int R, const double* u, long long ustride, const int* jdev, int nk, double* out,
                   bool dir) {
    const Precond& P = c->pre;
    const int blocks = P.npb * P.chunks + div_up(P.nplain > 0 ? P.nplain : 1, kApplyThreads);
    const size_t smem = sizeof(float2) * (size_t)std::max(1, P.maxn);
    static bool attr = false;
    if (!attr) {
        IBP_CUDA(cudaFuncSetAttribute(precond_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(float2) * kPrecondMaxBeads)));
        attr = true;
    }
    precond_apply_kernel<<<dim3(blocks, R), kApplyThreads, smem, c->stream>>>(
        dir, P.npb, P.chunks, nk, ustride, jdev, P.pb_shape.as<int>(), P.pb_first.as<int>(), P.pb_psi.as<int>(),
        P.pb_n.as<int>(), P.shape_off.as<long long>(), P.shape_goff.as<long long>(), P.minv.as<float>(),
        P.gvec.as<float>(),
        P.sinv.as<double>(), P.nplain, P.plain.as<int>(), u, out);
    IBP_CHECK_LAUNCH();
}

}  // namespace ibp
