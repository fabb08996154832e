// krylov.cu -- the induced-charge solve of Sec. III.B (Eq. saddle) by
// restarted GMRES(m) with every vector and scalar on the device.
//
// Unknowns.  Single-bead bodies (ions) have q = Q fixed, so the saddle system
// reduces exactly to the beads of multi-bead bodies ("free" beads) and their
// body potentials: with q_I the ion charges,
//   -M_FF q_F + Sigma_F^T (Psi - Psi_0) = -r.E0 + M_FI q_I,    Sigma_F q_F = Q_F.
// The ion rows of the full system then hold exactly, and the ions'
// Psi - Psi_0 = (M q)_ion - r.E0 follow from the final evaluation.
//
// Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation (CGS2),
// the Hessenberg least-squares problem is kept triangular by Givens rotations
// (Saad & Schultz), and each restart cycle recomputes the residual.  In mixed
// precision the cycles run on the FP32-mesh operator inside an iterative
// refinement whose residual b - A x always uses the FP64 operator; in FP64 the
// same loop is plain restarted GMRES.  Several right-hand sides (field
// directions) iterate in lockstep and share every PME evaluation.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace ibp {

struct Krylov {
    int nk = 0, R = 0, m = 0, nblk = 0;
    DevBuf V, H, cs, sn, g, y, w, x, d, r, rc, part, scal, active, qop, psi, psi_tot, qtot, Ax, norms, jdev;
    // one captured Arnoldi iteration per mesh precision, replayed for every j
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<long long> sig[2];
    long long nodes[2] = {0, 0};   // library kernels captured in each graph (counted per replay)
    ~Krylov() {
        for (auto& e : exec)
            if (e) cudaGraphExecDestroy(e);
    }
};

namespace {

constexpr int kChunk = 2048;   // vector elements per block in the Arnoldi kernels
constexpr int kThreads = 256;

// scal[r][*] slots
enum { S_BETA = 0, S_RES = 1, S_INVH = 2, S_COUNT = 4 };

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;   // valid in warp 0
}

// part[r][blk][i] = sum over this block's chunk of V_i . w, i = 0..j
__global__ void __launch_bounds__(kThreads) dots_kernel(int nk, int m, const int* __restrict__ jdev,
                                                         const double* __restrict__ V, const double* __restrict__ w,
                                                         const int* __restrict__ active, double* __restrict__ part) {
    const int j = *jdev;
    const int r = blockIdx.y;
    if (!active[r]) return;
    const int nblk = gridDim.x;
    const long long t0 = (long long)blockIdx.x * kChunk;
    const long long t1 = min((long long)nk, t0 + kChunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* wr = w + (size_t)r * nk;
    for (int i = warp; i <= j; i += kThreads / 32) {
        const double* vi = V + ((size_t)r * (m + 1) + i) * nk;
        double acc = 0.0;
        for (long long t = t0 + lane; t < t1; t += 32) acc += vi[t] * wr[t];
        acc = warp_sum(acc);
        if (lane == 0) part[((size_t)r * nblk + blockIdx.x) * (m + 2) + i] = acc;
    }
}

// w -= sum_i h_i V_i with h_i = sum over blocks of part; H[:, j] (+)= h.
// In the second pass also the partial sums of |w|^2 go to part[.., m+1].
__global__ void __launch_bounds__(kThreads) update_kernel(int nk, int m, const int* __restrict__ jdev, int pass,
                                                           const double* __restrict__ V, double* __restrict__ w,
                                                           double* __restrict__ H, const int* __restrict__ active,
                                                           double* __restrict__ part) {
    const int j = *jdev;
    const int r = blockIdx.y;
    if (!active[r]) return;
    const int nblk = gridDim.x;
    __shared__ double hc[130];
    __shared__ double sh[32];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double s = 0.0;
        for (int bb = 0; bb < nblk; ++bb) s += part[((size_t)r * nblk + bb) * (m + 2) + i];
        hc[i] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        double* Hc = H + ((size_t)r * m + j) * (m + 1);
        for (int i = threadIdx.x; i <= j; i += blockDim.x) Hc[i] = (pass == 0 ? 0.0 : Hc[i]) + hc[i];
    }
    const long long t0 = (long long)blockIdx.x * kChunk;
    const long long t1 = min((long long)nk, t0 + kChunk);
    double* wr = w + (size_t)r * nk;
    const double* Vr = V + (size_t)r * (m + 1) * nk;
    double acc = 0.0;
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        double v = wr[t];
        for (int i = 0; i <= j; ++i) v -= hc[i] * Vr[(size_t)i * nk + t];
        wr[t] = v;
        acc += v * v;
    }
    __syncthreads();   // part[] slots 0..j are read above by every block before any block writes slot m+1
    if (pass == 1) {
        const double s = block_sum(acc, sh);
        if (threadIdx.x == 0) part[((size_t)r * nblk + blockIdx.x) * (m + 2) + m + 1] = s;
    }
}

// h_{j+1,j} = |w|; Givens rotations on column j; g update; residual estimate |g_{j+1}|.
// Givens rotations of column j of H and the residual estimate; shared by the
// multi-block and the single-block Arnoldi paths.
__device__ void givens_column(int m, int j, int r, double h, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, double* __restrict__ scal) {
    double* Hc = H + ((size_t)r * m + j) * (m + 1);
    double* c = cs + (size_t)r * m;
    double* sg = sn + (size_t)r * m;
    double* gr = g + (size_t)r * (m + 1);
    Hc[j + 1] = h;
    for (int i = 0; i < j; ++i) {
        const double t = c[i] * Hc[i] + sg[i] * Hc[i + 1];
        Hc[i + 1] = -sg[i] * Hc[i] + c[i] * Hc[i + 1];
        Hc[i] = t;
    }
    const double den = hypot(Hc[j], Hc[j + 1]);
    if (den > 0.0) {
        c[j] = Hc[j] / den;
        sg[j] = Hc[j + 1] / den;
    } else {
        c[j] = 1.0;
        sg[j] = 0.0;
    }
    Hc[j] = den;
    Hc[j + 1] = 0.0;
    gr[j + 1] = -sg[j] * gr[j];
    gr[j] = c[j] * gr[j];
    double* sc = scal + (size_t)r * S_COUNT;
    sc[S_RES] = fabs(gr[j + 1]);
    // happy breakdown: the Krylov space is invariant, the estimate above is exact (0)
    sc[S_INVH] = (h > 1e-300 && h > 1e-14 * den) ? 1.0 / h : 0.0;
}

__global__ void finish_kernel(int m, const int* __restrict__ jdev, int nblk, const double* __restrict__ part,
                              double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ scal, const int* __restrict__ active) {
    const int j = *jdev;
    const int r = blockIdx.x;
    const int lane = threadIdx.x;
    if (!active[r]) return;
    double s = 0.0;
    for (int bb = lane; bb < nblk; bb += 32) s += part[((size_t)r * nblk + bb) * (m + 2) + m + 1];
    s = warp_sum(s);
    if (lane != 0) return;
    givens_column(m, j, r, sqrt(s), H, cs, sn, g, scal);
}

__global__ void normalize_kernel(int nk, int m, const int* __restrict__ jdev, int R, const double* __restrict__ w,
                                 const double* __restrict__ scal, const int* __restrict__ active,
                                 double* __restrict__ V) {
    const int j = *jdev;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk);
    const long long e = t - (long long)r * nk;
    if (!active[r]) return;
    V[((size_t)r * (m + 1) + j + 1) * nk + e] = w[t] * scal[(size_t)r * S_COUNT + S_INVH];
}

__global__ void advance_kernel(int* __restrict__ jdev) { *jdev += 1; }

// One Arnoldi step (CGS2 + Givens + normalisation) by a single block per
// right-hand side, for Krylov vectors short enough that one block streams them
// faster than a chain of six grid-wide launches.  Ends by advancing j.
constexpr int kSmallThreads = 1024;
constexpr int kSmallMaxNk = 32 * kSmallThreads;

__global__ void __launch_bounds__(kSmallThreads)
arnoldi_small_kernel(int nk, int m, int* __restrict__ jdev, const double* __restrict__ V, double* __restrict__ w,
                     double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                     double* __restrict__ scal, const int* __restrict__ active, double* __restrict__ Vout) {
    __shared__ double hc[130];
    __shared__ double sh[32];
    __shared__ double inv_h;
    const int j = *jdev;
    const int r = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const bool act = active[r] != 0;
    double* wr = w + (size_t)r * nk;
    const double* Vr = V + (size_t)r * (m + 1) * nk;
    double* Hc = H + ((size_t)r * m + j) * (m + 1);
    if (act) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = warp; i <= j; i += nwarp) {
                const double* vi = Vr + (size_t)i * nk;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;   // independent chains for ILP
                int t = lane;
                for (; t + 96 < nk; t += 128) {
                    a0 += vi[t] * wr[t];
                    a1 += vi[t + 32] * wr[t + 32];
                    a2 += vi[t + 64] * wr[t + 64];
                    a3 += vi[t + 96] * wr[t + 96];
                }
                for (; t < nk; t += 32) a0 += vi[t] * wr[t];
                const double acc = warp_sum((a0 + a1) + (a2 + a3));
                if (lane == 0) hc[i] = acc;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < nk; t += blockDim.x) {
                double v0 = wr[t], v1 = 0.0, v2 = 0.0, v3 = 0.0;
                int i = 0;
                for (; i + 3 <= j; i += 4) {
                    v0 -= hc[i] * Vr[(size_t)i * nk + t];
                    v1 -= hc[i + 1] * Vr[(size_t)(i + 1) * nk + t];
                    v2 -= hc[i + 2] * Vr[(size_t)(i + 2) * nk + t];
                    v3 -= hc[i + 3] * Vr[(size_t)(i + 3) * nk + t];
                }
                for (; i <= j; ++i) v0 -= hc[i] * Vr[(size_t)i * nk + t];
                wr[t] = (v0 + v1) + (v2 + v3);
            }
            if (threadIdx.x <= j) Hc[threadIdx.x] = (pass == 0 ? 0.0 : Hc[threadIdx.x]) + hc[threadIdx.x];
            __syncthreads();
        }
        double acc = 0.0;
        for (int t = threadIdx.x; t < nk; t += blockDim.x) acc += wr[t] * wr[t];
        const double nrm2 = block_sum(acc, sh);
        if (threadIdx.x == 0) {
            givens_column(m, j, r, sqrt(nrm2), H, cs, sn, g, scal);
            inv_h = scal[(size_t)r * S_COUNT + S_INVH];
        }
        __syncthreads();
        double* vn = Vout + ((size_t)r * (m + 1) + j + 1) * nk;
        for (int t = threadIdx.x; t < nk; t += blockDim.x) vn[t] = wr[t] * inv_h;
    }
    // with one block, every thread has read j by now: advance it here (with several
    // right-hand sides a separate launch advances it, after all blocks are done)
    __syncthreads();
    if (gridDim.x == 1 && threadIdx.x == 0) *jdev = j + 1;
}

// Back substitution H(0:k,0:k) y = g(0:k) per right-hand side.
__global__ void trisolve_kernel(int m, int k, const double* __restrict__ H, const double* __restrict__ g,
                                const int* __restrict__ active, double* __restrict__ y) {
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    double* yr = y + (size_t)r * m;
    if (!active[r]) {
        for (int i = 0; i < k; ++i) yr[i] = 0.0;
        return;
    }
    for (int i = k - 1; i >= 0; --i) {
        double s = g[(size_t)r * (m + 1) + i];
        for (int l = i + 1; l < k; ++l) s -= H[((size_t)r * m + l) * (m + 1) + i] * yr[l];
        const double hii = H[((size_t)r * m + i) * (m + 1) + i];
        yr[i] = hii != 0.0 ? s / hii : 0.0;
    }
}

__global__ void xupdate_kernel(int nk, int m, int k, int R, const double* __restrict__ V, const double* __restrict__ y,
                               double* __restrict__ x) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk);
    const long long e = t - (long long)r * nk;
    double s = x[t];
    for (int i = 0; i < k; ++i) s += y[(size_t)r * m + i] * V[((size_t)r * (m + 1) + i) * nk + e];
    x[t] = s;
}

__global__ void axpby_kernel(long long len, double a, const double* __restrict__ u, double b,
                             const double* __restrict__ v, double* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < len) out[t] = a * u[t] + b * v[t];
}

// norms[r] += sum_t v[r][t]^2
__global__ void norm2_kernel(int nk, const double* __restrict__ v, double* __restrict__ norms) {
    __shared__ double sh[32];
    const int r = blockIdx.y;
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nk; t += (long long)gridDim.x * blockDim.x) {
        const double e = v[(size_t)r * nk + t];
        acc += e * e;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(norms + r, s);
}

// Start of a cycle: beta = |r|, V_0 = r / beta, g = beta e_1 (inactive systems: V_0 = 0).
__global__ void start_kernel(int nk, int m, int R, const double* __restrict__ rr, const double* __restrict__ norms,
                             const int* __restrict__ active, double* __restrict__ V, double* __restrict__ g,
                             double* __restrict__ scal) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)R * (m + 1)) {
        const int r = (int)(t / (m + 1)), i = (int)(t % (m + 1));
        g[t] = (i == 0 && active[r]) ? sqrt(norms[r]) : 0.0;
        if (i == 0) scal[(size_t)r * S_COUNT + S_BETA] = sqrt(norms[r]);
    }
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk);
    const long long e = t - (long long)r * nk;
    const double beta = sqrt(norms[r]);
    V[(size_t)r * (m + 1) * nk + e] = (active[r] && beta > 0.0) ? rr[t] / beta : 0.0;
}

// ---- the reduced saddle operator ----
// u of right-hand side r starts at u + r * ustride (+ j * nk when jdev is given: V_j)
__global__ void scatter_kernel(int nfree, long long ustride, int n, int R, const int* __restrict__ free_idx,
                               const double* __restrict__ u, const int* __restrict__ jdev, int nk,
                               double* __restrict__ qop) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nfree * R) return;
    if (jdev) u += (size_t)(*jdev) * nk;
    const int r = (int)(t / nfree), i = (int)(t % nfree);
    qop[(size_t)r * n + free_idx[i]] = u[(size_t)r * ustride + i];
}

// y_F = -psi_F + Psi'(body); y_B = sum of the body's charges
__global__ void assemble_kernel(int nfree, int nmb, int nk, long long ustride, int n, int R,
                                const int* __restrict__ free_idx, const int* __restrict__ mb_of_free,
                                const int* __restrict__ free_off, const double* __restrict__ psi,
                                const double* __restrict__ u, const int* __restrict__ jdev, double* __restrict__ y) {
    if (jdev) u += (size_t)(*jdev) * nk;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long top = (long long)nfree * R;
    if (t < top) {
        const int r = (int)(t / nfree), i = (int)(t % nfree);
        y[(size_t)r * nk + i] = -psi[(size_t)r * n + free_idx[i]] + u[(size_t)r * ustride + nfree + mb_of_free[i]];
        return;
    }
    // one warp per (rhs, body) for the constraint rows; the warp section starts on a
    // 32-thread boundary so that every logical warp is one hardware warp
    const long long top_pad = (top + 31) / 32 * 32;
    if (t < top_pad) return;
    const long long wt = t - top_pad;
    const long long wid = wt >> 5;
    const int lane = (int)(wt & 31);
    if (wid >= (long long)nmb * R) return;
    const int r = (int)(wid / nmb), b = (int)(wid % nmb);
    double s = 0.0;
    for (int i = free_off[b] + lane; i < free_off[b + 1]; i += 32) s += u[(size_t)r * ustride + i];
    s = warp_sum(s);
    if (lane == 0) y[(size_t)r * nk + nfree + b] = s;
}

// |b_full|^2 = sum_all beads (r.E0)^2 + sum_bodies Q^2 (Eq. saddle right-hand side)
__global__ void bfull_kernel(int n, int nb, int R, const double* __restrict__ rel, const double* __restrict__ E0,
                             const double* __restrict__ Q, double* __restrict__ norms) {
    __shared__ double sh[32];
    const int r = blockIdx.y;
    const double* e = E0 + 3 * r;
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n + nb;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < n) {
            const double v = rel[3 * t] * e[0] + rel[3 * t + 1] * e[1] + rel[3 * t + 2] * e[2];
            acc += v * v;
        } else {
            const double v = Q[t - n];
            acc += v * v;
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(norms + r, s);
}

// all bead charges of the current iterate: free beads from x, ions fixed at Q
__global__ void compose_kernel(int n, int nk, int R, const int* __restrict__ free_pos,
                               const int* __restrict__ bead_body, const double* __restrict__ Q,
                               const double* __restrict__ x, double* __restrict__ qtot) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int f = free_pos[j];
    qtot[t] = f >= 0 ? x[(size_t)r * nk + f] : Q[bead_body[j]];
}

// Least-squares body potentials for given charges: Psi'_b = mean over the body's
// beads of ((M q)_j - r_j.E0), the value that minimises the bead rows' residual.
__global__ void fit_psi_kernel(int nfree, int nmb, int nk, int n, int R, const int* __restrict__ free_idx,
                               const int* __restrict__ free_off, const double* __restrict__ rel,
                               const double* __restrict__ E0, const double* __restrict__ psi,
                               double* __restrict__ x) {
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)nmb * R) return;
    const int r = (int)(wid / nmb), b = (int)(wid % nmb);
    const double* e = E0 + 3 * r;
    double sm = 0.0;
    for (int i = free_off[b] + lane; i < free_off[b + 1]; i += 32) {
        const int j = free_idx[i];
        sm += psi[(size_t)r * n + j] - (rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2]);
    }
    sm = warp_sum(sm);
    if (lane == 0) x[(size_t)r * nk + nfree + b] = sm / (double)(free_off[b + 1] - free_off[b]);
}

// residual of the full saddle system on the free rows (the ion rows hold exactly):
//   r_F = -r.E0 - (-(M q)_F + Psi'_body),   r_B = Q - sum of the body's charges
__global__ void residual_kernel(int nfree, int nmb, int nk, int n, int R, const int* __restrict__ free_idx,
                                const int* __restrict__ mb_of_free, const int* __restrict__ free_off,
                                const int* __restrict__ mb_body, const double* __restrict__ rel,
                                const double* __restrict__ E0, const double* __restrict__ Q,
                                const double* __restrict__ psi, const double* __restrict__ x,
                                double* __restrict__ res) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long top = (long long)nfree * R;
    if (t < top) {
        const int r = (int)(t / nfree), i = (int)(t % nfree);
        const int j = free_idx[i];
        const double* e = E0 + 3 * r;
        const double rE = rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2];
        res[(size_t)r * nk + i] = -rE + psi[(size_t)r * n + j] - x[(size_t)r * nk + nfree + mb_of_free[i]];
        return;
    }
    const long long top_pad = (top + 31) / 32 * 32;   // warp section aligned to hardware warps
    if (t < top_pad) return;
    const long long wt = t - top_pad;
    const long long wid = wt >> 5;
    const int lane = (int)(wt & 31);
    if (wid >= (long long)nmb * R) return;
    const int r = (int)(wid / nmb), b = (int)(wid % nmb);
    double sm = 0.0;
    for (int i = free_off[b] + lane; i < free_off[b + 1]; i += 32) sm += x[(size_t)r * nk + i];
    sm = warp_sum(sm);
    if (lane == 0) res[(size_t)r * nk + nfree + b] = Q[mb_body[b]] - sm;
}

__global__ void guess_kernel(int nfree, int nmb, int nk, int n, int nb, int R, const int* __restrict__ free_idx,
                             const int* __restrict__ mb_body, const double* __restrict__ q_in,
                             const double* __restrict__ psi_in, double* __restrict__ x) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk), i = (int)(t % nk);
    if (i < nfree)
        x[t] = q_in[(size_t)r * n + free_idx[i]];
    else
        x[t] = psi_in ? psi_in[(size_t)r * nb + mb_body[i - nfree]] : 0.0;
}

// q_out (free beads from x, ions = Q); psi_out (multi-bead bodies from x, ions from M q of the
// last full-system evaluation: Psi - Psi_0 = (M q)_ion - r.E0)
__global__ void extract_kernel(int n, int nb, int nfree, int nk, int R, const int* __restrict__ bead_body,
                               const int* __restrict__ off, const int* __restrict__ free_idx,
                               const int* __restrict__ mb_body, const double* __restrict__ x,
                               const double* __restrict__ Q, const double* __restrict__ rel,
                               const double* __restrict__ E0, const double* __restrict__ psi_tot,
                               double* __restrict__ q_out, double* __restrict__ psi_out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)nfree * R) {
        const int r = (int)(t / nfree), i = (int)(t % nfree);
        q_out[(size_t)r * n + free_idx[i]] = x[(size_t)r * nk + i];
        if (psi_out && i < nk - nfree) psi_out[(size_t)r * nb + mb_body[i]] = x[(size_t)r * nk + nfree + i];
    }
    if (t < (long long)n * R) {
        const int r = (int)(t / n), j = (int)(t % n);
        const int b = bead_body[j];
        if (off[b + 1] - off[b] == 1) {
            q_out[t] = Q[b];
            if (psi_out) {
                const double* e = E0 + 3 * r;
                psi_out[(size_t)r * nb + b] =
                    psi_tot[t] - (rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2]);
            }
        }
    }
}

inline int blocks_for(long long work, int threads = 256) { return div_up(work > 0 ? work : 1, threads); }

struct Solver {
    ibpme_ctx* c;
    Krylov* k;
    const SolveArgs& a;
    int n, R, nk, nfree, nmb, nb, m;
    int iters = 0, matvec64 = 0;
    std::vector<double> bnorm;   // |b_full| per rhs

    Solver(ibpme_ctx* c_, const SolveArgs& a_) : c(c_), k(c_->kry), a(a_) {
        n = a.n;
        R = a.nrhs;
        nfree = c->bodies.nfree;
        nmb = c->bodies.nmb;
        nb = c->bodies.nb;
        nk = nfree + nmb;
        m = a.restart;
    }

    cudaStream_t s() const { return c->stream; }
    double* D(DevBuf& b) const { return b.as<double>(); }

    void alloc() {
        k->nk = nk;
        k->R = R;
        k->m = m;
        k->nblk = div_up(nk > 0 ? nk : 1, kChunk);
        const size_t v = (size_t)R * (nk > 0 ? nk : 1);
        k->V.ensure(sizeof(double) * v * (m + 1));
        k->H.ensure(sizeof(double) * (size_t)R * m * (m + 1));
        k->cs.ensure(sizeof(double) * (size_t)R * m);
        k->sn.ensure(sizeof(double) * (size_t)R * m);
        k->g.ensure(sizeof(double) * (size_t)R * (m + 1));
        k->y.ensure(sizeof(double) * (size_t)R * m);
        for (DevBuf* b : {&k->w, &k->x, &k->d, &k->r, &k->rc, &k->Ax}) b->ensure(sizeof(double) * v);
        k->part.ensure(sizeof(double) * (size_t)R * k->nblk * (m + 2));
        k->scal.ensure(sizeof(double) * (size_t)R * S_COUNT);
        k->active.ensure(sizeof(int) * R);
        k->norms.ensure(sizeof(double) * R);
        k->jdev.ensure(sizeof(int));
        const size_t full = (size_t)R * n;
        for (DevBuf* b : {&k->qop, &k->psi, &k->psi_tot, &k->qtot}) b->ensure(sizeof(double) * full);
    }

    // y = A(prec) u for the reduced saddle operator; u[r] starts at u + r * ustride
    // (+ j * nk with j read on the device when jdev is given)
    void apply(int prec, const double* u, double* y, long long ustride = -1, const int* jdev = nullptr) {
        const BodyData& bd = c->bodies;
        if (ustride < 0) ustride = nk;
        scatter_kernel<<<blocks_for((long long)nfree * R), 256, 0, s()>>>(nfree, ustride, n, R,
                                                                          bd.free_idx.as<int>(), u, jdev, nk,
                                                                          D(k->qop));
        IBP_CHECK_LAUNCH();
        pme_apply(c, n, a.xw, D(k->qop), R, prec, D(k->psi), nullptr, true);
        const long long work = ((long long)nfree * R + 31) / 32 * 32 + 32LL * nmb * R;
        assemble_kernel<<<blocks_for(work), 256, 0, s()>>>(nfree, nmb, nk, ustride, n, R, bd.free_idx.as<int>(),
                                                           bd.mb_of_free.as<int>(), bd.free_off.as<int>(), D(k->psi),
                                                           u, jdev, y);
        IBP_CHECK_LAUNCH();
    }

    // One Arnoldi iteration entirely on the device: w = A V_j, CGS2 against
    // V_0..V_j, Givens on column j, V_{j+1} = w / h_{j+1,j}, j += 1.
    void iterate(int prec) {
        int* jd = k->jdev.as<int>();
        apply(prec, D(k->V), D(k->w), (long long)(m + 1) * nk, jd);
        ProfScope ps(ST_KRYLOV, s());
        if (nk <= kSmallMaxNk) {
            arnoldi_small_kernel<<<R, kSmallThreads, 0, s()>>>(nk, m, jd, D(k->V), D(k->w), D(k->H), D(k->cs),
                                                               D(k->sn), D(k->g), D(k->scal), k->active.as<int>(),
                                                               D(k->V));
            IBP_CHECK_LAUNCH();
            if (R > 1) {
                advance_kernel<<<1, 1, 0, s()>>>(jd);
                IBP_CHECK_LAUNCH();
            }
            return;
        }
        dim3 ag(k->nblk, R);
        for (int pass = 0; pass < 2; ++pass) {   // CGS2
            dots_kernel<<<ag, kThreads, 0, s()>>>(nk, m, jd, D(k->V), D(k->w), k->active.as<int>(), D(k->part));
            IBP_CHECK_LAUNCH();
            update_kernel<<<ag, kThreads, 0, s()>>>(nk, m, jd, pass, D(k->V), D(k->w), D(k->H),
                                                    k->active.as<int>(), D(k->part));
            IBP_CHECK_LAUNCH();
        }
        finish_kernel<<<R, 32, 0, s()>>>(m, jd, k->nblk, D(k->part), D(k->H), D(k->cs), D(k->sn), D(k->g),
                                         D(k->scal), k->active.as<int>());
        IBP_CHECK_LAUNCH();
        normalize_kernel<<<blocks_for((long long)nk * R), 256, 0, s()>>>(nk, m, jd, R, D(k->w), D(k->scal),
                                                                        k->active.as<int>(), D(k->V));
        IBP_CHECK_LAUNCH();
        advance_kernel<<<1, 1, 0, s()>>>(jd);
        IBP_CHECK_LAUNCH();
    }

    // The captured iteration for this precision, re-captured when any size,
    // buffer or the profiling mask differs from the last capture.
    cudaGraphExec_t iteration_graph(int prec) {
        const Mesh<float>& m32 = c->mesh32;
        const Mesh<double>& m64 = c->mesh64;
        std::vector<long long> sig = {prec, R, nk, n, m, nfree, nmb, (long long)prof_mask(),
                                      (long long)(size_t)k->V.p, (long long)(size_t)k->w.p, (long long)(size_t)k->qop.p,
                                      (long long)(size_t)k->psi.p, (long long)(size_t)k->H.p,
                                      (long long)(size_t)c->psi_r.p, (long long)(size_t)c->psi_k.p,
                                      (long long)(size_t)c->scalars.p, (long long)(size_t)c->near.col.p,
                                      (long long)(size_t)c->near.val.p, (long long)(size_t)c->near.rowptr.p,
                                      (long long)(size_t)a.xw, (long long)(size_t)c->bodies.free_idx.p,
                                      (long long)(size_t)c->bodies.mb_of_free.p,
                                      (long long)(size_t)c->bodies.free_off.p,
                                      (long long)(size_t)(prec == IBPME_MIXED ? m32.grid.p : m64.grid.p),
                                      (long long)(size_t)(prec == IBPME_MIXED ? m32.work.p : m64.work.p)};
        const int gi = prec == IBPME_MIXED ? 1 : 0;
        if (k->exec[gi] && k->sig[gi] == sig) return k->exec[gi];
        if (k->exec[gi]) {
            IBP_CUDA(cudaGraphExecDestroy(k->exec[gi]));
            k->exec[gi] = nullptr;
        }
        // make every lazily created resource exist before capture
        if (prec == IBPME_MIXED) c->mesh32.plans(R, s()); else c->mesh64.plans(R, s());
        prof_capture_begin(gi);
        const long long launches0 = launch_count();
        cudaGraph_t graph = nullptr;
        IBP_CUDA(cudaStreamBeginCapture(s(), cudaStreamCaptureModeThreadLocal));
        try {
            iterate(prec);
        } catch (...) {
            cudaStreamEndCapture(s(), &graph);
            if (graph) cudaGraphDestroy(graph);
            prof_capture_end();
            throw;
        }
        IBP_CUDA(cudaStreamEndCapture(s(), &graph));
        prof_capture_end();
        k->nodes[gi] = launch_count() - launches0;
        count_launch(-k->nodes[gi]);   // capturing is not launching
        cudaGraphExec_t exec = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        IBP_CUDA(e);
        k->exec[gi] = exec;
        k->sig[gi] = sig;
        return exec;
    }

    static bool use_graphs() {
        static const bool off = std::getenv("IBPME_NO_GRAPHS") != nullptr;
        return !off;
    }

    // host copy of R doubles
    std::vector<double> fetch(const double* dev, int count, size_t stride = 1) {
        const size_t elems = (size_t)(count - 1) * stride + 1;
        double* h = static_cast<double*>(pinned_host(c, sizeof(double) * elems));
        IBP_CUDA(cudaMemcpyAsync(h, dev, sizeof(double) * elems, cudaMemcpyDeviceToHost, s()));
        IBP_CUDA(cudaStreamSynchronize(s()));
        std::vector<double> out(count);
        for (int i = 0; i < count; ++i) out[i] = h[i * stride];
        return out;
    }

    std::vector<double> norms(const double* v) {
        IBP_CUDA(cudaMemsetAsync(k->norms.p, 0, sizeof(double) * R, s()));
        dim3 grid(std::min(blocks_for(nk), 152 * 4), R);
        norm2_kernel<<<grid, 256, 0, s()>>>(nk, v, D(k->norms));
        IBP_CHECK_LAUNCH();
        std::vector<double> h = fetch(D(k->norms), R);
        for (double& e : h) e = std::sqrt(e);
        return h;
    }

    void set_active(const std::vector<int>& act) {
        int* h = static_cast<int*>(pinned_host(c, sizeof(int) * R));
        for (int r = 0; r < R; ++r) h[r] = act[r];
        IBP_CUDA(cudaMemcpyAsync(k->active.p, h, sizeof(int) * R, cudaMemcpyHostToDevice, s()));
        IBP_CUDA(cudaStreamSynchronize(s()));   // the pinned scratch is reused right after
    }

    // Residual of the full saddle system at the iterate x with the operator of the
    // given precision: one PME evaluation of all charges (free beads and ions).
    // Leaves r, and psi_tot = M q_total for the ions' potentials.  Returns |r| per rhs.
    // With fit_psi the body potentials of x are first replaced by their
    // least-squares fit to the charges (initial guess).
    std::vector<double> residual(int prec, bool fit_psi = false) {
        const BodyData& bd = c->bodies;
        compose_kernel<<<blocks_for((long long)n * R), 256, 0, s()>>>(n, nk, R, bd.free_pos.as<int>(),
                                                                       bd.bead_body.as<int>(), bd.Q.as<double>(),
                                                                       D(k->x), D(k->qtot));
        IBP_CHECK_LAUNCH();
        pme_apply(c, n, a.xw, D(k->qtot), R, prec, D(k->psi_tot), nullptr, true);
        if (prec == IBPME_FP64) ++matvec64;
        if (fit_psi && nmb > 0) {
            fit_psi_kernel<<<blocks_for(32LL * nmb * R), 256, 0, s()>>>(nfree, nmb, nk, n, R, bd.free_idx.as<int>(),
                                                                        bd.free_off.as<int>(), bd.rel.as<double>(),
                                                                        a.E0, D(k->psi_tot), D(k->x));
            IBP_CHECK_LAUNCH();
        }
        const long long work = ((long long)nfree * R + 31) / 32 * 32 + 32LL * nmb * R;
        residual_kernel<<<blocks_for(work), 256, 0, s()>>>(nfree, nmb, nk, n, R, bd.free_idx.as<int>(),
                                                           bd.mb_of_free.as<int>(), bd.free_off.as<int>(),
                                                           bd.mb_body.as<int>(), bd.rel.as<double>(), a.E0,
                                                           bd.Q.as<double>(), D(k->psi_tot), D(k->x), D(k->r));
        IBP_CHECK_LAUNCH();
        return norms(D(k->r));
    }

    // GMRES on A(prec) d = rhs (d = 0 on entry), cycles of at most m iterations,
    // until |rhs - A d| <= target per rhs or the iteration budget is spent.
    void gmres(int prec, const double* rhs, double* dd, const std::vector<double>& target) {
        const long long len = (long long)nk * R;
        IBP_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * len, s()));
        const double* res_vec = rhs;   // residual the next cycle starts from
        std::vector<double> rn = norms(rhs);
        for (;;) {
            std::vector<int> act(R);
            bool any = false;
            for (int r = 0; r < R; ++r) {
                act[r] = rn[r] > target[r] ? 1 : 0;
                any = any || act[r];
            }
            if (!any || iters >= a.max_iter) return;
            set_active(act);
            // V_0 = res / |res|, g = |res| e_1 (k->norms still holds |res|^2 from norms())
            const long long work = std::max(len, (long long)R * (m + 1));
            start_kernel<<<blocks_for(work), 256, 0, s()>>>(nk, m, R, res_vec, D(k->norms), k->active.as<int>(),
                                                             D(k->V), D(k->g), D(k->scal));
            IBP_CHECK_LAUNCH();
            int kk = 0;
            bool cycle_converged = false;
            IBP_CUDA(cudaMemsetAsync(k->jdev.p, 0, sizeof(int), s()));
            const bool graphs = use_graphs();
            const int gi = prec == IBPME_MIXED ? 1 : 0;
            cudaGraphExec_t exec = graphs ? iteration_graph(prec) : nullptr;
            for (int j = 0; j < m; ++j) {
                if (graphs) {
                    IBP_CUDA(cudaGraphLaunch(exec, s()));
                    count_launch(k->nodes[gi]);
                } else {
                    iterate(prec);
                }
                if (prec == IBPME_FP64) ++matvec64;
                ++iters;
                kk = j + 1;
                std::vector<double> est = fetch(D(k->scal) + S_RES, R, S_COUNT);   // synchronises
                if (graphs) prof_graph_collect(gi);
                bool done = true;
                for (int r = 0; r < R; ++r) {
                    if (!act[r]) continue;
                    if (!std::isfinite(est[r])) fail(IBPME_ERR_NONFINITE, "non-finite Krylov residual estimate");
                    if (!(est[r] <= target[r])) done = false;
                }
                cycle_converged = done;
                if (done || iters >= a.max_iter) break;
            }
            trisolve_kernel<<<R, 32, 0, s()>>>(m, kk, D(k->H), D(k->g), k->active.as<int>(), D(k->y));
            IBP_CHECK_LAUNCH();
            xupdate_kernel<<<blocks_for(len), 256, 0, s()>>>(nk, m, kk, R, D(k->V), D(k->y), dd);
            IBP_CHECK_LAUNCH();
            // the estimate reached the target: the caller's full-system residual decides
            if (cycle_converged || iters >= a.max_iter) return;
            // restart: residual of this operator for the next cycle
            apply(prec, dd, D(k->Ax));
            if (prec == IBPME_FP64) ++matvec64;
            axpby_kernel<<<blocks_for(len), 256, 0, s()>>>(len, 1.0, rhs, -1.0, D(k->Ax), D(k->rc));
            IBP_CHECK_LAUNCH();
            res_vec = D(k->rc);
            rn = norms(res_vec);
        }
    }

    void run(ibpme_solve_stats* st) {
        const BodyData& bd = c->bodies;
        alloc();
        const long long len = (long long)nk * R;
        IBP_CUDA(cudaMemsetAsync(k->qop.p, 0, sizeof(double) * (size_t)R * n, s()));   // ions stay 0
        // |b| of the full system of Eq. saddle, b = [-r.E0 ; Q]
        IBP_CUDA(cudaMemsetAsync(k->norms.p, 0, sizeof(double) * R, s()));
        bfull_kernel<<<dim3(std::min(blocks_for((long long)n + nb), 152 * 4), R), 256, 0, s()>>>(
            n, nb, R, bd.rel.as<double>(), a.E0, bd.Q.as<double>(), D(k->norms));
        IBP_CHECK_LAUNCH();
        bnorm = fetch(D(k->norms), R);
        for (double& e : bnorm) e = std::sqrt(e);
        std::vector<double> tol_abs(R);
        for (int r = 0; r < R; ++r) tol_abs[r] = a.rtol * bnorm[r];

        if (nk > 0 && a.user_guess) {
            guess_kernel<<<blocks_for(len), 256, 0, s()>>>(nfree, nmb, nk, n, nb, R, bd.free_idx.as<int>(),
                                                           bd.mb_body.as<int>(), a.q, nullptr, D(k->x));
            IBP_CHECK_LAUNCH();
        } else if (nk > 0) {
            IBP_CUDA(cudaMemsetAsync(k->x.p, 0, sizeof(double) * len, s()));
        }
        // Iterative refinement on the full system.  Every residual uses the FP64
        // operator; in mixed precision the corrections come from the FP32-mesh
        // operator, whose rounding then scales with the residual, not with the
        // (possibly much larger) potentials of the guess itself.
        const bool mixed = a.prec == IBPME_MIXED;
        std::vector<double> res = residual(IBPME_FP64, true);
        int fell_back = 0;
        if (a.learned && nk > 0) {
            // the learned guess must beat the zero guess, whose residual is |b| up to the ions' share
            bool worse = false;
            for (int r = 0; r < R; ++r)
                if (!(res[r] < bnorm[r])) worse = true;
            if (worse) {
                IBP_CUDA(cudaMemsetAsync(k->x.p, 0, sizeof(double) * len, s()));
                res = residual(IBPME_FP64, true);
                fell_back = 1;
            }
        }
        double init_worst = 0.0;
        for (int r = 0; r < R; ++r) init_worst = std::max(init_worst, bnorm[r] > 0 ? res[r] / bnorm[r] : res[r]);
        const bool verbose = std::getenv("IBPME_VERBOSE") != nullptr;
        if (verbose)
            for (int r = 0; r < R; ++r)
                std::fprintf(stderr, "[ibpme] start rhs %d: nk %d |b| = %.6e |r0|/|b| = %.3e\n", r, nk, bnorm[r],
                             res[r] / bnorm[r]);
        bool res_is_fp64 = true;
        int outer = 0;
        auto converged = [&]() {
            if (!res_is_fp64) return false;
            for (int r = 0; r < R; ++r)
                if (!(res[r] <= tol_abs[r])) return false;
            return true;
        };
        while (nk > 0 && !converged() && iters < a.max_iter && outer < 50) {
            ++outer;
            // FP64: plain restarted GMRES (one cycle per outer step, the same operator).
            // Mixed: the FP32-mesh solve aims below the target so that a single FP64
            // check usually confirms it.
            std::vector<double> tgt(R);
            for (int r = 0; r < R; ++r) tgt[r] = (mixed ? 0.25 : 0.9) * tol_abs[r];
            gmres(a.prec, D(k->r), D(k->d), tgt);
            axpby_kernel<<<blocks_for(len), 256, 0, s()>>>(len, 1.0, D(k->x), 1.0, D(k->d), D(k->x));
            IBP_CHECK_LAUNCH();
            res = residual(IBPME_FP64);
            res_is_fp64 = true;
            if (verbose)
                for (int r = 0; r < R; ++r)
                    std::fprintf(stderr, "[ibpme] outer %d rhs %d: iters %d  |r|/|b| = %.3e (fp64 matvecs %d)\n",
                                 outer, r, iters, res[r] / bnorm[r], matvec64);
        }
        if (!res_is_fp64) res = residual(IBPME_FP64);
        // outputs
        extract_kernel<<<blocks_for((long long)n * R), 256, 0, s()>>>(
            n, nb, nfree, nk, R, bd.bead_body.as<int>(), bd.off.as<int>(), bd.free_idx.as<int>(),
            bd.mb_body.as<int>(), D(k->x), bd.Q.as<double>(), bd.rel.as<double>(), a.E0, D(k->psi_tot), a.q, a.psi);
        IBP_CHECK_LAUNCH();
        double worst = 0.0;
        for (int r = 0; r < R; ++r) {
            const double rel = bnorm[r] > 0 ? res[r] / bnorm[r] : res[r];
            if (!std::isfinite(rel)) {
                worst = rel;
                break;
            }
            worst = std::max(worst, rel);
        }
        st->iters = iters;
        st->outer = outer;
        st->matvecs_fp64 = matvec64;
        st->rel_residual = worst;
        st->fell_back = fell_back;
        st->init_rel_residual = init_worst;
    }
};

}  // namespace

void solve(ibpme_ctx* c, const SolveArgs& a, ibpme_solve_stats* st) {
    if (!c->kry) c->kry = new Krylov();
    // The solve runs on the context's own non-blocking stream (graph capture is not
    // possible on the legacy default stream), ordered after and before the caller's.
    cudaStream_t user = c->stream;
    IBP_CUDA(cudaEventRecord(c->ev_in, user));
    IBP_CUDA(cudaStreamWaitEvent(c->work, c->ev_in, 0));
    c->stream = c->work;
    try {
        near_build(c, a.n, a.xw, false);
        Solver sv(c, a);
        sv.run(st);
    } catch (...) {
        c->stream = user;
        cudaEventRecord(c->ev_out, c->work);
        cudaStreamWaitEvent(user, c->ev_out, 0);
        throw;
    }
    c->stream = user;
    IBP_CUDA(cudaEventRecord(c->ev_out, c->work));
    IBP_CUDA(cudaStreamWaitEvent(user, c->ev_out, 0));
}

void krylov_destroy(ibpme_ctx* c) {
    delete c->kry;
    c->kry = nullptr;
}

}  // namespace ibp
