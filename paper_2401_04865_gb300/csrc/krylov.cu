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
// Systems.  A call solves S = (configurations) x (right-hand sides)
// independent systems in lockstep: system s = cfg * R + r owns the segment
// [uo[cfg], uo[cfg+1]) of row r of every Krylov vector, its own Hessenberg
// matrix, Givens rotations and convergence flag; every PME evaluation serves
// all systems at once (batched mesh channels, batched FFTs).
//
// Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation (CGS2),
// the Hessenberg least-squares problem is kept triangular by Givens rotations
// (Saad & Schultz), and each restart cycle recomputes the residual.  In mixed
// precision the cycles run on the FP32-mesh operator inside an iterative
// refinement whose residual b - A x always uses the FP64 operator; in FP64 the
// same loop is plain restarted GMRES.  One Arnoldi iteration (operator and
// orthogonalisation) is captured once as a CUDA graph and replayed.
#include "common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace ibp {

struct Krylov {
    int nk = 0, R = 0, S = 0, m = 0, nblk = 0;
    DevBuf V, H, cs, sn, g, y, w, x, d, r, rc, part, scal, active, qop, psi, psi_tot, qtot, Ax, norms, jdev;
    DevBuf pu, pt, pz;   // preconditioned operand, cycle update before and after P^{-1}
    DevBuf qc, psif;     // [R][nfree] charges and potentials of the free beads (free-bead operator)
    DevBuf qkeep, dqf;   // charges whose spread the FP64 grid holds [R][n]; their change on the free beads
    // one captured Arnoldi iteration per mesh precision, replayed for every j
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<long long> sig[2];
    long long nodes[2] = {0, 0};   // library kernels captured in each graph (counted per replay)
    // host mirror of the device flags in `active` (uploaded only when they change) and
    // the pinned staging the uploads read; every upload is followed by a synchronising
    // fetch before the staging is written again
    std::vector<int> act_mirror;
    const void* act_buf = nullptr;
    int* act_pin = nullptr;
    int act_cap = 0;
    ~Krylov() {
        for (auto& e : exec)
            if (e) cudaGraphExecDestroy(e);
        if (act_pin) cudaFreeHost(act_pin);
    }
};

namespace {

constexpr int kChunk = 512;   // vector elements per block in the multi-block Arnoldi kernels (FP64-pipe
                              // bound: short chunks spread a 41,152-unknown system over 81 SMs)
constexpr int kThreads = 256;

// scal[s][*] slots
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

// ---- multi-block Arnoldi (one configuration, long vectors) ----

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
    __syncthreads();
    if (pass == 1) {
        const double s = block_sum(acc, sh);
        if (threadIdx.x == 0) part[((size_t)r * nblk + blockIdx.x) * (m + 2) + m + 1] = s;
    }
}

// Givens rotations of column j of system s's H and its residual estimate.
__device__ void givens_column(int m, int j, int s, double h, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, double* __restrict__ scal) {
    double* Hc = H + ((size_t)s * m + j) * (m + 1);
    double* c = cs + (size_t)s * m;
    double* sg = sn + (size_t)s * m;
    double* gr = g + (size_t)s * (m + 1);
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
    double* sc = scal + (size_t)s * S_COUNT;
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

// ---- cluster Arnoldi: one thread-block cluster per system ----
// GB300 executes FP64 at a small fraction of its FP32 rate on every SM, so the
// orthogonalisation of even a few hundred unknowns is bound by the FP64 pipe of
// the SM that runs it.  Each system is therefore spread over a cluster of
// kClusterCtas CTAs (one slice of the unknowns each); partial projections and
// norms are exchanged through distributed shared memory between hardware
// cluster barriers, and every CTA repeats the short serial Givens sweep so that
// no further exchange is needed.
namespace cg = cooperative_groups;
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxNk = 32768;
constexpr size_t kStageSmem = 160 * 1024;   // dynamic shared memory of the staged variant (opt-in)

// STAGE: the CTA's slice of V_0..V_j and of w is copied to shared memory once
// (one round of independent loads), and both CGS passes run from there; used
// when a slice of every Krylov vector fits (chunk <= threads, (m + 2) chunk
// doubles of shared memory).
template <bool STAGE>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
arnoldi_cluster_kernel(int nk, int m, int R, int chunk_max, const int* __restrict__ uo,
                       const int* __restrict__ jdev, const double* __restrict__ V, double* __restrict__ w,
                       double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                       double* __restrict__ g, double* __restrict__ scal, const int* __restrict__ active,
                       double* __restrict__ Vout) {
    extern __shared__ double stage_buf[];   // STAGE: [j + 1][chunk_max] slice of V, then [chunk_max] of w
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double part[130];    // this CTA's partial sums: projections, then |w|^2
    __shared__ double hc[130];      // projections of this pass (whole system)
    __shared__ double hcol[130];    // column j of H (both passes), rotated in place
    __shared__ double c_s[130], s_s[130];
    __shared__ double sh[32];
    __shared__ double inv_h;
    const int crank = (int)cl.block_rank();
    const int s = blockIdx.x / kClusterCtas;
    if (active[s] == 0) return;   // uniform over the cluster: no barrier is left waiting
    const int j = *jdev;
    const int r = s % R, cfg = s / R;
    const int base = uo[cfg], len = uo[cfg + 1] - base;
    const int chunk = (len + kClusterCtas - 1) / kClusterCtas;
    const int lo = min(len, crank * chunk), hi = min(len, lo + chunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = kClusterThreads / 32;
    double* wr = w + (size_t)r * nk + base;
    const double* Vr = V + (size_t)r * (m + 1) * nk + base;
    // STAGE: the slice re-based at lo with row stride chunk_max, w after the V rows
    double* vst = stage_buf;
    double* wst = stage_buf + (size_t)(j + 1) * chunk_max;
    const int cnt = hi - lo;
    for (int i = threadIdx.x; i < j; i += kClusterThreads) {
        c_s[i] = cs[(size_t)s * m + i];
        s_s[i] = sn[(size_t)s * m + i];
    }
    if (STAGE) {
        for (int e = threadIdx.x; e < (j + 1) * cnt; e += kClusterThreads) {
            const int i = e / cnt, t = e - i * cnt;
            vst[(size_t)i * chunk_max + t] = Vr[(size_t)i * nk + lo + t];
        }
        if (threadIdx.x < cnt) wst[threadIdx.x] = wr[lo + threadIdx.x];
        __syncthreads();
    }
    // element t of this CTA's slice of V_i and of w
    auto vat = [&](int i, int t) -> double {
        return STAGE ? vst[(size_t)i * chunk_max + (t - lo)] : Vr[(size_t)i * nk + t];
    };
    auto wat = [&](int t) -> double { return STAGE ? wst[t - lo] : wr[t]; };
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = warp; i <= j; i += nwarp) {
            double a0 = 0.0, a1 = 0.0;
            int t = lo + lane;
            for (; t + 32 < hi; t += 64) {
                a0 += vat(i, t) * wat(t);
                a1 += vat(i, t + 32) * wat(t + 32);
            }
            if (t < hi) a0 += vat(i, t) * wat(t);
            const double acc = warp_sum(a0 + a1);
            if (lane == 0) part[i] = acc;
        }
        cl.sync();
        if (threadIdx.x <= j) {
            double h = 0.0;
            for (int c = 0; c < kClusterCtas; ++c) h += *cl.map_shared_rank(&part[threadIdx.x], c);
            hc[threadIdx.x] = h;
            hcol[threadIdx.x] = (pass == 0 ? 0.0 : hcol[threadIdx.x]) + h;
        }
        cl.sync();   // every CTA has read the partials (and sees hc) before part is reused
        for (int t = lo + threadIdx.x; t < hi; t += kClusterThreads) {
            double v0 = wat(t), v1 = 0.0;
            int i = 0;
            for (; i + 1 <= j; i += 2) {
                v0 -= hc[i] * vat(i, t);
                v1 -= hc[i + 1] * vat(i + 1, t);
            }
            if (i <= j) v0 -= hc[i] * vat(i, t);
            if (STAGE)
                wst[t - lo] = v0 + v1;
            else
                wr[t] = v0 + v1;
        }
        __syncthreads();
    }
    double acc = 0.0;
    for (int t = lo + threadIdx.x; t < hi; t += kClusterThreads) acc += wat(t) * wat(t);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[0] = acc;
    cl.sync();
    if (threadIdx.x == 0) {
        double nrm2 = 0.0;
        for (int c = 0; c < kClusterCtas; ++c) nrm2 += *cl.map_shared_rank(&part[0], c);
        // Givens: apply rotations 0..j-1 to column j, then make the new one (as givens_column);
        // every CTA computes the same values, CTA 0 stores them
        const double h = sqrt(nrm2);
        hcol[j + 1] = h;
        for (int i = 0; i < j; ++i) {
            const double t = c_s[i] * hcol[i] + s_s[i] * hcol[i + 1];
            hcol[i + 1] = -s_s[i] * hcol[i] + c_s[i] * hcol[i + 1];
            hcol[i] = t;
        }
        const double den = hypot(hcol[j], hcol[j + 1]);
        double cj = 1.0, sj = 0.0;
        if (den > 0.0) {
            cj = hcol[j] / den;
            sj = hcol[j + 1] / den;
        }
        hcol[j] = den;
        hcol[j + 1] = 0.0;
        // happy breakdown: the Krylov space is invariant, the estimate is exact (0)
        const double ih = (h > 1e-300 && h > 1e-14 * den) ? 1.0 / h : 0.0;
        inv_h = ih;
        if (crank == 0) {
            cs[(size_t)s * m + j] = cj;
            sn[(size_t)s * m + j] = sj;
            double* gr = g + (size_t)s * (m + 1);
            const double gj = gr[j];
            gr[j + 1] = -sj * gj;
            gr[j] = cj * gj;
            double* sc = scal + (size_t)s * S_COUNT;
            sc[S_RES] = fabs(sj * gj);
            sc[S_INVH] = ih;
        }
    }
    cl.sync();   // no CTA leaves while another may still read its partial norm
    if (crank == 0) {
        double* Hc = H + ((size_t)s * m + j) * (m + 1);
        for (int i = threadIdx.x; i <= j + 1; i += kClusterThreads) Hc[i] = hcol[i];
    }
    double* vn = Vout + ((size_t)r * (m + 1) + j + 1) * nk + base;
    for (int t = lo + threadIdx.x; t < hi; t += kClusterThreads) vn[t] = wat(t) * inv_h;
}

// Back substitution H(0:k,0:k) y = g(0:k) per system.
__global__ void trisolve_kernel(int m, int k, const double* __restrict__ H, const double* __restrict__ g,
                                const int* __restrict__ active, double* __restrict__ y) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    double* ys = y + (size_t)s * m;
    if (!active[s]) {
        for (int i = 0; i < k; ++i) ys[i] = 0.0;
        return;
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = g[(size_t)s * (m + 1) + i];
        for (int l = i + 1; l < k; ++l) v -= H[((size_t)s * m + l) * (m + 1) + i] * ys[l];
        const double hii = H[((size_t)s * m + i) * (m + 1) + i];
        ys[i] = hii != 0.0 ? v / hii : 0.0;
    }
}

// x[r][t] += sum_i y[s][i] V_i[r][t], s the system of unknown t in row r
__global__ void xupdate_kernel(int nk, int m, int k, int R, const int* __restrict__ unk_cfg,
                               const double* __restrict__ V, const double* __restrict__ y, double* __restrict__ x) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk);
    const long long e = t - (long long)r * nk;
    const int s = unk_cfg[e] * R + r;
    double v = x[t];
    for (int i = 0; i < k; ++i) v += y[(size_t)s * m + i] * V[((size_t)r * (m + 1) + i) * nk + e];
    x[t] = v;
}

__global__ void axpby_kernel(long long len, double a, const double* __restrict__ u, double b,
                             const double* __restrict__ v, double* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < len) out[t] = a * u[t] + b * v[t];
}

// norms[s] += sum over system s's segment of v^2  (grid: chunks x S)
__global__ void norm2_kernel(int nk, int R, const int* __restrict__ uo, const double* __restrict__ v,
                             double* __restrict__ norms) {
    __shared__ double sh[32];
    const int s = blockIdx.y;
    const int r = s % R, cfg = s / R;
    const int b0 = uo[cfg], b1 = uo[cfg + 1];
    double acc = 0.0;
    for (long long t = b0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b1;
         t += (long long)gridDim.x * blockDim.x) {
        const double e = v[(size_t)r * nk + t];
        acc += e * e;
    }
    const double sm = block_sum(acc, sh);
    if (threadIdx.x == 0 && sm != 0.0) atomicAdd(norms + s, sm);
}

// Start of a cycle: V_0 = res / |res| per system, g = |res| e_1 (inactive systems: V_0 = 0).
__global__ void start_kernel(int nk, int m, int R, int S, const int* __restrict__ unk_cfg,
                             const double* __restrict__ rr, const double* __restrict__ norms,
                             const int* __restrict__ active, double* __restrict__ V, double* __restrict__ g,
                             double* __restrict__ scal) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)S * (m + 1)) {
        const int s = (int)(t / (m + 1)), i = (int)(t % (m + 1));
        g[t] = (i == 0 && active[s]) ? sqrt(norms[s]) : 0.0;
        if (i == 0) scal[(size_t)s * S_COUNT + S_BETA] = sqrt(norms[s]);
    }
    if (t >= (long long)nk * R) return;
    const int r = (int)(t / nk);
    const long long e = t - (long long)r * nk;
    const int s = unk_cfg[e] * R + r;
    const double beta = sqrt(norms[s]);
    V[(size_t)r * (m + 1) * nk + e] = (active[s] && beta > 0.0) ? rr[t] / beta : 0.0;
}

// ---- the reduced saddle operator ----
// u of row r starts at u + r * ustride (+ j * nk when jdev is given: V_j)
__global__ void scatter_kernel(int nfree, long long ustride, int n, int R, const int* __restrict__ free_idx,
                               const int* __restrict__ free_unk, const double* __restrict__ u,
                               const int* __restrict__ jdev, int nk, double* __restrict__ qop) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nfree * R) return;
    if (jdev) u += (size_t)(*jdev) * nk;
    const int r = (int)(t / nfree), i = (int)(t % nfree);
    qop[(size_t)r * n + free_idx[i]] = u[(size_t)r * ustride + free_unk[i]];
}

// Free-bead charges of u in list order: qc[r][i] = u[r][free_unk[i]].
__global__ void gather_free_kernel(int nfree, long long ustride, int R, const int* __restrict__ free_unk,
                                   const double* __restrict__ u, const int* __restrict__ jdev, int nk,
                                   double* __restrict__ qc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nfree * R) return;
    if (jdev) u += (size_t)(*jdev) * nk;
    const int r = (int)(t / nfree), i = (int)(t % nfree);
    qc[t] = u[(size_t)r * ustride + free_unk[i]];
}

// y_bead = -psi_bead + Psi'(body); y_body = sum of the body's charges.
// Blocks [0, bead_blocks) take the bead rows; each later block sums the
// charges of one (right-hand side, multi-bead body) pair, so that a body of
// hundreds of beads is reduced by a whole block rather than a serial warp.
// psi holds [R][n] bead potentials (list == false) or [R][nfree] free-bead
// potentials in list order (list == true).
__global__ void assemble_kernel(int nfree, int nmb, int nk, long long ustride, int n, int R, int bead_blocks,
                                const int* __restrict__ free_idx, const int* __restrict__ free_unk,
                                const int* __restrict__ bead_body, const int* __restrict__ body_unk,
                                const int* __restrict__ mb_unk, const int* __restrict__ mb_first,
                                const int* __restrict__ mb_cnt, const double* __restrict__ psi, bool list,
                                bool dir, const double* __restrict__ u, const int* __restrict__ jdev,
                                double* __restrict__ y) {
    __shared__ double sh[32];
    if (jdev) u += (size_t)(*jdev) * nk;
    if ((int)blockIdx.x < bead_blocks) {
        const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (t >= (long long)nfree * R) return;
        const int r = (int)(t / nfree), i = (int)(t % nfree);
        const int j = free_idx[i];
        const double p = list ? psi[t] : psi[(size_t)r * n + j];
        y[(size_t)r * nk + free_unk[i]] = -p + (dir ? 0.0 : u[(size_t)r * ustride + body_unk[bead_body[j]]]);
        return;
    }
    const int wid = blockIdx.x - bead_blocks;
    if (wid >= nmb * R) return;   // the one block of an empty launch
    const int r = wid / nmb, b = wid % nmb;
    if (dir) {   // prescribed potentials: the body rows are the identity
        if (threadIdx.x == 0) y[(size_t)r * nk + mb_unk[b]] = u[(size_t)r * ustride + mb_unk[b]];
        return;
    }
    double acc = 0.0;
    for (int i = threadIdx.x; i < mb_cnt[b]; i += blockDim.x) acc += u[(size_t)r * ustride + mb_first[b] + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) y[(size_t)r * nk + mb_unk[b]] = acc;
}

// all bead charges of the current iterate: free beads from x, ions fixed at Q
__global__ void compose_kernel(int n, int nk, int R, const int* __restrict__ bead_unk,
                               const int* __restrict__ bead_body, const double* __restrict__ Q,
                               const double* __restrict__ x, double* __restrict__ qtot) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int f = bead_unk[j];
    qtot[t] = f >= 0 ? x[(size_t)r * nk + f] : Q[bead_body[j]];
}

// dqf[r][f] = qtot - qkeep at free bead f (the charges added since the kept FP64
// grid was spread), and qkeep takes qtot there (ion charges do not change in a solve)
__global__ void delta_kernel(int nfree, int n, int R, const int* __restrict__ free_idx,
                             const double* __restrict__ qtot, double* __restrict__ qkeep, double* __restrict__ dqf) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nfree * R) return;
    const int r = (int)(t / nfree), f = (int)(t % nfree);
    const size_t j = (size_t)r * n + free_idx[f];
    dqf[t] = qtot[j] - qkeep[j];
    qkeep[j] = qtot[j];
}

// Least-squares body potentials for given charges: Psi'_b = mean over the body's
// beads of ((M q)_j - r_j.E0), the value that minimises the bead rows' residual.
__global__ void fit_psi_kernel(int nmb, int nk, int n, int R, const int* __restrict__ mb_body,
                               const int* __restrict__ mb_unk, const int* __restrict__ off,
                               const double* __restrict__ rel, const double* __restrict__ E0,
                               const double* __restrict__ psi, double* __restrict__ x) {
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)nmb * R) return;
    const int r = (int)(wid / nmb), b = (int)(wid % nmb);
    const int body = mb_body[b];
    const double* e = E0 + 3 * r;
    double sm = 0.0;
    for (int j = off[body] + lane; j < off[body + 1]; j += 32)
        sm += psi[(size_t)r * n + j] - (rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2]);
    sm = warp_sum(sm);
    if (lane == 0) x[(size_t)r * nk + mb_unk[b]] = sm / (double)(off[body + 1] - off[body]);
}

// residual of the full saddle system on the free rows (the ion rows hold exactly):
//   r_bead = -r.E0 - (-(M q)_bead + Psi'_body),   r_body = Q - sum of the body's charges
// (block roles as in assemble_kernel)
__global__ void residual_kernel(int nfree, int nmb, int nk, int n, int R, int bead_blocks,
                                const int* __restrict__ free_idx, const int* __restrict__ free_unk,
                                const int* __restrict__ bead_body, const int* __restrict__ body_unk,
                                const int* __restrict__ mb_body, const int* __restrict__ mb_unk,
                                const int* __restrict__ mb_first, const int* __restrict__ mb_cnt,
                                const double* __restrict__ rel, const double* __restrict__ E0,
                                const double* __restrict__ bead_psi, const double* __restrict__ Q,
                                const double* __restrict__ psi, const double* __restrict__ x,
                                double* __restrict__ res) {
    __shared__ double sh[32];
    const bool dir = bead_psi != nullptr;
    if ((int)blockIdx.x < bead_blocks) {
        const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (t >= (long long)nfree * R) return;
        const int r = (int)(t / nfree), i = (int)(t % nfree);
        const int j = free_idx[i];
        if (dir) {   // M q = bead_psi: r_bead = -bead_psi + (M q)_bead
            res[(size_t)r * nk + free_unk[i]] = -bead_psi[(size_t)r * n + j] + psi[(size_t)r * n + j];
            return;
        }
        const double* e = E0 + 3 * r;
        const double rE = rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2];
        res[(size_t)r * nk + free_unk[i]] = -rE + psi[(size_t)r * n + j] - x[(size_t)r * nk + body_unk[bead_body[j]]];
        return;
    }
    const int wid = blockIdx.x - bead_blocks;
    if (wid >= nmb * R) return;   // the one block of an empty launch
    const int r = wid / nmb, b = wid % nmb;
    if (dir) {
        if (threadIdx.x == 0) res[(size_t)r * nk + mb_unk[b]] = -x[(size_t)r * nk + mb_unk[b]];
        return;
    }
    double acc = 0.0;
    for (int i = threadIdx.x; i < mb_cnt[b]; i += blockDim.x) acc += x[(size_t)r * nk + mb_first[b] + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) res[(size_t)r * nk + mb_unk[b]] = Q[mb_body[b]] - acc;
}

// |b_s|^2 = sum over the configuration's beads of (r.E0_r)^2 + sum over its bodies of Q^2
// (Eq. saddle right-hand side), grid: chunks x S
// (with bead_psi, the prescribed-potential problem: sum of bead_psi^2 over the beads)
__global__ void bfull_kernel(int R, int n, const int* __restrict__ cfg_beads, const int* __restrict__ cfg_bodies,
                             const double* __restrict__ rel, const double* __restrict__ E0,
                             const double* __restrict__ bead_psi, const double* __restrict__ Q,
                             double* __restrict__ norms) {
    __shared__ double sh[32];
    const int s = blockIdx.y;
    const int r = s % R, cfg = s / R;
    const double* e = E0 + 3 * r;
    const long long nb0 = cfg_beads[cfg], nb1 = cfg_beads[cfg + 1];
    const long long q0 = cfg_bodies[cfg], q1 = cfg_bodies[cfg + 1];
    const long long len = (nb1 - nb0) + (q1 - q0);
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x) {
        if (t < nb1 - nb0) {
            const long long j = nb0 + t;
            const double v = bead_psi ? bead_psi[(size_t)r * n + j]
                                      : rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2];
            acc += v * v;
        } else if (!bead_psi) {
            const double v = Q[q0 + t - (nb1 - nb0)];
            acc += v * v;
        }
    }
    const double sm = block_sum(acc, sh);
    if (threadIdx.x == 0 && sm != 0.0) atomicAdd(norms + s, sm);
}

__global__ void guess_kernel(int nfree, int nk, int n, int R, const int* __restrict__ free_idx,
                             const int* __restrict__ free_unk, const double* __restrict__ q_in,
                             double* __restrict__ x) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nfree * R) return;
    const int r = (int)(t / nfree), i = (int)(t % nfree);
    x[(size_t)r * nk + free_unk[i]] = q_in[(size_t)r * n + free_idx[i]];
}

// q_out (free beads from x, ions = Q); psi_out per body (multi-bead bodies from x, ions from
// M q of the last full-system evaluation: Psi - Psi_0 = (M q)_ion - r.E0)
__global__ void extract_kernel(int n, int nb, int nk, int R, const int* __restrict__ bead_body,
                               const int* __restrict__ off, const int* __restrict__ bead_unk,
                               const int* __restrict__ body_unk, const double* __restrict__ x,
                               const double* __restrict__ Q, const double* __restrict__ rel,
                               const double* __restrict__ E0, const double* __restrict__ psi_tot,
                               double* __restrict__ q_out, double* __restrict__ psi_out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)n * R) {
        const int r = (int)(t / n), j = (int)(t % n);
        const int u = bead_unk[j];
        q_out[t] = u >= 0 ? x[(size_t)r * nk + u] : Q[bead_body[j]];
    }
    if (psi_out && t < (long long)nb * R) {
        const int r = (int)(t / nb), b = (int)(t % nb);
        const int u = body_unk[b];
        if (u >= 0) {
            psi_out[t] = x[(size_t)r * nk + u];
        } else {
            const int j = off[b];
            const double* e = E0 + 3 * r;
            psi_out[t] = psi_tot[(size_t)r * n + j] - (rel[3 * j] * e[0] + rel[3 * j + 1] * e[1] + rel[3 * j + 2] * e[2]);
        }
    }
}

inline int blocks_for(long long work, int threads = 256) { return div_up(work > 0 ? work : 1, threads); }

struct Solver {
    ibpme_ctx* c;
    Krylov* k;
    const SolveArgs& a;
    int n, R, S, ncfg, nk, nfree, nmb, nb, m;
    int iters = 0, matvec64 = 0;
    bool pre_on = false;         // body-block preconditioner active for this solve
    bool use_free = false;       // the Krylov operator evaluates the free beads alone
    bool dir = false;            // prescribed bead potentials (M q = a.bead_psi), not Eq. saddle
    std::vector<double> bnorm;   // |b| per system
    bool want_b = false;         // the next norms() call also fetches |b|
    // The FP64 grid of this solve's last FP64 residual: the double-float transforms
    // leave it intact, so the next FP64 residual spreads only the free beads' change
    // (while no other spread has written the FP64 mesh since: the mesh counts its
    // spreads, and an FP64 Krylov cycle, whose spreads run in graph replays, drops it)
    bool keep = false;
    unsigned long long keep_writes = 0;
    bool ions_stale = false;   // the last FP64 residual gathered the mesh at the free beads only

    Solver(ibpme_ctx* c_, const SolveArgs& a_) : c(c_), k(c_->kry), a(a_) {
        n = a.n;
        R = a.nrhs;
        ncfg = c->bodies.ncfg;
        S = ncfg * R;
        nfree = c->bodies.nfree;
        nmb = c->bodies.nmb;
        nb = c->bodies.nb;
        nk = c->bodies.nk;
        m = a.restart;
        dir = a.bead_psi != nullptr;
    }

    cudaStream_t s() const { return c->stream; }
    double* D(DevBuf& b) const { return b.as<double>(); }
    const int* I(const DevBuf& b) const { return b.as<int>(); }
    bool clustered() const { return ncfg > 1 || nk <= kClusterMaxNk; }

    void alloc() {
        // opt in to the staged Arnoldi's shared memory (on the current device; before any capture)
        IBP_CUDA(cudaFuncSetAttribute(arnoldi_cluster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kStageSmem));
        k->nk = nk;
        k->R = R;
        k->S = S;
        k->m = m;
        k->nblk = div_up(nk > 0 ? nk : 1, kChunk);
        const size_t v = (size_t)R * (nk > 0 ? nk : 1);
        k->V.ensure(sizeof(double) * v * (m + 1));
        k->H.ensure(sizeof(double) * (size_t)S * m * (m + 1));
        k->cs.ensure(sizeof(double) * (size_t)S * m);
        k->sn.ensure(sizeof(double) * (size_t)S * m);
        k->g.ensure(sizeof(double) * (size_t)S * (m + 1));
        k->y.ensure(sizeof(double) * (size_t)S * m);
        for (DevBuf* b : {&k->w, &k->x, &k->d, &k->r, &k->rc, &k->Ax, &k->pu, &k->pt, &k->pz})
            b->ensure(sizeof(double) * v);
        k->part.ensure(sizeof(double) * (size_t)R * k->nblk * (m + 2));
        k->scal.ensure(sizeof(double) * (size_t)S * S_COUNT);
        k->active.ensure(sizeof(int) * S);
        k->norms.ensure(sizeof(double) * 2 * S);   // |v|^2 per system, then |b|^2 per system
        k->jdev.ensure(sizeof(int));
        const size_t full = (size_t)R * n;
        for (DevBuf* b : {&k->qop, &k->psi, &k->psi_tot, &k->qtot, &k->qkeep}) b->ensure(sizeof(double) * full);
        const size_t fr = (size_t)R * (nfree > 0 ? nfree : 1);
        for (DevBuf* b : {&k->qc, &k->psif, &k->dqf}) b->ensure(sizeof(double) * fr);
    }

    // y = A(prec) u for the reduced saddle operator; u[r] starts at u + r * ustride
    // (+ j * nk with j read on the device when jdev is given); with pre, y = A P^{-1} u
    void apply(int prec, const double* u, double* y, long long ustride = -1, const int* jdev = nullptr,
               bool pre = false) {
        const BodyData& bd = c->bodies;
        if (ustride < 0) ustride = nk;
        if (pre && pre_on) {
            precond_apply(c, R, u, ustride, jdev, nk, D(k->pu), dir);
            u = D(k->pu);
            ustride = nk;
            jdev = nullptr;
        }
        const double* psi_op;
        if (use_free) {
            // the Krylov vector's charges sit on the free beads only, and only their
            // potentials enter the reduced operator: evaluate the free beads alone
            gather_free_kernel<<<blocks_for((long long)nfree * R), 256, 0, s()>>>(nfree, ustride, R, I(bd.free_unk),
                                                                                  u, jdev, nk, D(k->qc));
            IBP_CHECK_LAUNCH();
            pme_apply_free(c, D(k->qc), R, prec, D(k->psif), prec == IBPME_MIXED);
            psi_op = D(k->psif);
        } else {
            scatter_kernel<<<blocks_for((long long)nfree * R), 256, 0, s()>>>(nfree, ustride, n, R, I(bd.free_idx),
                                                                              I(bd.free_unk), u, jdev, nk, D(k->qop));
            IBP_CHECK_LAUNCH();
            pme_apply(c, n, a.xw, D(k->qop), R, prec, D(k->psi), nullptr, true, prec == IBPME_MIXED);
            psi_op = D(k->psi);
        }
        const int bb = div_up((long long)nfree * R, 256);
        assemble_kernel<<<std::max(1, bb + nmb * R), 256, 0, s()>>>(nfree, nmb, nk, ustride, n, R, bb, I(bd.free_idx),
                                                           I(bd.free_unk), I(bd.bead_body), I(bd.body_unk),
                                                           I(bd.mb_unk), I(bd.mb_first), I(bd.mb_cnt), psi_op,
                                                           use_free, dir, u, jdev, y);
        IBP_CHECK_LAUNCH();
    }

    // One Arnoldi iteration entirely on the device: w = A V_j, CGS2 against
    // V_0..V_j, Givens on column j, V_{j+1} = w / h_{j+1,j}, j += 1 (every system).
    void iterate(int prec) {
        int* jd = k->jdev.as<int>();
        apply(prec, D(k->V), D(k->w), (long long)(m + 1) * nk, jd, true);
        ProfScope ps(ST_KRYLOV, s());
        if (clustered()) {
            int max_len = 0;
            const std::vector<int>& uo = c->bodies.uo_h;
            for (size_t q = 0; q + 1 < uo.size(); ++q) max_len = std::max(max_len, uo[q + 1] - uo[q]);
            const int chunk = std::max(1, div_up(max_len, kClusterCtas));
            const size_t smem = sizeof(double) * (size_t)(m + 2) * chunk;
            if (chunk <= kClusterThreads && smem <= kStageSmem) {
                arnoldi_cluster_kernel<true><<<S * kClusterCtas, kClusterThreads, smem, s()>>>(
                    nk, m, R, chunk, I(c->bodies.uo), jd, D(k->V), D(k->w), D(k->H), D(k->cs), D(k->sn), D(k->g),
                    D(k->scal), k->active.as<int>(), D(k->V));
            } else {
                arnoldi_cluster_kernel<false><<<S * kClusterCtas, kClusterThreads, 0, s()>>>(
                    nk, m, R, chunk, I(c->bodies.uo), jd, D(k->V), D(k->w), D(k->H), D(k->cs), D(k->sn), D(k->g),
                    D(k->scal), k->active.as<int>(), D(k->V));
            }
            IBP_CHECK_LAUNCH();
            advance_kernel<<<1, 1, 0, s()>>>(jd);
            IBP_CHECK_LAUNCH();
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

    static bool use_graphs() {
        static const bool off = std::getenv("IBPME_NO_GRAPHS") != nullptr;
        return !off;
    }

    // The captured iteration for this precision, re-captured when any size,
    // buffer or the profiling mask differs from the last capture.
    cudaGraphExec_t iteration_graph(int prec) {
        const BodyData& bd = c->bodies;
        const Mesh<float>& m32 = c->mesh32;
        const Mesh<double>& m64 = c->mesh64;
        // make every lazily created resource exist before capture (this may grow the meshes
        // and build the stencil cache of these positions)
        const int ng = mesh_groups(c);   // mesh channel groups: radius classes or configurations
        if (prec == IBPME_MIXED) c->mesh32.plans(R * ng, s()); else c->mesh64.plans(R * ng, s());
        stencil_cache(c, n, a.xw);
        pme_reserve(c, n, R, false);
        auto P = [](const void* p) { return (long long)(size_t)p; };
        std::vector<long long> sig = {prec, R, S, ncfg, nk, n, m, nfree, nmb, (long long)prof_mask(), (long long)dir,
                                      P(k->V.p), P(k->w.p), P(k->qop.p), P(k->psi.p), P(k->H.p), P(k->scal.p),
                                      P(c->psi_r.p), P(c->psi_k.p), P(c->scalars.p), P(c->near.col.p),
                                      P(c->near.val.p), P(c->near.pair32.p), P(c->near.qf.p), P(c->near.qs.p), P(c->near.cell_beads.p), P(c->near.rowptr.p), P(a.xw), P(bd.free_idx.p),
                                      P(bd.free_unk.p), P(bd.bead_body.p), P(bd.body_unk.p), P(bd.mb_unk.p),
                                      P(bd.mb_first.p), P(bd.mb_cnt.p), P(bd.uo.p), P(c->bcfg),
                                      (long long)cls_key(c), P(c->cls.p), P(c->near.self_b.p), P(c->fs.cls_f.p),
                                      P(c->fs.self_f.p),
                                      (long long)c->stencils.valid, P(c->stencils.start.p), P(c->stencils.frac.p), P(c->stencils.frac32.p),
                                      (long long)c->stencils.tiles, (long long)c->stencils.tile_n[0],
                                      (long long)c->stencils.tile_n[1], (long long)c->stencils.tile_n[2],
                                      P(c->stencils.tile_sorted.p), P(c->stencils.tile_key.p), P(c->stencils.w64.p),
                                      (long long)c->near.cb_on, (long long)c->near.cb_ntasks,
                                      P(c->near.cb_flag.p), P(c->near.cb_hi.p), P(c->near.cb_lo.p),
                                      P(c->near.cb_tasks.p), P(c->near.tab32.p), P(c->near.tab_df.p),
                                      (long long)pre_on, (long long)c->pre.npb, (long long)c->pre.nplain,
                                      (long long)c->pre.chunks, P(k->pu.p), P(c->pre.minv.p), P(c->pre.gvec.p),
                                      P(c->pre.sinv.p), P(c->pre.pb_shape.p), P(c->pre.pb_first.p),
                                      P(c->pre.pb_psi.p), P(c->pre.pb_n.p), P(c->pre.plain.p),
                                      P(c->pre.shape_off.p), P(c->pre.shape_goff.p),
                                      P(prec == IBPME_MIXED ? m32.grid.p : m64.grid.p),
                                      P(prec == IBPME_MIXED ? m32.spec.p : m64.spec.p),
                                      P(prec == IBPME_MIXED ? m32.work.p : m64.work.p), P(m64.df_buf.p), P(m64.grid_df.p),
                                      P(m32.green.p), P(m64.green.p), P(m64.green_df.p), P(m64.df_tw[0].p),
                                      P(m64.df_tw[1].p), P(m64.df_tw[2].p)};
        if (use_free) {
            const FreeSet& fs = c->fs;
            const StencilCache& fc = fs.sc;
            for (long long v : {1LL, (long long)fs.nfree, (long long)fs.cb_ntasks, P(fs.xf.p), P(fs.rowptr.p),
                                P(fs.col.p), P(fs.val.p), P(fs.pair32.p), P(fs.qf.p), P(fs.qs.p), P(fs.cb_hi.p),
                                P(fs.cb_lo.p), P(fs.cb_tasks.p), P(fs.psi_r.p), P(fs.psi_k.p), P(fs.qsum.p),
                                (long long)fc.valid, (long long)fc.tiles, (long long)fc.tile_n[0],
                                (long long)fc.tile_n[1], (long long)fc.tile_n[2], P(fc.start.p), P(fc.frac.p),
                                P(fc.frac32.p), P(fc.w64.p), P(fc.tile_sorted.p), P(fc.tile_key.p), P(bd.iota.p),
                                P(bd.free_cfg.p), P(k->qc.p), P(k->psif.p)})
                sig.push_back(v);
        }
        const int gi = prec == IBPME_MIXED ? 1 : 0;
        if (k->exec[gi] && k->sig[gi] == sig) return k->exec[gi];
        if (k->exec[gi]) {
            IBP_CUDA(cudaGraphExecDestroy(k->exec[gi]));
            k->exec[gi] = nullptr;
        }
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

    // host copy of `count` doubles, `stride` apart
    std::vector<double> fetch(const double* dev, int count, size_t stride = 1) {
        const size_t elems = (size_t)(count - 1) * stride + 1;
        double* h = static_cast<double*>(pinned_host(c, sizeof(double) * elems));
        IBP_CUDA(cudaMemcpyAsync(h, dev, sizeof(double) * elems, cudaMemcpyDeviceToHost, s()));
        IBP_CUDA(cudaStreamSynchronize(s()));
        std::vector<double> out(count);
        for (int i = 0; i < count; ++i) out[i] = h[i * stride];
        return out;
    }

    // |v| per system (k->norms keeps the squares)
    std::vector<double> norms(const double* v) {
        IBP_CUDA(cudaMemsetAsync(k->norms.p, 0, sizeof(double) * S, s()));
        const int per = nk / std::max(1, ncfg) + 1;
        const int chunks = std::max(1, std::min(blocks_for(per), 608 / S + 1));
        norm2_kernel<<<dim3(chunks, S), 256, 0, s()>>>(nk, R, I(c->bodies.uo), v, D(k->norms));
        IBP_CHECK_LAUNCH();
        // the first fetch of a solve also brings |b|^2 (second half), saving one synchronisation
        std::vector<double> h = fetch(D(k->norms), want_b ? 2 * S : S);
        for (double& e : h) e = std::sqrt(e);
        if (want_b) {
            bnorm.assign(h.begin() + S, h.end());
            h.resize(S);
            want_b = false;
        }
        return h;
    }

    void set_active(const std::vector<int>& act) {
        if (k->act_buf == k->active.p && k->act_mirror == act) return;   // the device already holds them
        if (k->act_cap < S) {
            if (k->act_pin) IBP_CUDA(cudaFreeHost(k->act_pin));
            k->act_pin = nullptr;
            k->act_cap = 0;
            IBP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&k->act_pin), sizeof(int) * S, cudaHostAllocDefault));
            k->act_cap = S;
        }
        for (int i = 0; i < S; ++i) k->act_pin[i] = act[i];
        IBP_CUDA(cudaMemcpyAsync(k->active.p, k->act_pin, sizeof(int) * S, cudaMemcpyHostToDevice, s()));
        k->act_mirror = act;
        k->act_buf = k->active.p;
    }

    // Residual of the full saddle system at the iterate x with the operator of the
    // given precision: one PME evaluation of all charges (free beads and ions).
    // Leaves r, and psi_tot = M q_total for the ions' potentials.  Returns |r| per system.
    // With fit_psi the body potentials of x are first replaced by their
    // least-squares fit to the charges (initial guess).
    // zero_charges: every bead charge of the current x is zero (x = 0 without ions), so
    // the potentials are exactly zero and no evaluation is needed
    std::vector<double> residual(int prec, bool fit_psi = false, bool zero_charges = false) {
        const BodyData& bd = c->bodies;
        if (zero_charges) {
            IBP_CUDA(cudaMemsetAsync(k->psi_tot.p, 0, sizeof(double) * (size_t)R * n, s()));
            c->grid64_final = false;   // no evaluation: the grid holds other charges
        } else {
            compose_kernel<<<blocks_for((long long)n * R), 256, 0, s()>>>(n, nk, R, I(bd.bead_unk), I(bd.bead_body),
                                                                           bd.Q.as<double>(), D(k->x), D(k->qtot));
            IBP_CHECK_LAUNCH();
            const bool fp64 = prec == IBPME_FP64;
            const bool can_keep = fp64 && use_free && c->mesh64.df && nfree > 0;
            const StencilCache* fsc = can_keep ? free_stencil_cache(c) : nullptr;
            FreeMesh fm{nfree, c->fs.xf.as<double>(), I(bd.free_idx),
                        c->ncls > 1 ? c->fs.cls_f.as<int>() : (ncfg > 1 ? bd.free_cfg.as<int>() : nullptr), fsc,
                        nullptr, nullptr};
            // a residual that may be the last one gathers the mesh field with the potential
            // when the force pass follows (one field, one configuration)
            const bool field = fp64 && a.want_field && R == 1 && ncfg == 1 && !(can_keep && fsc && fit_psi);
            if (field) {
                pme_reserve(c, n, 1, true);
                fm.ek = c->E_k.as<double>();
                fm.er = c->E_r.as<double>();
            }
            if (can_keep && fsc && keep && c->mesh64.writes == keep_writes) {
                delta_kernel<<<blocks_for((long long)nfree * R), 256, 0, s()>>>(nfree, n, R, I(bd.free_idx), D(k->qtot),
                                                                                 D(k->qkeep), D(k->dqf));
                IBP_CHECK_LAUNCH();
                fm.dq = D(k->dqf);
                pme_apply(c, n, a.xw, D(k->qtot), R, prec, D(k->psi_tot), nullptr, true, false, &fm);
                ions_stale = false;
            } else {
                // the initial residual of an FP64 start: a later FP64 residual follows (or
                // is forced), so the mesh potential is gathered at the free beads only
                const bool partial = can_keep && fsc && fit_psi;
                fm.tmp = partial ? D(k->psif) : nullptr;
                pme_apply(c, n, a.xw, D(k->qtot), R, prec, D(k->psi_tot), nullptr, true, false,
                          partial || field ? &fm : nullptr);
                ions_stale = partial;
                keep = can_keep && fsc;
                if (keep)
                    IBP_CUDA(cudaMemcpyAsync(k->qkeep.p, k->qtot.p, sizeof(double) * (size_t)R * n,
                                             cudaMemcpyDeviceToDevice, s()));
            }
            keep_writes = c->mesh64.writes;
            if (prec == IBPME_FP64) ++matvec64;
            c->grid64_final = prec == IBPME_FP64;
        }
        if (fit_psi && nmb > 0 && !dir) {
            fit_psi_kernel<<<blocks_for(32LL * nmb * R), 256, 0, s()>>>(nmb, nk, n, R, I(bd.mb_body), I(bd.mb_unk),
                                                                        I(bd.off), bd.rel.as<double>(), a.E0,
                                                                        D(k->psi_tot), D(k->x));
            IBP_CHECK_LAUNCH();
        }
        const int bb = div_up((long long)nfree * R, 256);
        residual_kernel<<<std::max(1, bb + nmb * R), 256, 0, s()>>>(nfree, nmb, nk, n, R, bb, I(bd.free_idx),
                                                                    I(bd.free_unk),
                                                           I(bd.bead_body), I(bd.body_unk), I(bd.mb_body),
                                                           I(bd.mb_unk), I(bd.mb_first), I(bd.mb_cnt),
                                                           bd.rel.as<double>(), a.E0, a.bead_psi,
                                                           bd.Q.as<double>(), D(k->psi_tot), D(k->x), D(k->r));
        IBP_CHECK_LAUNCH();
        return norms(D(k->r));
    }

    // GMRES on A(prec) d = rhs (d = 0 on entry) for every system, cycles of at most m
    // iterations, until |rhs - A d| <= target per system or the iteration budget is spent.
    // rn0: |rhs| per system, from the norms() call that left |rhs|^2 in k->norms
    void gmres(int prec, const double* rhs, double* dd, const std::vector<double>& target,
               const std::vector<double>& rn0) {
        const long long len = (long long)nk * R;
        // FP64 iterations spread into the FP64 mesh inside graph replays, which the
        // mesh's host-side write count does not see: the kept grid is gone
        if (prec == IBPME_FP64) keep = false;
        IBP_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * len, s()));
        const double* res_vec = rhs;   // residual the next cycle starts from
        std::vector<double> rn = rn0;
        for (;;) {
            std::vector<int> act(S);
            bool any = false;
            for (int i = 0; i < S; ++i) {
                act[i] = rn[i] > target[i] ? 1 : 0;
                any = any || act[i];
            }
            if (!any || iters >= a.max_iter) return;
            set_active(act);
            // V_0 = res / |res|, g = |res| e_1 (k->norms still holds |res|^2 from norms())
            const long long work = std::max(len, (long long)S * (m + 1));
            start_kernel<<<blocks_for(work), 256, 0, s()>>>(nk, m, R, S, I(c->bodies.unk_cfg), res_vec, D(k->norms),
                                                             k->active.as<int>(), D(k->V), D(k->g), D(k->scal));
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
                std::vector<double> est = fetch(D(k->scal) + S_RES, S, S_COUNT);   // synchronises
                if (graphs) prof_graph_collect(gi);
                bool done = true;
                for (int i = 0; i < S; ++i) {
                    if (!act[i]) continue;
                    if (!std::isfinite(est[i])) fail(IBPME_ERR_NONFINITE, "non-finite Krylov residual estimate");
                    if (!(est[i] <= target[i])) done = false;
                }
                cycle_converged = done;
                if (done || iters >= a.max_iter) break;
            }
            trisolve_kernel<<<S, 32, 0, s()>>>(m, kk, D(k->H), D(k->g), k->active.as<int>(), D(k->y));
            IBP_CHECK_LAUNCH();
            if (pre_on) {   // the cycle's correction is P^{-1} (V y)
                IBP_CUDA(cudaMemsetAsync(k->pt.p, 0, sizeof(double) * len, s()));
                xupdate_kernel<<<blocks_for(len), 256, 0, s()>>>(nk, m, kk, R, I(c->bodies.unk_cfg), D(k->V),
                                                                 D(k->y), D(k->pt));
                IBP_CHECK_LAUNCH();
                precond_apply(c, R, D(k->pt), nk, nullptr, nk, D(k->pz), dir);
                axpby_kernel<<<blocks_for(len), 256, 0, s()>>>(len, 1.0, dd, 1.0, D(k->pz), dd);
                IBP_CHECK_LAUNCH();
            } else {
                xupdate_kernel<<<blocks_for(len), 256, 0, s()>>>(nk, m, kk, R, I(c->bodies.unk_cfg), D(k->V),
                                                                 D(k->y), dd);
                IBP_CHECK_LAUNCH();
            }
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
        pre_on = a.precond && nk > 0 && precond_prepare(c);
        use_free = nk > 0 && nfree > 0 && free_prepare(c, a.xw, R);
        const long long len = (long long)nk * R;
        IBP_CUDA(cudaMemsetAsync(k->qop.p, 0, sizeof(double) * (size_t)R * n, s()));   // ions stay 0
        // |b| of the full system of Eq. saddle, b = [-r.E0 ; Q], per system
        IBP_CUDA(cudaMemsetAsync(D(k->norms) + S, 0, sizeof(double) * S, s()));
        const int per = (n + nb) / ncfg + 1;
        bfull_kernel<<<dim3(std::max(1, std::min(blocks_for(per), 608 / S + 1)), S), 256, 0, s()>>>(
            R, n, I(bd.cfg_beads), I(bd.cfg_bodies), bd.rel.as<double>(), a.E0, a.bead_psi, bd.Q.as<double>(),
            D(k->norms) + S);
        IBP_CHECK_LAUNCH();
        want_b = true;   // fetched with the initial residual

        if (nk > 0) IBP_CUDA(cudaMemsetAsync(k->x.p, 0, sizeof(double) * len, s()));
        if (nk > 0 && a.user_guess) {
            guess_kernel<<<blocks_for((long long)nfree * R), 256, 0, s()>>>(nfree, nk, n, R, I(bd.free_idx),
                                                                            I(bd.free_unk), a.q, D(k->x));
            IBP_CHECK_LAUNCH();
        }
        // Iterative refinement on the full system.  Every residual that decides
        // convergence uses the FP64 operator; in mixed precision the corrections come
        // from the FP32-mesh operator, whose rounding then scales with the residual,
        // not with the (possibly much larger) potentials of the guess itself.
        const bool mixed = a.prec == IBPME_MIXED;
        // the zero guess of a system without ions has no charge anywhere: r0 follows from b alone
        const bool zero_start = nk > 0 && !a.user_guess && !a.learned && bd.nmb == bd.nb;
        // Mixed precision at tolerances of 1e-7 and looser: the first residual takes the
        // FP32-mesh operator.  Its rounding enters the correction once and the FP64
        // residual after it still decides convergence, so a step usually needs one FP64
        // evaluation instead of two.  Where that rounding is not small against |b| (many
        // ions around a weakly charged body) the first FP64 check fails; the context then
        // starts the next 32 solves from the FP64 residual.
        bool start32 = mixed && !zero_start && a.rtol >= 1e-7;
        if (start32 && c->start32_skip > 0) {
            --c->start32_skip;
            start32 = false;
        }
        bool check32 = start32;   // the first FP64 check still has to decide on the FP32 start
        const int prec0 = start32 ? IBPME_MIXED : IBPME_FP64;
        std::vector<double> res = residual(prec0, true, zero_start);
        std::vector<double> tol_abs(S);
        for (int i = 0; i < S; ++i) tol_abs[i] = a.rtol * bnorm[i];
        bool res64 = !start32;
        int fell_back = 0;
        if (a.learned && nk > 0) {
            // the learned guess must beat the zero guess, whose residual is |b| up to the ions' share
            bool worse = false;
            for (int i = 0; i < S; ++i)
                if (!(res[i] < bnorm[i])) worse = true;
            if (worse) {
                IBP_CUDA(cudaMemsetAsync(k->x.p, 0, sizeof(double) * len, s()));
                res = residual(prec0, true);
                fell_back = 1;
            }
        }
        auto relres = [&](int i) { return bnorm[i] > 0 ? res[i] / bnorm[i] : res[i]; };
        std::vector<double> init(S);
        for (int i = 0; i < S; ++i) init[i] = relres(i);
        const bool verbose = std::getenv("IBPME_VERBOSE") != nullptr;
        if (verbose)
            for (int i = 0; i < S; ++i)
                std::fprintf(stderr, "[ibpme] start system %d: nk %d |b| = %.6e |r0|/|b| = %.3e\n", i, nk, bnorm[i],
                             relres(i));
        int outer = 0;
        auto converged = [&]() {
            for (int i = 0; i < S; ++i)
                if (!(res[i] <= tol_abs[i])) return false;
            return true;
        };
        while (nk > 0 && iters < a.max_iter && outer < 50) {
            if (converged()) {
                if (res64) break;
                res = residual(IBPME_FP64);   // a guess that looks converged: confirm with FP64
                res64 = true;
                if (check32) {
                    c->start32_skip = converged() ? 0 : 32;
                    check32 = false;
                }
                if (converged()) break;
            }
            ++outer;
            // FP64: plain restarted GMRES (one cycle per outer step, the same operator).
            // Mixed: the FP32-mesh solve aims below the target so that a single FP64
            // check usually confirms it.
            std::vector<double> tgt(S);
            for (int i = 0; i < S; ++i) tgt[i] = (mixed ? 0.25 : 0.9) * tol_abs[i];
            gmres(a.prec, D(k->r), D(k->d), tgt, res);   // res: norms of k->r, the last norms() call
            axpby_kernel<<<blocks_for(len), 256, 0, s()>>>(len, 1.0, D(k->x), 1.0, D(k->d), D(k->x));
            IBP_CHECK_LAUNCH();
            res = residual(IBPME_FP64);
            res64 = true;
            if (check32) {
                c->start32_skip = converged() ? 0 : 32;
                check32 = false;
            }
            if (verbose)
                for (int i = 0; i < S; ++i)
                    std::fprintf(stderr, "[ibpme] outer %d system %d: iters %d  |r|/|b| = %.3e (fp64 matvecs %d)\n",
                                 outer, i, iters, relres(i), matvec64);
        }
        // the reported residual and the ions' potentials come from an FP64 evaluation
        if (!res64 || ions_stale) res = residual(IBPME_FP64);
        // outputs
        extract_kernel<<<blocks_for((long long)std::max(n, nb) * R), 256, 0, s()>>>(
            n, nb, nk, R, I(bd.bead_body), I(bd.off), I(bd.bead_unk), I(bd.body_unk), D(k->x), bd.Q.as<double>(),
            bd.rel.as<double>(), a.E0, D(k->psi_tot), a.q, a.psi);
        IBP_CHECK_LAUNCH();
        // statistics per configuration (worst of its right-hand sides)
        for (int cfg = 0; cfg < ncfg; ++cfg) {
            double worst = 0.0, iw = 0.0;
            for (int r = 0; r < R; ++r) {
                const int i = cfg * R + r;
                const double v = relres(i);
                worst = std::isfinite(v) && std::isfinite(worst) ? std::max(worst, v) : NAN;
                iw = std::max(iw, init[i]);
            }
            ibpme_solve_stats& o = st[cfg];
            o.iters = iters;
            o.outer = outer;
            o.matvecs_fp64 = matvec64;
            o.rel_residual = worst;
            o.fell_back = fell_back;
            o.init_rel_residual = iw;
        }
    }
};

}  // namespace

const double* solve_potentials(ibpme_ctx* c) {
    return c->kry && c->grid64_final ? c->kry->psi_tot.as<double>() : nullptr;
}

void solve(ibpme_ctx* c, const SolveArgs& a, ibpme_solve_stats* st) {
    if (!c->kry) c->kry = new Krylov();
    c->grid64_final = false;
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
