// mesh.cu -- wave-space half of the spectral Ewald sum (Sec. III.D.2 and
// steps 2-6 of Sec. III.D.3): Gaussian spreading onto the grid, forward FFT,
// Green's-function scaling, inverse FFT and trapezoid-rule gather (with the
// gradient for the field).
//
// Spreading and gathering use one warp per bead.  The Gaussian window is
// separable, exp(-2 xi^2 |x_g - x|^2 / eta) = w_x(i) w_y(j) w_z(k), so a warp
// evaluates 3P exponentials and then streams the P^3 products; lane
// (i, row) owns one x offset i of the stencil and walks the (j, k) rows, so
// the addresses of neighbouring lanes are contiguous along x.
#include "common.cuh"
#include "dfloat.cuh"

#include <cuda.h>   // CUtensorMap (tensor maps of the TMA region loads)
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace ibp {

namespace {

constexpr int kWarpsPerBlock = 4;

template <typename T> __device__ __forceinline__ T dexp(T v);
template <> __device__ __forceinline__ float dexp<float>(float v) { return expf(v); }
template <> __device__ __forceinline__ double dexp<double>(double v) { return exp(v); }

// Per-warp stencil set-up: for axis d, node indices (periodic) and window
// weights of the P closest nodes, first node floor(u - P/2) + 1, u = x / h.
template <typename T, bool DIST>
__device__ __forceinline__ void stencil_setup(const MeshGeom& g, const double* __restrict__ xw, int bead, int lane,
                                              T (*sw)[kMaxP], int (*sidx)[kMaxP], T (*sdist)[kMaxP]) {
    const int P = g.P;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double u = xw[3 * bead + d] * g.inv_h[d];
        const double sf = floor(u - 0.5 * P) + 1.0;
        if (lane < P) {
            const T f = (T)(sf - u) + (T)lane;          // (node - x) / h, exact to rounding of T
            sw[d][lane] = dexp<T>(-(T)g.kappa[d] * f * f);
            if (DIST) sdist[d][lane] = f * (T)g.h[d];
            int idx = ((int)sf + lane) % g.N[d];
            if (idx < 0) idx += g.N[d];
            sidx[d][lane] = idx;
        }
    }
    __syncwarp();
}

// Spreading, one bead per WPB warps.  Lane (i, rsub) of warp w of the bead
// owns stencil column i and walks the rows rsub + rows_per (w + WPB t) of the
// P^2 (j, k) rows; NR right-hand sides share the window weights.
template <typename T, int NR, int WPB>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
spread_kernel(int n, const double* __restrict__ xw, const double* __restrict__ q, const int* __restrict__ bead_cfg,
              MeshGeom g, T* __restrict__ grid) {
    __shared__ T s_w[kWarpsPerBlock][3][kMaxP];
    __shared__ int s_idx[kWarpsPerBlock][3][kMaxP];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bead = (blockIdx.x * kWarpsPerBlock + wib) / WPB;
    const int part = wib % WPB;
    if (bead >= n) return;
    stencil_setup<T, false>(g, xw, bead, lane, s_w[wib], s_idx[wib], nullptr);
    const int P = g.P;
    const int rows_per = 32 / P;
    const int i = lane % P, rsub = lane / P;
    if (rsub >= rows_per) return;
    const T wx = s_w[wib][0][i];
    const int ix = s_idx[wib][0][i];
    if (bead_cfg) grid += (size_t)bead_cfg[bead] * NR * g.G;
    T qc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) qc[r] = (T)(g.c * q[(size_t)r * n + bead]) * wx;
    const int P2 = P * P;
    const int step = rows_per * WPB;
    int row = rsub + rows_per * part;
    int k = row / P, j = row - k * P;
    const int nxy = g.N[0] * g.N[1];
    for (; row < P2; row += step) {
        const T wyz = s_w[wib][1][j] * s_w[wib][2][k];
        const int off = s_idx[wib][2][k] * nxy + s_idx[wib][1][j] * g.N[0] + ix;
#pragma unroll
        for (int r = 0; r < NR; ++r) atomicAdd(grid + (size_t)r * g.G + off, qc[r] * wyz);
        j += step;
        while (j >= P) {
            j -= P;
            ++k;
        }
    }
}

// Gather (trapezoid rule, Eq. psi_wave) and, with GRAD, the gradient of the
// window for the field; WPB warps per bead combine their partial sums in
// shared memory.
template <typename T, int NR, int WPB, bool GRAD>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
gather_kernel(int n, const double* __restrict__ xw, const int* __restrict__ bead_cfg, MeshGeom g,
              const T* __restrict__ grid, const float2* __restrict__ gdf, double* __restrict__ psi,
              double* __restrict__ E) {
    __shared__ T s_w[kWarpsPerBlock][3][kMaxP];
    __shared__ T s_d[kWarpsPerBlock][3][kMaxP];
    __shared__ int s_idx[kWarpsPerBlock][3][kMaxP];
    __shared__ double s_part[kWarpsPerBlock][GRAD ? 4 * NR : NR];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bead = (blockIdx.x * kWarpsPerBlock + wib) / WPB;
    const int part = wib % WPB;
    const bool valid = bead < n;   // no early exit: every warp must reach the block barrier below
    if (valid) stencil_setup<T, GRAD>(g, xw, bead, lane, s_w[wib], s_idx[wib], s_d[wib]);
    const int P = g.P;
    const int rows_per = 32 / P;
    const int i = lane % P, rsub = lane / P;
    const bool active = valid && rsub < rows_per;
    T acc[NR], accy[NR], accz[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = accy[r] = accz[r] = (T)0;
    T wx = 0, dx = 0;
    if (active) {
        wx = s_w[wib][0][i];
        if (GRAD) dx = s_d[wib][0][i];
        const int ix = s_idx[wib][0][i];
        if (bead_cfg) {
            grid += (size_t)bead_cfg[bead] * NR * g.G;
            if (gdf) gdf += (size_t)bead_cfg[bead] * NR * g.G;
        }
        const int P2 = P * P;
        const int step = rows_per * WPB;
        int row = rsub + rows_per * part;
        int k = row / P, j = row - k * P;
        const int nxy = g.N[0] * g.N[1];
#pragma unroll 4
        for (; row < P2; row += step) {
            const T wyz = s_w[wib][1][j] * s_w[wib][2][k];
            const int off = s_idx[wib][2][k] * nxy + s_idx[wib][1][j] * g.N[0] + ix;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                T gv;
                if constexpr (sizeof(T) == 8) {
                    if (gdf) {
                        const float2 t = __ldg(gdf + (size_t)r * g.G + off);
                        gv = df_join(df{t.x, t.y});
                    } else {
                        gv = __ldg(grid + (size_t)r * g.G + off);
                    }
                } else {
                    gv = __ldg(grid + (size_t)r * g.G + off);
                }
                const T v = gv * wyz;
                acc[r] += v;
                if (GRAD) {
                    accy[r] += v * s_d[wib][1][j];
                    accz[r] += v * s_d[wib][2][k];
                }
            }
            j += step;
            while (j >= P) {
                j -= P;
                ++k;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double p = warp_sum((double)(wx * acc[r]));
        double ex = 0, ey = 0, ez = 0;
        if (GRAD) {
            ex = warp_sum((double)(wx * dx * acc[r]));
            ey = warp_sum((double)(wx * accy[r]));
            ez = warp_sum((double)(wx * accz[r]));
        }
        if (lane == 0) {
            if (GRAD) {
                s_part[wib][4 * r] = p;
                s_part[wib][4 * r + 1] = ex;
                s_part[wib][4 * r + 2] = ey;
                s_part[wib][4 * r + 3] = ez;
            } else {
                s_part[wib][r] = p;
            }
        }
    }
    if (WPB > 1) __syncthreads();
    if (!valid || part != 0 || lane != 0) return;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double p = 0, ex = 0, ey = 0, ez = 0;
#pragma unroll
        for (int w = 0; w < WPB; ++w) {
            if (GRAD) {
                p += s_part[wib + w][4 * r];
                ex += s_part[wib + w][4 * r + 1];
                ey += s_part[wib + w][4 * r + 2];
                ez += s_part[wib + w][4 * r + 3];
            } else {
                p += s_part[wib + w][r];
            }
        }
        psi[(size_t)r * n + bead] = g.gather * p;
        if (GRAD) {
            double* e = E + ((size_t)r * n + bead) * 3;
            // E = -grad psi; d/dx_alpha of the window gives (4 xi^2/eta)(x_g - x_alpha)
            e[0] = -g.grad * ex;
            e[1] = -g.grad * ey;
            e[2] = -g.grad * ez;
        }
    }
}

// warps per bead: enough warps to fill the GPU at small bead counts
int warps_per_bead(int n) {
    const long long want = 152LL * 48;   // about 48 resident warps per SM
    if ((long long)n * 2 > want) return 1;
    if ((long long)n * 4 > want) return 2;
    return 4;
}

template <typename T, int NR, int WPB>
void launch_spread(int n, const double* xw, const double* q, const int* cfg, const MeshGeom& g, T* grid,
                   cudaStream_t s) {
    const int blocks = div_up((long long)n * WPB, kWarpsPerBlock);
    spread_kernel<T, NR, WPB><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(n, xw, q, cfg, g, grid);
}

template <typename T, int NR>
void launch_spread_w(int n, const double* xw, const double* q, const int* cfg, const MeshGeom& g, T* grid,
                     cudaStream_t s) {
    switch (warps_per_bead(n)) {
        case 1: launch_spread<T, NR, 1>(n, xw, q, cfg, g, grid, s); break;
        case 2: launch_spread<T, NR, 2>(n, xw, q, cfg, g, grid, s); break;
        default: launch_spread<T, NR, 4>(n, xw, q, cfg, g, grid, s); break;
    }
}

template <typename T>
void spread_dispatch(int n, const double* xw, const double* q, int nrhs, const int* cfg, const MeshGeom& g, T* grid,
                     cudaStream_t s) {
    switch (nrhs) {
        case 1: launch_spread_w<T, 1>(n, xw, q, cfg, g, grid, s); break;
        case 2: launch_spread_w<T, 2>(n, xw, q, cfg, g, grid, s); break;
        case 3: launch_spread_w<T, 3>(n, xw, q, cfg, g, grid, s); break;
        case 4: launch_spread_w<T, 4>(n, xw, q, cfg, g, grid, s); break;
        case 5: launch_spread_w<T, 5>(n, xw, q, cfg, g, grid, s); break;
        case 6: launch_spread_w<T, 6>(n, xw, q, cfg, g, grid, s); break;
        case 7: launch_spread_w<T, 7>(n, xw, q, cfg, g, grid, s); break;
        default: launch_spread_w<T, 8>(n, xw, q, cfg, g, grid, s); break;
    }
}

template <typename T, int NR, int WPB, bool GRAD>
void launch_gather(int n, const double* xw, const int* cfg, const MeshGeom& g, const T* grid, const float2* gdf, double* psi,
                   double* E, cudaStream_t s) {
    const int blocks = div_up((long long)n * WPB, kWarpsPerBlock);
    gather_kernel<T, NR, WPB, GRAD><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(n, xw, cfg, g, grid, gdf, psi, E);
}

template <typename T, int NR, bool GRAD>
void launch_gather_w(int n, const double* xw, const int* cfg, const MeshGeom& g, const T* grid, const float2* gdf,
                     double* psi, double* E, cudaStream_t s) {
    switch (warps_per_bead(n)) {
        case 1: launch_gather<T, NR, 1, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 2: launch_gather<T, NR, 2, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        default: launch_gather<T, NR, 4, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
    }
}

template <typename T, bool GRAD>
void gather_dispatch(int n, const double* xw, int nrhs, const int* cfg, const MeshGeom& g, const T* grid,
                     const float2* gdf, double* psi, double* E, cudaStream_t s) {
    switch (nrhs) {
        case 1: launch_gather_w<T, 1, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 2: launch_gather_w<T, 2, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 3: launch_gather_w<T, 3, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 4: launch_gather_w<T, 4, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 5: launch_gather_w<T, 5, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 6: launch_gather_w<T, 6, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        case 7: launch_gather_w<T, 7, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
        default: launch_gather_w<T, 8, GRAD>(n, xw, cfg, g, grid, gdf, psi, E, s); break;
    }
}

// ---------------------------------------------------------------------------
// Pair-lane spreading and gathering with cached stencils.
//
// For a fixed set of positions (a whole Krylov solve) every bead's first
// stencil node and fractional offset are computed once (stencil_cache_kernel).
// A warp sets up the bead's 3P one-dimensional windows once (lane l < P holds
// node l of each axis); its lanes then own (x, y) column pairs (i, j) of the
// stencil, taking their weights and node indices by shuffle, and walk the P
// z-nodes of their column: per z-node one shuffle, one index update and one
// atomic add (spread) or load (gather).  While the beads alone cannot fill the
// GPU, the P^2 columns of a bead are split over several warps.
// ---------------------------------------------------------------------------
constexpr int kPairWarps = 4;   // warps per block

// One thread per (bead, axis, stencil node l < P): the first node of the axis, the
// fractional offset and the FP64 window of node l (GB300 evaluates FP64 exp at a small
// fraction of its FP32 rate, so the windows are spread over the whole GPU).  The
// thread of node 0 writes the axis's start and offsets; axis 0 also the configuration.
__global__ void stencil_cache_kernel(int n, const double* __restrict__ xw, const int* __restrict__ bcfg, MeshGeom g,
                                     int4* __restrict__ start, double4* __restrict__ frac, float4* __restrict__ frac32,
                                     double* __restrict__ w64, float2* __restrict__ wdf, float4* __restrict__ frac_df) {
    // one thread per (bead, axis): the P window weights w_l = exp(-kappa (f + l)^2) by the
    // recurrence w_{l+1} = w_l r_l, r_l = exp(-kappa (2 (f + l) + 1)), r_{l+1} = r_l exp(-2 kappa):
    // two FP64 exponentials per axis instead of P (the relative error grows by about
    // 2^-53 per node)
    const int P = g.P;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3LL * n) return;
    const int b = (int)(t / 3), d = (int)(t - 3LL * b);
    const double u = xw[3 * b + d] * g.inv_h[d];
    const double sf = floor(u - 0.5 * P) + 1.0;
    const double f = sf - u;
    const double kap = g.kappa[d];
    double w = exp(-kap * f * f);
    double r = exp(-kap * (2.0 * f + 1.0));
    const double B = exp(-2.0 * kap);
    double* wo = w64 + ((size_t)b * 3 + d) * P;
    float2* wdo = wdf + ((size_t)b * 3 + d) * P;
    for (int l = 0; l < P; ++l) {
        wo[l] = w;
        const df wd = df_split(w);
        wdo[l] = make_float2(wd.hi, wd.lo);
        w *= r;
        r *= B;
    }
    const df fd = df_split(f);
    reinterpret_cast<float*>(frac_df + 2 * b)[d] = fd.hi;
    reinterpret_cast<float*>(frac_df + 2 * b + 1)[d] = fd.lo;
    int idx = (int)sf % g.N[d];
    if (idx < 0) idx += g.N[d];
    reinterpret_cast<int*>(start + b)[d] = idx;
    reinterpret_cast<double*>(frac + b)[d] = f;
    reinterpret_cast<float*>(frac32 + b)[d] = (float)f;
    if (d == 0) {
        reinterpret_cast<int*>(start + b)[3] = bcfg ? bcfg[b] : 0;
        reinterpret_cast<double*>(frac + b)[3] = 0.0;
        reinterpret_cast<float*>(frac32 + b)[3] = 0.0f;
        reinterpret_cast<float*>(frac_df + 2 * b)[3] = 0.0f;
        reinterpret_cast<float*>(frac_df + 2 * b + 1)[3] = 0.0f;
    }
}

// FP32 kernels take every constant and offset in FP32: GB300 issues FP64
// instructions (conversions included) at a small fraction of the FP32 rate, and
// a handful per bead made the FP64 pipe the busiest unit of the FP32 gather.
struct PairArgs {
    MeshGeom g;
    int wpb;            // warps per bead
    int rounds;         // blocks of 32 (i, j) pairs per warp: wpb * rounds * 32 >= P^2
    const int4* start;
    const double4* frac;
    const float4* frac32;   // the same offsets rounded to FP32
    const double* w64;  // cached FP64 windows [n][3][P] (NULL: evaluate them)
    const float2* wdf;  // the same as hi + lo floats
    const float4* frac_df;   // per bead two float4: the offsets as hi, lo floats
    float hdf[3][2];    // h per axis as hi, lo floats
    float kappa32[3], h32[3], c32, gather32, grad32;   // MeshGeom's constants in FP32
    const float2* gdf;  // FP64 gathers: the transformed grid as hi + lo floats, or NULL (FP64 grid)
};

// A mesh constant in the kernel's precision.
template <typename T>
__device__ __forceinline__ T cst(double v64, float v32) {
    if constexpr (sizeof(T) == 4) return v32;
    else return v64;
}

template <typename T>
__device__ __forceinline__ T window(T f, T kappa) { return dexp<T>(-kappa * f * f); }

// Window l of axis d of a bead: the cached FP64 value (FP64 meshes), else evaluated.
template <typename T>
__device__ __forceinline__ T bead_window(const PairArgs& A, int bead, int d, T f, int l, bool in) {
    if constexpr (sizeof(T) == 8) {
        if (A.w64) return in ? A.w64[((size_t)bead * 3 + d) * A.g.P + l] : 0.0;
    }
    return in ? window<T>(f, cst<T>(A.g.kappa[d], A.kappa32[d])) : (T)0;
}

// (node l - x) / h per axis for lane l of a bead's stencil.
template <typename T>
__device__ __forceinline__ void bead_offsets(const PairArgs& A, int bead, int lane, T& fx, T& fy, T& fz) {
    if constexpr (sizeof(T) == 4) {
        const float4 fr = A.frac32[bead];
        fx = fr.x + (float)lane;
        fy = fr.y + (float)lane;
        fz = fr.z + (float)lane;
    } else {
        const double4 fr = A.frac[bead];
        fx = fr.x + (double)lane;
        fy = fr.y + (double)lane;
        fz = fr.z + (double)lane;
    }
}

// One-dimensional windows of a bead, lane l < P holding node l of each axis:
// weight, distance (node - x) and periodic node index.
template <typename T>
struct Windows {
    T wx, wy, wz, dx, dy, dz;
    T wdz;   // wz dz: the z walk of a gradient gather takes two fused multiply-adds per node
    int ix, iy, iz;
};

template <typename T, bool DIST>
__device__ __forceinline__ Windows<T> bead_windows(const PairArgs& A, int bead, int lane) {
    const MeshGeom& g = A.g;
    const int P = g.P;
    const int4 st = A.start[bead];
    Windows<T> W;
    T fx, fy, fz;
    bead_offsets<T>(A, bead, lane, fx, fy, fz);
    const bool in = lane < P;
    W.wx = bead_window<T>(A, bead, 0, fx, lane, in);
    W.wy = bead_window<T>(A, bead, 1, fy, lane, in);
    W.wz = bead_window<T>(A, bead, 2, fz, lane, in);
    if (DIST) {
        W.dx = fx * cst<T>(g.h[0], A.h32[0]);
        W.dy = fy * cst<T>(g.h[1], A.h32[1]);
        W.dz = fz * cst<T>(g.h[2], A.h32[2]);
        W.wdz = W.wz * W.dz;
    }
    W.ix = st.x + lane;
    W.iy = st.y + lane;
    W.iz = st.z + lane;
    if (W.ix >= g.N[0]) W.ix -= g.N[0];   // P <= N: one wrap at most
    if (W.iy >= g.N[1]) W.iy -= g.N[1];
    if (W.iz >= g.N[2]) W.iz -= g.N[2];
    return W;
}

// ---- FP64 gathers in double-float arithmetic ----
// The double-float transforms leave the FP64 potential as hi + lo floats.  A gather
// from it keeps every product and sum on the FP32 pipes: the bead's windows are split
// into hi + lo floats once per lane, each column's walk, its weight and the bead's
// running sums are double-float, and each result is joined to FP64 once (GB300
// issues FP64 instructions at 1/64 of its FP32 rate, and an FP64 multiply-add per
// column or per node made the FP64 pipe the limit of these gathers).

// One-dimensional windows of a bead as double-float, lane l < P holding node l.
struct DfWindows {
    df wx, wy, wz, dx, dy, wdz;
    int ix, iy, iz;
};

template <bool GRAD>
__device__ __forceinline__ DfWindows df_bead_windows(const PairArgs& A, int bead, int lane) {
    const MeshGeom& g = A.g;
    const int P = g.P;
    const bool in = lane < P;
    const float2* wb = A.wdf + (size_t)bead * 3 * P;
    DfWindows D;
    const float2 zero = make_float2(0.0f, 0.0f);
    const float2 wx = in ? wb[lane] : zero, wy = in ? wb[P + lane] : zero, wz = in ? wb[2 * P + lane] : zero;
    D.wx = df{wx.x, wx.y};
    D.wy = df{wy.x, wy.y};
    D.wz = df{wz.x, wz.y};
    if (GRAD) {   // distance (node l - x) = (f + l) h per axis, f the bead's offset
        const float4 fh = A.frac_df[2 * bead], fl = A.frac_df[2 * bead + 1];
        const float lf = (float)lane;
        D.dx = df_mul(df_add(df{fh.x, fl.x}, df{lf, 0.0f}), df{A.hdf[0][0], A.hdf[0][1]});
        D.dy = df_mul(df_add(df{fh.y, fl.y}, df{lf, 0.0f}), df{A.hdf[1][0], A.hdf[1][1]});
        const df dz = df_mul(df_add(df{fh.z, fl.z}, df{lf, 0.0f}), df{A.hdf[2][0], A.hdf[2][1]});
        D.wdz = df_mul(D.wz, dz);
    } else {
        D.dx = D.dy = D.wdz = df{0.0f, 0.0f};
    }
    const int4 st = A.start[bead];
    D.ix = st.x + lane;
    D.iy = st.y + lane;
    D.iz = st.z + lane;
    if (D.ix >= g.N[0]) D.ix -= g.N[0];   // P <= N: one wrap at most
    if (D.iy >= g.N[1]) D.iy -= g.N[1];
    if (D.iz >= g.N[2]) D.iz -= g.N[2];
    return D;
}

__device__ __forceinline__ df df_shfl(df v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// Adds one column's walk (sa = sum of node w_z, sz = sum of node w_z dz) with the
// column's weight w_x w_y (and distances dx, dy for the gradient) to the bead's sums.
template <int NR, bool GRAD>
__device__ __forceinline__ void df_column_add(df wxy, df dx, df dy, const df (&sa)[NR], const df (&sz)[NR],
                                              df (&sp)[NR], df (&ex)[NR], df (&ey)[NR], df (&ez)[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const df t = df_mul(wxy, sa[r]);
        sp[r] = df_add(sp[r], t);
        if (GRAD) {
            ex[r] = df_add(ex[r], df_mul(t, dx));
            ey[r] = df_add(ey[r], df_mul(t, dy));
            ez[r] = df_add(ez[r], df_mul(wxy, sz[r]));
        }
    }
}

// The bead's columns pair = first .. first + 31 (lane: first + lane) of its P^2 (x, y)
// columns, read from the global hi + lo grid of its configuration (gr: channel 0).
template <int NR, bool GRAD, int PC>
__device__ __forceinline__ void df_round_global(const DfWindows& D, int P_rt, int lane, int first, int n0,
                                                long long nxy, long long G, const float2* __restrict__ gr,
                                                df (&sp)[NR], df (&ex)[NR], df (&ey)[NR], df (&ez)[NR]) {
    const int P = PC ? PC : P_rt, P2 = P * P;
    const int pair = first + lane;
    const bool on = pair < P2;
    int j = pair / P, i = pair - j * P;
    if (!on) i = j = 0;
    const df wx = df_shfl(D.wx, i), wy = df_shfl(D.wy, j);
    const df wxy = on ? df_mul(wx, wy) : df{0.0f, 0.0f};
    df dx = {0.0f, 0.0f}, dy = {0.0f, 0.0f};
    if (GRAD) {
        dx = df_shfl(D.dx, i);
        dy = df_shfl(D.dy, j);
    }
    const long long base = (long long)__shfl_sync(0xffffffffu, D.iy, j) * n0 + __shfl_sync(0xffffffffu, D.ix, i);
    df sa[NR], sz[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sa[r] = sz[r] = df{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const df wz = df_shfl(D.wz, k);
        const int iz = __shfl_sync(0xffffffffu, D.iz, k);
        df wdz = {0.0f, 0.0f};
        if (GRAD) wdz = df_shfl(D.wdz, k);
        if (on) {
            const size_t off = (size_t)iz * nxy + base;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 v = __ldg(gr + (size_t)r * G + off);
                const df vd = {v.x, v.y};
                sa[r] = df_add(sa[r], df_mul(vd, wz));
                if (GRAD) sz[r] = df_add(sz[r], df_mul(vd, wdz));
            }
        }
    }
    df_column_add<NR, GRAD>(wxy, dx, dy, sa, sz, sp, ex, ey, ez);
}

// Sums of the lanes of a warp into psi (and E) for bead `bead`, scaled by the gather and
// gradient constants; accumulate adds (several warps share a bead), else it stores.
template <int NR, bool GRAD>
__device__ __forceinline__ void df_bead_store(const MeshGeom& g, int n, int bead, int lane, bool accumulate,
                                              df (&sp)[NR], df (&ex)[NR], df (&ey)[NR], df (&ez)[NR],
                                              double* __restrict__ psi, double* __restrict__ E) {
    // the constants as double-float (a float pair is exact to 2^-48 of them)
    const float gh = (float)g.gather, dh = (float)(-g.grad);
    const df cg = {gh, (float)(g.gather - (double)gh)}, cd = {dh, (float)(-g.grad - (double)dh)};
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        // every lane holds every sum after the shuffles; lane k < 4 joins result k
        // (one FP64 addition per bead for the potential and the three field components)
        const df s0 = df_mul(df_warp_sum(sp[r]), cg);
        df v = s0;
        if (GRAD) {
            const df e0 = df_mul(df_warp_sum(ex[r]), cd);
            const df e1 = df_mul(df_warp_sum(ey[r]), cd);
            const df e2 = df_mul(df_warp_sum(ez[r]), cd);
            v = lane == 1 ? e0 : (lane == 2 ? e1 : (lane == 3 ? e2 : s0));
        }
        if (lane > (GRAD ? 3 : 0)) continue;
        const double x = df_join(v);
        double* dst = lane == 0 ? psi + (size_t)r * n + bead : E + ((size_t)r * n + bead) * 3 + (lane - 1);
        if (accumulate) atomicAdd(dst, x);
        else *dst = x;
    }
}

// Direct FP64 gather of one bead (one warp) from the hi + lo grid.
template <int NR, bool GRAD, int PC>
__device__ __forceinline__ void gather_bead_df(const PairArgs& A, int n, int bead, int lane, double* __restrict__ psi,
                                               double* __restrict__ E) {
    const MeshGeom& g = A.g;
    const int P = PC ? PC : g.P, P2 = P * P;
    const DfWindows D = df_bead_windows<GRAD>(A, bead, lane);
    const float2* gr = A.gdf + (size_t)A.start[bead].w * NR * g.G;
    const long long nxy = (long long)g.N[0] * g.N[1];
    df sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sp[r] = ex[r] = ey[r] = ez[r] = df{0.0f, 0.0f};
#pragma unroll
    for (int first = 0; first < P2; first += 32)
        df_round_global<NR, GRAD, PC>(D, P, lane, first, g.N[0], nxy, g.G, gr, sp, ex, ey, ez);
    df_bead_store<NR, GRAD>(g, n, bead, lane, false, sp, ex, ey, ez, psi, E);
}

template <typename T, int NR, int PC>
__global__ void __launch_bounds__(32 * kPairWarps)
spread_pairs_kernel(PairArgs A, int n, const double* __restrict__ q, T* __restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kPairWarps + (threadIdx.x >> 5);
    const long long slot = gw / A.wpb;
    if (slot >= n) return;   // warp-uniform
    const int part = (int)(gw - slot * A.wpb);
    const int bead = (int)slot;
    const MeshGeom& g = A.g;
    const int P = PC ? PC : g.P, P2 = P * P;
    const Windows<T> W = bead_windows<T, false>(A, bead, lane);
    T* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    T qc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) qc[r] = cst<T>(g.c, A.c32) * (T)q[(size_t)r * n + bead];
    const long long nxy = (long long)g.N[0] * g.N[1];
    for (int rd = 0; rd < A.rounds; ++rd) {
        const int first = (part * A.rounds + rd) * 32;
        if (first >= P2) break;   // warp-uniform
        const int pair = first + lane;
        const bool on = pair < P2;
        int j = pair / P, i = pair - j * P;
        if (!on) i = j = 0;
        const T wxy = __shfl_sync(0xffffffffu, W.wx, i) * __shfl_sync(0xffffffffu, W.wy, j);
        const long long base = (long long)__shfl_sync(0xffffffffu, W.iy, j) * g.N[0] + __shfl_sync(0xffffffffu, W.ix, i);
        T qw[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) qw[r] = qc[r] * wxy;
        #pragma unroll
        for (int k = 0; k < P; ++k) {
            const T wz = __shfl_sync(0xffffffffu, W.wz, k);
            const int iz = __shfl_sync(0xffffffffu, W.iz, k);
            if (on) {
                const size_t off = (size_t)iz * nxy + base;
#pragma unroll
                for (int r = 0; r < NR; ++r) atomicAdd(gr + (size_t)r * g.G + off, qw[r] * wz);
            }
        }
    }
}

// The z walk of one (x, y) column of a gather from the double-float grid (FP64
// meshes with double-float transforms): products and sums on the FP32 pipes, one
// FP64 addition per column and field to join the result (GB300 runs FP64 at a small
// fraction of its FP32 rate).  wzl, wdzl: this lane's window and window x distance
// as hi + lo floats; lane k supplies node k of the column.
template <int NR, bool GRAD, int PC>
__device__ __forceinline__ void column_walk_df(const float2* __restrict__ gr, long long G, long long nxy,
                                               long long base, bool on, int P_rt, df wzl, df wdzl, int izl,
                                               double (&a)[NR], double (&az)[NR]) {
    const unsigned full = 0xffffffffu;
    const int P = PC ? PC : P_rt;
    df sa[NR], sz[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sa[r] = sz[r] = df{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const df wz = {__shfl_sync(full, wzl.hi, k), __shfl_sync(full, wzl.lo, k)};
        const int iz = __shfl_sync(full, izl, k);
        df wdz = {0.0f, 0.0f};
        if (GRAD) wdz = df{__shfl_sync(full, wdzl.hi, k), __shfl_sync(full, wdzl.lo, k)};
        if (on) {
            const size_t off = (size_t)iz * nxy + base;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 v = __ldg(gr + (size_t)r * G + off);
                const df vd = {v.x, v.y};
                sa[r] = df_add(sa[r], df_mul(vd, wz));
                if (GRAD) sz[r] = df_add(sz[r], df_mul(vd, wdz));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        a[r] = df_join(sa[r]);
        az[r] = GRAD ? df_join(sz[r]) : 0.0;
    }
}

template <typename T, int NR, bool GRAD, int PC>
__global__ void __launch_bounds__(32 * kPairWarps)
gather_pairs_kernel(PairArgs A, int n, const T* __restrict__ grid, double* __restrict__ psi, double* __restrict__ E) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kPairWarps + (threadIdx.x >> 5);
    const long long slot = gw / A.wpb;
    if (slot >= n) return;   // warp-uniform
    const int part = (int)(gw - slot * A.wpb);
    const int bead = (int)slot;
    const MeshGeom& g = A.g;
    const int P = PC ? PC : g.P, P2 = P * P;
    if constexpr (sizeof(T) == 8) {
        if (A.gdf) {   // FP64 potential as hi + lo floats: double-float throughout
            const DfWindows D = df_bead_windows<GRAD>(A, bead, lane);
            const float2* gr2 = A.gdf + (size_t)A.start[bead].w * NR * g.G;
            const long long nxy2 = (long long)g.N[0] * g.N[1];
            df dsp[NR], dex[NR], dey[NR], dez[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) dsp[r] = dex[r] = dey[r] = dez[r] = df{0.0f, 0.0f};
            for (int rd = 0; rd < A.rounds; ++rd) {
                const int first = (part * A.rounds + rd) * 32;
                if (first >= P2) break;   // warp-uniform
                df_round_global<NR, GRAD, PC>(D, P, lane, first, g.N[0], nxy2, g.G, gr2, dsp, dex, dey, dez);
            }
            df_bead_store<NR, GRAD>(g, n, bead, lane, A.wpb > 1, dsp, dex, dey, dez, psi, E);
            return;
        }
    }
    const Windows<T> W = bead_windows<T, GRAD>(A, bead, lane);
    const T* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    T sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sp[r] = ex[r] = ey[r] = ez[r] = (T)0;
    const long long nxy = (long long)g.N[0] * g.N[1];
    df wz_df = {0.0f, 0.0f}, wdz_df = {0.0f, 0.0f};   // this lane's z window as hi + lo (double-float grid)
    if constexpr (sizeof(T) == 8) {
        if (A.gdf) {
            wz_df = df_split(W.wz);
            if (GRAD) wdz_df = df_split(W.wdz);
        }
    }
    for (int rd = 0; rd < A.rounds; ++rd) {
        const int first = (part * A.rounds + rd) * 32;
        if (first >= P2) break;   // warp-uniform
        const int pair = first + lane;
        const bool on = pair < P2;
        int j = pair / P, i = pair - j * P;
        if (!on) i = j = 0;
        // every lane takes part in every shuffle (full mask); off lanes then drop their weight
        const T wx = __shfl_sync(0xffffffffu, W.wx, i), wy = __shfl_sync(0xffffffffu, W.wy, j);
        const T wxy = on ? wx * wy : (T)0;
        T dx = (T)0, dy = (T)0;
        if (GRAD) {
            dx = __shfl_sync(0xffffffffu, W.dx, i);
            dy = __shfl_sync(0xffffffffu, W.dy, j);
        }
        const long long base = (long long)__shfl_sync(0xffffffffu, W.iy, j) * g.N[0] + __shfl_sync(0xffffffffu, W.ix, i);
        T a[NR], az[NR];
        bool walked = false;
        if constexpr (sizeof(T) == 8) {
            if (A.gdf) {
                column_walk_df<NR, GRAD, PC>(A.gdf + (size_t)A.start[bead].w * NR * g.G, g.G, nxy, base, on, P,
                                             wz_df, wdz_df, W.iz, a, az);
                walked = true;
            }
        }
        if (!walked) {
#pragma unroll
            for (int r = 0; r < NR; ++r) a[r] = az[r] = (T)0;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const T wz = __shfl_sync(0xffffffffu, W.wz, k);
                const int iz = __shfl_sync(0xffffffffu, W.iz, k);
                T wdz = (T)0;
                if (GRAD) wdz = __shfl_sync(0xffffffffu, W.wdz, k);
                if (on) {
                    const size_t off = (size_t)iz * nxy + base;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const T v = __ldg(gr + (size_t)r * g.G + off);
                        a[r] = fma(v, wz, a[r]);
                        if (GRAD) az[r] = fma(v, wdz, az[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            sp[r] += wxy * a[r];
            if (GRAD) {
                ex[r] += wxy * dx * a[r];
                ey[r] += wxy * dy * a[r];
                ez[r] += wxy * az[r];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const T s0 = warp_sum(sp[r]);
        if (GRAD) {
            const T e0 = warp_sum(ex[r]);
            const T e1 = warp_sum(ey[r]);
            const T e2 = warp_sum(ez[r]);
            if (lane == 0) {
                double* e = E + ((size_t)r * n + bead) * 3;
                if (A.wpb == 1) {
                    e[0] = (double)(-cst<T>(g.grad, A.grad32) * e0);
                    e[1] = (double)(-cst<T>(g.grad, A.grad32) * e1);
                    e[2] = (double)(-cst<T>(g.grad, A.grad32) * e2);
                } else {
                    atomicAdd(e + 0, (double)(-cst<T>(g.grad, A.grad32) * e0));
                    atomicAdd(e + 1, (double)(-cst<T>(g.grad, A.grad32) * e1));
                    atomicAdd(e + 2, (double)(-cst<T>(g.grad, A.grad32) * e2));
                }
            }
        }
        if (lane == 0) {
            if (A.wpb == 1)
                psi[(size_t)r * n + bead] = (double)(cst<T>(g.gather, A.gather32) * s0);
            else
                atomicAdd(psi + (size_t)r * n + bead, (double)(cst<T>(g.gather, A.gather32) * s0));
        }
    }
}

template <typename T, int NR>
void launch_pairs(bool spread, bool grad, const PairArgs& A, int n, const double* q, T* grid, double* psi,
                  double* E, cudaStream_t s) {
    const int blocks = div_up((long long)n * A.wpb, kPairWarps);
    // compile-time P = 9 (tolerance 1e-6) for the usual field counts: the z walk unrolls
    bool p9 = false;
    if constexpr (NR <= 3) p9 = A.g.P == 9;
    if (spread) {
        if constexpr (NR <= 3) {
            if (p9) {
                spread_pairs_kernel<T, NR, 9><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, q, grid);
                return;
            }
        }
        spread_pairs_kernel<T, NR, 0><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, q, grid);
    } else if (grad) {
        if constexpr (NR <= 3) {
            if (p9) {
                gather_pairs_kernel<T, NR, true, 9><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, grid, psi, E);
                return;
            }
        }
        gather_pairs_kernel<T, NR, true, 0><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, grid, psi, E);
    } else {
        if constexpr (NR <= 3) {
            if (p9) {
                gather_pairs_kernel<T, NR, false, 9><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, grid, psi, nullptr);
                return;
            }
        }
        gather_pairs_kernel<T, NR, false, 0><<<blocks, 32 * kPairWarps, 0, s>>>(A, n, grid, psi, nullptr);
    }
}

template <typename T>
void pairs_dispatch(int nrhs, bool spread, bool grad, const PairArgs& A, int n, const double* q, T* grid,
                    double* psi, double* E, cudaStream_t s) {
    switch (nrhs) {
        case 1: launch_pairs<T, 1>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 2: launch_pairs<T, 2>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 3: launch_pairs<T, 3>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 4: launch_pairs<T, 4>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 5: launch_pairs<T, 5>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 6: launch_pairs<T, 6>(spread, grad, A, n, q, grid, psi, E, s); break;
        case 7: launch_pairs<T, 7>(spread, grad, A, n, q, grid, psi, E, s); break;
        default: launch_pairs<T, 8>(spread, grad, A, n, q, grid, psi, E, s); break;
    }
}

// Warps per bead: split a bead's P^2 columns over several warps while the bead
// count alone cannot fill the GPU (about two waves of resident warps), else one
// warp walks all of them and sets its window up once.
void pair_consts(PairArgs& A, const MeshGeom& g, const StencilCache& b) {
    A.g = g;
    A.start = b.start.as<int4>();
    A.frac = b.frac.as<double4>();
    A.frac32 = b.frac32.as<float4>();
    A.w64 = b.w64.as<double>();
    A.wdf = b.wdf.as<float2>();
    A.frac_df = b.frac_df.as<float4>();
    for (int d = 0; d < 3; ++d) {
        const float hi = (float)g.h[d];
        A.hdf[d][0] = hi;
        A.hdf[d][1] = (float)(g.h[d] - (double)hi);
    }
    for (int d = 0; d < 3; ++d) {
        A.kappa32[d] = (float)g.kappa[d];
        A.h32[d] = (float)g.h[d];
    }
    A.c32 = (float)g.c;
    A.gather32 = (float)g.gather;
    A.grad32 = (float)g.grad;
}

PairArgs pair_args(const MeshGeom& g, const StencilCache& b, int n) {
    PairArgs A{};
    pair_consts(A, g, b);
    const int blocks32 = (g.P * g.P + 31) / 32;
    const bool split = (long long)n * blocks32 <= 152LL * 64 * 2;
    A.wpb = split ? blocks32 : 1;
    A.rounds = split ? 1 : blocks32;
    return A;
}

// ---------------------------------------------------------------------------
// Tiled spreading and gathering through shared memory.
//
// On dense bead surfaces hundreds of beads share every grid node, and their
// global atomics queue on the same L2 addresses.  Beads are binned (once per
// set of positions) by configuration and by the tile of kTileNodes^3 nodes that
// holds their first stencil node; every stencil of a tile then lies inside one
// region of E^3 nodes, E = kTileNodes + P - 1.  A block takes kTileChunk
// consecutive sorted beads and splits them into runs of one tile.  A run of at
// least kTileMin beads is spread into the region in shared memory and the region
// is added to the grid once (one atomic per non-zero node); a gather stages the
// region in shared memory and reads every stencil from there.  Beads of
// shorter runs (isolated ions) use the direct per-bead path.
// ---------------------------------------------------------------------------
constexpr int kTileChunk = 128;     // most sorted beads per block
constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileMin = 24;        // beads of one tile that go through shared memory: a sphere's
                                    // surface puts 5-20 beads in a tile, which the direct path
                                    // serves faster than staging a whole region
constexpr size_t kTileSmemMax = 192 * 1024;
constexpr size_t kTmaPad = 128;     // dynamic shared memory a gather adds to align its region

struct TileArgs {
    bool tma = false;       // the kernel's tensor map describes this grid: regions that do not
                            // wrap are loaded with cp.async.bulk.tensor
    int* tma_err = nullptr; // set when a bounded wait for a tensor copy ran out (1) or a check failed (2-6)
    int tma_zext = 0;       // z extent of the tensor map (N_z x channels)
    PairArgs A;             // geometry and cached stencils (one warp per bead)
    const int* sorted;      // bead at each sorted position
    const int* key;         // configuration * ntiles + tile at each sorted position
    int tn[3];              // tiles per axis
    int ntiles;
    int E;                  // region edge in nodes
    int chunk;              // sorted beads per block (<= kTileChunk)
};

// ---- TMA region loads ------------------------------------------------------------
// A gather's region of E^3 nodes per channel, when it does not wrap around the box,
// comes in as one 3-D tensor copy per channel (the grid described as N_x x N_y x
// (N_z channels), channel c's region at z = c N_z + oz) into the block's shared
// memory, completing on an mbarrier.  x offsets are multiples of 8 nodes and the box
// edge E times the element size a multiple of 16 bytes (checked on the host).
constexpr int kTmaWaitLimit = 1 << 22;   // polls of the mbarrier before the load is given up

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_barrier_init(uint64_t* mbar) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

__device__ __forceinline__ bool tma_poll(uint64_t* mbar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the current phase; true when it completed.
__device__ __forceinline__ bool tma_wait(uint64_t* mbar, unsigned phase) {
    for (int it = 0; it < kTmaWaitLimit; ++it) {
        if (tma_poll(mbar, phase)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

// Thread 0 checks and issues the nr copies (bytes each) of the region at (ox, oy,
// z0 + c zstep) into dst + c bytes; every thread then waits.  Returns (block-uniform)
// 1 when the region is in shared memory, -1 when a check failed before any copy was
// issued (the code is recorded in *err, the caller loads the region itself: the
// destination and the mbarrier aligned, x a multiple of 16 bytes, the boxes inside the
// z extent, the tensor map aligned), 0 when the wait ran out (recorded; the copies are
// waited for once more and the caller returns).
__device__ int tma_region(const CUtensorMap* tm, unsigned char* dst, int nr, unsigned bytes, int es, int E, int ox,
                          int oy, int z0, int zstep, int zext, uint64_t* mbar, unsigned& phase, int* err) {
    __shared__ int verdict;
    if (threadIdx.x == 0) {
        int code = 0;
        if ((smem_addr(dst) & 127u) != 0u) code = 2;
        else if ((smem_addr(mbar) & 7u) != 0u) code = 3;
        else if (((long long)ox * es) % 16 != 0 || ox < 0 || oy < 0 || z0 < 0) code = 4;
        else if (z0 + (nr - 1) * zstep + E > zext) code = 5;
        else if ((reinterpret_cast<unsigned long long>(tm) & 63ull) != 0ull) code = 6;
        verdict = code;
        if (code) {
            if (err) atomicExch(err, code);
        } else {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the region are done
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
                         "r"(bytes * (unsigned)nr)
                         : "memory");
            for (int c = 0; c < nr; ++c)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4}], [%5];" ::"r"(smem_addr(dst + (size_t)c * bytes)),
                    "l"(reinterpret_cast<unsigned long long>(tm)), "r"(ox), "r"(oy), "r"(z0 + c * zstep),
                    "r"(smem_addr(mbar))
                    : "memory");
        }
    }
    __syncthreads();
    if (verdict != 0) return -1;
    const bool done = tma_wait(mbar, phase);
    const bool bad = __syncthreads_or(!done);
    if (bad) {
        if (threadIdx.x == 0 && err) atomicExch(err, 1);
        tma_wait(mbar, phase);   // the copies may still land: give them the time once more
        __syncthreads();
    }
    phase ^= 1u;
    return bad ? 0 : 1;
}

__global__ void tile_count_kernel(int n, const int4* __restrict__ start, int tn0, int tn1, int tn2,
                                  int* __restrict__ count, int* __restrict__ key) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int4 s = start[b];
    const int k = ((s.w * tn2 + s.z / kTileNodes) * tn1 + s.y / kTileNodes) * tn0 + s.x / kTileNodes;
    key[b] = k;
    atomicAdd(count + k, 1);
}

__global__ void tile_fill_kernel(int n, const int* __restrict__ bead_key, const long long* __restrict__ off,
                                 int* __restrict__ cursor, int* __restrict__ sorted, int* __restrict__ skey) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int k = bead_key[b];
    const long long p = off[k] + atomicAdd(cursor + k, 1);
    sorted[p] = b;
    skey[p] = k;
}

// Runs of equal keys among the block's sorted positions [p0, p0 + m): run r
// covers [run_start[r], run_start[r + 1]); run_of[t] is the run of position t.
struct TileRuns {
    int start[kTileChunk + 1];
    int of[kTileChunk];
    int wcount[kTileChunk / 32];
    int count;
};

__device__ void tile_runs(const int* __restrict__ key, int p0, int m, TileRuns& R) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const bool in = t < m;   // m <= kTileChunk <= blockDim.x
    const int k = in ? key[p0 + t] : -1;
    const bool head = in && (t == 0 || key[p0 + t - 1] != k);
    const unsigned bal = __ballot_sync(0xffffffffu, head);
    if (lane == 0 && w < kTileChunk / 32) R.wcount[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int u = 0; u < w && u < kTileChunk / 32; ++u) before += R.wcount[u];
    if (head) R.start[before + __popc(bal & ((1u << lane) - 1u))] = t;
    if (in) R.of[t] = before + __popc(bal & ((2u << lane) - 1u)) - 1;   // lane 31: mask wraps to all ones
    if (t == 0) {
        int tot = 0;
        for (int u = 0; u < kTileChunk / 32; ++u) tot += R.wcount[u];
        R.count = tot;
        R.start[tot] = m;
    }
    __syncthreads();
}

__device__ __forceinline__ int wrap_once(int v, int N) { return v >= N ? v - N : v; }

// ---- FP32 direct paths with 16-byte accesses ----
// With N_x a multiple of four and the stencil width known at compile time, a lane
// takes one (y, z) row of a bead's stencil; the row's P x-nodes lie in G4 aligned
// groups of four consecutive nodes (periodic wrap at a group boundary), which are
// added with float4 atomics (spread) or read with float4 loads (gather), zeros in
// the slots outside the stencil: for P = 9 three vector accesses per row instead of
// nine scalar ones.  Every lane holds the 4 G4 slot weights of the x axis (the same for
// all rows of the bead).
template <int P>
struct V4 {
    static constexpr int G4 = (P + 6) / 4;   // groups covering offsets sh .. sh + P - 1, sh < 4
};

template <int P>
__device__ __forceinline__ void x_slots(float wl, int sh, float (&w)[4 * V4<P>::G4]) {
#pragma unroll
    for (int m = 0; m < 4 * V4<P>::G4; ++m) {
        const int idx = m - sh;   // warp-uniform
        const float v = __shfl_sync(0xffffffffu, wl, idx < 0 ? 0 : (idx >= P ? 0 : idx));
        w[m] = (idx >= 0 && idx < P) ? v : 0.0f;
    }
}

template <int NR, int P>
__device__ __forceinline__ void spread_bead_v4(const PairArgs& A, int n, int bead, int lane,
                                               const double* __restrict__ q, float* __restrict__ grid) {
    constexpr int G4 = V4<P>::G4, P2 = P * P;
    const MeshGeom& g = A.g;
    const Windows<float> W = bead_windows<float, false>(A, bead, lane);
    const int ix0 = __shfl_sync(0xffffffffu, W.ix, 0);
    const int sh = ix0 & 3, gx0 = ix0 >> 2, ngx = g.N[0] >> 2;
    float wx[4 * G4];
    x_slots<P>(W.wx, sh, wx);
    float* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    float qc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) qc[r] = A.c32 * (float)q[(size_t)r * n + bead];
#pragma unroll
    for (int first = 0; first < P2; first += 32) {
        const int row = first + lane;
        const bool on = row < P2;
        int k = row / P, j = row - k * P;
        if (!on) j = k = 0;
        const float wyz = __shfl_sync(0xffffffffu, W.wy, j) * __shfl_sync(0xffffffffu, W.wz, k);
        const int iy = __shfl_sync(0xffffffffu, W.iy, j), iz = __shfl_sync(0xffffffffu, W.iz, k);
        if (on) {
            float4* row4 = reinterpret_cast<float4*>(gr + ((size_t)iz * g.N[1] + iy) * g.N[0]);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float s = qc[r] * wyz;
                float4* rp = row4 + (size_t)r * (g.G >> 2);
#pragma unroll
                for (int t = 0; t < G4; ++t) {
                    int gx = gx0 + t;
                    if (gx >= ngx) gx -= ngx;
                    atomicAdd(rp + gx, make_float4(s * wx[4 * t], s * wx[4 * t + 1], s * wx[4 * t + 2],
                                                   s * wx[4 * t + 3]));
                }
            }
        }
    }
}

template <int NR, bool GRAD, int P>
__device__ __forceinline__ void gather_bead_v4(const PairArgs& A, int n, int bead, int lane,
                                               const float* __restrict__ grid, double* __restrict__ psi,
                                               double* __restrict__ E) {
    constexpr int G4 = V4<P>::G4, P2 = P * P;
    const MeshGeom& g = A.g;
    const Windows<float> W = bead_windows<float, GRAD>(A, bead, lane);
    const int ix0 = __shfl_sync(0xffffffffu, W.ix, 0);
    const int sh = ix0 & 3, gx0 = ix0 >> 2, ngx = g.N[0] >> 2;
    float wx[4 * G4], wxd[4 * G4];
    x_slots<P>(W.wx, sh, wx);
    if (GRAD) x_slots<P>(W.wx * W.dx, sh, wxd);
    const float* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    float sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sp[r] = ex[r] = ey[r] = ez[r] = 0.0f;
#pragma unroll
    for (int first = 0; first < P2; first += 32) {
        const int row = first + lane;
        const bool on = row < P2;
        int k = row / P, j = row - k * P;
        if (!on) j = k = 0;
        const float wy = __shfl_sync(0xffffffffu, W.wy, j), wz = __shfl_sync(0xffffffffu, W.wz, k);
        float wyz = wy * wz, wdy = 0.0f, wdz = 0.0f;
        if (GRAD) {
            wdy = wy * __shfl_sync(0xffffffffu, W.dy, j) * wz;
            wdz = wy * __shfl_sync(0xffffffffu, W.wdz, k);
        }
        const int iy = __shfl_sync(0xffffffffu, W.iy, j), iz = __shfl_sync(0xffffffffu, W.iz, k);
        if (!on) wyz = wdy = wdz = 0.0f;
        if (on) {
            const float4* row4 = reinterpret_cast<const float4*>(gr + ((size_t)iz * g.N[1] + iy) * g.N[0]);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float4* rp = row4 + (size_t)r * (g.G >> 2);
                float a = 0.0f, ax = 0.0f;
#pragma unroll
                for (int t = 0; t < G4; ++t) {
                    int gx = gx0 + t;
                    if (gx >= ngx) gx -= ngx;
                    const float4 v = __ldg(rp + gx);
                    a = fmaf(v.x, wx[4 * t], fmaf(v.y, wx[4 * t + 1], fmaf(v.z, wx[4 * t + 2], fmaf(v.w, wx[4 * t + 3], a))));
                    if (GRAD)
                        ax = fmaf(v.x, wxd[4 * t], fmaf(v.y, wxd[4 * t + 1],
                                  fmaf(v.z, wxd[4 * t + 2], fmaf(v.w, wxd[4 * t + 3], ax))));
                }
                sp[r] = fmaf(wyz, a, sp[r]);
                if (GRAD) {
                    ex[r] = fmaf(wyz, ax, ex[r]);
                    ey[r] = fmaf(wdy, a, ey[r]);
                    ez[r] = fmaf(wdz, a, ez[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const float s0 = warp_sum(sp[r]);
        if (GRAD) {
            const float e0 = warp_sum(ex[r]), e1 = warp_sum(ey[r]), e2 = warp_sum(ez[r]);
            if (lane == 0) {
                double* e = E + ((size_t)r * n + bead) * 3;
                e[0] = (double)(-A.grad32 * e0);
                e[1] = (double)(-A.grad32 * e1);
                e[2] = (double)(-A.grad32 * e2);
            }
        }
        if (lane == 0) psi[(size_t)r * n + bead] = (double)(A.gather32 * s0);
    }
}

// Direct spreading of one bead (one warp, global atomics).
template <typename T, int NR, int PC>
__device__ __forceinline__ void spread_bead_direct(const PairArgs& A, int n, int bead, int lane,
                                                   const double* __restrict__ q, T* __restrict__ grid) {
    const MeshGeom& g = A.g;
    const int P = PC ? PC : g.P, P2 = P * P;
    const Windows<T> W = bead_windows<T, false>(A, bead, lane);
    T* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    T qc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) qc[r] = cst<T>(g.c, A.c32) * (T)q[(size_t)r * n + bead];
    const long long nxy = (long long)g.N[0] * g.N[1];
    #pragma unroll
    for (int first = 0; first < P2; first += 32) {
        const int pair = first + lane;
        const bool on = pair < P2;
        int j = pair / P, i = pair - j * P;
        if (!on) i = j = 0;
        const T wxy = __shfl_sync(0xffffffffu, W.wx, i) * __shfl_sync(0xffffffffu, W.wy, j);
        const long long base = (long long)__shfl_sync(0xffffffffu, W.iy, j) * g.N[0] + __shfl_sync(0xffffffffu, W.ix, i);
        T qw[NR];   // the column's weight: one multiplication per node below
#pragma unroll
        for (int r = 0; r < NR; ++r) qw[r] = qc[r] * wxy;
        #pragma unroll
        for (int k = 0; k < P; ++k) {
            const T wz = __shfl_sync(0xffffffffu, W.wz, k);
            const int iz = __shfl_sync(0xffffffffu, W.iz, k);
            if (on) {
                const size_t off = (size_t)iz * nxy + base;
#pragma unroll
                for (int r = 0; r < NR; ++r) atomicAdd(gr + (size_t)r * g.G + off, qw[r] * wz);
            }
        }
    }
}

template <typename T, int NR, int PC>
__global__ void __launch_bounds__(kTileThreads)
spread_tiles_kernel(TileArgs TA, int n, const double* __restrict__ q, T* __restrict__ grid) {
    extern __shared__ __align__(16) unsigned char tile_smem_base[];
    unsigned char* tile_smem = tile_smem_base;
    T* reg = reinterpret_cast<T*>(tile_smem);
    __shared__ TileRuns R;
    const int p0 = blockIdx.x * TA.chunk;
    const int m = min(TA.chunk, n - p0);
    tile_runs(TA.key, p0, m, R);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const PairArgs& A = TA.A;
    const MeshGeom& g = A.g;
    // isolated beads: direct atomics (FP32 rows as float4 groups when the stencil width is fixed)
    const bool v4x = (g.N[0] & 3) == 0;
    for (int t = w; t < m; t += kTileWarps) {
        const int r = R.of[t];
        if (R.start[r + 1] - R.start[r] < kTileMin) {
            if constexpr (sizeof(T) == 4 && PC > 0) {
                if (v4x) {
                    spread_bead_v4<NR, PC>(A, n, TA.sorted[p0 + t], lane, q, reinterpret_cast<float*>(grid));
                    continue;
                }
            }
            spread_bead_direct<T, NR, PC>(A, n, TA.sorted[p0 + t], lane, q, grid);
        }
    }
    const int E = TA.E, E2 = E * E, E3 = E2 * E;
    const int P = PC ? PC : g.P, P2 = P * P;
    for (int r = 0; r < R.count; ++r) {
        const int a = R.start[r], b = R.start[r + 1];
        if (b - a < kTileMin) continue;   // block-uniform
        const int key = TA.key[p0 + a];
        const int tile = key % TA.ntiles, cfg = key / TA.ntiles;
        const int ox = (tile % TA.tn[0]) * kTileNodes;
        const int oy = ((tile / TA.tn[0]) % TA.tn[1]) * kTileNodes;
        const int oz = (tile / (TA.tn[0] * TA.tn[1])) * kTileNodes;
        for (int u = threadIdx.x; u < NR * E3; u += kTileThreads) reg[u] = (T)0;
        __syncthreads();
        for (int t = a + w; t < b; t += kTileWarps) {
            const int bead = TA.sorted[p0 + t];
            const int4 st = A.start[bead];
            const bool in = lane < P;
            T fx, fy, fz;
            bead_offsets<T>(A, bead, lane, fx, fy, fz);
            const T wx = bead_window<T>(A, bead, 0, fx, lane, in);
            const T wy = bead_window<T>(A, bead, 1, fy, lane, in);
            const T wz_l = bead_window<T>(A, bead, 2, fz, lane, in);
            const int lx = st.x - ox, ly = st.y - oy, lz = st.z - oz;   // in [0, kTileNodes)
            T qc[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) qc[c] = cst<T>(g.c, A.c32) * (T)q[(size_t)c * n + bead];
            #pragma unroll
    for (int first = 0; first < P2; first += 32) {
                const int pair = first + lane;
                const bool on = pair < P2;
                int j = pair / P, i = pair - j * P;
                if (!on) i = j = 0;
                const T wxy = __shfl_sync(0xffffffffu, wx, i) * __shfl_sync(0xffffffffu, wy, j);
                const int base = (lz * E + ly + j) * E + lx + i;
                T qw[NR];   // the column's weight: one multiplication per node below
#pragma unroll
                for (int c = 0; c < NR; ++c) qw[c] = qc[c] * wxy;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const T wz = __shfl_sync(0xffffffffu, wz_l, k);
                    if (on) {
#pragma unroll
                        for (int c = 0; c < NR; ++c) atomicAdd(reg + c * E3 + base + k * E2, qw[c] * wz);
                    }
                }
            }
        }
        __syncthreads();
        T* gr = grid + (size_t)cfg * NR * g.G;
        bool flushed = false;
        if constexpr (sizeof(T) == 4) {
            if (v4x && (E & 3) == 0) {   // groups of four x-nodes: float4 atomics (a group never wraps)
                const int E4 = E >> 2;
                for (int u = threadIdx.x; u < NR * (E3 >> 2); u += kTileThreads) {
                    const float4 v = reinterpret_cast<const float4*>(reg)[u];
                    if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f) {
                        const int c = u / (E3 >> 2), rem = u - c * (E3 >> 2);
                        const int z = rem / (E2 >> 2), y = (rem / E4) % E, x = 4 * (rem % E4);
                        const size_t off = ((size_t)wrap_once(oz + z, g.N[2]) * g.N[1] + wrap_once(oy + y, g.N[1])) *
                                               g.N[0] + wrap_once(ox + x, g.N[0]);
                        atomicAdd(reinterpret_cast<float4*>(gr + (size_t)c * g.G + off), v);
                    }
                }
                flushed = true;
            }
        }
        if (!flushed) {
            for (int u = threadIdx.x; u < NR * E3; u += kTileThreads) {
                const T v = reg[u];
                if (v != (T)0) {
                    const int c = u / E3, rem = u - c * E3;
                    const int z = rem / E2, y = (rem / E) % E, x = rem % E;
                    const size_t off = ((size_t)wrap_once(oz + z, g.N[2]) * g.N[1] + wrap_once(oy + y, g.N[1])) *
                                           g.N[0] + wrap_once(ox + x, g.N[0]);
                    atomicAdd(gr + (size_t)c * g.G + off, v);
                }
            }
        }
        __syncthreads();
    }
}

// Direct gather of one bead (one warp) into psi / E.
template <typename T, int NR, bool GRAD, int PC>
__device__ __forceinline__ void gather_bead_direct(const PairArgs& A, int n, int bead, int lane,
                                                   const T* __restrict__ grid, double* __restrict__ psi,
                                                   double* __restrict__ E) {
    const MeshGeom& g = A.g;
    const int P = PC ? PC : g.P, P2 = P * P;
    const Windows<T> W = bead_windows<T, GRAD>(A, bead, lane);
    const T* gr = grid + (size_t)A.start[bead].w * NR * g.G;
    T sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) sp[r] = ex[r] = ey[r] = ez[r] = (T)0;
    const long long nxy = (long long)g.N[0] * g.N[1];
    df wz_df = {0.0f, 0.0f}, wdz_df = {0.0f, 0.0f};   // this lane's z window as hi + lo (double-float grid)
    if constexpr (sizeof(T) == 8) {
        if (A.gdf) {
            wz_df = df_split(W.wz);
            if (GRAD) wdz_df = df_split(W.wdz);
        }
    }
    #pragma unroll
    for (int first = 0; first < P2; first += 32) {
        const int pair = first + lane;
        const bool on = pair < P2;
        int j = pair / P, i = pair - j * P;
        if (!on) i = j = 0;
        const T wx = __shfl_sync(0xffffffffu, W.wx, i), wy = __shfl_sync(0xffffffffu, W.wy, j);
        const T wxy = on ? wx * wy : (T)0;
        T dx = (T)0, dy = (T)0;
        if (GRAD) {
            dx = __shfl_sync(0xffffffffu, W.dx, i);
            dy = __shfl_sync(0xffffffffu, W.dy, j);
        }
        const long long base = (long long)__shfl_sync(0xffffffffu, W.iy, j) * g.N[0] + __shfl_sync(0xffffffffu, W.ix, i);
        T acc[NR], accz[NR];
        bool walked = false;
        if constexpr (sizeof(T) == 8) {
            if (A.gdf) {
                column_walk_df<NR, GRAD, PC>(A.gdf + (size_t)A.start[bead].w * NR * g.G, g.G, nxy, base, on, P,
                                             wz_df, wdz_df, W.iz, acc, accz);
                walked = true;
            }
        }
        if (!walked) {
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = accz[r] = (T)0;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const T wz = __shfl_sync(0xffffffffu, W.wz, k);
                const int iz = __shfl_sync(0xffffffffu, W.iz, k);
                T wdz = (T)0;
                if (GRAD) wdz = __shfl_sync(0xffffffffu, W.wdz, k);
                if (on) {
                    const size_t off = (size_t)iz * nxy + base;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const T v = __ldg(gr + (size_t)r * g.G + off);
                        acc[r] = fma(v, wz, acc[r]);
                        if (GRAD) accz[r] = fma(v, wdz, accz[r]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            sp[r] += wxy * acc[r];
            if (GRAD) {
                ex[r] += wxy * dx * acc[r];
                ey[r] += wxy * dy * acc[r];
                ez[r] += wxy * accz[r];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const T s0 = warp_sum(sp[r]);
        if (GRAD) {
            const T e0 = warp_sum(ex[r]);
            const T e1 = warp_sum(ey[r]);
            const T e2 = warp_sum(ez[r]);
            if (lane == 0) {
                double* e = E + ((size_t)r * n + bead) * 3;
                e[0] = (double)(-cst<T>(g.grad, A.grad32) * e0);
                e[1] = (double)(-cst<T>(g.grad, A.grad32) * e1);
                e[2] = (double)(-cst<T>(g.grad, A.grad32) * e2);
            }
        }
        if (lane == 0) psi[(size_t)r * n + bead] = (double)(cst<T>(g.gather, A.gather32) * s0);
    }
}

// Dense tiles of an FP64 gather from the hi + lo grid: the region is staged in shared
// memory as hi + lo floats and every bead of the run is gathered from it in
// double-float arithmetic.
template <int NR, bool GRAD, int PC>
__device__ void gather_tiles_df(const TileArgs& TA, const TileRuns& R, int p0, int n, float2* __restrict__ reg,
                                double* __restrict__ psi, double* __restrict__ E, const CUtensorMap* tm,
                                uint64_t* mbar, unsigned& phase) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const PairArgs& A = TA.A;
    const MeshGeom& g = A.g;
    const int Ee = TA.E, E2 = Ee * Ee, E3 = E2 * Ee;
    const int P = PC ? PC : g.P, P2 = P * P;
    for (int r = 0; r < R.count; ++r) {
        const int a = R.start[r], b = R.start[r + 1];
        if (b - a < kTileMin) continue;   // block-uniform
        const int key = TA.key[p0 + a];
        const int tile = key % TA.ntiles, cfg = key / TA.ntiles;
        const int ox = (tile % TA.tn[0]) * kTileNodes;
        const int oy = ((tile / TA.tn[0]) % TA.tn[1]) * kTileNodes;
        const int oz = (tile / (TA.tn[0] * TA.tn[1])) * kTileNodes;
        const float2* gr = A.gdf + (size_t)cfg * NR * g.G;
        const bool inside = ox + Ee <= g.N[0] && oy + Ee <= g.N[1] && oz + Ee <= g.N[2];
        int got = -1;
        if (TA.tma && inside) {
            got = tma_region(tm, reinterpret_cast<unsigned char*>(reg), NR, (unsigned)(sizeof(float2) * E3),
                             (int)sizeof(float2), Ee, ox, oy, cfg * NR * g.N[2] + oz, g.N[2], TA.tma_zext, mbar, phase,
                             TA.tma_err);
            if (got == 0) return;
        }
        if (got < 0) {
            for (int u = threadIdx.x; u < NR * E3; u += kTileThreads) {
                const int c = u / E3, rem = u - c * E3;
                const int z = rem / E2, y = (rem / Ee) % Ee, x = rem % Ee;
                const size_t off = ((size_t)wrap_once(oz + z, g.N[2]) * g.N[1] + wrap_once(oy + y, g.N[1])) * g.N[0] +
                                   wrap_once(ox + x, g.N[0]);
                reg[u] = __ldg(gr + (size_t)c * g.G + off);
            }
            __syncthreads();
        }
        for (int t = a + w; t < b; t += kTileWarps) {
            const int bead = TA.sorted[p0 + t];
            const int4 st = A.start[bead];
            const DfWindows D = df_bead_windows<GRAD>(A, bead, lane);
            const int lx = st.x - ox, ly = st.y - oy, lz = st.z - oz;
            df sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) sp[c] = ex[c] = ey[c] = ez[c] = df{0.0f, 0.0f};
#pragma unroll
            for (int first = 0; first < P2; first += 32) {
                const int pair = first + lane;
                const bool on = pair < P2;
                int j = pair / P, i = pair - j * P;
                if (!on) i = j = 0;
                const df wx = df_shfl(D.wx, i), wy = df_shfl(D.wy, j);
                const df wxy = on ? df_mul(wx, wy) : df{0.0f, 0.0f};
                df dx = {0.0f, 0.0f}, dy = {0.0f, 0.0f};
                if (GRAD) {
                    dx = df_shfl(D.dx, i);
                    dy = df_shfl(D.dy, j);
                }
                const int base = (lz * Ee + ly + j) * Ee + lx + i;
                df sa[NR], sz[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) sa[c] = sz[c] = df{0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const df wz = df_shfl(D.wz, k);
                    df wdz = {0.0f, 0.0f};
                    if (GRAD) wdz = df_shfl(D.wdz, k);
                    if (on) {
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const float2 v = reg[c * E3 + base + k * E2];
                            const df vd = {v.x, v.y};
                            sa[c] = df_add(sa[c], df_mul(vd, wz));
                            if (GRAD) sz[c] = df_add(sz[c], df_mul(vd, wdz));
                        }
                    }
                }
                df_column_add<NR, GRAD>(wxy, dx, dy, sa, sz, sp, ex, ey, ez);
            }
            df_bead_store<NR, GRAD>(g, n, bead, lane, false, sp, ex, ey, ez, psi, E);
        }
        __syncthreads();
    }
}

template <typename T, int NR, bool GRAD, int PC>
__global__ void __launch_bounds__(kTileThreads)
gather_tiles_kernel(TileArgs TA, int n, const T* __restrict__ grid, double* __restrict__ psi, double* __restrict__ E,
                    const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char tile_smem_base[];
    // the region starts at the first 128-byte boundary of the dynamic shared memory
    // (a tensor copy's destination must be 128-byte aligned; kTmaPad bytes are reserved)
    unsigned char* tile_smem = tile_smem_base + ((128u - (smem_addr(tile_smem_base) & 127u)) & 127u);
    T* reg = reinterpret_cast<T*>(tile_smem);
    __shared__ TileRuns R;
    __shared__ uint64_t tma_bar;
    unsigned phase = 0;
    if (TA.tma && (smem_addr(tile_smem) & 127u) != 0u) {   // cannot happen: recorded, plain loads instead
        if (threadIdx.x == 0 && TA.tma_err) atomicExch(TA.tma_err, 2);
        TA.tma = false;
    }
    if (TA.tma) tma_barrier_init(&tma_bar);   // block-uniform
    const int p0 = blockIdx.x * TA.chunk;
    const int m = min(TA.chunk, n - p0);
    tile_runs(TA.key, p0, m, R);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const PairArgs& A = TA.A;
    const MeshGeom& g = A.g;
    bool dfg = false;   // FP64 potential as hi + lo floats: double-float throughout
    if constexpr (sizeof(T) == 8) dfg = A.gdf != nullptr;
    const bool v4x = (g.N[0] & 3) == 0;
    for (int t = w; t < m; t += kTileWarps) {
        const int r = R.of[t];
        if (R.start[r + 1] - R.start[r] < kTileMin) {
            if constexpr (sizeof(T) == 8) {
                if (dfg) {
                    gather_bead_df<NR, GRAD, PC>(A, n, TA.sorted[p0 + t], lane, psi, E);
                    continue;
                }
            }
            if constexpr (sizeof(T) == 4 && PC > 0) {
                if (v4x) {
                    gather_bead_v4<NR, GRAD, PC>(A, n, TA.sorted[p0 + t], lane, reinterpret_cast<const float*>(grid),
                                                 psi, E);
                    continue;
                }
            }
            gather_bead_direct<T, NR, GRAD, PC>(A, n, TA.sorted[p0 + t], lane, grid, psi, E);
        }
    }
    const int Ee = TA.E, E2 = Ee * Ee, E3 = E2 * Ee;
    const int P = PC ? PC : g.P, P2 = P * P;
    if constexpr (sizeof(T) == 8) {
        if (dfg) {
            gather_tiles_df<NR, GRAD, PC>(TA, R, p0, n, reinterpret_cast<float2*>(tile_smem), psi, E, &tmap, &tma_bar,
                                          phase);
            return;
        }
    }
    for (int r = 0; r < R.count; ++r) {
        const int a = R.start[r], b = R.start[r + 1];
        if (b - a < kTileMin) continue;   // block-uniform
        const int key = TA.key[p0 + a];
        const int tile = key % TA.ntiles, cfg = key / TA.ntiles;
        const int ox = (tile % TA.tn[0]) * kTileNodes;
        const int oy = ((tile / TA.tn[0]) % TA.tn[1]) * kTileNodes;
        const int oz = (tile / (TA.tn[0] * TA.tn[1])) * kTileNodes;
        const T* gr = grid + (size_t)cfg * NR * g.G;
        const bool inside = ox + Ee <= g.N[0] && oy + Ee <= g.N[1] && oz + Ee <= g.N[2];
        int got = -1;
        if (sizeof(T) == 4 && TA.tma && inside) {
            got = tma_region(&tmap, tile_smem, NR, (unsigned)(sizeof(T) * E3), (int)sizeof(T), Ee, ox, oy,
                             cfg * NR * g.N[2] + oz, g.N[2], TA.tma_zext, &tma_bar, phase, TA.tma_err);
            if (got == 0) return;
        }
        if (got < 0) {
            for (int u = threadIdx.x; u < NR * E3; u += kTileThreads) {
                const int c = u / E3, rem = u - c * E3;
                const int z = rem / E2, y = (rem / Ee) % Ee, x = rem % Ee;
                const size_t off = ((size_t)wrap_once(oz + z, g.N[2]) * g.N[1] + wrap_once(oy + y, g.N[1])) * g.N[0] +
                                   wrap_once(ox + x, g.N[0]);
                T v;
                if constexpr (sizeof(T) == 8) {
                    if (A.gdf) {
                        const float2 t = __ldg(A.gdf + (size_t)(cfg * NR + c) * g.G + off);
                        v = df_join(df{t.x, t.y});
                    } else {
                        v = __ldg(gr + (size_t)c * g.G + off);
                    }
                } else {
                    v = __ldg(gr + (size_t)c * g.G + off);
                }
                reg[u] = v;
            }
            __syncthreads();
        }
        for (int t = a + w; t < b; t += kTileWarps) {
            const int bead = TA.sorted[p0 + t];
            const int4 st = A.start[bead];
            const bool in = lane < P;
            T fx, fy, fz;
            bead_offsets<T>(A, bead, lane, fx, fy, fz);
            const T wx_l = bead_window<T>(A, bead, 0, fx, lane, in);
            const T wy_l = bead_window<T>(A, bead, 1, fy, lane, in);
            const T wz_l = bead_window<T>(A, bead, 2, fz, lane, in);
            const T dx_l = fx * cst<T>(g.h[0], A.h32[0]), dy_l = fy * cst<T>(g.h[1], A.h32[1]),
                    wdz_l = wz_l * (fz * cst<T>(g.h[2], A.h32[2]));
            const int lx = st.x - ox, ly = st.y - oy, lz = st.z - oz;
            T sp[NR], ex[NR], ey[NR], ez[NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) sp[c] = ex[c] = ey[c] = ez[c] = (T)0;
            #pragma unroll
    for (int first = 0; first < P2; first += 32) {
                const int pair = first + lane;
                const bool on = pair < P2;
                int j = pair / P, i = pair - j * P;
                if (!on) i = j = 0;
                const T wx = __shfl_sync(0xffffffffu, wx_l, i), wy = __shfl_sync(0xffffffffu, wy_l, j);
                const T wxy = on ? wx * wy : (T)0;
                T dx = (T)0, dy = (T)0;
                if (GRAD) {
                    dx = __shfl_sync(0xffffffffu, dx_l, i);
                    dy = __shfl_sync(0xffffffffu, dy_l, j);
                }
                const int base = (lz * Ee + ly + j) * Ee + lx + i;
                T acc[NR], accz[NR];
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] = accz[c] = (T)0;
                #pragma unroll
        for (int k = 0; k < P; ++k) {
                    const T wz = __shfl_sync(0xffffffffu, wz_l, k);
                    T wdz = (T)0;
                    if (GRAD) wdz = __shfl_sync(0xffffffffu, wdz_l, k);
                    if (on) {
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const T v = reg[c * E3 + base + k * E2];
                            acc[c] = fma(v, wz, acc[c]);
                            if (GRAD) accz[c] = fma(v, wdz, accz[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    sp[c] += wxy * acc[c];
                    if (GRAD) {
                        ex[c] += wxy * dx * acc[c];
                        ey[c] += wxy * dy * acc[c];
                        ez[c] += wxy * accz[c];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                const T s0 = warp_sum(sp[c]);
                if (GRAD) {
                    const T e0 = warp_sum(ex[c]);
                    const T e1 = warp_sum(ey[c]);
                    const T e2 = warp_sum(ez[c]);
                    if (lane == 0) {
                        double* e = E + ((size_t)c * n + bead) * 3;
                        e[0] = (double)(-cst<T>(g.grad, A.grad32) * e0);
                        e[1] = (double)(-cst<T>(g.grad, A.grad32) * e1);
                        e[2] = (double)(-cst<T>(g.grad, A.grad32) * e2);
                    }
                }
                if (lane == 0) psi[(size_t)c * n + bead] = (double)(cst<T>(g.gather, A.gather32) * s0);
            }
        }
        __syncthreads();
    }
}

// Blocks take fewer sorted beads when the beads are few, so that isolated
// beads (one warp each) still give every SM several blocks.
TileArgs tile_args(const MeshGeom& g, const StencilCache& b, int n) {
    TileArgs TA{};
    TA.chunk = n >= 152 * 4 * 128 ? 128 : (n >= 152 * 4 * 64 ? 64 : 32);
    pair_consts(TA.A, g, b);
    TA.A.wpb = 1;
    TA.A.rounds = (g.P * g.P + 31) / 32;
    TA.sorted = b.tile_sorted.as<int>();
    TA.key = b.tile_key.as<int>();
    for (int d = 0; d < 3; ++d) TA.tn[d] = b.tile_n[d];
    TA.ntiles = b.tile_n[0] * b.tile_n[1] * b.tile_n[2];
    TA.E = kTileNodes + g.P - 1;
    return TA;
}

template <typename T>
size_t tile_smem_bytes(const MeshGeom& g, int nrhs) {
    const size_t E = kTileNodes + g.P - 1;
    return sizeof(T) * (size_t)nrhs * E * E * E;
}

// Blocks of a tile kernel resident on the whole GPU at once (cached per kernel and
// shared-memory size; the dynamic shared memory attribute is set by then).
int tile_resident_blocks(const void* fn, size_t smem) {
    static std::map<std::pair<const void*, size_t>, int> cache;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 0, per = 0;
    IBP_CUDA(cudaGetDevice(&dev));
    IBP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IBP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kTileThreads, smem));
    const int r = std::max(1, per) * std::max(1, sms);
    cache.emplace(key, r);
    return r;
}

// Opt-in to more than 48 KB of dynamic shared memory for every tiled kernel,
// once per device (outside any stream capture: called when bins are built).
template <typename K>
void tile_smem_attr(K kernel) {
    IBP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemMax));
}

template <typename T, int NR>
void tile_attrs_nr() {
    tile_smem_attr(spread_tiles_kernel<T, NR, 0>);
    tile_smem_attr(gather_tiles_kernel<T, NR, true, 0>);
    tile_smem_attr(gather_tiles_kernel<T, NR, false, 0>);
    if constexpr (NR <= 3) {
        tile_smem_attr(spread_tiles_kernel<T, NR, 9>);
        tile_smem_attr(gather_tiles_kernel<T, NR, true, 9>);
        tile_smem_attr(gather_tiles_kernel<T, NR, false, 9>);
    }
}

template <typename T>
void tile_attrs() {
    tile_attrs_nr<T, 1>();
    tile_attrs_nr<T, 2>();
    tile_attrs_nr<T, 3>();
    tile_attrs_nr<T, 4>();
    tile_attrs_nr<T, 5>();
    tile_attrs_nr<T, 6>();
    tile_attrs_nr<T, 7>();
    tile_attrs_nr<T, 8>();
}

// The resident block counts of the tile kernels for this mesh's region size, queried
// here (outside any stream capture) so that launches inside captures find them cached.
template <typename T, int NR>
void tile_resident_nr(const MeshGeom& g) {
    const size_t b = tile_smem_bytes<T>(g, NR), bg = b + kTmaPad;
    if (bg > kTileSmemMax) return;
    tile_resident_blocks((const void*)spread_tiles_kernel<T, NR, 0>, b);
    tile_resident_blocks((const void*)gather_tiles_kernel<T, NR, true, 0>, bg);
    tile_resident_blocks((const void*)gather_tiles_kernel<T, NR, false, 0>, bg);
    if constexpr (NR <= 3) {
        if (g.P == 9) {
            tile_resident_blocks((const void*)spread_tiles_kernel<T, NR, 9>, b);
            tile_resident_blocks((const void*)gather_tiles_kernel<T, NR, true, 9>, bg);
            tile_resident_blocks((const void*)gather_tiles_kernel<T, NR, false, 9>, bg);
        }
    }
}

template <typename T>
void tile_resident(const MeshGeom& g) {
    tile_resident_nr<T, 1>(g);
    tile_resident_nr<T, 2>(g);
    tile_resident_nr<T, 3>(g);
    tile_resident_nr<T, 4>(g);
    tile_resident_nr<T, 5>(g);
    tile_resident_nr<T, 6>(g);
    tile_resident_nr<T, 7>(g);
    tile_resident_nr<T, 8>(g);
}

void tile_attrs_once() {
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    IBP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev) fail(IBPME_ERR_CUDA, "device ordinal %d out of range", dev);
    if (done[dev]) return;
    tile_attrs<float>();
    tile_attrs<double>();
    done[dev] = true;
}

template <typename T, int NR>
void launch_tiles(bool spread, bool grad, const TileArgs& TA0, int n, const double* q, T* grid, double* psi,
                  double* E, cudaStream_t s, const CUtensorMap* tm) {
    CUtensorMap tmv;
    memset(&tmv, 0, sizeof(tmv));
    if (tm) tmv = *tm;
    const size_t bytes = tile_smem_bytes<T>(TA0.A.g, NR) + (spread ? 0 : kTmaPad);
    bool p9 = false;
    if constexpr (NR <= 3) p9 = TA0.A.g.P == 9;
    const void* fn;
    if (spread) fn = p9 ? (const void*)spread_tiles_kernel<T, NR, 9> : (const void*)spread_tiles_kernel<T, NR, 0>;
    else if (grad) fn = p9 ? (const void*)gather_tiles_kernel<T, NR, true, 9> : (const void*)gather_tiles_kernel<T, NR, true, 0>;
    else fn = p9 ? (const void*)gather_tiles_kernel<T, NR, false, 9> : (const void*)gather_tiles_kernel<T, NR, false, 0>;
    // beads per block so that the grid fills whole waves of resident blocks (a
    // partial last wave runs at the cost of a full one)
    TileArgs TA = TA0;
    const int resident = tile_resident_blocks(fn, bytes);
    const int waves = div_up(n, resident * kTileChunk);
    TA.chunk = std::max(1, std::min(kTileChunk, div_up(n, waves * resident)));
    const int blocks = div_up(n, TA.chunk);
    if (spread) {
        if constexpr (NR <= 3) {
            if (p9) {
                spread_tiles_kernel<T, NR, 9><<<blocks, kTileThreads, bytes, s>>>(TA, n, q, grid);
                return;
            }
        }
        spread_tiles_kernel<T, NR, 0><<<blocks, kTileThreads, bytes, s>>>(TA, n, q, grid);
    } else if (grad) {
        if constexpr (NR <= 3) {
            if (p9) {
                gather_tiles_kernel<T, NR, true, 9><<<blocks, kTileThreads, bytes, s>>>(TA, n, grid, psi, E, tmv);
                return;
            }
        }
        gather_tiles_kernel<T, NR, true, 0><<<blocks, kTileThreads, bytes, s>>>(TA, n, grid, psi, E, tmv);
    } else {
        if constexpr (NR <= 3) {
            if (p9) {
                gather_tiles_kernel<T, NR, false, 9><<<blocks, kTileThreads, bytes, s>>>(TA, n, grid, psi, nullptr, tmv);
                return;
            }
        }
        gather_tiles_kernel<T, NR, false, 0><<<blocks, kTileThreads, bytes, s>>>(TA, n, grid, psi, nullptr, tmv);
    }
}

template <typename T>
void tiles_dispatch(int nrhs, bool spread, bool grad, const TileArgs& TA, int n, const double* q, T* grid,
                    double* psi, double* E, cudaStream_t s, const CUtensorMap* tm = nullptr) {
    switch (nrhs) {
        case 1: launch_tiles<T, 1>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 2: launch_tiles<T, 2>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 3: launch_tiles<T, 3>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 4: launch_tiles<T, 4>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 5: launch_tiles<T, 5>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 6: launch_tiles<T, 6>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        case 7: launch_tiles<T, 7>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
        default: launch_tiles<T, 8>(spread, grad, TA, n, q, grid, psi, E, s, tm); break;
    }
}

// The tensor map of the grid the tiled gathers read (base: the FP32 grid, or the
// double-float potential as (hi, lo) pairs of es = 8 bytes), built once per buffer and
// channel count; NULL when a region's box cannot be copied by TMA (the box edge or a
// grid row not a multiple of 16 bytes, a region larger than the grid) or IBPME_NO_TMA
// is set (the switch lets tests compare both paths).
const CUtensorMap* grid_tmap(unsigned char* bytes, const void*& tm_base, int& tm_ch, int& tm_es, int& tm_E,
                             bool& tm_ok, const MeshGeom& g, const void* base, int channels, int es) {
    if (std::getenv("IBPME_NO_TMA") != nullptr) return nullptr;
    const int E = kTileNodes + g.P - 1;
    if (tm_base == base && tm_ch == channels && tm_es == es && tm_E == E) {
        return tm_ok ? reinterpret_cast<const CUtensorMap*>(bytes) : nullptr;
    }
    tm_base = base;
    tm_ch = channels;
    tm_es = es;
    tm_E = E;
    tm_ok = false;
    if ((E * es) % 16 != 0 || ((size_t)g.N[0] * es) % 16 != 0 || E > 256 || E > g.N[0] || E > g.N[1] ||
        E > g.N[2] || (reinterpret_cast<size_t>(base) & 15) != 0)
        return nullptr;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn) {
                cudaGetLastError();
                return nullptr;
            }
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    const cuuint64_t dims[3] = {(cuuint64_t)g.N[0], (cuuint64_t)g.N[1], (cuuint64_t)g.N[2] * (cuuint64_t)channels};
    const cuuint64_t strides[2] = {(cuuint64_t)g.N[0] * es, (cuuint64_t)g.N[0] * g.N[1] * es};
    const cuuint32_t box[3] = {(cuuint32_t)E, (cuuint32_t)E, (cuuint32_t)E};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(bytes);
    const CUresult r = encode(m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                              const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    tm_ok = r == CUDA_SUCCESS;
    return tm_ok ? m : nullptr;
}

// The tiled path serves a call when the cache holds tile bins and the region of
// all its channels fits in shared memory.
template <typename T>
bool tiles_fit(const MeshGeom& g, const StencilCache* sc, int nrhs) {
    return sc && sc->tiles && nrhs <= 8 && tile_smem_bytes<T>(g, nrhs) + kTmaPad <= kTileSmemMax;
}

// |k| of half-spectrum entry t (x fastest, N_x / 2 + 1 entries per row).
__device__ __forceinline__ double half_spectrum_k2(const MeshGeom& g, long long t) {
    const int nxh = g.N[0] / 2 + 1;
    const double two_pi = 6.283185307179586476925286766559;
    const int kx_i = (int)(t % nxh);
    const long long rest = t / nxh;
    const int ky_i = (int)(rest % g.N[1]);
    const int kz_i = (int)(rest / g.N[1]);
    const int my = ky_i <= g.N[1] / 2 ? ky_i : ky_i - g.N[1];
    const int mz = kz_i <= g.N[2] / 2 ? kz_i : kz_i - g.N[2];
    const double kx = two_pi * kx_i / g.L[0], ky = two_pi * my / g.L[1], kz = two_pi * mz / g.L[2];
    return kx * kx + ky * ky + kz * kz;
}

// G(k)/(N_x N_y N_z) on the half spectrum, Eq. after H_hat:
// j0^2(k a) e^{-(1 - eta) k^2 / (4 xi^2)} / k^2, zero at k = 0 (Sec. II, k = 0 removed).
// a = 0 leaves the j0^2 factor out (radius classes apply theirs in mix_kernel).
template <typename T>
__global__ void green_kernel(MeshGeom g, double xi, double eta, double a, T* __restrict__ green) {
    const int nxh = g.N[0] / 2 + 1;
    const double two_pi = 6.283185307179586476925286766559;
    const double norm = 1.0 / ((double)g.N[0] * g.N[1] * g.N[2]);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.Gc;
         t += (long long)gridDim.x * blockDim.x) {
        const int kx_i = (int)(t % nxh);
        const long long rest = t / nxh;
        const int ky_i = (int)(rest % g.N[1]);
        const int kz_i = (int)(rest / g.N[1]);
        const int my = ky_i <= g.N[1] / 2 ? ky_i : ky_i - g.N[1];
        const int mz = kz_i <= g.N[2] / 2 ? kz_i : kz_i - g.N[2];
        const double kx = two_pi * kx_i / g.L[0], ky = two_pi * my / g.L[1], kz = two_pi * mz / g.L[2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        double v = 0.0;
        if (k2 > 0.0) {
            const double k = sqrt(k2);
            const double j0 = a > 0.0 ? sin(k * a) / (k * a) : 1.0;
            v = j0 * j0 * exp(-(1.0 - eta) * k2 / (4.0 * xi * xi)) / k2 * norm;
        }
        green[t] = (T)v;
    }
}

// j0(k a_c) = sin(k a_c) / (k a_c) of every class on the half spectrum (1 at k = 0).
struct ClassRadii {
    double a[IBPME_MAX_RADIUS_CLASSES];
};

template <typename T>
__global__ void class_j0_kernel(MeshGeom g, int ncls, ClassRadii R, T* __restrict__ jtab) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.Gc;
         t += (long long)gridDim.x * blockDim.x) {
        const double k = sqrt(half_spectrum_k2(g, t));
        for (int c = 0; c < ncls; ++c) {
            const double x = k * R.a[c];
            jtab[(size_t)c * g.Gc + t] = (T)(x > 0.0 ? sin(x) / x : 1.0);
        }
    }
}

// RPY wave space: the three force channels F(k) become fac (1 + k^2/(4 xi^2)) G(k)
// (I - k_hat k_hat) F(k) (Hasimoto's weight; G carries j0^2(ka) and the window's
// e^{-(1 - eta) k^2/(4 xi^2)}); zero at k = 0.
template <typename T>
__global__ void rpy_project_kernel(MeshGeom g, double fac, double xi, const T* __restrict__ green,
                                   typename Cplx<T>::type* __restrict__ spec) {
    const int nxh = g.N[0] / 2 + 1;
    const T two_pi = (T)6.283185307179586476925286766559;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.Gc;
         t += (long long)gridDim.x * blockDim.x) {
        const int kx_i = (int)(t % nxh);
        const long long rest = t / nxh;
        const int ky_i = (int)(rest % g.N[1]);
        const int kz_i = (int)(rest / g.N[1]);
        const int my = ky_i <= g.N[1] / 2 ? ky_i : ky_i - g.N[1];
        const int mz = kz_i <= g.N[2] / 2 ? kz_i : kz_i - g.N[2];
        const T k[3] = {two_pi * kx_i / (T)g.L[0], two_pi * my / (T)g.L[1], two_pi * mz / (T)g.L[2]};
        const T k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        typename Cplx<T>::type v[3];
        for (int c = 0; c < 3; ++c) v[c] = spec[(size_t)c * g.Gc + t];
        typename Cplx<T>::type o[3];
        if (k2 > (T)0) {
            const T w = green[t] * ((T)1 + k2 / (T)(4.0 * xi * xi)) * (T)fac;
            const T kr = k[0] * v[0].x + k[1] * v[1].x + k[2] * v[2].x;   // k . F
            const T ki = k[0] * v[0].y + k[1] * v[1].y + k[2] * v[2].y;
            for (int c = 0; c < 3; ++c) {
                o[c].x = w * (v[c].x - k[c] * kr / k2);
                o[c].y = w * (v[c].y - k[c] * ki / k2);
            }
        } else {
            for (int c = 0; c < 3; ++c) o[c].x = o[c].y = (T)0;
        }
        for (int c = 0; c < 3; ++c) spec[(size_t)c * g.Gc + t] = o[c];
    }
}

// Scaling with radius classes (the pair kernel j0(k a_c) j0(k a_d) G(k)): for each
// right-hand side r, S = sum_c j0(k a_c) H_hat(c, r), then channel (d, r) becomes
// G(k) j0(k a_d) S.  The source and the target factor of every pair are applied, so
// each bead's gather from its own class's channel sees every class's charges.
template <typename T>
__global__ void mix_kernel(long long Gc, int nrhs, int ncls, const T* __restrict__ green, const T* __restrict__ jtab,
                           typename Cplx<T>::type* __restrict__ spec) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Gc; t += (long long)gridDim.x * blockDim.x) {
        const T gk = green[t];
        T j[IBPME_MAX_RADIUS_CLASSES];
        for (int c = 0; c < ncls; ++c) j[c] = jtab[(size_t)c * Gc + t];
        for (int r = 0; r < nrhs; ++r) {
            T sx = 0, sy = 0;
            for (int c = 0; c < ncls; ++c) {
                const typename Cplx<T>::type v = spec[(size_t)(c * nrhs + r) * Gc + t];
                sx += j[c] * v.x;
                sy += j[c] * v.y;
            }
            for (int d = 0; d < ncls; ++d) {
                const T f = gk * j[d];
                typename Cplx<T>::type o;
                o.x = f * sx;
                o.y = f * sy;
                spec[(size_t)(d * nrhs + r) * Gc + t] = o;
            }
        }
    }
}

// The FP64 Green's table as unevaluated sums hi + lo of floats.
__global__ void green_split_kernel(long long Gc, const double* __restrict__ green, float2* __restrict__ out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Gc; t += (long long)gridDim.x * blockDim.x) {
        const double v = green[t];
        const float hi = (float)v;
        out[t] = make_float2(hi, (float)(v - (double)hi));
    }
}

// Scaling of the half spectrum by the Green's table; blockIdx.y is the
// right-hand side, so the table index needs no division.
template <typename T>
__global__ void scale_kernel(long long Gc, const T* __restrict__ green, typename Cplx<T>::type* __restrict__ spec) {
    typename Cplx<T>::type* sp = spec + (size_t)blockIdx.y * Gc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Gc; t += (long long)gridDim.x * blockDim.x) {
        const T gk = green[t];
        typename Cplx<T>::type v = sp[t];
        v.x *= gk;
        v.y *= gk;
        sp[t] = v;
    }
}

int grid_blocks(long long work, int threads) {
    long long b = (work + threads - 1) / threads;
    const long long cap = 152LL * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

template <typename T>
void Mesh<T>::init(const MeshGeom& geom, int channels, double xi, double eta, double a, cudaStream_t s, int nc,
                   const double* cls_a) {
    g = geom;
    rcap = 0;
    ncls = nc > 1 ? nc : 1;
    if (!tma_err_host) {   // here, outside any stream capture (the gathers only write it)
        IBP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&tma_err_host), sizeof(int), cudaHostAllocMapped));
        *tma_err_host = 0;
        IBP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&tma_err_dev), tma_err_host, 0));
    }
    df = sizeof(T) == 8 && df_fft_supported(g);
    if (df) df_fft_init(g, df_tw, s);
    ensure_channels(channels * ncls);
    green.ensure(sizeof(T) * (size_t)g.Gc);
    green_kernel<T><<<grid_blocks(g.Gc, 256), 256, 0, s>>>(g, xi, eta, ncls > 1 ? 0.0 : a, green.as<T>());
    IBP_CHECK_LAUNCH();
    if (ncls > 1) {
        ClassRadii R{};
        for (int c = 0; c < ncls; ++c) R.a[c] = cls_a[c];
        jtab.ensure(sizeof(T) * (size_t)g.Gc * ncls);
        class_j0_kernel<T><<<grid_blocks(g.Gc, 256), 256, 0, s>>>(g, ncls, R, jtab.as<T>());
        IBP_CHECK_LAUNCH();
    }
    if constexpr (sizeof(T) == 8) {
        if (df) {
            green_df.ensure(sizeof(float2) * (size_t)g.Gc);
            green_split_kernel<<<grid_blocks(g.Gc, 256), 256, 0, s>>>(g.Gc, green.as<double>(), green_df.as<float2>());
            IBP_CHECK_LAUNCH();
            if (ncls > 1) {
                jtab_df.ensure(sizeof(float2) * (size_t)g.Gc * ncls);
                green_split_kernel<<<grid_blocks(g.Gc * ncls, 256), 256, 0, s>>>(g.Gc * ncls, jtab.as<double>(),
                                                                                  jtab_df.as<float2>());
                IBP_CHECK_LAUNCH();
            }
        }
    }
}

template <typename T>
void Mesh<T>::ensure_channels(int ch) {
    if (ch <= rcap) return;
    grid.ensure(sizeof(T) * (size_t)g.G * ch);
    if (df) grid_df.ensure(sizeof(float2) * (size_t)g.G * ch);
    spec.ensure(sizeof(typename Cplx<T>::type) * (size_t)g.Gc * ch);
    rcap = ch;
}

template <typename T>
void Mesh<T>::plans(int ch, cudaStream_t s) {
    if (ch < 1) fail(IBPME_ERR_ARG, "channel count %d < 1", ch);
    ensure_channels(ch);
    if (df) {   // double-float transforms: one complex float4 buffer, no cuFFT plan
        df_buf.ensure(sizeof(float4) * (size_t)g.G * ch);
        return;
    }
    auto it = plan.find(ch);
    if (it == plan.end()) {
        int dims[3] = {g.N[2], g.N[1], g.N[0]};   // slowest to fastest: z, y, x
        const cufftType tf = sizeof(T) == 8 ? CUFFT_D2Z : CUFFT_R2C;
        const cufftType tb = sizeof(T) == 8 ? CUFFT_Z2D : CUFFT_C2R;
        size_t ws1 = 0, ws2 = 0;
        cufftHandle f = 0, b = 0;
        IBP_CUFFT(cufftCreate(&f));
        IBP_CUFFT(cufftCreate(&b));
        IBP_CUFFT(cufftSetAutoAllocation(f, 0));
        IBP_CUFFT(cufftSetAutoAllocation(b, 0));
        IBP_CUFFT(cufftMakePlanMany(f, 3, dims, nullptr, 1, (int)g.G, nullptr, 1, (int)g.Gc, tf, ch, &ws1));
        IBP_CUFFT(cufftMakePlanMany(b, 3, dims, nullptr, 1, (int)g.Gc, nullptr, 1, (int)g.G, tb, ch, &ws2));
        it = plan.emplace(ch, std::make_pair(f, b)).first;
        const size_t need = ws1 > ws2 ? ws1 : ws2;
        if (need > work.bytes) {
            work.ensure(need);
            for (auto& kv : plan) {
                IBP_CUFFT(cufftSetWorkArea(kv.second.first, work.p));
                IBP_CUFFT(cufftSetWorkArea(kv.second.second, work.p));
            }
        } else {
            IBP_CUFFT(cufftSetWorkArea(f, work.p));
            IBP_CUFFT(cufftSetWorkArea(b, work.p));
        }
    }
    IBP_CUFFT(cufftSetStream(it->second.first, s));
    IBP_CUFFT(cufftSetStream(it->second.second, s));
}

template <typename T>
void Mesh<T>::destroy() {
    for (auto& kv : plan) {
        cufftDestroy(kv.second.first);
        cufftDestroy(kv.second.second);
    }
    plan.clear();
    df_buf.release();
    for (auto& t : df_tw) t.release();
    grid.release();
    spec.release();
    green.release();
    jtab.release();
    jtab_df.release();
    green_df.release();
    grid_df.release();
    potential_df = false;
    work.release();
    rcap = 0;
    if (tma_err_host) cudaFreeHost(tma_err_host);
    tma_err_host = nullptr;
    tma_err_dev = nullptr;
    tm_base = nullptr;
    tm_ok = false;
}

template <typename T>
void Mesh<T>::spread(int n, const double* xw, const double* q, int nrhs, const int* bead_cfg, int ncfg,
                     cudaStream_t s, const StencilCache* sc, bool accumulate) {
    ProfScope ps(mesh_stage<T>(ST_SPREAD), s);
    ensure_channels(nrhs * ncfg);
    potential_df = false;
    ++writes;
    if (!accumulate) IBP_CUDA(cudaMemsetAsync(grid.p, 0, sizeof(T) * (size_t)g.G * nrhs * ncfg, s));
    if (n == 0) return;
    // Pair lanes while a bead's columns are split over warps (few beads); with one
    // warp per bead the row-walking kernel keeps its atomics of consecutive
    // instructions within one z-plane, which measured faster on dense surfaces.
    const PairArgs A = sc ? pair_args(g, *sc, n) : PairArgs{};
    if (tiles_fit<T>(g, sc, nrhs)) {
        tiles_dispatch<T>(nrhs, true, false, tile_args(g, *sc, n), n, q, grid.as<T>(), nullptr, nullptr, s);
    } else if (sc && A.wpb > 1) {
        pairs_dispatch<T>(nrhs, true, false, A, n, q, grid.as<T>(), nullptr, nullptr, s);
    } else {
        spread_dispatch<T>(n, xw, q, nrhs, bead_cfg, g, grid.as<T>(), s);
    }
    IBP_CHECK_LAUNCH();
}

template <typename T>
void Mesh<T>::transform(int ch, cudaStream_t s) {
    plans(ch, s);
    if constexpr (sizeof(T) == 8) {
        if (df) {
            df_fft_convolve(g, ch, green_df.as<float2>(), grid.as<double>(), grid_df.as<float2>(), df_buf.as<float4>(),
                            df_tw, s, ncls, jtab_df.as<float2>());
            potential_df = true;
            return;
        }
    }
    potential_df = false;
    const auto& pl = plan.at(ch);
    using C = typename Cplx<T>::type;
    {
        ProfScope ps(mesh_stage<T>(ST_FFT_FWD), s);
        if constexpr (sizeof(T) == 8) {
            IBP_CUFFT(cufftExecD2Z(pl.first, grid.as<double>(), spec.as<C>()));
        } else {
            IBP_CUFFT(cufftExecR2C(pl.first, grid.as<float>(), spec.as<C>()));
        }
    }
    {
        ProfScope ps(mesh_stage<T>(ST_SCALE), s);
        if (ncls > 1) {
            if (ch % ncls) fail(IBPME_ERR_ARG, "internal: %d channels for %d radius classes", ch, ncls);
            mix_kernel<T><<<grid_blocks(g.Gc, 256), 256, 0, s>>>(g.Gc, ch / ncls, ncls, green.as<T>(), jtab.as<T>(),
                                                               spec.as<C>());
        } else {
            scale_kernel<T><<<dim3(grid_blocks(g.Gc, 256), ch), 256, 0, s>>>(g.Gc, green.as<T>(), spec.as<C>());
        }
        IBP_CHECK_LAUNCH();
    }
    ProfScope ps(mesh_stage<T>(ST_FFT_INV), s);
    if constexpr (sizeof(T) == 8) {
        IBP_CUFFT(cufftExecZ2D(pl.second, spec.as<C>(), grid.as<double>()));
    } else {
        IBP_CUFFT(cufftExecC2R(pl.second, spec.as<C>(), grid.as<float>()));
    }
}

template <typename T>
void Mesh<T>::transform_rpy(double fac, double xi, cudaStream_t s) {
    if (ncls > 1) fail(IBPME_ERR_UNEQUAL_RADII, "the RPY mobility takes one bead radius");
    plans(3, s);
    if constexpr (sizeof(T) == 8) {
        if (df) {
            RpyScale R{{g.L[0], g.L[1], g.L[2]}, xi, fac};
            df_fft_convolve(g, 3, green_df.as<float2>(), grid.as<double>(), grid_df.as<float2>(), df_buf.as<float4>(),
                            df_tw, s, 1, nullptr, &R);
            potential_df = true;
            return;
        }
    }
    potential_df = false;
    const auto& pl = plan.at(3);
    using C = typename Cplx<T>::type;
    {
        ProfScope ps(mesh_stage<T>(ST_FFT_FWD), s);
        if constexpr (sizeof(T) == 8) {
            IBP_CUFFT(cufftExecD2Z(pl.first, grid.as<double>(), spec.as<C>()));
        } else {
            IBP_CUFFT(cufftExecR2C(pl.first, grid.as<float>(), spec.as<C>()));
        }
    }
    {
        ProfScope ps(mesh_stage<T>(ST_SCALE), s);
        rpy_project_kernel<T><<<grid_blocks(g.Gc, 256), 256, 0, s>>>(g, fac, xi, green.as<T>(), spec.as<C>());
        IBP_CHECK_LAUNCH();
    }
    ProfScope ps(mesh_stage<T>(ST_FFT_INV), s);
    if constexpr (sizeof(T) == 8) {
        IBP_CUFFT(cufftExecZ2D(pl.second, spec.as<C>(), grid.as<double>()));
    } else {
        IBP_CUFFT(cufftExecC2R(pl.second, spec.as<C>(), grid.as<float>()));
    }
}

template <typename T>
void Mesh<T>::gather(int n, const double* xw, int nrhs, const int* bead_cfg, double* psi, double* E,
                     cudaStream_t s, const StencilCache* sc) {
    if (n == 0) return;
    ProfScope ps(mesh_stage<T>(ST_GATHER), s);
    // the double-float transforms leave the potential as hi + lo floats
    const float2* gdf = sizeof(T) == 8 && potential_df ? grid_df.as<float2>() : nullptr;
    if (tiles_fit<T>(g, sc, nrhs)) {
        TileArgs TA = tile_args(g, *sc, n);
        TA.A.gdf = gdf;
        const CUtensorMap* tm = nullptr;
        if ((sizeof(T) == 4 || gdf) && tma_err_dev) {
            tm = gdf ? grid_tmap(tmap, tm_base, tm_ch, tm_es, tm_E, tm_ok, g, grid_df.p, rcap, 8)
                     : grid_tmap(tmap, tm_base, tm_ch, tm_es, tm_E, tm_ok, g, grid.p, rcap, 4);
        }
        TA.tma = tm != nullptr;
        TA.tma_err = tma_err_dev;
        TA.tma_zext = g.N[2] * rcap;
        tiles_dispatch<T>(nrhs, false, E != nullptr, TA, n, nullptr, grid.as<T>(), psi, E, s, tm);
        IBP_CHECK_LAUNCH();
        return;
    }
    if (sc) {   // several warps of a bead add their partial sums into zeroed outputs
        PairArgs A = pair_args(g, *sc, n);
        A.gdf = gdf;
        if (A.wpb > 1) {
            IBP_CUDA(cudaMemsetAsync(psi, 0, sizeof(double) * (size_t)nrhs * n, s));
            if (E) IBP_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * 3 * (size_t)nrhs * n, s));
        }
        pairs_dispatch<T>(nrhs, false, E != nullptr, A, n, nullptr, grid.as<T>(), psi, E, s);
        IBP_CHECK_LAUNCH();
        return;
    }
    if (E)
        gather_dispatch<T, true>(n, xw, nrhs, bead_cfg, g, grid.as<T>(), gdf, psi, E, s);
    else
        gather_dispatch<T, false>(n, xw, nrhs, bead_cfg, g, grid.as<T>(), gdf, psi, nullptr, s);
    IBP_CHECK_LAUNCH();
}

template <typename T>
int Mesh<T>::tma_failed() {
    if (!tma_err_host || *tma_err_host == 0) return 0;
    const int v = *tma_err_host;
    *tma_err_host = 0;
    return v;
}

template struct Mesh<float>;
template struct Mesh<double>;

namespace {

// Stencils (and tile bins) of n beads at xw, bead b of configuration bcfg[b], into b.
void build_stencils(ibpme_ctx* c, StencilCache& b, int n, const double* xw, const int* bcfg) {
    const MeshGeom& g = c->mesh64.g;   // both meshes share N, h and P
    b.valid = false;
    int4* start = static_cast<int4*>(b.start.ensure(sizeof(int4) * n));
    double4* frac = static_cast<double4*>(b.frac.ensure(sizeof(double4) * n));
    float4* frac32 = static_cast<float4*>(b.frac32.ensure(sizeof(float4) * n));
    double* w64 = static_cast<double*>(b.w64.ensure(sizeof(double) * 3 * (size_t)g.P * n));
    float2* wdf = static_cast<float2*>(b.wdf.ensure(sizeof(float2) * 3 * (size_t)g.P * n));
    float4* frac_df = static_cast<float4*>(b.frac_df.ensure(sizeof(float4) * 2 * (size_t)n));
    stencil_cache_kernel<<<div_up(3LL * n, 128), 128, 0, c->stream>>>(n, xw, bcfg, g, start, frac, frac32, w64,
                                                                     wdf, frac_df);
    IBP_CHECK_LAUNCH();
    // tile bins when one warp per bead already fills the GPU and a region of
    // E^3 nodes does not wrap onto itself
    const int E = kTileNodes + g.P - 1;
    const long long blocks32 = (g.P * g.P + 31) / 32;
    b.tiles = (long long)n * blocks32 > 152LL * 64 * 2 && g.N[0] >= E && g.N[1] >= E && g.N[2] >= E &&
              std::getenv("IBPME_NO_TILES") == nullptr;   // the switch lets tests compare both paths
    if (b.tiles) {
        for (int d = 0; d < 3; ++d) b.tile_n[d] = div_up(g.N[d], kTileNodes);
        const long long nkeys = (long long)b.tile_n[0] * b.tile_n[1] * b.tile_n[2] * mesh_groups(c);
        if (nkeys > (1LL << 30)) {
            b.tiles = false;
        } else {
            tile_attrs_once();
            tile_resident<float>(g);
            tile_resident<double>(g);
            const int nk = (int)nkeys;
            int* count = static_cast<int*>(b.tile_count.ensure(sizeof(int) * nk));
            int* cursor = static_cast<int*>(b.tile_cursor.ensure(sizeof(int) * nk));
            long long* off = static_cast<long long*>(b.tile_off.ensure(sizeof(long long) * (nk + 1)));
            int* bkey = static_cast<int*>(b.tile_bkey.ensure(sizeof(int) * n));
            int* sorted = static_cast<int*>(b.tile_sorted.ensure(sizeof(int) * n));
            int* skey = static_cast<int*>(b.tile_key.ensure(sizeof(int) * n));
            IBP_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * nk, c->stream));
            IBP_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * nk, c->stream));
            tile_count_kernel<<<div_up(n, 256), 256, 0, c->stream>>>(n, start, b.tile_n[0], b.tile_n[1], b.tile_n[2],
                                                                     count, bkey);
            IBP_CHECK_LAUNCH();
            scan_counts(count, off, nk, b.tile_tmp, c->stream);
            tile_fill_kernel<<<div_up(n, 256), 256, 0, c->stream>>>(n, bkey, off, cursor, sorted, skey);
            IBP_CHECK_LAUNCH();
        }
    }
    b.fp = c->near.fp;
    b.n = n;
    b.ncfg = mesh_groups(c);
    b.cls_key = cls_key(c);
    b.valid = true;
}

}  // namespace

const StencilCache* stencil_cache(ibpme_ctx* c, int n, const double* xw) {
    if (n == 0 || !c->near.fp_valid) return nullptr;   // no fingerprint of these positions: no cache key
    StencilCache& b = c->stencils;
    if (b.valid && b.fp == c->near.fp && b.n == n && b.ncfg == mesh_groups(c) && b.cls_key == cls_key(c)) return &b;
    build_stencils(c, b, n, xw, mesh_cfg(c));
    return &b;
}

const StencilCache* free_stencil_cache(ibpme_ctx* c) {
    const FreeSet& fs = c->fs;
    const int n = fs.nfree;
    if (n == 0 || !fs.valid) return nullptr;
    StencilCache& b = c->fs.sc;
    if (b.valid && b.fp == c->near.fp && b.n == n && b.ncfg == mesh_groups(c) && b.cls_key == cls_key(c)) return &b;
    const int* grp = c->ncls > 1 ? c->fs.cls_f.as<int>() : (c->ncfg > 1 ? c->bodies.free_cfg.as<int>() : nullptr);
    build_stencils(c, b, n, fs.xf.as<double>(), grp);
    return &b;
}

}  // namespace ibp


// ---------------------------------------------------------------------------
// Spreading for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs while a stream
// is being captured into a CUDA graph, engines whose device memory is owned
// by a pool or framework (for example a custom call inside a compiler-managed
// program), or loops that must never reach the allocator.  pme_spread needs a
// context, and the context allocates its meshes and scratch.  The variant
// below does the same spreading but keeps its only scratch -- the positions
// wrapped into the box -- in a fixed array compiled into the library, and
// writes straight into the caller's grid.
// ---------------------------------------------------------------------------
namespace ibp {

namespace {

// Scratch of pme_spread_noalloc: wrapped positions, [n][3] doubles for at
// most IBPME_NOALLOC_MAX_BEADS beads (6 MiB).  Every GPU that loads the
// library holds it until the process exits.  All calls share it.
static __device__ __align__(256) double g_noalloc_xw[3 * IBPME_NOALLOC_MAX_BEADS];

// Device address of g_noalloc_xw on each device, looked up once per device
// (host code cannot use the symbol's name as a device pointer).
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

double* noalloc_scratch(int dev) {
    if (dev < 0 || dev >= kMaxDevices) fail(IBPME_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_xw);
        if (e != cudaSuccess || !ptr)
            fail(IBPME_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_xw) failed on device %d: %s", dev,
                 cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<double*>(ptr);
    }
    return g_noalloc_ptr[dev];
}

__global__ void noalloc_wrap_kernel(int n, const double* __restrict__ x, double L0, double L1, double L2,
                                    double* __restrict__ xw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int d = i % 3;
    xw[i] = wrap_coord(x[i], d == 0 ? L0 : (d == 1 ? L1 : L2));
}

bool device_resident(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace ibp

IBP_API ibpme_status pme_spread_noalloc(const ibpme_params* params, int n, const double* x, const double* q,
                                        int nrhs, void* grid_out, void* cuda_stream) {
    using namespace ibp;
    try {
        set_error("%s", "");
        if (!params) fail(IBPME_ERR_ARG, "params is NULL");
        ibpme_params p{};
        resolve_params(params, &p);
        if (n < 0 || n > IBPME_NOALLOC_MAX_BEADS)
            fail(IBPME_ERR_ARG, "n = %d outside 0..%d, the fixed scratch of pme_spread_noalloc", n,
                 IBPME_NOALLOC_MAX_BEADS);
        if (nrhs < 1 || nrhs > kMaxRhs) fail(IBPME_ERR_ARG, "nrhs %d outside 1..%d", nrhs, kMaxRhs);
        if (!grid_out) fail(IBPME_ERR_ARG, "grid_out is required");
        if (n > 0 && (!x || !q)) fail(IBPME_ERR_ARG, "x and q are required");
        // no staging here: every array must already be on the device
        if (!device_resident(grid_out) || (n > 0 && (!device_resident(x) || !device_resident(q))))
            fail(IBPME_ERR_ARG, "pme_spread_noalloc takes device pointers only");
        int dev = 0;
        IBP_CUDA(cudaGetDevice(&dev));
        double* xw = noalloc_scratch(dev);
        const MeshGeom g = make_geom(p);
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        const bool f64 = p.precision == IBPME_FP64;
        IBP_CUDA(cudaMemsetAsync(grid_out, 0, (f64 ? sizeof(double) : sizeof(float)) * (size_t)g.G * nrhs, s));
        if (n > 0) {
            noalloc_wrap_kernel<<<div_up(3LL * n, 256), 256, 0, s>>>(n, x, p.box[0], p.box[1], p.box[2], xw);
            IBP_CHECK_LAUNCH();
            if (f64)
                spread_dispatch<double>(n, xw, q, nrhs, nullptr, g, static_cast<double*>(grid_out), s);
            else
                spread_dispatch<float>(n, xw, q, nrhs, nullptr, g, static_cast<float*>(grid_out), s);
            IBP_CHECK_LAUNCH();
        }
        return IBPME_OK;
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        set_error("unexpected internal exception");
        return IBPME_ERR_CUDA;
    }
}
