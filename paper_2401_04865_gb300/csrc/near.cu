// near.cu -- real-space half of the spectral Ewald sum (Sec. III.D.1, step 1
// of Sec. III.D.3): linked cells of side >= r_c, a CSR table of the pairs
// within r_c (minimum image) with the FP64 pair kernel and its radial
// derivative, and the SpMV / field passes that apply it.
//
// The table is built once per set of positions and reused by every Krylov
// iteration of a solve; GB300's FP64 rate makes re-evaluating erfc/exp per
// iteration far slower than streaming the stored values.
//
// Pair kernel.  The seven printed terms of Eq. psi_Re_1 (Heaviside sign read
// as -1/(4 pi r) + (4a - r)/(16 pi a^2)) regroup into a second difference:
//   phi_r(r) = [g(r + 2a) + g(r - 2a) - 2 g(r)] / r + H-term,
//   g(u) = -A u e^{-u^2 xi^2} + B (2 xi^2 u^2 + 1) erfc(u xi),
//   A = 1/(32 pi^{3/2} a^2 xi), B = 1/(64 pi a^2 xi^2),
// with g'(u) = -2A e^{-u^2 xi^2} + 4 B xi^2 u erfc(u xi); three exp and three
// erfc give both phi_r and phi_r'.
#include "common.cuh"

namespace ibp {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct PairConst {
    double a, xi, A, B, rc2, self;
    float rc2_cand;     // FP32 screen: (r_c + delta)^2, delta above the FP32 rounding of positions in the box
    double L[3];
    int nc[3];
    int lo[3], hi[3];   // neighbour cell offsets per axis
    // tabulated kernel on [2a, r_c]: node i at r = t0 + i h holds (phi, phi', phi'')
    const double* table;
    double t0, h, inv_h;
    int nt;
};

constexpr int kTableIntervals = 4096;

__device__ __forceinline__ void g_and_dg(double u, const PairConst& k, double& g, double& dg) {
    const double x2 = k.xi * k.xi;
    const double e = exp(-u * u * x2);
    const double ec = erfc(u * k.xi);
    g = -k.A * u * e + k.B * (2.0 * x2 * u * u + 1.0) * ec;
    dg = -2.0 * k.A * e + 4.0 * k.B * x2 * u * ec;
}

__device__ __forceinline__ void pair_kernel(double r, const PairConst& k, double& phi, double& dphi) {
    double gp, dgp, gm, dgm, g0, dg0;
    g_and_dg(r + 2.0 * k.a, k, gp, dgp);
    g_and_dg(r - 2.0 * k.a, k, gm, dgm);
    g_and_dg(r, k, g0, dg0);
    const double D = gp + gm - 2.0 * g0;
    const double dD = dgp + dgm - 2.0 * dg0;
    phi = D / r;
    dphi = dD / r - D / (r * r);
    if (r < 2.0 * k.a) {
        phi += -1.0 / (4.0 * kPi * r) + (4.0 * k.a - r) / (16.0 * kPi * k.a * k.a);
        dphi += 1.0 / (4.0 * kPi * r * r) - 1.0 / (16.0 * kPi * k.a * k.a);
    }
}

// phi_r, phi_r', phi_r'' for r >= 2a from the second-difference form, with
// g''(u) = 4 B xi^2 erfc(u xi) (the Heaviside term vanishes there).
__device__ void pair_kernel_d2(double r, const PairConst& k, double& phi, double& dphi, double& d2phi) {
    double gp, dgp, gm, dgm, g0, dg0;
    g_and_dg(r + 2.0 * k.a, k, gp, dgp);
    g_and_dg(r - 2.0 * k.a, k, gm, dgm);
    g_and_dg(r, k, g0, dg0);
    const double c2 = 4.0 * k.B * k.xi * k.xi;
    const double D = gp + gm - 2.0 * g0;
    const double dD = dgp + dgm - 2.0 * dg0;
    const double d2D = c2 * (erfc((r + 2.0 * k.a) * k.xi) + erfc((r - 2.0 * k.a) * k.xi) - 2.0 * erfc(r * k.xi));
    phi = D / r;
    dphi = dD / r - D / (r * r);
    d2phi = d2D / r - 2.0 * dD / (r * r) + 2.0 * D / (r * r * r);
}

__global__ void table_kernel(PairConst k, double* __restrict__ table) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > k.nt) return;
    double p, d, d2;
    pair_kernel_d2(k.t0 + i * k.h, k, p, d, d2);
    table[3 * i + 0] = p;
    table[3 * i + 1] = d;
    table[3 * i + 2] = d2;
}

// Cubic Hermite interpolation of phi (from phi, phi') and of phi' (from phi', phi'')
// between table nodes; r in [2a, r_c).
__device__ __forceinline__ void pair_table(double r, const PairConst& k, double& phi, double& dphi) {
    const double t = (r - k.t0) * k.inv_h;
    int i = (int)t;
    i = i < 0 ? 0 : (i >= k.nt ? k.nt - 1 : i);
    const double s = t - i;
    const double* a = k.table + 3 * i;
    const double p0 = a[0], d0 = a[1], e0 = a[2], p1 = a[3], d1 = a[4], e1 = a[5];
    const double s2 = s * s, s3 = s2 * s;
    const double h00 = 2.0 * s3 - 3.0 * s2 + 1.0, h10 = s3 - 2.0 * s2 + s;
    const double h01 = -2.0 * s3 + 3.0 * s2, h11 = s3 - s2;
    phi = h00 * p0 + h10 * k.h * d0 + h01 * p1 + h11 * k.h * d1;
    dphi = h00 * d0 + h10 * k.h * e0 + h01 * d1 + h11 * k.h * e1;
}

__device__ __forceinline__ int cell_coord(double x, double L, int nc) {
    int c = (int)(x * nc / L);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// 64-bit fingerprint of the wrapped positions (sum of splitmix64 of each word's
// bits mixed with its index) and a flag for non-finite coordinates.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void fingerprint_kernel(long long m, const double* __restrict__ xw, const int* __restrict__ bcfg,
                                   unsigned long long* __restrict__ out, int* __restrict__ bad) {
    unsigned long long acc = 0;
    int nonfinite = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const double v = xw[i];
        nonfinite |= !isfinite(v);
        acc += mix64((unsigned long long)__double_as_longlong(v) ^ mix64((unsigned long long)i));
        if (bcfg && i % 3 == 0) acc += mix64(0x5BD1E995ull * (unsigned long long)(bcfg[i / 3] + 1) + (unsigned long long)i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, acc);
        if (nonfinite) atomicOr(bad, 1);
    }
}

__global__ void cell_count_kernel(int n, const double* __restrict__ xw, PairConst k, const int* __restrict__ bcfg,
                                  int* __restrict__ cell_of, int* __restrict__ cell_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int base = bcfg ? bcfg[i] * (k.nc[0] * k.nc[1] * k.nc[2]) : 0;   // cells of the bead's configuration
    const int cx = cell_coord(xw[3 * i + 0], k.L[0], k.nc[0]);
    const int cy = cell_coord(xw[3 * i + 1], k.L[1], k.nc[1]);
    const int cz = cell_coord(xw[3 * i + 2], k.L[2], k.nc[2]);
    const int c = base + (cz * k.nc[1] + cy) * k.nc[0] + cx;
    cell_of[i] = c;
    atomicAdd(cell_count + c, 1);
}

__global__ void cell_fill_kernel(int n, const int* __restrict__ cell_of, int* __restrict__ cursor,
                                 int* __restrict__ cell_beads) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = atomicAdd(cursor + cell_of[i], 1);
    cell_beads[slot] = i;
}

// FP32 copy of the wrapped positions (x, y, z, 0) for the candidate filter.
__global__ void pos32_kernel(int n, const double* __restrict__ xw, float4* __restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xf[i] = make_float4((float)xw[3 * i], (float)xw[3 * i + 1], (float)xw[3 * i + 2], 0.0f);
}

// Visits every bead beta != alpha of the neighbouring cells, lanes striding
// over each cell; calls f(beta, slot, dx, dy, dz, r2, within) for every lane
// slot (within = false for idle lanes) so that warp-collective code can run in
// f; slot is beta's position in the cell-sorted bead order.
// Candidates are screened in FP32 with a margin far above its rounding, and
// the pairs that pass are decided exactly in FP64 (GB300's FP64 rate makes the
// FP64 test of every candidate the cost of the build).
template <typename F>
__device__ __forceinline__ void for_neighbours(int alpha, const double* __restrict__ xw,
                                               const float4* __restrict__ xf, const PairConst& k,
                                               const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                                               const int* __restrict__ cell_beads, int lane, F&& f) {
    const double x0 = xw[3 * alpha + 0], y0 = xw[3 * alpha + 1], z0 = xw[3 * alpha + 2];
    const float4 p0 = xf[alpha];
    const float Lx = (float)k.L[0], Ly = (float)k.L[1], Lz = (float)k.L[2];
    const float rc2f = k.rc2_cand;
    const int ncell = k.nc[0] * k.nc[1] * k.nc[2];
    const int base = (cell_of[alpha] / ncell) * ncell;   // first cell of the bead's configuration
    const int c = cell_of[alpha] - base;
    const int cx = c % k.nc[0], cy = (c / k.nc[0]) % k.nc[1], cz = c / (k.nc[0] * k.nc[1]);
    for (int oz = k.lo[2]; oz <= k.hi[2]; ++oz)
        for (int oy = k.lo[1]; oy <= k.hi[1]; ++oy)
            for (int ox = k.lo[0]; ox <= k.hi[0]; ++ox) {
                const int nx = (cx + ox + k.nc[0]) % k.nc[0];
                const int ny = (cy + oy + k.nc[1]) % k.nc[1];
                const int nz = (cz + oz + k.nc[2]) % k.nc[2];
                const int cell = base + (nz * k.nc[1] + ny) * k.nc[0] + nx;
                const int s = cell_start[cell], e = cell_start[cell + 1];
                for (int t0 = s; t0 < e; t0 += 32) {
                    const int t = t0 + lane;
                    bool within = false;
                    int beta = -1;
                    double dx = 0, dy = 0, dz = 0, r2 = 0;
                    if (t < e) {
                        beta = cell_beads[t];
                        const float4 pb = xf[beta];
                        const float fx = min_image_wrapped(p0.x - pb.x, Lx);
                        const float fy = min_image_wrapped(p0.y - pb.y, Ly);
                        const float fz = min_image_wrapped(p0.z - pb.z, Lz);
                        if (beta != alpha && fx * fx + fy * fy + fz * fz < rc2f) {
                            dx = min_image_wrapped(x0 - xw[3 * beta + 0], k.L[0]);
                            dy = min_image_wrapped(y0 - xw[3 * beta + 1], k.L[1]);
                            dz = min_image_wrapped(z0 - xw[3 * beta + 2], k.L[2]);
                            r2 = dx * dx + dy * dy + dz * dz;
                            within = r2 < k.rc2;
                        }
                    }
                    f(beta, t, dx, dy, dz, r2, within);
                }
            }
}

// The pair table is stored in the cell-sorted bead order: row t belongs to bead
// cell_beads[t] and its columns are sorted positions too, so the rows a block
// works on, and the charges they gather, sit close together in memory.
__global__ void pair_count_kernel(int n, const double* __restrict__ xw, const float4* __restrict__ xf, PairConst k,
                                  const int* __restrict__ cell_of,
                                  const int* __restrict__ cell_start, const int* __restrict__ cell_beads,
                                  int* __restrict__ row_count) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int alpha = cell_beads[t];
    int cnt = 0;
    for_neighbours(alpha, xw, xf, k, cell_of, cell_start, cell_beads, lane,
                   [&](int, int, double, double, double, double, bool within) { cnt += within ? 1 : 0; });
    cnt = warp_sum(cnt);
    if (lane == 0) row_count[t] = cnt;
}

__global__ void pair_fill_kernel(int n, const double* __restrict__ xw, const float4* __restrict__ xf, PairConst k,
                                 const int* __restrict__ cell_of,
                                 const int* __restrict__ cell_start, const int* __restrict__ cell_beads,
                                 const long long* __restrict__ rowptr, int* __restrict__ col,
                                 double* __restrict__ val, uint2* __restrict__ pair32, double* __restrict__ gfac) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int alpha = cell_beads[t];
    long long base = rowptr[t];
    const unsigned lt = (1u << lane) - 1u;
    for_neighbours(alpha, xw, xf, k, cell_of, cell_start, cell_beads, lane,
                   [&](int, int slot_b, double, double, double, double r2, bool within) {
                       const unsigned m = __ballot_sync(0xffffffffu, within);
                       if (within) {
                           const long long slot = base + __popc(m & lt);
                           const double r = sqrt(r2);
                           double phi, dphi;
                           if (r >= 2.0 * k.a) {
                               pair_table(r, k, phi, dphi);
                           } else if (r > 0.0) {
                               pair_kernel(r, k, phi, dphi);   // overlapping beads: exact form
                           } else {
                               phi = k.self;   // coincident beads: the r -> 0 limit
                               dphi = 0.0;
                           }
                           col[slot] = slot_b;
                           val[slot] = phi;
                           pair32[slot] = make_uint2((unsigned)slot_b, __float_as_uint((float)phi));
                           if (gfac) gfac[slot] = (r > 0.0) ? -dphi / r : 0.0;
                       }
                       base += __popc(m);
                   });
}

// psi_r[r][alpha] = (phi_self q_alpha + sum_pairs phi_r q_beta) / eps.
// One warp per row for NR right-hand sides; four independent accumulation
// chains per lane keep several gathers in flight on long rows.  The charges are
// first packed in the sorted order with the right-hand sides interleaved, so a
// pair gathers one NR-double run.
__global__ void pack_q64_kernel(int n, int nrhs, const int* __restrict__ order, const double* __restrict__ q,
                                double* __restrict__ qs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int b = order[t];
    for (int r = 0; r < nrhs; ++r) qs[(size_t)t * nrhs + r] = q[(size_t)r * n + b];
}

template <int NR>
__global__ void near_apply_kernel(int n, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                  const double* __restrict__ val, const int* __restrict__ order, double self,
                                  double inv_eps, const double* __restrict__ qs, const double* __restrict__ q,
                                  double* __restrict__ psi) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const long long s = rowptr[t], e = rowptr[t + 1];
    double acc[4][NR];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[u][r] = 0.0;
    long long p = s + lane;
    for (; p + 96 < e; p += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double* qb = qs + (size_t)col[p + 32 * u] * NR;
            const double v = val[p + 32 * u];
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[u][r] += v * qb[r];
        }
    }
    for (; p < e; p += 32) {
        const double* qb = qs + (size_t)col[p] * NR;
        const double v = val[p];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[0][r] += v * qb[r];
    }
    const int alpha = order[t];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double sum = warp_sum((acc[0][r] + acc[1][r]) + (acc[2][r] + acc[3][r]));
        if (lane == 0) psi[(size_t)r * n + alpha] = (sum + self * q[(size_t)r * n + alpha]) * inv_eps;
    }
}

// The inner operator of a mixed-precision solve: the same sum with the pair
// values rounded to FP32 and stored with their column as one 8-byte word, the
// charges of up to four right-hand sides packed per bead in one float4 (one
// 16-byte gather per pair instead of NR 8-byte ones), FP32 partial sums per
// lane, FP64 across the warp and for the self term.
__global__ void pack_q32_kernel(int n, int nrhs, const int* __restrict__ order, const double* __restrict__ q,
                                float4* __restrict__ qf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int b = order[t];
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = 0; r < nrhs; ++r) v[r] = (float)q[(size_t)r * n + b];
    qf[t] = make_float4(v[0], v[1], v[2], v[3]);
}

constexpr int kChains32 = 8;   // pairs per lane in flight in the FP32 pass

template <int NR>
__global__ void near_apply32_kernel(int n, const long long* __restrict__ rowptr, const uint2* __restrict__ pair32,
                                    const int* __restrict__ order, double self, double inv_eps,
                                    const float4* __restrict__ qf, const double* __restrict__ q,
                                    double* __restrict__ psi) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const long long s = rowptr[t], e = rowptr[t + 1];
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0f;
    long long p = s + lane;
    // kChains32 independent (column, value) loads, then their charge gathers
    for (; p + 32 * (kChains32 - 1) < e; p += 32 * kChains32) {
        uint2 cv[kChains32];
#pragma unroll
        for (int u = 0; u < kChains32; ++u) cv[u] = pair32[p + 32 * u];
        float4 b[kChains32];
#pragma unroll
        for (int u = 0; u < kChains32; ++u) b[u] = qf[cv[u].x];
#pragma unroll
        for (int u = 0; u < kChains32; ++u) {
            const float v = __uint_as_float(cv[u].y);
            const float qb[4] = {b[u].x, b[u].y, b[u].z, b[u].w};
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] += v * qb[r];
        }
    }
    for (; p < e; p += 32) {
        const uint2 cv = pair32[p];
        const float4 b = qf[cv.x];
        const float v = __uint_as_float(cv.y);
        const float qb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] += v * qb[r];
    }
    const int alpha = order[t];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double sum = warp_sum((double)acc[r]);
        if (lane == 0) psi[(size_t)r * n + alpha] = (sum + self * q[(size_t)r * n + alpha]) * inv_eps;
    }
}

// E_r[r][alpha] = sum_pairs (-phi_r'(r)/r) (x_alpha - x_beta) q_beta / eps
__global__ void near_field_kernel(int n, int nrhs, const double* __restrict__ xw, PairConst k,
                                  const long long* __restrict__ rowptr, const int* __restrict__ col,
                                  const int* __restrict__ order, const double* __restrict__ gfac, double inv_eps,
                                  const double* __restrict__ q, double* __restrict__ E) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int alpha = order[t];
    const long long s = rowptr[t], e = rowptr[t + 1];
    const double x0 = xw[3 * alpha + 0], y0 = xw[3 * alpha + 1], z0 = xw[3 * alpha + 2];
    double ex[kMaxRhs], ey[kMaxRhs], ez[kMaxRhs];
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r) ex[r] = ey[r] = ez[r] = 0.0;
    for (long long p = s + lane; p < e; p += 32) {
        const int b = order[col[p]];
        const double gf = gfac[p];
        const double dx = min_image_wrapped(x0 - xw[3 * b + 0], k.L[0]);
        const double dy = min_image_wrapped(y0 - xw[3 * b + 1], k.L[1]);
        const double dz = min_image_wrapped(z0 - xw[3 * b + 2], k.L[2]);
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nrhs) {
                const double w = gf * q[(size_t)r * n + b];
                ex[r] += w * dx;
                ey[r] += w * dy;
                ez[r] += w * dz;
            }
    }
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r) {
        if (r >= nrhs) break;
        const double a0 = warp_sum(ex[r]), a1 = warp_sum(ey[r]), a2 = warp_sum(ez[r]);
        if (lane == 0) {
            double* o = E + ((size_t)r * n + alpha) * 3;
            o[0] = a0 * inv_eps;
            o[1] = a1 * inv_eps;
            o[2] = a2 * inv_eps;
        }
    }
}

// ---- exclusive scan of int counts into 64-bit offsets (three passes) ----
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* s_warp, long long& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long ws = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
        long long wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = wi - ws;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const long long r = s_warp[w] + inc - v;
    total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void scan_blocks_kernel(const int* __restrict__ in, long long* __restrict__ out, int n,
                                   long long* __restrict__ block_sums) {
    __shared__ long long s_warp[33];
    const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        local += v[i];
    }
    long long total;
    long long ex = block_exclusive_scan(local, s_warp, total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(long long* __restrict__ block_sums, int nblocks, long long* __restrict__ total_out) {
    __shared__ long long s_warp[33];
    long long carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const long long v = b < nblocks ? block_sums[b] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, s_warp, total);
        if (b < nblocks) block_sums[b] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_add_kernel(long long* __restrict__ out, int n, const long long* __restrict__ block_sums) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_sums[i / kScanChunk];
}

__global__ void narrow_kernel(const long long* __restrict__ a, int* __restrict__ b, int* __restrict__ b2, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        b[i] = (int)a[i];
        b2[i] = (int)a[i];
    }
}

}  // namespace

void scan_counts(const int* in, long long* out, int n, DevBuf& tmp, cudaStream_t s) {
    const int nblocks = div_up(n > 0 ? n : 1, kScanChunk);
    long long* sums = static_cast<long long*>(tmp.ensure(sizeof(long long) * (nblocks + 1)));
    if (n > 0) {
        scan_blocks_kernel<<<nblocks, kScanThreads, 0, s>>>(in, out, n, sums);
        IBP_CHECK_LAUNCH();
    }
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, n > 0 ? nblocks : 0, out + n);
    IBP_CHECK_LAUNCH();
    if (n > 0) {
        scan_add_kernel<<<div_up(n, 256), 256, 0, s>>>(out, n, sums);
        IBP_CHECK_LAUNCH();
    }
}

namespace {

PairConst make_const(const ibpme_ctx* c) {
    PairConst k{};
    k.a = c->a;
    k.xi = c->xi;
    k.A = 1.0 / (32.0 * pow(kPi, 1.5) * c->a * c->a * c->xi);
    k.B = 1.0 / (64.0 * kPi * c->a * c->a * c->xi * c->xi);
    k.rc2 = c->rc * c->rc;
    {
        // each FP32 coordinate is within 2^-24 L of its FP64 value; a difference within
        // 2^-23 L per axis, the distance within sqrt(3) of that: delta = 8 L 2^-23 is ample
        const double Lmax = fmax(c->p.box[0], fmax(c->p.box[1], c->p.box[2]));
        const double delta = 8.0 * Lmax * 1.1920928955078125e-07;
        k.rc2_cand = (float)((c->rc + delta) * (c->rc + delta) * (1.0 + 1e-5));
    }
    k.self = (1.0 - exp(-4.0 * c->a * c->a * c->xi * c->xi)) / (8.0 * pow(kPi, 1.5) * c->a * c->a * c->xi) +
             erfc(2.0 * c->a * c->xi) / (4.0 * kPi * c->a);
    k.table = c->near.table.as<double>();
    k.nt = kTableIntervals;
    k.t0 = 2.0 * c->a;
    k.h = (c->rc > k.t0 ? c->rc - k.t0 : 0.0) / kTableIntervals;
    k.inv_h = k.h > 0.0 ? 1.0 / k.h : 0.0;
    for (int d = 0; d < 3; ++d) {
        k.L[d] = c->p.box[d];
        k.nc[d] = c->near.nc[d];
        if (k.nc[d] >= 3) { k.lo[d] = -1; k.hi[d] = 1; }
        else if (k.nc[d] == 2) { k.lo[d] = 0; k.hi[d] = 1; }
        else { k.lo[d] = 0; k.hi[d] = 0; }
    }
    return k;
}

}  // namespace

double self_term(const ibpme_ctx* c) { return make_const(c).self; }

void near_setup(ibpme_ctx* c) {
    NearList& nl = c->near;
    nl.table.ensure(sizeof(double) * 3 * (kTableIntervals + 1));
    const PairConst k = make_const(c);
    if (k.h > 0.0) {
        table_kernel<<<div_up(kTableIntervals + 1, 128), 128, 0, c->stream>>>(k, nl.table.as<double>());
        IBP_CHECK_LAUNCH();
    }
    nl.fp_valid = false;
}

void near_build(ibpme_ctx* c, int n, const double* xw, bool need_grad) {
    (void)need_grad;   // the table always carries the gradient factors
    NearList& nl = c->near;
    cudaStream_t s = c->stream;
    ProfScope ps(ST_NEAR_BUILD, s);
    // positions unchanged since the last build (solve -> forces -> BD step): reuse the table
    unsigned long long* fp = static_cast<unsigned long long*>(nl.fp_dev.ensure(2 * sizeof(unsigned long long)));
    int* bad = reinterpret_cast<int*>(fp + 1);
    IBP_CUDA(cudaMemsetAsync(fp, 0, 2 * sizeof(unsigned long long), s));
    if (n > 0) {
        fingerprint_kernel<<<div_up(3LL * n, 256) < 256 ? div_up(3LL * n, 256) : 256, 256, 0, s>>>(3LL * n, xw,
                                                                                                  c->bcfg, fp, bad);
        IBP_CHECK_LAUNCH();
    }
    unsigned long long* hfp = static_cast<unsigned long long*>(pinned_host(c, 2 * sizeof(unsigned long long)));
    IBP_CUDA(cudaMemcpyAsync(hfp, fp, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    if (*reinterpret_cast<int*>(hfp + 1) != 0) fail(IBPME_ERR_NONFINITE, "non-finite bead position");
    const unsigned long long print = hfp[0];
    if (nl.fp_valid && nl.n == n && nl.fp == print && nl.ncfg == c->ncfg) return;
    nl.fp_valid = false;
    nl.n = n;
    nl.rc = c->rc;
    int ncells = 1;
    for (int d = 0; d < 3; ++d) {
        nl.L[d] = c->p.box[d];
        int m = (int)floor(c->p.box[d] / c->rc);
        if (m < 1) m = 1;
        if (m > 1024) m = 1024;
        nl.nc[d] = m;
        ncells *= m;
    }
    nl.ncfg = c->ncfg;
    ncells *= c->ncfg;   // every configuration has its own cells
    const PairConst k = make_const(c);
    int* cell_of = static_cast<int*>(nl.cell_of.ensure(sizeof(int) * (n + 1)));
    int* cell_count = static_cast<int*>(nl.cell_count.ensure(sizeof(int) * (ncells + 1)));
    long long* cell_start64 = static_cast<long long*>(nl.cell_start64.ensure(sizeof(long long) * (ncells + 1)));
    int* cell_start = static_cast<int*>(nl.cell_start.ensure(sizeof(int) * (ncells + 1)));
    int* cursor = static_cast<int*>(nl.cursor.ensure(sizeof(int) * (ncells + 1)));
    int* cell_beads = static_cast<int*>(nl.cell_beads.ensure(sizeof(int) * (n + 1)));
    IBP_CUDA(cudaMemsetAsync(cell_count, 0, sizeof(int) * (ncells + 1), s));
    if (n > 0) {
        cell_count_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, k, c->bcfg, cell_of, cell_count);
        IBP_CHECK_LAUNCH();
    }
    scan_counts(cell_count, cell_start64, ncells, nl.scan_tmp, s);
    narrow_kernel<<<div_up(ncells + 1, 256), 256, 0, s>>>(cell_start64, cell_start, cursor, ncells + 1);
    IBP_CHECK_LAUNCH();
    if (n > 0) {
        cell_fill_kernel<<<div_up(n, 256), 256, 0, s>>>(n, cell_of, cursor, cell_beads);
        IBP_CHECK_LAUNCH();
    }
    // pair counts, offsets, fill
    int* row_count = static_cast<int*>(nl.row_count.ensure(sizeof(int) * (n + 1)));
    long long* rowptr = static_cast<long long*>(nl.rowptr.ensure(sizeof(long long) * (n + 1)));
    float4* xf = static_cast<float4*>(nl.xf.ensure(sizeof(float4) * (n + 1)));
    if (n > 0) {
        pos32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, xf);
        IBP_CHECK_LAUNCH();
        pair_count_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, xw, xf, k, cell_of, cell_start,
                                                                          cell_beads, row_count);
        IBP_CHECK_LAUNCH();
    }
    scan_counts(row_count, rowptr, n, nl.scan_tmp, s);
    long long* host_total = static_cast<long long*>(pinned_host(c, sizeof(long long)));
    IBP_CUDA(cudaMemcpyAsync(host_total, rowptr + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    nl.npairs = *host_total;
    nl.have_grad = true;
    const size_t np = (size_t)(nl.npairs > 0 ? nl.npairs : 1);
    int* col = static_cast<int*>(nl.col.ensure(sizeof(int) * np));
    double* val = static_cast<double*>(nl.val.ensure(sizeof(double) * np));
    double* gfac = static_cast<double*>(nl.gfac.ensure(sizeof(double) * np));
    uint2* pair32 = static_cast<uint2*>(nl.pair32.ensure(sizeof(uint2) * np));
    // packed charges of the two passes, allocated here, outside any graph capture
    nl.qf.ensure(sizeof(float4) * (n + 1));
    nl.qs.ensure(sizeof(double) * (size_t)(n + 1) * kMaxRhs);
    if (n > 0) {
        pair_fill_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, xw, xf, k, cell_of, cell_start,
                                                                         cell_beads, rowptr, col, val, pair32, gfac);
        IBP_CHECK_LAUNCH();
    }
    nl.fp = print;
    nl.fp_valid = true;
}

void near_apply(ibpme_ctx* c, int n, const double* q, int nrhs, double* psi_r, bool fp32) {
    if (n == 0) return;
    fp32 = fp32 && nrhs <= 4;
    ProfScope ps(fp32 ? ST_NEAR_APPLY32 : ST_NEAR_APPLY, c->stream);
    NearList& nl = c->near;
    const PairConst k = make_const(c);
    const int blocks = div_up((long long)n * 32, 128);
    const long long* rp = nl.rowptr.as<long long>();
    const int* cl = nl.col.as<int>();
    const double* vl = nl.val.as<double>();
    const double ie = 1.0 / c->eps;
    cudaStream_t s = c->stream;
    const int* od = nl.cell_beads.as<int>();
    if (fp32) {
        float4* qf = static_cast<float4*>(nl.qf.ensure(sizeof(float4) * n));
        pack_q32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, q, qf);
        IBP_CHECK_LAUNCH();
        const uint2* pc = nl.pair32.as<uint2>();
        switch (nrhs) {
            case 1: near_apply32_kernel<1><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, ie, qf, q, psi_r); break;
            case 2: near_apply32_kernel<2><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, ie, qf, q, psi_r); break;
            case 3: near_apply32_kernel<3><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, ie, qf, q, psi_r); break;
            default: near_apply32_kernel<4><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, ie, qf, q, psi_r); break;
        }
        IBP_CHECK_LAUNCH();
        return;
    }
    double* qs = static_cast<double*>(nl.qs.ensure(sizeof(double) * (size_t)n * nrhs));
    pack_q64_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, q, qs);
    IBP_CHECK_LAUNCH();
    switch (nrhs) {
        case 1: near_apply_kernel<1><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 2: near_apply_kernel<2><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 3: near_apply_kernel<3><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 4: near_apply_kernel<4><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 5: near_apply_kernel<5><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 6: near_apply_kernel<6><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        case 7: near_apply_kernel<7><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
        default: near_apply_kernel<8><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, ie, qs, q, psi_r); break;
    }
    IBP_CHECK_LAUNCH();
}

void near_field(ibpme_ctx* c, int n, const double* xw, const double* q, int nrhs, double* E_r) {
    if (n == 0) return;
    ProfScope ps(ST_NEAR_FIELD, c->stream);
    if (!c->near.have_grad) fail(IBPME_ERR_ARG, "internal: pair table built without gradients");
    NearList& nl = c->near;
    const PairConst k = make_const(c);
    near_field_kernel<<<div_up((long long)n * 32, 128), 128, 0, c->stream>>>(
        n, nrhs, xw, k, nl.rowptr.as<long long>(), nl.col.as<int>(), nl.cell_beads.as<int>(), nl.gfac.as<double>(),
        1.0 / c->eps, q, E_r);
    IBP_CHECK_LAUNCH();
}

}  // namespace ibp
