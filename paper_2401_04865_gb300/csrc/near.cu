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
#include "dfloat.cuh"

#include <cstdlib>
#include <mutex>
#include <vector>

namespace ibp {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct PairConst {
    double a, xi, A, B, rc2, self;
    float rc2_cand;     // FP32 screen: (r_c + delta)^2, delta above the FP32 rounding of positions in the box
    float rc2_in;       // FP32 screen: below (r_c - delta)^2 a pair is inside r_c without the FP64 test
    double L[3];
    int nc[3];
    int lo[3], hi[3];   // neighbour cell offsets per axis
    // tabulated kernel on [2a, r_c] in u = r^2 / (2a)^2: octave e (u in [2^e, 2^(e+1)))
    // holds kOctaveIntervals equal intervals; node j = e kOctaveIntervals + i sits at
    // u = 2^e (1 + i / kOctaveIntervals) and holds (phi, dphi/du, G, dG/du) with
    // G = -phi'(r) / r, the factor of the field
    const double* table;
    double inv4a2;      // 1 / (2a)^2
    int K;              // octaves (0: no table, every pair takes the exact kernel)
    // pairs inside one compact body are not tabulated (NULL: every pair is)
    const int* bbody;   // body of each bead
    const int* cflag;   // compact flag of each body
    // beads of unequal radii (ncls > 1): class of each bead, class radii and self terms
    int ncls;
    const int* cls;
    double ra[IBPME_MAX_RADIUS_CLASSES];
    double selfc[IBPME_MAX_RADIUS_CLASSES];
};

constexpr int kOctaveIntervals = 128;   // intervals per octave of u (a power of two)
constexpr int kMaxOctaves = 24;         // r_c / 2a up to 4096

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

// Two radii a and b (beads of unequal radii).  A bead's charge sits on a shell of
// its radius, so the pair kernel is the average of erfc(xi s)/(4 pi s) over both
// shells.  With g and A, B above taken at a b in place of a^2, the average is
//   phi_r = [g(r+a+b) - g(r+a-b) - g(r-a+b) + g(r-a-b)] / r
//           - sum over the negative arguments s of sign_s s^2 / (16 pi a b r)
// (the second line turns g, taken as printed for s < 0, into the odd extension
// the shell average needs; for a = b it is the Heaviside term of the one-radius
// kernel).  Coincident beads (r = 0) take the limit
//   [F'(a+b) - F'(|a-b|)] / (2ab),  F'(u) = (u erfc(xi u) - e^{-xi^2 u^2}/(xi sqrt(pi))) / (4 pi),
// which for a = b is the self term.
__device__ void pair_kernel2(double r, double a, double b, double xi, double& phi, double& dphi) {
    const double A = 1.0 / (32.0 * pow(kPi, 1.5) * a * b * xi);
    const double B = 1.0 / (64.0 * kPi * a * b * xi * xi);
    const double c2 = 1.0 / (16.0 * kPi * a * b);
    const double x2 = xi * xi;
    const double sv[4] = {r + a + b, r + a - b, r - a + b, r - a - b};
    const double sg[4] = {1.0, -1.0, -1.0, 1.0};
    double N = 0.0, dN = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double u = sv[i];
        const double e = exp(-u * u * x2);
        const double ec = erfc(u * xi);
        N += sg[i] * (-A * u * e + B * (2.0 * x2 * u * u + 1.0) * ec);
        dN += sg[i] * (-2.0 * A * e + 4.0 * B * x2 * u * ec);
        if (u < 0.0) {
            N -= c2 * sg[i] * u * u;
            dN -= 2.0 * c2 * sg[i] * u;
        }
    }
    phi = N / r;
    dphi = dN / r - N / (r * r);
}

__device__ double pair_limit2(double a, double b, double xi) {
    auto dF = [xi](double u) {
        return (u * erfc(xi * u) - exp(-xi * xi * u * u) / (xi * sqrt(kPi))) / (4.0 * kPi);
    };
    return (dF(a + b) - dF(fabs(a - b))) / (2.0 * a * b);
}

// phi_r, phi_r', phi_r'' of two radii for r >= a + b (every argument of g is >= 0
// there, so no correction term), with g''(u) = 4 B xi^2 erfc(u xi).
__device__ void pair_kernel2_d2(double r, double a, double b, double xi, double& phi, double& dphi, double& d2phi) {
    const double A = 1.0 / (32.0 * pow(kPi, 1.5) * a * b * xi);
    const double B = 1.0 / (64.0 * kPi * a * b * xi * xi);
    const double x2 = xi * xi;
    const double sv[4] = {r + a + b, r + a - b, r - a + b, r - a - b};
    const double sg[4] = {1.0, -1.0, -1.0, 1.0};
    double N = 0.0, dN = 0.0, d2N = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double u = sv[i];
        const double e = exp(-u * u * x2);
        const double ec = erfc(u * xi);
        N += sg[i] * (-A * u * e + B * (2.0 * x2 * u * u + 1.0) * ec);
        dN += sg[i] * (-2.0 * A * e + 4.0 * B * x2 * u * ec);
        d2N += sg[i] * 4.0 * B * x2 * ec;
    }
    phi = N / r;
    dphi = dN / r - N / (r * r);
    d2phi = d2N / r - 2.0 * dN / (r * r) + 2.0 * N / (r * r * r);
}

// The table of a pair of radii a, b in u = r^2 / (a + b)^2 (nodes as in table_kernel,
// with du/dr = 2 r / (a + b)^2).
__global__ void table2_kernel(double a, double b, double xi, int K, double* __restrict__ table) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > K * kOctaveIntervals) return;
    const int e = j / kOctaveIntervals, i = j % kOctaveIntervals;
    const double u = ldexp(1.0 + (double)i / kOctaveIntervals, e);
    const double r = (a + b) * sqrt(u);
    double p, d, d2;
    pair_kernel2_d2(r, a, b, xi, p, d, d2);
    const double s = (a + b) * (a + b) / (2.0 * r);
    table[4 * j + 0] = p;
    table[4 * j + 1] = d * s;
    table[4 * j + 2] = -d / r;
    table[4 * j + 3] = (d / (r * r) - d2 / r) * s;
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

// Node j of the table: u = 2^e (1 + i / M), r = 2a sqrt(u); with du/dr = r / (2 a^2),
// dphi/du = phi' 2a^2 / r and dG/du = (phi' / r^2 - phi'' / r) 2a^2 / r.
__global__ void table_kernel(PairConst k, double* __restrict__ table) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > k.K * kOctaveIntervals) return;
    const int e = j / kOctaveIntervals, i = j % kOctaveIntervals;
    const double u = ldexp(1.0 + (double)i / kOctaveIntervals, e);
    const double r = 2.0 * k.a * sqrt(u);
    double p, d, d2;
    pair_kernel_d2(r, k, p, d, d2);
    const double s = 2.0 * k.a * k.a / r;
    table[4 * j + 0] = p;
    table[4 * j + 1] = d * s;
    table[4 * j + 2] = -d / r;
    table[4 * j + 3] = (d / (r * r) - d2 / r) * s;
}

// Octave e, interval i and fraction s of u (>= about 1): u = 2^e (1 + (i + s) / M).
__device__ __forceinline__ int table_interval(double u, const PairConst& k, double& s, double& hu) {
    const long long bits = __double_as_longlong(u);
    int e = (int)((bits >> 52) & 0x7FF) - 1023;   // floor(log2 u) for normal u
    e = e < 0 ? 0 : (e > k.K - 1 ? k.K - 1 : e);
    const double w = u * __longlong_as_double((long long)(1023 - e) << 52);   // u / 2^e, exact
    const double t = (w - 1.0) * kOctaveIntervals;
    int i = (int)floor(t);
    i = i < 0 ? 0 : (i > kOctaveIntervals - 1 ? kOctaveIntervals - 1 : i);
    s = t - i;
    hu = __longlong_as_double((long long)(1023 + e) << 52) / kOctaveIntervals;   // interval width in u
    return e * kOctaveIntervals + i;
}

// Cubic Hermite interpolation of phi and of G = -phi'/r in u, for r^2 in [(2a)^2, r_c^2).
__device__ __forceinline__ void pair_table(double r2, const PairConst& k, double& phi, double& gfac) {
    double s, hu;
    const int j = table_interval(r2 * k.inv4a2, k, s, hu);
    const double* a = k.table + 4 * j;
    const double s2 = s * s, s3 = s2 * s;
    const double h00 = 2.0 * s3 - 3.0 * s2 + 1.0, h10 = s3 - 2.0 * s2 + s;
    const double h01 = -2.0 * s3 + 3.0 * s2, h11 = s3 - s2;
    phi = h00 * a[0] + h10 * hu * a[1] + h01 * a[4] + h11 * hu * a[5];
    gfac = h00 * a[2] + h10 * hu * a[3] + h01 * a[6] + h11 * hu * a[7];
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

// Order-dependent 64-bit hash of m ints: mix64(m) + sum of mix64(value ^ mix64(index)),
// added into *out (zeroed by the caller) by every block; the caller sets bit 0 so that
// a hash is never 0 (0 means unknown).
__global__ void hash_ints_kernel(const int* __restrict__ a, int m, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long sh[32];
    unsigned long long acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        acc += mix64((unsigned long long)(unsigned)a[i] ^ mix64(0xA24BAED4963EE407ull + (unsigned long long)i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = blockIdx.x == 0 ? mix64((unsigned long long)m) : 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(out, t);
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

// Visits every bead beta != alpha of the neighbouring cells, 32 candidates per
// round across the cells; calls f(beta, slot, within) for every lane slot
// (within = false for idle lanes) so that warp-collective code can run in f;
// slot is beta's position in the cell-sorted bead order.  Candidates are
// screened in FP32 between an outer and an inner bound, each a margin far above
// the FP32 rounding of positions in the box away from r_c: outside the outer
// one a candidate is no pair, inside the inner one it is, and only the thin
// shell between them takes the exact FP64 test (GB300's FP64 rate made the FP64
// test of every candidate the cost of the build).
template <typename F>
__device__ __forceinline__ void for_neighbours(int alpha, const double* __restrict__ xw,
                                               const float4* __restrict__ xf, const PairConst& k,
                                               const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                                               const int* __restrict__ cell_beads, int lane, F&& f) {
    const unsigned full = 0xffffffffu;
    const double x0 = xw[3 * alpha + 0], y0 = xw[3 * alpha + 1], z0 = xw[3 * alpha + 2];
    const float4 p0 = xf[alpha];
    const float Lx = (float)k.L[0], Ly = (float)k.L[1], Lz = (float)k.L[2];
    const float rc2f = k.rc2_cand;
    const int ncell = k.nc[0] * k.nc[1] * k.nc[2];
    const int base = (cell_of[alpha] / ncell) * ncell;   // first cell of the bead's configuration
    const int ba = k.cflag ? k.bbody[alpha] : -1;
    const int skip_body = (ba >= 0 && k.cflag[ba]) ? ba : -1;   // alpha's compact body, or -1
    const int c = cell_of[alpha] - base;
    const int cx = c % k.nc[0], cy = (c / k.nc[0]) % k.nc[1], cz = c / (k.nc[0] * k.nc[1]);
    const int wx = k.hi[0] - k.lo[0] + 1, wy = k.hi[1] - k.lo[1] + 1, wz = k.hi[2] - k.lo[2] + 1;
    const int nnb = wx * wy * wz;
    // Neighbour cells 32 at a time, lane l holding cell g0 + l of the (z, y, x)
    // offset order and its bead range; their candidates, concatenated in that
    // order, are then taken 32 per round.  A warp's dependent loads per row are
    // one round for the cell ranges plus one per 32 candidates, instead of one
    // chain per neighbour cell.
    for (int g0 = 0; g0 < nnb; g0 += 32) {
        const int g = g0 + lane;
        int s = 0, cnt = 0;
        if (g < nnb) {
            const int ox = k.lo[0] + g % wx, oy = k.lo[1] + (g / wx) % wy, oz = k.lo[2] + g / (wx * wy);
            const int nx = (cx + ox + k.nc[0]) % k.nc[0];
            const int ny = (cy + oy + k.nc[1]) % k.nc[1];
            const int nz = (cz + oz + k.nc[2]) % k.nc[2];
            const int cell = base + (nz * k.nc[1] + ny) * k.nc[0] + nx;
            s = cell_start[cell];
            cnt = cell_start[cell + 1] - s;
        }
        int incl = cnt;   // inclusive prefix of the counts over the lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(full, incl, d);
            if (lane >= d) incl += v;
        }
        const int excl = incl - cnt;
        const int total = __shfl_sync(full, incl, 31);
        for (int i0 = 0; i0 < total; i0 += 32) {
            const int i = i0 + lane;
            // the lane whose range holds candidate i: the largest j with excl_j <= i
            // (its count is then non-zero); j + step never passes lane 31
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int e = __shfl_sync(full, excl, j + step);
                if (e <= i) j += step;
            }
            const int t = __shfl_sync(full, s, j) + (i - __shfl_sync(full, excl, j));
            bool within = false;
            int beta = -1;
            if (i < total) {
                beta = cell_beads[t];
                const float4 pb = xf[beta];
                const float fx = min_image_wrapped(p0.x - pb.x, Lx);
                const float fy = min_image_wrapped(p0.y - pb.y, Ly);
                const float fz = min_image_wrapped(p0.z - pb.z, Lz);
                const float r2f = fx * fx + fy * fy + fz * fz;
                if (beta != alpha && r2f < rc2f && (skip_body < 0 || k.bbody[beta] != skip_body)) {
                    if (r2f < k.rc2_in) {
                        within = true;
                    } else {
                        const double dx = min_image_wrapped(x0 - xw[3 * beta + 0], k.L[0]);
                        const double dy = min_image_wrapped(y0 - xw[3 * beta + 1], k.L[1]);
                        const double dz = min_image_wrapped(z0 - xw[3 * beta + 2], k.L[2]);
                        within = dx * dx + dy * dy + dz * dz < k.rc2;
                    }
                }
            }
            f(beta, t, within);
        }
    }
}

// The pair table is stored in the cell-sorted bead order: row t belongs to bead
// cell_beads[t] and its columns are sorted positions too, so the rows a block
// works on, and the charges they gather, sit close together in memory.
// The pairs of each row counted (row_count[t]), its first cap columns kept in
// ell[t][0 .. cap) in the order pair_fill_kernel writes them, and the longest row
// in *row_max.
__global__ void pair_count_ell_kernel(int n, const double* __restrict__ xw, const float4* __restrict__ xf, PairConst k,
                                      const int* __restrict__ cell_of, const int* __restrict__ cell_start,
                                      const int* __restrict__ cell_beads, int cap, int* __restrict__ row_count,
                                      int* __restrict__ ell, int* __restrict__ row_max) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int alpha = cell_beads[t];
    int base = 0;
    const unsigned lt = (1u << lane) - 1u;
    int* row = ell + (size_t)t * cap;
    for_neighbours(alpha, xw, xf, k, cell_of, cell_start, cell_beads, lane, [&](int, int slot_b, bool within) {
        const unsigned m = __ballot_sync(0xffffffffu, within);
        if (within) {
            const int slot = base + __popc(m & lt);
            if (slot < cap) row[slot] = slot_b;
        }
        base += __popc(m);
    });
    if (lane == 0) {
        row_count[t] = base;
        atomicMax(row_max, base);
    }
}

// CSR table from the padded rows (every row at most cap long): one warp per row
__global__ void ell_compact_kernel(int n, int cap, const int* __restrict__ ell, const long long* __restrict__ rowptr,
                                   int* __restrict__ col, int* __restrict__ prow) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const long long s = rowptr[t];
    const int cnt = (int)(rowptr[t + 1] - s);
    const int* row = ell + (size_t)t * cap;
    for (int i = lane; i < cnt; i += 32) {
        col[s + i] = row[i];
        prow[s + i] = t;
    }
}

// The columns of each row (the same walk and decisions as the count) and the row of
// every pair; the FP64 values follow in pair_values_kernel, one thread per pair, so
// that the rows of beads beside a dense body (hundreds of real pairs each) do not
// hold one warp per row through their FP64 work.
__global__ void pair_fill_kernel(int n, const double* __restrict__ xw, const float4* __restrict__ xf, PairConst k,
                                 const int* __restrict__ cell_of,
                                 const int* __restrict__ cell_start, const int* __restrict__ cell_beads,
                                 const long long* __restrict__ rowptr, int* __restrict__ col,
                                 int* __restrict__ prow) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int alpha = cell_beads[t];
    long long base = rowptr[t];
    const unsigned lt = (1u << lane) - 1u;
    for_neighbours(alpha, xw, xf, k, cell_of, cell_start, cell_beads, lane,
                          [&](int, int slot_b, bool within) {
                              const unsigned m = __ballot_sync(0xffffffffu, within);
                              if (within) {
                                  const long long slot = base + __popc(m & lt);
                                  col[slot] = slot_b;
                                  prow[slot] = t;
                              }
                              base += __popc(m);
                          });
}

// phi_r and -phi_r'/r of every pair from its FP64 distance: the octave table at
// r >= 2a, the exact form for overlapping beads, the r -> 0 limit for coincident ones.
__global__ void pair_values_kernel(long long np, const double* __restrict__ xw, PairConst k,
                                   const int* __restrict__ prow, const int* __restrict__ col,
                                   const int* __restrict__ order, double* __restrict__ val,
                                   uint2* __restrict__ pair32, double* __restrict__ gfac) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int a = order[prow[p]], cb = col[p], b = order[cb];
    const double dx = min_image_wrapped(xw[3 * a + 0] - xw[3 * b + 0], k.L[0]);
    const double dy = min_image_wrapped(xw[3 * a + 1] - xw[3 * b + 1], k.L[1]);
    const double dz = min_image_wrapped(xw[3 * a + 2] - xw[3 * b + 2], k.L[2]);
    const double r2 = dx * dx + dy * dy + dz * dz;
    double phi, g;
    if (k.K > 0 && r2 * k.inv4a2 >= 1.0) {
        pair_table(r2, k, phi, g);
    } else if (r2 > 0.0) {
        const double r = sqrt(r2);
        double dphi;
        pair_kernel(r, k, phi, dphi);   // overlapping beads: exact form
        g = -dphi / r;
    } else {
        phi = k.self;   // coincident beads: the r -> 0 limit, no field
        g = 0.0;
    }
    val[p] = phi;
    pair32[p] = make_uint2((unsigned)cb, __float_as_uint((float)phi));
    if (gfac) gfac[p] = g;
}

// Pair values with radius classes: the exact two-radius kernel of each pair in FP64
// (every pair of classes has its own kernel; no table).
__global__ void pair_values_cls_kernel(long long np, const double* __restrict__ xw, PairConst k,
                                       const int* __restrict__ prow, const int* __restrict__ col,
                                       const int* __restrict__ order, double* __restrict__ val,
                                       uint2* __restrict__ pair32, double* __restrict__ gfac) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int a = order[prow[p]], cb = col[p], b = order[cb];
    const double dx = min_image_wrapped(xw[3 * a + 0] - xw[3 * b + 0], k.L[0]);
    const double dy = min_image_wrapped(xw[3 * a + 1] - xw[3 * b + 1], k.L[1]);
    const double dz = min_image_wrapped(xw[3 * a + 2] - xw[3 * b + 2], k.L[2]);
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double ra = k.ra[k.cls[a]], rb = k.ra[k.cls[b]];
    double phi, g;
    if (r2 > 0.0) {
        const double r = sqrt(r2);
        double dphi;
        pair_kernel2(r, ra, rb, k.xi, phi, dphi);
        g = -dphi / r;
    } else {
        phi = pair_limit2(ra, rb, k.xi);   // coincident beads: the r -> 0 limit, no field
        g = 0.0;
    }
    val[p] = phi;
    pair32[p] = make_uint2((unsigned)cb, __float_as_uint((float)phi));
    if (gfac) gfac[p] = g;
}

// Self term of each bead's class (radius classes).
__global__ void class_self_kernel(int n, const int* __restrict__ cls, PairConst k, double* __restrict__ self_b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) self_b[i] = k.selfc[cls[i]];
}

// psi_r[r][alpha] = (phi_self q_alpha + sum_pairs phi_r q_beta) / eps; with radius
// classes phi_self is selfv[alpha].
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
                                  const double* __restrict__ selfv, double inv_eps, const double* __restrict__ qs,
                                  const double* __restrict__ q, double* __restrict__ psi) {
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
    const double sf = selfv ? selfv[alpha] : self;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double sum = warp_sum((acc[0][r] + acc[1][r]) + (acc[2][r] + acc[3][r]));
        if (lane == 0) psi[(size_t)r * n + alpha] = (sum + sf * q[(size_t)r * n + alpha]) * inv_eps;
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
                                    const int* __restrict__ order, double self, const double* __restrict__ selfv,
                                    double inv_eps, const float4* __restrict__ qf, const double* __restrict__ q,
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
    const double sf = selfv ? selfv[alpha] : self;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double sum = warp_sum((double)acc[r]);
        if (lane == 0) psi[(size_t)r * n + alpha] = (sum + sf * q[(size_t)r * n + alpha]) * inv_eps;
    }
}

// E_r[r][alpha] += sum_pairs (-phi_r'(r)/r) (x_alpha - x_beta) q_beta / eps, one
// thread per pair (E_r zeroed first).  Pairs are stored row by row: a warp sums the
// runs of equal rows among its lanes (segmented doubling) and the first lane of each
// run adds the run's sum to its row, one atomic per component.  The rows beside a
// dense body hold hundreds of pairs; one warp per row left most of the GPU idle.
__global__ void near_field_kernel(long long np, int n, int nrhs, const double* __restrict__ xw, PairConst k,
                                  const int* __restrict__ prow, const int* __restrict__ col,
                                  const int* __restrict__ order, const double* __restrict__ gfac, double inv_eps,
                                  const double* __restrict__ q, double* __restrict__ E) {
    const unsigned full = 0xffffffffu;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool on = p < np;
    const int t = on ? prow[p] : -1;   // idle lanes (the grid's tail) only follow on lanes
    int a = 0, b = 0;
    double gf = 0.0, d[3] = {0.0, 0.0, 0.0};
    if (on) {
        a = order[t];
        b = order[col[p]];
        gf = gfac[p];
        d[0] = min_image_wrapped(xw[3 * a + 0] - xw[3 * b + 0], k.L[0]);
        d[1] = min_image_wrapped(xw[3 * a + 1] - xw[3 * b + 1], k.L[1]);
        d[2] = min_image_wrapped(xw[3 * a + 2] - xw[3 * b + 2], k.L[2]);
    }
    const int tprev = __shfl_up_sync(full, t, 1);
    const bool head = on && (lane == 0 || tprev != t);
    for (int r = 0; r < nrhs; ++r) {
        const double wq = on ? gf * q[(size_t)r * n + b] : 0.0;
        double v[3] = {wq * d[0], wq * d[1], wq * d[2]};
        // after the step of width w, lane l holds the sum over lanes [l, l + 2w) of its run
#pragma unroll
        for (int w = 1; w < 32; w <<= 1) {
            const int ot = __shfl_down_sync(full, t, w);
            double o[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = __shfl_down_sync(full, v[c], w);
            if (lane + w < 32 && ot == t)
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] += o[c];
        }
        if (head) {
            double* e = E + ((size_t)r * n + a) * 3;
            atomicAdd(e + 0, v[0] * inv_eps);
            atomicAdd(e + 1, v[1] * inv_eps);
            atomicAdd(e + 2, v[2] * inv_eps);
        }
    }
}

// ---------------------------------------------------------------------------
// Compact bodies: intra-body pairs evaluated directly.
//
// Within a body whose beads all lie within min(2 r_c, L/4) of its first bead, nearly
// every pair is inside r_c; such pairs are most of the table of a tessellated
// colloid (n_b^2 per body) and tabulating them needs FP64 per pair.  Instead,
// blocks of kCbThreads targets sweep the body's beads staged in shared memory
// and evaluate phi_r from cubic coefficients per table interval: FP32 for the
// inner operator of a mixed solve, double-float (dfloat.cuh) for the FP64
// operator and the field.  Positions are taken relative to the body's first bead,
// so every intra-body difference is its minimum image (|difference| <= L/2).
// Overlapping beads (r < 2a, rare within a tessellation) use the exact FP64
// kernel; coincident beads the r -> 0 limit, as in the table.
// ---------------------------------------------------------------------------
constexpr int kCbThreads = 128;    // targets per task and sources staged per round
constexpr int kCbBlocksPerSm = 6;  // resident blocks of the persistent compact kernels

// Tables per interval j = e M + i of u (see PairConst), with s in [0, 1):
//   tab32[j] = (p0, c1, c2, c3), phi = p0 + s (c1 + s (c2 + s c3))         (FP32)
//   tabdf[3j..3j+2] = (p0 hi, p0 lo, c1 hi, c1 lo), (c2, c3, g0 hi, g0 lo), (f1 hi, f1 lo, f2, f3)
// for phi and G = -phi'/r in double-float (linear terms) and FP32 (the smaller
// quadratic and cubic ones).
struct CbArgs {
    const int* flag;       // [nb] compact
    const int4* tasks;     // (body, first target bead, first source bead, target count << 20 | source count)
    int ntasks;
    const float4* hi;      // [n] position relative to the body's first bead, high parts
    const float4* lo;      // low parts
    const float4* tab32;
    const float4* tabdf;
    int nt;                // intervals (K M)
    int K;                 // octaves
    float rc2f, a2x4f, inv4a2f;
    df rc2, inv4a2;
    PairConst k;
};

// Interval and fraction of u = r^2 / (2a)^2 (FP32); u < 1 extrapolates the first interval.
__device__ __forceinline__ int cb_interval32(float u, int K, float& s) {
    int e = (__float_as_int(u) >> 23) - 127;
    e = min(max(e, 0), K - 1);
    const float w = __int_as_float(__float_as_int(u) - (e << 23));   // u / 2^e, exact
    const float t = (w - 1.0f) * (float)kOctaveIntervals;
    const int i = min(max((int)t, 0), kOctaveIntervals - 1);
    s = t - (float)i;
    return e * kOctaveIntervals + i;
}

// The same in double-float: w = u / 2^e scales both parts exactly, and the fraction
// keeps the low part.
__device__ __forceinline__ int cb_interval(df u, int K, df& s) {
    int e = (__float_as_int(u.hi) >> 23) - 127;
    e = min(max(e, 0), K - 1);
    const float sc = __int_as_float((127 - e) << 23);   // 2^-e
    const df w = {__fmul_rn(u.hi, sc), __fmul_rn(u.lo, sc)};
    const df t0 = two_sum(w.hi, -1.0f);
    const df t = fast_two_sum(__fmul_rn(t0.hi, (float)kOctaveIntervals),
                              __fmul_rn(__fadd_rn(t0.lo, w.lo), (float)kOctaveIntervals));
    int i = (int)floorf(t.hi);
    i = min(max(i, 0), kOctaveIntervals - 1);
    s = two_sum(__fsub_rn(t.hi, (float)i), t.lo);   // t.hi - i is exact
    return e * kOctaveIntervals + i;
}

__device__ __forceinline__ df cb_poly(float4 a, float c2, float c3, df s) {
    const df lin = df_add({a.x, a.y}, df_mul(s, {a.z, a.w}));
    return df_add(lin, {__fmul_rn(__fmul_rn(s.hi, s.hi), __fmaf_rn(s.hi, c3, c2)), 0.0f});
}

__device__ __forceinline__ df cb_diff(float ah, float al, float bh, float bl) {
    const df d = two_sum(ah, -bh);
    return fast_two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(al, bl)));
}

// Exact FP64 pair kernel for overlapping or coincident beads (phi and G = -phi'/r).
__device__ __noinline__ void cb_exact(const CbArgs& A, int ia, int ib, double& phi, double& g, double* d) {
    const float4 ah = A.hi[ia], al = A.lo[ia], bh = A.hi[ib], bl = A.lo[ib];
    d[0] = ((double)ah.x - (double)bh.x) + ((double)al.x - (double)bl.x);
    d[1] = ((double)ah.y - (double)bh.y) + ((double)al.y - (double)bl.y);
    d[2] = ((double)ah.z - (double)bh.z) + ((double)al.z - (double)bl.z);
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r > 0.0) {
        double dphi;
        pair_kernel(r, A.k, phi, dphi);
        g = -dphi / r;
    } else {
        phi = A.k.self;
        g = 0.0;
    }
}

__device__ __forceinline__ void cb_task(const CbArgs& A, int task, int& body, int& t0, int& s0, int& tc, int& sc) {
    const int4 w = A.tasks[task];
    body = w.x;
    t0 = w.y;
    s0 = w.z;
    tc = w.w >> 20;
    sc = w.w & 0xFFFFF;
}

// Overlapping (r < 2a) and coincident sources of one target with the exact FP64
// kernel: a rare second sweep over the task's sources, kept out of the main loop
// so that it stays free of calls.  The test matches the main loop's.
template <int NR, bool FIELD, bool DF>
__device__ __noinline__ void cb_overlaps(const CbArgs& A, int n, int alpha, int s0, int sc,
                                         const double* __restrict__ q, double* out) {
    const float4 pa = A.hi[alpha];
    for (int b = s0; b < s0 + sc; ++b) {
        if (b == alpha) continue;
        const float4 pb = A.hi[b];
        const float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 < A.a2x4f)) continue;
        double phi, g, d[3];
        cb_exact(A, alpha, b, phi, g, d);
        if (!DF) phi = (double)(float)phi;
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            const double qb = q[(size_t)c * n + b];
            if (FIELD) {
                out[3 * c + 0] += g * qb * d[0];
                out[3 * c + 1] += g * qb * d[1];
                out[3 * c + 2] += g * qb * d[2];
            } else {
                out[c] += phi * qb;
            }
        }
    }
}

// Copy n4 float4 of a table into shared memory.
__device__ __forceinline__ void cb_stage_table(float4* dst, const float4* __restrict__ src, int n4) {
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// Inner operator: psi_r[r][alpha] += sum over each task's sources, FP32 pairs from
// the shared-memory table, FP32 sums per staged round, FP64 across rounds.
// Persistent blocks stride over the tasks.
template <int NR>
__global__ void __launch_bounds__(kCbThreads)
compact_apply32_kernel(CbArgs A, int n, const double* __restrict__ q, double inv_eps, double* __restrict__ psi) {
    extern __shared__ float4 cb_tab[];
    __shared__ float4 sp[kCbThreads];
    __shared__ float4 sq[kCbThreads];   // charges of up to four fields
    cb_stage_table(cb_tab, A.tab32, A.nt);
    const int tid = threadIdx.x;
    for (int task = blockIdx.x; task < A.ntasks; task += gridDim.x) {
        int body, t0, s0, tc, sc;
        cb_task(A, task, body, t0, s0, tc, sc);
        if (!A.flag[body]) continue;   // block-uniform
        const int alpha = t0 + tid;
        const bool tin = tid < tc;
        const float4 pa = tin ? A.hi[alpha] : make_float4(0.f, 0.f, 0.f, 0.f);
        double accd[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) accd[r] = 0.0;
        bool ov = false;
        for (int u = 0; u < sc; u += kCbThreads) {
            const int m = min(kCbThreads, sc - u);
            __syncthreads();
            if (tid < m) {
                const int b = s0 + u + tid;
                sp[tid] = A.hi[b];
                float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int r = 0; r < NR; ++r) v[r] = (float)q[(size_t)r * n + b];
                sq[tid] = make_float4(v[0], v[1], v[2], v[3]);
            }
            __syncthreads();
            if (!tin) continue;
            float acc[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = 0.0f;
            const int self = alpha - (s0 + u);
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float4 pb = sp[j];
                const float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool near = r2 < A.a2x4f;   // the target itself, or an overlap
                ov |= near && j != self;
                const bool use = r2 < A.rc2f && !near;
                float s;
                const int i = cb_interval32(r2 * A.inv4a2f, A.K, s);
                const float4 c = cb_tab[use ? i : 0];
                const float phi = use ? fmaf(s, fmaf(s, fmaf(s, c.w, c.z), c.y), c.x) : 0.0f;
                const float4 qb = sq[j];
                const float qv[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = fmaf(phi, qv[r], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) accd[r] += (double)acc[r];
        }
        if (tin) {
            if (ov) cb_overlaps<NR, false, false>(A, n, alpha, s0, sc, q, accd);
#pragma unroll
            for (int r = 0; r < NR; ++r) atomicAdd(psi + (size_t)r * n + alpha, accd[r] * inv_eps);
        }
    }
}

// FP64 operator: the same sum in double-float arithmetic, the phi coefficients
// (two float4 per interval) in shared memory.
template <int NR>
__global__ void __launch_bounds__(kCbThreads)
compact_apply64_kernel(CbArgs A, int n, const double* __restrict__ q, double inv_eps, double* __restrict__ psi) {
    extern __shared__ float4 cb_tab[];
    __shared__ float4 sh[kCbThreads], sl[kCbThreads];
    __shared__ float2 sq[NR][kCbThreads];
    for (int i = threadIdx.x; i < A.nt; i += blockDim.x) {
        cb_tab[2 * i] = A.tabdf[3 * i];
        cb_tab[2 * i + 1] = A.tabdf[3 * i + 1];
    }
    __syncthreads();
    const int tid = threadIdx.x;
    for (int task = blockIdx.x; task < A.ntasks; task += gridDim.x) {
        int body, t0, s0, tc, sc;
        cb_task(A, task, body, t0, s0, tc, sc);
        if (!A.flag[body]) continue;   // block-uniform
        const int alpha = t0 + tid;
        const bool tin = tid < tc;
        const float4 ah = tin ? A.hi[alpha] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 al = tin ? A.lo[alpha] : make_float4(0.f, 0.f, 0.f, 0.f);
        df acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = {0.0f, 0.0f};
        bool ov = false;
        for (int u = 0; u < sc; u += kCbThreads) {
            const int m = min(kCbThreads, sc - u);
            __syncthreads();
            if (tid < m) {
                const int b = s0 + u + tid;
                sh[tid] = A.hi[b];
                sl[tid] = A.lo[b];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const df v = df_from_double(q[(size_t)r * n + b]);
                    sq[r][tid] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
            if (!tin) continue;
            const int self = alpha - (s0 + u);
#pragma unroll 2
            for (int j = 0; j < m; ++j) {
                const float4 bh = sh[j];
                const float fx = ah.x - bh.x, fy = ah.y - bh.y, fz = ah.z - bh.z;
                const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));   // the same test as the inner operator
                const bool near = r2f < A.a2x4f;
                ov |= near && j != self;
                if (near) continue;
                const float4 bl = sl[j];
                const df dx = cb_diff(ah.x, al.x, bh.x, bl.x);
                const df dy = cb_diff(ah.y, al.y, bh.y, bl.y);
                const df dz = cb_diff(ah.z, al.z, bh.z, bl.z);
                const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
                if (!(r2.hi < A.rc2.hi || (r2.hi == A.rc2.hi && r2.lo < A.rc2.lo))) continue;
                df s;
                const int i = cb_interval(df_mul(r2, A.inv4a2), A.K, s);
                const float4 a = cb_tab[2 * i], b = cb_tab[2 * i + 1];
                const df phi = cb_poly(a, b.x, b.y, s);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 qb = sq[r][j];
                    acc[r] = df_add(acc[r], df_mul(phi, {qb.x, qb.y}));
                }
            }
        }
        if (tin) {
            double out[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) out[r] = df_to_double(acc[r]);
            if (ov) cb_overlaps<NR, false, true>(A, n, alpha, s0, sc, q, out);
#pragma unroll
            for (int r = 0; r < NR; ++r) atomicAdd(psi + (size_t)r * n + alpha, out[r] * inv_eps);
        }
    }
}

// Field: E_r[r][alpha] += sum G(r) (x_alpha - x_beta) q_beta / eps, G = -phi'/r, double-float.
template <int NR>
__global__ void __launch_bounds__(kCbThreads)
compact_field_kernel(CbArgs A, int n, const double* __restrict__ q, double inv_eps, double* __restrict__ E) {
    extern __shared__ float4 cb_tab[];
    __shared__ float4 sh[kCbThreads], sl[kCbThreads];
    __shared__ float2 sq[NR][kCbThreads];
    for (int i = threadIdx.x; i < A.nt; i += blockDim.x) {
        cb_tab[2 * i] = A.tabdf[3 * i + 1];
        cb_tab[2 * i + 1] = A.tabdf[3 * i + 2];
    }
    __syncthreads();
    const int tid = threadIdx.x;
    for (int task = blockIdx.x; task < A.ntasks; task += gridDim.x) {
        int body, t0, s0, tc, sc;
        cb_task(A, task, body, t0, s0, tc, sc);
        if (!A.flag[body]) continue;   // block-uniform
        const int alpha = t0 + tid;
        const bool tin = tid < tc;
        const float4 ah = tin ? A.hi[alpha] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 al = tin ? A.lo[alpha] : make_float4(0.f, 0.f, 0.f, 0.f);
        df ex[NR], ey[NR], ez[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) ex[r] = ey[r] = ez[r] = {0.0f, 0.0f};
        bool ov = false;
        for (int u = 0; u < sc; u += kCbThreads) {
            const int m = min(kCbThreads, sc - u);
            __syncthreads();
            if (tid < m) {
                const int b = s0 + u + tid;
                sh[tid] = A.hi[b];
                sl[tid] = A.lo[b];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const df v = df_from_double(q[(size_t)r * n + b]);
                    sq[r][tid] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
            if (!tin) continue;
            const int self = alpha - (s0 + u);
            for (int j = 0; j < m; ++j) {
                const float4 bh = sh[j];
                const float fx = ah.x - bh.x, fy = ah.y - bh.y, fz = ah.z - bh.z;
                const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                const bool near = r2f < A.a2x4f;
                ov |= near && j != self;
                if (near) continue;
                const float4 bl = sl[j];
                const df dx = cb_diff(ah.x, al.x, bh.x, bl.x);
                const df dy = cb_diff(ah.y, al.y, bh.y, bl.y);
                const df dz = cb_diff(ah.z, al.z, bh.z, bl.z);
                const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
                if (!(r2.hi < A.rc2.hi || (r2.hi == A.rc2.hi && r2.lo < A.rc2.lo))) continue;
                df s;
                const int i = cb_interval(df_mul(r2, A.inv4a2), A.K, s);
                const float4 b4 = cb_tab[2 * i], c4 = cb_tab[2 * i + 1];
                const df g = cb_poly(make_float4(b4.z, b4.w, c4.x, c4.y), c4.z, c4.w, s);
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    const float2 qb = sq[c][j];
                    const df gq = df_mul(g, {qb.x, qb.y});
                    ex[c] = df_add(ex[c], df_mul(gq, dx));
                    ey[c] = df_add(ey[c], df_mul(gq, dy));
                    ez[c] = df_add(ez[c], df_mul(gq, dz));
                }
            }
        }
        if (tin) {
            double o[3 * NR];
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                o[3 * c + 0] = df_to_double(ex[c]);
                o[3 * c + 1] = df_to_double(ey[c]);
                o[3 * c + 2] = df_to_double(ez[c]);
            }
            if (ov) cb_overlaps<NR, true, true>(A, n, alpha, s0, sc, q, o);
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                double* e = E + ((size_t)c * n + alpha) * 3;
                atomicAdd(e + 0, o[3 * c + 0] * inv_eps);
                atomicAdd(e + 1, o[3 * c + 1] * inv_eps);
                atomicAdd(e + 2, o[3 * c + 2] * inv_eps);
            }
        }
    }
}

// Compact bodies: every bead within lim of the body's first bead (so that every
// intra-body difference of the relative positions below is its minimum image).
// Flags first (bodies of at least kCompactMin beads start compact), then one
// thread per bead: its position relative to the body's first bead as hi + lo
// floats, and a bead beyond lim clears its body's flag.
constexpr int kCompactMin = 32;    // smaller bodies stay in the table

__global__ void compact_flags_kernel(int nb, const int* __restrict__ off, int* __restrict__ flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) flag[b] = off[b + 1] - off[b] >= kCompactMin ? 1 : 0;
}

__global__ void compact_rel_kernel(int n, const int* __restrict__ bead_body, const int* __restrict__ off,
                                   const double* __restrict__ xw, double L0, double L1, double L2, double lim2,
                                   int* __restrict__ flag, float4* __restrict__ hi, float4* __restrict__ lo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int b = bead_body[j];
    const int o = off[b];
    if (off[b + 1] - o < kCompactMin) return;
    const double dx = min_image_wrapped(xw[3 * j] - xw[3 * o], L0);
    const double dy = min_image_wrapped(xw[3 * j + 1] - xw[3 * o + 1], L1);
    const double dz = min_image_wrapped(xw[3 * j + 2] - xw[3 * o + 2], L2);
    const float hx = (float)dx, hy = (float)dy, hz = (float)dz;
    hi[j] = make_float4(hx, hy, hz, 0.0f);
    lo[j] = make_float4((float)(dx - (double)hx), (float)(dy - (double)hy), (float)(dz - (double)hz), 0.0f);
    if (dx * dx + dy * dy + dz * dz > lim2) flag[b] = 0;   // every writer stores 0
}

// Cubic coefficients per interval j from the FP64 nodes (value and u-derivative of
// phi and of G): on [node j, node j+1] with s in [0, 1] and width h = 2^e / M,
//   phi = p0 + c1 s + c2 s^2 + c3 s^3,  c1 = h p'_0,  c2 = 3 (p1 - p0) - h (2 p'_0 + p'_1),
//   c3 = h (p'_0 + p'_1) - 2 (p1 - p0)   (the cubic Hermite interpolant), and the same for G.
__global__ void compact_table_kernel(int nt, const double* __restrict__ table, float4* __restrict__ tab32,
                                     float4* __restrict__ tabdf) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nt) return;
    const double h = ldexp(1.0, j / kOctaveIntervals) / kOctaveIntervals;
    const double* a = table + 4 * j;
    const double p0 = a[0], d0 = a[1], g0 = a[2], e0 = a[3];
    const double p1 = a[4], d1 = a[5], g1 = a[6], e1 = a[7];
    const double c1 = h * d0, c2 = 3.0 * (p1 - p0) - h * (2.0 * d0 + d1), c3 = h * (d0 + d1) - 2.0 * (p1 - p0);
    const double f1 = h * e0, f2 = 3.0 * (g1 - g0) - h * (2.0 * e0 + e1), f3 = h * (e0 + e1) - 2.0 * (g1 - g0);
    tab32[j] = make_float4((float)p0, (float)c1, (float)c2, (float)c3);
    const float ph = (float)p0, ch = (float)c1, gh = (float)g0, fh = (float)f1;
    tabdf[3 * j] = make_float4(ph, (float)(p0 - (double)ph), ch, (float)(c1 - (double)ch));
    tabdf[3 * j + 1] = make_float4((float)c2, (float)c3, gh, (float)(g0 - (double)gh));
    tabdf[3 * j + 2] = make_float4(fh, (float)(f1 - (double)fh), (float)f2, (float)f3);
}

// ---- pair values in double-float arithmetic ----
// GB300 issues FP64 at 1/64 of its FP32 rate, and the FP64 Hermite interpolation of
// every pair made the FP64 pipe the limit of the table build.  Pairs at r >= 2a take
// the table's per-interval coefficients in double-float arithmetic (linear terms hi +
// lo, quadratic and cubic terms FP32, as the compact-body kernels) from double-float
// positions, and join to FP64 once per value.  Overlapping beads (r < 2a) need the
// exact kernel (three exp and three erfc in FP64); they are rare, and within a warp of
// table pairs one of them stalled every lane, so they are listed and valued by a
// second kernel of one thread per such pair.

// Positions as hi, lo float4 per bead.
__global__ void pos_df_kernel(int n, const double* __restrict__ xw, float4* __restrict__ xdf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df x = df_split(xw[3 * i]), y = df_split(xw[3 * i + 1]), z = df_split(xw[3 * i + 2]);
    xdf[2 * i] = make_float4(x.hi, y.hi, z.hi, 0.0f);
    xdf[2 * i + 1] = make_float4(x.lo, y.lo, z.lo, 0.0f);
}

struct DfPairArgs {
    const float4* xdf;
    const float4* tabdf;
    int K;
    df inv4a2;
    df L[3];
    float halfL[3];
};

// Minimum image of a difference of two wrapped coordinates (in (-L, L)): one shift.
__device__ __forceinline__ df df_min_image(df d, df L, float halfL) {
    if (d.hi > halfL) return df_sub(d, L);
    if (d.hi < -halfL) return df_add(d, L);
    return d;
}

__global__ void pair_values_df_kernel(long long np, DfPairArgs A, const int* __restrict__ prow,
                                      const int* __restrict__ col, const int* __restrict__ order,
                                      double* __restrict__ val, uint2* __restrict__ pair32, double* __restrict__ gfac,
                                      int* __restrict__ ov_list, int* __restrict__ ov_count) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int a = order[prow[p]], cb = col[p], b = order[cb];
    const float4 ah = A.xdf[2 * a], al = A.xdf[2 * a + 1], bh = A.xdf[2 * b], bl = A.xdf[2 * b + 1];
    const df dx = df_min_image(df_sub(df{ah.x, al.x}, df{bh.x, bl.x}), A.L[0], A.halfL[0]);
    const df dy = df_min_image(df_sub(df{ah.y, al.y}, df{bh.y, bl.y}), A.L[1], A.halfL[1]);
    const df dz = df_min_image(df_sub(df{ah.z, al.z}, df{bh.z, bl.z}), A.L[2], A.halfL[2]);
    const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
    const df u = df_mul(r2, A.inv4a2);
    if (!(u.hi > 1.0f || (u.hi == 1.0f && u.lo >= 0.0f))) {   // r < 2a: the exact kernel, below
        ov_list[atomicAdd(ov_count, 1)] = (int)p;   // np < 2^31 (the table's pair count)
        return;
    }
    df s;
    const int j = cb_interval(u, A.K, s);
    const float4 t0 = A.tabdf[3 * j], t1 = A.tabdf[3 * j + 1], t2 = A.tabdf[3 * j + 2];
    const df phi = cb_poly(t0, t1.x, t1.y, s);
    const df g = cb_poly(make_float4(t1.z, t1.w, t2.x, t2.y), t2.z, t2.w, s);
    val[p] = df_join(phi);
    pair32[p] = make_uint2((unsigned)cb, __float_as_uint(__fadd_rn(phi.hi, phi.lo)));
    if (gfac) gfac[p] = df_join(g);
}

// The listed pairs of overlapping beads with the exact FP64 kernel (the r -> 0 limit
// for coincident ones); the grid strides over the list, whose length is on the device.
__global__ void pair_values_exact_kernel(const int* __restrict__ ov_count, const int* __restrict__ ov_list,
                                         const double* __restrict__ xw, PairConst k, const int* __restrict__ prow,
                                         const int* __restrict__ col, const int* __restrict__ order,
                                         double* __restrict__ val, uint2* __restrict__ pair32,
                                         double* __restrict__ gfac) {
    const int m = *ov_count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const long long p = ov_list[t];
        const int a = order[prow[p]], cb = col[p], b = order[cb];
        const double dx = min_image_wrapped(xw[3 * a + 0] - xw[3 * b + 0], k.L[0]);
        const double dy = min_image_wrapped(xw[3 * a + 1] - xw[3 * b + 1], k.L[1]);
        const double dz = min_image_wrapped(xw[3 * a + 2] - xw[3 * b + 2], k.L[2]);
        const double r2 = dx * dx + dy * dy + dz * dz;
        double phi, g;
        const double ra = k.ncls > 1 ? k.ra[k.cls[a]] : k.a, rb = k.ncls > 1 ? k.ra[k.cls[b]] : k.a;
        if (r2 > 0.0) {
            const double r = sqrt(r2);
            double dphi;
            if (k.ncls > 1)
                pair_kernel2(r, ra, rb, k.xi, phi, dphi);
            else
                pair_kernel(r, k, phi, dphi);
            g = -dphi / r;
        } else {
            // coincident beads: the r -> 0 limit, no field
            phi = k.ncls > 1 ? pair_limit2(ra, rb, k.xi) : k.self;
            g = 0.0;
        }
        val[p] = phi;
        pair32[p] = make_uint2((unsigned)cb, __float_as_uint((float)phi));
        if (gfac) gfac[p] = g;
    }
}

// Radius classes: the table of each pair of classes (c, d) at tabdf + (c ncls + d) stride,
// in u = r^2 inv_s2[c ncls + d] with inv_s2 = 1 / (a_c + a_d)^2.
struct DfClassArgs {
    const int* cls;
    int ncls;
    long long stride;
    df inv_s2[IBPME_MAX_RADIUS_CLASSES * IBPME_MAX_RADIUS_CLASSES];
};

__global__ void pair_values_df_cls_kernel(long long np, DfPairArgs A, DfClassArgs C, const int* __restrict__ prow,
                                          const int* __restrict__ col, const int* __restrict__ order,
                                          double* __restrict__ val, uint2* __restrict__ pair32,
                                          double* __restrict__ gfac, int* __restrict__ ov_list,
                                          int* __restrict__ ov_count) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int a = order[prow[p]], cb = col[p], b = order[cb];
    const float4 ah = A.xdf[2 * a], al = A.xdf[2 * a + 1], bh = A.xdf[2 * b], bl = A.xdf[2 * b + 1];
    const df dx = df_min_image(df_sub(df{ah.x, al.x}, df{bh.x, bl.x}), A.L[0], A.halfL[0]);
    const df dy = df_min_image(df_sub(df{ah.y, al.y}, df{bh.y, bl.y}), A.L[1], A.halfL[1]);
    const df dz = df_min_image(df_sub(df{ah.z, al.z}, df{bh.z, bl.z}), A.L[2], A.halfL[2]);
    const df r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
    const int pc = C.cls[a] * C.ncls + C.cls[b];
    const df u = df_mul(r2, C.inv_s2[pc]);
    if (!(u.hi > 1.0f || (u.hi == 1.0f && u.lo >= 0.0f))) {   // r < a_c + a_d: the exact kernel
        ov_list[atomicAdd(ov_count, 1)] = (int)p;
        return;
    }
    df s;
    const int j = cb_interval(u, A.K, s);
    const float4* tab = A.tabdf + (size_t)pc * C.stride;
    const float4 t0 = tab[3 * j], t1 = tab[3 * j + 1], t2 = tab[3 * j + 2];
    const df phi = cb_poly(t0, t1.x, t1.y, s);
    const df g = cb_poly(make_float4(t1.z, t1.w, t2.x, t2.y), t2.z, t2.w, s);
    val[p] = df_join(phi);
    pair32[p] = make_uint2((unsigned)cb, __float_as_uint(__fadd_rn(phi.hi, phi.lo)));
    if (gfac) gfac[p] = df_join(g);
}

// The real-space field of near_field_kernel in double-float arithmetic: differences
// from the double-float positions, products and the segmented warp sums on the FP32
// pipes, one FP64 addition per component of each run's sum (the FP64 differences,
// products and 15 FP64 additions of the segmented sums per pair made the FP64 pipe the
// limit of the force pass).
__global__ void near_field_df_kernel(long long np, int n, int nrhs, DfPairArgs A, const int* __restrict__ prow,
                                     const int* __restrict__ col, const int* __restrict__ order,
                                     const double* __restrict__ gfac, df inv_eps, const double* __restrict__ q,
                                     double* __restrict__ E) {
    const unsigned full = 0xffffffffu;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool on = p < np;
    const int t = on ? prow[p] : -1;   // idle lanes (the grid's tail) only follow on lanes
    int a = 0, b = 0;
    df gf = {0.0f, 0.0f}, d[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    if (on) {
        a = order[t];
        b = order[col[p]];
        gf = df_split(gfac[p]);
        const float4 ah = A.xdf[2 * a], al = A.xdf[2 * a + 1], bh = A.xdf[2 * b], bl = A.xdf[2 * b + 1];
        d[0] = df_min_image(df_sub(df{ah.x, al.x}, df{bh.x, bl.x}), A.L[0], A.halfL[0]);
        d[1] = df_min_image(df_sub(df{ah.y, al.y}, df{bh.y, bl.y}), A.L[1], A.halfL[1]);
        d[2] = df_min_image(df_sub(df{ah.z, al.z}, df{bh.z, bl.z}), A.L[2], A.halfL[2]);
    }
    const int tprev = __shfl_up_sync(full, t, 1);
    const bool head = on && (lane == 0 || tprev != t);
    for (int r = 0; r < nrhs; ++r) {
        const df wq = on ? df_mul(gf, df_split(q[(size_t)r * n + b])) : df{0.0f, 0.0f};
        df v[3] = {df_mul(wq, d[0]), df_mul(wq, d[1]), df_mul(wq, d[2])};
        // after the step of width w, lane l holds the sum over lanes [l, l + 2w) of its run
#pragma unroll
        for (int w = 1; w < 32; w <<= 1) {
            const int ot = __shfl_down_sync(full, t, w);
            df o[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = df{__shfl_down_sync(full, v[c].hi, w), __shfl_down_sync(full, v[c].lo, w)};
            if (lane + w < 32 && ot == t)
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = df_add(v[c], o[c]);
        }
        if (head) {
            double* e = E + ((size_t)r * n + a) * 3;
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(e + c, df_join(df_mul(v[c], inv_eps)));
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

constexpr size_t kCbSmemMax = 2 * sizeof(float4) * kOctaveIntervals * kMaxOctaves;   // two float4 per interval

template <typename K>
void cb_attr(K kernel) {
    IBP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmemMax));
}

template <int NR>
void cb_attrs_nr() {
    cb_attr(compact_apply64_kernel<NR>);
    cb_attr(compact_field_kernel<NR>);
}

// Opt-in to the shared-memory tables of the compact kernels, once per device
// (called at set-up, outside any stream capture).
void compact_attrs() {
    constexpr int kMaxDev = 64;
    static bool done[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    IBP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev) fail(IBPME_ERR_CUDA, "device ordinal %d out of range", dev);
    if (done[dev]) return;
    cb_attr(compact_apply32_kernel<1>);
    cb_attr(compact_apply32_kernel<2>);
    cb_attr(compact_apply32_kernel<3>);
    cb_attr(compact_apply32_kernel<4>);
    cb_attrs_nr<1>();
    cb_attrs_nr<2>();
    cb_attrs_nr<3>();
    cb_attrs_nr<4>();
    cb_attrs_nr<5>();
    cb_attrs_nr<6>();
    cb_attrs_nr<7>();
    cb_attrs_nr<8>();
    done[dev] = true;
}

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
        k.rc2_in = c->rc > delta ? (float)((c->rc - delta) * (c->rc - delta) * (1.0 - 1e-5)) : 0.0f;
    }
    k.self = (1.0 - exp(-4.0 * c->a * c->a * c->xi * c->xi)) / (8.0 * pow(kPi, 1.5) * c->a * c->a * c->xi) +
             erfc(2.0 * c->a * c->xi) / (4.0 * kPi * c->a);
    k.table = c->near.table.as<double>();
    k.inv4a2 = 1.0 / (4.0 * c->a * c->a);
    {
        const double uc = c->rc * c->rc * k.inv4a2;   // u at the cut-off
        k.K = 0;
        while (k.K < kMaxOctaves && ldexp(1.0, k.K) < uc) ++k.K;
        if (uc <= 1.0) k.K = 0;                        // r_c <= 2a: no tabulated range
    }
    k.ncls = c->ncls;
    k.cls = c->ncls > 1 ? c->cls.as<int>() : nullptr;
    for (int q = 0; q < c->ncls && c->ncls > 1; ++q) {
        const double a = c->cls_a[q];
        k.ra[q] = a;
        k.selfc[q] = (1.0 - exp(-4.0 * a * a * c->xi * c->xi)) / (8.0 * pow(kPi, 1.5) * a * a * c->xi) +
                     erfc(2.0 * a * c->xi) / (4.0 * kPi * a);
    }
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
    nl.table.ensure(sizeof(double) * 4 * (kMaxOctaves * kOctaveIntervals + 1));
    const PairConst k = make_const(c);
    if (k.K > 0) {
        const int nodes = k.K * kOctaveIntervals + 1;
        table_kernel<<<div_up(nodes, 128), 128, 0, c->stream>>>(k, nl.table.as<double>());
        IBP_CHECK_LAUNCH();
        const int nt = k.K * kOctaveIntervals;
        float4* t32 = static_cast<float4*>(nl.tab32.ensure(sizeof(float4) * nt));
        float4* tdf = static_cast<float4*>(nl.tab_df.ensure(sizeof(float4) * 3 * nt));
        compact_table_kernel<<<div_up(nt, 128), 128, 0, c->stream>>>(nt, nl.table.as<double>(), t32, tdf);
        IBP_CHECK_LAUNCH();
    }
    if (c->ncls > 1) {   // one table per pair of radius classes, octaves up to the largest u
        int K = 0;
        for (int a = 0; a < c->ncls; ++a)
            for (int b = 0; b < c->ncls; ++b) {
                const double uc = c->rc * c->rc / ((c->cls_a[a] + c->cls_a[b]) * (c->cls_a[a] + c->cls_a[b]));
                int ka = 0;
                while (ka < kMaxOctaves && ldexp(1.0, ka) < uc) ++ka;
                if (uc > 1.0) K = std::max(K, ka);
            }
        nl.cls_K = K;
        if (K > 0) {
            const int nodes = K * kOctaveIntervals + 1, nt = K * kOctaveIntervals, np = c->ncls * c->ncls;
            double* tab = static_cast<double*>(nl.cls_table.ensure(sizeof(double) * 4 * (size_t)nodes * np));
            float4* tdf = static_cast<float4*>(nl.cls_tabdf.ensure(sizeof(float4) * 3 * (size_t)nt * np));
            float4* t32 = static_cast<float4*>(nl.cls_tab32.ensure(sizeof(float4) * (size_t)nt * np));
            for (int a = 0; a < c->ncls; ++a)
                for (int b = 0; b < c->ncls; ++b) {
                    const int q = a * c->ncls + b;
                    table2_kernel<<<div_up(nodes, 128), 128, 0, c->stream>>>(c->cls_a[a], c->cls_a[b], c->xi, K,
                                                                            tab + 4 * (size_t)nodes * q);
                    IBP_CHECK_LAUNCH();
                    compact_table_kernel<<<div_up(nt, 128), 128, 0, c->stream>>>(
                        nt, tab + 4 * (size_t)nodes * q, t32 + (size_t)nt * q, tdf + 3 * (size_t)nt * q);
                    IBP_CHECK_LAUNCH();
                }
        }
    }
    compact_attrs();
    nl.fp_valid = false;
}

namespace {

df host_df(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

CbArgs cb_args(const ibpme_ctx* c) {
    const NearList& nl = c->near;
    const PairConst k = make_const(c);
    CbArgs A{};
    A.flag = nl.cb_flag.as<int>();
    A.tasks = nl.cb_tasks.as<int4>();
    A.ntasks = nl.cb_ntasks;
    A.hi = nl.cb_hi.as<float4>();
    A.lo = nl.cb_lo.as<float4>();
    A.tab32 = nl.tab32.as<float4>();
    A.tabdf = nl.tab_df.as<float4>();
    A.K = k.K;
    A.nt = k.K * kOctaveIntervals;
    A.rc2f = (float)k.rc2;
    A.a2x4f = (float)(4.0 * k.a * k.a);
    A.inv4a2f = (float)k.inv4a2;
    A.rc2 = host_df(k.rc2);
    A.inv4a2 = host_df(k.inv4a2);
    A.k = k;
    return A;
}

// Compact flags and relative positions of this set of positions, and the
// block tasks of the body structure: (body, 128 targets, a range of sources).
// Sources are split into ranges while the blocks would not give every SM
// several of them.
void compact_prepare(ibpme_ctx* c, int n, const double* xw) {
    NearList& nl = c->near;
    const BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    const int nb = bd.nb;
    int* flag = static_cast<int*>(nl.cb_flag.ensure(sizeof(int) * (nb + 1)));
    float4* hi = static_cast<float4*>(nl.cb_hi.ensure(sizeof(float4) * (n + 1)));
    float4* lo = static_cast<float4*>(nl.cb_lo.ensure(sizeof(float4) * (n + 1)));
    const double* L = c->p.box;
    // a body spanning at most 2 r_c (every bead within 2 r_c of the first bead), and
    // at most a quarter box so that intra-body differences are minimum images
    const double lim = fmin(2.0 * c->rc, 0.25 * fmin(L[0], fmin(L[1], L[2])));
    compact_flags_kernel<<<div_up(nb, 256), 256, 0, s>>>(nb, bd.off.as<int>(), flag);
    IBP_CHECK_LAUNCH();
    compact_rel_kernel<<<div_up(n, 256), 256, 0, s>>>(n, bd.bead_body.as<int>(), bd.off.as<int>(), xw, L[0], L[1], L[2],
                                                      lim * lim, flag, hi, lo);
    IBP_CHECK_LAUNCH();
    if (nl.cb_tasks_key == bd.version) return;
    const std::vector<int>& off = bd.host_off;
    auto blocks = [&](int S) {
        long long t = 0;
        for (int b = 0; b < nb; ++b) {
            const int m = off[b + 1] - off[b];
            if (m >= kCompactMin) t += (long long)div_up(m, kCbThreads) * div_up(m, S);
        }
        return t;
    };
    int S = 8;
    for (int cand : {1024, 512, 256, 128, 64, 32, 16}) {
        if (blocks(cand) >= 152LL * 8) {
            S = cand;
            break;
        }
    }
    std::vector<int4> tasks;
    for (int b = 0; b < nb; ++b) {
        const int o = off[b], m = off[b + 1] - off[b];
        if (m < kCompactMin) continue;
        for (int t = 0; t < m; t += kCbThreads)
            for (int u = 0; u < m; u += S)
                tasks.push_back(make_int4(b, o + t, o + u, (std::min(kCbThreads, m - t) << 20) | std::min(S, m - u)));
    }
    nl.cb_ntasks = (int)tasks.size();
    if (!tasks.empty()) {
        nl.cb_tasks.ensure(sizeof(int4) * tasks.size());
        IBP_CUDA(cudaMemcpyAsync(nl.cb_tasks.p, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice, s));
        IBP_CUDA(cudaStreamSynchronize(s));   // the host vector is replaced below
    }
    nl.cb_tasks_h = std::move(tasks);
    nl.cb_tasks_key = bd.version;
}

int cb_grid(int ntasks) { return ntasks < 152 * kCbBlocksPerSm ? ntasks : 152 * kCbBlocksPerSm; }

template <bool FP32>
void compact_apply(ibpme_ctx* c, const CbArgs& A, int n, const double* q, int nrhs, double* psi_r) {
    const int g = cb_grid(A.ntasks);
    const double ie = 1.0 / c->eps;
    cudaStream_t s = c->stream;
    if (FP32) {
        const size_t sm = sizeof(float4) * A.nt;
        switch (nrhs) {
            case 1: compact_apply32_kernel<1><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 2: compact_apply32_kernel<2><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 3: compact_apply32_kernel<3><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            default: compact_apply32_kernel<4><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
        }
    } else {
        const size_t sm = 2 * sizeof(float4) * A.nt;
        switch (nrhs) {
            case 1: compact_apply64_kernel<1><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 2: compact_apply64_kernel<2><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 3: compact_apply64_kernel<3><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 4: compact_apply64_kernel<4><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 5: compact_apply64_kernel<5><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 6: compact_apply64_kernel<6><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            case 7: compact_apply64_kernel<7><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
            default: compact_apply64_kernel<8><<<g, kCbThreads, sm, s>>>(A, n, q, ie, psi_r); break;
        }
    }
    IBP_CHECK_LAUNCH();
}

void compact_field(ibpme_ctx* c, int n, const double* q, int nrhs, double* E_r) {
    const CbArgs A = cb_args(c);
    const int g = cb_grid(A.ntasks);
    const double ie = 1.0 / c->eps;
    const size_t sm = 2 * sizeof(float4) * A.nt;
    cudaStream_t s = c->stream;
    switch (nrhs) {
        case 1: compact_field_kernel<1><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 2: compact_field_kernel<2><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 3: compact_field_kernel<3><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 4: compact_field_kernel<4><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 5: compact_field_kernel<5><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 6: compact_field_kernel<6><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        case 7: compact_field_kernel<7><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
        default: compact_field_kernel<8><<<g, kCbThreads, sm, s>>>(A, n, q, ie, E_r); break;
    }
    IBP_CHECK_LAUNCH();
}

}  // namespace

unsigned long long near_prefetch(ibpme_ctx* c, int n, const double* xw, const int* off, int noff) {
    NearList& nl = c->near;
    cudaStream_t s = c->stream;
    unsigned long long* fp = static_cast<unsigned long long*>(nl.fp_dev.ensure(3 * sizeof(unsigned long long)));
    IBP_CUDA(cudaMemsetAsync(fp, 0, 3 * sizeof(unsigned long long), s));
    if (n > 0) {
        fingerprint_kernel<<<div_up(3LL * n, 256) < 256 ? div_up(3LL * n, 256) : 256, 256, 0, s>>>(
            3LL * n, xw, nullptr, fp, reinterpret_cast<int*>(fp + 1));
        IBP_CHECK_LAUNCH();
    }
    hash_ints_kernel<<<std::max(1, std::min(div_up(noff, 256), 152)), 256, 0, s>>>(off, noff, fp + 2);
    IBP_CHECK_LAUNCH();
    unsigned long long* h = static_cast<unsigned long long*>(pinned_host(c, 3 * sizeof(unsigned long long)));
    IBP_CUDA(cudaMemcpyAsync(h, fp, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    nl.fp_pre[0] = h[0];
    nl.fp_pre[1] = (unsigned long long)*reinterpret_cast<int*>(h + 1);
    nl.fp_pre_n = n;
    nl.fp_pre_xw = xw;
    nl.fp_pre_valid = true;
    return h[2] | 1ull;
}

void near_build(ibpme_ctx* c, int n, const double* xw, bool need_grad) {
    (void)need_grad;   // the table always carries the gradient factors
    NearList& nl = c->near;
    cudaStream_t s = c->stream;
    ProfScope ps(ST_NEAR_BUILD, s);
    // positions unchanged since the last build (solve -> forces -> BD step): reuse the table
    unsigned long long print = 0;
    if (nl.fp_pre_valid && nl.fp_pre_n == n && nl.fp_pre_xw == xw) {   // fetched by the entry point
        nl.fp_pre_valid = false;
        if (nl.fp_pre[1] != 0) fail(IBPME_ERR_NONFINITE, "non-finite bead position");
        print = nl.fp_pre[0];
    } else {
        nl.fp_pre_valid = false;
        unsigned long long* fp = static_cast<unsigned long long*>(nl.fp_dev.ensure(3 * sizeof(unsigned long long)));
        int* bad = reinterpret_cast<int*>(fp + 1);
        IBP_CUDA(cudaMemsetAsync(fp, 0, 2 * sizeof(unsigned long long), s));
        if (n > 0) {
            fingerprint_kernel<<<div_up(3LL * n, 256) < 256 ? div_up(3LL * n, 256) : 256, 256, 0, s>>>(
                3LL * n, xw, c->bcfg, fp, bad);
            IBP_CHECK_LAUNCH();
        }
        unsigned long long* hfp = static_cast<unsigned long long*>(pinned_host(c, 2 * sizeof(unsigned long long)));
        IBP_CUDA(cudaMemcpyAsync(hfp, fp, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        IBP_CUDA(cudaStreamSynchronize(s));
        if (*reinterpret_cast<int*>(hfp + 1) != 0) fail(IBPME_ERR_NONFINITE, "non-finite bead position");
        print = hfp[0];
    }
    // compact bodies whenever the call has bodies (their structure is part of the cache key)
    const BodyData& bd = c->bodies;
    // (the compact kernels and the double-float pair values take one bead radius)
    const bool want_cb = c->bodies_current && bd.nmb > 0 && bd.host_n == n && make_const(c).K > 0 &&
                         c->ncls == 1 &&
                         std::getenv("IBPME_NO_COMPACT") == nullptr;   // the switch lets tests compare both paths
    const unsigned long long cb_key = want_cb ? bd.version : 0;
    if (nl.fp_valid && nl.n == n && nl.fp == print && nl.ncfg == c->ncfg && nl.cb_key == cb_key &&
        nl.cls_key == cls_key(c))
        return;
    nl.fp_valid = false;
    nl.ov_valid = false;
    nl.cb_on = false;
    nl.cb_key = cb_key;
    nl.cls_key = cls_key(c);
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
    PairConst k = make_const(c);
    if (want_cb && n > 0) {
        compact_prepare(c, n, xw);
        k.bbody = bd.bead_body.as<int>();
        k.cflag = nl.cb_flag.as<int>();
        nl.cb_on = true;
    }
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
    int* row_max = static_cast<int*>(nl.row_max.ensure(sizeof(int)));
    IBP_CUDA(cudaMemsetAsync(row_max, 0, sizeof(int), s));
    // padded rows only while they stay small next to the table itself
    const int cap = (long long)nl.ell_cap * n <= (1LL << 28) ? nl.ell_cap : 0;
    int* ell = cap > 0 ? static_cast<int*>(nl.ell.ensure(sizeof(int) * (size_t)cap * n)) : nullptr;
    if (n > 0) {
        pos32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, xf);
        IBP_CHECK_LAUNCH();
        pair_count_ell_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, xw, xf, k, cell_of, cell_start,
                                                                              cell_beads, cap, row_count, ell,
                                                                              row_max);
        IBP_CHECK_LAUNCH();
    }
    scan_counts(row_count, rowptr, n, nl.scan_tmp, s);
    long long* host_total = static_cast<long long*>(pinned_host(c, 2 * sizeof(long long)));
    IBP_CUDA(cudaMemcpyAsync(host_total, rowptr + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaMemcpyAsync(host_total + 1, row_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    nl.npairs = host_total[0];
    const int longest = *reinterpret_cast<const int*>(host_total + 1);
    const bool from_ell = n > 0 && cap > 0 && longest <= cap;
    nl.ell_cap = ((longest + longest / 4 + 8) + 7) / 8 * 8;   // the next build's padding
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
        int* prow = static_cast<int*>(nl.prow.ensure(sizeof(int) * np));
        if (from_ell)
            ell_compact_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, cap, ell, rowptr, col, prow);
        else
            pair_fill_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, xw, xf, k, cell_of, cell_start,
                                                                             cell_beads, rowptr, col, prow);
        IBP_CHECK_LAUNCH();
        if (c->ncls > 1) {   // beads of unequal radii: the exact two-radius kernel per pair
            double* self_b = static_cast<double*>(nl.self_b.ensure(sizeof(double) * (size_t)n));
            class_self_kernel<<<div_up(n, 256), 256, 0, s>>>(n, k.cls, k, self_b);
            IBP_CHECK_LAUNCH();
            if (nl.npairs > 0 && nl.cls_K > 0 && nl.npairs < (1LL << 31)) {
                // double-float tables per pair of classes, overlapping shells listed and valued exactly
                float4* xdf = static_cast<float4*>(nl.xdf.ensure(sizeof(float4) * 2 * (size_t)(n + 1)));
                pos_df_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, xdf);
                IBP_CHECK_LAUNCH();
                int* ov_list = static_cast<int*>(nl.ov_list.ensure(sizeof(int) * np));
                int* ov_count = static_cast<int*>(nl.ov_count.ensure(sizeof(int)));
                IBP_CUDA(cudaMemsetAsync(ov_count, 0, sizeof(int), s));
                DfPairArgs A{};
                A.xdf = xdf;
                A.tabdf = nl.cls_tabdf.as<float4>();
                A.K = nl.cls_K;
                for (int d = 0; d < 3; ++d) {
                    A.L[d] = host_df(k.L[d]);
                    A.halfL[d] = (float)(0.5 * k.L[d]);
                }
                DfClassArgs CA{};
                CA.cls = k.cls;
                CA.ncls = c->ncls;
                CA.stride = 3LL * nl.cls_K * kOctaveIntervals;
                for (int a2 = 0; a2 < c->ncls; ++a2)
                    for (int b2 = 0; b2 < c->ncls; ++b2) {
                        const double sab = c->cls_a[a2] + c->cls_a[b2];
                        CA.inv_s2[a2 * c->ncls + b2] = host_df(1.0 / (sab * sab));
                    }
                pair_values_df_cls_kernel<<<div_up(nl.npairs, 256), 256, 0, s>>>(
                    nl.npairs, A, CA, prow, col, cell_beads, val, pair32, gfac, ov_list, ov_count);
                IBP_CHECK_LAUNCH();
                pair_values_exact_kernel<<<152 * 4, 128, 0, s>>>(ov_count, ov_list, xw, k, prow, col, cell_beads, val,
                                                                 pair32, gfac);
                IBP_CHECK_LAUNCH();
                nl.ov_valid = true;
            } else if (nl.npairs > 0) {
                pair_values_cls_kernel<<<div_up(nl.npairs, 256), 256, 0, s>>>(nl.npairs, xw, k, prow, col,
                                                                              cell_beads, val, pair32, gfac);
                IBP_CHECK_LAUNCH();
            }
        } else if (nl.npairs > 0 && k.K > 0 && nl.npairs < (1LL << 31)) {
            // table pairs in double-float arithmetic, overlapping beads listed and valued exactly
            float4* xdf = static_cast<float4*>(nl.xdf.ensure(sizeof(float4) * 2 * (size_t)(n + 1)));
            pos_df_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, xdf);
            IBP_CHECK_LAUNCH();
            int* ov_list = static_cast<int*>(nl.ov_list.ensure(sizeof(int) * np));
            int* ov_count = static_cast<int*>(nl.ov_count.ensure(sizeof(int)));
            IBP_CUDA(cudaMemsetAsync(ov_count, 0, sizeof(int), s));
            DfPairArgs A{};
            A.xdf = xdf;
            A.tabdf = nl.tab_df.as<float4>();
            A.K = k.K;
            A.inv4a2 = host_df(k.inv4a2);
            for (int d = 0; d < 3; ++d) {
                A.L[d] = host_df(k.L[d]);
                A.halfL[d] = (float)(0.5 * k.L[d]);
            }
            pair_values_df_kernel<<<div_up(nl.npairs, 256), 256, 0, s>>>(nl.npairs, A, prow, col, cell_beads, val,
                                                                        pair32, gfac, ov_list, ov_count);
            IBP_CHECK_LAUNCH();
            pair_values_exact_kernel<<<152 * 4, 128, 0, s>>>(ov_count, ov_list, xw, k, prow, col, cell_beads, val,
                                                             pair32, gfac);
            IBP_CHECK_LAUNCH();
            nl.ov_valid = true;
        } else if (nl.npairs > 0) {
            pair_values_kernel<<<div_up(nl.npairs, 256), 256, 0, s>>>(nl.npairs, xw, k, prow, col, cell_beads, val,
                                                                     pair32, gfac);
            IBP_CHECK_LAUNCH();
        }
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
    const double* sv = c->ncls > 1 ? nl.self_b.as<double>() : nullptr;   // self term of each bead's class
    if (fp32) {
        float4* qf = static_cast<float4*>(nl.qf.ensure(sizeof(float4) * n));
        pack_q32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, q, qf);
        IBP_CHECK_LAUNCH();
        const uint2* pc = nl.pair32.as<uint2>();
        switch (nrhs) {
            case 1: near_apply32_kernel<1><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, q, psi_r); break;
            case 2: near_apply32_kernel<2><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, q, psi_r); break;
            case 3: near_apply32_kernel<3><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, q, psi_r); break;
            default: near_apply32_kernel<4><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, q, psi_r); break;
        }
        IBP_CHECK_LAUNCH();
        if (nl.cb_on && nl.cb_ntasks > 0) compact_apply<true>(c, cb_args(c), n, q, nrhs, psi_r);
        return;
    }
    double* qs = static_cast<double*>(nl.qs.ensure(sizeof(double) * (size_t)n * nrhs));
    pack_q64_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, q, qs);
    IBP_CHECK_LAUNCH();
    switch (nrhs) {
        case 1: near_apply_kernel<1><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 2: near_apply_kernel<2><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 3: near_apply_kernel<3><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 4: near_apply_kernel<4><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 5: near_apply_kernel<5><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 6: near_apply_kernel<6><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        case 7: near_apply_kernel<7><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
        default: near_apply_kernel<8><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, q, psi_r); break;
    }
    IBP_CHECK_LAUNCH();
    if (nl.cb_on && nl.cb_ntasks > 0) compact_apply<false>(c, cb_args(c), n, q, nrhs, psi_r);
}

void near_field(ibpme_ctx* c, int n, const double* xw, const double* q, int nrhs, double* E_r) {
    if (n == 0) return;
    ProfScope ps(ST_NEAR_FIELD, c->stream);
    if (!c->near.have_grad) fail(IBPME_ERR_ARG, "internal: pair table built without gradients");
    NearList& nl = c->near;
    const PairConst k = make_const(c);
    IBP_CUDA(cudaMemsetAsync(E_r, 0, sizeof(double) * 3 * (size_t)nrhs * n, c->stream));
    if (nl.npairs > 0 && nl.ov_valid) {   // double-float positions of this table are current
        DfPairArgs A{};
        A.xdf = nl.xdf.as<float4>();
        for (int d = 0; d < 3; ++d) {
            A.L[d] = host_df(k.L[d]);
            A.halfL[d] = (float)(0.5 * k.L[d]);
        }
        near_field_df_kernel<<<div_up(nl.npairs, 256), 256, 0, c->stream>>>(
            nl.npairs, n, nrhs, A, nl.prow.as<int>(), nl.col.as<int>(), nl.cell_beads.as<int>(), nl.gfac.as<double>(),
            host_df(1.0 / c->eps), q, E_r);
        IBP_CHECK_LAUNCH();
    } else if (nl.npairs > 0) {
        near_field_kernel<<<div_up(nl.npairs, 256), 256, 0, c->stream>>>(
            nl.npairs, n, nrhs, xw, k, nl.prow.as<int>(), nl.col.as<int>(), nl.cell_beads.as<int>(),
            nl.gfac.as<double>(), 1.0 / c->eps, q, E_r);
        IBP_CHECK_LAUNCH();
    }
    if (nl.cb_on && nl.cb_ntasks > 0) compact_field(c, n, q, nrhs, E_r);
}

namespace {

// ---- the free beads on their own (the Krylov operator's sources and targets) ----

// Pair-table row (cell-sorted position) of every bead.
__global__ void invert_order_kernel(int n, const int* __restrict__ order, int* __restrict__ inv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) inv[order[t]] = t;
}

// Wrapped positions of the free beads in list order.
__global__ void free_positions_kernel(int nfree, const int* __restrict__ free_idx, const double* __restrict__ xw,
                                      double* __restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * nfree) return;
    const int f = i / 3, d = i - 3 * f;
    xf[i] = xw[3 * free_idx[f] + d];
}

// Radius class and self term of each free bead.
__global__ void free_class_kernel(int nfree, const int* __restrict__ free_idx, const int* __restrict__ cls,
                                  const double* __restrict__ self_b, int* __restrict__ cls_f,
                                  double* __restrict__ self_f) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfree) return;
    cls_f[f] = cls[free_idx[f]];
    self_f[f] = self_b[free_idx[f]];
}

// Compact-body relative positions in list order.
__global__ void free_rel_kernel(int nfree, const int* __restrict__ free_idx, const float4* __restrict__ hi,
                                const float4* __restrict__ lo, float4* __restrict__ fhi, float4* __restrict__ flo) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfree) return;
    fhi[f] = hi[free_idx[f]];
    flo[f] = lo[free_idx[f]];
}

// Pairs of free bead f's table row whose other bead is free too (one thread per row).
__global__ void ff_count_kernel(int nfree, const int* __restrict__ free_idx, const int* __restrict__ sorted_of,
                                const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ order, const int* __restrict__ free_pos,
                                int* __restrict__ count) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfree) return;
    const int t = sorted_of[free_idx[f]];
    int k = 0;
    for (long long p = rowptr[t]; p < rowptr[t + 1]; ++p) k += free_pos[order[col[p]]] >= 0 ? 1 : 0;
    count[f] = k;
}

// Those pairs in list indices: column, FP64 value and the (column, FP32 value) word.
__global__ void ff_fill_kernel(int nfree, const int* __restrict__ free_idx, const int* __restrict__ sorted_of,
                               const long long* __restrict__ rowptr, const int* __restrict__ col,
                               const int* __restrict__ order, const int* __restrict__ free_pos,
                               const double* __restrict__ val, const uint2* __restrict__ pair32,
                               const long long* __restrict__ fptr, int* __restrict__ fcol, double* __restrict__ fval,
                               uint2* __restrict__ fpair32) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfree) return;
    const int t = sorted_of[free_idx[f]];
    long long k = fptr[f];
    for (long long p = rowptr[t]; p < rowptr[t + 1]; ++p) {
        const int g = free_pos[order[col[p]]];
        if (g < 0) continue;
        fcol[k] = g;
        fval[k] = val[p];
        fpair32[k] = make_uint2((unsigned)g, pair32[p].y);
        ++k;
    }
}

CbArgs cb_args_free(const ibpme_ctx* c) {
    CbArgs A = cb_args(c);
    A.tasks = c->fs.cb_tasks.as<int4>();
    A.ntasks = c->fs.cb_ntasks;
    A.hi = c->fs.cb_hi.as<float4>();
    A.lo = c->fs.cb_lo.as<float4>();
    return A;
}

}  // namespace

bool near_free_build(ibpme_ctx* c, const double* xw) {
    NearList& nl = c->near;
    FreeSet& fs = c->fs;
    const BodyData& bd = c->bodies;
    const int n = nl.n, nf = bd.nfree;
    if (!nl.fp_valid || !c->bodies_current || bd.host_n != n || nf == 0) return false;
    if (fs.valid && fs.fp == nl.fp && fs.version == bd.version && fs.nfree == nf && fs.cls_key == cls_key(c))
        return true;
    cudaStream_t s = c->stream;
    fs.valid = false;
    fs.nfree = nf;
    const int* fidx = bd.free_idx.as<int>();
    if (c->ncls > 1) {   // class and self term of each free bead
        int* cf = static_cast<int*>(fs.cls_f.ensure(sizeof(int) * (size_t)nf));
        double* sf = static_cast<double*>(fs.self_f.ensure(sizeof(double) * (size_t)nf));
        free_class_kernel<<<div_up(nf, 256), 256, 0, s>>>(nf, fidx, c->cls.as<int>(), nl.self_b.as<double>(), cf, sf);
        IBP_CHECK_LAUNCH();
    }
    fs.cls_key = cls_key(c);
    double* xf = static_cast<double*>(fs.xf.ensure(sizeof(double) * 3 * (size_t)nf));
    free_positions_kernel<<<div_up(3LL * nf, 256), 256, 0, s>>>(nf, fidx, xw, xf);
    IBP_CHECK_LAUNCH();
    // the table's pairs between two free beads, re-indexed into the list
    int* sorted_of = static_cast<int*>(fs.sorted_of.ensure(sizeof(int) * (n + 1)));
    invert_order_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nl.cell_beads.as<int>(), sorted_of);
    IBP_CHECK_LAUNCH();
    int* cnt = static_cast<int*>(fs.row_count.ensure(sizeof(int) * (nf + 1)));
    long long* fptr = static_cast<long long*>(fs.rowptr.ensure(sizeof(long long) * (nf + 1)));
    ff_count_kernel<<<div_up(nf, 128), 128, 0, s>>>(nf, fidx, sorted_of, nl.rowptr.as<long long>(), nl.col.as<int>(),
                                                    nl.cell_beads.as<int>(), bd.free_pos.as<int>(), cnt);
    IBP_CHECK_LAUNCH();
    scan_counts(cnt, fptr, nf, fs.scan_tmp, s);
    long long* host_total = static_cast<long long*>(pinned_host(c, sizeof(long long)));
    IBP_CUDA(cudaMemcpyAsync(host_total, fptr + nf, sizeof(long long), cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    fs.npairs = *host_total;
    const size_t np = (size_t)(fs.npairs > 0 ? fs.npairs : 1);
    int* fcol = static_cast<int*>(fs.col.ensure(sizeof(int) * np));
    double* fval = static_cast<double*>(fs.val.ensure(sizeof(double) * np));
    uint2* fp32 = static_cast<uint2*>(fs.pair32.ensure(sizeof(uint2) * np));
    if (fs.npairs > 0) {
        ff_fill_kernel<<<div_up(nf, 128), 128, 0, s>>>(nf, fidx, sorted_of, nl.rowptr.as<long long>(), nl.col.as<int>(),
                                                       nl.cell_beads.as<int>(), bd.free_pos.as<int>(),
                                                       nl.val.as<double>(), nl.pair32.as<uint2>(), fptr, fcol, fval,
                                                       fp32);
        IBP_CHECK_LAUNCH();
    }
    fs.qf.ensure(sizeof(float4) * (nf + 1));
    fs.qs.ensure(sizeof(double) * (size_t)(nf + 1) * kMaxRhs);
    // compact bodies: relative positions in list order, tasks in list indices (a task's
    // targets and sources lie in one body, whose free beads are consecutive in the list)
    if (nl.cb_on && nl.cb_ntasks > 0) {
        float4* fhi = static_cast<float4*>(fs.cb_hi.ensure(sizeof(float4) * (nf + 1)));
        float4* flo = static_cast<float4*>(fs.cb_lo.ensure(sizeof(float4) * (nf + 1)));
        free_rel_kernel<<<div_up(nf, 256), 256, 0, s>>>(nf, fidx, nl.cb_hi.as<float4>(), nl.cb_lo.as<float4>(), fhi,
                                                         flo);
        IBP_CHECK_LAUNCH();
        if (fs.cb_tasks_key != nl.cb_tasks_key || fs.cb_ntasks != nl.cb_ntasks) {
            std::vector<int4> t(nl.cb_tasks_h);
            for (int4& w : t) {
                w.y = bd.free_pos_h[w.y];
                w.z = bd.free_pos_h[w.z];
                if (w.y < 0 || w.z < 0) fail(IBPME_ERR_ARG, "internal: compact-body task outside the free beads");
            }
            fs.cb_tasks.ensure(sizeof(int4) * t.size());
            IBP_CUDA(cudaMemcpyAsync(fs.cb_tasks.p, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice, s));
            IBP_CUDA(cudaStreamSynchronize(s));   // the host vector goes out of scope
            fs.cb_ntasks = (int)t.size();
            fs.cb_tasks_key = nl.cb_tasks_key;
        }
    } else {
        fs.cb_ntasks = 0;
        fs.cb_tasks_key = 0;
    }
    fs.fp = nl.fp;
    fs.version = bd.version;
    fs.valid = true;
    return true;
}

void near_apply_free(ibpme_ctx* c, const double* qc, int nrhs, double* psi_r, bool fp32) {
    FreeSet& fs = c->fs;
    const int n = fs.nfree;
    if (n == 0) return;
    fp32 = fp32 && nrhs <= 4;
    ProfScope ps(fp32 ? ST_NEAR_APPLY32 : ST_NEAR_APPLY, c->stream);
    const PairConst k = make_const(c);
    const int blocks = div_up((long long)n * 32, 128);
    const long long* rp = fs.rowptr.as<long long>();
    const double ie = 1.0 / c->eps;
    cudaStream_t s = c->stream;
    const int* od = c->bodies.iota.as<int>();   // rows are list positions already
    const bool cb = c->near.cb_on && fs.cb_ntasks > 0;
    const double* sv = c->ncls > 1 ? fs.self_f.as<double>() : nullptr;
    if (fp32) {
        float4* qf = fs.qf.as<float4>();
        pack_q32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, qc, qf);
        IBP_CHECK_LAUNCH();
        const uint2* pc = fs.pair32.as<uint2>();
        switch (nrhs) {
            case 1: near_apply32_kernel<1><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, qc, psi_r); break;
            case 2: near_apply32_kernel<2><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, qc, psi_r); break;
            case 3: near_apply32_kernel<3><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, qc, psi_r); break;
            default: near_apply32_kernel<4><<<blocks, 128, 0, s>>>(n, rp, pc, od, k.self, sv, ie, qf, qc, psi_r); break;
        }
        IBP_CHECK_LAUNCH();
        if (cb) compact_apply<true>(c, cb_args_free(c), n, qc, nrhs, psi_r);
        return;
    }
    double* qs = fs.qs.as<double>();
    pack_q64_kernel<<<div_up(n, 256), 256, 0, s>>>(n, nrhs, od, qc, qs);
    IBP_CHECK_LAUNCH();
    const int* cl = fs.col.as<int>();
    const double* vl = fs.val.as<double>();
    switch (nrhs) {
        case 1: near_apply_kernel<1><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 2: near_apply_kernel<2><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 3: near_apply_kernel<3><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 4: near_apply_kernel<4><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 5: near_apply_kernel<5><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 6: near_apply_kernel<6><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        case 7: near_apply_kernel<7><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
        default: near_apply_kernel<8><<<blocks, 128, 0, s>>>(n, rp, cl, vl, od, k.self, sv, ie, qs, qc, psi_r); break;
    }
    IBP_CHECK_LAUNCH();
    if (cb) compact_apply<false>(c, cb_args_free(c), n, qc, nrhs, psi_r);
}

}  // namespace ibp
