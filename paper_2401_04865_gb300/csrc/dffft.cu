// dffft.cu -- the FP64 mesh's 3-D transforms in double-float arithmetic.
//
// The true residual of a mixed-precision solve and every FP64-context PME
// evaluation (Sec. III.D.3 steps 3-5) transform the FP64 grid.  GB300 executes
// FP64 at a small fraction of its FP32 rate, and cuFFT's D2Z/Z2D of a 128^3 grid
// is bound by that FP64 pipe.  Here each value is carried as an unevaluated sum
// of two floats (hi + lo, about 48 significant bits; error-free transformations
// of Dekker and Knuth: two-sum, and two-product with a fused multiply-add), so
// the butterflies run on the FP32 pipes.  The transforms are Stockham passes
// (radix 3 when 3 divides the size, radix 8, then radix 4 or 2) in shared memory
// along x (two real lines packed into one complex line), y and z on the half
// spectrum; the Green's-function scaling of the FP64 table is fused between the
// forward and inverse z passes, and the real lines come back as FP64.  Sizes
// 2^k and 3 2^k (16 to 1024); other sizes use cuFFT.
#include "common.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ibp {

namespace {

constexpr int kDfPoints = 1024;   // points per block (lines x line length)
constexpr int kDfThreads = 128;   // eight points per thread in each radix-8 pass
constexpr int kDfMinBlocks = 8;   // resident blocks per SM the register budget is set for
// Shared memory: point i of a line at line * ls + i + i / 8 (a stride-8 store of the
// first pass then spreads over the banks), ls = n + n / 8 + 1 (odd: column loads spread too)
constexpr int kDfSmem = kDfPoints + kDfPoints / 8 + kDfPoints / 16;
__host__ __device__ constexpr int df_ls(int n) { return n + n / 8 + 1; }
__device__ __forceinline__ int sw(int i) { return i + (i >> 3); }

// Accuracy of the double-float operations (dfloat.cuh): each is exact to about
// 2^-44 of its operands' magnitude, so a length-N transform keeps a normwise
// error near log2(N) 2^-44, far below the FP32 mesh and the 1e-6 residual test
// it serves.
struct dfc {
    df re, im;
};

__device__ __forceinline__ dfc load_c(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 store_c(const dfc& c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }

// (a + ib) (c + id) with w = c + id; conj selects c - id
__device__ __forceinline__ dfc cmul(const dfc& x, const dfc& w, bool conj) {
    const df wi = conj ? df_neg(w.im) : w.im;
    const df re = df_add(df_mul(x.re, w.re), df_neg(df_mul(x.im, wi)));
    const df im = df_add(df_mul(x.re, wi), df_mul(x.im, w.re));
    return {re, im};
}

// Multiplication by (1 -+ i) / sqrt(2) (forward / inverse) and by -+i.
__device__ __forceinline__ dfc mul_w8(const dfc& x, bool inv) {
    constexpr float ch = 0.70710677f;
    constexpr float cl = (float)(0.70710678118654752440 - (double)ch);
    const df c = {ch, cl};
    // forward: (x + iy)(1 - i) = (x + y) + i (y - x); inverse: (x - y) + i (x + y)
    const df a = df_add(x.re, inv ? df_neg(x.im) : x.im);
    const df b = inv ? df_add(x.re, x.im) : df_add(x.im, df_neg(x.re));
    return {df_mul(a, c), df_mul(b, c)};
}

__device__ __forceinline__ dfc mul_mi(const dfc& x, bool inv) {   // forward -i x, inverse +i x
    return inv ? dfc{df_neg(x.im), x.re} : dfc{x.im, df_neg(x.re)};
}

__device__ __forceinline__ dfc cadd(const dfc& a, const dfc& b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc csub(const dfc& a, const dfc& b) {
    return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))};
}

// R-point DFTs in registers, y_q = sum_m v_m exp(-+2 pi i m q / R).
template <bool INV>
__device__ __forceinline__ void dft2(dfc* v) {
    const dfc a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(dfc* v) {
    const dfc a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    const dfc a2 = cadd(v[1], v[3]), a3 = mul_mi(csub(v[1], v[3]), INV);
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <bool INV>
__device__ __forceinline__ void dft8(dfc* v) {
    dfc e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    o[1] = mul_w8(o[1], INV);
    o[2] = mul_mi(o[2], INV);
    o[3] = mul_mi(mul_w8(o[3], INV), INV);   // w8^3 = w8 w4
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = cadd(e[q], o[q]);
        v[q + 4] = csub(e[q], o[q]);
    }
}

// Radix-3 DFT: t1 = v1 + v2, t2 = v0 - t1/2, t3 = -+i (sqrt(3)/2)(v1 - v2);
// y0 = v0 + t1, y1 = t2 + t3, y2 = t2 - t3.
template <bool INV>
__device__ __forceinline__ void dft3(dfc* v) {
    constexpr float ch = 0.86602540f;
    constexpr float cl = (float)(0.86602540378443864676 - (double)ch);
    const df c = {ch, cl};
    const dfc t1 = cadd(v[1], v[2]);
    const dfc t2 = {df_add(v[0].re, df_neg(df_half(t1.re))), df_add(v[0].im, df_neg(df_half(t1.im)))};
    const dfc d = csub(v[1], v[2]);
    // forward: -i c d = c (d.im, -d.re); inverse: +i c d = c (-d.im, d.re)
    const dfc t3 = INV ? dfc{df_neg(df_mul(d.im, c)), df_mul(d.re, c)} : dfc{df_mul(d.im, c), df_neg(df_mul(d.re, c))};
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
}

// One Stockham pass of radix R over the block's lines (pts = lines x n points) in
// shared memory, natural order in and out: butterfly j of a line takes the points
// j + r n/R, applies the twiddles exp(-+2 pi i k r / (Ns R)), k = j mod Ns, and
// writes its R outputs to (j - k) R + k + r Ns.  tw[t] = exp(-2 pi i t / n), t < n.
// A thread holds all its butterflies in registers between the loads and the stores.
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(float4* buf, int ls, int n, int pts, int Ns,
                                              const float4* __restrict__ tw) {
    constexpr int per = (kDfPoints / R + kDfThreads - 1) / kDfThreads;   // butterflies per thread at most
    const int nb = n / R, nbf = pts / R;
    dfc v[per][R];
    int out[per];
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int b = threadIdx.x + q * kDfThreads;
        out[q] = -1;
        if (b >= nbf) continue;
        const int line = b / nb, j = b - line * nb;
        const int k = j % Ns;
        const float4* x = buf + line * ls;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = load_c(x[sw(j + r * nb)]);
        if (Ns > 1) {   // the first pass (Ns = 1) has k = 0: every twiddle is 1
            const int step = k * (n / (Ns * R));
#pragma unroll
            for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], load_c(tw[r * step]), INV);
        }
        if (R == 8) dft8<INV>(v[q]);
        else if (R == 4) dft4<INV>(v[q]);
        else if (R == 3) dft3<INV>(v[q]);
        else dft2<INV>(v[q]);
        out[q] = line * ls + (j - k) * R + k;   // line offset + first output (before the swizzle)
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < per; ++q) {
        if (out[q] < 0) continue;
        const int b = threadIdx.x + q * kDfThreads;
        const int line = b / nb;
        const int o = out[q] - line * ls;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[line * ls + sw(o + r * Ns)] = store_c(v[q][r]);
    }
    __syncthreads();
}

// Length-n transforms (n = 2^m or 3 2^m) of every line of the block (natural order in
// and out): a radix-3 pass first when 3 divides n, then radix-8 passes, then one
// radix-4 or radix-2 pass.
template <bool INV>
__device__ void fft_lines(float4* buf, int n, int logm, int pts, const float4* __restrict__ tw) {
    const int ls = df_ls(n);
    int Ns = 1, l = logm;
    if (n % 3 == 0) {
        stockham_pass<3, INV>(buf, ls, n, pts, Ns, tw);
        Ns = 3;
    }
    for (; l >= 3; l -= 3, Ns *= 8) stockham_pass<8, INV>(buf, ls, n, pts, Ns, tw);
    if (l == 2) stockham_pass<4, INV>(buf, ls, n, pts, Ns, tw);
    else if (l == 1) stockham_pass<2, INV>(buf, ls, n, pts, Ns, tw);
}

struct DfGeom {
    int n[3], logn[3];   // size and log2 of its power-of-two factor per axis
    int pl[3];           // lines (x) or columns (y, z) per block: lines x n <= kDfPoints
    int h;          // half-spectrum row length N_x / 2 + 1
    long long G;    // real points per channel
    long long Gh;   // half-spectrum points per channel (N_y N_z h)
};


// x pass, forward.  Two real lines a, b travel as one complex line a + i b; after
// its transform Z, A[k] = (Z[k] + conj Z[N-k]) / 2 and B[k] = (Z[k] - conj Z[N-k]) / 2i
// are the spectra of a and b; their halves k = 0 .. N/2 go to S.
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
dfx_forward_kernel(DfGeom d, const double* __restrict__ grid, float4* __restrict__ S, const float4* __restrict__ tw) {
    __shared__ float4 buf[kDfSmem];
    const int n = d.n[0], pl = d.pl[0], ls = df_ls(n), pts = pl * n;   // packed lines per block
    const size_t ch = blockIdx.y;
    const long long line0 = (long long)blockIdx.x * 2 * pl;   // first real line
    const double* src = grid + ch * d.G + line0 * n;
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int p = e / n, i = e % n;
        const df a = df_split(src[(size_t)(2 * p) * n + i]);
        const df b = df_split(src[(size_t)(2 * p + 1) * n + i]);
        buf[p * ls + sw(i)] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    __syncthreads();
    fft_lines<false>(buf, n, d.logn[0], pts, tw);
    float4* dst = S + ch * d.Gh + line0 * d.h;
    for (int e = threadIdx.x; e < pl * d.h; e += kDfThreads) {
        const int p = e / d.h, k = e % d.h;
        const dfc zk = load_c(buf[p * ls + sw(k)]);
        const dfc zm = load_c(buf[p * ls + sw(k == 0 ? 0 : n - k)]);   // Z[N - k], conjugated below
        const dfc A = {df_half(df_add(zk.re, zm.re)), df_half(df_add(zk.im, df_neg(zm.im)))};
        // (Z[k] - conj Z[N-k]) / 2i: re = (zk.im + zm.im) / 2, im = -(zk.re - zm.re) / 2
        const dfc B = {df_half(df_add(zk.im, zm.im)), df_half(df_add(zm.re, df_neg(zk.re)))};
        dst[(size_t)(2 * p) * d.h + k] = store_c(A);
        dst[(size_t)(2 * p + 1) * d.h + k] = store_c(B);
    }
}

// x pass, inverse: the half spectra A, B of two lines rebuild Z = A + i B on all
// N points (Z[N-k] = conj A[k] + i conj B[k]); the inverse transform's real and
// imaginary parts are the two real lines, returned as hi + lo floats (the gathers
// read them in double-float arithmetic).
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
dfx_inverse_kernel(DfGeom d, const float4* __restrict__ S, float2* __restrict__ grid, const float4* __restrict__ tw) {
    __shared__ float4 buf[kDfSmem];
    const int n = d.n[0], pl = d.pl[0], ls = df_ls(n), pts = pl * n;
    const size_t ch = blockIdx.y;
    const long long line0 = (long long)blockIdx.x * 2 * pl;
    const float4* src = S + ch * d.Gh + line0 * d.h;
    for (int e = threadIdx.x; e < pl * d.h; e += kDfThreads) {
        const int p = e / d.h, k = e % d.h;
        const dfc A = load_c(src[(size_t)(2 * p) * d.h + k]);
        const dfc B = load_c(src[(size_t)(2 * p + 1) * d.h + k]);
        // Z[k] = A + i B
        const dfc zk = {df_add(A.re, df_neg(B.im)), df_add(A.im, B.re)};
        buf[p * ls + sw(k)] = store_c(zk);
        if (k > 0 && k < n / 2) {   // Z[N-k] = conj A + i conj B
            const dfc zm = {df_add(A.re, B.im), df_add(df_neg(A.im), B.re)};
            buf[p * ls + sw(n - k)] = store_c(zm);
        }
    }
    __syncthreads();
    fft_lines<true>(buf, n, d.logn[0], pts, tw);
    float2* dst = grid + ch * d.G + line0 * n;
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int p = e / n, i = e % n;
        const float4 v = buf[p * ls + sw(i)];
        dst[(size_t)(2 * p) * n + i] = make_float2(v.x, v.y);
        dst[(size_t)(2 * p + 1) * n + i] = make_float2(v.z, v.w);
    }
}

// y pass (either direction) on the half spectrum: columns x0 .. x0 + cols of one
// z-plane (the last group of columns may be partial)
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
dfy_kernel(DfGeom d, float4* __restrict__ S, const float4* __restrict__ tw, int inverse) {
    __shared__ float4 buf[kDfSmem];
    const int n = d.n[1], cols = d.pl[1], h = d.h, ls = df_ls(n), pts = cols * n;
    const size_t ch = blockIdx.y;
    const int blocks_x = (h + cols - 1) / cols;
    const int z = blockIdx.x / blocks_x, x0 = (blockIdx.x % blocks_x) * cols;
    float4* plane = S + ch * d.Gh + (size_t)z * n * h;
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int y = e / cols, c = e % cols;   // consecutive threads: consecutive x (coalesced)
        buf[c * ls + sw(y)] = x0 + c < h ? plane[(size_t)y * h + x0 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (inverse)
        fft_lines<true>(buf, n, d.logn[1], pts, tw);
    else
        fft_lines<false>(buf, n, d.logn[1], pts, tw);
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int y = e / cols, c = e % cols;
        if (x0 + c < h) plane[(size_t)y * h + x0 + c] = buf[c * ls + sw(y)];
    }
}

// z pass on the half spectrum: forward FFT, Green's-function scaling (the FP64
// half-spectrum table split into hi + lo floats), inverse FFT, for columns
// x0 .. x0 + cols at one y.  mode 1 stops after the forward FFT and mode 2 runs the
// inverse FFT alone (radius classes: the scaling mixes the channels in between).
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
dfz_scale_kernel(DfGeom d, float4* __restrict__ S, const float4* __restrict__ tw, const float2* __restrict__ green,
                 int mode) {
    __shared__ float4 buf[kDfSmem];
    const int n = d.n[2], cols = d.pl[2], ny = d.n[1], h = d.h, ls = df_ls(n), pts = cols * n;
    const size_t ch = blockIdx.y;
    const int blocks_x = (h + cols - 1) / cols;
    const int y = blockIdx.x / blocks_x, x0 = (blockIdx.x % blocks_x) * cols;
    const size_t zstride = (size_t)h * ny;
    float4* col = S + ch * d.Gh + (size_t)y * h + x0;
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int z = e / cols, c = e % cols;
        buf[c * ls + sw(z)] = x0 + c < h ? col[(size_t)z * zstride + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (mode != 2) fft_lines<false>(buf, n, d.logn[2], pts, tw);
    if (mode == 0) {
        for (int e = threadIdx.x; e < pts; e += kDfThreads) {
            const int c = e / n, z = e % n;
            if (x0 + c >= h) continue;
            const float2 gv = green[((size_t)z * ny + y) * h + x0 + c];
            const df gk = {gv.x, gv.y};
            float4& slot = buf[c * ls + sw(z)];
            dfc v = load_c(slot);
            v.re = df_mul(v.re, gk);
            v.im = df_mul(v.im, gk);
            slot = store_c(v);
        }
        __syncthreads();
    }
    if (mode != 1) fft_lines<true>(buf, n, d.logn[2], pts, tw);
    for (int e = threadIdx.x; e < pts; e += kDfThreads) {
        const int z = e / cols, c = e % cols;
        if (x0 + c < h) col[(size_t)z * zstride + c] = buf[c * ls + sw(z)];
    }
}

// Scaling with radius classes between the z passes, in double-float arithmetic: for
// every right-hand side r, S = sum_c j0(k a_c) H(c, r), then H(d, r) = G(k) j0(k a_d) S,
// G and j0 as hi + lo floats ([Gh] and [ncls][Gh]).
__global__ void dfz_mix_kernel(long long Gh, int nrhs, int ncls, float4* __restrict__ S,
                               const float2* __restrict__ green, const float2* __restrict__ jtab) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < Gh; t += (long long)gridDim.x * blockDim.x) {
        const df gk = {green[t].x, green[t].y};
        df j[IBPME_MAX_RADIUS_CLASSES];
        for (int c = 0; c < ncls; ++c) j[c] = df{jtab[(size_t)c * Gh + t].x, jtab[(size_t)c * Gh + t].y};
        for (int r = 0; r < nrhs; ++r) {
            dfc sum = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            for (int c = 0; c < ncls; ++c) {
                const dfc v = load_c(S[(size_t)(c * nrhs + r) * Gh + t]);
                sum.re = df_add(sum.re, df_mul(v.re, j[c]));
                sum.im = df_add(sum.im, df_mul(v.im, j[c]));
            }
            for (int dd = 0; dd < ncls; ++dd) {
                const df f = df_mul(gk, j[dd]);
                S[(size_t)(dd * nrhs + r) * Gh + t] = store_c(dfc{df_mul(sum.re, f), df_mul(sum.im, f)});
            }
        }
    }
}

// RPY wave space between the z passes (three force channels): F(k) becomes
// fac (1 + k^2/(4 xi^2)) G(k) (I - k_hat k_hat) F(k), the scalar and the projection
// formed in FP64 per k and applied in double-float arithmetic; zero at k = 0.
__global__ void dfz_rpy_kernel(DfGeom d, RpyScale R, float4* __restrict__ S, const float2* __restrict__ green) {
    const double two_pi = 6.283185307179586476925286766559;
    const int h = d.h, ny = d.n[1], nz = d.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d.Gh;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % h);
        const long long rest = t / h;
        const int y = (int)(rest % ny), z = (int)(rest / ny);
        const int my = y <= ny / 2 ? y : y - ny, mz = z <= nz / 2 ? z : z - nz;
        const double k[3] = {two_pi * x / R.L[0], two_pi * my / R.L[1], two_pi * mz / R.L[2]};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        dfc v[3];
        for (int c = 0; c < 3; ++c) v[c] = load_c(S[(size_t)c * d.Gh + t]);
        if (k2 == 0.0) {
            for (int c = 0; c < 3; ++c) S[(size_t)c * d.Gh + t] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const double w = ((double)green[t].x + (double)green[t].y) * (1.0 + k2 / (4.0 * R.xi * R.xi)) * R.fac;
        for (int c = 0; c < 3; ++c) {
            dfc o = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            for (int e = 0; e < 3; ++e) {
                const df p = df_split(w * ((c == e ? 1.0 : 0.0) - k[c] * k[e] / k2));
                o.re = df_add(o.re, df_mul(v[e].re, p));
                o.im = df_add(o.im, df_mul(v[e].im, p));
            }
            S[(size_t)c * d.Gh + t] = store_c(o);
        }
    }
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

namespace {

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// power-of-two factor of a supported size: n itself, or n / 3
int pow2_part(int n) { return n % 3 == 0 ? n / 3 : n; }

// lines (or columns) per block: the largest power of two p with p n <= kDfPoints
int df_lines(int n) {
    int p = 1;
    while (2 * p * n <= kDfPoints) p *= 2;
    return p;
}

}  // namespace

bool df_fft_supported(const MeshGeom& g) {
    for (int d = 0; d < 3; ++d) {
        const int n = g.N[d], m = pow2_part(n);
        if (!pow2(m) || n < 16 || n > kDfPoints || (m != n && m < 8)) return false;   // 2^k or 3 2^k
    }
    // the x pass takes 2 df_lines(N_x) whole real lines per block
    return (long long)g.N[1] * g.N[2] % (2 * df_lines(g.N[0])) == 0;
}

// Twiddles exp(-2 pi i k / N_d), k < N_d, per axis (double -> hi + lo floats).
void df_fft_init(const MeshGeom& g, DevBuf tw[3], cudaStream_t s) {
    for (int d = 0; d < 3; ++d) {
        const int n = g.N[d];
        std::vector<float4> h(n);
        for (int k = 0; k < n; ++k) {
            const double th = 2.0 * 3.14159265358979323846264338327950288 * k / n;
            const double c = std::cos(th), sn = -std::sin(th);
            const float ch = (float)c, sh = (float)sn;
            h[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(sn - (double)sh));
        }
        tw[d].ensure(sizeof(float4) * h.size());
        IBP_CUDA(cudaMemcpyAsync(tw[d].p, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice, s));
    }
    IBP_CUDA(cudaStreamSynchronize(s));   // the host table goes out of scope
}

// grid (FP64, [ch][G]) -> out ([ch][G], hi + lo floats): the inverse transform of G(k)
// times the grid's transform.
void df_fft_convolve(const MeshGeom& g, int ch, const float2* green, const double* grid, float2* out, float4* S,
                     DevBuf tw[3], cudaStream_t s, int ncls, const float2* jtab, const RpyScale* rpy) {
    DfGeom d;
    for (int a = 0; a < 3; ++a) {
        d.n[a] = g.N[a];
        d.logn[a] = ilog2(pow2_part(g.N[a]));
        d.pl[a] = df_lines(g.N[a]);
    }
    d.h = g.N[0] / 2 + 1;
    d.G = g.G;
    d.Gh = (long long)g.N[1] * g.N[2] * d.h;
    const int pl = d.pl[0];
    const dim3 gx((unsigned)((long long)g.N[1] * g.N[2] / (2 * pl)), ch);
    const int cy = d.pl[1], cz = d.pl[2];
    const dim3 gy((unsigned)(g.N[2] * ((d.h + cy - 1) / cy)), ch);
    const dim3 gz((unsigned)(g.N[1] * ((d.h + cz - 1) / cz)), ch);
    {
        ProfScope ps(ST_FFT_FWD64, s);
        dfx_forward_kernel<<<gx, kDfThreads, 0, s>>>(d, grid, S, tw[0].as<float4>());
        IBP_CHECK_LAUNCH();
        dfy_kernel<<<gy, kDfThreads, 0, s>>>(d, S, tw[1].as<float4>(), 0);
        IBP_CHECK_LAUNCH();
    }
    {
        ProfScope ps(ST_SCALE64, s);
        if (rpy) {
            if (ch != 3) fail(IBPME_ERR_ARG, "internal: the RPY scaling takes three channels, not %d", ch);
            dfz_scale_kernel<<<gz, kDfThreads, 0, s>>>(d, S, tw[2].as<float4>(), green, 1);
            IBP_CHECK_LAUNCH();
            const long long blocks = std::min<long long>((d.Gh + 255) / 256, 152LL * 16);
            dfz_rpy_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, *rpy, S, green);
            IBP_CHECK_LAUNCH();
            dfz_scale_kernel<<<gz, kDfThreads, 0, s>>>(d, S, tw[2].as<float4>(), green, 2);
        } else if (ncls > 1) {
            if (ch % ncls) fail(IBPME_ERR_ARG, "internal: %d channels for %d radius classes", ch, ncls);
            dfz_scale_kernel<<<gz, kDfThreads, 0, s>>>(d, S, tw[2].as<float4>(), green, 1);
            IBP_CHECK_LAUNCH();
            const long long blocks = std::min<long long>((d.Gh + 255) / 256, 152LL * 16);
            dfz_mix_kernel<<<(unsigned)blocks, 256, 0, s>>>(d.Gh, ch / ncls, ncls, S, green, jtab);
            IBP_CHECK_LAUNCH();
            dfz_scale_kernel<<<gz, kDfThreads, 0, s>>>(d, S, tw[2].as<float4>(), green, 2);
        } else {
            dfz_scale_kernel<<<gz, kDfThreads, 0, s>>>(d, S, tw[2].as<float4>(), green, 0);
        }
        IBP_CHECK_LAUNCH();
    }
    ProfScope ps(ST_FFT_INV64, s);
    dfy_kernel<<<gy, kDfThreads, 0, s>>>(d, S, tw[1].as<float4>(), 1);
    IBP_CHECK_LAUNCH();
    dfx_inverse_kernel<<<gx, kDfThreads, 0, s>>>(d, S, out, tw[0].as<float4>());
    IBP_CHECK_LAUNCH();
}

}  // namespace ibp
