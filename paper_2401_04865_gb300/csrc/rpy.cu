// rpy.cu -- the periodic Rotne-Prager-Yamakawa mobility U = M^H F through the
// spectral-Ewald machinery of the electrostatics.
//
// The paper leaves hydrodynamic interactions out and names the RPY tensor as the
// way to add them (Sec. V.A, Eq. velocity).  The RPY tensor of beads of radius a is
// the Oseen tensor averaged over both beads' surfaces; its transform is
//     M_hat(k) = j0^2(ka) (I - k_hat k_hat) / (mu k^2),
// the same j0^2(ka) shape factor as Eq. M00_Fourier, with the k = 0 mode left out.
// Hasimoto's weight H(k) = (1 + k^2/(4 xi^2)) e^{-k^2/(4 xi^2)} splits it:
//   * wave space: the three force components are spread onto three mesh channels,
//     transformed, multiplied by (1 + k^2/(4 xi^2)) G(k) (I - k_hat k_hat) (G the
//     electrostatic Green's table, which holds j0^2(ka) and the window's share of the
//     Gaussian) and gathered back (Mesh::transform_rpy);
//   * real space: M_r = M_RPY - M_w, where M_w is the inverse transform of the wave
//     kernel over all k.  An isotropic kernel f(k)(I - k_hat k_hat) is A(r) I + B(r)
//     r_hat r_hat in real space, with
//       A = 1/(2 pi^2) int f k^2 [j0(kr) - j1(kr)/(kr)] dk,
//       B = 1/(2 pi^2) int f k^2 [3 j1(kr)/(kr) - j0(kr)] dk;
//     the integrand of M_w falls like e^{-k^2/(4 xi^2)}, so panels of Gauss-Legendre
//     nodes on [0, 14 xi] give it to rounding.  M_r decays like e^{-xi^2 r^2} and needs
//     no k = 0 correction ((1 - H)/k^2 vanishes at k = 0).  A and B are tabulated once
//     per (a, xi, r_c) on nodes spaced 2a/m (a node at r = 2a, where the RPY form
//     changes) and interpolated with cubic Catmull-Rom weights; every pair of the
//     electrostatic pair table within r_c adds A F_beta + B r_hat (r_hat . F_beta).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ibp {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kRpyTableNodes = 4096;   // table nodes across [0, r_c] (about)
constexpr int kRpyPanels = 160;        // Gauss-Legendre panels of the wave integral
constexpr int kRpyOrder = 32;          // nodes per panel

// Gauss-Legendre nodes and weights of the given order on [-1, 1]: Newton's method on
// P_n from the Chebyshev guesses, P_n and P_n' by the three-term recurrence.
void gauss_legendre(int order, std::vector<double>& x, std::vector<double>& w) {
    x.resize(order);
    w.resize(order);
    for (int i = 0; i < order; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (order + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= order; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = order * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= order; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = order * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

__device__ __forceinline__ double j1_over_x(double x) {
    if (fabs(x) < 1e-2) {
        const double x2 = x * x;
        return 1.0 / 3.0 - x2 / 30.0 + x2 * x2 / 840.0;
    }
    double sn, cs;
    sincos(x, &sn, &cs);
    return (sn - x * cs) / (x * x * x);
}

// Free-space RPY tensor A I + B r_hat r_hat at mu = 1: Rotne-Prager for r >= 2a,
// Yamakawa's overlapping form below (the shell-averaged Oseen tensor in both).
__device__ __forceinline__ void rpy_free(double r, double a, double& A, double& B) {
    if (r >= 2.0 * a) {
        A = (1.0 + 2.0 * a * a / (3.0 * r * r)) / (8.0 * kPi * r);
        B = (1.0 - 2.0 * a * a / (r * r)) / (8.0 * kPi * r);
    } else {
        A = (1.0 - 9.0 * r / (32.0 * a)) / (6.0 * kPi * a);
        B = (3.0 * r / (32.0 * a)) / (6.0 * kPi * a);
    }
}

// Node i of the table (r = i h): A_r = A_RPY - A_w, B_r likewise, the wave integrals over
// the nk quadrature points (k_j, W_j), W_j holding the weight times j0^2(k a) H(k).
__global__ void rpy_table_kernel(int nodes, double h, double a, const double* __restrict__ kq,
                                 const double* __restrict__ wq, int nk, double2* __restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    const double r = i * h;
    double sa = 0.0, sb = 0.0;
    for (int j = 0; j < nk; ++j) {
        const double x = kq[j] * r;
        const double j0 = x == 0.0 ? 1.0 : sin(x) / x;
        const double jx = j1_over_x(x);
        sa += wq[j] * (j0 - jx);
        sb += wq[j] * (3.0 * jx - j0);
    }
    double A, B;
    rpy_free(r, a, A, B);
    const double c = 1.0 / (2.0 * kPi * kPi);
    tab[i] = make_double2(A - c * sa, B - c * sb);
}

// F [n][3] -> three channels [3][n]
__global__ void rpy_pack_kernel(int n, const double* __restrict__ F, double* __restrict__ Fc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 3LL * n) return;
    const int i = (int)(t / 3), d = (int)(t % 3);
    Fc[(size_t)d * n + i] = F[t];
}

struct RpyTab {
    const double2* tab;
    int nodes;
    double inv_h;
};

// A, B at distance r (< r_c) by cubic Catmull-Rom weights on the uniform nodes; below
// the second node the missing node is the linear extrapolation of the first two.
__device__ __forceinline__ double2 rpy_interp(const RpyTab& T, double r) {
    const double u = r * T.inv_h;
    int i = (int)u;
    i = i > T.nodes - 3 ? T.nodes - 3 : i;
    const double t = u - i;
    const double2 p1 = T.tab[i], p2 = T.tab[i + 1], p3 = T.tab[i + 2];
    const double2 p0 = i > 0 ? T.tab[i - 1] : make_double2(2.0 * p1.x - p2.x, 2.0 * p1.y - p2.y);
    const double t2 = t * t, t3 = t2 * t;
    const double w0 = -0.5 * t3 + t2 - 0.5 * t, w1 = 1.5 * t3 - 2.5 * t2 + 1.0;
    const double w2 = -1.5 * t3 + 2.0 * t2 + 0.5 * t, w3 = 0.5 * t3 - 0.5 * t2;
    return make_double2(w0 * p0.x + w1 * p1.x + w2 * p2.x + w3 * p3.x, w0 * p0.y + w1 * p1.y + w2 * p2.y + w3 * p3.y);
}

// Real space: one warp per row of the pair table (cell-sorted order); U[alpha] =
// (self F_alpha + sum_pairs A F_beta + B r_hat (r_hat . F_beta)) / mu.
__global__ void rpy_near_kernel(int n, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ order, const double* __restrict__ xw, double L0, double L1,
                                double L2, RpyTab T, double self, double inv_mu, const double* __restrict__ F,
                                double* __restrict__ U) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int al = order[t];
    const double x0 = xw[3 * al], y0 = xw[3 * al + 1], z0 = xw[3 * al + 2];
    double u[3] = {0.0, 0.0, 0.0};
    for (long long p = rowptr[t] + lane; p < rowptr[t + 1]; p += 32) {
        const int be = order[col[p]];
        const double d[3] = {min_image_wrapped(x0 - xw[3 * be], L0), min_image_wrapped(y0 - xw[3 * be + 1], L1),
                             min_image_wrapped(z0 - xw[3 * be + 2], L2)};
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double2 ab = rpy_interp(T, r);
        const double f[3] = {F[3 * be], F[3 * be + 1], F[3 * be + 2]};
        const double ef = r > 0.0 ? (d[0] * f[0] + d[1] * f[1] + d[2] * f[2]) / (r * r) : 0.0;
        for (int c = 0; c < 3; ++c) u[c] += ab.x * f[c] + ab.y * ef * d[c];
    }
    for (int c = 0; c < 3; ++c) u[c] = warp_sum(u[c]);
    if (lane == 0)
        for (int c = 0; c < 3; ++c) U[3 * al + c] = (u[c] + self * F[3 * al + c]) * inv_mu;
}

// The same in FP32 for a mixed-precision context (its mesh is FP32 too): FP32 positions
// of the pair search, a float copy of the table and the forces, FP32 sums per lane and
// FP64 across the warp.  GB300's FP64 rate made the FP64 pass the cost of the product.
struct RpyTab32 {
    const float2* tab;
    int nodes;
    float inv_h;
};

__device__ __forceinline__ float2 rpy_interp32(const RpyTab32& T, float r) {
    const float u = r * T.inv_h;
    int i = (int)u;
    i = i > T.nodes - 3 ? T.nodes - 3 : i;
    const float t = u - (float)i;
    const float2 p1 = T.tab[i], p2 = T.tab[i + 1], p3 = T.tab[i + 2];
    const float2 p0 = i > 0 ? T.tab[i - 1] : make_float2(2.0f * p1.x - p2.x, 2.0f * p1.y - p2.y);
    const float t2 = t * t, t3 = t2 * t;
    const float w0 = -0.5f * t3 + t2 - 0.5f * t, w1 = 1.5f * t3 - 2.5f * t2 + 1.0f;
    const float w2 = -1.5f * t3 + 2.0f * t2 + 0.5f * t, w3 = 0.5f * t3 - 0.5f * t2;
    return make_float2(w0 * p0.x + w1 * p1.x + w2 * p2.x + w3 * p3.x, w0 * p0.y + w1 * p1.y + w2 * p2.y + w3 * p3.y);
}

__global__ void rpy_near32_kernel(int n, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                  const int* __restrict__ order, const float4* __restrict__ xf, float L0, float L1,
                                  float L2, RpyTab32 T, double self, double inv_mu, const float4* __restrict__ F4,
                                  const double* __restrict__ F, double* __restrict__ U) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n) return;
    const int al = order[t];
    const float4 pa = xf[al];
    float u[3] = {0.0f, 0.0f, 0.0f};
    for (long long p = rowptr[t] + lane; p < rowptr[t + 1]; p += 32) {
        const int be = order[col[p]];
        const float4 pb = xf[be];
        const float d[3] = {min_image_wrapped(pa.x - pb.x, L0), min_image_wrapped(pa.y - pb.y, L1),
                            min_image_wrapped(pa.z - pb.z, L2)};
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const float r = sqrtf(r2);
        const float2 ab = rpy_interp32(T, r);
        const float4 f = F4[be];
        const float ef = r2 > 0.0f ? (d[0] * f.x + d[1] * f.y + d[2] * f.z) / r2 : 0.0f;
        u[0] += ab.x * f.x + ab.y * ef * d[0];
        u[1] += ab.x * f.y + ab.y * ef * d[1];
        u[2] += ab.x * f.z + ab.y * ef * d[2];
    }
    double v[3];
    for (int c = 0; c < 3; ++c) v[c] = warp_sum((double)u[c]);
    if (lane == 0)
        for (int c = 0; c < 3; ++c) U[3 * al + c] = (v[c] + self * F[3 * al + c]) * inv_mu;
}

// forces as float4 (x, y, z, 0) and the table as float2, for the FP32 pass
__global__ void rpy_f4_kernel(int n, const double* __restrict__ F, float4* __restrict__ F4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) F4[i] = make_float4((float)F[3 * i], (float)F[3 * i + 1], (float)F[3 * i + 2], 0.0f);
}

__global__ void rpy_tab32_kernel(int nodes, const double2* __restrict__ tab, float2* __restrict__ t32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nodes) t32[i] = make_float2((float)tab[i].x, (float)tab[i].y);
}

// U[i][d] += Uk[d][i]
__global__ void rpy_combine_kernel(int n, const double* __restrict__ Uk, double* __restrict__ U) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 3LL * n) return;
    const int i = (int)(t / 3), d = (int)(t % 3);
    U[t] += Uk[(size_t)d * n + i];
}

// The radial table of the context's (a, xi, r_c), built on first use.
void rpy_table(ibpme_ctx* c) {
    if (c->rpy_nodes > 0 && c->rpy_key[0] == c->a && c->rpy_key[1] == c->xi && c->rpy_key[2] == c->rc) return;
    const double a = c->a, xi = c->xi, rc = c->rc;
    const int m = std::max(1, (int)std::ceil(2.0 * a * kRpyTableNodes / rc));   // nodes per 2a
    const double h = 2.0 * a / m;
    const int nodes = (int)std::floor(rc / h) + 4;
    std::vector<double> gx, gw;
    gauss_legendre(kRpyOrder, gx, gw);
    const double kmax = 14.0 * xi, pw = kmax / kRpyPanels;
    std::vector<double> kq, wq;
    for (int p = 0; p < kRpyPanels; ++p)
        for (int j = 0; j < kRpyOrder; ++j) {
            const double k = p * pw + 0.5 * pw * (gx[j] + 1.0);
            const double j0 = std::sin(k * a) / (k * a);
            const double q = k * k / (4.0 * xi * xi);
            kq.push_back(k);
            wq.push_back(0.5 * pw * gw[j] * j0 * j0 * (1.0 + q) * std::exp(-q));
        }
    const int nk = (int)kq.size();
    DevBuf dk, dw;
    dk.ensure(sizeof(double) * nk);
    dw.ensure(sizeof(double) * nk);
    IBP_CUDA(cudaMemcpyAsync(dk.p, kq.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream));
    IBP_CUDA(cudaMemcpyAsync(dw.p, wq.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream));
    double2* tab = static_cast<double2*>(c->rpy_tab.ensure(sizeof(double2) * (size_t)nodes));
    rpy_table_kernel<<<div_up(nodes, 128), 128, 0, c->stream>>>(nodes, h, a, dk.as<double>(), dw.as<double>(), nk,
                                                                tab);
    IBP_CHECK_LAUNCH();
    double2 self{};
    IBP_CUDA(cudaMemcpyAsync(&self, tab, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    IBP_CUDA(cudaStreamSynchronize(c->stream));   // the host vectors and the quadrature buffers go out of scope
    float2* t32 = static_cast<float2*>(c->rpy_tab32.ensure(sizeof(float2) * (size_t)nodes));
    rpy_tab32_kernel<<<div_up(nodes, 128), 128, 0, c->stream>>>(nodes, tab, t32);
    IBP_CHECK_LAUNCH();
    IBP_CUDA(cudaStreamSynchronize(c->stream));
    c->rpy_self = self.x;
    c->rpy_h = h;
    c->rpy_nodes = nodes;
    c->rpy_key[0] = a;
    c->rpy_key[1] = xi;
    c->rpy_key[2] = rc;
}

// ---- rigid-body mobility problem (the paper's last equation, physical sign) ----
// Unknowns z = [f (n x 3 bead constraint forces); W (n_b x 6 body motions U, Omega)], operator
//     [ M f - K W ;  K^T f ]   with (K W)_j = U_b + Omega_b x r_j,  K^T f = (sum f, sum r x f),
// right-hand side [0; (F, L)].  A single-bead body moves by U alone: its Omega rows hold Omega
// itself (right-hand side 0), so the system stays regular.

// y_f -= K W
__global__ void rigid_kw_kernel(int n, const int* __restrict__ bead_body, const int* __restrict__ off,
                                const double* __restrict__ rel, const double* __restrict__ W,
                                double* __restrict__ y) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int b = bead_body[j];
    const double* w = W + 6 * (size_t)b;
    double u[3] = {w[0], w[1], w[2]};
    if (off[b + 1] - off[b] > 1) {
        const double r[3] = {rel[3 * j], rel[3 * j + 1], rel[3 * j + 2]};
        u[0] += w[4] * r[2] - w[5] * r[1];
        u[1] += w[5] * r[0] - w[3] * r[2];
        u[2] += w[3] * r[1] - w[4] * r[0];
    }
    for (int d = 0; d < 3; ++d) y[3 * j + d] -= u[d];
}

// y_W = (F, L) of the bead forces per body; Omega for single-bead bodies
__global__ void rigid_body_rows_kernel(int nb, const int* __restrict__ off, const double* __restrict__ F,
                                       const double* __restrict__ L, const double* __restrict__ W,
                                       double* __restrict__ yW) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const bool multi = off[b + 1] - off[b] > 1;
    for (int d = 0; d < 3; ++d) {
        yW[6 * b + d] = F[3 * b + d];
        yW[6 * b + 3 + d] = multi ? L[3 * b + d] : W[6 * b + 3 + d];
    }
}

// b = [0; (F, L)] with the torque rows of single-bead bodies zero
__global__ void rigid_rhs_kernel(int n, int nb, const int* __restrict__ off, const double* __restrict__ FL,
                                 double* __restrict__ b) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < 3LL * n) {
        b[t] = 0.0;
        return;
    }
    const long long k = t - 3LL * n;
    if (k >= 6LL * nb) return;
    const int body = (int)(k / 6), c = (int)(k % 6);
    b[t] = (c < 3 || off[body + 1] - off[body] > 1) ? FL[k] : 0.0;
}

// out[v] += sum_i V[v][i] w[i] for v < nv (out zeroed by the caller); blockIdx.y = v
__global__ void multi_dot_kernel(long long N, const double* __restrict__ V, long long ldv,
                                 const double* __restrict__ w, double* __restrict__ out) {
    __shared__ double sh[32];
    const double* v = V + (size_t)blockIdx.y * ldv;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        acc += v[i] * w[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out + blockIdx.y, t);
    }
}

// w[i] += s sum_v coef[v] V[v][i]
__global__ void multi_axpy_kernel(long long N, const double* __restrict__ V, long long ldv, int nv,
                                  const double* __restrict__ coef, double s, double* __restrict__ w) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int v = 0; v < nv; ++v) acc += coef[v] * V[(size_t)v * ldv + i];
        w[i] += s * acc;
    }
}

// dst = s src
__global__ void scale_copy_kernel(long long N, double s, const double* __restrict__ src, double* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        dst[i] = s * src[i];
}

}  // namespace

void rpy_apply(ibpme_ctx* c, int n, const double* xw, const double* F, double mu, double* U) {
    if (c->ncls > 1) fail(IBPME_ERR_UNEQUAL_RADII, "the RPY mobility takes one bead radius");
    if (n == 0) return;
    cudaStream_t s = c->stream;
    rpy_table(c);
    c->grid64_final = false;   // the meshes are about to hold the force channels
    c->field64_ready = false;
    c->near_field_ready = false;
    near_build(c, n, xw, false);
    const StencilCache* sc = stencil_cache(c, n, xw);
    double* Fc = static_cast<double*>(c->rpy_F.ensure(sizeof(double) * 3 * (size_t)n));
    double* Uk = static_cast<double*>(c->rpy_Uk.ensure(sizeof(double) * 3 * (size_t)n));
    rpy_pack_kernel<<<div_up(3LL * n, 256), 256, 0, s>>>(n, F, Fc);
    IBP_CHECK_LAUNCH();
    const double fac = c->eps / mu;   // the gather carries 1/eps_f
    if (c->p.precision == IBPME_MIXED) {
        c->mesh32.spread(n, xw, Fc, 3, nullptr, 1, s, sc);
        c->mesh32.transform_rpy(fac, c->xi, s);
        c->mesh32.gather(n, xw, 3, nullptr, Uk, nullptr, s, sc);
    } else {
        c->mesh64.spread(n, xw, Fc, 3, nullptr, 1, s, sc);
        c->mesh64.transform_rpy(fac, c->xi, s);
        c->mesh64.gather(n, xw, 3, nullptr, Uk, nullptr, s, sc);
    }
    const NearList& nl = c->near;
    RpyTab T{c->rpy_tab.as<double2>(), c->rpy_nodes, 1.0 / c->rpy_h};
    ProfScope ps(ST_RPY_NEAR, s);
    if (c->p.precision == IBPME_MIXED) {
        float4* F4 = static_cast<float4*>(c->rpy_F4.ensure(sizeof(float4) * (size_t)n));
        rpy_f4_kernel<<<div_up(n, 256), 256, 0, s>>>(n, F, F4);
        IBP_CHECK_LAUNCH();
        RpyTab32 T32{c->rpy_tab32.as<float2>(), c->rpy_nodes, (float)(1.0 / c->rpy_h)};
        rpy_near32_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(
            n, nl.rowptr.as<long long>(), nl.col.as<int>(), nl.cell_beads.as<int>(), nl.xf.as<float4>(),
            (float)c->p.box[0], (float)c->p.box[1], (float)c->p.box[2], T32, c->rpy_self, 1.0 / mu, F4, F, U);
    } else {
        rpy_near_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(
            n, nl.rowptr.as<long long>(), nl.col.as<int>(), nl.cell_beads.as<int>(), xw, c->p.box[0], c->p.box[1],
            c->p.box[2], T, c->rpy_self, 1.0 / mu, F, U);
    }
    IBP_CHECK_LAUNCH();
    rpy_combine_kernel<<<div_up(3LL * n, 256), 256, 0, s>>>(n, Uk, U);
    IBP_CHECK_LAUNCH();
}

namespace {

// ---- body-block preconditioner of the rigid-body mobility problem ----
// For every multi-bead body the exact inverse of its own block with the free-space RPY
// tensor of its beads M_b (3 n_b x 3 n_b, FP32 inverse): [M_b -K_b; K_b^T 0]^{-1} [v; g] is
//     t = M_b^{-1} v,  W = S^{-1} (g - K_b^T t),  f = t + G W,   G = M_b^{-1} K_b, S = K_b^T G;
// for a single bead (self mobility m = 1/(6 pi mu a)) f = g_F, U = m g_F - v, Omega = g_Omega.
// GMRES then iterates on A P^{-1}, whose remaining coupling is between bodies.

// M_b of one body: entry (3i+p, 3j+q) = (A delta_pq + B r_p r_q / r^2) / mu (free-space RPY)
__global__ void rigid_block_kernel(int nb, const double* __restrict__ rel, double a, double inv_mu,
                                   float* __restrict__ M) {
    const long long m3 = 3LL * nb;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= m3 * m3) return;
    const int row = (int)(t / m3), col = (int)(t % m3);
    const int i = row / 3, p = row % 3, j = col / 3, q = col % 3;
    const double d[3] = {rel[3 * i] - rel[3 * j], rel[3 * i + 1] - rel[3 * j + 1], rel[3 * i + 2] - rel[3 * j + 2]};
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double A, B;
    rpy_free(r, a, A, B);
    const double v = (p == q ? A : 0.0) + (r > 0.0 ? B * d[p] * d[q] / (r * r) : 0.0);
    M[t] = (float)(v * inv_mu);
}

// G = M_b^{-1} K_b (3 n_b x 6, row-major), one thread per entry
__global__ void rigid_g_kernel(int nb, const float* __restrict__ Minv, const double* __restrict__ rel,
                               double* __restrict__ G) {
    const int m3 = 3 * nb;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m3 * 6) return;
    const int row = t / 6, k = t % 6;
    double acc = 0.0;
    for (int col = 0; col < m3; ++col) {
        const int j = col / 3, q = col % 3;
        double kv;
        if (k < 3) {
            kv = q == k ? 1.0 : 0.0;
        } else {   // (e_{k-3} x r_j)_q
            const double* r = rel + 3 * j;
            const int e = k - 3;
            kv = e == 0 ? (q == 1 ? -r[2] : (q == 2 ? r[1] : 0.0))
               : e == 1 ? (q == 0 ? r[2] : (q == 2 ? -r[0] : 0.0))
                        : (q == 0 ? -r[1] : (q == 1 ? r[0] : 0.0));
        }
        acc += (double)Minv[(size_t)row * m3 + col] * kv;
    }
    G[t] = acc;
}

// t = M_b^{-1} v for every preconditioned body: blockIdx.y = body, one warp per row
__global__ void rigid_pre_minv_kernel(const int4* __restrict__ pb, const long long* __restrict__ moff,
                                      const float* __restrict__ Minv, const double* __restrict__ v,
                                      double* __restrict__ tvec) {
    const int4 P = pb[blockIdx.y];   // (body, first bead, beads, -)
    const int m3 = 3 * P.z;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m3) return;
    const float* Mr = Minv + moff[blockIdx.y] + (size_t)row * m3;
    const double* vb = v + 3 * (size_t)P.y;
    double acc = 0.0;
    for (int col = lane; col < m3; col += 32) acc += (double)Mr[col] * vb[col];
    acc = warp_sum(acc);
    if (lane == 0) tvec[3 * (size_t)P.y + row] = acc;
}

// W_b = S^{-1} (g_b - K_b^T t) per preconditioned body (one block each)
__global__ void rigid_pre_body_kernel(const int4* __restrict__ pb, const double* __restrict__ rel,
                                      const double* __restrict__ Sinv, const double* __restrict__ tvec,
                                      const double* __restrict__ gW, double* __restrict__ outW) {
    __shared__ double sh[6][32];
    const int4 P = pb[blockIdx.x];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int j = P.y + threadIdx.x; j < P.y + P.z; j += blockDim.x) {
        const double* t = tvec + 3 * (size_t)j;
        const double* r = rel + 3 * (size_t)j;
        acc[0] += t[0];
        acc[1] += t[1];
        acc[2] += t[2];
        acc[3] += r[1] * t[2] - r[2] * t[1];
        acc[4] += r[2] * t[0] - r[0] * t[2];
        acc[5] += r[0] * t[1] - r[1] * t[0];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double h[6];
        for (int k = 0; k < 6; ++k) {
            double v = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += sh[k][q];
            h[k] = gW[6 * (size_t)P.x + k] - v;
        }
        const double* Si = Sinv + 36 * (size_t)blockIdx.x;
        for (int k = 0; k < 6; ++k) {
            double v = 0.0;
            for (int l = 0; l < 6; ++l) v += Si[6 * k + l] * h[l];
            outW[6 * (size_t)P.x + k] = v;
        }
    }
}

// f_j = t_j + G_j W_b for beads of preconditioned bodies; single beads exactly; (body index of
// each bead's preconditioned block in pre_of, -1 for single beads)
__global__ void rigid_pre_bead_kernel(int n, const int* __restrict__ bead_body, const int* __restrict__ off,
                                      const int* __restrict__ pre_first, const long long* __restrict__ goff,
                                      const int* __restrict__ pre_of, const double* __restrict__ G,
                                      const double* __restrict__ tvec, double mself, const double* __restrict__ v,
                                      double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int b = bead_body[j];
    const long long nw = 3LL * n;
    const double* gW = v + nw + 6 * (size_t)b;
    double* oW = out + nw + 6 * (size_t)b;
    if (off[b + 1] - off[b] == 1) {
        for (int d = 0; d < 3; ++d) {
            out[3 * (size_t)j + d] = gW[d];
            oW[d] = mself * gW[d] - v[3 * (size_t)j + d];
            oW[3 + d] = gW[3 + d];
        }
        return;
    }
    const int q = pre_of[b];
    const double* W = out + nw + 6 * (size_t)b;
    const double* Gj = G + goff[q] + 18 * (size_t)(j - pre_first[q]);
    for (int d = 0; d < 3; ++d) {
        double acc = tvec[3 * (size_t)j + d];
        for (int k = 0; k < 6; ++k) acc += Gj[6 * d + k] * W[k];
        out[3 * (size_t)j + d] = acc;
    }
}

// y = A z for the rigid-body mobility operator (bodies uploaded, positions xw)
void rigid_apply(ibpme_ctx* c, int n, const double* xw, double mu, const double* z, double* y) {
    const BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    const int nb = bd.nb;
    rpy_apply(c, n, xw, z, mu, y);
    rigid_kw_kernel<<<div_up(n, 256), 256, 0, s>>>(n, bd.bead_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(),
                                                    z + 3 * (size_t)n, y);
    IBP_CHECK_LAUNCH();
    double* FL = static_cast<double*>(c->rig_FL.ensure(sizeof(double) * 6 * (size_t)nb));
    body_reduce_force_torque(c, n, z, FL, FL + 3 * (size_t)nb);
    rigid_body_rows_kernel<<<div_up(nb, 256), 256, 0, s>>>(nb, bd.off.as<int>(), FL, FL + 3 * (size_t)nb,
                                                           z + 3 * (size_t)n, y + 3 * (size_t)n);
    IBP_CHECK_LAUNCH();
}

int vec_blocks(long long N) { return (int)std::min<long long>(div_up(N, 256), 152LL * 8); }

// The blocks of every multi-bead body at the current positions; false when a body is too
// large for the dense inverse (the solve then runs unpreconditioned).
bool rigid_precond_build(ibpme_ctx* c, int n, double mu) {
    const BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    const std::vector<int>& off = bd.host_off;
    const int nb = bd.nb;
    std::vector<int4> pb;
    std::vector<long long> moff, goff;
    std::vector<int> pre_of(nb, -1), pre_first;
    long long mtot = 0, gtot = 0;
    int maxn = 0;
    for (int b = 0; b < nb; ++b) {
        const int k = off[b + 1] - off[b];
        if (k < 2) continue;
        if (3 * k > kPrecondMaxBeads) return false;
        pre_of[b] = (int)pb.size();
        pb.push_back(make_int4(b, off[b], k, 0));
        pre_first.push_back(off[b]);
        moff.push_back(mtot);
        goff.push_back(gtot);
        mtot += 9LL * k * k;
        gtot += 18LL * k;
        maxn = std::max(maxn, k);
    }
    const int nmb = (int)pb.size();
    c->rig_nmb = nmb;
    c->rig_maxn = maxn;
    if (nmb == 0) return true;
    float* minv = static_cast<float*>(c->rig_minv.ensure(sizeof(float) * (size_t)mtot));
    double* G = static_cast<double*>(c->rig_G.ensure(sizeof(double) * (size_t)gtot));
    std::vector<double> rel(3 * (size_t)n);
    IBP_CUDA(cudaMemcpyAsync(rel.data(), bd.rel.p, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
    IBP_CUDA(cudaStreamSynchronize(s));
    std::vector<double> Sinv(36 * (size_t)nmb), Gh;
    for (int q = 0; q < nmb; ++q) {
        const int k = pb[q].z, first = pb[q].y, m3 = 3 * k;
        float* A = minv + moff[q];
        const double* relb = bd.rel.as<double>() + 3 * (size_t)first;
        rigid_block_kernel<<<(unsigned)div_up((long long)m3 * m3, 256), 256, 0, s>>>(k, relb, c->a, 1.0 / mu, A);
        IBP_CHECK_LAUNCH();
        invert_spd(c, m3, A);
        rigid_g_kernel<<<div_up(m3 * 6, 128), 128, 0, s>>>(k, A, relb, G + goff[q]);
        IBP_CHECK_LAUNCH();
        Gh.resize((size_t)m3 * 6);
        IBP_CUDA(cudaMemcpyAsync(Gh.data(), G + goff[q], sizeof(double) * Gh.size(), cudaMemcpyDeviceToHost, s));
        IBP_CUDA(cudaStreamSynchronize(s));
        // S = K^T G (6 x 6), then its inverse by Gauss-Jordan with partial pivoting
        double S[6][12] = {};
        for (int j = 0; j < k; ++j) {
            const double* r = rel.data() + 3 * (size_t)(first + j);
            for (int qq = 0; qq < 3; ++qq) {
                const double* g = Gh.data() + 6 * (size_t)(3 * j + qq);
                // K row (3j+qq): translation e_qq, rotation columns (e_e x r)_qq
                double kr[6] = {0, 0, 0, 0, 0, 0};
                kr[qq] = 1.0;
                kr[3] = qq == 1 ? -r[2] : (qq == 2 ? r[1] : 0.0);
                kr[4] = qq == 0 ? r[2] : (qq == 2 ? -r[0] : 0.0);
                kr[5] = qq == 0 ? -r[1] : (qq == 1 ? r[0] : 0.0);
                for (int a2 = 0; a2 < 6; ++a2)
                    for (int l = 0; l < 6; ++l) S[a2][l] += kr[a2] * g[l];
            }
        }
        for (int a2 = 0; a2 < 6; ++a2) S[a2][6 + a2] = 1.0;
        for (int col = 0; col < 6; ++col) {
            int piv = col;
            for (int r2 = col + 1; r2 < 6; ++r2)
                if (std::fabs(S[r2][col]) > std::fabs(S[piv][col])) piv = r2;
            if (!(std::fabs(S[piv][col]) > 0.0))
                fail(IBPME_ERR_ARG, "body %d: its beads are collinear (no resistance to spin about its axis)",
                     pb[q].x);
            for (int l = 0; l < 12; ++l) std::swap(S[col][l], S[piv][l]);
            const double d = S[col][col];
            for (int l = 0; l < 12; ++l) S[col][l] /= d;
            for (int r2 = 0; r2 < 6; ++r2) {
                if (r2 == col) continue;
                const double f = S[r2][col];
                for (int l = 0; l < 12; ++l) S[r2][l] -= f * S[col][l];
            }
        }
        for (int a2 = 0; a2 < 6; ++a2)
            for (int l = 0; l < 6; ++l) Sinv[36 * (size_t)q + 6 * a2 + l] = S[a2][6 + l];
    }
    auto up = [&](DevBuf& dst, const void* src, size_t bytes) {
        dst.ensure(bytes > 0 ? bytes : 4);
        if (bytes) IBP_CUDA(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyHostToDevice, s));
    };
    up(c->rig_Sinv, Sinv.data(), sizeof(double) * Sinv.size());
    up(c->rig_pb, pb.data(), sizeof(int4) * pb.size());
    up(c->rig_moff, moff.data(), sizeof(long long) * moff.size());
    up(c->rig_goff, goff.data(), sizeof(long long) * goff.size());
    std::vector<int> idx(pre_of);
    idx.insert(idx.end(), pre_first.begin(), pre_first.end());   // [nb] pre_of, then [nmb] first beads
    up(c->rig_idx, idx.data(), sizeof(int) * idx.size());
    IBP_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
    return true;
}

// out = P^{-1} v
void rigid_precond_apply(ibpme_ctx* c, int n, double mu, const double* v, double* out) {
    const BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    double* t = static_cast<double*>(c->rig_t.ensure(sizeof(double) * 3 * (size_t)n));
    const int nmb = c->rig_nmb;
    if (nmb > 0) {
        rigid_pre_minv_kernel<<<dim3(div_up(3 * c->rig_maxn, 8), nmb), 256, 0, s>>>(
            c->rig_pb.as<int4>(), c->rig_moff.as<long long>(), c->rig_minv.as<float>(), v, t);
        IBP_CHECK_LAUNCH();
        rigid_pre_body_kernel<<<nmb, 128, 0, s>>>(c->rig_pb.as<int4>(), bd.rel.as<double>(), c->rig_Sinv.as<double>(),
                                                  t, v + 3 * (size_t)n, out + 3 * (size_t)n);
        IBP_CHECK_LAUNCH();
    }
    const int* idx = c->rig_idx.as<int>();
    rigid_pre_bead_kernel<<<div_up(n, 256), 256, 0, s>>>(
        n, bd.bead_body.as<int>(), bd.off.as<int>(), nmb > 0 ? idx + bd.nb : nullptr, c->rig_goff.as<long long>(),
        idx, c->rig_G.as<double>(), t, 1.0 / (6.0 * kPi * mu * c->a), v, out);
    IBP_CHECK_LAUNCH();
}

}  // namespace

void rigid_solve(ibpme_ctx* c, int n, const double* xw, const double* FL, double mu, double rtol, int m,
                 int max_iter, double* W_out, double* f_out, ibpme_solve_stats* st, bool precond) {
    cudaStream_t s = c->stream;
    const int nb = c->bodies.nb;
    const long long N = 3LL * n + 6LL * nb;
    // right preconditioning: Arnoldi on A P^{-1}, x = P^{-1} (V y)
    const bool pre = precond && rigid_precond_build(c, n, mu);
    double* zb = pre ? static_cast<double*>(c->rig_z.ensure(sizeof(double) * (size_t)N)) : nullptr;
    double* ub = pre ? static_cast<double*>(c->rig_u.ensure(sizeof(double) * (size_t)N)) : nullptr;
    double* V = static_cast<double*>(c->rig_V.ensure(sizeof(double) * (size_t)N * (m + 1)));
    double* w = static_cast<double*>(c->rig_w.ensure(sizeof(double) * (size_t)N));
    double* b = static_cast<double*>(c->rig_b.ensure(sizeof(double) * (size_t)N));
    double* x = static_cast<double*>(c->rig_x.ensure(sizeof(double) * (size_t)N));
    double* dd = static_cast<double*>(c->rig_dot.ensure(sizeof(double) * (size_t)(m + 2)));
    const int vb = vec_blocks(N);
    std::vector<double> hh(m + 2);
    auto dots = [&](const double* Vs, int nv, const double* v) {   // V[0..nv) . v -> hh
        IBP_CUDA(cudaMemsetAsync(dd, 0, sizeof(double) * nv, s));
        multi_dot_kernel<<<dim3(vb, nv), 256, 0, s>>>(N, Vs, N, v, dd);
        IBP_CHECK_LAUNCH();
        IBP_CUDA(cudaMemcpyAsync(hh.data(), dd, sizeof(double) * nv, cudaMemcpyDeviceToHost, s));
        IBP_CUDA(cudaStreamSynchronize(s));
    };
    auto axpy = [&](const double* Vs, int nv, const double* coef_h, double sc, double* v) {   // v += sc V coef
        IBP_CUDA(cudaMemcpyAsync(dd, coef_h, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
        multi_axpy_kernel<<<vb, 256, 0, s>>>(N, Vs, N, nv, dd, sc, v);
        IBP_CHECK_LAUNCH();
        IBP_CUDA(cudaStreamSynchronize(s));   // coef_h is reused
    };
    rigid_rhs_kernel<<<(unsigned)div_up(N, 256), 256, 0, s>>>(n, nb, c->bodies.off.as<int>(), FL, b);
    IBP_CHECK_LAUNCH();
    IBP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)N, s));
    dots(b, 1, b);
    const double bnorm = std::sqrt(hh[0]);
    int iters = 0, outer = 0;
    double rel = 0.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (true) {
        // r = b - A x into V_0
        if (iters == 0) {
            IBP_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, s));
        } else {
            rigid_apply(c, n, xw, mu, x, w);
            scale_copy_kernel<<<vb, 256, 0, s>>>(N, 1.0, b, V);
            IBP_CHECK_LAUNCH();
            const double one = 1.0;
            axpy(w, 1, &one, -1.0, V);
        }
        dots(V, 1, V);
        const double beta = std::sqrt(hh[0]);
        rel = bnorm > 0.0 ? beta / bnorm : 0.0;
        if (bnorm == 0.0 || rel <= rtol || iters >= max_iter) break;
        ++outer;
        scale_copy_kernel<<<vb, 256, 0, s>>>(N, 1.0 / beta, V, V);
        IBP_CHECK_LAUNCH();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && iters < max_iter; ++j) {
            double* vj1 = V + (size_t)(j + 1) * N;
            if (pre) {
                rigid_precond_apply(c, n, mu, V + (size_t)j * N, zb);
                rigid_apply(c, n, xw, mu, zb, vj1);
            } else {
                rigid_apply(c, n, xw, mu, V + (size_t)j * N, vj1);
            }
            std::vector<double> h(j + 2, 0.0);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                dots(V, j + 1, vj1);
                for (int i = 0; i <= j; ++i) h[i] += hh[i];
                axpy(V, j + 1, hh.data(), -1.0, vj1);
            }
            dots(vj1, 1, vj1);
            h[j + 1] = std::sqrt(hh[0]);
            if (h[j + 1] > 0.0) {
                scale_copy_kernel<<<vb, 256, 0, s>>>(N, 1.0 / h[j + 1], vj1, vj1);
                IBP_CHECK_LAUNCH();
            }
            for (int i = 0; i < j; ++i) {   // earlier rotations
                const double t = cs[i] * h[i] + sn[i] * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t;
            }
            const double den = std::hypot(h[j], h[j + 1]);
            cs[j] = den > 0.0 ? h[j] / den : 1.0;
            sn[j] = den > 0.0 ? h[j + 1] / den : 0.0;
            h[j] = den;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
            ++iters;
            k = j + 1;
            if (std::fabs(g[j + 1]) <= rtol * bnorm || h[j + 1] == 0.0) break;
        }
        for (int i = k - 1; i >= 0; --i) {   // H y = g, upper triangular
            double t = g[i];
            for (int l = i + 1; l < k; ++l) t -= H[(size_t)i * m + l] * y[l];
            y[i] = t / H[(size_t)i * m + i];
        }
        if (pre) {
            IBP_CUDA(cudaMemsetAsync(ub, 0, sizeof(double) * (size_t)N, s));
            axpy(V, k, y.data(), 1.0, ub);
            rigid_precond_apply(c, n, mu, ub, zb);
            const double one = 1.0;
            axpy(zb, 1, &one, 1.0, x);
        } else {
            axpy(V, k, y.data(), 1.0, x);
        }
    }
    IBP_CUDA(cudaMemcpyAsync(W_out, x + 3 * (size_t)n, sizeof(double) * 6 * (size_t)nb, cudaMemcpyDeviceToDevice, s));
    if (f_out)
        IBP_CUDA(cudaMemcpyAsync(f_out, x, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    if (st) {
        st->iters = iters;
        st->outer = outer;
        st->rel_residual = rel;
    }
    if (!(rel <= rtol)) fail(IBPME_ERR_NOT_CONVERGED, "rigid mobility: relative residual %.3g after %d iterations",
                             rel, iters);
}

}  // namespace ibp
