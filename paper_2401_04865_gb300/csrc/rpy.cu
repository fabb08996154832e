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

}  // namespace ibp
