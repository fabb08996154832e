// api.cu -- the C ABI: context set-up (automatic parameters of Sec. III.D.2),
// staging of host arrays, and the entry points declared in include/ibpme.h.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace ibp {

namespace {
thread_local char g_err[1024] = "";
constexpr double kPi = 3.14159265358979323846264338327950288;
}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void fail(ibpme_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    throw Error(s);
}

namespace {

template <typename F>
ibpme_status guard(F&& f) {
    try {
        g_err[0] = '\0';
        return f();
    } catch (const Error& e) {
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return IBPME_ERR_OOM;
    } catch (...) {
        set_error("unexpected internal exception");
        return IBPME_ERR_CUDA;
    }
}

// Keeps the context's device current for the duration of a call.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        IBP_CUDA(cudaGetDevice(&prev));
        if (prev != dev) IBP_CUDA(cudaSetDevice(dev));
    }
    ~DeviceScope() {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown pointer
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Input array: device pointers pass through, host arrays are copied into the stage.
const void* stage_in(ibpme_ctx* c, const void* p, size_t bytes, DevBuf& st) {
    if (!p || bytes == 0 || is_device_ptr(p)) return p;
    void* d = st.ensure(bytes);
    IBP_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, c->stream));
    return d;
}

// Output array: returns a device pointer to write to; host arrays get a stage
// that finish_out() copies back.
struct OutArg {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool host = false;
};

OutArg stage_out(ibpme_ctx* c, void* p, size_t bytes, DevBuf& st, bool read_first = false) {
    OutArg o;
    o.user = p;
    o.bytes = bytes;
    if (!p || bytes == 0) return o;
    if (is_device_ptr(p)) {
        o.dev = p;
        return o;
    }
    o.host = true;
    o.dev = st.ensure(bytes);
    if (read_first) IBP_CUDA(cudaMemcpyAsync(o.dev, p, bytes, cudaMemcpyHostToDevice, c->stream));
    return o;
}

void finish_out(ibpme_ctx* c, const OutArg& o) {
    if (o.host && o.bytes) IBP_CUDA(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, c->stream));
}

__global__ void wrap_kernel(int n, const double* __restrict__ x, double L0, double L1, double L2,
                            double* __restrict__ xw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int d = i % 3;
    const double L = d == 0 ? L0 : (d == 1 ? L1 : L2);
    xw[i] = wrap_coord(x[i], L);
}

__global__ void add_kernel(long long m, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < m) out[i] = a[i] + b[i];
}

// qsum[cfg * nrhs + r] += sum of the charges of right-hand side r in configuration cfg
__global__ void qsum_kernel(int n, int nrhs, const double* __restrict__ q, const int* __restrict__ bcfg,
                            double* __restrict__ qsum) {
    const int r = blockIdx.y;
    if (!bcfg) {
        double acc = 0.0;
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x)
            acc += q[(size_t)r * n + t];
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) atomicAdd(qsum + r, acc);
        return;
    }
    // configurations are contiguous bead ranges: a warp whose beads share one
    // configuration adds once, a warp on a boundary adds per bead
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w0 < n; w0 += stride) {
        const long long t = w0 + lane;
        const bool ok = t < n;
        const int cf = ok ? bcfg[t] : -1;
        double v = ok ? q[(size_t)r * n + t] : 0.0;
        const int c0 = __shfl_sync(0xffffffffu, cf, 0);
        if (__all_sync(0xffffffffu, !ok || cf == c0)) {
            v = warp_sum(v);
            if (lane == 0) atomicAdd(qsum + (size_t)c0 * nrhs + r, v);
        } else if (ok) {
            atomicAdd(qsum + (size_t)cf * nrhs + r, v);
        }
    }
}

// psi = psi_real + psi_wave - k0 * sum(q): the real-space image sum carries the
// k = 0 Fourier mode 1/(4 xi^2 V eps) that M (Sec. II) excludes (per configuration).
__global__ void combine_kernel(long long m, int n, int nrhs, const double* __restrict__ a,
                               const double* __restrict__ b, const double* __restrict__ qsum,
                               const int* __restrict__ bcfg, double k0, double* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int r = (int)(i / n);
    const int cfg = bcfg ? bcfg[i - (long long)r * n] : 0;
    out[i] = a[i] + b[i] - k0 * qsum[(size_t)cfg * nrhs + r];
}

bool good_fft_size(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

}  // namespace

void resolve_params(const ibpme_params* in, ibpme_params* p) {
    *p = *in;
    for (int d = 0; d < 3; ++d)
        if (!(p->box[d] > 0.0) || !std::isfinite(p->box[d])) fail(IBPME_ERR_ARG, "box[%d] must be > 0", d);
    if (p->n_radius_classes < 0 || p->n_radius_classes > IBPME_MAX_RADIUS_CLASSES)
        fail(IBPME_ERR_ARG, "n_radius_classes must be in 0..%d", IBPME_MAX_RADIUS_CLASSES);
    if (p->n_radius_classes >= 2) {   // the largest class radius stands for a in the rules below
        double amax = 0.0;
        for (int k = 0; k < p->n_radius_classes; ++k) {
            const double r = p->class_radius[k];
            if (!(r > 0.0) || !std::isfinite(r)) fail(IBPME_ERR_ARG, "class_radius[%d] must be > 0", k);
            amax = std::fmax(amax, r);
        }
        p->bead_radius = amax;
    } else {
        p->n_radius_classes = 0;
    }
    if (!(p->bead_radius > 0.0)) fail(IBPME_ERR_ARG, "bead_radius must be > 0");
    if (!(p->eps_f > 0.0)) fail(IBPME_ERR_ARG, "eps_f must be > 0");
    if (p->precision != IBPME_FP64 && p->precision != IBPME_MIXED) fail(IBPME_ERR_ARG, "unknown precision");
    if (p->max_rhs == 0) p->max_rhs = 3;
    if (p->max_rhs < 1 || p->max_rhs > kMaxRhs) fail(IBPME_ERR_ARG, "max_rhs must be in 1..%d", kMaxRhs);
    if (p->tol == 0.0) p->tol = 1e-6;
    if (!(p->tol > 0.0 && p->tol < 1.0)) fail(IBPME_ERR_ARG, "tol must be in (0, 1)");
    const double lnt = std::log(1.0 / p->tol);
    const bool mesh_auto = p->mesh[0] == 0 && p->mesh[1] == 0 && p->mesh[2] == 0;
    if (mesh_auto) {
        if (!(p->xi > 0.0)) fail(IBPME_ERR_ARG, "mesh = 0 needs xi > 0");
        const double kc = 2.0 * p->xi * std::sqrt(lnt);
        for (int d = 0; d < 3; ++d) {
            int m = (int)std::ceil(1.0 + p->box[d] * kc / kPi);
            if (m < 8) m = 8;
            while (!good_fft_size(m)) ++m;
            p->mesh[d] = m;
        }
    }
    for (int d = 0; d < 3; ++d)
        if (p->mesh[d] < 2 || p->mesh[d] > 2048) fail(IBPME_ERR_ARG, "mesh[%d] = %d outside 2..2048", d, p->mesh[d]);
    double kc = 1e300, h = 0.0, lmin = 1e300;
    for (int d = 0; d < 3; ++d) {
        kc = std::fmin(kc, kPi * (p->mesh[d] - 1) / p->box[d]);
        h = std::fmax(h, p->box[d] / p->mesh[d]);
        lmin = std::fmin(lmin, p->box[d]);
    }
    if (p->xi == 0.0) p->xi = kc / (2.0 * std::sqrt(lnt));
    if (!(p->xi > 0.0)) fail(IBPME_ERR_ARG, "xi must be > 0");
    if (p->P == 0) p->P = (int)std::ceil(2.0 * lnt / kPi);
    if (p->P < 1 || p->P > kMaxP) fail(IBPME_ERR_ARG, "P = %d outside 1..%d", p->P, kMaxP);
    for (int d = 0; d < 3; ++d)
        if (p->mesh[d] < p->P) fail(IBPME_ERR_ARG, "mesh[%d] = %d smaller than P = %d", d, p->mesh[d], p->P);
    if (p->eta == 0.0) p->eta = h * h * p->xi * p->xi * p->P / kPi;
    if (!(p->eta > 0.0)) fail(IBPME_ERR_ARG, "eta must be > 0");
    if (p->r_cut == 0.0) p->r_cut = std::sqrt(lnt) / p->xi + 2.0 * p->bead_radius;
    if (!(p->r_cut > 0.0) || p->r_cut >= 0.5 * lmin)
        fail(IBPME_ERR_ARG, "r_cut = %g must be in (0, L/2 = %g); use a finer mesh or a larger xi", p->r_cut,
             0.5 * lmin);
}

MeshGeom make_geom(const ibpme_params& p) {
    MeshGeom g{};
    const double xi = p.xi, eta = p.eta;
    double vh = 1.0;
    for (int d = 0; d < 3; ++d) {
        g.L[d] = p.box[d];
        g.N[d] = p.mesh[d];
        g.h[d] = p.box[d] / p.mesh[d];
        g.inv_h[d] = p.mesh[d] / p.box[d];
        g.kappa[d] = 2.0 * xi * xi * g.h[d] * g.h[d] / eta;
        vh *= g.h[d];
    }
    g.P = p.P;
    g.c = std::pow(2.0 * xi * xi / (kPi * eta), 1.5);
    g.gather = g.c * vh / p.eps_f;
    g.grad = g.gather * 4.0 * xi * xi / eta;
    g.G = (long long)p.mesh[0] * p.mesh[1] * p.mesh[2];
    g.Gc = (long long)(p.mesh[0] / 2 + 1) * p.mesh[1] * p.mesh[2];
    return g;
}

namespace {

void check_n(int n) {
    if (n < 0) fail(IBPME_ERR_ARG, "n must be >= 0");
}

// A context with radius classes needs them bound for the call's bead count.
void check_classes(const ibpme_ctx* c, int n) {
    if (c->ncls > 1 && n > 0 && c->cls_n != n)
        fail(IBPME_ERR_ARG, "radius classes are bound for %d beads, the call has %d (ibpme_set_radius_classes)",
             c->cls_n, n);
}

}  // namespace

void* pinned_host(ibpme_ctx* c, size_t bytes) {
    if (bytes > c->pinned_bytes) {
        if (c->pinned) cudaFreeHost(c->pinned);
        c->pinned = nullptr;
        c->pinned_bytes = 0;
        size_t want = bytes < 4096 ? 4096 : bytes;
        IBP_CUDA(cudaMallocHost(&c->pinned, want));
        c->pinned_bytes = want;
    }
    return c->pinned;
}

void wrap_positions(ibpme_ctx* c, int n, const double* x, double* xw) {
    if (n == 0) return;
    wrap_kernel<<<div_up(3LL * n, 256), 256, 0, c->stream>>>(n, x, c->p.box[0], c->p.box[1], c->p.box[2], xw);
    IBP_CHECK_LAUNCH();
}

void pme_reserve(ibpme_ctx* c, int n, int nrhs, bool field) {
    const size_t m = (size_t)nrhs * n;
    c->psi_r.ensure(sizeof(double) * (m ? m : 1));
    c->psi_k.ensure(sizeof(double) * (m ? m : 1));
    if (field) {
        c->E_r.ensure(sizeof(double) * 3 * (m ? m : 1));
        c->E_k.ensure(sizeof(double) * 3 * (m ? m : 1));
    }
    c->scalars.ensure(sizeof(double) * (size_t)(nrhs * c->ncfg));
}

namespace {

// out[r][free_idx[f]] = v[r][f]
__global__ void free_scatter_kernel(int nf, int n, int R, const int* __restrict__ free_idx, const double* __restrict__ v,
                                    double* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nf * R) return;
    const int r = (int)(t / nf), f = (int)(t % nf);
    out[(size_t)r * n + free_idx[f]] = v[t];
}

}  // namespace

void tma_check(ibpme_ctx* c) {
    const int e32 = c->have32 ? c->mesh32.tma_failed() : 0;
    const int e64 = c->mesh64.tma_failed();
    if (e32 == 1 || e64 == 1) fail(IBPME_ERR_TIMEOUT, "a tensor copy of a tiled mesh gather was not complete in time");
    if (e32 || e64)   // a check before the copy failed: the gather loaded the region itself
        fail(IBPME_ERR_CUDA, "tensor copy of a tiled mesh gather refused by its check %d", e32 ? e32 : e64);
}

void pme_apply(ibpme_ctx* c, int n, const double* xw, const double* q, int nrhs, int prec, double* psi,
               double* E, bool near_ready, bool near32, const FreeMesh* fm) {
    c->grid64_final = false;   // the meshes are about to hold other charges
    c->field64_ready = false;
    c->near_field_ready = false;
    if (!near_ready) near_build(c, n, xw, E != nullptr);
    const size_t m = (size_t)nrhs * n;
    pme_reserve(c, n, nrhs, E != nullptr);
    double* pr = c->psi_r.as<double>();
    double* pk = c->psi_k.as<double>();
    double* er = nullptr;
    double* ek = nullptr;
    if (E) {
        er = c->E_r.as<double>();
        ek = c->E_k.as<double>();
    }
    // The real-space pass and the mesh pass are independent until they are
    // combined: the near field runs on the context's second stream, forked from
    // and joined back into the calling stream (two branches of a captured graph).
    const cudaStream_t main = c->stream;
    IBP_CUDA(cudaEventRecord(c->ev_fork, main));
    IBP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    {
        struct Restore {
            ibpme_ctx* c;
            cudaStream_t s;
            ~Restore() { c->stream = s; }
        } restore{c, main};
        c->stream = c->aux;
        near_apply(c, n, q, nrhs, pr, near32 && prec == IBPME_MIXED);
        if (E) near_field(c, n, xw, q, nrhs, er);
        else if (fm && fm->er) near_field(c, n, xw, q, nrhs, fm->er);
    }
    IBP_CUDA(cudaEventRecord(c->ev_join, c->aux));
    // mesh channel groups: the radius classes, else the configurations
    const int* mg = mesh_cfg(c);
    const int ng = mesh_groups(c);
    const int ch = nrhs * ng;
    const StencilCache* sc = stencil_cache(c, n, xw);
    if (prec == IBPME_MIXED) {
        if (!c->have32) fail(IBPME_ERR_ARG, "mixed precision needs a context created with IBPME_MIXED");
        c->mesh32.spread(n, xw, q, nrhs, mg, ng, c->stream, sc);
        c->mesh32.transform(ch, c->stream);
        c->mesh32.gather(n, xw, nrhs, mg, pk, ek, c->stream, sc);
    } else {
        if (fm && fm->dq)
            c->mesh64.spread(fm->nf, fm->xf, fm->dq, nrhs, fm->cfg, ng, c->stream, fm->sc, true);
        else
            c->mesh64.spread(n, xw, q, nrhs, mg, ng, c->stream, sc);
        c->mesh64.transform(ch, c->stream);
        if (fm && fm->tmp && !E) {
            c->mesh64.gather(fm->nf, fm->xf, nrhs, fm->cfg, fm->tmp, nullptr, c->stream, fm->sc);
            free_scatter_kernel<<<div_up((long long)fm->nf * nrhs, 256), 256, 0, c->stream>>>(
                fm->nf, n, nrhs, fm->free_idx, fm->tmp, pk);
            IBP_CHECK_LAUNCH();
        } else {
            c->mesh64.gather(n, xw, nrhs, mg, pk, ek ? ek : (fm ? fm->ek : nullptr), c->stream, sc);
            c->field64_ready = !E && fm && fm->ek;
            c->near_field_ready = !E && fm && fm->er;
        }
    }
    IBP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (m) {
        const int nq = nrhs * c->ncfg;   // k = 0 sums per configuration
        double* qsum = static_cast<double*>(c->scalars.ensure(sizeof(double) * (size_t)nq));
        IBP_CUDA(cudaMemsetAsync(qsum, 0, sizeof(double) * nq, c->stream));
        qsum_kernel<<<dim3(div_up(n, 256) < 64 ? div_up(n, 256) : 64, nrhs), 256, 0, c->stream>>>(n, nrhs, q,
                                                                                                c->bcfg, qsum);
        IBP_CHECK_LAUNCH();
        const double V = c->p.box[0] * c->p.box[1] * c->p.box[2];
        const double k0 = 1.0 / (4.0 * c->xi * c->xi * V * c->eps);
        combine_kernel<<<div_up((long long)m, 256), 256, 0, c->stream>>>((long long)m, n, nrhs, pr, pk, qsum,
                                                                         c->bcfg, k0, psi);
        IBP_CHECK_LAUNCH();
        if (E) {
            add_kernel<<<div_up(3LL * m, 256), 256, 0, c->stream>>>(3LL * (long long)m, er, ek, E);
            IBP_CHECK_LAUNCH();
        }
    }
}

bool free_prepare(ibpme_ctx* c, const double* xw, int nrhs) {
    if (std::getenv("IBPME_FULL_OPERATOR")) return false;   // the switch lets tests compare both paths
    if (!near_free_build(c, xw)) return false;
    if (!free_stencil_cache(c)) return false;
    FreeSet& fs = c->fs;
    const size_t m = (size_t)nrhs * fs.nfree;
    fs.psi_r.ensure(sizeof(double) * (m ? m : 1));
    fs.psi_k.ensure(sizeof(double) * (m ? m : 1));
    fs.qsum.ensure(sizeof(double) * (size_t)(nrhs * c->ncfg));
    return true;
}

void pme_apply_free(ibpme_ctx* c, const double* qc, int nrhs, int prec, double* psi_f, bool near32) {
    FreeSet& fs = c->fs;
    const int n = fs.nfree;
    c->grid64_final = false;   // the meshes are about to hold other charges
    c->field64_ready = false;
    c->near_field_ready = false;
    if (n == 0) return;
    double* pr = fs.psi_r.as<double>();
    double* pk = fs.psi_k.as<double>();
    const double* xf = fs.xf.as<double>();
    const int* fcfg = c->ncfg > 1 ? c->bodies.free_cfg.as<int>() : nullptr;
    const int* fmg = c->ncls > 1 ? c->fs.cls_f.as<int>() : fcfg;   // mesh channel group of each free bead
    const int ng = mesh_groups(c);
    // near field on the second stream, as in pme_apply
    const cudaStream_t main = c->stream;
    IBP_CUDA(cudaEventRecord(c->ev_fork, main));
    IBP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    {
        struct Restore {
            ibpme_ctx* c;
            cudaStream_t s;
            ~Restore() { c->stream = s; }
        } restore{c, main};
        c->stream = c->aux;
        near_apply_free(c, qc, nrhs, pr, near32 && prec == IBPME_MIXED);
    }
    IBP_CUDA(cudaEventRecord(c->ev_join, c->aux));
    const int ch = nrhs * ng;
    const StencilCache* sc = free_stencil_cache(c);
    if (prec == IBPME_MIXED) {
        if (!c->have32) fail(IBPME_ERR_ARG, "mixed precision needs a context created with IBPME_MIXED");
        c->mesh32.spread(n, xf, qc, nrhs, fmg, ng, c->stream, sc);
        c->mesh32.transform(ch, c->stream);
        c->mesh32.gather(n, xf, nrhs, fmg, pk, nullptr, c->stream, sc);
    } else {
        c->mesh64.spread(n, xf, qc, nrhs, fmg, ng, c->stream, sc);
        c->mesh64.transform(ch, c->stream);
        c->mesh64.gather(n, xf, nrhs, fmg, pk, nullptr, c->stream, sc);
    }
    IBP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    double* qsum = fs.qsum.as<double>();
    IBP_CUDA(cudaMemsetAsync(qsum, 0, sizeof(double) * nrhs * c->ncfg, c->stream));
    qsum_kernel<<<dim3(div_up(n, 256) < 64 ? div_up(n, 256) : 64, nrhs), 256, 0, c->stream>>>(n, nrhs, qc, fcfg, qsum);
    IBP_CHECK_LAUNCH();
    const double V = c->p.box[0] * c->p.box[1] * c->p.box[2];
    const double k0 = 1.0 / (4.0 * c->xi * c->xi * V * c->eps);
    const long long m = (long long)nrhs * n;
    combine_kernel<<<div_up(m, 256), 256, 0, c->stream>>>(m, n, nrhs, pr, pk, qsum, fcfg, k0, psi_f);
    IBP_CHECK_LAUNCH();
}

}  // namespace ibp

using namespace ibp;

IBP_API const char* ibpme_last_error(void) { return g_err; }

IBP_API ibpme_status pme_setup(ibpme_ctx** ctx, const ibpme_params* params, void* cuda_stream) {
    if (!ctx) {
        set_error("ctx is NULL");
        return IBPME_ERR_ARG;
    }
    *ctx = nullptr;
    return guard([&]() -> ibpme_status {
        if (!params) fail(IBPME_ERR_ARG, "params is NULL");
        ibpme_ctx* c = new ibpme_ctx();
        try {
            resolve_params(params, &c->p);
            IBP_CUDA(cudaGetDevice(&c->device));
            c->stream = static_cast<cudaStream_t>(cuda_stream);
            c->xi = c->p.xi;
            c->eta = c->p.eta;
            c->rc = c->p.r_cut;
            c->a = c->p.bead_radius;
            c->eps = c->p.eps_f;
            c->P = c->p.P;
            c->geom = make_geom(c->p);
            if (c->p.n_radius_classes >= 2) {
                c->ncls = c->p.n_radius_classes;
                for (int k = 0; k < c->ncls; ++k) c->cls_a[k] = c->p.class_radius[k];
            }
            c->mesh64.init(c->geom, c->p.max_rhs, c->xi, c->eta, c->a, c->stream, c->ncls, c->cls_a);
            c->mesh64.plans(c->ncls, c->stream);
            if (c->p.precision == IBPME_MIXED) {
                c->mesh32.init(c->geom, c->p.max_rhs, c->xi, c->eta, c->a, c->stream, c->ncls, c->cls_a);
                c->mesh32.plans(c->ncls, c->stream);
                c->have32 = true;
            }
            IBP_CUDA(cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking));
            IBP_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
            IBP_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
            IBP_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
            IBP_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
            IBP_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
            near_setup(c);
            pinned_host(c, 4096);
            IBP_CUDA(cudaStreamSynchronize(c->stream));
        } catch (...) {
            pme_destroy(c);
            throw;
        }
        *ctx = c;
        return IBPME_OK;
    });
}

IBP_API ibpme_status pme_destroy(ibpme_ctx* c) {
    if (!c) return IBPME_OK;
    cudaStreamSynchronize(c->stream);
    krylov_destroy(c);
    if (c->work) {
        cudaStreamSynchronize(c->work);
        cudaStreamDestroy(c->work);
    }
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaStreamDestroy(c->aux);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    c->mesh64.destroy();
    c->mesh32.destroy();
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    if (c->pre.hm_pin) cudaFreeHost(c->pre.hm_pin);
    c->pre.hm_pin = nullptr;
    delete c;
    return IBPME_OK;
}

IBP_API ibpme_status ibpme_set_stream(ibpme_ctx* c, void* cuda_stream) {
    if (!c) {
        set_error("ctx is NULL");
        return IBPME_ERR_ARG;
    }
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return IBPME_OK;
}

IBP_API ibpme_status ibpme_set_radius_classes(ibpme_ctx* c, int n, const int* cls) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        if (c->ncls < 2) fail(IBPME_ERR_ARG, "the context was created without radius classes");
        check_n(n);
        if (n > 0 && !cls) fail(IBPME_ERR_ARG, "cls is required");
        if (n > 0 && is_device_ptr(cls)) fail(IBPME_ERR_ARG, "cls must be a host array");
        std::vector<int> h(cls, cls + n);
        for (int i = 0; i < n; ++i)
            if (h[i] < 0 || h[i] >= c->ncls) fail(IBPME_ERR_ARG, "cls[%d] = %d outside 0..%d", i, h[i], c->ncls - 1);
        IBP_CUDA(cudaStreamSynchronize(c->stream));   // no earlier call still reads the old binding
        c->cls.ensure(sizeof(int) * (size_t)(n ? n : 1));
        if (n > 0) {
            IBP_CUDA(cudaMemcpyAsync(c->cls.p, h.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
            IBP_CUDA(cudaStreamSynchronize(c->stream));
        }
        c->cls_h = std::move(h);
        c->cls_n = n > 0 ? n : -1;
        ++c->cls_version;
        // everything keyed by the bead classes is rebuilt by the next call
        c->near.fp_valid = false;
        c->stencils.valid = false;
        c->fs.valid = false;
        c->fs.sc.valid = false;
        c->grid64_final = false;
        c->field64_ready = false;
        c->near_field_ready = false;
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_get_params(const ibpme_ctx* c, ibpme_params* out) {
    if (!c || !out) {
        set_error("NULL argument");
        return IBPME_ERR_ARG;
    }
    *out = c->p;
    return IBPME_OK;
}

IBP_API ibpme_status pme_spread(ibpme_ctx* c, int n, const double* x, const double* q, int nrhs, void* grid_out) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        check_n(n);
        if (nrhs < 1 || nrhs > c->p.max_rhs) fail(IBPME_ERR_ARG, "nrhs %d outside 1..%d", nrhs, c->p.max_rhs);
        if (n > 0 && (!x || !q)) fail(IBPME_ERR_ARG, "x and q are required");
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        const double* dq = static_cast<const double*>(stage_in(c, q, sizeof(double) * (size_t)nrhs * n, c->st_q));
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * (n ? n : 1)));
        wrap_positions(c, n, dx, xw);
        c->bodies_current = false;
        c->near.fp_pre_valid = false;
        const bool mixed = c->p.precision == IBPME_MIXED;
        const size_t gb = (mixed ? sizeof(float) : sizeof(double)) * (size_t)c->geom.G * nrhs;
        if (mixed)
            c->mesh32.spread(n, xw, dq, nrhs, nullptr, 1, c->stream);
        else
            c->mesh64.spread(n, xw, dq, nrhs, nullptr, 1, c->stream);
        if (grid_out) {
            const void* src = mixed ? c->mesh32.grid.p : c->mesh64.grid.p;
            const cudaMemcpyKind kind = is_device_ptr(grid_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            IBP_CUDA(cudaMemcpyAsync(grid_out, src, gb, kind, c->stream));
            if (kind == cudaMemcpyDeviceToHost) IBP_CUDA(cudaStreamSynchronize(c->stream));
        }
        return IBPME_OK;
    });
}

IBP_API ibpme_status pme_field(ibpme_ctx* c, int n, const double* x, const double* q, int nrhs, double* psi,
                               double* E) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        tma_check(c);
        check_n(n);
        check_classes(c, n);
        if (nrhs < 1 || nrhs > c->p.max_rhs) fail(IBPME_ERR_ARG, "nrhs %d outside 1..%d", nrhs, c->p.max_rhs);
        if (n > 0 && (!x || !q || !psi)) fail(IBPME_ERR_ARG, "x, q and psi are required");
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        const double* dq = static_cast<const double*>(stage_in(c, q, sizeof(double) * (size_t)nrhs * n, c->st_q));
        OutArg op = stage_out(c, psi, sizeof(double) * (size_t)nrhs * n, c->st_out1);
        OutArg oe = stage_out(c, E, sizeof(double) * 3 * (size_t)nrhs * n, c->st_out2);
        if (n == 0) return IBPME_OK;
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        c->bodies_current = false;   // beads without bodies: every pair goes through the table
        c->near.fp_pre_valid = false;
        pme_apply(c, n, xw, dq, nrhs, c->p.precision, static_cast<double*>(op.dev), static_cast<double*>(oe.dev),
                  false);
        finish_out(c, op);
        finish_out(c, oe);
        if (op.host || oe.host) {
            IBP_CUDA(cudaStreamSynchronize(c->stream));
            tma_check(c);
        }
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_rpy_mobility(ibpme_ctx* c, int n, const double* x, const double* F, double mu,
                                        double* U) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        tma_check(c);
        check_n(n);
        if (!(mu > 0.0) || !std::isfinite(mu)) fail(IBPME_ERR_ARG, "mu must be > 0");
        if (c->ncls > 1) fail(IBPME_ERR_UNEQUAL_RADII, "the RPY mobility takes one bead radius");
        if (n > 0 && (!x || !F || !U)) fail(IBPME_ERR_ARG, "x, F and U are required");
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        const double* dF = static_cast<const double*>(stage_in(c, F, sizeof(double) * 3 * n, c->st_q));
        OutArg ou = stage_out(c, U, sizeof(double) * 3 * (size_t)n, c->st_out1);
        if (n == 0) return IBPME_OK;
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        c->bodies_current = false;   // beads without bodies: every pair goes through the table
        c->near.fp_pre_valid = false;
        rpy_apply(c, n, xw, dF, mu, static_cast<double*>(ou.dev));
        finish_out(c, ou);
        if (ou.host) {
            IBP_CUDA(cudaStreamSynchronize(c->stream));
            tma_check(c);
        }
        return IBPME_OK;
    });
}

namespace {

struct BodiesDev {
    ibpme_bodies b{};
};

// Stages the body arrays and uploads the bookkeeping; returns the device-side view.
void prepare_bodies(ibpme_ctx* c, int n, const ibpme_bodies* bodies, const double* xw, int ncfg = 1,
                    const int* cfg_bodies = nullptr) {
    if (!bodies) fail(IBPME_ERR_ARG, "bodies is NULL");
    const int nb = bodies->n_bodies;
    if (nb < 1) fail(IBPME_ERR_ARG, "n_bodies must be >= 1");
    if (!bodies->body_offsets || !bodies->X || !bodies->Q) fail(IBPME_ERR_ARG, "body arrays are required");
    ibpme_bodies d{};
    d.n_bodies = nb;
    d.body_offsets = static_cast<const int*>(stage_in(c, bodies->body_offsets, sizeof(int) * (nb + 1), c->st_off));
    d.X = static_cast<const double*>(stage_in(c, bodies->X, sizeof(double) * 3 * nb, c->st_X));
    d.Q = static_cast<const double*>(stage_in(c, bodies->Q, sizeof(double) * nb, c->st_Q));
    // one synchronisation for the body structure and the position fingerprint
    const unsigned long long h = near_prefetch(c, n, xw, d.body_offsets, nb + 1);
    bodies_upload(c, n, &d, xw, ncfg, nullptr, cfg_bodies, &h);
}

// The configuration split of a batched call, undone when the call ends so that
// every other entry point sees one configuration.
struct ConfigScope {
    ibpme_ctx* c;
    ConfigScope(ibpme_ctx* c_, int ncfg) : c(c_) {
        c->ncfg = ncfg;
        c->bcfg = ncfg > 1 ? c->bodies.bead_cfg.as<int>() : nullptr;
    }
    ~ConfigScope() {
        c->ncfg = 1;
        c->bcfg = nullptr;
    }
};

// One solve call up to its device outputs (shared by induced_charge_solve,
// induced_charge_solve_batch and ibpme_bd_advance); the caller finishes the outputs.
struct SolveCall {
    SolveArgs a{};
    OutArg oq, op, os;
    std::vector<ibpme_solve_stats> st;
};

void solve_run(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies, int ncfg, const int* cfg_bodies,
               const double* E0, int nrhs, const ibpme_solve_opts* opts, double* q_out, double* psi_out,
               double* S_out, SolveCall& call) {
    check_n(n);
    if (n == 0) fail(IBPME_ERR_ARG, "a solve needs at least one bead");
    if (c->ncls > 1 && ncfg > 1)
        fail(IBPME_ERR_UNEQUAL_RADII, "the batched solve takes one bead radius (this context has radius classes)");
    check_classes(c, n);
    if (nrhs < 1 || nrhs > c->p.max_rhs) fail(IBPME_ERR_ARG, "nrhs %d outside 1..%d", nrhs, c->p.max_rhs);
    if (!x || !E0 || !q_out) fail(IBPME_ERR_ARG, "x, E0 and q_out are required");
    if (ncfg < 1) fail(IBPME_ERR_ARG, "n_configs must be >= 1");
    if (ncfg > 1 && !cfg_bodies) fail(IBPME_ERR_ARG, "cfg_bodies is required");
    if (cfg_bodies && is_device_ptr(cfg_bodies)) fail(IBPME_ERR_ARG, "cfg_bodies must be a host array");
    ibpme_solve_opts o{};
    o.precision = -1;
    if (opts) o = *opts;
    SolveArgs& a = call.a;
    a.n = n;
    a.nrhs = nrhs;
    a.prec = o.precision < 0 ? c->p.precision : o.precision;
    if (a.prec != IBPME_FP64 && a.prec != IBPME_MIXED) fail(IBPME_ERR_ARG, "unknown solve precision");
    if (a.prec == IBPME_MIXED && !c->have32) fail(IBPME_ERR_ARG, "mixed solve needs a mixed context");
    a.rtol = o.rtol > 0 ? o.rtol : 1e-6;
    a.restart = o.restart > 0 ? o.restart : 50;
    if (a.restart > 128) fail(IBPME_ERR_ARG, "restart must be <= 128");
    a.max_iter = o.max_iter > 0 ? o.max_iter : 3000;
    const bool learned = o.guess == IBPME_GUESS_LEARNED || o.guess == IBPME_GUESS_LEARNED_STEP;
    if (learned && !o.mlp) fail(IBPME_ERR_ARG, "a learned guess needs opts->mlp");
    if (o.guess != IBPME_GUESS_ZERO && o.guess != IBPME_GUESS_USER && !learned) fail(IBPME_ERR_ARG, "unknown guess mode");
    if (learned && cfg_bodies) fail(IBPME_ERR_ARG, "a batched solve takes no learned guess");
    if (learned && c->ncls > 1)
        fail(IBPME_ERR_UNEQUAL_RADII, "the learned guess takes one bead radius (this context has radius classes)");
    if (o.precond != IBPME_PRECOND_BODY && o.precond != IBPME_PRECOND_NONE) fail(IBPME_ERR_ARG, "unknown precond");
    a.precond = o.precond == IBPME_PRECOND_BODY;
    a.user_guess = o.guess == IBPME_GUESS_USER || learned;
    a.learned = learned;
    const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
    a.E0 = static_cast<const double*>(stage_in(c, E0, sizeof(double) * 3 * nrhs, c->st_E0));
    double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
    wrap_positions(c, n, dx, xw);
    a.xw = xw;
    prepare_bodies(c, n, bodies, xw, ncfg, cfg_bodies);
    ConfigScope scope(c, ncfg);
    const int nb = bodies->n_bodies;
    call.oq = stage_out(c, q_out, sizeof(double) * (size_t)nrhs * n, c->st_out1, a.user_guess);
    call.op = stage_out(c, psi_out, sizeof(double) * (size_t)nrhs * nb, c->st_out2);
    call.os = stage_out(c, S_out, sizeof(double) * 3 * (size_t)nrhs * nb, c->st_out3);
    a.q = static_cast<double*>(call.oq.dev);
    a.psi = static_cast<double*>(call.op.dev);
    if (a.learned)
        learned_guess(c, static_cast<const ibpme_mlp*>(o.mlp), n, xw, a.E0, nrhs, a.q,
                      o.guess == IBPME_GUESS_LEARNED_STEP);
    call.st.assign(ncfg, ibpme_solve_stats{});
    tma_check(c);   // a gather of an earlier call, finished by now
    solve(c, a, call.st.data());
    tma_check(c);   // the solve's last residual has synchronised
    if (a.learned) learned_check(static_cast<const ibpme_mlp*>(o.mlp));   // the solve has synchronised
    if (S_out) body_dipoles(c, n, a.q, nrhs, static_cast<double*>(call.os.dev));
}

// Statistics of a finished solve call into stats[ncfg]; the call's status.
ibpme_status solve_status(SolveCall& call, std::chrono::steady_clock::time_point t0, ibpme_solve_stats* stats) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    double worst = 0.0;
    bool finite = true;
    for (auto& e : call.st) {
        e.time_ms = ms;
        finite = finite && std::isfinite(e.rel_residual);
        worst = std::max(worst, e.rel_residual);
    }
    if (stats)
        for (size_t k = 0; k < call.st.size(); ++k) stats[k] = call.st[k];
    if (!finite) fail(IBPME_ERR_NONFINITE, "non-finite residual in the solve");
    if (!(worst <= call.a.rtol)) {
        set_error("not converged: relative residual %.3e after %d iterations", worst, call.st[0].iters);
        return IBPME_ERR_NOT_CONVERGED;
    }
    return IBPME_OK;
}

ibpme_status solve_entry(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies, int ncfg,
                         const int* cfg_bodies, const double* E0, int nrhs, const ibpme_solve_opts* opts,
                         double* q_out, double* psi_out, double* S_out, ibpme_solve_stats* stats) {
    if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
    DeviceScope ds(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    SolveCall call;
    solve_run(c, n, x, bodies, ncfg, cfg_bodies, E0, nrhs, opts, q_out, psi_out, S_out, call);
    finish_out(c, call.oq);
    finish_out(c, call.op);
    finish_out(c, call.os);
    // the last convergence check has synchronised; device outputs are stream-ordered,
    // host outputs must have arrived before the call returns
    if (call.oq.host || call.op.host || call.os.host) IBP_CUDA(cudaStreamSynchronize(c->stream));
    return solve_status(call, t0, stats);
}

// Potential psi [n] and field E [n][3] of the charges q at the positions of the
// solve that just produced them (near table and stencils current).  The FP64 mesh
// grid of the solve's final residual already holds these charges' transformed
// potential and the Krylov state their FP64 potentials: the field is one gradient
// gather of that grid plus the near field, and the potentials are taken as they are.
// Without that evaluation (the solve skipped it) one full evaluation.
const double* solution_field(ibpme_ctx* c, int n, const double* xw, const double* q, double* psi, double* E) {
    const double* psi64 = solve_potentials(c);
    if (!psi64) {
        pme_apply(c, n, xw, q, 1, c->p.precision, psi, E, true);
        return psi;
    }
    pme_reserve(c, n, 1, true);
    double* er = c->E_r.as<double>();
    double* ek = c->E_k.as<double>();
    const cudaStream_t main = c->stream;
    if (!c->near_field_ready) {   // the final residual did not compute the real-space field beside its mesh pass
        IBP_CUDA(cudaEventRecord(c->ev_fork, main));
        IBP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
        {
            struct Restore {
                ibpme_ctx* c;
                cudaStream_t s;
                ~Restore() { c->stream = s; }
            } restore{c, main};
            c->stream = c->aux;
            near_field(c, n, xw, q, 1, er);
        }
    } else {
        IBP_CUDA(cudaEventRecord(c->ev_fork, main));   // nothing on the second stream: join at once
        IBP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    }
    IBP_CUDA(cudaEventRecord(c->ev_join, c->aux));
    if (!c->field64_ready) {   // the final residual did not gather the mesh field with its potential
        const StencilCache* sc = stencil_cache(c, n, xw);
        c->mesh64.gather(n, xw, 1, mesh_cfg(c), c->psi_k.as<double>(), ek, c->stream, sc);
    }
    IBP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    add_kernel<<<div_up(3LL * n, 256), 256, 0, c->stream>>>(3LL * n, er, ek, E);
    IBP_CHECK_LAUNCH();
    c->grid64_final = false;
    c->field64_ready = false;
    c->near_field_ready = false;
    return psi64;
}

}  // namespace

IBP_API ibpme_status ibpme_rigid_mobility(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                          const double* FL, double mu, const ibpme_solve_opts* opts, double* W,
                                          double* f_out, ibpme_solve_stats* stats) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        const auto t0 = std::chrono::steady_clock::now();
        tma_check(c);
        check_n(n);
        if (n == 0) fail(IBPME_ERR_ARG, "the mobility problem needs at least one bead");
        if (!(mu > 0.0) || !std::isfinite(mu)) fail(IBPME_ERR_ARG, "mu must be > 0");
        if (c->ncls > 1) fail(IBPME_ERR_UNEQUAL_RADII, "the RPY mobility takes one bead radius");
        if (!x || !bodies || !FL || !W) fail(IBPME_ERR_ARG, "x, bodies, FL and W are required");
        ibpme_solve_opts o{};
        if (opts) o = *opts;
        const double rtol = o.rtol > 0 ? o.rtol : 1e-6;
        const int restart = o.restart > 0 ? o.restart : 50;
        if (restart > 200) fail(IBPME_ERR_ARG, "restart must be <= 200");
        const int max_iter = o.max_iter > 0 ? o.max_iter : 3000;
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        prepare_bodies(c, n, bodies, xw);
        c->bodies_current = false;   // the RPY pass takes every pair from the table (no compact bodies)
        const int nb = bodies->n_bodies;
        const double* dFL = static_cast<const double*>(stage_in(c, FL, sizeof(double) * 6 * nb, c->st_E0));
        OutArg ow = stage_out(c, W, sizeof(double) * 6 * (size_t)nb, c->st_out1);
        OutArg of = stage_out(c, f_out, sizeof(double) * 3 * (size_t)n, c->st_out2);
        ibpme_solve_stats st{};
        ibpme_status status = IBPME_OK;
        try {
            rigid_solve(c, n, xw, dFL, mu, rtol, restart, max_iter, static_cast<double*>(ow.dev),
                        static_cast<double*>(of.dev), &st, o.precond != IBPME_PRECOND_NONE);
        } catch (const Error& e) {
            if (e.status != IBPME_ERR_NOT_CONVERGED) throw;
            status = IBPME_ERR_NOT_CONVERGED;   // outputs hold the last iterate
        }
        finish_out(c, ow);
        finish_out(c, of);
        IBP_CUDA(cudaStreamSynchronize(c->stream));
        st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (stats) *stats = st;
        if (status != IBPME_OK) fail(status, "rigid mobility did not reach rtol %g in %d iterations", rtol, st.iters);
        return IBPME_OK;
    });
}

IBP_API ibpme_status induced_charge_solve(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                          const double* E0, int nrhs, const ibpme_solve_opts* opts,
                                          double* q_out, double* psi_out, double* S_out,
                                          ibpme_solve_stats* stats) {
    return guard([&]() -> ibpme_status {
        return solve_entry(c, n, x, bodies, 1, nullptr, E0, nrhs, opts, q_out, psi_out, S_out, stats);
    });
}

IBP_API ibpme_status induced_charge_solve_batch(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                                int n_configs, const int* cfg_bodies, const double* E0, int nrhs,
                                                const ibpme_solve_opts* opts, double* q_out, double* psi_out,
                                                double* S_out, ibpme_solve_stats* stats) {
    return guard([&]() -> ibpme_status {
        return solve_entry(c, n, x, bodies, n_configs, cfg_bodies, E0, nrhs, opts, q_out, psi_out, S_out, stats);
    });
}

IBP_API ibpme_status body_force_torque(ibpme_ctx* c, int n, const double* x, const double* q,
                                       const ibpme_bodies* bodies, const double* E0, double* f_bead, double* F,
                                       double* L, double* U) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        check_n(n);
        check_classes(c, n);
        if (n == 0) fail(IBPME_ERR_ARG, "n must be >= 1");
        if (!x || !q || !E0 || !F || !L) fail(IBPME_ERR_ARG, "x, q, E0, F and L are required");
        const int nb = bodies ? bodies->n_bodies : 0;
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        const double* dq = static_cast<const double*>(stage_in(c, q, sizeof(double) * n, c->st_q));
        const double* dE0 = static_cast<const double*>(stage_in(c, E0, sizeof(double) * 3, c->st_E0));
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        prepare_bodies(c, n, bodies, xw);
        OutArg of = stage_out(c, f_bead, sizeof(double) * 3 * n, c->st_out1);
        OutArg oF = stage_out(c, F, sizeof(double) * 3 * nb, c->st_out2);
        OutArg oL = stage_out(c, L, sizeof(double) * 3 * nb, c->st_out3);
        OutArg oU = stage_out(c, U, sizeof(double), c->st_out4);
        double* psi = static_cast<double*>(c->qfull.ensure(sizeof(double) * 4 * n));   // psi [n] then E [n][3]
        double* E = psi + n;
        pme_apply(c, n, xw, dq, 1, c->p.precision, psi, E, false);
        double* f = of.dev ? static_cast<double*>(of.dev) : static_cast<double*>(c->st_f.ensure(sizeof(double) * 3 * n));
        bead_forces(c, n, dq, dE0, E, f);
        body_reduce_force_torque(c, n, f, static_cast<double*>(oF.dev), static_cast<double*>(oL.dev));
        if (U) body_energy(c, n, dq, psi, dE0, static_cast<double*>(oU.dev));
        finish_out(c, of);
        finish_out(c, oF);
        finish_out(c, oL);
        finish_out(c, oU);
        if (of.host || oF.host || oL.host || oU.host) IBP_CUDA(cudaStreamSynchronize(c->stream));
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_bd_advance(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                      const double* E0, const ibpme_solve_opts* opts, const ibpme_bd_params* bd,
                                      double* q_io, double* psi_out, double* f_bead, double* F, double* L,
                                      double* U, double* x_out, double* X_out, ibpme_solve_stats* stats) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        const auto t0 = std::chrono::steady_clock::now();
        if (!bd || !F || !L || !x_out || !X_out) fail(IBPME_ERR_ARG, "bd, F, L, x_out and X_out are required");
        if (!(bd->dt > 0) || !(bd->gamma > 0) || !(bd->kT >= 0)) fail(IBPME_ERR_ARG, "need dt > 0, gamma > 0, kT >= 0");
        // the solve: positions staged and wrapped, bodies uploaded and the near table
        // built once for the whole step
        SolveCall call;
        call.a.want_field = true;   // the force pass follows
        solve_run(c, n, x, bodies, 1, nullptr, E0, 1, opts, q_io, psi_out, nullptr, call);
        const ibpme_status status = solve_status(call, t0, stats);
        if (status != IBPME_OK) {   // not converged: charges written, nothing moves
            finish_out(c, call.oq);
            finish_out(c, call.op);
            IBP_CUDA(cudaStreamSynchronize(c->stream));
            return status;
        }
        const int nb = bodies->n_bodies;
        const double* xw = call.a.xw;
        const double* q = call.a.q;
        const double* dE0 = call.a.E0;
        OutArg of = stage_out(c, f_bead, sizeof(double) * 3 * n, c->st_out5);
        OutArg oF = stage_out(c, F, sizeof(double) * 3 * nb, c->st_out3);
        OutArg oL = stage_out(c, L, sizeof(double) * 3 * nb, c->st_out4);
        OutArg oU = stage_out(c, U, sizeof(double), c->st_out6);
        OutArg ox = stage_out(c, x_out, sizeof(double) * 3 * n, c->st_out7);
        OutArg oX = stage_out(c, X_out, sizeof(double) * 3 * nb, c->st_out8);
        // forces, torques and energy of the solution (Eq. beadforce, Sec. III.C, Eq. pot_syst)
        double* buf = static_cast<double*>(c->qfull.ensure(sizeof(double) * 4 * n));   // psi [n] then E [n][3]
        double* E = buf + n;
        const double* psi = solution_field(c, n, xw, q, buf, E);
        double* f = of.dev ? static_cast<double*>(of.dev) : static_cast<double*>(c->st_f.ensure(sizeof(double) * 3 * n));
        bead_forces(c, n, q, dE0, E, f);
        body_reduce_force_torque(c, n, f, static_cast<double*>(oF.dev), static_cast<double*>(oL.dev));
        if (U) body_energy(c, n, q, psi, dE0, static_cast<double*>(oU.dev));
        // the Euler-Maruyama step (Eq. forward) with the hard-sphere forces of Eq. hardsphereFD
        bd_step(c, n, xw, f, bd, static_cast<double*>(ox.dev), static_cast<double*>(oX.dev));
        for (const OutArg* o : {&call.oq, &call.op, &of, &oF, &oL, &oU, &ox, &oX}) finish_out(c, *o);
        bool host = false;
        for (const OutArg* o : {&call.oq, &call.op, &of, &oF, &oL, &oU, &ox, &oX}) host = host || o->host;
        if (host) IBP_CUDA(cudaStreamSynchronize(c->stream));
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_bd_step(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                   const double* f_bead, const ibpme_bd_params* bd, double* x_out,
                                   double* X_out) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        check_n(n);
        check_classes(c, n);
        if (n == 0) fail(IBPME_ERR_ARG, "n must be >= 1");
        if (!x || !f_bead || !bd || !x_out || !X_out) fail(IBPME_ERR_ARG, "missing argument");
        if (!(bd->dt > 0) || !(bd->gamma > 0) || !(bd->kT >= 0)) fail(IBPME_ERR_ARG, "need dt > 0, gamma > 0, kT >= 0");
        const int nb = bodies ? bodies->n_bodies : 0;
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        const double* df = static_cast<const double*>(stage_in(c, f_bead, sizeof(double) * 3 * n, c->st_q));
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        prepare_bodies(c, n, bodies, xw);
        near_build(c, n, xw, false);
        OutArg ox = stage_out(c, x_out, sizeof(double) * 3 * n, c->st_out1);
        OutArg oX = stage_out(c, X_out, sizeof(double) * 3 * nb, c->st_out2);
        bd_step(c, n, xw, df, bd, static_cast<double*>(ox.dev), static_cast<double*>(oX.dev));
        finish_out(c, ox);
        finish_out(c, oX);
        if (ox.host || oX.host) IBP_CUDA(cudaStreamSynchronize(c->stream));
        return IBPME_OK;
    });
}

// ---------------------------------------------------------------------------
// Grand capacitance tensor (Sec. III.B, Eq. QS_capacitance)
// ---------------------------------------------------------------------------
namespace ibp {
namespace {

// Column k0 + r of Sigma'^T as bead potentials (r < R): column k < nb puts 1 on the
// beads of body k, column nb + 3 i + d puts r_ij,d on the beads of body i.
__global__ void cap_rhs_kernel(int n, int R, int k0, int nb, const int* __restrict__ bead_body,
                               const double* __restrict__ rel, double* __restrict__ psi) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int k = k0 + r, b = bead_body[j];
    double v = 0.0;
    if (k < nb) {
        v = b == k ? 1.0 : 0.0;
    } else {
        const int i = (k - nb) / 3, d = (k - nb) % 3;
        v = b == i ? rel[3 * j + d] : 0.0;
    }
    psi[t] = v;
}

// Rows of C for columns k0 .. k0 + R - 1: C[i][k] = sum over body i of q, C[nb + 3 i + d][k] =
// sum over body i of r_d q (Sigma' q).  One block per (column, body).
__global__ void cap_columns_kernel(int n, int nb, int R, int k0, const int* __restrict__ off,
                                   const double* __restrict__ rel, const double* __restrict__ q,
                                   double* __restrict__ C) {
    __shared__ double sh[4][32];
    const int r = blockIdx.y, i = blockIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = off[i] + threadIdx.x; j < off[i + 1]; j += blockDim.x) {
        const double qj = q[(size_t)r * n + j];
        v[0] += qj;
        v[1] += rel[3 * j] * qj;
        v[2] += rel[3 * j + 1] * qj;
        v[3] += rel[3 * j + 2] * qj;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        v[c] = warp_sum(v[c]);
        if (lane == 0) sh[c][w] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long ld = 4LL * nb, k = k0 + r;
        double tot[4] = {0.0, 0.0, 0.0, 0.0};
        for (int u = 0; u < (int)(blockDim.x >> 5); ++u)
            for (int c = 0; c < 4; ++c) tot[c] += sh[c][u];
        C[(size_t)i * ld + k] = tot[0];
        for (int d = 0; d < 3; ++d) C[(size_t)(nb + 3 * i + d) * ld + k] = tot[1 + d];
    }
}

}  // namespace
}  // namespace ibp

IBP_API ibpme_status ibpme_capacitance(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                       const ibpme_solve_opts* opts, double* C_out, ibpme_solve_stats* stats) {
    return guard([&]() -> ibpme_status {
        if (!c) fail(IBPME_ERR_ARG, "ctx is NULL");
        DeviceScope ds(c->device);
        const auto t0 = std::chrono::steady_clock::now();
        check_n(n);
        check_classes(c, n);
        if (n == 0) fail(IBPME_ERR_ARG, "the capacitance needs at least one body");
        if (!x || !bodies || !C_out) fail(IBPME_ERR_ARG, "x, bodies and C_out are required");
        const int nb = bodies->n_bodies;
        if (nb < 1) fail(IBPME_ERR_ARG, "n_bodies must be >= 1");
        ibpme_solve_opts o{};
        o.precision = -1;
        if (opts) o = *opts;
        if (o.guess != IBPME_GUESS_ZERO) fail(IBPME_ERR_ARG, "the capacitance solves start from the zero guess");
        if (o.precond != IBPME_PRECOND_BODY && o.precond != IBPME_PRECOND_NONE) fail(IBPME_ERR_ARG, "unknown precond");
        SolveArgs a{};
        a.n = n;
        a.prec = o.precision < 0 ? c->p.precision : o.precision;
        if (a.prec != IBPME_FP64 && a.prec != IBPME_MIXED) fail(IBPME_ERR_ARG, "unknown solve precision");
        if (a.prec == IBPME_MIXED && !c->have32) fail(IBPME_ERR_ARG, "mixed solve needs a mixed context");
        a.rtol = o.rtol > 0 ? o.rtol : 1e-6;
        a.restart = o.restart > 0 ? o.restart : 50;
        if (a.restart > 128) fail(IBPME_ERR_ARG, "restart must be <= 128");
        a.max_iter = o.max_iter > 0 ? o.max_iter : 3000;
        a.precond = o.precond == IBPME_PRECOND_BODY;
        const double* dx = static_cast<const double*>(stage_in(c, x, sizeof(double) * 3 * n, c->st_x));
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, dx, xw);
        a.xw = xw;
        // the net charges play no part (the body potentials are given): zeros where none are passed
        const int R = std::min(c->p.max_rhs, 4 * nb);
        double* zero = static_cast<double*>(c->cap_zero.ensure(sizeof(double) * (size_t)std::max(nb, 3 * R)));
        IBP_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * (size_t)std::max(nb, 3 * R), c->stream));
        ibpme_bodies b = *bodies;
        if (!b.Q) b.Q = zero;
        prepare_bodies(c, n, &b, xw);
        if (c->bodies.nmb != nb)
            fail(IBPME_ERR_ARG, "every body needs two beads or more (single-bead bodies are not conductors here)");
        a.E0 = zero;
        OutArg oc = stage_out(c, C_out, sizeof(double) * 16 * (size_t)nb * nb, c->st_out1);
        double* psi = static_cast<double*>(c->cap_psi.ensure(sizeof(double) * (size_t)R * n));
        double* q = static_cast<double*>(c->cap_q.ensure(sizeof(double) * (size_t)R * n));
        ibpme_solve_stats agg{};
        agg.outer = 0;
        for (int k0 = 0; k0 < 4 * nb; k0 += R) {
            const int r = std::min(R, 4 * nb - k0);
            cap_rhs_kernel<<<div_up((long long)n * r, 256), 256, 0, c->stream>>>(n, r, k0, nb,
                                                                              c->bodies.bead_body.as<int>(),
                                                                              c->bodies.rel.as<double>(), psi);
            IBP_CHECK_LAUNCH();
            a.nrhs = r;
            a.q = q;
            a.psi = nullptr;
            a.bead_psi = psi;
            ibpme_solve_stats st{};
            solve(c, a, &st);
            cap_columns_kernel<<<dim3(nb, r), 256, 0, c->stream>>>(n, nb, r, k0, c->bodies.off.as<int>(),
                                                                  c->bodies.rel.as<double>(), q,
                                                                  static_cast<double*>(oc.dev));
            IBP_CHECK_LAUNCH();
            agg.iters = std::max(agg.iters, st.iters);
            agg.outer = std::max(agg.outer, st.outer);
            agg.matvecs_fp64 += st.matvecs_fp64;
            agg.rel_residual = std::isfinite(st.rel_residual) && std::isfinite(agg.rel_residual)
                                   ? std::max(agg.rel_residual, st.rel_residual) : NAN;
            agg.init_rel_residual = std::max(agg.init_rel_residual, st.init_rel_residual);
        }
        finish_out(c, oc);
        IBP_CUDA(cudaStreamSynchronize(c->stream));
        agg.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (stats) *stats = agg;
        if (!std::isfinite(agg.rel_residual)) fail(IBPME_ERR_NONFINITE, "non-finite residual in the solve");
        if (!(agg.rel_residual <= a.rtol)) {
            set_error("not converged: relative residual %.3e after %d iterations", agg.rel_residual, agg.iters);
            return IBPME_ERR_NOT_CONVERGED;
        }
        return IBPME_OK;
    });
}
