// common.cuh -- internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <exception>
#include <string>
#include <map>
#include <utility>
#include <vector>

#include "../../include/ibpme.h"

#define IBP_API extern "C" __attribute__((visibility("default")))

namespace ibp {

// ---------------------------------------------------------------------------
// Errors: internal code throws ibp::Error; the C ABI converts it to a status.
// ---------------------------------------------------------------------------
struct Error : std::exception {
    ibpme_status status;
    explicit Error(ibpme_status s) : status(s) {}
};

void set_error(const char* fmt, ...);
[[noreturn]] void fail(ibpme_status s, const char* fmt, ...);

#define IBP_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            ::ibp::fail(e_ == cudaErrorMemoryAllocation ? IBPME_ERR_OOM : IBPME_ERR_CUDA,  \
                        "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
    } while (0)

#define IBP_CUFFT(call)                                                                           \
    do {                                                                                          \
        cufftResult r_ = (call);                                                                  \
        if (r_ != CUFFT_SUCCESS)                                                                  \
            ::ibp::fail(IBPME_ERR_CUFFT, "%s:%d %s: cufft error %d", __FILE__, __LINE__, #call, \
                        (int)r_);                                                                 \
    } while (0)

// Every kernel launch of the library is followed by IBP_CHECK_LAUNCH(), which
// also counts it (cuFFT's own launches are not counted).
void count_launch(long long k = 1);
long long launch_count();
#define IBP_CHECK_LAUNCH()                 \
    do {                                   \
        ::ibp::count_launch();             \
        IBP_CUDA(cudaGetLastError());      \
    } while (0)

// ---------------------------------------------------------------------------
// Device buffer that only grows.
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void* ensure(size_t b) {
        if (b > bytes) {
            release();
            size_t want = b < 256 ? 256 : b;
            IBP_CUDA(cudaMalloc(&p, want));
            bytes = want;
        }
        return p;
    }
    // grow to at least b bytes keeping the content (stream-ordered copy); the
    // capacity grows by half at least, so repeated growth copies O(final size)
    void* grow(size_t b, cudaStream_t s) {
        if (b <= bytes) return p;
        if (b < bytes + bytes / 2) b = bytes + bytes / 2;
        void* q = nullptr;
        IBP_CUDA(cudaMalloc(&q, b));
        if (p) {
            IBP_CUDA(cudaMemcpyAsync(q, p, bytes, cudaMemcpyDeviceToDevice, s));
            IBP_CUDA(cudaStreamSynchronize(s));
            cudaFree(p);
        }
        p = q;
        bytes = b;
        return p;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------------------
// Geometry of the spectral-Ewald mesh (Sec. III.D.2), passed to kernels by value.
// ---------------------------------------------------------------------------
struct MeshGeom {
    double L[3];       // box
    double h[3];       // L_d / N_d
    double inv_h[3];
    double kappa[3];   // 2 xi^2 h_d^2 / eta: Gaussian exponent in grid units
    double c;          // (2 xi^2 / (pi eta))^{3/2}: spreading normalisation
    double gather;     // c * h_x h_y h_z / eps_f: trapezoid weight of the gather
    double grad;       // gather * 4 xi^2 / eta: prefactor of the gradient gather
    int N[3];
    int P;
    long long G;       // N_x N_y N_z real grid points
    long long Gc;      // N_z N_y (N_x/2+1) complex points of the half spectrum
};

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = cufftComplex; };
template <> struct Cplx<double> { using type = cufftDoubleComplex; };

constexpr int kMaxRhs = 8;
constexpr int kMaxP = 32;

// Stencils cached for a set of positions: each bead's first stencil node per
// axis (and its configuration) and fractional offset (first node - x / h).
// Built once per set of positions and shared by every spread and gather of a
// solve in either precision.
struct StencilCache {
    bool valid = false;
    unsigned long long fp = 0;   // position fingerprint the cache belongs to
    int n = 0, ncfg = 0;
    unsigned long long cls_key = 0;   // radius-class binding the channels belong to (0: none)
    DevBuf start;                // int4 per bead: first node (x, y, z), configuration
    DevBuf frac;                 // double4 per bead: (first node - x / h) per axis
    DevBuf frac32;               // float4 per bead: the same offsets in FP32 (FP32 kernels)
    DevBuf w64;                  // FP64 window weights [n][3][P] (GB300's FP64 exp is slow: once per positions)
    DevBuf wdf;                  // the same windows as hi + lo floats [n][3][P] (double-float gathers)
    DevBuf frac_df;              // float4 pairs per bead: the offsets of frac as hi + lo floats
    // Tile bins for spreading and gathering through shared memory (many beads
    // only): beads sorted by (configuration, tile of kTileNodes^3 nodes holding
    // their first stencil node).
    bool tiles = false;
    int tile_n[3] = {0, 0, 0};   // tiles per axis
    DevBuf tile_count, tile_cursor, tile_off, tile_tmp, tile_bkey;
    DevBuf tile_sorted;          // int per sorted position: bead
    DevBuf tile_key;             // int per sorted position: configuration * tiles + tile
};

constexpr int kTileNodes = 8;    // tile edge in grid nodes

// Spectral-Ewald mesh engine in one precision: grids, spectrum, Green's table, plans.
// A grid "channel" holds one right-hand side of one configuration: channel
// cfg * nrhs + r (a single system is configuration 0).  With beads of unequal
// radii the channels group the beads by radius class instead (channel
// class * nrhs + r) and the scaling combines them (see transform).
template <typename T>
struct Mesh {
    MeshGeom g{};
    int rcap = 0;   // channels the buffers hold
    DevBuf grid;    // [rcap][G] real
    DevBuf spec;    // [rcap][Gc] complex
    DevBuf green;   // [Gc] real: G(k) / (N_x N_y N_z), 0 at k = 0 (without j0^2 with radius classes)
    int ncls = 1;   // radius classes (1: one radius, its j0^2 inside green)
    DevBuf jtab;    // [ncls][Gc] real: j0(k a_c) of each class
    DevBuf work;    // cuFFT work area shared by the plans
    std::map<int, std::pair<cufftHandle, cufftHandle>> plan;   // R2C and C2R plans by channel count
    // FP64 meshes of power-of-two sizes: double-float transforms instead of cuFFT (dffft.cu)
    bool df = false;
    DevBuf df_tw[3], df_buf;
    DevBuf green_df;   // the Green's table as (hi, lo) float pairs for the double-float transforms
    DevBuf jtab_df;    // [ncls][Gc] j0(k a_c) as (hi, lo) float pairs (radius classes)
    DevBuf grid_df;    // [rcap][G] (hi, lo) floats: the transformed grid of the double-float transforms
    bool potential_df = false;   // the last transform left the potential in grid_df (gathers read it)
    unsigned long long writes = 0;   // spreads into grid so far (a kept grid is intact while this holds)
    // tensor map (CUtensorMap bytes) of the grid the tiled gathers stage their regions
    // from with cp.async.bulk.tensor, for the buffer, channel count and element size below
    alignas(64) unsigned char tmap[128] = {};
    const void* tm_base = nullptr;
    int tm_ch = 0, tm_es = 0, tm_E = 0;
    bool tm_ok = false;
    int* tma_err_host = nullptr;   // mapped host flag: a bounded wait for a tensor copy ran out
    int* tma_err_dev = nullptr;
    int tma_failed();              // read and clear the flag (after a synchronisation): 0, or its code
    // ncls > 1: radius classes of radii cls_a[0 .. ncls) (no double-float transforms then)
    void init(const MeshGeom& geom, int channels, double xi, double eta, double a, cudaStream_t s, int ncls = 1,
              const double* cls_a = nullptr);
    void destroy();
    void ensure_channels(int ch);
    void plans(int ch, cudaStream_t s);   // every resource a transform of ch channels needs
    // bead_cfg (device, or NULL for one configuration) maps each bead to its configuration
    // sc: cached stencils of these positions, or NULL to derive them in the kernels
    // accumulate: add to the grid as it is instead of zeroing it first
    void spread(int n, const double* xw, const double* q, int nrhs, const int* bead_cfg, int ncfg, cudaStream_t s,
                const StencilCache* sc = nullptr, bool accumulate = false);
    // R2C, scale, C2R over ch channels; the double-float transforms leave grid as it was.
    // With radius classes the ch channels are ncls groups of ch / ncls right-hand sides and
    // the scaling sets channel (d, r) to G(k) j0(k a_d) sum_c j0(k a_c) channel (c, r)
    void transform(int ch, cudaStream_t s);
    void gather(int n, const double* xw, int nrhs, const int* bead_cfg, double* psi, double* E, cudaStream_t s,
                const StencilCache* sc = nullptr);
    // The RPY mobility's wave space on three force channels (one system): R2C, then every
    // k takes fac (1 + k^2/(4 xi^2)) G(k) (I - k_hat k_hat) of the three transforms, C2R
    void transform_rpy(double fac, double xi, cudaStream_t s);
};

// Scaling of the RPY wave space (Hasimoto's weight and the transverse projection).
struct RpyScale {
    double L[3];
    double xi, fac;
};

// Cell list and real-space pair table (Sec. III.D.1, Sec. III.D.3 step 1).
struct NearList {
    int n = 0;
    long long npairs = 0;
    int nc[3] = {1, 1, 1};
    double L[3] = {0, 0, 0};
    double rc = 0;
    bool have_grad = false;
    DevBuf cell_of, cell_count, cell_start64, cell_start, cursor;
    DevBuf cell_beads;             // beads sorted by cell: row t of the pair table is bead cell_beads[t]
    DevBuf row_count, rowptr;
    // the count pass also keeps each row's first ell_cap columns (rows padded to ell_cap,
    // sized from the previous build's longest row); when no row is longer, the table
    // is a copy of them and the second search pass is skipped
    DevBuf ell, row_max;
    int ell_cap = 0;
    DevBuf prow;                   // row (sorted position) of every pair
    DevBuf col, val, gfac;
    DevBuf pair32;                 // (col, FP32 val) per pair: inner operator of mixed-precision solves
    DevBuf qf;                     // charges packed per bead (float4) for the FP32 pass
    DevBuf qs;                     // charges [n][nrhs] in the sorted order for the FP64 pass
    DevBuf scan_tmp, flag;
    DevBuf xf;                     // FP32 positions (x, y, z, 0) for the candidate filter
    DevBuf xdf;                    // positions as hi, lo float4 pairs per bead (double-float pair values)
    DevBuf ov_list;                // pairs of overlapping beads (r < 2a), valued exactly in FP64
    DevBuf ov_count;
    bool ov_valid = false;         // ov_list holds every overlapping pair of the current table
    DevBuf table;                  // tabulated pair kernel (phi, phi', phi'') on [2a, r_c]
    DevBuf fp_dev;                 // fingerprint of the positions + non-finite flag
    unsigned long long fp = 0;     // fingerprint of the positions the table was built for
    bool fp_valid = false;
    // fingerprint already fetched by the entry point (with the body-structure hash, one
    // synchronisation for both), consumed by the next near_build for these positions
    bool fp_pre_valid = false;
    unsigned long long fp_pre[2] = {0, 0};
    int fp_pre_n = -1;
    const double* fp_pre_xw = nullptr;
    int ncfg = 1;
    unsigned long long cls_key = 0;   // radius-class binding of the pair values (0: none)
    DevBuf self_b;                 // [n] self term of each bead's radius class (radius classes only)
    DevBuf cls_table, cls_tab32, cls_tabdf;   // radius classes: the tables of every pair of classes
    int cls_K = 0;                 // their octaves (0: no tables, every pair takes the exact kernel)
    // Compact bodies: multi-bead bodies within min(r_c, L/4) of their centre.
    // Their intra-body pairs are left out of the table and evaluated directly
    // by the compact kernels (FP32 for the inner operator, double-float for the
    // FP64 operator and the field).
    bool cb_on = false;            // the table was built with compact bodies taken out
    unsigned long long cb_key = 0; // body structure the compact data belong to (0: none)
    DevBuf cb_flag;                // [nb] 1 if the body is compact
    DevBuf cb_hi, cb_lo;           // [n] float4: position relative to the body's first bead, hi + lo parts
    DevBuf cb_tasks;               // int4 per block: (body, first target, first source, counts)
    std::vector<int4> cb_tasks_h;  // host copy of the tasks
    int cb_ntasks = 0;
    unsigned long long cb_tasks_key = 0;
    DevBuf tab32;                  // [nt] float4: FP32 cubic coefficients of phi per interval
    DevBuf tab_df;                 // [nt][3] float4: double-float phi and phi' coefficients
};

// Body bookkeeping on the device for solves, forces and BD steps.
// Unknowns of the reduced saddle system (krylov.cu), configuration by
// configuration: the configuration's free beads (beads of multi-bead bodies,
// in bead order), then its multi-bead bodies (one body potential each).
struct BodyData {
    int nb = 0;         // bodies
    int nmb = 0;        // multi-bead bodies
    int nfree = 0;      // beads of multi-bead bodies (the unknown charges)
    int nk = 0;         // unknowns (nfree + nmb)
    int ncfg = 1;       // configurations
    DevBuf off;         // [nb+1] int body offsets
    DevBuf bead_body;   // [n] body of each bead
    DevBuf X, Q;        // [nb][3], [nb]
    DevBuf free_idx;    // [nfree] bead of each free bead
    DevBuf free_unk;    // [nfree] unknown index of each free bead
    DevBuf mb_body;     // [nmb] body of each multi-bead body
    DevBuf mb_unk;      // [nmb] unknown index of its potential
    DevBuf mb_first;    // [nmb] unknown index of its first bead (its beads' unknowns are contiguous)
    DevBuf mb_cnt;      // [nmb] its bead count
    DevBuf bead_unk;    // [n] unknown index of a bead's charge, -1 for ions
    DevBuf body_unk;    // [nb] unknown index of a body's potential, -1 for ions
    DevBuf unk_cfg;     // [nk] configuration of each unknown
    DevBuf bead_cfg;    // [n] configuration of each bead
    DevBuf uo;          // [ncfg+1] unknown offsets of the configurations
    DevBuf cfg_beads;   // [ncfg+1] bead offsets of the configurations
    DevBuf cfg_bodies;  // [ncfg+1] body offsets of the configurations
    DevBuf rel;         // [n][3] r_ij = minimum image of x_ij - X_i
    DevBuf scratch;     // reductions and BD temporaries
    DevBuf free_pos;    // [n] position of a bead in the free-bead list, -1 for ions
    DevBuf free_cfg;    // [nfree] configuration of each free bead
    DevBuf iota;        // [nfree] 0, 1, ..., nfree - 1 (identity order of the free-bead list)
    std::vector<int> free_pos_h;   // host copy of free_pos
    std::vector<int> uo_h, cfg_beads_h, cfg_bodies_h;
    std::vector<int> host_off, host_cfg;   // structure of the last upload (to skip rebuilding the lists)
    int host_n = -1;
    int max_beads = 0;                     // beads of the largest body of the last upload
    unsigned long long version = 0;        // changes whenever the body structure changes
    unsigned long long off_hash = 0;       // hash of the offsets of the last upload (0: unknown)
};

struct Krylov;   // krylov.cu

// The free beads (beads of multi-bead bodies) on their own.  A Krylov vector
// carries charges on these beads only (ion charges are fixed and eliminated) and
// only their potentials enter the reduced saddle operator, so the operator of
// the Krylov iterations evaluates sources and targets of this list alone: the
// mesh pass spreads and gathers the free beads through their own stencil cache,
// the real-space pass takes the table's pairs between two free beads (re-indexed
// into the list) and the compact bodies' pairs.  Everything is indexed by the
// position f in the list (bodies.free_idx[f] is the bead).
struct FreeSet {
    bool valid = false;
    unsigned long long fp = 0;        // position fingerprint the data belong to
    unsigned long long version = 0;   // body structure they belong to
    int nfree = 0;
    DevBuf xf;                        // [nfree][3] wrapped positions
    StencilCache sc;                  // their stencils (and tile bins)
    DevBuf sorted_of;                 // [n] pair-table row (cell-sorted position) of each bead
    long long npairs = 0;             // pairs between two free beads outside the compact bodies
    DevBuf row_count, rowptr, col, val, pair32, scan_tmp;   // that table in list indices
    DevBuf qf, qs;                    // packed charges of its FP32 and FP64 passes
    DevBuf cb_hi, cb_lo;              // [nfree] compact-body relative positions in list order
    DevBuf cb_tasks;                  // compact-body tasks in list indices
    int cb_ntasks = 0;
    unsigned long long cb_tasks_key = 0;
    DevBuf psi_r, psi_k, qsum;        // [R][nfree] partial potentials, [channels] charge sums
    DevBuf cls_f, self_f;             // radius classes: class and self term of each free bead
    unsigned long long cls_key = 0;   // the binding they belong to
};

// Body-block preconditioner (precond.cu): inverses of the bodies' free-space
// saddle blocks, cached per body shape for the life of the context.
constexpr int kPrecondMaxBeads = 8192;                      // larger bodies are left unpreconditioned
constexpr long long kPrecondCacheBytes = 24LL << 30;        // FP32 inverses kept at most
struct Precond {
    struct Shape {
        int nb;
        double m2, m4;        // rotation-invariant moments of the bead cloud
        unsigned long long ckey;   // hash of the beads' radius classes in bead order (0: one radius)
        long long off, goff;  // element offsets of M^{-1} and of g in minv / gvec
    };
    std::vector<Shape> shapes;
    long long used = 0, gused = 0;
    DevBuf minv, gvec, sinv, shape_off, shape_goff;   // per shape
    DevBuf pb_shape, pb_first, pb_psi, pb_n, plain;   // per solve: preconditioned bodies, identity unknowns
    DevBuf moments, gj_d, gj_c, gj_r, gj_bad;          // set-up scratch (blocked Gauss-Jordan)
    int npb = 0, nplain = 0, chunks = 0, maxn = 0;
    // steady state: the body structure the tables were laid out for, the shape of
    // every multi-bead body (-1: identity), and the moments of the last positions
    // (copied asynchronously into pinned memory, checked at the next solve)
    unsigned long long prep_version = 0;
    unsigned long long prep_cls = 0;        // radius-class binding of that preparation
    bool prep_valid = false;
    std::vector<int> assign;
    double* hm_pin = nullptr;
    size_t hm_cap = 0;
};

// Optional per-stage timing with CUDA events on the launching stream.
enum Stage {
    ST_NEAR_BUILD = 0,   // cell list + pair table
    ST_NEAR_APPLY,       // real-space SpMV / field
    ST_SPREAD,           // FP32 mesh: spread (grid clear + atomics)
    ST_FFT_FWD,          //            cuFFT R2C
    ST_SCALE,            //            Green's-function scaling
    ST_FFT_INV,          //            cuFFT C2R
    ST_GATHER,           //            gather
    ST_KRYLOV,           // Arnoldi / Givens / update kernels of one iteration
    ST_BODIES,           // body reductions and the BD step
    ST_SPREAD64,         // FP64 mesh: the same five stages
    ST_FFT_FWD64,
    ST_SCALE64,
    ST_FFT_INV64,
    ST_GATHER64,
    ST_NEAR_APPLY32,     // real-space SpMV, FP32 pass (inner operator of mixed solves)
    ST_NEAR_FIELD,       // real-space field (force pass)
    ST_RPY_NEAR,         // real-space share of the RPY mobility
    ST_COUNT
};
// stage of a mesh step for the mesh precision T
template <typename T>
constexpr int mesh_stage(int st32) { return sizeof(T) == 8 ? st32 - ST_SPREAD + ST_SPREAD64 : st32; }
struct ProfScope {
    int stage;
    cudaStream_t s;
    bool on;
    ProfScope(int stage, cudaStream_t s);
    ~ProfScope();
};
unsigned prof_mask();
// Scopes opened between begin and end are being captured into CUDA graph `gid`:
// their events become graph nodes, re-recorded by every replay, and
// prof_graph_collect(gid) adds the last replay's times (call it after a sync).
void prof_capture_begin(int gid);
void prof_capture_end();
void prof_graph_collect(int gid);

}  // namespace ibp

// The context (opaque in the C ABI).
struct ibpme_ctx {
    ibpme_params p{};              // resolved parameters
    int device = 0;
    cudaStream_t stream = nullptr;
    double xi = 0, eta = 0, rc = 0, a = 0, eps = 1;
    int P = 0;
    ibp::MeshGeom geom{};
    ibp::Mesh<double> mesh64;
    ibp::Mesh<float> mesh32;
    bool have32 = false;
    ibp::NearList near;
    ibp::BodyData bodies;
    ibp::Krylov* kry = nullptr;
    // working vectors
    ibp::DevBuf xw;          // [n][3] wrapped positions
    ibp::DevBuf psi_r, psi_k, E_r, E_k;   // [R][n], [R][n][3]
    ibp::DevBuf qfull;       // [R][n]
    // staging of host arrays
    ibp::DevBuf st_x, st_q, st_out1, st_out2, st_out3, st_out4, st_out5, st_out6, st_out7, st_out8, st_E0, st_off, st_X,
        st_Q, st_f;
    ibp::DevBuf scalars;     // small device scratch
    void* pinned = nullptr;  // small pinned host scratch
    size_t pinned_bytes = 0;
    cudaStream_t work = nullptr;              // the context's own stream (solves, graph capture)
    // batch of independent configurations (1 and NULL outside a batched call):
    // bead b belongs to configuration bcfg[b]
    int ncfg = 1;
    const int* bcfg = nullptr;
    bool bodies_current = false;   // the uploaded bodies belong to the running call
    // mixed solves whose first residual takes the FP64 operator after an FP32-mesh start
    // missed the tolerance at the first FP64 check (counts down once per solve)
    int start32_skip = 0;
    // the FP64 mesh grid and the Krylov potentials hold the last solve's final FP64
    // residual evaluation (the field of the solution charges can be gathered from it)
    bool grid64_final = false;
    // E_k holds the mesh field of that evaluation at every bead (gathered with its potential),
    // E_r its real-space field
    bool field64_ready = false;
    bool near_field_ready = false;
    ibp::DevBuf ml_feat, ml_scratch, ml_scales, ml_y, ml_part;   // learned warm start
    ibp::DevBuf ml_g, ml_gprev;               // [nrhs][n] learned guesses of this and of the last call
    unsigned long long ml_prev_version = 0;   // body structure, bead and field count of ml_gprev
    int ml_prev_n = -1, ml_prev_R = 0;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ibp::StencilCache stencils;               // stencils of the current positions
    ibp::FreeSet fs;                          // the free beads on their own (Krylov operator)
    ibp::DevBuf cap_psi, cap_q, cap_zero;     // grand capacitance: bead potentials, charges, zeros
    // beads of unequal radii: ncls classes of radii cls_a (ncls = 1: every bead has radius a);
    // cls [cls_n] binds a class to each bead of the calls with cls_n beads
    int ncls = 1;
    double cls_a[IBPME_MAX_RADIUS_CLASSES] = {};
    int cls_n = -1;
    ibp::DevBuf cls;
    std::vector<int> cls_h;
    unsigned long long cls_version = 0;       // bumped by every binding (cache keys; 0: none)
    // RPY mobility: real-space radial table (A, B at mu = 1) for (a, xi, r_c) of rpy_key
    ibp::DevBuf rpy_tab, rpy_tab32, rpy_F, rpy_F4, rpy_Uk;
    ibp::DevBuf rig_V, rig_w, rig_b, rig_x, rig_dot, rig_FL;   // rigid-body mobility GMRES
    ibp::DevBuf rig_z, rig_u, rig_t, rig_minv, rig_G, rig_Sinv, rig_pb, rig_moff, rig_goff, rig_idx;   // and its
    int rig_nmb = 0, rig_maxn = 0;   // body-block preconditioner
    double rpy_key[3] = {0.0, 0.0, 0.0};
    double rpy_h = 0.0, rpy_self = 0.0;
    int rpy_nodes = 0;
    ibp::Precond pre;                         // body-block preconditioner
    cudaStream_t aux = nullptr;               // second branch of a PME evaluation (near field)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace ibp {

// The mesh channel group of each bead (device, or NULL for one group) and the number of
// groups: the radius classes with beads of unequal radii, else the configurations.
inline const int* mesh_cfg(const ibpme_ctx* c) {
    return c->ncls > 1 ? static_cast<const int*>(c->cls.p) : c->bcfg;
}
inline int mesh_groups(const ibpme_ctx* c) { return c->ncls > 1 ? c->ncls : c->ncfg; }
// The binding key of the radius classes (0 with one radius).
inline unsigned long long cls_key(const ibpme_ctx* c) { return c->ncls > 1 ? c->cls_version : 0; }

// ---- near.cu ----
// exclusive scan of n int counts into n + 1 int64 offsets (out[n] = total)
void scan_counts(const int* in, long long* out, int n, DevBuf& tmp, cudaStream_t s);
void near_setup(ibpme_ctx* c);   // tabulates the pair kernel (once per context)
void near_build(ibpme_ctx* c, int n, const double* xw, bool need_grad);
// Position fingerprint of xw and a hash of the noff body offsets (device), fetched with one
// synchronisation; the fingerprint is kept for the next near_build of these positions.
// Returns the offsets hash.
unsigned long long near_prefetch(ibpme_ctx* c, int n, const double* xw, const int* off, int noff);
// overwrite; fp32: FP32 pair values and charges (the mixed solve's inner operator)
void near_apply(ibpme_ctx* c, int n, const double* q, int nrhs, double* psi_r, bool fp32 = false);
void near_field(ibpme_ctx* c, int n, const double* xw, const double* q, int nrhs, double* E_r);  // overwrite
double self_term(const ibpme_ctx* c);   // phi_self (without 1/eps)

// The free-bead data of the current positions and body structure (call after
// near_build, outside any stream capture): positions, stencils, the free-free pair
// table and the compact-body tasks in list indices.  False when the free-bead
// operator cannot be used (no free beads, or the table was built without bodies).
bool near_free_build(ibpme_ctx* c, const double* xw);
// psi_r [nrhs][nfree] = real-space potential at the free beads of the charges qc
// [nrhs][nfree] on the free beads (self term, free-free table, compact bodies)
void near_apply_free(ibpme_ctx* c, const double* qc, int nrhs, double* psi_r, bool fp32);

// ---- dffft.cu ----
bool df_fft_supported(const MeshGeom& g);
void df_fft_init(const MeshGeom& g, DevBuf tw[3], cudaStream_t s);
// ncls > 1: radius classes, the channels mixed by j0(k a_c) j0(k a_d) (jtab [ncls][Gc] hi + lo)
// rpy != NULL: three force channels scaled as in Mesh::transform_rpy
void df_fft_convolve(const MeshGeom& g, int ch, const float2* green, const double* grid, float2* out, float4* S,
                     DevBuf tw[3], cudaStream_t s, int ncls = 1, const float2* jtab = nullptr,
                     const RpyScale* rpy = nullptr);

// ---- rpy.cu ----
// U [n][3] = periodic RPY mobility (viscosity mu) times F [n][3] at the wrapped positions xw
void rpy_apply(ibpme_ctx* c, int n, const double* xw, const double* F, double mu, double* U);
// Rigid-body mobility problem on the uploaded bodies: FL [nb][6] (F, L) -> W_out [nb][6] (U, Omega),
// f_out [n][3] (or NULL) bead constraint forces; restarted GMRES(m) to rtol (IBPME_ERR_NOT_CONVERGED
// past max_iter iterations, outputs hold the last iterate); all pointers device
void rigid_solve(ibpme_ctx* c, int n, const double* xw, const double* FL, double mu, double rtol, int m,
                 int max_iter, double* W_out, double* f_out, ibpme_solve_stats* st, bool precond = true);
// ---- precond.cu ----
// A (nb x nb, FP32, symmetric positive definite) -> A^{-1} in place (blocked Gauss-Jordan)
void invert_spd(ibpme_ctx* c, int nb, float* A);

// ---- mesh.cu ----
// Cached stencils for the current positions (rebuilt when the position
// fingerprint of the last near_build changed), or NULL without a fingerprint.
const StencilCache* stencil_cache(ibpme_ctx* c, int n, const double* xw);
// Stencils of the free beads (c->fs.xf), keyed like stencil_cache.
const StencilCache* free_stencil_cache(ibpme_ctx* c);

// ---- api.cu helpers ----
void resolve_params(const ibpme_params* in, ibpme_params* out);   // rules of Sec. III.D.2; throws on bad input
MeshGeom make_geom(const ibpme_params& p);
void wrap_positions(ibpme_ctx* c, int n, const double* x, double* xw);
// psi = M q (real + self + wave) in the given precision; E optional
// near32: real-space pass in FP32 too (only the inner operator of a mixed solve)
// every buffer pme_apply needs for n beads and nrhs fields (before a stream capture)
void pme_reserve(ibpme_ctx* c, int n, int nrhs, bool field);
// IBPME_ERR_TIMEOUT if a tiled gather's bounded wait for its tensor copies ran out
// since the last check (read after the gather's stream has synchronised)
void tma_check(ibpme_ctx* c);
// The FP64 mesh pass on the free beads only (nf beads at xf, bead free_idx[f] of the
// full list, configuration cfg[f] or NULL for one, stencils sc):
//   dq != NULL: add the charges dq [nrhs][nf] to a grid that still holds an earlier
//               spread (the caller guarantees it holds the spread of q - dq);
//   tmp != NULL: gather the mesh potential at the free beads only (through tmp
//               [nrhs][nf]); the other beads' results are then not written.
struct FreeMesh {
    int nf;
    const double* xf;
    const int* free_idx;
    const int* cfg;
    const StencilCache* sc;
    const double* dq;
    double* tmp;
    double* ek = nullptr;   // also gather the mesh field at every bead into ek [nrhs][n][3]
    double* er = nullptr;   // and the real-space field into er (on the second stream, beside the mesh)
};
// With fm (FP64 only) the mesh pass takes the free-bead forms above; the real-space
// pass and the k = 0 term still take q on every bead.
void pme_apply(ibpme_ctx* c, int n, const double* xw, const double* q, int nrhs, int prec,
               double* psi, double* E, bool near_ready, bool near32 = false, const FreeMesh* fm = nullptr);
// Prepare the free-bead operator for the positions xw of the last near_build and nrhs
// fields (after near_build, before any capture); false if it cannot serve this call.
bool free_prepare(ibpme_ctx* c, const double* xw, int nrhs);
// psi_f = M q restricted to the free beads: charges qc [nrhs][nfree] on the free beads
// (every other charge zero), potentials psi_f [nrhs][nfree] at the free beads.
void pme_apply_free(ibpme_ctx* c, const double* qc, int nrhs, int prec, double* psi_f, bool near32);
void* pinned_host(ibpme_ctx* c, size_t bytes);

// ---- bodies.cu ----
// cfg_beads / cfg_bodies: host [ncfg+1] offsets of the configurations (NULL for one)
// off_hash: hash of the body offsets from near_prefetch, or NULL (read the offsets back)
void bodies_upload(ibpme_ctx* c, int n, const ibpme_bodies* b, const double* xw, int ncfg = 1,
                   const int* cfg_beads = nullptr, const int* cfg_bodies = nullptr,
                   const unsigned long long* off_hash = nullptr);
void body_dipoles(ibpme_ctx* c, int n, const double* q, int nrhs, double* S);
void bead_forces(ibpme_ctx* c, int n, const double* q, const double* E0, const double* E, double* f);
void body_reduce_force_torque(ibpme_ctx* c, int n, const double* f, double* F, double* L);
void body_energy(ibpme_ctx* c, int n, const double* q, const double* psi, const double* E0, double* U);
void bd_step(ibpme_ctx* c, int n, const double* x, const double* f, const ibpme_bd_params* bd,
             double* x_out, double* X_out);

// ---- mlp.cu ----
void compute_features(ibpme_ctx* c, int n, const double* xw, const double* E0, int nrhs, float* feat,
                      DevBuf& scratch, DevBuf& scales);
void learned_guess(ibpme_ctx* c, const ibpme_mlp* mlp, int n, const double* xw, const double* E0, int nrhs,
                   double* q, bool step);
// IBPME_ERR_TIMEOUT if the tensor-core pass of the last learned_guess gave up waiting
// (call after a synchronisation of the stream that ran it).
void learned_check(const ibpme_mlp* mlp);

// ---- krylov.cu ----
struct SolveArgs {
    int n, nrhs, prec;
    const double* xw;
    const double* E0;   // device [nrhs][3]
    double* q;          // device [nrhs][n] (guess in, solution out)
    double* psi;        // device [nrhs][nb] or nullptr
    bool user_guess;
    bool learned;       // the guess came from the learned model: fall back to zero if it is worse
    double rtol;
    int restart, max_iter;
    bool precond;       // body-block right preconditioner
    // Prescribed bead potentials [nrhs][n] (device), or NULL for Eq. saddle.  Given,
    // the solve finds the charges of M q = bead_psi instead: the body potentials are
    // no unknowns (their rows become the identity with zero right-hand side), every
    // body must have two beads or more, and E0, Q and psi are not used.
    const double* bead_psi = nullptr;
    // The caller needs the field of the solution next (the BD step): the FP64 residuals
    // after the first also gather the mesh field into the context (one field, one
    // configuration), so that the force pass does not gather the mesh again.
    bool want_field = false;
};
void solve(ibpme_ctx* c, const SolveArgs& a, ibpme_solve_stats* st);
// FP64 potentials [nrhs][n] of the last solve's final residual evaluation (its FP64
// mesh grid still holds the same charges), or NULL when that evaluation was skipped
const double* solve_potentials(ibpme_ctx* c);
// precond.cu
bool precond_prepare(ibpme_ctx* c);   // false: no body qualifies
// dir: the block [-M_b 0; 0 1] of the prescribed-potential problem (SolveArgs::bead_psi)
void precond_apply(ibpme_ctx* c, int R, const double* u, long long ustride, const int* jdev, int nk, double* out,
                   bool dir = false);
void krylov_destroy(ibpme_ctx* c);

// small device helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__host__ __device__ __forceinline__ double wrap_coord(double x, double L) {
    double w = x - L * floor(x / L);
    return (w >= L) ? w - L : w;   // guard x/L rounding to exactly 1
}

__host__ __device__ __forceinline__ double min_image(double d, double L) {
    return d - L * floor(d / L + 0.5);
}

// Minimum image of a difference of two wrapped coordinates (both in [0, L)):
// d lies in (-L, L), so one conditional shift suffices (no division).
template <typename T>
__host__ __device__ __forceinline__ T min_image_wrapped(T d, T L) {
    return d > T(0.5) * L ? d - L : (d < T(-0.5) * L ? d + L : d);
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace ibp
