// mlp.cu -- learned warm start for the induced-charge solve (not in the paper).
//
// A small fully connected network maps per-bead features (the local field
// driving the induced charge, the bead's place on its body, the body's net
// charge and size) to a first guess of the induced bead charge.  Everything
// runs in this file's kernels: feature extraction, inference, and training
// (forward, backward and Adam).  Architecture (fixed): IN -> 64 -> 64 -> 1 with
// tanh hidden units; FP32 weights and arithmetic.
//
// Layout of the flat parameter vector: W1[H][IN], b1[H], W2[H][H], b2[H],
// W3[H], b3 (row-major, out x in).
#include "common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

struct ibpme_mlp {
    int device = 0;
    ibp::DevBuf params, grad, m1, m2, perm, loss;
    ibp::DevBuf tc_err;   // set by the tensor-core forward if its mbarrier wait ran out
    int* tc_err_host = nullptr;   // pinned copy of tc_err
    long long step = 0;
};

namespace ibp {

namespace {

constexpr int IN = IBPME_MLP_IN;
constexpr int H = IBPME_MLP_HIDDEN;
constexpr int NP = IBPME_MLP_NPARAM;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H;
static_assert(OFF_B3 + 1 == NP, "parameter layout");
constexpr int TILE = 128;   // samples per block in the training kernel
constexpr int HS = H + 1;   // padded row stride of the hidden activations (no bank conflicts)

// ---- inference: one thread per sample, weights broadcast from shared memory ----
__global__ void __launch_bounds__(128) mlp_forward_kernel(int n, const float* __restrict__ P,
                                                          const float* __restrict__ X, float* __restrict__ Y) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[IN];
#pragma unroll
    for (int f = 0; f < IN; ++f) x[f] = X[(size_t)s * IN + f];
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) {
        float a = w[OFF_B1 + o];
#pragma unroll
        for (int f = 0; f < IN; ++f) a += w[OFF_W1 + o * IN + f] * x[f];
        h1[o] = tanhf(a);
    }
    float y = w[OFF_B3];
    for (int o = 0; o < H; ++o) {
        float a = w[OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < H; ++i) a += w[OFF_W2 + o * H + i] * h1[i];
        y += w[OFF_W3 + o] * tanhf(a);
    }
    Y[s] = y;
}

// ---- inference on the 5th-generation tensor cores (tcgen05) ----
// One CTA of 128 threads takes 128 samples.  Layer 1 (IN -> H) runs on the
// CUDA cores, one sample per thread, and writes tanh(h1) as BF16 into shared
// memory in the tensor cores' K-major layout without swizzle: 8 x 8 core
// matrices of 8 rows x 16 bytes, byte offset of element (row, k) =
// ((row / 8) * (H / 8) + k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2, so
// adjacent core matrices along K are 128 B apart and along the rows
// (H / 8) * 128 B apart.  W2 (H x H, out x in) is staged the same way.  One
// elected thread issues four tcgen05.mma (M = 128, N = H, K = 16 each, BF16
// inputs, FP32 accumulator in tensor memory), commits them to an mbarrier,
// and every warp then reads its 32 rows of the accumulator with tcgen05.ld;
// layer 2's bias and tanh and layer 3 finish on the CUDA cores in FP32.
namespace tc {

constexpr int kRows = 128;                    // M: samples per CTA (one TMEM lane each)
constexpr int kABytes = kRows * H * 2;        // BF16 activations
constexpr int kBBytes = H * H * 2;            // BF16 W2
constexpr int kCoreBytes = 128;               // one 8 x 16-byte core matrix
constexpr uint32_t kLbo = kCoreBytes;         // next core matrix along K
constexpr uint32_t kSbo = (H / 8) * kCoreBytes;   // next group of 8 rows
constexpr int kTmemCols = H;                  // FP32 accumulator columns (a power of two >= 32)
constexpr int kWaitLimit = 1 << 22;           // bounded mbarrier polling (about 0.4 s with back-off)
constexpr size_t kSmem = 1024 + kABytes + kBBytes + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05: start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A and
// B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t core_offset(int row, int k) {
    return (uint32_t)(((row >> 3) * (H / 8) + (k >> 3)) * kCoreBytes + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (int it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(100);
    }
    return false;
}

__global__ void __launch_bounds__(kRows) mlp_forward_tc_kernel(int n, const float* __restrict__ P,
                                                               const float* __restrict__ X, float* __restrict__ Y,
                                                               int* __restrict__ err) {
    extern __shared__ uint8_t dyn[];
    __shared__ float w1[H * IN], b1[H], b2[H], w3[H];
    __shared__ float b3;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    // 1024-byte aligned operand tiles inside the dynamic buffer
    const uint32_t dyn_base = smem_u32(dyn);
    const uint32_t pad = (1024u - (dyn_base & 1023u)) & 1023u;
    uint8_t* a_tile = dyn + pad;
    uint8_t* b_tile = a_tile + kABytes;
    const uint32_t a_addr = dyn_base + pad, b_addr = a_addr + kABytes;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar_addr = smem_u32(&mbar);

    if (warp == 0) {   // 64 TMEM columns for the accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_addr) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < H * IN; i += kRows) w1[i] = P[OFF_W1 + i];
    for (int i = tid; i < H; i += kRows) {
        b1[i] = P[OFF_B1 + i];
        b2[i] = P[OFF_B2 + i];
        w3[i] = P[OFF_W3 + i];
    }
    if (tid == 0) b3 = P[OFF_B3];
    // W2 -> BF16 core matrices: 8 consecutive inputs of one output per 16-byte store
    for (int c = tid; c < H * (H / 8); c += kRows) {
        const int o = c / (H / 8), kg = c % (H / 8);
        const float* src = P + OFF_W2 + o * H + kg * 8;
        uint4 v;
        v.x = pack_bf16(src[0], src[1]);
        v.y = pack_bf16(src[2], src[3]);
        v.z = pack_bf16(src[4], src[5]);
        v.w = pack_bf16(src[6], src[7]);
        *reinterpret_cast<uint4*>(b_tile + core_offset(o, kg * 8)) = v;
    }
    __syncthreads();
    // layer 1 on the CUDA cores, one sample per thread -> BF16 A tile
    const int s = blockIdx.x * kRows + tid;
    float x[IN];
#pragma unroll
    for (int f = 0; f < IN; ++f) x[f] = s < n ? X[(size_t)s * IN + f] : 0.0f;
#pragma unroll
    for (int kg = 0; kg < H / 8; ++kg) {
        float h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int o = kg * 8 + u;
            float a = b1[o];
#pragma unroll
            for (int f = 0; f < IN; ++f) a += w1[o * IN + f] * x[f];
            h[u] = tanhf(a);
        }
        uint4 v;
        v.x = pack_bf16(h[0], h[1]);
        v.y = pack_bf16(h[2], h[3]);
        v.z = pack_bf16(h[4], h[5]);
        v.w = pack_bf16(h[6], h[7]);
        *reinterpret_cast<uint4*>(a_tile + core_offset(tid, kg * 8)) = v;
    }
    // generic-proxy writes of the tiles -> visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(kRows, H);
#pragma unroll
        for (int kk = 0; kk < H / 16; ++kk) {   // K = 16 per instruction: two core matrices along K
            const uint64_t da = smem_desc(a_addr + kk * 2 * kCoreBytes, kLbo, kSbo);
            const uint64_t db = smem_desc(b_addr + kk * 2 * kCoreBytes, kLbo, kSbo);
            const uint32_t acc = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(da), "l"(db), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_addr)
                     : "memory");
    }
    const bool ok = mbar_wait(mbar_addr, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // this warp's 32 accumulator rows (TMEM lanes 32 warp ..), 16 columns per load
        float y = b3;
        const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += 16) {
            uint32_t r[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(row_addr + (uint32_t)c0)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int u = 0; u < 16; ++u) y += w3[c0 + u] * tanhf(__uint_as_float(r[u]) + b2[c0 + u]);
        }
        if (s < n) Y[s] = y;
    } else if (tid == 0) {
        atomicExch(err, 1);
        mbar_wait(mbar_addr, 0);   // give the tensor cores a second bounded chance to finish
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace tc

// Tensor-core forward pass of n samples; returns IBPME_ERR_TIMEOUT (after the
// kernel has freed its tensor memory) if a wait for the tensor cores ran out.
// IBPME_ERR_TIMEOUT if the last tensor-core forward pass (already complete: the
// caller has synchronised its stream) gave up waiting for the tensor cores.
void forward_tc_check(const ibpme_mlp* m) {
    if (m->tc_err_host && *m->tc_err_host) {
        *m->tc_err_host = 0;
        fail(IBPME_ERR_TIMEOUT, "tensor-core MLP forward: the wait for the tensor cores ran out");
    }
}

// The tensor-core forward pass.  Its bounded waits report through a device flag;
// with check the call synchronises and raises IBPME_ERR_TIMEOUT if it is set,
// without it the flag is left for forward_tc_check (after a later synchronisation).
void forward_tc(const ibpme_mlp* m, int n, const float* feat, float* out, cudaStream_t s, bool check = true) {
    if (n <= 0) return;
    ibpme_mlp* mm = const_cast<ibpme_mlp*>(m);
    int* err = static_cast<int*>(mm->tc_err.ensure(sizeof(int)));
    IBP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    IBP_CUDA(cudaFuncSetAttribute(tc::mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc::kSmem));
    tc::mlp_forward_tc_kernel<<<div_up(n, tc::kRows), tc::kRows, tc::kSmem, s>>>(n, m->params.as<float>(), feat,
                                                                                    out, err);
    IBP_CHECK_LAUNCH();
    if (!mm->tc_err_host) {
        IBP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&mm->tc_err_host), sizeof(int), cudaHostAllocDefault));
        *mm->tc_err_host = 0;
    }
    IBP_CUDA(cudaMemcpyAsync(mm->tc_err_host, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (check) {
        IBP_CUDA(cudaStreamSynchronize(s));
        forward_tc_check(m);
    }
}

// ---- gradient of the mean squared error over a batch ----
// Block of TILE threads owns TILE samples (rows idx[base .. base + TILE) of X
// through the permutation, or rows base.. when idx is NULL).  Forward pass
// kept in shared memory, then the backward pass as small products over the
// tile's samples; the block's gradient is added to G.
__global__ void __launch_bounds__(TILE) mlp_grad_kernel(int n, int base, int count, const int* __restrict__ idx,
                                                         const float* __restrict__ P, const float* __restrict__ X,
                                                         const float* __restrict__ T, float inv_batch,
                                                         float* __restrict__ G, float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* w = sm;                       // NP
    float* xs = w + NP;                  // TILE x IN
    float* h1 = xs + TILE * IN;          // TILE x HS (later dH1)
    float* h2 = h1 + TILE * HS;          // TILE x HS (later dH2)
    float* dy = h2 + TILE * HS;          // TILE
    const int tid = threadIdx.x;
    for (int i = tid; i < NP; i += blockDim.x) w[i] = P[i];
    const int first = base + blockIdx.x * TILE;
    const int s = first + tid;
    const bool valid = tid < count - blockIdx.x * TILE && s < n;
    const int row = valid ? (idx ? idx[s] : s) : 0;
    for (int f = 0; f < IN; ++f) xs[tid * IN + f] = valid ? X[(size_t)row * IN + f] : 0.f;
    __syncthreads();
    // forward
    for (int o = 0; o < H; ++o) {
        float a = w[OFF_B1 + o];
        for (int f = 0; f < IN; ++f) a += w[OFF_W1 + o * IN + f] * xs[tid * IN + f];
        h1[tid * HS + o] = tanhf(a);
    }
    float y = w[OFF_B3];
    for (int o = 0; o < H; ++o) {
        float a = w[OFF_B2 + o];
        for (int i = 0; i < H; ++i) a += w[OFF_W2 + o * H + i] * h1[tid * HS + i];
        const float t = tanhf(a);
        h2[tid * HS + o] = t;
        y += w[OFF_W3 + o] * t;
    }
    const float err = valid ? y - T[row] : 0.f;
    dy[tid] = 2.f * err * inv_batch;
    float l = err * err * inv_batch;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) atomicAdd(loss, l);
    __syncthreads();
    // output layer: dW3[o] = sum_s dy h2[s][o], db3 = sum_s dy
    if (tid < H) {
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += dy[q] * h2[q * HS + tid];
        atomicAdd(G + OFF_W3 + tid, a);
    }
    if (tid == H) {
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += dy[q];
        atomicAdd(G + OFF_B3, a);
    }
    __syncthreads();
    // dH2 = dy W3 (1 - h2^2), in place
    for (int o = 0; o < H; ++o) {
        const float t = h2[tid * HS + o];
        h2[tid * HS + o] = dy[tid] * w[OFF_W3 + o] * (1.f - t * t);
    }
    __syncthreads();
    // dW2[o][i] = sum_s dH2[s][o] h1[s][i]; db2[o] = sum_s dH2[s][o]
    for (int e = tid; e < H * H; e += blockDim.x) {
        const int o = e / H, i = e % H;
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += h2[q * HS + o] * h1[q * HS + i];
        atomicAdd(G + OFF_W2 + e, a);
    }
    if (tid < H) {
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += h2[q * HS + tid];
        atomicAdd(G + OFF_B2 + tid, a);
    }
    // dH1[s][i] = (sum_o W2[o][i] dH2[s][o]) (1 - h1^2): each thread its own sample
    float d1[H];
    for (int i = 0; i < H; ++i) {
        float a = 0.f;
        for (int o = 0; o < H; ++o) a += w[OFF_W2 + o * H + i] * h2[tid * HS + o];
        const float t = h1[tid * HS + i];
        d1[i] = a * (1.f - t * t);
    }
    __syncthreads();   // every dW2 sum has read h1 before it is overwritten
    for (int i = 0; i < H; ++i) h1[tid * HS + i] = d1[i];
    __syncthreads();
    // dW1[o][f] = sum_s dH1[s][o] x[s][f]; db1[o] = sum_s dH1[s][o]
    for (int e = tid; e < H * IN; e += blockDim.x) {
        const int o = e / IN, f = e % IN;
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += h1[q * HS + o] * xs[q * IN + f];
        atomicAdd(G + OFF_W1 + e, a);
    }
    if (tid < H) {
        float a = 0.f;
        for (int q = 0; q < TILE; ++q) a += h1[q * HS + tid];
        atomicAdd(G + OFF_B1 + tid, a);
    }
}

constexpr size_t kGradSmem = sizeof(float) * (NP + TILE * IN + 2 * TILE * HS + TILE);

// Adam (Kingma & Ba 2015) with bias correction; clears the gradient.
__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ G, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float b1, float b2, float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float g = G[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    P[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    G[i] = 0.f;
}

void grad_launch(ibpme_mlp* m, int n, int base, int count, const int* idx, const float* X, const float* T,
                 float inv_batch, cudaStream_t s) {
    const int blocks = div_up(count, TILE);
    mlp_grad_kernel<<<blocks, TILE, kGradSmem, s>>>(n, base, count, idx, m->params.as<float>(), X, T, inv_batch,
                                                     m->grad.as<float>(), m->loss.as<float>());
    IBP_CHECK_LAUNCH();
}

void init_params(std::vector<float>& p, unsigned long long seed) {
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    p.assign(NP, 0.f);
    for (int i = 0; i < H * IN; ++i) p[OFF_W1 + i] = (float)(nd(rng) / std::sqrt((double)IN));
    for (int i = 0; i < H * H; ++i) p[OFF_W2 + i] = (float)(nd(rng) / std::sqrt((double)H));
    for (int i = 0; i < H; ++i) p[OFF_W3 + i] = (float)(nd(rng) / std::sqrt((double)H));
}

// ---- features -----------------------------------------------------------------
// Every feature comes from the body's own geometry, E0, the net charges and the
// free-space potential and field of the other bodies' fixed charges near the body;
// no mesh evaluation.
constexpr int kBs = 6;    // per (rhs, body): R, A, S, <r.E0>, <phi>, h
constexpr int kGeo = 8;   // per bead: d1, dk, n (3), kappa, unused (2)
constexpr int kSrcThreads = 256;

// Every bead as a source: wrapped position in FP32 and its fixed charge (an ion's
// own charge, Q/N on a bead of a multi-bead body).
__global__ void source_kernel(int n, const double* __restrict__ xw, const int* __restrict__ bead_body,
                              const int* __restrict__ off, const double* __restrict__ Q, float4* __restrict__ src) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = bead_body[k];
    src[k] = make_float4((float)xw[3 * k], (float)xw[3 * k + 1], (float)xw[3 * k + 2],
                         (float)(Q[b] / (double)(off[b + 1] - off[b])));
}

// Per multi-bead body (one warp): R = mean |r|, R_max, the reference point wrapped
// into the box with the source cutoff R_max + 6R (FP32), the relative positions as
// floats.
__global__ void body_geom_kernel(int nmb, const int* __restrict__ mb_body, const int* __restrict__ off,
                                 const double* __restrict__ rel, const double* __restrict__ X, double Lx, double Ly,
                                 double Lz, float4* __restrict__ rel32, double* __restrict__ Rb,
                                 float4* __restrict__ bgeo) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nmb) return;
    const int b = mb_body[i];
    const int s = off[b], e = off[b + 1];
    double rs = 0.0, rm = 0.0;
    for (int j = s + lane; j < e; j += 32) {
        const double x = rel[3 * j], y = rel[3 * j + 1], z = rel[3 * j + 2];
        const double r = sqrt(x * x + y * y + z * z);
        rs += r;
        rm = fmax(rm, r);
        rel32[j] = make_float4((float)x, (float)y, (float)z, 0.0f);
    }
    rs = warp_sum(rs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    if (lane == 0) {
        const double R = rs / (e - s);
        Rb[b] = R;
        const double xb = X[3 * b] - Lx * floor(X[3 * b] / Lx), yb = X[3 * b + 1] - Ly * floor(X[3 * b + 1] / Ly),
                     zb = X[3 * b + 2] - Lz * floor(X[3 * b + 2] / Lz);
        bgeo[b] = make_float4((float)xb, (float)yb, (float)zb, (float)(rm + 6.0 * R));
    }
}

// Partial phi and Es at the beads of one multi-bead body from one slice of the
// candidate sources (grid.x: the body's place among the multi-bead bodies, grid.y:
// chunks of 256 beads, grid.z: slices of the bead list): a source is a bead of
// another body with a fixed charge whose minimum image lies within the body's cutoff
// of its reference point; those of a 256-bead tile are compacted into shared memory
// and summed with the regularised free-space kernel (FP32).  part[z][j] =
// (phi, Es) before the 1/eps.
__global__ void __launch_bounds__(kSrcThreads) body_field_kernel(
    int n, int slice, const int* __restrict__ mb_body, const int* __restrict__ off,
    const int* __restrict__ bead_body, const float4* __restrict__ src, const float4* __restrict__ rel32,
    const float4* __restrict__ bgeo, float Lx, float Ly, float Lz, float a, float4* __restrict__ part) {
    const int b = mb_body[blockIdx.x];
    const int s = off[b], e = off[b + 1];
    if (s + (int)blockIdx.y * kSrcThreads >= e) return;   // the whole block: no bead of this chunk
    __shared__ float4 tile[kSrcThreads];
    __shared__ int wcount[kSrcThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = s + blockIdx.y * kSrcThreads + threadIdx.x;
    const float4 g = bgeo[b];
    const float4 rj = j < e ? rel32[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float c4 = 0.0795774715459476678f;                 // 1 / (4 pi)
    const float c16 = 0.0198943678864869170f / (a * a);      // 1 / (16 pi a^2)
    const float a2 = 2.0f * a;
    float p = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    const int k0 = blockIdx.z * slice, k1 = min(n, k0 + slice);
    for (int base = k0; base < k1; base += kSrcThreads) {
        const int k = base + threadIdx.x;
        bool ok = false;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < k1) {
            const float4 sk = src[k];
            if (sk.w != 0.f && bead_body[k] != b) {
                float dx = sk.x - g.x, dy = sk.y - g.y, dz = sk.z - g.z;
                dx -= Lx * rintf(dx / Lx);
                dy -= Ly * rintf(dy / Ly);
                dz -= Lz * rintf(dz / Lz);
                if (dx * dx + dy * dy + dz * dz < g.w * g.w) {
                    ok = true;
                    c = make_float4(dx, dy, dz, sk.w);
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) wcount[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int i = 0; i < kSrcThreads / 32; ++i) {
            const int cnt = wcount[i];
            before += i < w ? cnt : 0;
            total += cnt;
        }
        if (ok) tile[before + __popc(m & ((1u << lane) - 1u))] = c;
        __syncthreads();
        if (j < e) {
            for (int i = 0; i < total; ++i) {
                const float4 q = tile[i];
                const float vx = rj.x - q.x, vy = rj.y - q.y, vz = rj.z - q.z;
                const float r = sqrtf(vx * vx + vy * vy + vz * vz);
                float pot, gr;   // M(r) and -M'(r) / r
                if (r >= a2) {
                    const float ir = 1.0f / r;
                    pot = c4 * ir;
                    gr = pot * ir * ir;
                } else {
                    pot = c16 * (2.0f * a2 - r);
                    gr = r > 0.f ? c16 / r : 0.f;
                }
                p += q.w * pot;
                ex += q.w * gr * vx;
                ey += q.w * gr * vy;
                ez += q.w * gr * vz;
            }
        }
        __syncthreads();
    }
    if (j < e) part[(size_t)blockIdx.z * n + j] = make_float4(p, ex, ey, ez);
}

// phi and Es of every bead of a multi-bead body: the slices' partial sums added in
// slice order (the same result on every run), times 1/eps.
__global__ void body_field_sum_kernel(int n, int slices, const int* __restrict__ bead_body,
                                      const int* __restrict__ off, const float4* __restrict__ part, double inv_eps,
                                      double* __restrict__ phi, double* __restrict__ Es) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int b = bead_body[j];
    if (off[b + 1] - off[b] < 2) return;
    float p = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    for (int z = 0; z < slices; ++z) {
        const float4 v = part[(size_t)z * n + j];
        p += v.x;
        ex += v.y;
        ey += v.z;
        ez += v.w;
    }
    phi[j] = (double)p * inv_eps;
    Es[3 * j] = (double)ex * inv_eps;
    Es[3 * j + 1] = (double)ey * inv_eps;
    Es[3 * j + 2] = (double)ez * inv_eps;
}

// Unit eigenvector of the smallest eigenvalue of the symmetric positive
// semi-definite 3 x 3 matrix C = (c00, c11, c22, c01, c02, c12), in FP32 without
// transcendental functions: the adjugate adj(C) has the same eigenvectors, with
// eigenvalues the products of the other two of C's, so its dominant direction is
// C's smallest one (also when C is singular, as for a flat neighbourhood).  Start
// from adj(C)'s longest column and refine by six power steps (each shrinks the other
// directions by lambda_min / lambda_mid).  false if adj(C) vanishes (the smallest
// eigenvalue is not simple).
__device__ bool smallest_eigvec(float c00, float c11, float c22, float c01, float c02, float c12, float* v) {
    const float t = c00 + c11 + c22;
    if (!(t > 0.f)) return false;
    const float it = 1.0f / t;   // scale to trace 1
    c00 *= it; c11 *= it; c22 *= it; c01 *= it; c02 *= it; c12 *= it;
    const float a00 = c11 * c22 - c12 * c12, a11 = c00 * c22 - c02 * c02, a22 = c00 * c11 - c01 * c01;
    const float a01 = c02 * c12 - c01 * c22, a02 = c01 * c12 - c02 * c11, a12 = c01 * c02 - c00 * c12;
    const float n0 = a00 * a00 + a01 * a01 + a02 * a02, n1 = a01 * a01 + a11 * a11 + a12 * a12,
                n2 = a02 * a02 + a12 * a12 + a22 * a22;
    float x, y, z;
    if (n0 >= n1 && n0 >= n2) {
        x = a00; y = a01; z = a02;
    } else if (n1 >= n2) {
        x = a01; y = a11; z = a12;
    } else {
        x = a02; y = a12; z = a22;
    }
    float nn = x * x + y * y + z * z;
    if (!(nn > 1e-30f)) return false;
    for (int k = 0; k < 6; ++k) {
        const float inv = rsqrtf(nn);
        x *= inv; y *= inv; z *= inv;
        const float u = a00 * x + a01 * y + a02 * z, w = a01 * x + a11 * y + a12 * z, q = a02 * x + a12 * y + a22 * z;
        x = u; y = w; z = q;
        nn = x * x + y * y + z * z;
        if (!(nn > 1e-30f)) return false;
    }
    const float inv = rsqrtf(nn);
    v[0] = x * inv;
    v[1] = y * inv;
    v[2] = z * inv;
    return true;
}

// Per bead of a multi-bead body (one warp over the body's other beads): the
// nearest and k-th nearest distances (k = min(6, N-1)), and the Gaussian
// neighbourhood sums (weights exp(-d^2/h^2), h = sqrt(4 pi R^2 / N)) giving the
// normal (smallest principal direction of the weighted neighbour offsets) and the
// curvature, all in FP32.
__global__ void bead_geom_kernel(int n, const int* __restrict__ bead_body, const int* __restrict__ off,
                                 const float4* __restrict__ rel32, const double* __restrict__ Rb,
                                 float* __restrict__ geo) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int b = bead_body[j];
    const int s = off[b], e = off[b + 1], N = e - s;
    if (N < 2) return;
    const float h = sqrtf(12.566370614359172f / (float)N) * (float)Rb[b];
    const float ih2 = 1.0f / (h * h);
    const float4 rj = rel32[j];
    constexpr int K = 6;
    float best[K];
#pragma unroll
    for (int i = 0; i < K; ++i) best[i] = INFINITY;
    // W, m (3), s2, C (6: xx yy zz xy xz yz)
    float acc[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = 0.f;
    for (int k = s + lane; k < e; k += 32) {
        if (k == j) continue;
        const float4 rk = rel32[k];
        const float dx = rk.x - rj.x, dy = rk.y - rj.y, dz = rk.z - rj.z;
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < best[K - 1]) {   // insertion into this lane's sorted K smallest
            float v = d2;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (v < best[i]) {
                    const float tmp = best[i];
                    best[i] = v;
                    v = tmp;
                }
            }
        }
        const float w = __expf(-d2 * ih2);
        acc[0] += w;
        acc[1] += w * dx;
        acc[2] += w * dy;
        acc[3] += w * dz;
        acc[4] += w * d2;
        acc[5] += w * dx * dx;
        acc[6] += w * dy * dy;
        acc[7] += w * dz * dz;
        acc[8] += w * dx * dy;
        acc[9] += w * dx * dz;
        acc[10] += w * dy * dz;
    }
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = warp_sum(acc[i]);
    // merge: K rounds, each removing the warp's smallest head (lowest lane on ties)
    const int kk = N - 1 < K ? N - 1 : K;
    float d1 = 0.f, dk = 0.f;
    for (int i = 0; i < kk; ++i) {
        float m = best[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const unsigned who = __ballot_sync(0xffffffffu, best[0] == m);
        if (lane == __ffs(who) - 1) {
#pragma unroll
            for (int q = 0; q < K - 1; ++q) best[q] = best[q + 1];
            best[K - 1] = INFINITY;
        }
        if (i == 0) d1 = sqrtf(m);
        if (i == kk - 1) dk = sqrtf(m);
    }
    if (lane == 0) {
        const float iW = 1.0f / acc[0];
        const float mx = acc[1] * iW, my = acc[2] * iW, mz = acc[3] * iW, s2 = acc[4] * iW;
        float nv[3];
        if (!smallest_eigvec(acc[5] * iW, acc[6] * iW, acc[7] * iW, acc[8] * iW, acc[9] * iW, acc[10] * iW, nv)) {
            const float rr = sqrtf(rj.x * rj.x + rj.y * rj.y + rj.z * rj.z);
            nv[0] = rr > 0.f ? rj.x / rr : 0.f;
            nv[1] = rr > 0.f ? rj.y / rr : 0.f;
            nv[2] = rr > 0.f ? rj.z / rr : 1.f;
        }
        if (nv[0] * rj.x + nv[1] * rj.y + nv[2] * rj.z < 0.f) {
            nv[0] = -nv[0];
            nv[1] = -nv[1];
            nv[2] = -nv[2];
        }
        float* g = geo + (size_t)j * kGeo;
        g[0] = d1;
        g[1] = dk;
        g[2] = nv[0];
        g[3] = nv[1];
        g[4] = nv[2];
        g[5] = s2 > 0.f ? -2.0f * (mx * nv[0] + my * nv[1] + mz * nv[2]) / s2 : 0.f;
        g[6] = 0.f;
        g[7] = 0.f;
    }
}

// Per (rhs, multi-bead body), one warp: <r.E0>, <phi>, rms |Es|, S.
__global__ void body_stats_kernel(int nb, int nmb, int R, const int* __restrict__ mb_body,
                                  const int* __restrict__ off, const double* __restrict__ rel,
                                  const double* __restrict__ E0, const double* __restrict__ phi,
                                  const double* __restrict__ Es, const double* __restrict__ Rb, double eps,
                                  double* __restrict__ bs) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long long)nmb * R) return;
    const int r = (int)(w / nmb), b = mb_body[(int)(w % nmb)];
    const int s = off[b], e = off[b + 1], N = e - s;
    double* o = bs + ((size_t)r * nb + b) * kBs;
    const double ex = E0[3 * r], ey = E0[3 * r + 1], ez = E0[3 * r + 2];
    double re = 0.0, pm = 0.0, e2 = 0.0;
    for (int j = s + lane; j < e; j += 32) {
        re += rel[3 * j] * ex + rel[3 * j + 1] * ey + rel[3 * j + 2] * ez;
        pm += phi[j];
        e2 += Es[3 * j] * Es[3 * j] + Es[3 * j + 1] * Es[3 * j + 1] + Es[3 * j + 2] * Es[3 * j + 2];
    }
    re = warp_sum(re) / N;
    pm = warp_sum(pm) / N;
    e2 = warp_sum(e2) / N;
    if (lane == 0) {
        const double Rv = Rb[b];
        const double A = 4.0 * 3.14159265358979323846 * Rv * Rv / N;
        o[0] = Rv;
        o[1] = A;
        o[2] = eps * A * (sqrt(ex * ex + ey * ey + ez * ez) + sqrt(e2));   // S
        o[3] = re;
        o[4] = pm;
        o[5] = sqrt(A);
    }
}

__global__ void feature_kernel(int n, int nb, int R, const int* __restrict__ bead_body, const int* __restrict__ off,
                               const double* __restrict__ rel, const double* __restrict__ E0,
                               const double* __restrict__ phi, const double* __restrict__ Es,
                               const float* __restrict__ geo, const double* __restrict__ Q,
                               const double* __restrict__ bs, double eps, double a, float* __restrict__ feat) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int b = bead_body[j];
    const int N = off[b + 1] - off[b];
    float* f = feat + (size_t)t * IN;
    const double* o = bs + ((size_t)r * nb + b) * kBs;
    const double Rv = o[0], A = o[1], S = o[2], re = o[3], pm = o[4], h = o[5];
    if (N < 2 || !(S > 0.0)) {
        for (int k = 0; k < IN; ++k) f[k] = 0.f;
        return;
    }
    const float* g = geo + (size_t)j * kGeo;
    const double nx = g[2], ny = g[3], nz = g[4];
    const double ex = E0[3 * r], ey = E0[3 * r + 1], ez = E0[3 * r + 2];
    const double sx = Es[3 * j], sy = Es[3 * j + 1], sz = Es[3 * j + 2];
    const double rx = rel[3 * j], ry = rel[3 * j + 1], rz = rel[3 * j + 2];
    const double en = ex * nx + ey * ny + ez * nz, sn = sx * nx + sy * ny + sz * nz;
    const double tx = ex - en * nx, ty = ey - en * ny, tz = ez - en * nz;
    const double ux = sx - sn * nx, uy = sy - sn * ny, uz = sz - sn * nz;
    const double c = eps * A / S, cr = c / Rv;
    const double qb = Q[b] / N / S;
    f[0] = (float)(c * en);
    f[1] = (float)(c * sqrt(tx * tx + ty * ty + tz * tz));
    f[2] = (float)(cr * (rx * ex + ry * ey + rz * ez - re));
    f[3] = (float)(cr * (phi[j] - pm));
    f[4] = (float)(c * sn);
    f[5] = (float)(c * sqrt(ux * ux + uy * uy + uz * uz));
    f[6] = (float)((double)g[5] * Rv);
    f[7] = (float)(sqrt(rx * rx + ry * ry + rz * rz) / Rv - 1.0);
    f[8] = (float)(qb > 10.0 ? 10.0 : (qb < -10.0 ? -10.0 : qb));
    f[9] = (float)(10.0 * a / Rv);
    f[10] = (float)((double)g[0] / h);
    f[11] = (float)(((double)g[1] - (double)g[0]) / h);
}

// training target y = (q - Q/N) / S on beads of multi-bead bodies (0 elsewhere)
__global__ void target_kernel(int n, int nb, int R, const int* __restrict__ bead_body, const int* __restrict__ off,
                              const double* __restrict__ Q, const double* __restrict__ bs,
                              const double* __restrict__ q, float* __restrict__ y) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int b = bead_body[j];
    const int N = off[b + 1] - off[b];
    const double S = bs[((size_t)r * nb + b) * kBs + 2];
    y[t] = (N > 1 && S > 0.0) ? (float)((q[t] - Q[b] / N) / S) : 0.f;
}

// charge q = Q/N + S y on the beads of multi-bead bodies
__global__ void guess_from_net_kernel(int n, int nb, int R, const int* __restrict__ bead_body,
                                      const int* __restrict__ off, const double* __restrict__ Q,
                                      const double* __restrict__ bs, const float* __restrict__ y,
                                      double* __restrict__ q) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * R) return;
    const int r = (int)(t / n), j = (int)(t % n);
    const int b = bead_body[j];
    const int N = off[b + 1] - off[b];
    const double S = bs[((size_t)r * nb + b) * kBs + 2];
    double v = Q[b] / N;
    if (N > 1 && S > 0.0) v += S * (double)y[t];
    q[t] = v;
}

// restore the constraint sum_j q_ij = Q_i of every multi-bead body (uniform shift)
__global__ void project_kernel(int nmb, int n, int R, const int* __restrict__ mb_body, const int* __restrict__ off,
                               const double* __restrict__ Q, double* __restrict__ q) {
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)nmb * R) return;
    const int r = (int)(wid / nmb), b = mb_body[(int)(wid % nmb)];
    const int s = off[b], e = off[b + 1];
    double sm = 0.0;
    for (int j = s + lane; j < e; j += 32) sm += q[(size_t)r * n + j];
    sm = warp_sum(sm);
    const double shift = (Q[b] - sm) / (e - s);
    for (int j = s + lane; j < e; j += 32) q[(size_t)r * n + j] += shift;
}

}  // namespace

// Features of every bead for nrhs fields E0 [nrhs][3] (bodies already uploaded,
// positions wrapped, context stream current).  Leaves the per-body scales in
// `scales` [nrhs][nb][kBs].
void compute_features(ibpme_ctx* c, int n, const double* xw, const double* E0, int nrhs, float* feat,
                      DevBuf& scratch, DevBuf& scales) {
    BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    // scratch: phi [n], Es [n][3], R_b [nb] doubles; src, rel32 [n] and bgeo [nb] float4; geo [n][kGeo] floats
    auto up = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const size_t o_Es = up(sizeof(double) * (size_t)n), o_R = o_Es + up(sizeof(double) * 3 * (size_t)n);
    const size_t o_src = o_R + up(sizeof(double) * (size_t)bd.nb), o_rel = o_src + sizeof(float4) * (size_t)n;
    const size_t o_bg = o_rel + sizeof(float4) * (size_t)n, o_geo = o_bg + sizeof(float4) * (size_t)bd.nb;
    char* base = static_cast<char*>(scratch.ensure(o_geo + sizeof(float) * kGeo * (size_t)n));
    double* phi = reinterpret_cast<double*>(base);
    double* Es = reinterpret_cast<double*>(base + o_Es);
    double* Rb = reinterpret_cast<double*>(base + o_R);
    float4* src = reinterpret_cast<float4*>(base + o_src);
    float4* rel32 = reinterpret_cast<float4*>(base + o_rel);
    float4* bgeo = reinterpret_cast<float4*>(base + o_bg);
    float* geo = reinterpret_cast<float*>(base + o_geo);
    const double* L = c->p.box;
    source_kernel<<<div_up(n, 256), 256, 0, s>>>(n, xw, bd.bead_body.as<int>(), bd.off.as<int>(), bd.Q.as<double>(),
                                                 src);
    IBP_CHECK_LAUNCH();
    if (bd.nmb > 0) {
        body_geom_kernel<<<div_up((long long)bd.nmb * 32, 128), 128, 0, s>>>(
            bd.nmb, bd.mb_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(), bd.X.as<double>(), L[0], L[1], L[2],
            rel32, Rb, bgeo);
        IBP_CHECK_LAUNCH();
    }
    if (bd.nmb > 0) {
        // slices of the source list so that the grid fills the GPU about twice
        const int chunks = div_up(bd.max_beads, kSrcThreads);
        const long long cells = (long long)bd.nmb * chunks;
        int slices = (int)std::min<long long>(64, std::max<long long>(1, (2 * 152 + cells - 1) / cells));
        const int slice = div_up(div_up(n, slices), kSrcThreads) * kSrcThreads;
        slices = div_up(n, slice);
        float4* part = static_cast<float4*>(c->ml_part.ensure(sizeof(float4) * (size_t)slices * n));
        const dim3 grid(bd.nmb, chunks, slices);
        body_field_kernel<<<grid, kSrcThreads, 0, s>>>(n, slice, bd.mb_body.as<int>(), bd.off.as<int>(),
                                                        bd.bead_body.as<int>(), src, rel32, bgeo, (float)L[0],
                                                        (float)L[1], (float)L[2], (float)c->a, part);
        IBP_CHECK_LAUNCH();
        body_field_sum_kernel<<<div_up(n, 256), 256, 0, s>>>(n, slices, bd.bead_body.as<int>(), bd.off.as<int>(),
                                                             part, 1.0 / c->eps, phi, Es);
        IBP_CHECK_LAUNCH();
    }
    bead_geom_kernel<<<div_up((long long)n * 32, 128), 128, 0, s>>>(n, bd.bead_body.as<int>(), bd.off.as<int>(),
                                                                    rel32, Rb, geo);
    IBP_CHECK_LAUNCH();
    double* bs = static_cast<double*>(scales.ensure(sizeof(double) * kBs * (size_t)bd.nb * nrhs));
    if (bd.nmb > 0) {
        body_stats_kernel<<<div_up((long long)bd.nmb * nrhs * 32, 128), 128, 0, s>>>(
            bd.nb, bd.nmb, nrhs, bd.mb_body.as<int>(), bd.off.as<int>(), bd.rel.as<double>(), E0, phi, Es, Rb, c->eps,
            bs);
        IBP_CHECK_LAUNCH();
    }
    feature_kernel<<<div_up((long long)n * nrhs, 256), 256, 0, s>>>(n, bd.nb, nrhs, bd.bead_body.as<int>(),
                                                                    bd.off.as<int>(), bd.rel.as<double>(), E0, phi, Es,
                                                                    geo, bd.Q.as<double>(), bs, c->eps, c->a, feat);
    IBP_CHECK_LAUNCH();
}

// q += g - gprev for every bead of a multi-bead body (the learned change added to
// the previous charges); single beads keep q.
__global__ void step_guess_kernel(long long len, int n, const int* __restrict__ bead_body, const int* __restrict__ off,
                                  const double* __restrict__ g, const double* __restrict__ gprev,
                                  double* __restrict__ q) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= len) return;
    const int b = bead_body[(int)(t % n)];
    if (off[b + 1] - off[b] > 1) q[t] += g[t] - gprev[t];
}

// Learned initial charges q [nrhs][n] (constraint restored body by body); with
// step, q (in) holds the previous call's charges and gets the learned change.
void learned_guess(ibpme_ctx* c, const ibpme_mlp* mlp, int n, const double* xw, const double* E0, int nrhs,
                   double* q, bool step) {
    DevBuf& feat = c->ml_feat;
    DevBuf& scratch = c->ml_scratch;
    DevBuf& scales = c->ml_scales;
    DevBuf& y = c->ml_y;
    BodyData& bd = c->bodies;
    cudaStream_t s = c->stream;
    const long long len = (long long)n * nrhs;
    const bool have_prev = c->ml_prev_n == n && c->ml_prev_R == nrhs && c->ml_prev_version == bd.version &&
                           c->ml_gprev.bytes >= sizeof(double) * (size_t)len;
    double* g = step && have_prev ? static_cast<double*>(c->ml_g.ensure(sizeof(double) * (size_t)len)) : q;
    float* f = static_cast<float*>(feat.ensure(sizeof(float) * IN * (size_t)len));
    compute_features(c, n, xw, E0, nrhs, f, scratch, scales);
    float* yy = static_cast<float*>(y.ensure(sizeof(float) * (size_t)len));
    forward_tc(mlp, (int)len, f, yy, s, false);   // checked after the solve (which synchronises)
    guess_from_net_kernel<<<div_up(len, 256), 256, 0, s>>>(n, bd.nb, nrhs, bd.bead_body.as<int>(), bd.off.as<int>(),
                                                           bd.Q.as<double>(), scales.as<double>(), yy, g);
    IBP_CHECK_LAUNCH();
    if (bd.nmb > 0) {
        project_kernel<<<div_up((long long)bd.nmb * nrhs * 32, 128), 128, 0, s>>>(
            bd.nmb, n, nrhs, bd.mb_body.as<int>(), bd.off.as<int>(), bd.Q.as<double>(), g);
        IBP_CHECK_LAUNCH();
    }
    double* gp = static_cast<double*>(c->ml_gprev.ensure(sizeof(double) * (size_t)len));
    if (g != q) {
        step_guess_kernel<<<div_up(len, 256), 256, 0, s>>>(len, n, bd.bead_body.as<int>(), bd.off.as<int>(), g, gp, q);
        IBP_CHECK_LAUNCH();
    }
    IBP_CUDA(cudaMemcpyAsync(gp, g, sizeof(double) * (size_t)len, cudaMemcpyDeviceToDevice, s));
    c->ml_prev_n = n;
    c->ml_prev_R = nrhs;
    c->ml_prev_version = bd.version;
}

void learned_check(const ibpme_mlp* mlp) { forward_tc_check(mlp); }

}  // namespace ibp

using namespace ibp;

namespace {

template <typename F>
ibpme_status mlp_guard(F&& f) {
    try {
        set_error("%s", "");
        return f();
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        set_error("unexpected internal exception");
        return IBPME_ERR_CUDA;
    }
}

}  // namespace

IBP_API ibpme_status ibpme_mlp_create(ibpme_mlp** out, unsigned long long seed) {
    if (!out) {
        set_error("out is NULL");
        return IBPME_ERR_ARG;
    }
    *out = nullptr;
    return mlp_guard([&]() -> ibpme_status {
        ibpme_mlp* m = new ibpme_mlp();
        try {
            IBP_CUDA(cudaGetDevice(&m->device));
            std::vector<float> p;
            init_params(p, seed);
            m->params.ensure(sizeof(float) * NP);
            m->grad.ensure(sizeof(float) * NP);
            m->m1.ensure(sizeof(float) * NP);
            m->m2.ensure(sizeof(float) * NP);
            m->loss.ensure(sizeof(float));
            IBP_CUDA(cudaMemcpy(m->params.p, p.data(), sizeof(float) * NP, cudaMemcpyHostToDevice));
            IBP_CUDA(cudaMemset(m->grad.p, 0, sizeof(float) * NP));
            IBP_CUDA(cudaMemset(m->m1.p, 0, sizeof(float) * NP));
            IBP_CUDA(cudaMemset(m->m2.p, 0, sizeof(float) * NP));
            IBP_CUDA(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kGradSmem));
        } catch (...) {
            delete m;
            throw;
        }
        *out = m;
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_destroy(ibpme_mlp* m) {
    if (m && m->tc_err_host) cudaFreeHost(m->tc_err_host);
    delete m;
    return IBPME_OK;
}

IBP_API ibpme_status ibpme_mlp_get(const ibpme_mlp* m, float* params) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || !params) fail(IBPME_ERR_ARG, "NULL argument");
        IBP_CUDA(cudaMemcpy(params, m->params.p, sizeof(float) * NP, cudaMemcpyDefault));
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_set(ibpme_mlp* m, const float* params) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || !params) fail(IBPME_ERR_ARG, "NULL argument");
        IBP_CUDA(cudaMemcpy(m->params.p, params, sizeof(float) * NP, cudaMemcpyDefault));
        IBP_CUDA(cudaMemset(m->m1.p, 0, sizeof(float) * NP));
        IBP_CUDA(cudaMemset(m->m2.p, 0, sizeof(float) * NP));
        m->step = 0;
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_forward(ibpme_mlp* m, int n, const float* feat, float* out, void* cuda_stream) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || n < 0 || (n > 0 && (!feat || !out))) fail(IBPME_ERR_ARG, "bad argument");
        if (n == 0) return IBPME_OK;
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        mlp_forward_kernel<<<div_up(n, 128), 128, 0, s>>>(n, m->params.as<float>(), feat, out);
        IBP_CHECK_LAUNCH();
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_forward_tc(ibpme_mlp* m, int n, const float* feat, float* out, void* cuda_stream) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || n < 0 || (n > 0 && (!feat || !out))) fail(IBPME_ERR_ARG, "bad argument");
        forward_tc(m, n, feat, out, static_cast<cudaStream_t>(cuda_stream));
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_gradient(ibpme_mlp* m, int n, const float* feat, const float* target, float* grad,
                                        float* loss, void* cuda_stream) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || n < 1 || !feat || !target || !grad) fail(IBPME_ERR_ARG, "bad argument");
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        IBP_CUDA(cudaMemsetAsync(m->grad.p, 0, sizeof(float) * NP, s));
        IBP_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(float), s));
        grad_launch(m, n, 0, n, nullptr, feat, target, 1.0f / n, s);
        IBP_CUDA(cudaMemcpyAsync(grad, m->grad.p, sizeof(float) * NP, cudaMemcpyDefault, s));
        if (loss) IBP_CUDA(cudaMemcpyAsync(loss, m->loss.p, sizeof(float), cudaMemcpyDefault, s));
        IBP_CUDA(cudaMemsetAsync(m->grad.p, 0, sizeof(float) * NP, s));
        IBP_CUDA(cudaStreamSynchronize(s));
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_mlp_train(ibpme_mlp* m, int n, const float* feat, const float* target, int batch,
                                     int epochs, float lr, unsigned long long seed, float* loss_out,
                                     void* cuda_stream) {
    return mlp_guard([&]() -> ibpme_status {
        if (!m || n < 1 || !feat || !target || batch < 1 || epochs < 0) fail(IBPME_ERR_ARG, "bad argument");
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        int* perm = static_cast<int*>(m->perm.ensure(sizeof(int) * n));
        std::vector<int> hp(n);
        std::mt19937_64 rng(seed);
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        float last = 0.f;
        for (int ep = 0; ep < epochs; ++ep) {
            for (int i = 0; i < n; ++i) hp[i] = i;
            std::shuffle(hp.begin(), hp.end(), rng);
            IBP_CUDA(cudaMemcpyAsync(perm, hp.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
            IBP_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(float), s));
            int batches = 0;
            for (int base = 0; base < n; base += batch) {
                const int cnt = (n - base < batch) ? n - base : batch;
                grad_launch(m, n, base, cnt, perm, feat, target, 1.0f / cnt, s);
                ++m->step;
                const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
                adam_kernel<<<div_up(NP, 256), 256, 0, s>>>(m->params.as<float>(), m->grad.as<float>(),
                                                            m->m1.as<float>(), m->m2.as<float>(), lr, b1, b2, c1, c2,
                                                            eps);
                IBP_CHECK_LAUNCH();
                ++batches;
            }
            float h = 0.f;
            IBP_CUDA(cudaMemcpyAsync(&h, m->loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
            IBP_CUDA(cudaStreamSynchronize(s));   // also keeps hp alive until the copy is done
            last = batches ? h / batches : 0.f;
        }
        if (loss_out) *loss_out = last;
        return IBPME_OK;
    });
}

IBP_API ibpme_status ibpme_features(ibpme_ctx* c, int n, const double* x, const ibpme_bodies* bodies,
                                    const double* E0, int nrhs, float* feat, const double* q, float* target) {
    return mlp_guard([&]() -> ibpme_status {
        if (!c || n < 1 || !x || !bodies || !E0 || !feat || nrhs < 1 || nrhs > c->p.max_rhs)
            fail(IBPME_ERR_ARG, "bad argument");
        bool dev_ok = true;
        for (const void* p : {(const void*)x, (const void*)E0, (const void*)feat, (const void*)bodies->body_offsets,
                              (const void*)bodies->X, (const void*)bodies->Q, (const void*)q, (const void*)target}) {
            if (!p) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
                !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
                cudaGetLastError();
                dev_ok = false;
            }
        }
        if (!dev_ok) fail(IBPME_ERR_ARG, "ibpme_features takes device pointers");
        double* xw = static_cast<double*>(c->xw.ensure(sizeof(double) * 3 * n));
        wrap_positions(c, n, x, xw);
        c->near.fp_pre_valid = false;
        bodies_upload(c, n, bodies, xw);
        compute_features(c, n, xw, E0, nrhs, feat, c->ml_scratch, c->ml_scales);
        if (q && target) {
            const BodyData& bd = c->bodies;
            target_kernel<<<div_up((long long)n * nrhs, 256), 256, 0, c->stream>>>(
                n, bd.nb, nrhs, bd.bead_body.as<int>(), bd.off.as<int>(), bd.Q.as<double>(), c->ml_scales.as<double>(),
                q, target);
            IBP_CHECK_LAUNCH();
        }
        return IBPME_OK;
    });
}
