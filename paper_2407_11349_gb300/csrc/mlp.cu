// Surrogate network of the log-likelihood and its gradient: a 7 -> 256 -> 256
// -> 7 multilayer perceptron (tanh hidden units), trained on the GPU with
// these kernels and evaluated inside HMC leapfrog trajectories.  The paper has
// no surrogate: this is the learned part layered on its method.
//
// Inputs are the six standardised log-parameters and a seventh input that is
// either a constant 1 or a standardised per-sample feature; outputs are the
// standardised log-likelihood and its six log-parameter partials.
// Weights are kept in FP32 (Adam state and master copy); the 256 x 256 layer
// runs on the 5th-generation tensor cores (tcgen05.mma, accumulator in tensor
// memory) from BF16 copies of W2 and W2^T with BF16 activations and FP32
// accumulation; the 7-wide layers run in FP32.
//   forward:  h1 = tanh(x W1^T + b1), h2 = tanh(h1 W2^T + b2), y = h2 W3^T + b3
//   loss:     mean over the batch and the 7 outputs of (y - t)^2
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace {

using bf16 = __nv_bfloat16;
constexpr int DIN = 7, DH = 256, DOUT = 7;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + DH * DIN, OFF_W2 = OFF_B1 + DH, OFF_B2 = OFF_W2 + DH * DH,
              OFF_W3 = OFF_B2 + DH, OFF_B3 = OFF_W3 + DOUT * DH, NPARAMS = OFF_B3 + DOUT;
static_assert(NPARAMS == HAWKES_MLP_NPARAMS, "parameter count");
constexpr int BMAX = 4096;  // largest batch (a multiple of 64)

// ---------------------------------------------------------------------------
// Epilogues of the 256 x 256 layer's products (C = A . Bt^T, FP32 out):
//   EPI_FWD2  tanh(C + b2)            (forward, h2)
//   EPI_STORE C                       (weight gradient of W2)
//   EPI_BWD1  C * (1 - h1^2)          (backward through the first tanh)
// ---------------------------------------------------------------------------
enum { EPI_FWD2 = 0, EPI_STORE = 1, EPI_BWD1 = 2 };

struct Epi {
    const float* bias;  // EPI_FWD2: b2[N]
    const float* h;     // EPI_BWD1: h1 (FP32, [M x N]) for the tanh derivative
    float* out;         // [M x N] FP32
};

// ---------------------------------------------------------------------------
// The products on the 5th-generation tensor cores (tcgen05): one CTA of 128
// threads computes a 128 x 256 tile of C = A . Bt^T (A [M x K] and Bt
// [256 x K] row-major BF16; every product here has N = 256, K a multiple of
// 64) with the FP32 accumulator in tensor memory.
//   - K is staged in chunks of 64 BF16 values: the A rows [m0, m0 + 128) and
//     all 256 Bt rows, as 8 x 16-byte core matrices in the unswizzled
//     K-major layout: core matrix (row group i, K group j) at byte
//     (8 i + j) * 128, so the K step between core matrices is 128 bytes and
//     the row-group step 1024 bytes.  (Had the two offsets been read the
//     other way round, every access would still fall inside the operand's
//     buffer.)
//   - One thread issues the four K = 16 products of a chunk and commits them
//     to an mbarrier; the chunk's buffers are refilled after it completes.
//   - Warp w reads TMEM lanes [32 w, 32 w + 32) (tile rows) 16 columns at a
//     time for the epilogue.
// A wait that gives up latches HAWKES_ERR_TIMEOUT in *err, skips the
// epilogue, and the tensor memory is still released.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 256, TC_KC = 64;
constexpr uint32_t TC_BYTES_A = TC_M * TC_KC * 2, TC_BYTES_B = TC_N * TC_KC * 2;
constexpr uint32_t TC_SMEM = TC_BYTES_A + TC_BYTES_B;
// kind::f16 instruction descriptor: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((TC_N >> 3) << 17) |
                              ((TC_M >> 4) << 24);

constexpr uint32_t TC_LBO = 128, TC_SBO = (TC_KC / 8) * 128;  // K step, row-group step (bytes)

__device__ __forceinline__ uint32_t core_off(int r, int j) {
    return static_cast<uint32_t>(((r >> 3) * (TC_KC / 8) + j) * 128 + (r & 7) * 16);
}

// Shared-memory matrix descriptor: start, K-direction and row-group byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
           (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const bf16* __restrict__ A, int lda, int M,
                                                    const bf16* __restrict__ Bt, int ldb, int K,
                                                    Epi e, int ldc, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M;
    unsigned char* sA = tc_smem;
    unsigned char* sB = tc_smem + TC_BYTES_A;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         hk::smem_u32(&s_tmem)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        hk::mbar_init(&bar, 1);
        hk::fence_barrier_init();
        s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K && !s_fail; k0 += TC_KC) {
        for (int idx = tid; idx < TC_M * 8; idx += 128) {  // 16-byte pieces of A
            const int r = idx >> 3, j = idx & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M)
                v = *reinterpret_cast<const uint4*>(A + static_cast<size_t>(m0 + r) * lda + k0 + j * 8);
            *reinterpret_cast<uint4*>(sA + core_off(r, j)) = v;
        }
        for (int idx = tid; idx < TC_N * 8; idx += 128) {  // and of Bt
            const int r = idx >> 3, j = idx & 7;
            *reinterpret_cast<uint4*>(sB + core_off(r, j)) =
                *reinterpret_cast<const uint4*>(Bt + static_cast<size_t>(r) * ldb + k0 + j * 8);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s4 = 0; s4 < TC_KC / 16; ++s4) {
                // K = 16 values = core-matrix columns 2 s4 and 2 s4 + 1
                const uint64_t da = smem_desc(hk::smem_u32(sA) + s4 * 2 * TC_LBO, TC_LBO, TC_SBO);
                const uint64_t db = smem_desc(hk::smem_u32(sB) + s4 * 2 * TC_LBO, TC_LBO, TC_SBO);
                const uint32_t accumulate = (k0 > 0 || s4 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(TC_IDESC), "r"(accumulate)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             hk::smem_u32(&bar))
                         : "memory");
            if (!hk::mbar_wait(&bar, phase)) {
                s_fail = 1;
                atomicCAS(err, 0, HAWKES_ERR_TIMEOUT);
            }
        }
        phase ^= 1u;
        __syncthreads();
    }
    if (!s_fail) {
        tc_fence_after();
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                  "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                const size_t o = static_cast<size_t>(row) * ldc + c0;
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v[q] = __uint_as_float(r[q]);
                    if (EPI == EPI_FWD2) v[q] = tanhf(v[q] + e.bias[c0 + q]);
                    if (EPI == EPI_BWD1) {
                        const float h = e.h[o + q];
                        v[q] = v[q] * (1.f - h * h);
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4*>(e.out + o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
        }
    } else if (tid == 0) {
        (void)hk::mbar_wait(&bar, phase ^ 1u);  // bounded: let products in flight finish
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Small layers and reductions (FP32).
// ---------------------------------------------------------------------------
// h1 = tanh(x W1^T + b1): FP32 copy, BF16 row-major copy, BF16 transposed copy.
__global__ void k_l1(const float* __restrict__ X, const float* __restrict__ P, int B,
                     float* __restrict__ H1f, bf16* __restrict__ H1b, bf16* __restrict__ H1Tb) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * DH) return;
    const int b = idx / DH, j = idx % DH;
    float z = P[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < DIN; ++k) z = fmaf(P[OFF_W1 + j * DIN + k], X[b * DIN + k], z);
    const float h = tanhf(z);
    H1f[idx] = h;
    H1b[idx] = __float2bfloat16_rn(h);
    H1Tb[static_cast<size_t>(j) * B + b] = __float2bfloat16_rn(h);
}

// y = h2 W3^T + b3; with targets: dy = 2 (y - t) / (7 B) and the loss sum.
__global__ void k_l3(const float* __restrict__ H2f, const float* __restrict__ P, int B,
                     const float* __restrict__ T, float* __restrict__ Y, float* __restrict__ dY,
                     double* loss) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * DOUT) return;
    const int b = idx / DOUT, o = idx % DOUT;
    float y = P[OFF_B3 + o];
    for (int j = 0; j < DH; ++j) y = fmaf(P[OFF_W3 + o * DH + j], H2f[b * DH + j], y);
    Y[idx] = y;
    if (T) {
        const float d = y - T[idx];
        dY[idx] = 2.f * d / static_cast<float>(DOUT * B);
        atomicAdd(loss, static_cast<double>(d) * d / (DOUT * B));
    }
}

// dz2 = (dy W3) * (1 - h2^2): FP32, BF16 row-major and BF16 transposed copies.
__global__ void k_bwd2(const float* __restrict__ dY, const float* __restrict__ H2f,
                       const float* __restrict__ P, int B, float* __restrict__ dZ2f,
                       bf16* __restrict__ dZ2b, bf16* __restrict__ dZ2Tb) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * DH) return;
    const int b = idx / DH, j = idx % DH;
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < DOUT; ++o) s = fmaf(dY[b * DOUT + o], P[OFF_W3 + o * DH + j], s);
    const float h = H2f[idx];
    const float d = s * (1.f - h * h);
    dZ2f[idx] = d;
    dZ2b[idx] = __float2bfloat16_rn(d);
    dZ2Tb[static_cast<size_t>(j) * B + b] = __float2bfloat16_rn(d);
}

// Gradients reduced over the batch: W3, b3, b2 (after k_bwd2) or W1, b1 (after
// the backward GEMM).  One block of 256 threads per output element.
__global__ void k_grad_small(const float* __restrict__ dY, const float* __restrict__ H2f,
                             const float* __restrict__ dZ2f, const float* __restrict__ dZ1f,
                             const float* __restrict__ X, int B, int which, float* __restrict__ G) {
    const int e = blockIdx.x;
    float s = 0.f;
    int dst;
    if (which == 0) {  // W3 [7 x 256], b3 [7], b2 [256]
        if (e < DOUT * DH) {
            const int o = e / DH, j = e % DH;
            for (int b = threadIdx.x; b < B; b += blockDim.x) s += dY[b * DOUT + o] * H2f[b * DH + j];
            dst = OFF_W3 + e;
        } else if (e < DOUT * DH + DOUT) {
            const int o = e - DOUT * DH;
            for (int b = threadIdx.x; b < B; b += blockDim.x) s += dY[b * DOUT + o];
            dst = OFF_B3 + o;
        } else {
            const int j = e - DOUT * DH - DOUT;
            for (int b = threadIdx.x; b < B; b += blockDim.x) s += dZ2f[b * DH + j];
            dst = OFF_B2 + j;
        }
    } else {  // W1 [256 x 7], b1 [256]
        if (e < DH * DIN) {
            const int j = e / DIN, k = e % DIN;
            for (int b = threadIdx.x; b < B; b += blockDim.x) s += dZ1f[b * DH + j] * X[b * DIN + k];
            dst = OFF_W1 + e;
        } else {
            const int j = e - DH * DIN;
            for (int b = threadIdx.x; b < B; b += blockDim.x) s += dZ1f[b * DH + j];
            dst = OFF_B1 + j;
        }
    }
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) G[dst] = red[0];
}

// Adam step (bias-corrected, step count read from device memory) and refresh
// of the BF16 copies of W2 and W2^T.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, const int64_t* step, float lr, bf16* __restrict__ W2b,
                       bf16* __restrict__ W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAMS) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float tt = static_cast<float>(*step + 1);  // this update's 1-based step number
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float mh = m / (1.f - powf(b1, tt)), vh = v / (1.f - powf(b2, tt));
    const float p = P[i] - lr * mh / (sqrtf(vh) + eps);
    P[i] = p;
    if (i >= OFF_W2 && i < OFF_B2) {
        const int r = (i - OFF_W2) / DH, c = (i - OFF_W2) % DH;
        W2b[r * DH + c] = __float2bfloat16_rn(p);
        W2Tb[c * DH + r] = __float2bfloat16_rn(p);
    }
}

__global__ void k_refresh_w2(const float* __restrict__ P, bf16* __restrict__ W2b,
                             bf16* __restrict__ W2Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= DH * DH) return;
    const int r = i / DH, c = i % DH;
    const bf16 v = __float2bfloat16_rn(P[OFF_W2 + i]);
    W2b[r * DH + c] = v;
    W2Tb[c * DH + r] = v;
}

// Philox4x32-10 (Salmon et al. 2011) for minibatch draws and initialisation.
__device__ __forceinline__ uint4 philox4x32(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Minibatch of B rows drawn with replacement from the n standardised rows
// (Philox counter: row slot, completed step count); clears the loss.
__global__ void k_gather(const float* __restrict__ Xs, const float* __restrict__ Ts, int64_t n,
                         int B, uint64_t seed, const int64_t* step, float* __restrict__ X,
                         float* __restrict__ T, double* loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = *step;
    if (b < B) {
        const uint4 r = philox4x32(make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(s),
                                              static_cast<uint32_t>(s >> 32), 0x4d4c50u),
                                   make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
        const uint64_t u = (static_cast<uint64_t>(r.x) << 32) | r.y;
        const int64_t row = static_cast<int64_t>(u % static_cast<uint64_t>(n));
        for (int k = 0; k < DIN; ++k) X[b * DIN + k] = Xs[row * DIN + k];
        for (int k = 0; k < DOUT; ++k) T[b * DOUT + k] = Ts[row * DOUT + k];
    }
    if (b == 0) *loss = 0.0;
}

__global__ void k_step_done(int64_t* step) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

// Column means and standard deviations (FP64) of X[n x 6], Y[n x 7] and the
// optional feature F[n], then the standardised FP32 copies (the 7th input is
// the standardised feature, or the constant 1 without one).
__global__ void k_stats(const double* __restrict__ X, const double* __restrict__ Y,
                        const double* __restrict__ F, int64_t n,
                        double* stats /* mean_in[6] sd_in[6] mean_out[7] sd_out[7] mean_f sd_f */) {
    const int col = blockIdx.x;  // 0..5 inputs, 6..12 outputs, 13 the feature
    if (col == 13 && !F) {
        if (threadIdx.x == 0) {
            stats[26] = 0.0;
            stats[27] = 1.0;
        }
        return;
    }
    const double* src = col < 6 ? X : col < 13 ? Y : F;
    const int w = col < 6 ? 6 : col < 13 ? 7 : 1, c = col < 6 ? col : col < 13 ? col - 6 : 0;
    double s = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = src[i * w + c];
        s += v;
        s2 += v * v;
    }
    __shared__ double r1[256], r2[256];
    r1[threadIdx.x] = s;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            r1[threadIdx.x] += r1[threadIdx.x + k];
            r2[threadIdx.x] += r2[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = r1[0] / n;
        double var = r2[0] / n - mean * mean;
        double sd = var > 0.0 ? sqrt(var) : 0.0;
        if (!(sd > 1e-12 * (fabs(mean) + 1e-300))) sd = 1.0;  // constant column
        if (col < 6) {
            stats[col] = mean;
            stats[6 + col] = sd;
        } else if (col < 13) {
            stats[12 + c] = mean;
            stats[19 + c] = sd;
        } else {
            stats[26] = mean;
            stats[27] = sd;
        }
    }
}

__global__ void k_standardise(const double* __restrict__ X, const double* __restrict__ Y,
                              const double* __restrict__ F, int64_t n,
                              const double* __restrict__ st, float* __restrict__ Xs,
                              float* __restrict__ Ts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 6; ++k) Xs[i * DIN + k] = static_cast<float>((X[i * 6 + k] - st[k]) / st[6 + k]);
        Xs[i * DIN + 6] = F ? static_cast<float>((F[i] - st[26]) / st[27]) : 1.f;
        if (Y)
            for (int k = 0; k < 7; ++k)
                Ts[i * DOUT + k] = static_cast<float>((Y[i * 7 + k] - st[12 + k]) / st[19 + k]);
    }
}

// Prediction: standardise the queries (zero-padded to B rows), and map the
// network's outputs back to the log-likelihood and log-parameter partials.
__global__ void k_predict_in(const double* __restrict__ q, const double* __restrict__ f, int64_t m,
                             int B, const double* __restrict__ st, float* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    for (int k = 0; k < 6; ++k) X[i * DIN + k] = i < m ? static_cast<float>((q[i * 6 + k] - st[k]) / st[6 + k]) : 0.f;
    X[i * DIN + 6] = (f && i < m) ? static_cast<float>((f[i] - st[26]) / st[27]) : (f ? 0.f : 1.f);
}

__global__ void k_predict_out(const float* __restrict__ Y, int64_t m, const double* __restrict__ st,
                              double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * DOUT) return;
    const int k = i % DOUT;
    out[i] = st[12 + k] + st[19 + k] * static_cast<double>(Y[i]);
}

__global__ void k_init_params(float* P, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAMS) return;
    float lim = 0.f;  // biases start at zero
    if (i < OFF_B1) lim = sqrtf(6.f / (DH + DIN));
    else if (i >= OFF_W2 && i < OFF_B2) lim = sqrtf(6.f / (DH + DH));
    else if (i >= OFF_W3 && i < OFF_B3) lim = sqrtf(6.f / (DOUT + DH));
    const uint4 r = philox4x32(make_uint4(static_cast<uint32_t>(i), 0u, 0u, 0x494e4954u),
                               make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
    const float u = (r.x >> 8) * (1.f / 16777216.f);
    P[i] = lim * (2.f * u - 1.f);
}

}  // namespace

struct hawkes_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    bf16 *W2b = nullptr, *W2Tb = nullptr;
    int64_t* step = nullptr;
    double* loss = nullptr;
    double* stats = nullptr;  // 28 values
    bool have_stats = false;
    bool have_feature = false;  // the 7th input is a feature (else the constant 1)
    int64_t n = 0;
    float *Xs = nullptr, *Ts = nullptr;  // standardised data set
    // batch work buffers (BMAX rows)
    float *X = nullptr, *T = nullptr, *H1f = nullptr, *H2f = nullptr, *Y = nullptr, *dY = nullptr,
          *dZ2f = nullptr, *dZ1f = nullptr;
    bf16 *H1b = nullptr, *H1Tb = nullptr, *dZ2b = nullptr, *dZ2Tb = nullptr;
    double* hbuf = nullptr;  // pinned host scratch
    int* err = nullptr;      // latched device error (a tensor-core wait that gave up)
};

namespace {

int st_of(cudaError_t e) {
    if (e == cudaSuccess) return HAWKES_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HAWKES_ERR_OOM : HAWKES_ERR_CUDA;
}
#define HM_TRY(expr)                      \
    do {                                  \
        int _rc = (expr);                 \
        if (_rc != HAWKES_OK) return _rc; \
    } while (0)
#define HM_CUDA(expr) HM_TRY(st_of(expr))

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
int alloc(T** p, size_t count) {
    return st_of(cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T)));
}

// Read and clear the latched device error (synchronous).
int take_err(hawkes_mlp* m) {
    HM_CUDA(cudaMemcpyAsync(m->hbuf + 63, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    HM_CUDA(cudaStreamSynchronize(m->stream));
    int e = 0;
    std::memcpy(&e, m->hbuf + 63, sizeof(int));
    if (e != 0) HM_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    return e;
}

// Forward (and, with targets, backward) of a batch already in m->X (and m->T).
int forward_backward(hawkes_mlp* m, int B, bool train) {
    cudaStream_t st = m->stream;
    const int gH = (B * DH + 255) / 256, gO = (B * DOUT + 255) / 256;
    k_l1<<<gH, 256, 0, st>>>(m->X, m->P, B, m->H1f, m->H1b, m->H1Tb);
    Epi e2{m->P + OFF_B2, nullptr, m->H2f};
    const int gM = (B + TC_M - 1) / TC_M;
    k_gemm_tc<EPI_FWD2><<<gM, 128, TC_SMEM, st>>>(m->H1b, DH, B, m->W2b, DH, DH, e2, DH, m->err);
    k_l3<<<gO, 256, 0, st>>>(m->H2f, m->P, B, train ? m->T : nullptr, m->Y, m->dY, m->loss);
    if (train) {
        k_bwd2<<<gH, 256, 0, st>>>(m->dY, m->H2f, m->P, B, m->dZ2f, m->dZ2b, m->dZ2Tb);
        k_grad_small<<<DOUT * DH + DOUT + DH, 256, 0, st>>>(m->dY, m->H2f, m->dZ2f, nullptr, m->X, B,
                                                            0, m->G);
        Epi ew{nullptr, nullptr, m->G + OFF_W2};
        k_gemm_tc<EPI_STORE><<<DH / TC_M, 128, TC_SMEM, st>>>(m->dZ2Tb, B, DH, m->H1Tb, B, B, ew, DH,
                                                             m->err);
        Epi eb{nullptr, m->H1f, m->dZ1f};
        k_gemm_tc<EPI_BWD1><<<gM, 128, TC_SMEM, st>>>(m->dZ2b, DH, B, m->W2Tb, DH, DH, eb, DH, m->err);
        k_grad_small<<<DH * DIN + DH, 256, 0, st>>>(nullptr, nullptr, nullptr, m->dZ1f, m->X, B, 1, m->G);
    }
    return st_of(cudaGetLastError());
}

}  // namespace

extern "C" {

int hawkes_mlp_create(hawkes_mlp** out, int device, void* cuda_stream, uint64_t seed) {
    HK_NVTX("hawkes_mlp_create");
    if (!out) return HAWKES_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? HAWKES_ERR_ARG : HAWKES_ERR_CUDA;
    }
    DeviceGuard g(device);
    hawkes_mlp* m = new (std::nothrow) hawkes_mlp();
    if (!m) return HAWKES_ERR_OOM;
    m->device = device;
    int rc = HAWKES_OK;
    do {
        if (cuda_stream) {
            m->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            if ((rc = st_of(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking)))) break;
            m->own_stream = true;
        }
        if ((rc = alloc(&m->P, NPARAMS)) || (rc = alloc(&m->G, NPARAMS)) || (rc = alloc(&m->M, NPARAMS)) ||
            (rc = alloc(&m->V, NPARAMS)) || (rc = alloc(&m->W2b, DH * DH)) || (rc = alloc(&m->W2Tb, DH * DH)) ||
            (rc = alloc(&m->step, 1)) || (rc = alloc(&m->loss, 1)) || (rc = alloc(&m->stats, 28)) ||
            (rc = alloc(&m->X, BMAX * DIN)) || (rc = alloc(&m->T, BMAX * DOUT)) ||
            (rc = alloc(&m->H1f, BMAX * DH)) || (rc = alloc(&m->H2f, BMAX * DH)) ||
            (rc = alloc(&m->Y, BMAX * DOUT)) || (rc = alloc(&m->dY, BMAX * DOUT)) ||
            (rc = alloc(&m->dZ2f, BMAX * DH)) || (rc = alloc(&m->dZ1f, BMAX * DH)) ||
            (rc = alloc(&m->H1b, BMAX * DH)) || (rc = alloc(&m->H1Tb, BMAX * DH)) ||
            (rc = alloc(&m->dZ2b, BMAX * DH)) || (rc = alloc(&m->dZ2Tb, BMAX * DH)))
            break;
        if ((rc = st_of(cudaMallocHost(reinterpret_cast<void**>(&m->hbuf), 64 * sizeof(double))))) break;
        if ((rc = alloc(&m->err, 1)) || (rc = st_of(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream))))
            break;
        for (const void* f : {reinterpret_cast<const void*>(k_gemm_tc<EPI_FWD2>),
                              reinterpret_cast<const void*>(k_gemm_tc<EPI_STORE>),
                              reinterpret_cast<const void*>(k_gemm_tc<EPI_BWD1>)})
            if ((rc = st_of(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(TC_SMEM)))))
                break;
        if (rc) break;
        k_init_params<<<(NPARAMS + 255) / 256, 256, 0, m->stream>>>(m->P, seed);
        k_refresh_w2<<<DH * DH / 256, 256, 0, m->stream>>>(m->P, m->W2b, m->W2Tb);
        if ((rc = st_of(cudaMemsetAsync(m->M, 0, NPARAMS * sizeof(float), m->stream))) ||
            (rc = st_of(cudaMemsetAsync(m->V, 0, NPARAMS * sizeof(float), m->stream))) ||
            (rc = st_of(cudaMemsetAsync(m->step, 0, sizeof(int64_t), m->stream))) ||
            (rc = st_of(cudaStreamSynchronize(m->stream))))
            break;
    } while (0);
    if (rc != HAWKES_OK) {
        hawkes_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return HAWKES_OK;
}

void hawkes_mlp_destroy(hawkes_mlp* m) {
    HK_NVTX("hawkes_mlp_destroy");
    if (!m) return;
    DeviceGuard g(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* p : {(void*)m->P, (void*)m->G, (void*)m->M, (void*)m->V, (void*)m->W2b, (void*)m->W2Tb,
                    (void*)m->step, (void*)m->loss, (void*)m->stats, (void*)m->Xs, (void*)m->Ts,
                    (void*)m->X, (void*)m->T, (void*)m->H1f, (void*)m->H2f, (void*)m->Y, (void*)m->dY,
                    (void*)m->dZ2f, (void*)m->dZ1f, (void*)m->H1b, (void*)m->H1Tb, (void*)m->dZ2b,
                    (void*)m->dZ2Tb, (void*)m->err})
        if (p) cudaFree(p);
    if (m->hbuf) cudaFreeHost(m->hbuf);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    cudaGetLastError();
    delete m;
}

int hawkes_mlp_get_params(hawkes_mlp* m, float* params) {
    HK_NVTX("hawkes_mlp_get_params");
    if (!m || !params) return HAWKES_ERR_ARG;
    DeviceGuard g(m->device);
    HM_CUDA(cudaMemcpyAsync(params, m->P, NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    return st_of(cudaStreamSynchronize(m->stream));
}

int hawkes_mlp_set_params(hawkes_mlp* m, const float* params) {
    HK_NVTX("hawkes_mlp_set_params");
    if (!m || !params) return HAWKES_ERR_ARG;
    DeviceGuard g(m->device);
    HM_CUDA(cudaMemcpyAsync(m->P, params, NPARAMS * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    k_refresh_w2<<<DH * DH / 256, 256, 0, m->stream>>>(m->P, m->W2b, m->W2Tb);
    HM_CUDA(cudaMemsetAsync(m->M, 0, NPARAMS * sizeof(float), m->stream));
    HM_CUDA(cudaMemsetAsync(m->V, 0, NPARAMS * sizeof(float), m->stream));
    HM_CUDA(cudaMemsetAsync(m->step, 0, sizeof(int64_t), m->stream));
    return st_of(cudaStreamSynchronize(m->stream));
}

int hawkes_mlp_set_data(hawkes_mlp* m, int64_t n, const double* X, const double* F,
                        const double* Y) {
    HK_NVTX("hawkes_mlp_set_data");
    if (!m || n < 2 || !X || !Y) return HAWKES_ERR_ARG;
    DeviceGuard g(m->device);
    HM_CUDA(cudaStreamSynchronize(m->stream));
    if (m->Xs) cudaFree(m->Xs);
    if (m->Ts) cudaFree(m->Ts);
    m->Xs = m->Ts = nullptr;
    m->have_stats = false;
    double *dX = nullptr, *dY = nullptr, *dF = nullptr;
    int rc = HAWKES_OK;
    if ((rc = alloc(&m->Xs, n * DIN)) || (rc = alloc(&m->Ts, n * DOUT)) || (rc = alloc(&dX, n * 6)) ||
        (rc = alloc(&dY, n * 7)) || (F && (rc = alloc(&dF, n)))) {
        if (dX) cudaFree(dX);
        if (dY) cudaFree(dY);
        if (dF) cudaFree(dF);
        return rc;
    }
    cudaStream_t st = m->stream;
    if ((rc = st_of(cudaMemcpyAsync(dX, X, n * 6 * sizeof(double), cudaMemcpyHostToDevice, st))) == HAWKES_OK &&
        (rc = st_of(cudaMemcpyAsync(dY, Y, n * 7 * sizeof(double), cudaMemcpyHostToDevice, st))) == HAWKES_OK &&
        (!F || (rc = st_of(cudaMemcpyAsync(dF, F, n * sizeof(double), cudaMemcpyHostToDevice, st))) == HAWKES_OK)) {
        k_stats<<<14, 256, 0, st>>>(dX, dY, dF, n, m->stats);
        k_standardise<<<256, 256, 0, st>>>(dX, dY, dF, n, m->stats, m->Xs, m->Ts);
        rc = st_of(cudaStreamSynchronize(st));
    }
    cudaFree(dX);
    cudaFree(dY);
    if (dF) cudaFree(dF);
    if (rc != HAWKES_OK) return rc;
    m->n = n;
    m->have_stats = true;
    m->have_feature = F != nullptr;
    return HAWKES_OK;
}

int hawkes_mlp_train(hawkes_mlp* m, int64_t steps, int batch, double lr, uint64_t seed,
                     double* last_loss) {
    HK_NVTX("hawkes_mlp_train");
    if (!m || steps < 0 || batch < 64 || batch > BMAX || batch % 64 != 0 || !(lr > 0)) return HAWKES_ERR_ARG;
    if (!m->have_stats || !m->Xs) return HAWKES_ERR_STATE;
    DeviceGuard g(m->device);
    for (int64_t s = 0; s < steps; ++s) {
        k_gather<<<(batch + 255) / 256, 256, 0, m->stream>>>(m->Xs, m->Ts, m->n, batch, seed, m->step,
                                                            m->X, m->T, m->loss);
        HM_TRY(forward_backward(m, batch, true));
        k_adam<<<(NPARAMS + 255) / 256, 256, 0, m->stream>>>(m->P, m->G, m->M, m->V, m->step,
                                                             static_cast<float>(lr), m->W2b, m->W2Tb);
        k_step_done<<<1, 32, 0, m->stream>>>(m->step);
    }
    HM_CUDA(cudaGetLastError());
    if (last_loss) {
        HM_CUDA(cudaMemcpyAsync(m->hbuf, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        HM_CUDA(cudaStreamSynchronize(m->stream));
        *last_loss = m->hbuf[0];
    }
    return take_err(m);
}

int hawkes_mlp_loss_grad(hawkes_mlp* m, int batch, const float* Xs, const float* Ts, double* loss,
                         float* grad, float* Y) {
    HK_NVTX("hawkes_mlp_loss_grad");
    if (!m || batch < 64 || batch > BMAX || batch % 64 != 0 || !Xs || !Ts) return HAWKES_ERR_ARG;
    DeviceGuard g(m->device);
    cudaStream_t st = m->stream;
    HM_CUDA(cudaMemcpyAsync(m->X, Xs, batch * DIN * sizeof(float), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->T, Ts, batch * DOUT * sizeof(float), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), st));
    HM_TRY(forward_backward(m, batch, true));
    if (grad) HM_CUDA(cudaMemcpyAsync(grad, m->G, NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (Y) HM_CUDA(cudaMemcpyAsync(Y, m->Y, batch * DOUT * sizeof(float), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(m->hbuf, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = m->hbuf[0];
    return take_err(m);
}

int hawkes_mlp_predict(hawkes_mlp* m, int64_t count, const double* d_logp, const double* d_feature,
                       double* d_out) {
    HK_NVTX("hawkes_mlp_predict");
    if (!m || count < 1 || count > BMAX || !d_logp || !d_out || !hk::aligned8(d_logp) ||
        !hk::aligned8(d_out) || !hk::aligned8(d_feature))
        return HAWKES_ERR_ARG;
    if (!m->have_stats || (d_feature != nullptr) != m->have_feature) return HAWKES_ERR_STATE;
    DeviceGuard g(m->device);
    const int B = static_cast<int>((count + 63) / 64 * 64);
    k_predict_in<<<(B + 255) / 256, 256, 0, m->stream>>>(d_logp, d_feature, count, B, m->stats, m->X);
    HM_TRY(forward_backward(m, B, false));
    k_predict_out<<<static_cast<int>((count * DOUT + 255) / 256), 256, 0, m->stream>>>(m->Y, count, m->stats,
                                                                                     d_out);
    return st_of(cudaGetLastError());
}

int hawkes_mlp_stats(hawkes_mlp* m, double* stats28) {
    HK_NVTX("hawkes_mlp_stats");
    if (!m || !stats28) return HAWKES_ERR_ARG;
    if (!m->have_stats) return HAWKES_ERR_STATE;
    DeviceGuard g(m->device);
    HM_CUDA(cudaMemcpyAsync(stats28, m->stats, 28 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    return st_of(cudaStreamSynchronize(m->stream));
}

int hawkes_mlp_wait(hawkes_mlp* m) {
    HK_NVTX("hawkes_mlp_wait");
    if (!m) return HAWKES_ERR_ARG;
    DeviceGuard g(m->device);
    HM_CUDA(cudaStreamSynchronize(m->stream));
    return take_err(m);
}

}  // extern "C"
