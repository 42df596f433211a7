// Shared definitions of the libhawkes CUDA sources: the context, the staged
// event record, per-call constants and small PTX wrappers (mbarrier, bulk
// TMA copy, SFU exp2).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hawkes.h"

namespace hk {

// ---------------------------------------------------------------------------
// Tiling of the N x N pair matrix.
//   A CTA has WARPS warps; a warp owns 32 x R rows (R per lane, strided by 32,
//   R a kernel-variant parameter).  Source (column) events are streamed
//   through shared memory in tiles of TC events, one TMA bulk copy each, and
//   a work item covers up to CHUNK consecutive tiles.  Times are stored
//   relative to the first event of their block of TB = TC events.  Event
//   arrays are padded to a multiple of NPAD_MULT (the largest row tile).
// ---------------------------------------------------------------------------
// NVTX range around one C-ABI call (visible in Nsight timelines; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define HK_NVTX(name) ::hk::NvtxRange hk_nvtx_range_(name)

// HAWKES_DEBUG build: kernels check the indices they derive from work lists
// and fix-up lists before using them; a failed check latches
// HAWKES_ERR_BOUNDS and skips the access.  Release builds compile the checks
// out.
#ifdef HAWKES_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

// Device pointers handed to the library point at doubles: 8-byte alignment.
inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Every flag bit the log-likelihood calls accept.
constexpr uint32_t kFlagsAll = HAWKES_F64 | HAWKES_MODEL1 | HAWKES_SKIP_UNDERFLOW | HAWKES_BG_TIME |
                               HAWKES_SKIP_SPATIAL | HAWKES_LOGLIK_ONLY;
// The flag bits that k_prep and the FP64 kernels read as the call's model.
constexpr uint32_t kModelBits = HAWKES_MODEL1 | HAWKES_BG_TIME | HAWKES_LOGLIK_ONLY;

struct SpatialState;  // the spatial-skip order of a context (sweep_spatial.cu)

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int TC = 256;
constexpr int TB = TC;
constexpr int CHUNK = 16;
constexpr int NPAD_MULT = 2048;
static_assert(TC == THREADS, "column flush maps one thread to one column");

// Staged per-event record (64 B), rebuilt every call from the FP64 inputs and
// the parameters.  Values are negated and duplicated so that a packed f32x2
// add with a pair of rows forms both differences:
//   q0 = (-t~, -t~, -xh, -xh)   q1 = (-xl, -xl, -yh, -yh)
//   q2 = (-yl, -yl, -beta, -beta)   q3 = (ce, ce, 0, 0)
// with coordinates pre-scaled so that a background exponent is
// -(r~^2 + dt~^2) in base 2:
//   x~ = x sqrt(a_x), a_x = log2(e) / (2 tau_x^2), split hi + lo in FP32
//   t~ = (t - T_block) sqrt(a_t), a_t = log2(e) / (2 tau_t^2)
//   beta = tau_x^2 / (h^2 s^2)    (excitation spatial exponent is beta r~^2)
//   ce = -2 log2(s)               (the 1 / s^2 of the source's density)
// In device memory the records of each tile of TC events are stored as four
// planes, q0[TC] q1[TC] q2[TC] q3[TC], so that lanes reading consecutive
// events touch consecutive 16-byte words (no shared-memory bank conflicts);
// one tile is one contiguous 64 x TC-byte block for the TMA copy.
struct __align__(16) Rec {
    float v[16];
};
static_assert(sizeof(Rec) == 64, "Rec is four 16-byte vectors");

// Address of plane q of event e's record in the tiled layout.
__host__ __device__ __forceinline__ float4* rec_q(Rec* base, int64_t e, int q) {
    return reinterpret_cast<float4*>(base) + (e / TC) * 4 * TC + q * TC + (e % TC);
}
__host__ __device__ __forceinline__ const float4* rec_q(const Rec* base, int64_t e, int q) {
    return reinterpret_cast<const float4*>(base) + (e / TC) * 4 * TC + q * TC + (e % TC);
}

// Time value given to padding events: far after every real event, so that
// every pair term with a padding event is exactly 0 (and finite products).
constexpr float PAD_T = 1.0e15f;

// One problem of the pair sweep: its staged records, tie ranges, time bases,
// per-call constants and accumulators (all device pointers).
struct ProbDesc {
    const double* t;  // FP64 times (for the underflow-skip bounds)
    const Rec* rec;
    const int32_t* lo;
    const int32_t* hi;
    const double* tb;
    const double* cc;
    double* acc;
    int64_t n, npad;
};

// A group of chains with identical event times, swept kc at a time by the
// group kernel (sweep_group.cu): the group's tile records (TC / 2 + 3 kc TC
// float4 per tile of TC events: the shared time plane, then three planes per
// chain), the shared tie ranges and time bases, and each chain's per-call
// constants and FP64 moment accumulators.
constexpr int KMAX = 4;
__host__ __device__ constexpr int gt_f4(int kc) { return TC / 2 + 3 * kc * TC; }
struct GroupDesc {
    const float4* tiles;
    const int32_t* lo;
    const double* tb;
    const double* cc[KMAX];
    double* acc[KMAX];
    int64_t n, npad;
};

// Per-call constants, computed on the device from the parameters.
enum {
    CC_KX = 0,      // sqrt(a_x)
    CC_KT,          // sqrt(a_t)
    CC_OMT,         // omega log2(e) / sqrt(a_t): excitation time exponent per unit t~
    CC_SR,          // 1 / a_x : r~^2 -> r^2
    CC_ST,          // 1 / a_t : t~^2 -> t^2
    CC_SET,         // 1 / sqrt(a_t) : t~ -> t
    CC_SEQ,         // 2 h^2 / log2(e) : beta r~^2 -> r^2 / s^2
    CC_CB,          // background normalisation 1 / ((2 pi)^{3/2} tau_x^2 tau_t)
    CC_CE,          // excitation normalisation omega / (2 pi h^2)
    CC_MU, CC_TX, CC_TT, CC_TH, CC_OM, CC_H,
    CC_TN,          // t_N
    CC_FLAGTHR,     // rows with lambda below this are recomputed in FP64
    CC_SKIPDT,      // > 0: skip tiles whose smallest time gap (scaled) exceeds this
    CC_SKIPDTB,     // the background-only part of that bound (sqrt(128))
    CC_VALID,       // 1 if the parameters are valid
    CC_CEMAX,       // max(0, max_j ce_j) of the call's model (0 for Model 1)
    CC_BGT,         // 1 for the time-only background
    CC_LLONLY,      // 1 when only the log-likelihood is evaluated
    CC_FTHR,        // [7] flush-bound thresholds per output (< 0: nothing to recompute)
    CC_COUNT = CC_FTHR + 7
};

// Per-block partials of k_finalize: the 7 outputs, then the 7 flush bounds.
constexpr int PART_STRIDE = 16;
// fix7 buffer: [0, 8) sums over rows recomputed because their rate is near the
// FP32 floor, [8, 16) corrections of rows recomputed because of the flush bound.
constexpr int FIX_DOUBLES = 16;
// Relative share of an output's magnitude that the bound on the FP32 sweep's
// flushed terms may reach before the rows that carry it are recomputed in FP64.
constexpr double FLUSH_TAU = 1e-8;

// Device counters.
enum {
    CT_WORK = 0,    // persistent work-queue cursor
    CT_FIX,         // number of rows queued for FP64 recomputation
    CT_ERR,         // latched error status (0 or a HAWKES_ERR_* value)
    CT_DONE,        // finished-block counter
    CT_CEMAX,       // bits of max(0, max_j -2 log2 s_j), set when the events are loaded
    CT_COUNT = 8
};

constexpr double LOG2E = 1.4426950408889634;
constexpr double CLIP = 1e-40;
constexpr double TWO_PI = 6.283185307179586;

// Bounded waits: a wait on an mbarrier gives up after WAIT_CYCLES SM clock
// cycles (about 2 s at 2 GHz) or SPIN_LIMIT polls, whichever comes first.
constexpr long long SPIN_LIMIT = 1ll << 30;
constexpr long long WAIT_CYCLES = 4000000000ll;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared through the TMA unit; completion
// is signalled on `bar` as transferred bytes.  Addresses 16-byte aligned,
// size a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete; false if the bounded wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (long long k = 0; k < SPIN_LIMIT; ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 63) == 63 && clock64() - t0 > WAIT_CYCLES) return false;
    }
    return false;
}

// 2^x on the special-function unit; results below 2^-126 flush to zero.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void set_error(int* ctr, int code) {
    atomicCAS(ctr + CT_ERR, 0, code);
}

}  // namespace hk

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct hawkes_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;

    int64_t n = 0, npad = 0;
    int32_t n_counties = 0;
    int64_t nblk = 0;

    double* t = nullptr;       // [npad] FP64 times (padding = t_N)
    double* x = nullptr;       // [npad] current locations
    double* y = nullptr;
    double* s = nullptr;       // [npad] per-event source scale
    double* scale_c = nullptr; // [n_counties]
    int32_t* county = nullptr; // [n]
    int32_t* lo = nullptr;     // [npad] first index with t_j == t_i
    int32_t* hi = nullptr;     // [npad] one past the last index with t_j == t_i
    double* tb = nullptr;      // [npad / TB] block time bases
    hk::Rec* rec = nullptr;    // [npad] staged FP32 records
    int4* items = nullptr;     // symmetric-sweep work list
    int nitems = 0;
    int items_variant = -1;    // variant the work list was built for
    int variant = 0;           // sweep kernel variant in use
    int variant_bpsm = 1;      // its resident CTAs per SM
    double* acc = nullptr;     // [6 * npad] per-row moment sums (natural units)
    double* partials = nullptr;// [final_blocks * 8]
    double* fix7 = nullptr;    // [8] sums over FP64-recomputed rows
    int* fixlist = nullptr;    // [npad]
    int* ctr = nullptr;        // [CT_COUNT]
    double* cc = nullptr;      // [CC_COUNT]
    hawkes_params* params_dev = nullptr;
    double* out_dev = nullptr; // [8]
    double* out_host = nullptr;// pinned [8]
    double* rows9 = nullptr;   // [9 * n] optional per-row output (allocated on demand)
    int64_t rows9_cap = 0;
    int final_blocks = 0;

    int32_t n_tri = 0;
    bool counties_ok = false;
    int32_t* tri_county = nullptr;
    double* tri_xy = nullptr;
    double* tri_cum = nullptr;
    int32_t* cfirst = nullptr;
    int32_t* clast = nullptr;

    bool prof = false;
    cudaEvent_t pev[2] = {nullptr, nullptr};
    hawkes_profile pacc{};

    hk::SpatialState* sp = nullptr;  // HAWKES_SKIP_SPATIAL order (built on first use)

    // Work list of one shard of the symmetric sweep (hawkes_shard_moments),
    // for (nshards, shard, variant) = shard_key; rebuilt when any changes.
    int4* shard_items = nullptr;
    int shard_nitems = 0;
    int shard_key[3] = {-1, -1, -1};
};
