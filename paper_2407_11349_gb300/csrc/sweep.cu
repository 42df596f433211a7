// FP32 pair sweep: the O(N^2) part of the Hawkes log-likelihood (eq. 4) and of
// its gradient, as six moment sums per row.
//
// For every ordered pair (target i, source j) the model has a background term
// (if t_j != t_i) and an excitation term (if t_j < t_i); see Sec. 2.1, eqs.
// 2-3.  With the parameters mu, theta and the normalising constants factored
// out, each row needs
//   SB = sum B',  SBr = sum B' r^2,  SBt = sum B' dt^2       B' = exp(-r^2/2tau_x^2 - dt^2/2tau_t^2)
//   SE = sum E',  SEt = sum E' dt,   SEq = sum E' r^2/s_j^2  E' = s_j^-2 exp(-omega dt - r^2/2h^2 s_j^2)
// from which lambda_i and its six partial derivatives follow in closed form.
//
// Symmetric mode (the whole sum): B' is symmetric in (i, j), so each unordered
// pair j < i is visited once and its B' is added to both row i and row j.  A
// warp holds 32 x R rows in registers; the 32 lanes walk a chunk of 32 source
// columns in rotated order (lane k takes column (k + step) mod 32), so the
// column partial sums travel around the warp by one shuffle per step and end
// at their column's lane.  Tie and triangle masks use the index range
// [lo_i, hi_i) of events with t_j == t_i, computed in FP64 from the sorted
// times, so FP32 rounding never changes an indicator.
//
// Window mode (rows [row_begin, row_end) only, Sec. 2.3.2): every row sweeps
// all sources without the symmetric shortcut.
//
// Precision: pair terms in FP32 with exp2 on the SFU; per-row partials are
// folded into FP64 after every 256-column tile; column partials are added to
// FP64 accumulators per tile.
#include "common.cuh"

namespace hk {

enum { M_NONE = 0, M_LOWER = 1, M_TWO = 2 };

struct RowRegs {
    float t0[R], tp[R], xh[R], xl[R], yh[R], yl[R];
    int lo[R], hi[R];
    float sB[R], sBr[R], sBt[R], sE[R], sEt[R], sEq[R];
};

// One tile of TC source columns against the warp's rows.
//   MASK   M_NONE: every pair valid; M_LOWER: valid iff j < lo_i (lower
//          triangle without ties); M_TWO: background iff j < lo_i or j >= hi_i,
//          excitation iff j < lo_i
//   EXC    evaluate the excitation term (sources strictly earlier)
//   COL    also accumulate the background into the source columns
template <int MASK, bool EXC, bool COL>
__device__ __forceinline__ void tile_pass(const Ev* __restrict__ tile, int j0, int lane,
                                          RowRegs& rr, float om_t, float* __restrict__ colacc) {
#pragma unroll 1
    for (int ch = 0; ch < TC / 32; ++ch) {
        float cB = 0.f, cBr = 0.f, cBt = 0.f;
#pragma unroll 2
        for (int s = 0; s < 32; ++s) {
            const int c = ch * 32 + ((lane + s) & 31);
            const float4 a = reinterpret_cast<const float4*>(tile + c)[0];  // t, xh, yh, beta
            const float4 b = reinterpret_cast<const float4*>(tile + c)[1];  // xl, yl, ce, -
            const int j = j0 + c;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dt = rr.tp[r] - a.x;
                const float dx = (rr.xh[r] - a.y) + (rr.xl[r] - b.x);
                const float dy = (rr.yh[r] - a.z) + (rr.yl[r] - b.y);
                const float r2 = fmaf(dy, dy, dx * dx);
                const float dt2 = dt * dt;
                float B = ex2(-(dt2 + r2));
                if (MASK == M_LOWER) B = (j < rr.lo[r]) ? B : 0.f;
                if (MASK == M_TWO) B = (j < rr.lo[r] || j >= rr.hi[r]) ? B : 0.f;
                rr.sB[r] += B;
                rr.sBr[r] = fmaf(B, r2, rr.sBr[r]);
                rr.sBt[r] = fmaf(B, dt2, rr.sBt[r]);
                if (COL) {
                    cB += B;
                    cBr = fmaf(B, r2, cBr);
                    cBt = fmaf(B, dt2, cBt);
                }
                if (EXC) {
                    const float v = a.w * r2;
                    float E = ex2(b.z - fmaf(om_t, dt, v));
                    if (MASK != M_NONE) E = (j < rr.lo[r]) ? E : 0.f;
                    rr.sE[r] += E;
                    rr.sEt[r] = fmaf(E, dt, rr.sEt[r]);
                    rr.sEq[r] = fmaf(E, v, rr.sEq[r]);
                }
            }
            if (COL) {
                const int src = (lane + 1) & 31;
                cB = __shfl_sync(0xffffffffu, cB, src);
                cBr = __shfl_sync(0xffffffffu, cBr, src);
                cBt = __shfl_sync(0xffffffffu, cBt, src);
            }
        }
        if (COL) {  // lane k now holds column ch*32 + k, summed over the warp's rows
            atomicAdd(colacc + 0 * TC + ch * 32 + lane, cB);
            atomicAdd(colacc + 1 * TC + ch * 32 + lane, cBr);
            atomicAdd(colacc + 2 * TC + ch * 32 + lane, cBt);
        }
    }
}

constexpr size_t SMEM_TILES = 2 * TC * sizeof(Ev);
constexpr size_t SMEM_COLACC = 2 * 3 * TC * sizeof(float);
constexpr size_t SMEM_ROWACC = 6 * R * THREADS * sizeof(double);
constexpr size_t SWEEP_SMEM = SMEM_TILES + SMEM_COLACC + SMEM_ROWACC;

// Persistent sweep.  Work item = one row tile of TR rows; SYM takes them
// largest first (row tile I has I + 1 column-tile strips of work).
template <bool SYM>
__global__ void __launch_bounds__(THREADS, 2)
    k_sweep(const Ev* __restrict__ ev, const int32_t* __restrict__ lo,
            const int32_t* __restrict__ hi, const double* __restrict__ tb,
            const double* __restrict__ cc, double* __restrict__ acc, int* __restrict__ ctr,
            int64_t n, int64_t npad, int64_t row_begin, int64_t row_end, int nitems, int item0) {
    extern __shared__ __align__(128) unsigned char smem[];
    Ev* tiles = reinterpret_cast<Ev*>(smem);
    float* colacc = reinterpret_cast<float*>(smem + SMEM_TILES);
    double* racc = reinterpret_cast<double*>(smem + SMEM_TILES + SMEM_COLACC);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (cc[CC_VALID] == 0.0) return;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    for (int k = tid; k < 2 * 3 * TC; k += THREADS) colacc[k] = 0.f;
    __syncthreads();

    const float om_t = static_cast<float>(cc[CC_OMT]);
    const double kt = cc[CC_KT];
    const double sr = cc[CC_SR], st = cc[CC_ST], set = cc[CC_SET], seq = cc[CC_SEQ];
    const int ncol_tiles = static_cast<int>((n + TC - 1) / TC);
    uint32_t parbits = 0u;   // bit b: parity of the next phase of buffer b
    uint32_t pendbits = 0u;  // thread 0, bit b: a copy into buffer b is in flight

    for (;;) {
        if (tid == 0) s_item = atomicAdd(ctr + CT_WORK, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems || s_abort) break;
        const int64_t I = SYM ? static_cast<int64_t>(nitems - 1 - item) : item0 + item;
        const int64_t rc0 = I * TR;
        const int64_t r0 = rc0 + warp * WROWS;
        const int nJ = SYM ? static_cast<int>((min(rc0 + TR, n) + TC - 1) / TC) : ncol_tiles;

        RowRegs rr;
        bool live = r0 < n;
        if (!SYM) live = live && r0 < row_end && r0 + WROWS > row_begin;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t i = r0 + lane + 32 * r;
            const Ev e = ev[i];
            rr.t0[r] = e.t;
            rr.xh[r] = e.xh; rr.xl[r] = e.xl;
            rr.yh[r] = e.yh; rr.yl[r] = e.yl;
            rr.lo[r] = lo[i];
            rr.hi[r] = hi[i];
            rr.sB[r] = rr.sBr[r] = rr.sBt[r] = rr.sE[r] = rr.sEt[r] = rr.sEq[r] = 0.f;
        }
        const int lo_first = live ? lo[r0] : 0;
        const int hi_last = live ? hi[min(r0 + WROWS, n) - 1] : 0;
        const double trow = tb[r0 / TB];
        for (int k = 0; k < 6 * R; ++k) racc[k * THREADS + tid] = 0.0;

        if (tid == 0) {
            for (int q = 0; q < 2 && q < nJ; ++q) {
                mbar_arrive_expect_tx(&bars[q], TC * sizeof(Ev));
                tma_load_1d(tiles + q * TC, ev + static_cast<int64_t>(q) * TC, TC * sizeof(Ev), &bars[q]);
                pendbits |= 1u << q;
            }
        }

        for (int J = 0; J < nJ; ++J) {
            const int buf = J & 1;
            if (!mbar_wait(&bars[buf], (parbits >> buf) & 1u)) {
                set_error(ctr, HAWKES_ERR_TIMEOUT);
                s_abort = 1;
            }
            parbits ^= 1u << buf;
            pendbits &= ~(1u << buf);
            const int j0 = J * TC;
            if (live) {
                const float dT = static_cast<float>((trow - tb[J]) * kt);
#pragma unroll
                for (int r = 0; r < R; ++r) rr.tp[r] = rr.t0[r] + dT;
                const Ev* tile = tiles + buf * TC;
                float* ca = colacc + buf * 3 * TC;
                if (SYM) {
                    if (j0 < r0 + WROWS) {
                        if (j0 + TC > lo_first)
                            tile_pass<M_LOWER, true, true>(tile, j0, lane, rr, om_t, ca);
                        else
                            tile_pass<M_NONE, true, true>(tile, j0, lane, rr, om_t, ca);
                    }
                } else {
                    if (j0 + TC <= lo_first)
                        tile_pass<M_NONE, true, false>(tile, j0, lane, rr, om_t, ca);
                    else if (j0 >= hi_last)
                        tile_pass<M_NONE, false, false>(tile, j0, lane, rr, om_t, ca);
                    else
                        tile_pass<M_TWO, true, false>(tile, j0, lane, rr, om_t, ca);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double* q = racc + r * THREADS + tid;
                    q[0 * R * THREADS] += static_cast<double>(rr.sB[r]);
                    q[1 * R * THREADS] += static_cast<double>(rr.sBr[r]);
                    q[2 * R * THREADS] += static_cast<double>(rr.sBt[r]);
                    q[3 * R * THREADS] += static_cast<double>(rr.sE[r]);
                    q[4 * R * THREADS] += static_cast<double>(rr.sEt[r]);
                    q[5 * R * THREADS] += static_cast<double>(rr.sEq[r]);
                    rr.sB[r] = rr.sBr[r] = rr.sBt[r] = rr.sE[r] = rr.sEt[r] = rr.sEq[r] = 0.f;
                }
            }
            __syncthreads();
            if (tid == 0 && J + 2 < nJ && !s_abort) {
                mbar_arrive_expect_tx(&bars[buf], TC * sizeof(Ev));
                tma_load_1d(tiles + buf * TC, ev + static_cast<int64_t>(J + 2) * TC, TC * sizeof(Ev),
                            &bars[buf]);
                pendbits |= 1u << buf;
            }
            if (SYM) {
                float* ca = colacc + buf * 3 * TC;
                const float v0 = ca[tid], v1 = ca[TC + tid], v2 = ca[2 * TC + tid];
                if (v0 != 0.f || v1 != 0.f || v2 != 0.f) {
                    const int64_t j = static_cast<int64_t>(j0) + tid;
                    atomicAdd(acc + 0 * npad + j, static_cast<double>(v0));
                    atomicAdd(acc + 1 * npad + j, static_cast<double>(v1) * sr);
                    atomicAdd(acc + 2 * npad + j, static_cast<double>(v2) * st);
                    ca[tid] = 0.f;
                    ca[TC + tid] = 0.f;
                    ca[2 * TC + tid] = 0.f;
                }
            }
            if (s_abort) break;
        }

        if (live && !s_abort) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t i = r0 + lane + 32 * r;
                if (i >= n || (!SYM && (i < row_begin || i >= row_end))) continue;
                const double* q = racc + r * THREADS + tid;
                const double vB = q[0], vBr = q[1 * R * THREADS] * sr, vBt = q[2 * R * THREADS] * st;
                if (SYM) {
                    atomicAdd(acc + 0 * npad + i, vB);
                    atomicAdd(acc + 1 * npad + i, vBr);
                    atomicAdd(acc + 2 * npad + i, vBt);
                } else {
                    acc[0 * npad + i] = vB;
                    acc[1 * npad + i] = vBr;
                    acc[2 * npad + i] = vBt;
                }
                acc[3 * npad + i] = q[3 * R * THREADS];
                acc[4 * npad + i] = q[4 * R * THREADS] * set;
                acc[5 * npad + i] = q[5 * R * THREADS] * seq;
            }
        }
        __syncthreads();
        if (s_abort) break;
    }
    // A wait that gave up may leave bulk copies in flight: let them land
    // (bounded) before the CTA's shared memory is released.
    if (tid == 0)
        for (int q = 0; q < 2; ++q)
            if ((pendbits >> q) & 1u) (void)mbar_wait(&bars[q], (parbits >> q) & 1u);
}

}  // namespace hk

// Host-side launch helpers (called from api.cu).
namespace hk {

cudaError_t sweep_setup_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SWEEP_SMEM));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(SWEEP_SMEM));
}

int sweep_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<true>, THREADS, SWEEP_SMEM) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_sweep(hawkes_ctx* c, bool sym, int64_t row_begin, int64_t row_end) {
    int nitems, item0;
    if (sym) {
        nitems = static_cast<int>(c->npad / TR);
        item0 = 0;
    } else {
        item0 = static_cast<int>(row_begin / TR);
        nitems = static_cast<int>((row_end + TR - 1) / TR) - item0;
    }
    const int grid = nitems < c->sweep_grid ? nitems : c->sweep_grid;
    if (grid <= 0) return cudaSuccess;
    if (sym)
        k_sweep<true><<<grid, THREADS, SWEEP_SMEM, c->stream>>>(c->ev, c->lo, c->hi, c->tb, c->cc,
                                                                c->acc, c->ctr, c->n, c->npad,
                                                                row_begin, row_end, nitems, item0);
    else
        k_sweep<false><<<grid, THREADS, SWEEP_SMEM, c->stream>>>(c->ev, c->lo, c->hi, c->tb, c->cc,
                                                                 c->acc, c->ctr, c->n, c->npad,
                                                                 row_begin, row_end, nitems, item0);
    return cudaGetLastError();
}

}  // namespace hk
