// FP32 pair sweep: the O(N^2) part of the Hawkes log-likelihood (eq. 4) and of
// its gradient, as six moment sums per row.
//
// For every ordered pair (target i, source j) the model has a background term
// (if t_j != t_i) and an excitation term (if t_j < t_i); see Sec. 2.1, eqs.
// 2-3.  With mu, theta and the normalising constants factored out, each row
// needs
//   SB = sum B',  SBr = sum B' r^2,  SBt = sum B' dt^2       B' = exp(-r^2/2tau_x^2 - dt^2/2tau_t^2)
//   SE = sum E',  SEt = sum E' dt,   SEq = sum E' r^2/s_j^2  E' = s_j^-2 exp(-omega dt - r^2/2h^2 s_j^2)
// from which lambda_i and its six partial derivatives follow in closed form.
//
// Symmetric mode (the whole sum): B' is symmetric in (i, j), so each unordered
// pair j < i is visited once and its B' is added to both row i and row j.  A
// warp holds 32 x R rows in registers, two rows per packed f32x2 register
// pair, so every pair operation is one FFMA2/FADD2/FMUL2 for two rows.  The
// 32 lanes walk a chunk of 32 source columns in rotated order (lane k takes
// column (k + step) mod 32), so the column partial sums travel around the
// warp by one shuffle per step and end at their column's lane.  Source
// records hold negated, duplicated values, so every difference is a packed
// add with the column value already in both halves.
//
// Tie and triangle masks use the index range [lo_i, hi_i) of events with
// t_j == t_i, computed in FP64 from the sorted times, so FP32 rounding never
// changes an indicator.
//
// Window mode (rows [row_begin, row_end) only, Sec. 2.3.2): every row sweeps
// all sources without the symmetric shortcut.
//
// Time-only background (eq. 2 as printed, flag HAWKES_BG_TIME): B' keeps only
// its time factor, so the pair loop drops r^2 from the background exponent
// and the SBr moment; the excitation is unchanged.  The flag is a template
// parameter, so the default kernels are compiled exactly as without it.
//
// Log-likelihood only (flag HAWKES_LOGLIK_ONLY, template parameter LL): the
// rows keep SB and SE, the columns SB, and the other moments are not formed
// (13 algorithmic FP32 operations per unordered pair instead of 19).
//
// Work is split into items (row tile x chunk of column tiles) taken from an
// atomic queue, longest first.  Pair terms are FP32 with exp2 on the SFU;
// row sums are FP32 within an item (CHUNK x TC sources) and FP64 across
// items; column sums are FP32 within a tile and FP64 across tiles.
#pragma once
#include "common.cuh"

namespace hk {

enum { M_NONE = 0, M_LOWER = 1, M_TWO = 2 };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int RP>
struct Rows {
    float2 tp[RP], xh[RP], xl[RP], yh[RP], yl[RP];
    float2 sB[RP], sBr[RP], sBt[RP], sE[RP], sEt[RP], sEq[RP];
};

// One tile of TC source columns against the warp's 2 RP rows per lane.
//   MASK   M_NONE: every pair valid; M_LOWER: valid iff j < lo_i (lower
//          triangle without ties); M_TWO: background iff j < lo_i or
//          j >= hi_i, excitation iff j < lo_i
//   EXC    evaluate the excitation term (sources strictly earlier)
//   COL    also accumulate the background into the source columns
//   BGT    time-only background (eq. 2): B' = exp(-dt^2/2tau_t^2), no SBr
//   LL     log-likelihood only: SB and SE (and the column SB) alone
// rlo/rhi: shared-memory lo/hi of the lane's rows (masked tiles only).
// racc: the thread's FP32 row accumulators in shared memory (see fold_rows;
// time-only background only).
//
// Summation order.  An FP32 running sum of many equal terms drifts by a
// rounding bias that grows with the length of the chain.  With the time-only
// background every pair at the same time gap has the same B', and
// integer-day times make whole runs of them, so the BGT kernels keep every
// chain short: a row's register sums cover one 32-column chunk before they
// are folded into racc, and a column's sum takes each step's 2 RP rows as one
// partial (at N = 100,000 on integer days this takes the d/dtau_t error from
// 8e-5 to 7e-7 of its value).  With the space-time background the spatial
// factor makes the terms differ and the plain chains stay within 2e-7 of the
// FP64 path up to N = 1,000,000 on integer days, so those kernels keep the
// cheaper order.
__device__ __forceinline__ void fold2(float4* q, float2 a, float2 b) {
    const float4 v = *q;
    const float2 lo = add2(f2(v.x, v.y), a), hi = add2(f2(v.z, v.w), b);
    *q = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// racc layout per thread (stride THREADS float4): for each row pair p,
// (SB, SBr), (SBt, SE), (SEt, SEq), each a float2 over the pair's two rows.
template <int RP>
__device__ __forceinline__ void fold_rows(Rows<RP>& rr, float4* __restrict__ racc) {
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        fold2(racc + (3 * p + 0) * THREADS, rr.sB[p], rr.sBr[p]);
        fold2(racc + (3 * p + 1) * THREADS, rr.sBt[p], rr.sE[p]);
        fold2(racc + (3 * p + 2) * THREADS, rr.sEt[p], rr.sEq[p]);
        rr.sB[p] = rr.sBr[p] = rr.sBt[p] = rr.sE[p] = rr.sEt[p] = rr.sEq[p] = f2(0.f, 0.f);
    }
}

template <int RP, int UNROLL, int MASK, bool EXC, bool COL, bool BGT, bool LL>
__device__ __forceinline__ void tile_pass(const float4* __restrict__ tile, int j0, int lane,
                                          Rows<RP>& rr, float2 nomt,
                                          const int* __restrict__ rlo,
                                          const int* __restrict__ rhi, float* __restrict__ colacc,
                                          float4* __restrict__ racc) {
#pragma unroll 1
    for (int ch = 0; ch < TC / 32; ++ch) {
        float2 cB = f2(0.f, 0.f), cBr = f2(0.f, 0.f), cBt = f2(0.f, 0.f);
#pragma unroll UNROLL
        for (int s = 0; s < 32; ++s) {
            const int c = ch * 32 + ((lane + s) & 31);
            const float4 q0 = tile[0 * TC + c];  // -t, -t, -xh, -xh
            const float4 q1 = tile[1 * TC + c];  // -xl, -xl, -yh, -yh
            const float4 q2 = tile[2 * TC + c];  // -yl, -yl, -beta, -beta
            const float4 q3 = tile[3 * TC + c];  // ce, ce, -, -
            const float2 nT = f2(q0.x, q0.y), nXH = f2(q0.z, q0.w);
            const float2 nXL = f2(q1.x, q1.y), nYH = f2(q1.z, q1.w);
            const float2 nYL = f2(q2.x, q2.y), NB = f2(q2.z, q2.w);
            const float2 CE = f2(q3.x, q3.y);
            const int j = j0 + c;
            float2 pB, pBt;  // BGT: this step's column partial over the lane's rows
#pragma unroll
            for (int p = 0; p < RP; ++p) {
                const float2 dt = add2(rr.tp[p], nT);
                const float2 dx = add2(add2(rr.xh[p], nXH), add2(rr.xl[p], nXL));
                const float2 dy = add2(add2(rr.yh[p], nYH), add2(rr.yl[p], nYL));
                const float2 r2 = fma2(dy, dy, mul2(dx, dx));
                const float2 dt2 = mul2(dt, dt);
                const float2 aB = BGT ? dt2 : add2(dt2, r2);
                float2 B = f2(ex2(-aB.x), ex2(-aB.y));
                if (MASK != M_NONE) {
                    const int l0 = rlo[2 * p], l1 = rlo[2 * p + 1];
                    if (MASK == M_LOWER) {
                        B.x = (j < l0) ? B.x : 0.f;
                        B.y = (j < l1) ? B.y : 0.f;
                    } else {
                        B.x = (j < l0 || j >= rhi[2 * p]) ? B.x : 0.f;
                        B.y = (j < l1 || j >= rhi[2 * p + 1]) ? B.y : 0.f;
                    }
                }
                rr.sB[p] = add2(rr.sB[p], B);
                if (!BGT && !LL) rr.sBr[p] = fma2(B, r2, rr.sBr[p]);
                if (!LL) rr.sBt[p] = fma2(B, dt2, rr.sBt[p]);
                if (COL && !BGT) {
                    cB = add2(cB, B);
                    if (!LL) {
                        cBr = fma2(B, r2, cBr);
                        cBt = fma2(B, dt2, cBt);
                    }
                }
                if (COL && BGT) {  // per-step partial (no SBr moment here)
                    pB = (p == 0) ? B : add2(pB, B);
                    if (!LL) pBt = (p == 0) ? mul2(B, dt2) : fma2(B, dt2, pBt);
                }
                if (EXC) {
                    const float2 nv = mul2(NB, r2);                  // -beta r~^2
                    const float2 arg = add2(fma2(nomt, dt, nv), CE); // ce - omega~ dt - beta r~^2
                    float2 E = f2(ex2(arg.x), ex2(arg.y));
                    if (MASK != M_NONE) {
                        E.x = (j < rlo[2 * p]) ? E.x : 0.f;
                        E.y = (j < rlo[2 * p + 1]) ? E.y : 0.f;
                    }
                    rr.sE[p] = add2(rr.sE[p], E);
                    if (!LL) {
                        rr.sEt[p] = fma2(E, dt, rr.sEt[p]);
                        rr.sEq[p] = fma2(E, nv, rr.sEq[p]);  // accumulates -sum E beta r~^2
                    }
                }
            }
            if (COL) {
                if (BGT) {
                    cB = add2(cB, pB);
                    if (!LL) cBt = add2(cBt, pBt);
                }
                const int src = (lane + 1) & 31;
                cB.x = __shfl_sync(0xffffffffu, cB.x, src);
                cB.y = __shfl_sync(0xffffffffu, cB.y, src);
                if (!BGT && !LL) {
                    cBr.x = __shfl_sync(0xffffffffu, cBr.x, src);
                    cBr.y = __shfl_sync(0xffffffffu, cBr.y, src);
                }
                if (!LL) {
                    cBt.x = __shfl_sync(0xffffffffu, cBt.x, src);
                    cBt.y = __shfl_sync(0xffffffffu, cBt.y, src);
                }
            }
        }
        if (COL) {  // lane k now holds column ch*32 + k, summed over the warp's rows
            atomicAdd(colacc + 0 * TC + ch * 32 + lane, cB.x + cB.y);
            if (!BGT && !LL) atomicAdd(colacc + 1 * TC + ch * 32 + lane, cBr.x + cBr.y);
            if (!LL) atomicAdd(colacc + 2 * TC + ch * 32 + lane, cBt.x + cBt.y);
        }
        if (BGT) fold_rows<RP>(rr, racc);
    }
}

template <int RP>
struct Geo {
    static constexpr int R = 2 * RP;          // rows per lane
    static constexpr int WROWS = 32 * R;      // rows per warp
    static constexpr int TR = WARPS * WROWS;  // rows per row tile
    static_assert(TB % WROWS == 0, "a warp's rows share one time block");
    static constexpr size_t SMEM_TILES = 2 * TC * sizeof(Rec);
    static constexpr size_t SMEM_COLACC = 2 * 3 * TC * sizeof(float);
    static constexpr size_t SMEM_LOHI = 2 * THREADS * R * sizeof(int);
    static constexpr size_t SMEM_RACC = 3 * RP * THREADS * sizeof(float4);  // BGT kernels only
    static constexpr size_t SMEM = SMEM_TILES + SMEM_COLACC + SMEM_LOHI;
    static constexpr size_t smem(bool bgt) { return SMEM + (bgt ? SMEM_RACC : 0); }
};

enum { MODE_WIN = 0, MODE_SYM = 1, MODE_BATCH = 2 };

// Persistent sweep over work items.
//   MODE_SYM:   item k = items[k] = (row tile, first column tile, end column
//               tile) of problem `one`
//   MODE_BATCH: as MODE_SYM, item.w = index into probs[] (many problems, one
//               launch, one queue)
//   MODE_WIN:   item k -> row tile item0 + k / nch, column chunk k % nch of
//               problem `one`, rows [row_begin, row_end) only
// In MODE_BATCH, nch is the number of problems (checked in debug builds).
template <int RP, int MINB, int UNROLL, int MODE, bool BGT, bool LL>
__global__ void __launch_bounds__(THREADS, MINB)
    k_sweep(ProbDesc one, const ProbDesc* __restrict__ probs, const int4* __restrict__ items,
            int nitems, int* __restrict__ ctr, int64_t row_begin, int64_t row_end, int item0,
            int nch) {
    using G = Geo<RP>;
    constexpr int R = G::R;
    constexpr bool SYM = MODE != MODE_WIN;
    extern __shared__ __align__(128) unsigned char smem[];
    Rec* tiles = reinterpret_cast<Rec*>(smem);
    float* colacc = reinterpret_cast<float*>(smem + G::SMEM_TILES);
    int* slo = reinterpret_cast<int*>(smem + G::SMEM_TILES + G::SMEM_COLACC);
    int* shi = slo + THREADS * R;
    float4* racc = reinterpret_cast<float4*>(smem + G::SMEM_TILES + G::SMEM_COLACC + G::SMEM_LOHI) +
                   threadIdx.x;
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_abort, s_bad;
    // The current item's problem.  In batch mode it is re-read from shared
    // memory (volatile: not kept in registers) wherever it is needed outside
    // the pair loop, so the pair loop is compiled as in the one-problem modes.
    __shared__ __align__(16) ProbDesc s_pd;
    volatile ProbDesc* vpd = &s_pd;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (MODE != MODE_BATCH && one.cc[CC_VALID] == 0.0) return;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    for (int k = tid; k < 2 * 3 * TC; k += THREADS) colacc[k] = 0.f;
    __syncthreads();

    uint32_t parbits = 0u;   // bit b: parity of the next phase of buffer b
    uint32_t pendbits = 0u;  // thread 0, bit b: a copy into buffer b is in flight
    int* mylo = slo + tid * R;
    int* myhi = shi + tid * R;

    for (;;) {
        if (tid == 0) {
            const int k = atomicAdd(ctr + CT_WORK, 1);
            s_item = k;
            if (kDebug) s_bad = 0;
            if (kDebug && MODE == MODE_BATCH && k < nitems && !(items[k].w >= 0 && items[k].w < nch)) {
                s_bad = 1;  // problem index out of range: do not read its descriptor
            } else if (MODE == MODE_BATCH && k < nitems) {
                const ProbDesc d = probs[items[k].w];
                // every field the item reads (the times for the underflow skip)
                vpd->t = d.t; vpd->rec = d.rec; vpd->lo = d.lo; vpd->hi = d.hi; vpd->tb = d.tb;
                vpd->cc = d.cc; vpd->acc = d.acc; vpd->n = d.n; vpd->npad = d.npad;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems || s_abort) break;
        int64_t I;
        int jb, je;
#define HK_PD(field) (MODE == MODE_BATCH ? vpd->field : one.field)
        if (SYM) {
            const int4 it = items[item];
            I = it.x;
            jb = it.y;
            je = it.z;
        } else {
            const int ncol_tiles = static_cast<int>((one.n + TC - 1) / TC);
            I = item0 + item / nch;
            jb = (item % nch) * CHUNK;
            je = min(jb + CHUNK, ncol_tiles);
        }
        if (kDebug) {  // the item must lie inside its problem's causal triangle
            bool ok = !s_bad;
            const int64_t nn = ok ? HK_PD(n) : 0, np = ok ? HK_PD(npad) : 0;
            const int64_t nI = (nn + G::TR - 1) / G::TR;
            const int64_t rows_end = SYM ? min((I + 1) * G::TR, nn) : nn;
            const int64_t jmax = (rows_end + TC - 1) / TC;
            ok = ok && I >= 0 && I < nI && (I + 1) * G::TR <= np && jb >= 0 && jb < je &&
                 je <= jmax && static_cast<int64_t>(je) * TC <= np;
            if (!ok) {
                if (tid == 0) set_error(ctr, HAWKES_ERR_BOUNDS);
                __syncthreads();
                continue;
            }
        }
        const double* cc = HK_PD(cc);
        if (MODE == MODE_BATCH && cc[CC_VALID] == 0.0) {  // problem with invalid parameters
            __syncthreads();
            continue;
        }
        const float omt = static_cast<float>(cc[CC_OMT]);
        const float2 nomt = f2(-omt, -omt);
        const double kt = cc[CC_KT];
        const int64_t n = HK_PD(n);
        const double skipdt = cc[CC_SKIPDT], skipdtb = cc[CC_SKIPDTB];
        if (SYM && skipdt > 0.0) {  // whole item below the FP32 underflow bound
            const double* tt = HK_PD(t);
            const int64_t lastc = min(static_cast<int64_t>(je) * TC, n) - 1;
            const double gap = (tt[min(I * G::TR, n - 1)] - tt[lastc]) * kt;
            if (gap > skipdt) {
                __syncthreads();
                continue;
            }
        }

        const int64_t r0 = I * G::TR + warp * G::WROWS;  // warp's first row
        bool live = r0 < n;
        if (!SYM) live = live && r0 < row_end && r0 + G::WROWS > row_begin;

        Rows<RP> rr;
        float t0[R];
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            const Rec* rec = HK_PD(rec);
            const int32_t* plo = HK_PD(lo);
            const int32_t* phi = HK_PD(hi);
            const int64_t i0 = r0 + lane + 64 * p, i1 = i0 + 32;
            const float4 a0 = *rec_q(rec, i0, 0), b0 = *rec_q(rec, i0, 1), c0 = *rec_q(rec, i0, 2);
            const float4 a1 = *rec_q(rec, i1, 0), b1 = *rec_q(rec, i1, 1), c1 = *rec_q(rec, i1, 2);
            t0[2 * p] = -a0.x;
            t0[2 * p + 1] = -a1.x;
            rr.xh[p] = f2(-a0.z, -a1.z);
            rr.xl[p] = f2(-b0.x, -b1.x);
            rr.yh[p] = f2(-b0.z, -b1.z);
            rr.yl[p] = f2(-c0.x, -c1.x);
            rr.sB[p] = rr.sBr[p] = rr.sBt[p] = rr.sE[p] = rr.sEt[p] = rr.sEq[p] = f2(0.f, 0.f);
            if (BGT)
                for (int q = 0; q < 3; ++q) racc[(3 * p + q) * THREADS] = make_float4(0.f, 0.f, 0.f, 0.f);
            mylo[2 * p] = plo[i0];
            mylo[2 * p + 1] = plo[i1];
            myhi[2 * p] = phi[i0];
            myhi[2 * p + 1] = phi[i1];
        }
        const int lo_first = live ? HK_PD(lo)[r0] : 0;
        const int hi_last = live ? HK_PD(hi)[min(r0 + G::WROWS, n) - 1] : 0;
        const double trow = HK_PD(tb)[r0 / TB];
        const int nJ = je - jb;

        if (tid == 0) {
            for (int q = 0; q < 2 && q < nJ; ++q) {
                mbar_arrive_expect_tx(&bars[q], TC * sizeof(Rec));
                tma_load_1d(tiles + q * TC, HK_PD(rec) + static_cast<int64_t>(jb + q) * TC,
                            TC * sizeof(Rec), &bars[q]);
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
            const int jt = jb + J;
            const int j0 = jt * TC;
            bool run = live;
            if (live && skipdt > 0.0) {  // this warp's rows against this tile
                const double* tt = HK_PD(t);
                const int64_t rl = min(r0 + G::WROWS, n) - 1;
                const int64_t cf = j0, cl = min(static_cast<int64_t>(j0) + TC, n) - 1;
                const double before = (tt[r0] - tt[cl]) * kt;   // columns entirely earlier
                const double after = (tt[cf] - tt[rl]) * kt;    // columns entirely later
                if (before > skipdt || (after > skipdtb)) run = false;
            }
            if (run) {
                const float dT = static_cast<float>((trow - HK_PD(tb)[jt]) * kt);
#pragma unroll
                for (int p = 0; p < RP; ++p) rr.tp[p] = f2(t0[2 * p] + dT, t0[2 * p + 1] + dT);
                const float4* tile = reinterpret_cast<const float4*>(tiles + buf * TC);
                float* ca = colacc + buf * 3 * TC;
                if (SYM) {
                    if (j0 < r0 + G::WROWS) {
                        if (j0 + TC > lo_first)
                            tile_pass<RP, UNROLL, M_LOWER, true, true, BGT, LL>(tile, j0, lane, rr, nomt, mylo, myhi, ca, racc);
                        else
                            tile_pass<RP, UNROLL, M_NONE, true, true, BGT, LL>(tile, j0, lane, rr, nomt, mylo, myhi, ca, racc);
                    }
                } else {
                    if (j0 + TC <= lo_first)
                        tile_pass<RP, UNROLL, M_NONE, true, false, BGT, LL>(tile, j0, lane, rr, nomt, mylo, myhi, ca, racc);
                    else if (j0 >= hi_last)
                        tile_pass<RP, UNROLL, M_NONE, false, false, BGT, LL>(tile, j0, lane, rr, nomt, mylo, myhi, ca, racc);
                    else
                        tile_pass<RP, UNROLL, M_TWO, true, false, BGT, LL>(tile, j0, lane, rr, nomt, mylo, myhi, ca, racc);
                }
            }
            __syncthreads();
            if (tid == 0 && J + 2 < nJ && !s_abort) {
                mbar_arrive_expect_tx(&bars[buf], TC * sizeof(Rec));
                tma_load_1d(tiles + buf * TC, HK_PD(rec) + static_cast<int64_t>(jt + 2) * TC,
                            TC * sizeof(Rec), &bars[buf]);
                pendbits |= 1u << buf;
            }
            if (SYM) {
                float* ca = colacc + buf * 3 * TC;
                const float v0 = ca[tid], v1 = ca[TC + tid], v2 = ca[2 * TC + tid];
                if (v0 != 0.f || v1 != 0.f || v2 != 0.f) {
                    const int64_t j = static_cast<int64_t>(j0) + tid;
                    double* acc = HK_PD(acc);
                    const int64_t npad = HK_PD(npad);
                    atomicAdd(acc + 0 * npad + j, static_cast<double>(v0));
                    if (!LL) {
                        atomicAdd(acc + 1 * npad + j, static_cast<double>(v1) * cc[CC_SR]);
                        atomicAdd(acc + 2 * npad + j, static_cast<double>(v2) * cc[CC_ST]);
                    }
                    ca[tid] = 0.f;
                    ca[TC + tid] = 0.f;
                    ca[2 * TC + tid] = 0.f;
                }
            }
            if (s_abort) break;
        }

        if (live && !s_abort) {
            double* acc = HK_PD(acc);
            const int64_t npad = HK_PD(npad);
            const double sr = cc[CC_SR], st = cc[CC_ST], set = cc[CC_SET], seq = cc[CC_SEQ];
#pragma unroll
            for (int p = 0; p < RP; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t i = r0 + lane + 64 * p + 32 * h;
                    if (i >= n || (!SYM && (i < row_begin || i >= row_end))) continue;
                    float vB, vBr, vBt, vE, vEt, vEq;
                    if (BGT) {  // racc holds (SB, SBr), (SBt, SE), (SEt, SEq) of rows (x, y)
                        const float4 a = racc[(3 * p + 0) * THREADS];
                        const float4 b = racc[(3 * p + 1) * THREADS];
                        const float4 e = racc[(3 * p + 2) * THREADS];
                        vB = h ? a.y : a.x; vBr = h ? a.w : a.z;
                        vBt = h ? b.y : b.x; vE = h ? b.w : b.z;
                        vEt = h ? e.y : e.x; vEq = h ? e.w : e.z;
                    } else {
                        vB = h ? rr.sB[p].y : rr.sB[p].x;
                        vBr = h ? rr.sBr[p].y : rr.sBr[p].x;
                        vBt = h ? rr.sBt[p].y : rr.sBt[p].x;
                        vE = h ? rr.sE[p].y : rr.sE[p].x;
                        vEt = h ? rr.sEt[p].y : rr.sEt[p].x;
                        vEq = h ? rr.sEq[p].y : rr.sEq[p].x;
                    }
                    if (LL) {
                        if (vB != 0.f) atomicAdd(acc + 0 * npad + i, static_cast<double>(vB));
                        if (vE != 0.f) atomicAdd(acc + 3 * npad + i, static_cast<double>(vE));
                        continue;
                    }
                    if (vB != 0.f || vBr != 0.f || vBt != 0.f) {
                        atomicAdd(acc + 0 * npad + i, static_cast<double>(vB));
                        atomicAdd(acc + 1 * npad + i, static_cast<double>(vBr) * sr);
                        atomicAdd(acc + 2 * npad + i, static_cast<double>(vBt) * st);
                    }
                    if (vE != 0.f || vEt != 0.f || vEq != 0.f) {
                        atomicAdd(acc + 3 * npad + i, static_cast<double>(vE));
                        atomicAdd(acc + 4 * npad + i, static_cast<double>(vEt) * set);
                        atomicAdd(acc + 5 * npad + i, -static_cast<double>(vEq) * seq);
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
#undef HK_PD
    }
    // A wait that gave up may leave bulk copies in flight: let them land
    // (bounded) before the CTA's shared memory is released.
    if (tid == 0)
        for (int q = 0; q < 2; ++q)
            if ((pendbits >> q) & 1u) (void)mbar_wait(&bars[q], (parbits >> q) & 1u);
}

// ---------------------------------------------------------------------------
// Kernel tables.  Each translation unit that expands HK_SWEEP_VARIANTS(BGT, LL)
// instantiates one kernel family (space-time background, time-only
// background, log-likelihood only), so the families compile in parallel.
// ---------------------------------------------------------------------------
using SweepFn = void (*)(ProbDesc, const ProbDesc*, const int4*, int, int*, int64_t, int64_t, int,
                         int);

struct Variant {
    int rp, minb;
    SweepFn win, sym, batch;
    size_t smem;
    int tr;
};

#define HK_VARIANT(RP, MINB, U, BGT, LL)                                                      \
    {RP, MINB, k_sweep<RP, MINB, U, MODE_WIN, BGT, LL>, k_sweep<RP, MINB, U, MODE_SYM, BGT, LL>, \
     k_sweep<RP, MINB, U, MODE_BATCH, BGT, LL>, Geo<RP>::smem(BGT), Geo<RP>::TR}
// (rows-per-lane pairs, resident CTAs per SM, unroll of the 32-step pair loop)
#define HK_SWEEP_VARIANTS(BGT, LL)                                                           \
    {HK_VARIANT(4, 1, 8, BGT, LL), HK_VARIANT(4, 1, 16, BGT, LL), HK_VARIANT(4, 1, 32, BGT, LL), \
     HK_VARIANT(4, 1, 4, BGT, LL), HK_VARIANT(2, 2, 8, BGT, LL)}
constexpr int kNumVariants = 5;

// The time-only background's table and the log-likelihood-only table (same
// order as the default one).
const Variant* sweep_variants_bgt();
const Variant* sweep_variants_ll();

}  // namespace hk
