// Exact spatial skip of the pair sweep (flag HAWKES_SKIP_SPATIAL).
//
// At the sizes of the paper most pair terms are exact FP32 zeros because the
// two events are far apart: a background term B' = 2^-(dt~^2 + r~^2) flushes
// to zero once its exponent passes 126, and an excitation term once
// omega~ dt~ + beta r~^2 - ce passes 126 (ex2.approx.ftz).  The symmetric
// sweep visits 256-event tiles in time order, and such a tile spans the whole
// map, so no tile pair is ever entirely zero by distance.  This path orders
// the events so that tiles are compact in space and time, and skips every
// tile pair whose terms are all provably zero:
//   - time windows of about `window` consecutive events, cut only between
//     distinct times (a tie group never straddles two windows);
//   - inside each window, events ordered along a Morton curve of their
//     locations at the time the order is built;
//   - per 256-event tile of that order: the time range and the smallest and
//     largest s_j (fixed), and the bounding box of the current locations
//     (recomputed every call, so a resample moves it with the events);
//   - a tile pair is skipped when, with 2 units of margin, the smallest
//     possible background exponent exceeds 128 and the smallest possible
//     excitation exponent (or the absence of an earlier source) makes every
//     excitation term zero as well.
// The kept pairs are evaluated without the symmetric shortcut (each row
// against the kept column tiles); the tie and causality indicators come from
// each event's index in the time order, carried in its record, so the masks
// are exact.  Times are split into FP32 hi + lo parts like the coordinates,
// because a tile now spans many days.  Row sums go to the FP64 accumulators
// of the events' original indices; finalisation is shared with the other
// paths.  The result equals the full sweep's up to FP32 summation order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sweep_kernel.cuh"

namespace hk {

struct SpatialState {
    int64_t window = 131072;  // target events per time window
    bool built = false;
    int ntiles = 0;           // npad / TC
    int32_t* perm = nullptr;  // [npad] time-order index at each position (-1: padding)
    double* tmeta = nullptr;  // [4 ntiles] time min, time max, s min, s max of each tile
    double* box = nullptr;    // [4 ntiles] x min, x max, y min, y max of the current locations
};

constexpr int SP_CH = THREADS;  // column tiles per work item (one per thread when listing)
constexpr int SP_RP = 4, SP_R = 2 * SP_RP, SP_WROWS = 32 * SP_R, SP_TR = WARPS * SP_WROWS;
static_assert(SP_WROWS == TC, "a warp's rows are one tile of the spatial order");
constexpr int32_t SP_PAD_RANK = 0x7fffffff;

void spatial_free(hawkes_ctx* c) {
    if (!c->sp) return;
    SpatialState* s = c->sp;
    if (s->perm) cudaFree(s->perm);
    if (s->tmeta) cudaFree(s->tmeta);
    if (s->box) cudaFree(s->box);
    delete s;
    c->sp = nullptr;
}

void spatial_invalidate(hawkes_ctx* c) {
    if (c->sp) c->sp->built = false;
}

int spatial_set_window(hawkes_ctx* c, int64_t window) {
    if (window < TC) return HAWKES_ERR_ARG;
    if (!c->sp) {
        c->sp = new (std::nothrow) SpatialState();
        if (!c->sp) return HAWKES_ERR_OOM;
    }
    if (c->sp->window != window) {
        c->sp->window = window;
        c->sp->built = false;
    }
    return HAWKES_OK;
}

static uint32_t spread16(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Build the order and its fixed tile data from the current events
// (synchronous; the locations used for the order are the current ones).
int spatial_build(hawkes_ctx* c) {
    if (!c->sp) {
        const int rc = spatial_set_window(c, 131072);
        if (rc != HAWKES_OK) return rc;
    }
    SpatialState* sp = c->sp;
    if (sp->built) return HAWKES_OK;
    const int64_t n = c->n, npad = c->npad;
    std::vector<double> t(n), x(n), y(n), s(n);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(t.data(), c->t, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(x.data(), c->x, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(y.data(), c->y, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(s.data(), c->s, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
    for (int64_t i = 1; i < n; ++i) {
        x0 = std::min(x0, x[i]); x1 = std::max(x1, x[i]);
        y0 = std::min(y0, y[i]); y1 = std::max(y1, y[i]);
    }
    const double gx = 65535.0 / std::max(x1 - x0, 1e-300), gy = 65535.0 / std::max(y1 - y0, 1e-300);
    std::vector<uint64_t> key(n);
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t cx = static_cast<uint32_t>(std::min(65535.0, std::max(0.0, (x[i] - x0) * gx)));
        const uint32_t cy = static_cast<uint32_t>(std::min(65535.0, std::max(0.0, (y[i] - y0) * gy)));
        key[i] = (static_cast<uint64_t>(spread16(cx) | (spread16(cy) << 1)) << 32) | static_cast<uint64_t>(i);
    }
    std::vector<int32_t> perm(npad, -1);
    for (int64_t a = 0; a < n;) {  // windows cut between distinct times only
        int64_t b = std::min(n, a + sp->window);
        while (b < n && t[b] == t[b - 1]) ++b;
        std::sort(key.begin() + a, key.begin() + b);
        for (int64_t p = a; p < b; ++p) perm[p] = static_cast<int32_t>(key[p] & 0xFFFFFFFFu);
        a = b;
    }
    const int ntiles = static_cast<int>(npad / TC);
    std::vector<double> meta(4 * static_cast<size_t>(ntiles));
    for (int k = 0; k < ntiles; ++k) {
        double t0 = 1e300, t1 = -1e300, s0 = 1e300, s1 = -1e300;
        for (int q = 0; q < TC; ++q) {
            const int32_t e = perm[static_cast<size_t>(k) * TC + q];
            if (e < 0) continue;
            t0 = std::min(t0, t[e]); t1 = std::max(t1, t[e]);
            s0 = std::min(s0, s[e]); s1 = std::max(s1, s[e]);
        }
        meta[4 * k + 0] = t0; meta[4 * k + 1] = t1; meta[4 * k + 2] = s0; meta[4 * k + 3] = s1;
    }
    if (sp->ntiles != ntiles || !sp->perm) {
        if (sp->perm) cudaFree(sp->perm);
        if (sp->tmeta) cudaFree(sp->tmeta);
        if (sp->box) cudaFree(sp->box);
        sp->perm = nullptr; sp->tmeta = nullptr; sp->box = nullptr;
        if (cudaMalloc(&sp->perm, npad * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&sp->tmeta, 4 * static_cast<size_t>(ntiles) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&sp->box, 4 * static_cast<size_t>(ntiles) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return HAWKES_ERR_OOM;
        }
        sp->ntiles = ntiles;
    }
    if (cudaMemcpy(sp->perm, perm.data(), npad * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(sp->tmeta, meta.data(), meta.size() * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return HAWKES_ERR_CUDA;
    sp->built = true;
    return HAWKES_OK;
}

// Stage the records in the spatial order: times relative to their tile's
// earliest time, split into FP32 hi + lo; the time-order index of the event
// in the last word (padding: an index no row ever admits).
__global__ void k_sp_prep(const int32_t* __restrict__ perm, const double* __restrict__ tmeta,
                          const double* __restrict__ t, const double* __restrict__ x,
                          const double* __restrict__ y, const double* __restrict__ s,
                          const double* __restrict__ cc, int model1, int64_t npad, Rec* rec) {
    if (cc[CC_VALID] == 0.0) return;
    const double kx = cc[CC_KX], kt = cc[CC_KT];
    const double beta0 = (cc[CC_TX] * cc[CC_TX]) / (cc[CC_H] * cc[CC_H]);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm[p];
        float4 q0, q1, q2, q3;
        if (e >= 0) {
            const double tt = (t[e] - tmeta[4 * (p / TC)]) * kt;
            const float th = static_cast<float>(tt), tl = static_cast<float>(tt - static_cast<double>(th));
            const double xs = x[e] * kx, ys = y[e] * kx;
            const float xh = static_cast<float>(xs), yh = static_cast<float>(ys);
            const float xl = static_cast<float>(xs - static_cast<double>(xh));
            const float yl = static_cast<float>(ys - static_cast<double>(yh));
            const double se = model1 ? 1.0 : s[e];
            const float nb = -static_cast<float>(beta0 / (se * se));
            const float ce = static_cast<float>(-2.0 * log2(se));
            q0 = make_float4(-th, -th, -xh, -xh);
            q1 = make_float4(-xl, -xl, -yh, -yh);
            q2 = make_float4(-yl, -yl, nb, nb);
            q3 = make_float4(ce, ce, -tl, __int_as_float(e));
        } else {
            q0 = make_float4(-PAD_T, -PAD_T, 0.f, 0.f);
            q1 = make_float4(0.f, 0.f, 0.f, 0.f);
            q2 = make_float4(0.f, 0.f, 0.f, 0.f);
            q3 = make_float4(0.f, 0.f, 0.f, __int_as_float(SP_PAD_RANK));
        }
        *rec_q(rec, p, 0) = q0;
        *rec_q(rec, p, 1) = q1;
        *rec_q(rec, p, 2) = q2;
        *rec_q(rec, p, 3) = q3;
    }
}

// Bounding box of the current locations of each tile of the order (one warp
// per tile).  Tiles of padding only get an empty box (min > max).
__global__ void k_sp_box(const int32_t* __restrict__ perm, const double* __restrict__ x,
                         const double* __restrict__ y, int ntiles, double* box) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < ntiles;
         k += (gridDim.x * blockDim.x) >> 5) {
        double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
        for (int q = lane; q < TC; q += 32) {
            const int32_t e = perm[static_cast<int64_t>(k) * TC + q];
            if (e < 0) continue;
            x0 = fmin(x0, x[e]); x1 = fmax(x1, x[e]);
            y0 = fmin(y0, y[e]); y1 = fmax(y1, y[e]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, o));
            x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, o));
            y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, o));
            y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        }
        if (lane == 0) {
            box[4 * k + 0] = x0; box[4 * k + 1] = x1;
            box[4 * k + 2] = y0; box[4 * k + 3] = y1;
        }
    }
}

// Everything the sweep needs to know about a set of tiles for the zero test.
struct SpRange {
    double x0, x1, y0, y1;  // bounding box (km)
    double t0, t1;          // time range (days)
    double s0, s1;          // s_j range
    bool empty;
};

__device__ __forceinline__ SpRange sp_tile(const double* __restrict__ tmeta,
                                           const double* __restrict__ box, int k) {
    SpRange r;
    r.x0 = box[4 * k + 0]; r.x1 = box[4 * k + 1]; r.y0 = box[4 * k + 2]; r.y1 = box[4 * k + 3];
    r.t0 = tmeta[4 * k + 0]; r.t1 = tmeta[4 * k + 1];
    r.s0 = tmeta[4 * k + 2]; r.s1 = tmeta[4 * k + 3];
    r.empty = !(r.t0 <= r.t1);
    return r;
}

__device__ __forceinline__ void sp_union(SpRange& a, const SpRange& b) {
    if (b.empty) return;
    if (a.empty) {
        a = b;
        return;
    }
    a.x0 = fmin(a.x0, b.x0); a.x1 = fmax(a.x1, b.x1);
    a.y0 = fmin(a.y0, b.y0); a.y1 = fmax(a.y1, b.y1);
    a.t0 = fmin(a.t0, b.t0); a.t1 = fmax(a.t1, b.t1);
    a.s0 = fmin(a.s0, b.s0); a.s1 = fmax(a.s1, b.s1);
}

// True if every background and excitation term of a row in `rw` against a
// source in `col` is an exact FP32 zero (2 units of margin on each exponent).
__device__ __forceinline__ bool sp_all_zero(const SpRange& rw, const SpRange& col,
                                            const double* __restrict__ cc, int model1) {
    if (rw.empty || col.empty) return true;
    const double ax = cc[CC_KX] * cc[CC_KX], kt = cc[CC_KT], omt = cc[CC_OMT];
    const double dx = fmax(0.0, fmax(col.x0 - rw.x1, rw.x0 - col.x1));
    const double dy = fmax(0.0, fmax(col.y0 - rw.y1, rw.y0 - col.y1));
    const double r2 = (dx * dx + dy * dy) * ax;
    const double gap = fmax(0.0, fmax(col.t0 - rw.t1, rw.t0 - col.t1)) * kt;
    if (gap * gap + r2 <= 128.0) return false;
    if (col.t0 >= rw.t1) return true;  // no source earlier than any row: no excitation
    const double causal = fmax(0.0, rw.t0 - col.t1) * kt;
    const double smin = model1 ? 1.0 : col.s0, smax = model1 ? 1.0 : col.s1;
    const double ce_max = -2.0 * log2(smin);
    const double beta_min = (cc[CC_TX] * cc[CC_TX]) / (cc[CC_H] * cc[CC_H] * smax * smax);
    return ce_max - omt * causal - beta_min * r2 < -128.0;
}

// One tile of the spatial order against the warp's rows (no symmetry).
//   MASK  per-pair indicators from the time-order indices (rows' tie ranges
//         [lo, hi) against the source's index); else every pair counts and
//   EXC   says whether the sources are all earlier (excitation) or all later.
template <int UNROLL, bool MASK, bool EXC>
__device__ __forceinline__ void sp_tile_pass(const float4* __restrict__ tile, int lane,
                                             Rows<SP_RP>& rr, const float2 (&tl)[SP_RP],
                                             float2 nomt, const int (&lo)[SP_R],
                                             const int (&hi)[SP_R]) {
#pragma unroll 1
    for (int ch = 0; ch < TC / 32; ++ch) {
#pragma unroll UNROLL
        for (int s = 0; s < 32; ++s) {
            const int c = ch * 32 + ((lane + s) & 31);
            const float4 q0 = tile[0 * TC + c];  // -t, -t, -xh, -xh
            const float4 q1 = tile[1 * TC + c];  // -xl, -xl, -yh, -yh
            const float4 q2 = tile[2 * TC + c];  // -yl, -yl, -beta, -beta
            const float4 q3 = tile[3 * TC + c];  // ce, ce, -t lo, time-order index
            const float2 nT = f2(q0.x, q0.y), nXH = f2(q0.z, q0.w);
            const float2 nXL = f2(q1.x, q1.y), nYH = f2(q1.z, q1.w);
            const float2 nYL = f2(q2.x, q2.y), NB = f2(q2.z, q2.w);
            const float2 CE = f2(q3.x, q3.y), nTL = f2(q3.z, q3.z);
            const int rank = __float_as_int(q3.w);
#pragma unroll
            for (int p = 0; p < SP_RP; ++p) {
                const float2 dt = add2(add2(rr.tp[p], nT), add2(tl[p], nTL));
                const float2 dx = add2(add2(rr.xh[p], nXH), add2(rr.xl[p], nXL));
                const float2 dy = add2(add2(rr.yh[p], nYH), add2(rr.yl[p], nYL));
                const float2 r2 = fma2(dy, dy, mul2(dx, dx));
                const float2 dt2 = mul2(dt, dt);
                const float2 aB = add2(dt2, r2);
                float2 B = f2(ex2(-aB.x), ex2(-aB.y));
                if (MASK) {
                    B.x = (rank < lo[2 * p] || rank >= hi[2 * p]) ? B.x : 0.f;
                    B.y = (rank < lo[2 * p + 1] || rank >= hi[2 * p + 1]) ? B.y : 0.f;
                }
                rr.sB[p] = add2(rr.sB[p], B);
                rr.sBr[p] = fma2(B, r2, rr.sBr[p]);
                rr.sBt[p] = fma2(B, dt2, rr.sBt[p]);
                if (MASK || EXC) {
                    const float2 nv = mul2(NB, r2);
                    const float2 arg = add2(fma2(nomt, dt, nv), CE);
                    float2 E = f2(ex2(arg.x), ex2(arg.y));
                    if (MASK) {
                        E.x = rank < lo[2 * p] ? E.x : 0.f;
                        E.y = rank < lo[2 * p + 1] ? E.y : 0.f;
                    }
                    rr.sE[p] = add2(rr.sE[p], E);
                    rr.sEt[p] = fma2(E, dt, rr.sEt[p]);
                    rr.sEq[p] = fma2(E, nv, rr.sEq[p]);
                }
            }
        }
    }
}

struct SpArgs {
    const Rec* rec;
    const int32_t* lo;
    const int32_t* hi;
    const double* cc;
    double* acc;
    const double* tmeta;
    const double* box;
    int64_t n, npad;
    int ntiles, nI, nch, model1;
    int chunk;  // column tiles per item (<= SP_CH)
};

// Persistent sweep over items (row tile I of the spatial order x a chunk of
// SP_CH column tiles).  The CTA first lists the chunk's column tiles that are
// not entirely zero against its 8 row tiles, then streams only those through
// shared memory (TMA, double-buffered); each warp re-tests them against its
// own row tile.
__global__ void __launch_bounds__(THREADS, 1) k_sweep_sp(SpArgs a, int* __restrict__ ctr, int nitems) {
    extern __shared__ __align__(128) unsigned char smem[];
    Rec* tiles = reinterpret_cast<Rec*>(smem);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_abort, s_nlist;
    __shared__ int s_list[SP_CH];
    __shared__ int s_wcount[WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.cc[CC_VALID] == 0.0) return;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t parbits = 0u, pendbits = 0u;
    const double* cc = a.cc;
    const float omt = static_cast<float>(cc[CC_OMT]);
    const float2 nomt = f2(-omt, -omt);
    const double kt = cc[CC_KT];

    for (;;) {
        if (tid == 0) s_item = atomicAdd(ctr + CT_WORK, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems || s_abort) break;
        const int I = item / a.nch;
        const int cb = (item % a.nch) * a.chunk;
        const int cend = min(cb + a.chunk, a.ntiles);
        // the CTA's rows: tiles 8 I .. 8 I + 7 of the order
        SpRange rows;
        rows.empty = true;
        for (int w = 0; w < WARPS; ++w) sp_union(rows, sp_tile(a.tmeta, a.box, I * WARPS + w));
        // list the chunk's column tiles that can hold a nonzero term
        const int jt_mine = cb + tid;
        const bool keep = jt_mine < cend && !sp_all_zero(rows, sp_tile(a.tmeta, a.box, jt_mine), cc, a.model1);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wcount[warp] = __popc(bal);
        __syncthreads();
        int base = 0;
        for (int w = 0; w < warp; ++w) base += s_wcount[w];
        if (keep) s_list[base + __popc(bal & ((1u << lane) - 1u))] = jt_mine;
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < WARPS; ++w) tot += s_wcount[w];
            s_nlist = tot;
        }
        __syncthreads();
        const int nJ = s_nlist;
        if (nJ == 0) continue;  // the next item is fetched after the barrier at the loop top

        // rows of this warp: one tile of the order
        const int wtile = I * WARPS + warp;
        const int64_t r0 = static_cast<int64_t>(wtile) * TC;
        const SpRange mine = sp_tile(a.tmeta, a.box, wtile);
        const bool live = !mine.empty;
        Rows<SP_RP> rr;
        float t0h[SP_R], t0l[SP_R];
        int lo[SP_R], hi[SP_R], rk[SP_R];
#pragma unroll
        for (int p = 0; p < SP_RP; ++p) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t i = r0 + lane + 64 * p + 32 * h;
                const float4 qa = *rec_q(a.rec, i, 0), qb = *rec_q(a.rec, i, 1);
                const float4 qc = *rec_q(a.rec, i, 2), qd = *rec_q(a.rec, i, 3);
                const int e = __float_as_int(qd.w);
                rk[2 * p + h] = e;
                const bool real = e >= 0 && e < a.n;
                lo[2 * p + h] = real ? a.lo[e] : 0;
                hi[2 * p + h] = real ? a.hi[e] : 0;
                t0h[2 * p + h] = -qa.x;
                t0l[2 * p + h] = -qd.z;
                if (h == 0) {
                    rr.xh[p].x = -qa.z; rr.xl[p].x = -qb.x; rr.yh[p].x = -qb.z; rr.yl[p].x = -qc.x;
                } else {
                    rr.xh[p].y = -qa.z; rr.xl[p].y = -qb.x; rr.yh[p].y = -qb.z; rr.yl[p].y = -qc.x;
                }
            }
            rr.sB[p] = rr.sBr[p] = rr.sBt[p] = rr.sE[p] = rr.sEt[p] = rr.sEq[p] = f2(0.f, 0.f);
        }

        if (tid == 0) {
            for (int q = 0; q < 2 && q < nJ; ++q) {
                mbar_arrive_expect_tx(&bars[q], TC * sizeof(Rec));
                tma_load_1d(tiles + q * TC, a.rec + static_cast<int64_t>(s_list[q]) * TC, TC * sizeof(Rec),
                            &bars[q]);
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
            const int jt = s_list[J];
            const SpRange col = sp_tile(a.tmeta, a.box, jt);
            if (live && !s_abort && !sp_all_zero(mine, col, cc, a.model1)) {
                // row times against this tile's base: two-word sums, exact in the hi part
                const double dT = (mine.t0 - col.t0) * kt;
                const float dTh = static_cast<float>(dT), dTl = static_cast<float>(dT - static_cast<double>(dTh));
                float2 tl[SP_RP];
#pragma unroll
                for (int p = 0; p < SP_RP; ++p) {
                    float hv[2], lv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float u = t0h[2 * p + h], v = dTh;
                        const float sm = __fadd_rn(u, v);
                        const float vb = __fsub_rn(sm, u);
                        const float ua = __fsub_rn(sm, vb);
                        const float err = __fadd_rn(__fsub_rn(u, ua), __fsub_rn(v, vb));
                        hv[h] = sm;
                        lv[h] = __fadd_rn(err, __fadd_rn(t0l[2 * p + h], dTl));
                    }
                    rr.tp[p] = f2(hv[0], hv[1]);
                    tl[p] = f2(lv[0], lv[1]);
                }
                const float4* tile = reinterpret_cast<const float4*>(tiles + buf * TC);
                const bool partial = (static_cast<int64_t>(jt) + 1) * TC > a.n;
                if (!partial && col.t1 < mine.t0)  // every source strictly earlier
                    sp_tile_pass<8, false, true>(tile, lane, rr, tl, nomt, lo, hi);
                else if (!partial && col.t0 > mine.t1)  // every source strictly later
                    sp_tile_pass<8, false, false>(tile, lane, rr, tl, nomt, lo, hi);
                else
                    sp_tile_pass<8, true, true>(tile, lane, rr, tl, nomt, lo, hi);
            }
            __syncthreads();
            if (tid == 0 && J + 2 < nJ && !s_abort) {
                mbar_arrive_expect_tx(&bars[buf], TC * sizeof(Rec));
                tma_load_1d(tiles + buf * TC, a.rec + static_cast<int64_t>(s_list[J + 2]) * TC,
                            TC * sizeof(Rec), &bars[buf]);
                pendbits |= 1u << buf;
            }
            if (s_abort) break;
        }
        if (live && !s_abort) {
            const double sr = cc[CC_SR], st = cc[CC_ST], set = cc[CC_SET], seq = cc[CC_SEQ];
#pragma unroll
            for (int p = 0; p < SP_RP; ++p) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = rk[2 * p + h];
                    if (e < 0 || e >= a.n) continue;
                    const float vB = h ? rr.sB[p].y : rr.sB[p].x, vBr = h ? rr.sBr[p].y : rr.sBr[p].x;
                    const float vBt = h ? rr.sBt[p].y : rr.sBt[p].x, vE = h ? rr.sE[p].y : rr.sE[p].x;
                    const float vEt = h ? rr.sEt[p].y : rr.sEt[p].x, vEq = h ? rr.sEq[p].y : rr.sEq[p].x;
                    if (vB != 0.f || vBr != 0.f || vBt != 0.f) {
                        atomicAdd(a.acc + 0 * a.npad + e, static_cast<double>(vB));
                        atomicAdd(a.acc + 1 * a.npad + e, static_cast<double>(vBr) * sr);
                        atomicAdd(a.acc + 2 * a.npad + e, static_cast<double>(vBt) * st);
                    }
                    if (vE != 0.f || vEt != 0.f || vEq != 0.f) {
                        atomicAdd(a.acc + 3 * a.npad + e, static_cast<double>(vE));
                        atomicAdd(a.acc + 4 * a.npad + e, static_cast<double>(vEt) * set);
                        atomicAdd(a.acc + 5 * a.npad + e, -static_cast<double>(vEq) * seq);
                    }
                }
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

// Queue the spatial path's staging and sweep (after k_prep has written the
// per-call constants and zeroed the accumulators).
cudaError_t spatial_launch(hawkes_ctx* c, int model1) {
    SpatialState* sp = c->sp;
    const int g = c->sms * 8;
    k_sp_prep<<<g, 256, 0, c->stream>>>(sp->perm, sp->tmeta, c->t, c->x, c->y, c->s, c->cc, model1, c->npad,
                                         c->rec);
    k_sp_box<<<(sp->ntiles * 32 + 255) / 256, 256, 0, c->stream>>>(sp->perm, c->x, c->y, sp->ntiles, sp->box);
    SpArgs a;
    a.rec = c->rec; a.lo = c->lo; a.hi = c->hi; a.cc = c->cc; a.acc = c->acc;
    a.tmeta = sp->tmeta; a.box = sp->box; a.n = c->n; a.npad = c->npad;
    a.ntiles = sp->ntiles;
    a.nI = static_cast<int>(c->npad / SP_TR);
    // column chunks of up to SP_CH tiles, halved until there are at least 4
    // items per SM (smaller problems would otherwise leave SMs idle)
    a.chunk = SP_CH;
    while (a.chunk > 32 && static_cast<int64_t>(a.nI) * ((sp->ntiles + a.chunk - 1) / a.chunk) <
                               4LL * c->sms)
        a.chunk /= 2;
    a.nch = (sp->ntiles + a.chunk - 1) / a.chunk;
    a.model1 = model1;
    const int nitems = a.nI * a.nch;
    const size_t smem = 2 * TC * sizeof(Rec);  // 32 KB: below the default dynamic limit
    const int grid = std::min(nitems, c->sms);
    if (grid <= 0) return cudaSuccess;
    k_sweep_sp<<<grid, THREADS, smem, c->stream>>>(a, c->ctr, nitems);
    return cudaGetLastError();
}

}  // namespace hk
