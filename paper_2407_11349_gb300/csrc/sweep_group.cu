// Batched pair sweep with several chains per CTA.
//
// MCMC chains of one data set share their event times (and so their tie
// ranges and time blocks) and differ in their location draws (Sec. 2.2) and
// parameters.  A group of KC such chains is swept by one kernel in which each
// CTA takes a row tile of the shared event order and streams the matching
// column tiles of all KC chains through shared memory in one TMA copy per
// tile.  For every pair the time difference and its square are formed once
// and serve all KC chains; each chain adds its own spatial difference,
// exponents and moments (Sec. 2.1, eqs. 2-3, as in sweep_kernel.cuh).
//
// Times are therefore carried unscaled (days, relative to each 256-event
// block's FP64 base), and each chain's background exponent is formed as
// fma(dt^2, a_t, r~^2) with its own a_t = log2(e) / (2 tau_t^2); the
// excitation exponent is ce - omega log2(e) dt - beta r~^2.  Per unordered
// pair and chain this is 21 executed FP32 lane ops plus 2 / KC for the shared
// dt and dt^2, against 23 for one chain per CTA.
//
// Group tile layout (device memory and shared memory alike), per tile of TC
// events, in float4 units:
//   [0, TC/2)                       the time plane: (-tau, -tau) per event
//   [TC/2 + (3k + q) TC, ... + TC)   chain k, plane q:
//        q = 0: (-xh, -xh, -xl, -xl)   q = 1: (-yh, -yh, -yl, -yl)
//        q = 2: (-beta, -beta, ce, ce)
// with the spatial values of the chain's own staged records (k_prep).
// Symmetric mode only: each unordered pair j < i is visited once, the
// background added to row i and to column j, the excitation to row i.
#include <algorithm>
#include <vector>

#include "sweep_kernel.cuh"

namespace hk {

struct GroupStage {
    const Rec* rec[KMAX];  // each chain's staged records (k_prep)
    const double* t;       // the shared FP64 times
};

// Repack the chains' staged records into the group tile layout.
__global__ void k_group_stage(GroupStage gs, GroupDesc gd, int kc, float4* __restrict__ out) {
    const int64_t n = gd.n, npad = gd.npad;
    const int gt = gt_f4(kc);
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < npad;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float4* base = out + (e / TC) * gt;
        const int c = static_cast<int>(e % TC);
        const float nt = e < n ? -static_cast<float>(gs.t[e] - gd.tb[e / TB]) : -PAD_T;
        reinterpret_cast<float2*>(base)[c] = make_float2(nt, nt);
        for (int k = 0; k < kc; ++k) {
            const float4 a = *rec_q(gs.rec[k], e, 0);  // (-t~, -t~, -xh, -xh)
            const float4 b = *rec_q(gs.rec[k], e, 1);  // (-xl, -xl, -yh, -yh)
            const float4 q = *rec_q(gs.rec[k], e, 2);  // (-yl, -yl, -beta, -beta)
            const float4 d = *rec_q(gs.rec[k], e, 3);  // (ce, ce, 0, 0)
            base[TC / 2 + (3 * k + 0) * TC + c] = make_float4(a.z, a.z, b.x, b.x);
            base[TC / 2 + (3 * k + 1) * TC + c] = make_float4(b.z, b.z, q.x, q.x);
            base[TC / 2 + (3 * k + 2) * TC + c] = make_float4(q.z, q.z, d.x, d.x);
        }
    }
}

template <int RPC, int KC>
struct GRows {
    float2 tp[RPC];
    float2 xh[KC][RPC], xl[KC][RPC], yh[KC][RPC], yl[KC][RPC];
    float2 sB[KC][RPC], sBr[KC][RPC], sBt[KC][RPC], sE[KC][RPC], sEt[KC][RPC], sEq[KC][RPC];
};

// One tile of TC source columns against the warp's 2 RPC rows per lane, for
// all KC chains.  MASK M_NONE: every pair valid; M_LOWER: valid iff
// j < lo_i.  at / nomt: each chain's a_t and -omega log2(e), duplicated.
template <int RPC, int KC, int UNROLL, int MASK>
__device__ __forceinline__ void gtile_pass(const float4* __restrict__ tile, int j0, int lane,
                                           GRows<RPC, KC>& rr, const float2 (&at)[KC],
                                           const float2 (&nomt)[KC], const int* __restrict__ rlo,
                                           float* __restrict__ colacc) {
    const float2* tT = reinterpret_cast<const float2*>(tile);
    const float4* tC = tile + TC / 2;
#pragma unroll 1
    for (int ch = 0; ch < TC / 32; ++ch) {
        float2 cB[KC], cBr[KC], cBt[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) cB[k] = cBr[k] = cBt[k] = f2(0.f, 0.f);
#pragma unroll UNROLL
        for (int s = 0; s < 32; ++s) {
            const int c = ch * 32 + ((lane + s) & 31);
            const int j = j0 + c;
            const float2 nT = tT[c];
            float4 q0[KC], q1[KC], q2[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                q0[k] = tC[(3 * k + 0) * TC + c];
                q1[k] = tC[(3 * k + 1) * TC + c];
                q2[k] = tC[(3 * k + 2) * TC + c];
            }
#pragma unroll
            for (int p = 0; p < RPC; ++p) {
                const float2 dt = add2(rr.tp[p], nT);
                const float2 dt2 = mul2(dt, dt);
                bool v0 = true, v1 = true;
                if (MASK == M_LOWER) {
                    v0 = j < rlo[2 * p];
                    v1 = j < rlo[2 * p + 1];
                }
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    const float2 nXH = f2(q0[k].x, q0[k].y), nXL = f2(q0[k].z, q0[k].w);
                    const float2 nYH = f2(q1[k].x, q1[k].y), nYL = f2(q1[k].z, q1[k].w);
                    const float2 NB = f2(q2[k].x, q2[k].y), CE = f2(q2[k].z, q2[k].w);
                    const float2 dx = add2(add2(rr.xh[k][p], nXH), add2(rr.xl[k][p], nXL));
                    const float2 dy = add2(add2(rr.yh[k][p], nYH), add2(rr.yl[k][p], nYL));
                    const float2 r2 = fma2(dy, dy, mul2(dx, dx));
                    const float2 aB = fma2(dt2, at[k], r2);
                    float2 B = f2(ex2(-aB.x), ex2(-aB.y));
                    if (MASK == M_LOWER) {
                        B.x = v0 ? B.x : 0.f;
                        B.y = v1 ? B.y : 0.f;
                    }
                    rr.sB[k][p] = add2(rr.sB[k][p], B);
                    rr.sBr[k][p] = fma2(B, r2, rr.sBr[k][p]);
                    rr.sBt[k][p] = fma2(B, dt2, rr.sBt[k][p]);
                    cB[k] = add2(cB[k], B);
                    cBr[k] = fma2(B, r2, cBr[k]);
                    cBt[k] = fma2(B, dt2, cBt[k]);
                    const float2 nv = mul2(NB, r2);                      // -beta r~^2
                    const float2 arg = add2(fma2(nomt[k], dt, nv), CE);  // ce - omega' dt - beta r~^2
                    float2 E = f2(ex2(arg.x), ex2(arg.y));
                    if (MASK == M_LOWER) {
                        E.x = v0 ? E.x : 0.f;
                        E.y = v1 ? E.y : 0.f;
                    }
                    rr.sE[k][p] = add2(rr.sE[k][p], E);
                    rr.sEt[k][p] = fma2(E, dt, rr.sEt[k][p]);
                    rr.sEq[k][p] = fma2(E, nv, rr.sEq[k][p]);  // accumulates -sum E beta r~^2
                }
            }
            const int src = (lane + 1) & 31;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                cB[k].x = __shfl_sync(0xffffffffu, cB[k].x, src);
                cB[k].y = __shfl_sync(0xffffffffu, cB[k].y, src);
                cBr[k].x = __shfl_sync(0xffffffffu, cBr[k].x, src);
                cBr[k].y = __shfl_sync(0xffffffffu, cBr[k].y, src);
                cBt[k].x = __shfl_sync(0xffffffffu, cBt[k].x, src);
                cBt[k].y = __shfl_sync(0xffffffffu, cBt[k].y, src);
            }
        }
        // lane l now holds column ch*32 + l, summed over the warp's rows
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            atomicAdd(colacc + (3 * k + 0) * TC + ch * 32 + lane, cB[k].x + cB[k].y);
            atomicAdd(colacc + (3 * k + 1) * TC + ch * 32 + lane, cBr[k].x + cBr[k].y);
            atomicAdd(colacc + (3 * k + 2) * TC + ch * 32 + lane, cBt[k].x + cBt[k].y);
        }
    }
}

template <int RPC, int KC>
struct GGeo {
    static constexpr int R = 2 * RPC;
    static constexpr int WROWS = 32 * R;
    static constexpr int TR = WARPS * WROWS;
    static_assert(TB % WROWS == 0, "a warp's rows share one time block");
    static_assert(NPAD_MULT % TR == 0, "row tiles cover the padded arrays");
    static constexpr int GT = gt_f4(KC);
    static constexpr size_t SMEM_TILES = 2 * GT * sizeof(float4);
    static constexpr size_t SMEM_COLACC = 2 * 3 * KC * TC * sizeof(float);
    static constexpr size_t SMEM_LO = THREADS * R * sizeof(int);
    static constexpr size_t SMEM = SMEM_TILES + SMEM_COLACC + SMEM_LO;
};

// Persistent sweep over group items: item k = (row tile, first column tile,
// end column tile, group).  ctr[CT_WORK] is the work cursor.
template <int RPC, int KC, int UNROLL>
__global__ void __launch_bounds__(THREADS, 1)
    k_sweep_group(const GroupDesc* __restrict__ groups, int ngroups, const int4* __restrict__ items,
                  int nitems, int* __restrict__ ctr) {
    using G = GGeo<RPC, KC>;
    constexpr int R = G::R;
    constexpr int GT = G::GT;
    extern __shared__ __align__(128) unsigned char smem[];
    float4* tiles = reinterpret_cast<float4*>(smem);
    float* colacc = reinterpret_cast<float*>(smem + G::SMEM_TILES);
    int* slo = reinterpret_cast<int*>(smem + G::SMEM_TILES + G::SMEM_COLACC);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_abort, s_bad;
    // The current item's group.  Read through a volatile pointer wherever it
    // is needed outside the pair loop, so that the pair loop keeps its
    // registers for the rows.
    __shared__ __align__(16) GroupDesc s_gd;
    volatile GroupDesc* vgd = &s_gd;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    for (int k = tid; k < 2 * 3 * KC * TC; k += THREADS) colacc[k] = 0.f;
    __syncthreads();

    uint32_t parbits = 0u;   // bit b: parity of the next phase of buffer b
    uint32_t pendbits = 0u;  // thread 0, bit b: a copy into buffer b is in flight
    int* mylo = slo + tid * R;

    for (;;) {
        if (tid == 0) {
            const int k = atomicAdd(ctr + CT_WORK, 1);
            s_item = k;
            s_bad = 0;
            if (k < nitems) {
                const int g = items[k].w;
                if (kDebug && !(g >= 0 && g < ngroups)) {
                    s_bad = 1;  // group index out of range: do not read its descriptor
                } else {
                    const GroupDesc d = groups[g];
                    vgd->tiles = d.tiles; vgd->lo = d.lo; vgd->tb = d.tb;
                    for (int q = 0; q < KMAX; ++q) {
                        vgd->cc[q] = d.cc[q];
                        vgd->acc[q] = d.acc[q];
                    }
                    vgd->n = d.n; vgd->npad = d.npad;
                }
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nitems || s_abort) break;
        const int4 it = items[item];
        const int64_t I = it.x;
        const int jb = it.y, je = it.z;
        if (kDebug) {  // the item must lie inside its group's causal triangle
            bool ok = !s_bad;
            const int64_t nn = ok ? vgd->n : 0, np = ok ? vgd->npad : 0;
            const int64_t nI = (nn + G::TR - 1) / G::TR;
            const int64_t rows_end = (I + 1) * G::TR < nn ? (I + 1) * G::TR : nn;
            const int64_t jmax = (rows_end + TC - 1) / TC;
            ok = ok && I >= 0 && I < nI && (I + 1) * G::TR <= np && jb >= 0 && jb < je &&
                 je <= jmax && static_cast<int64_t>(je) * TC <= np;
            if (!ok) {
                if (tid == 0) set_error(ctr, HAWKES_ERR_BOUNDS);
                __syncthreads();
                continue;
            }
        }
        const int64_t n = vgd->n;
        float2 at[KC], nomt[KC];
        bool valid[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const double* cc = vgd->cc[k];
            valid[k] = cc[CC_VALID] != 0.0;
            const double kt = cc[CC_KT];
            const float a = valid[k] ? static_cast<float>(kt * kt) : 1.f;
            const float w = valid[k] ? -static_cast<float>(cc[CC_OM] * LOG2E) : -1.f;
            at[k] = f2(a, a);
            nomt[k] = f2(w, w);
        }

        const int64_t r0 = I * G::TR + warp * G::WROWS;  // warp's first row
        const bool live = r0 < n;
        const float4* gtiles = vgd->tiles;

        GRows<RPC, KC> rr;
        float t0[R];
#pragma unroll
        for (int p = 0; p < RPC; ++p) {
            const int64_t i0 = r0 + lane + 64 * p, i1 = i0 + 32;
            const float4* b0 = gtiles + (i0 / TC) * GT;  // both rows lie in one tile
            const int c0 = static_cast<int>(i0 % TC), c1 = static_cast<int>(i1 % TC);
            t0[2 * p] = -reinterpret_cast<const float2*>(b0)[c0].x;
            t0[2 * p + 1] = -reinterpret_cast<const float2*>(b0)[c1].x;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const float4* pl = b0 + TC / 2 + 3 * k * TC;
                const float4 a0 = pl[c0], a1 = pl[c1];
                const float4 e0 = pl[TC + c0], e1 = pl[TC + c1];
                rr.xh[k][p] = f2(-a0.x, -a1.x);
                rr.xl[k][p] = f2(-a0.z, -a1.z);
                rr.yh[k][p] = f2(-e0.x, -e1.x);
                rr.yl[k][p] = f2(-e0.z, -e1.z);
                rr.sB[k][p] = rr.sBr[k][p] = rr.sBt[k][p] = f2(0.f, 0.f);
                rr.sE[k][p] = rr.sEt[k][p] = rr.sEq[k][p] = f2(0.f, 0.f);
            }
            const int32_t* plo = vgd->lo;
            mylo[2 * p] = plo[i0];
            mylo[2 * p + 1] = plo[i1];
        }
        const int lo_first = live ? vgd->lo[r0] : 0;
        const double trow = vgd->tb[r0 / TB];
        const int nJ = je - jb;

        if (tid == 0) {
            for (int q = 0; q < 2 && q < nJ; ++q) {
                mbar_arrive_expect_tx(&bars[q], GT * sizeof(float4));
                tma_load_1d(tiles + q * GT, gtiles + static_cast<int64_t>(jb + q) * GT,
                            GT * sizeof(float4), &bars[q]);
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
            float* ca = colacc + buf * 3 * KC * TC;
            if (live && j0 < r0 + G::WROWS) {
                const float dT = static_cast<float>(trow - vgd->tb[jt]);
#pragma unroll
                for (int p = 0; p < RPC; ++p) rr.tp[p] = f2(t0[2 * p] + dT, t0[2 * p + 1] + dT);
                const float4* tile = tiles + buf * GT;
                if (j0 + TC > lo_first)
                    gtile_pass<RPC, KC, UNROLL, M_LOWER>(tile, j0, lane, rr, at, nomt, mylo, ca);
                else
                    gtile_pass<RPC, KC, UNROLL, M_NONE>(tile, j0, lane, rr, at, nomt, mylo, ca);
            }
            __syncthreads();
            if (tid == 0 && J + 2 < nJ && !s_abort) {
                mbar_arrive_expect_tx(&bars[buf], GT * sizeof(float4));
                tma_load_1d(tiles + buf * GT, gtiles + static_cast<int64_t>(jt + 2) * GT,
                            GT * sizeof(float4), &bars[buf]);
                pendbits |= 1u << buf;
            }
            // column sums of this tile, one thread per column, chain by chain
            const int64_t npad = vgd->npad;
            const int64_t j = static_cast<int64_t>(j0) + tid;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                float* ck = ca + 3 * k * TC;
                const float v0 = ck[tid], v1 = ck[TC + tid], v2 = ck[2 * TC + tid];
                if (v0 != 0.f || v1 != 0.f || v2 != 0.f) {
                    if (valid[k]) {
                        double* acc = vgd->acc[k];
                        atomicAdd(acc + 0 * npad + j, static_cast<double>(v0));
                        atomicAdd(acc + 1 * npad + j, static_cast<double>(v1) * vgd->cc[k][CC_SR]);
                        atomicAdd(acc + 2 * npad + j, static_cast<double>(v2));
                    }
                    ck[tid] = 0.f;
                    ck[TC + tid] = 0.f;
                    ck[2 * TC + tid] = 0.f;
                }
            }
            if (s_abort) break;
        }

        if (live && !s_abort) {
            const int64_t npad = vgd->npad;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                if (!valid[k]) continue;
                double* acc = vgd->acc[k];
                const double sr = vgd->cc[k][CC_SR], seq = vgd->cc[k][CC_SEQ];
#pragma unroll
                for (int p = 0; p < RPC; ++p) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int64_t i = r0 + lane + 64 * p + 32 * h;
                        if (i >= n) continue;
                        const float vB = h ? rr.sB[k][p].y : rr.sB[k][p].x;
                        const float vBr = h ? rr.sBr[k][p].y : rr.sBr[k][p].x;
                        const float vBt = h ? rr.sBt[k][p].y : rr.sBt[k][p].x;
                        const float vE = h ? rr.sE[k][p].y : rr.sE[k][p].x;
                        const float vEt = h ? rr.sEt[k][p].y : rr.sEt[k][p].x;
                        const float vEq = h ? rr.sEq[k][p].y : rr.sEq[k][p].x;
                        if (vB != 0.f || vBr != 0.f || vBt != 0.f) {
                            atomicAdd(acc + 0 * npad + i, static_cast<double>(vB));
                            atomicAdd(acc + 1 * npad + i, static_cast<double>(vBr) * sr);
                            atomicAdd(acc + 2 * npad + i, static_cast<double>(vBt));
                        }
                        if (vE != 0.f || vEt != 0.f || vEq != 0.f) {
                            atomicAdd(acc + 3 * npad + i, static_cast<double>(vE));
                            atomicAdd(acc + 4 * npad + i, static_cast<double>(vEt));
                            atomicAdd(acc + 5 * npad + i, -static_cast<double>(vEq) * seq);
                        }
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using GroupFn = void (*)(const GroupDesc*, int, const int4*, int, int*);

struct GroupVariant {
    int kc, rpc;
    GroupFn fn;
    size_t smem;
    int tr;
};

#define HK_GROUP_VARIANT(RPC, KC, U) \
    {KC, RPC, k_sweep_group<RPC, KC, U>, GGeo<RPC, KC>::SMEM, GGeo<RPC, KC>::TR}
// (rows-per-lane pairs, chains per CTA, unroll of the 32-step pair loop)
static const GroupVariant kGroupVariants[] = {HK_GROUP_VARIANT(2, 2, 8), HK_GROUP_VARIANT(1, 4, 8)};

static const GroupVariant* group_variant(int kc) {
    for (const GroupVariant& v : kGroupVariants)
        if (v.kc == kc) return &v;
    return nullptr;
}

bool group_kc_supported(int kc) { return group_variant(kc) != nullptr; }
int group_tile_rows(int kc) { return group_variant(kc)->tr; }
size_t group_tile_bytes(int kc) { return static_cast<size_t>(gt_f4(kc)) * sizeof(float4); }

cudaError_t group_setup_attributes() {
    for (const GroupVariant& v : kGroupVariants) {
        const cudaError_t e = cudaFuncSetAttribute(
            v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(v.smem));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int group_blocks_per_sm(int kc) {
    const GroupVariant* v = group_variant(kc);
    int nb = 0;
    if (!v || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, v->fn, THREADS, v->smem) !=
                  cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

// Work list of the groups (sizes ns[]) for kc chains per CTA: items (row
// tile, column tiles [jb, je), group) in chunks of `chunk` column tiles,
// longest first over all groups (ties: later row tiles first).
std::vector<int4> group_items(const std::vector<int64_t>& ns, int kc, int chunk) {
    const int tr = group_tile_rows(kc);
    std::vector<int4> items;
    for (size_t g = 0; g < ns.size(); ++g) {
        const int64_t n = ns[g];
        const int64_t nI = (n + tr - 1) / tr;
        for (int64_t I = 0; I < nI; ++I) {
            const int nJ = static_cast<int>((std::min<int64_t>((I + 1) * tr, n) + TC - 1) / TC);
            for (int jb = 0; jb < nJ; jb += chunk)
                items.push_back(make_int4(static_cast<int>(I), jb, std::min(jb + chunk, nJ),
                                          static_cast<int>(g)));
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& b) {
        return (a.z - a.y) > (b.z - b.y) || ((a.z - a.y) == (b.z - b.y) && a.x > b.x);
    });
    return items;
}

// Stage group g's tiles from its chains' records (k_prep must have run).
cudaError_t launch_group_stage(cudaStream_t st, int sms, const GroupDesc& gd,
                               const Rec* const* recs, const double* t, int kc, float4* out) {
    GroupStage gs{};
    for (int k = 0; k < kc; ++k) gs.rec[k] = recs[k];
    gs.t = t;
    int g = static_cast<int>((gd.npad + 255) / 256);
    if (g > 8 * sms) g = 8 * sms;
    k_group_stage<<<g, 256, 0, st>>>(gs, gd, kc, out);
    return cudaGetLastError();
}

// One persistent launch over the group items; ctr[CT_WORK] must be zero.
cudaError_t launch_sweep_group(cudaStream_t st, int kc, int grid, const GroupDesc* groups,
                               int ngroups, const int4* items, int nitems, int* ctr) {
    const GroupVariant* v = group_variant(kc);
    if (!v) return cudaErrorInvalidValue;
    if (grid > nitems) grid = nitems;
    if (grid <= 0) return cudaSuccess;
    v->fn<<<grid, THREADS, v->smem, st>>>(groups, ngroups, items, nitems, ctr);
    return cudaGetLastError();
}

}  // namespace hk
