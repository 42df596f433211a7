// O(N) kernels around the pair sweep: event set-up (validation, tie ranges,
// time blocks), per-call staging of the FP32 event table, the FP64 pair rows,
// per-row finalisation (lambda_i, Lambda_i, the gradient of eq. 4), the
// global reduction, and the cut-posterior location resample (Sec. 2.2).
#include <math_constants.h>

#include "common.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// Set-up: validate the events, per-event source scale, tie ranges, bases.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t lower_bound_d(const double* a, int64_t n, double v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t upper_bound_d(const double* a, int64_t n, double v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_setup(double* t, double* x, double* y, const int32_t* county, int32_t nc,
                        const double* scale_c, int64_t n, int64_t npad, int xy_given, double* s,
                        int32_t* lo, int32_t* hi, double* tb, int* ctr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n) {
            const double te = t[e];
            if (!(te > 0.0) || !isfinite(te) || (e + 1 < n && !(te <= t[e + 1])))
                set_error(ctr, HAWKES_ERR_UNSORTED);
            const int32_t c = county[e];
            double se = 1.0;
            if (c < 0 || c >= nc) set_error(ctr, HAWKES_ERR_ARG);
            else se = scale_c[c];
            if (!(se > 0.0) || !isfinite(se)) set_error(ctr, HAWKES_ERR_ARG);
            s[e] = se;
            const float ce = static_cast<float>(-2.0 * log2(se));
            if (ce > 0.f) atomicMax(ctr + CT_CEMAX, __float_as_int(ce));
            if (xy_given) {
                if (!isfinite(x[e]) || !isfinite(y[e])) set_error(ctr, HAWKES_ERR_ARG);
            } else {
                x[e] = 0.0;
                y[e] = 0.0;
            }
            lo[e] = static_cast<int32_t>(lower_bound_d(t, n, te));
            hi[e] = static_cast<int32_t>(upper_bound_d(t, n, te));
        } else {
            t[e] = t[n - 1];
            x[e] = 0.0;
            y[e] = 0.0;
            s[e] = 1.0;
            lo[e] = 0;
            hi[e] = 0;
        }
        if (e % TB == 0) tb[e / TB] = t[e < n ? e : n - 1];
    }
}

// ---------------------------------------------------------------------------
// Per-call constants (every thread derives them; block 0 publishes them).
// ---------------------------------------------------------------------------
struct Consts {
    double mu, tx, tt, th, om, h;
    double kx, kt, omt, sr, st, set, seq, cB, cE;
    bool valid;
};

__device__ __forceinline__ Consts make_consts(const hawkes_params* P, bool bg_time) {
    Consts k;
    k.mu = P->mu; k.tx = P->tau_x; k.tt = P->tau_t; k.th = P->theta; k.om = P->omega; k.h = P->h;
    k.valid = isfinite(k.mu) && isfinite(k.tx) && isfinite(k.tt) && isfinite(k.th) &&
              isfinite(k.om) && isfinite(k.h) && k.mu >= 0.0 && k.th >= 0.0 && k.tx > 0.0 &&
              k.tt > 0.0 && k.om > 0.0 && k.h > 0.0;
    const double ax = LOG2E / (2.0 * k.tx * k.tx), at = LOG2E / (2.0 * k.tt * k.tt);
    k.kx = sqrt(ax);
    k.kt = sqrt(at);
    k.omt = k.om * LOG2E / k.kt;
    k.sr = 1.0 / ax;
    k.st = 1.0 / at;
    k.set = 1.0 / k.kt;
    k.seq = 2.0 * k.h * k.h / LOG2E;
    // Space-time background phi2(r; tau_x) phi1(dt; tau_t), or the time-only
    // background phi1(dt; tau_t) / tau_x^2 (eq. 2, tau_x^2 read as the area).
    k.cB = bg_time ? 1.0 / (sqrt(TWO_PI) * k.tx * k.tx * k.tt)
                   : 1.0 / (TWO_PI * sqrt(TWO_PI) * k.tx * k.tx * k.tt);
    k.cE = k.om / (TWO_PI * k.h * k.h);
    return k;
}

// Zero the accumulators, reset the counters and (FP32 path) stage the event table.
// model: the HAWKES_MODEL1, HAWKES_BG_TIME and HAWKES_LOGLIK_ONLY bits of the
// call's flags.
// skip: evaluate only tiles whose terms can be nonzero in FP32 (see CC_SKIPDT).
__global__ void k_prep(const double* __restrict__ t, const double* __restrict__ x,
                       const double* __restrict__ y, const double* __restrict__ s,
                       const double* __restrict__ tb, const hawkes_params* P, int model,
                       int stage, int skip, int64_t n, int64_t npad, Rec* __restrict__ rec,
                       double* __restrict__ acc, double* __restrict__ cc, int* ctr,
                       double* fix7) {
    const bool model1 = (model & HAWKES_MODEL1) != 0;
    const Consts k = make_consts(P, (model & HAWKES_BG_TIME) != 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cc[CC_KX] = k.kx; cc[CC_KT] = k.kt; cc[CC_OMT] = k.omt;
        cc[CC_SR] = k.sr; cc[CC_ST] = k.st; cc[CC_SET] = k.set; cc[CC_SEQ] = k.seq;
        cc[CC_CB] = k.cB; cc[CC_CE] = k.cE;
        cc[CC_MU] = k.mu; cc[CC_TX] = k.tx; cc[CC_TT] = k.tt;
        cc[CC_TH] = k.th; cc[CC_OM] = k.om; cc[CC_H] = k.h;
        cc[CC_TN] = t[n - 1];
        // Terms below 2^-126 flush to zero in the FP32 path; rows whose rate is
        // within 1e9 x (n such terms) of that are recomputed in FP64.
        cc[CC_FLAGTHR] = 1e9 * (double)n * 1.1754943508222875e-38 * (k.mu * k.cB + k.th * k.cE);
        // A background term is exactly 0 in FP32 (flush to zero) when its
        // base-2 exponent dt~^2 + r~^2 exceeds 126; an excitation term when
        // omega~ dt~ + beta r~^2 - ce exceeds 126.  With 2 units of margin, a
        // tile whose smallest scaled time gap exceeds both bounds contributes
        // exactly nothing.
        const double cemax = model1 ? 0.0 : static_cast<double>(__int_as_float(ctr[CT_CEMAX]));
        cc[CC_SKIPDTB] = skip ? sqrt(128.0) : 0.0;
        cc[CC_SKIPDT] = skip ? fmax(sqrt(128.0), (cemax + 128.0) / k.omt) : 0.0;
        cc[CC_VALID] = k.valid ? 1.0 : 0.0;
        cc[CC_CEMAX] = cemax;
        cc[CC_BGT] = (model & HAWKES_BG_TIME) ? 1.0 : 0.0;
        cc[CC_LLONLY] = (model & HAWKES_LOGLIK_ONLY) ? 1.0 : 0.0;
        for (int q = 0; q < 7; ++q) cc[CC_FTHR + q] = -1.0;
        ctr[CT_WORK] = 0;
        ctr[CT_FIX] = 0;
        ctr[CT_DONE] = 0;
        for (int q = 0; q < FIX_DOUBLES; ++q) fix7[q] = 0.0;
        if (!k.valid) set_error(ctr, HAWKES_ERR_ARG);
    }
    const double beta0 = (k.tx * k.tx) / (k.h * k.h);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad;
         e += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q * npad + e] = 0.0;
        if (!stage) continue;
        float nt, nxh, nxl, nyh, nyl, nb, ce;
        if (e < n) {
            const double tt = (t[e] - tb[e / TB]) * k.kt;
            const double xs = x[e] * k.kx, ys = y[e] * k.kx;
            const float xh = static_cast<float>(xs), yh = static_cast<float>(ys);
            const double se = model1 ? 1.0 : s[e];
            nt = -static_cast<float>(tt);
            nxh = -xh;
            nyh = -yh;
            nxl = -static_cast<float>(xs - static_cast<double>(xh));
            nyl = -static_cast<float>(ys - static_cast<double>(yh));
            nb = -static_cast<float>(beta0 / (se * se));
            ce = static_cast<float>(-2.0 * log2(se));
        } else {
            nt = -PAD_T;
            nxh = nyh = nxl = nyl = 0.f;
            nb = 0.f;
            ce = 0.f;
        }
        *rec_q(rec, e, 0) = make_float4(nt, nt, nxh, nxh);
        *rec_q(rec, e, 1) = make_float4(nxl, nxl, nyh, nyh);
        *rec_q(rec, e, 2) = make_float4(nyl, nyl, nb, nb);
        *rec_q(rec, e, 3) = make_float4(ce, ce, 0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------
// Row finalisation: lambda_i, clip, Lambda_i and the gradient (FP64).
// sums = SB, SBr, SBt, SE, SEt, SEq in natural units (unnormalised).
// ---------------------------------------------------------------------------
__device__ void row_terms(const double* sums, double ti, const double* __restrict__ cc,
                          double out[9]) {
    const double mu = cc[CC_MU], tx = cc[CC_TX], tt = cc[CC_TT];
    const double th = cc[CC_TH], om = cc[CC_OM], h = cc[CC_H];
    const double cB = cc[CC_CB], cE = cc[CC_CE], tN = cc[CC_TN];
    const double SB = cB * sums[0], SBr = cB * sums[1], SBt = cB * sums[2];
    const double SE = cE * sums[3], SEt = cE * sums[4], SEq = cE * sums[5];
    const double lam = mu * SB + th * SE;
    double d[6] = {0, 0, 0, 0, 0, 0};
    double loglam;
    if (cc[CC_LLONLY] != 0.0) {  // the sweep formed SB and SE only: no gradient
        loglam = lam < CLIP ? log(CLIP) : log(lam);
        const double a = (tN - ti) / tt, b = -ti / tt;
        const double Lam = mu * (normcdf(a) - normcdf(b)) + th * (1.0 - exp(-om * (tN - ti)));
        out[0] = loglam - Lam;
        for (int q = 1; q < 7; ++q) out[q] = CUDART_NAN;
        out[7] = loglam;
        out[8] = Lam;
        return;
    }
    if (lam < CLIP) {
        loglam = log(CLIP);
    } else {
        loglam = log(lam);
        const double il = 1.0 / lam;
        d[0] = SB * il;
        d[1] = mu * (SBr / (tx * tx * tx) - 2.0 * SB / tx) * il;
        d[2] = mu * (SBt / (tt * tt * tt) - SB / tt) * il;
        d[3] = SE * il;
        d[4] = th * (SE / om - SEt) * il;
        d[5] = th * (SEq / (h * h * h) - 2.0 * SE / h) * il;
    }
    const double a = (tN - ti) / tt, b = -ti / tt;
    const double Pa = normcdf(a), Pb = normcdf(b);
    const double pa = exp(-0.5 * a * a) * 0.3989422804014327;
    const double pb = exp(-0.5 * b * b) * 0.3989422804014327;
    const double ea = exp(-om * (tN - ti));
    const double Lam = mu * (Pa - Pb) + th * (1.0 - ea);
    out[0] = loglam - Lam;
    out[1] = d[0] - (Pa - Pb);
    out[2] = d[1];
    out[3] = d[2] - mu * (-pa * a + pb * b) / tt;
    out[4] = d[3] - (1.0 - ea);
    out[5] = d[4] - th * (tN - ti) * ea;
    out[6] = d[5];
    out[7] = loglam;
    out[8] = Lam;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* dst) {
    __shared__ double red[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < NV; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int q = 0; q < NV; ++q) {
            double u = lane < nw ? red[lane][q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
            if (lane == 0) dst[q] = u;
        }
    }
}

// ---------------------------------------------------------------------------
// Bound on what the FP32 sweep's flushed terms can move in a row.
//
// ex2.approx.ftz returns 0 for every term below 2^-126, and a product below
// 2^-126 in an accumulation flushes too, so each FP32 moment sum of row i
// lacks a nonnegative part that is at most (per source, natural units):
//   SB  : F                         SE  : F
//   SBr : F 126 / a_x               SEt : F max(t_i - t_1, 1 / sqrt(a_t))
//   SBt : F 126 / a_t               SEq : F (ce_max + 127) 2 h^2 / log2(e)
// with F = 2^-126 (plus margin for the approximation), summed over the row's
// background sources (t_j != t_i) and excitation sources (t_j < t_i).  The
// r^2 and dt^2 factors follow from 2^-a a <= 126 2^-126 for a >= 126; the
// excitation's from 2^g (ce_max - g) <= 2^-126 (ce_max + 126) for g <= -126.
// The row's outputs are N_k / lambda with N_k linear in the moments, so each
// output moves by at most (|dN_k| + |N_k| dlambda / lambda) / lambda, and the
// log-likelihood by dlambda / lambda.  A clipped row whose true rate could
// reach the clip gets an infinite bound.
// ---------------------------------------------------------------------------
__device__ void row_flush_bound(const double* sums, double ti, double t1, int64_t nb, int64_t ne,
                                const double* __restrict__ cc, double b[7]) {
    constexpr double F = 1.2e-38;  // 2^-126 = 1.1755e-38, with margin
    const double mu = cc[CC_MU], tx = cc[CC_TX], tt = cc[CC_TT];
    const double th = cc[CC_TH], om = cc[CC_OM], h = cc[CC_H];
    const double cB = cc[CC_CB], cE = cc[CC_CE];
    const double fb = F * static_cast<double>(nb), fe = F * static_cast<double>(ne);
    const double DB = cB * fb;
    const double DBr = cc[CC_BGT] != 0.0 ? 0.0 : cB * fb * 126.0 * cc[CC_SR];
    const double DBt = cB * fb * 126.0 * cc[CC_ST];
    const double DE = cE * fe;
    const double DEt = cE * fe * fmax(ti - t1, cc[CC_SET]);
    const double DEq = cE * fe * (cc[CC_CEMAX] + 127.0) * cc[CC_SEQ];
    const double SB = cB * sums[0], SBr = cB * sums[1], SBt = cB * sums[2];
    const double SE = cE * sums[3], SEt = cE * sums[4], SEq = cE * sums[5];
    const double lam = mu * SB + th * SE, dlam = mu * DB + th * DE;
    if (lam < CLIP) {
        const double inf = CUDART_INF;
        for (int q = 0; q < 7; ++q) b[q] = (lam + dlam >= CLIP) ? inf : 0.0;
        return;
    }
    const double il = 1.0 / lam, r = dlam * il;
    const double N[6] = {SB, mu * (SBr / (tx * tx * tx) - 2.0 * SB / tx),
                         mu * (SBt / (tt * tt * tt) - SB / tt), SE, th * (SE / om - SEt),
                         th * (SEq / (h * h * h) - 2.0 * SE / h)};
    const double dN[6] = {DB, mu * (DBr / (tx * tx * tx) + 2.0 * DB / tx),
                          mu * (DBt / (tt * tt * tt) + DB / tt), DE, th * (DE / om + DEt),
                          th * (DEq / (h * h * h) + 2.0 * DE / h)};
    b[0] = r;
    for (int q = 0; q < 6; ++q) b[1 + q] = (dN[q] + fabs(N[q]) * r) * il;
}

// Finalise rows [rb, re).  With `check` (FP32 sweep), rows whose rate could be
// moved by FP32 underflow are queued for FP64 recomputation instead, and each
// block's partials also carry the summed flush bounds of its other rows.
__global__ void k_finalize(const double* __restrict__ acc, const double* __restrict__ t,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const double* __restrict__ cc, int64_t n, int64_t npad, int64_t rb,
                           int64_t re, int check, int* fixlist, int* ctr, double* partials,
                           double* rows9) {
    double v[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const bool valid = cc[CC_VALID] != 0.0;
    const double thr = cc[CC_FLAGTHR];
    const double mu = cc[CC_MU], th = cc[CC_TH], cB = cc[CC_CB], cE = cc[CC_CE];
    const double t1 = t[0];
    for (int64_t i = rb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; valid && i < re;
         i += (int64_t)gridDim.x * blockDim.x) {
        double sums[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) sums[q] = acc[q * npad + i];
        if (check) {
            const double lam = mu * cB * sums[0] + th * cE * sums[3];
            if (lam < thr) {
                const int k = atomicAdd(ctr + CT_FIX, 1);
                if (kDebug && !(k >= 0 && k < npad)) {
                    set_error(ctr, HAWKES_ERR_BOUNDS);
                    continue;
                }
                fixlist[k] = static_cast<int>(i);
                continue;
            }
        }
        double o[9];
        row_terms(sums, t[i], cc, o);
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] += o[q];
        if (check) {
            double bd[7];
            const int64_t l = lo[i];
            row_flush_bound(sums, t[i], t1, l + (n - hi[i]), l, cc, bd);
#pragma unroll
            for (int q = 0; q < 7; ++q) v[7 + q] += bd[q];
        }
        if (rows9)
            for (int q = 0; q < 9; ++q) rows9[9 * i + q] = o[q];
    }
    block_reduce_store<14>(v, partials + PART_STRIDE * blockIdx.x);
}

// This thread's share (sources j = threadIdx.x + k blockDim.x) of row i's six
// FP64 moment sums, in natural units: the pair terms of eqs. 2-3 written out.
// ix2 = 1/(2 tau_x^2) (0 for the time-only background), it2 = 1/(2 tau_t^2),
// ih2 = 1/(2 h^2).
__device__ __forceinline__ void row_sums64(int64_t i, const double* __restrict__ t,
                                           const double* __restrict__ x,
                                           const double* __restrict__ y,
                                           const double* __restrict__ s,
                                           const int32_t* __restrict__ lo,
                                           const int32_t* __restrict__ hi, bool model1, int64_t n,
                                           double ix2, double it2, double ih2, double om,
                                           double v[6]) {
    const double ti = t[i], xi = x[i], yi = y[i];
    const int64_t li = lo[i], hj = hi[i];
    for (int q = 0; q < 6; ++q) v[q] = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double dt = ti - t[j], dx = xi - x[j], dy = yi - y[j];
        const double r2 = dx * dx + dy * dy;
        if (j < li || j >= hj) {
            const double b = exp(-r2 * ix2 - dt * dt * it2);
            v[0] += b;
            v[1] += ix2 != 0.0 ? b * r2 : 0.0;
            v[2] += b * dt * dt;
        }
        if (j < li) {
            const double sj = model1 ? 1.0 : s[j];
            const double is2 = 1.0 / (sj * sj);
            const double e = is2 * exp(-om * dt - r2 * ih2 * is2);
            v[3] += e;
            v[4] += e * dt;
            v[5] += e * r2 * is2;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 pair rows: one CTA per row, threads stride over all sources.
// mode 0: rows row_begin + [0, count) -> write natural-unit sums to acc
// mode 1: rows fixlist[0 .. ctr[CT_FIX]) -> finalise and add into fix7
// ---------------------------------------------------------------------------
__global__ void k_rows64(const double* __restrict__ t, const double* __restrict__ x,
                         const double* __restrict__ y, const double* __restrict__ s,
                         const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                         const double* __restrict__ cc, int model, int64_t n, int64_t npad,
                         int64_t row_begin, int64_t count, int mode, const int* fixlist, int* ctr,
                         double* acc, double* fix7, double* rows9) {
    if (cc[CC_VALID] == 0.0) return;
    const bool model1 = (model & HAWKES_MODEL1) != 0;
    const double tx = cc[CC_TX], tt = cc[CC_TT], om = cc[CC_OM], h = cc[CC_H];
    // Time-only background: no spatial factor in B and no r^2 moment.
    const double ix2 = (model & HAWKES_BG_TIME) ? 0.0 : 1.0 / (2.0 * tx * tx);
    const double it2 = 1.0 / (2.0 * tt * tt), ih2 = 1.0 / (2.0 * h * h);
    const int64_t total = mode ? static_cast<int64_t>(ctr[CT_FIX]) : count;
    for (int64_t k = blockIdx.x; k < total; k += gridDim.x) {
        const int64_t i = mode ? fixlist[k] : row_begin + k;
        if (kDebug && !(i >= 0 && i < n && (mode || k < npad))) {
            if (threadIdx.x == 0) set_error(ctr, HAWKES_ERR_BOUNDS);
            continue;  // uniform over the block: i depends on k only
        }
        const double ti = t[i];
        double v[6];
        row_sums64(i, t, x, y, s, lo, hi, model1, n, ix2, it2, ih2, om, v);
        __shared__ double sums[8];
        block_reduce_store<6>(v, sums);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (mode == 0) {
                for (int q = 0; q < 6; ++q) acc[q * npad + i] = sums[q];
            } else {
                double o[9];
                row_terms(sums, ti, cc, o);
                for (int q = 0; q < 7; ++q) atomicAdd(fix7 + q, o[q]);
                if (rows9)
                    for (int q = 0; q < 9; ++q) rows9[9 * i + q] = o[q];
            }
        }
        __syncthreads();
    }
}

// Sum the per-block partials in a fixed order, add the FP64-recomputed rows,
// write the 7 outputs.  One CTA.  The summed flush bounds of the FP32 sweep
// (zero on the FP64 path) decide, per output, whether rows must be recomputed
// by k_flushfix: when an output's bound exceeds FLUSH_TAU of its magnitude,
// every row whose own bound exceeds FLUSH_TAU |output| / nrows is, so the rows
// left in FP32 can move it by at most FLUSH_TAU of its magnitude.
__global__ void k_reduce(const double* __restrict__ partials, int nparts,
                         const double* __restrict__ fix7, double* __restrict__ cc, int64_t nrows,
                         double* out, int* ctr) {
    double v[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int q = 0; q < 14; ++q) v[q] += partials[PART_STRIDE * b + q];
    __shared__ double tot[16];
    block_reduce_store<14>(v, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool valid = cc[CC_VALID] != 0.0;
        const bool llonly = cc[CC_LLONLY] != 0.0;
        bool finite = true;
        for (int q = 0; q < 7; ++q) {
            const double r = valid ? tot[q] + fix7[q] : CUDART_NAN;
            if (q == 0 || !llonly) finite = finite && isfinite(r);
            out[q] = r;
            const double g = fabs(r), bound = tot[7 + q];
            cc[CC_FTHR + q] = (valid && (q == 0 || !llonly) && bound > FLUSH_TAU * g)
                                  ? FLUSH_TAU * g / static_cast<double>(nrows > 0 ? nrows : 1)
                                  : -1.0;
        }
        if (valid && !finite) set_error(ctr, HAWKES_ERR_NONFINITE);
    }
}

// Recompute in FP64 the rows that k_reduce's thresholds select (a row whose
// flush bound for some output exceeds that output's threshold; rows already
// recomputed for their low rate are left out), replace their FP32 values by
// the FP64 ones in the outputs, and write their per-row values.  Each block
// takes 256-row chunks; the last block to finish adds the corrections to out.
// Returns at once when no output needs it (the usual case).
__global__ void k_flushfix(const double* __restrict__ acc, const double* __restrict__ t,
                           const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ s, const int32_t* __restrict__ lo,
                           const int32_t* __restrict__ hi, const double* __restrict__ cc,
                           int model, int64_t n, int64_t npad, int64_t rb, int64_t re, int* ctr,
                           double* fix7, double* out, double* rows9) {
    if (cc[CC_VALID] == 0.0) return;
    double thr[7];
    bool any = false;
    for (int q = 0; q < 7; ++q) {
        thr[q] = cc[CC_FTHR + q];
        any = any || thr[q] >= 0.0;
    }
    if (!any) return;  // uniform over the grid
    const bool model1 = (model & HAWKES_MODEL1) != 0;
    const double tx = cc[CC_TX], tt = cc[CC_TT], om = cc[CC_OM], h = cc[CC_H];
    const double ix2 = cc[CC_BGT] != 0.0 ? 0.0 : 1.0 / (2.0 * tx * tx);
    const double it2 = 1.0 / (2.0 * tt * tt), ih2 = 1.0 / (2.0 * h * h);
    const double flagthr = cc[CC_FLAGTHR];
    const double mu = cc[CC_MU], th = cc[CC_TH], cB = cc[CC_CB], cE = cc[CC_CE];
    const double t1 = t[0];
    __shared__ int list[256];
    __shared__ int cnt;
    __shared__ double sums[8];
    __shared__ int last;
    double mine[7] = {0, 0, 0, 0, 0, 0, 0};  // thread 0: this block's corrections
    for (int64_t base = rb + static_cast<int64_t>(blockIdx.x) * 256; base < re;
         base += static_cast<int64_t>(gridDim.x) * 256) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        const int64_t i = base + threadIdx.x;
        if (threadIdx.x < 256 && i < re) {
            double sm[6];
            for (int q = 0; q < 6; ++q) sm[q] = acc[q * npad + i];
            if (!(mu * cB * sm[0] + th * cE * sm[3] < flagthr)) {
                double bd[7];
                const int64_t l = lo[i];
                row_flush_bound(sm, t[i], t1, l + (n - hi[i]), l, cc, bd);
                bool f = false;
                for (int q = 0; q < 7; ++q) f = f || (thr[q] >= 0.0 && bd[q] > thr[q]);
                if (f) list[atomicAdd(&cnt, 1)] = threadIdx.x;
            }
        }
        __syncthreads();
        const int m = cnt;
        for (int k = 0; k < m; ++k) {
            const int64_t r = base + list[k];
            double v[6];
            row_sums64(r, t, x, y, s, lo, hi, model1, n, ix2, it2, ih2, om, v);
            block_reduce_store<6>(v, sums);
            if (threadIdx.x == 0) {
                double s32[6], o64[9], o32[9];
                for (int q = 0; q < 6; ++q) s32[q] = acc[q * npad + r];
                row_terms(sums, t[r], cc, o64);
                row_terms(s32, t[r], cc, o32);
                for (int q = 0; q < 7; ++q) mine[q] += o64[q] - o32[q];
                if (rows9)
                    for (int q = 0; q < 9; ++q) rows9[9 * r + q] = o64[q];
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 7; ++q)
            if (mine[q] != 0.0) atomicAdd(fix7 + 8 + q, mine[q]);
        __threadfence();
        last = atomicAdd(ctr + CT_DONE, 1) == static_cast<int>(gridDim.x) - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double* fb = fix7 + 8;
        const bool llonly = cc[CC_LLONLY] != 0.0;
        bool finite = true;
        for (int q = 0; q < 7; ++q) {
            const double r = out[q] + fb[q];
            out[q] = r;
            if (q == 0 || !llonly) finite = finite && isfinite(r);
        }
        if (!finite) set_error(ctr, HAWKES_ERR_NONFINITE);
    }
}

// ---------------------------------------------------------------------------
// Location resample (cut posterior, Sec. 2.2).
// ---------------------------------------------------------------------------
// Triangle areas, evaluated exactly as documented (no fused multiply-add).
__global__ void k_tri_area(const double* __restrict__ xy, int32_t n_tri, double* area, int* ctr) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_tri; k += gridDim.x * blockDim.x) {
        const double* v = xy + 6 * (int64_t)k;
        for (int q = 0; q < 6; ++q)
            if (!isfinite(v[q])) set_error(ctr, HAWKES_ERR_ARG);
        const double cr = __dsub_rn(__dmul_rn(__dsub_rn(v[2], v[0]), __dsub_rn(v[5], v[1])),
                                    __dmul_rn(__dsub_rn(v[4], v[0]), __dsub_rn(v[3], v[1])));
        area[k] = __dmul_rn(0.5, fabs(cr));
    }
}

// Per county: its triangle range and the running area sums (in triangle order).
__global__ void k_tri_county(const int32_t* __restrict__ tri_county, int32_t n_tri,
                             int32_t n_counties, double* cum, int32_t* first, int32_t* last,
                             int* ctr) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_counties;
         c += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_tri;  // first triangle with county >= c
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (tri_county[mid] < c) lo = mid + 1; else hi = mid;
        }
        int k = lo;
        if (k >= n_tri || tri_county[k] != c) {
            first[c] = -1;
            last[c] = -1;
            set_error(ctr, HAWKES_ERR_ARG);
            continue;
        }
        first[c] = k;
        double run = cum[k];  // cum holds the areas on entry
        for (++k; k < n_tri && tri_county[k] == c; ++k) {
            run = __dadd_rn(run, cum[k]);
            cum[k] = run;
        }
        last[c] = k - 1;
        if (!(run > 0.0)) set_error(ctr, HAWKES_ERR_ARG);
    }
}

__global__ void k_tri_check(const int32_t* __restrict__ tri_county, int32_t n_tri,
                            int32_t n_counties, int* ctr) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_tri; k += gridDim.x * blockDim.x) {
        const int32_t c = tri_county[k];
        if (c < 0 || c >= n_counties || (k > 0 && tri_county[k - 1] > c))
            set_error(ctr, HAWKES_ERR_ARG);
    }
}

// Philox4x64-10 (Salmon et al., SC 2011): ten rounds of two 64x64->128-bit
// multiplies mixing the counter with a Weyl-bumped key.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int rd = 0; rd < 10; ++rd) {
        if (rd) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double unit53(uint64_t w) {
    return __dmul_rn(static_cast<double>(w >> 11), 1.0 / 9007199254740992.0);
}

__global__ void k_resample(const int32_t* __restrict__ county, int64_t n,
                           const double* __restrict__ tri_xy, const double* __restrict__ cum,
                           const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                           uint64_t seed, uint64_t stream, uint64_t iteration,
                           const uint64_t* d_iteration, double* x, double* y) {
    if (d_iteration) iteration = *d_iteration;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = county[i];
        uint64_t w[4] = {static_cast<uint64_t>(i), iteration, 0ull, 0ull};
        philox4x64_10(w, seed, stream);
        const double u0 = unit53(w[0]), u1 = unit53(w[1]), u2 = unit53(w[2]);
        int32_t a = first[c], b = last[c];
        const double target = __dmul_rn(u0, cum[b]);
        // first k in [a, b] with target < cum[k]; b if there is none
        while (a < b) {
            const int32_t mid = (a + b) >> 1;
            if (target < cum[mid]) b = mid; else a = mid + 1;
        }
        const double* v = tri_xy + 6 * (int64_t)a;
        const double r1 = __dsqrt_rn(u1);
        const double w0 = __dsub_rn(1.0, r1);
        const double w1 = __dmul_rn(r1, __dsub_rn(1.0, u2));
        const double w2 = __dmul_rn(r1, u2);
        x[i] = __dadd_rn(__dadd_rn(__dmul_rn(w0, v[0]), __dmul_rn(w1, v[2])), __dmul_rn(w2, v[4]));
        y[i] = __dadd_rn(__dadd_rn(__dmul_rn(w0, v[1]), __dmul_rn(w1, v[3])), __dmul_rn(w2, v[5]));
    }
}

// Self-check of the bounded wait: one thread waits on an mbarrier that nothing
// ever completes; the wait must give up and latch HAWKES_ERR_TIMEOUT.
__global__ void k_wait_selftest(int* ctr) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) set_error(ctr, HAWKES_ERR_TIMEOUT);
}

}  // namespace hk
