/*
 * Plain CPU oracle for the spatiotemporal Hawkes log-likelihood, its gradient
 * in (mu, tau_x, tau_t, theta, omega, h), and the cut-posterior location
 * resample.  TEST INFRASTRUCTURE ONLY: nothing in the product path links,
 * loads or calls this file; only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark do.
 *
 * It is written to be checked by eye against the paper, not to be fast:
 * ordered pairs (i, j), j != i, one row at a time, no symmetry, no tiling, no
 * reordering.  The input times need not be sorted.
 *
 * The same source is compiled twice: REAL = double (the oracle proper) and
 * REAL = long double (binary128 on aarch64, x87 extended on x86_64), which is
 * used only to bound the rounding error of the double build.
 *
 * Model (Sec. 2.1, eqs. 2-4, with the readings listed in the design notes):
 *   background pair term, for every j with t_j != t_i:
 *       B_ij = mu * phi2(r_ij; tau_x) * phi1(t_i - t_j; tau_t)
 *   or, with the time-only background of eq. 2 (App. A writes its 1/A(X)
 *   factor as tau_x^-2, so tau_x^2 stands for the domain area):
 *       B_ij = mu * phi1(t_i - t_j; tau_t) / tau_x^2
 *   excitation pair term, for every j with t_j < t_i (eq. 3, the bandwidth
 *   belongs to the source event j):
 *       E_ij = theta * omega * exp(-omega (t_i - t_j)) * phi2(r_ij; h s_j)
 *   phi2(r; sd) = exp(-r^2 / (2 sd^2)) / (2 pi sd^2)   (2-D spherical Gaussian)
 *   phi1(d; sd) = exp(-d^2 / (2 sd^2)) / (sqrt(2 pi) sd)
 *   lambda_i = max(sum_j B_ij + sum_j E_ij, 1e-40)    (Sec. 2.3.1 clip)
 *   Lambda_i = mu [Phi((t_N - t_i)/tau_t) - Phi(-t_i/tau_t)]
 *              + theta [1 - exp(-omega (t_N - t_i))]    (Sec. 2.1, t_N = max t)
 *   ell = sum_i (log lambda_i - Lambda_i)                (eq. 4)
 * The gradient is the analytic derivative of ell (the paper gives none).
 *
 * Resample (Sec. 2.2, cut posterior): each location is drawn uniformly in
 * its county polygon, given as a fan of triangles: a triangle is picked with
 * probability proportional to its area, then a uniform point inside it
 * (Osada et al. 2002, square-root barycentric map).  Random numbers come from
 * Philox4x64-10 (Salmon et al. 2011) keyed (seed, stream), counter
 * (event index, iteration, 0, 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_LONG
typedef double REAL;
#define SUF(name) name##_f64
#define EXP exp
#define LOG log
#define ERFC erfc
#define SQRT sqrt
#else
typedef long double REAL;
#define SUF(name) name##_ld
#define EXP expl
#define LOG logl
#define ERFC erfcl
#define SQRT sqrtl
#endif

#define PI_R ((REAL)3.14159265358979323846264338327950288L)
#define CLIP_R ((REAL)1e-40L)

/* Standard normal CDF through the complementary error function. */
static REAL std_normal_cdf(REAL z) {
    return (REAL)0.5 * ERFC(-z / SQRT((REAL)2));
}

/* Standard normal density. */
static REAL std_normal_pdf(REAL z) {
    return EXP(-z * z / 2) / SQRT(2 * PI_R);
}

/* 2-D spherical Gaussian density at squared distance r2, standard deviation sd. */
static REAL phi2(REAL r2, REAL sd) {
    return EXP(-r2 / (2 * sd * sd)) / (2 * PI_R * sd * sd);
}

/* 1-D Gaussian density at offset d, standard deviation sd. */
static REAL phi1(REAL d, REAL sd) {
    return EXP(-d * d / (2 * sd * sd)) / (SQRT(2 * PI_R) * sd);
}

/*
 * One row i of eq. 4 and its gradient.  out9 receives
 *   [ell_i, d ell_i/d(mu, tau_x, tau_t, theta, omega, h), log lambda_i, Lambda_i].
 */
static void one_row(int64_t n, const double* t, const double* x, const double* y,
                    const double* s, const REAL p[6], REAL tN, int64_t i, int bg_time_only,
                    REAL out9[9]) {
    const REAL mu = p[0], tx = p[1], tt = p[2], th = p[3], om = p[4], h = p[5];
    REAL SB = 0, SBr = 0, SBt = 0, SE = 0, SEt = 0, SEq = 0;
    const REAL ti = t[i], xi = x[i], yi = y[i];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const REAL tj = t[j];
        const REAL dt = ti - tj;
        const REAL dx = xi - (REAL)x[j], dy = yi - (REAL)y[j];
        const REAL r2 = dx * dx + dy * dy;
        if (tj != ti) {                         /* background, indicator t_j != t_i */
            if (bg_time_only) {
                const REAL b = phi1(dt, tt) / (tx * tx);
                SB += b;                            /* no spatial moment: SBr stays 0 */
                SBt += b * dt * dt;
            } else {
                const REAL b = phi2(r2, tx) * phi1(dt, tt);
                SB += b;
                SBr += b * r2;
                SBt += b * dt * dt;
            }
        }
        if (tj < ti) {                          /* excitation from earlier source j */
            const REAL sj = s ? (REAL)s[j] : (REAL)1;
            const REAL e = om * EXP(-om * dt) * phi2(r2, h * sj);
            SE += e;
            SEt += e * dt;
            SEq += e * r2 / (sj * sj);
        }
    }
    REAL lam = mu * SB + th * SE;
    REAL dlog[6] = {0, 0, 0, 0, 0, 0};
    REAL loglam;
    if (lam < CLIP_R) {
        loglam = LOG(CLIP_R);                  /* clipped: constant, zero gradient */
    } else {
        loglam = LOG(lam);
        dlog[0] = SB / lam;
        dlog[1] = mu * (SBr / (tx * tx * tx) - 2 * SB / tx) / lam;
        dlog[2] = mu * (SBt / (tt * tt * tt) - SB / tt) / lam;
        dlog[3] = SE / lam;
        dlog[4] = th * (SE / om - SEt) / lam;
        dlog[5] = th * (SEq / (h * h * h) - 2 * SE / h) / lam;
    }
    /* Lambda_i and its derivatives (the spatial kernels integrate to 1 over R^2). */
    const REAL a = (tN - ti) / tt, b = -ti / tt;
    const REAL ea = EXP(-om * (tN - ti));
    const REAL Lam = mu * (std_normal_cdf(a) - std_normal_cdf(b)) + th * (1 - ea);
    REAL dLam[6];
    dLam[0] = std_normal_cdf(a) - std_normal_cdf(b);
    dLam[1] = 0;
    dLam[2] = mu * (-std_normal_pdf(a) * a + std_normal_pdf(b) * b) / tt;
    dLam[3] = 1 - ea;
    dLam[4] = th * (tN - ti) * ea;
    dLam[5] = 0;
    out9[0] = loglam - Lam;
    for (int k = 0; k < 6; ++k) out9[1 + k] = dlog[k] - dLam[k];
    out9[7] = loglam;
    out9[8] = Lam;
}

/*
 * Log-likelihood (eq. 4) and gradient over rows [row_begin, row_end).
 *   n        number of events; t, x, y: event times and coordinates [n]
 *   s        per-event source bandwidth scale s_j [n], or NULL for s_j = 1
 *            (the fixed-bandwidth model, eq. 2)
 *   params   mu, tau_x, tau_t, theta, omega, h
 *   out7     ell, then the six partial derivatives, summed over the rows
 *   rows9    optional [(row_end - row_begin) * 9] per-row values (see one_row)
 *   threads  OpenMP threads (<= 0: the OpenMP default); rows are summed in
 *            row order afterwards, so the result does not depend on it
 *   bg_time_only  nonzero: the time-only background of eq. 2 (see above)
 * t_N is the largest time of all n events, also for a row window.
 * Returns 0, or -1 on bad arguments.
 */
int SUF(oracle_loglik_grad)(int64_t n, const double* t, const double* x, const double* y,
                            const double* s, const double* params, int64_t row_begin,
                            int64_t row_end, double* out7, double* rows9, int threads,
                            int bg_time_only) {
    if (n < 1 || !t || !x || !y || !params || !out7) return -1;
    if (row_begin < 0 || row_end > n || row_begin > row_end) return -1;
    REAL p[6];
    for (int k = 0; k < 6; ++k) p[k] = params[k];
    REAL tN = t[0];
    for (int64_t j = 1; j < n; ++j)
        if (t[j] > tN) tN = t[j];
    const int64_t m = row_end - row_begin;
    REAL* rows = (REAL*)malloc(sizeof(REAL) * 9 * (size_t)(m > 0 ? m : 1));
    if (!rows) return -1;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads)
#endif
    for (int64_t r = 0; r < m; ++r)
        one_row(n, t, x, y, s, p, tN, row_begin + r, bg_time_only, rows + 9 * r);
    REAL acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t r = 0; r < m; ++r)
        for (int k = 0; k < 7; ++k) acc[k] += rows[9 * r + k];
    for (int k = 0; k < 7; ++k) out7[k] = (double)acc[k];
    if (rows9)
        for (int64_t r = 0; r < 9 * m; ++r) rows9[r] = (double)rows[r];
    free(rows);
    (void)threads;
    return 0;
}

/* Threads the OpenMP runtime would use by default (1 without OpenMP). */
int SUF(oracle_max_threads)(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifndef ORACLE_LONG
/* ---------------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011).  State: four 64-bit counter words, two key words.
 * One round multiplies counter words 0 and 2 by the two round multipliers,
 * keeping the 128-bit products, and mixes the high halves with the other two
 * counter words and the key:
 *   (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2
 *   c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
 * Between rounds the key is bumped by the Weyl constants (golden ratio and
 * sqrt(3) - 1 in 64-bit fixed point).
 * ------------------------------------------------------------------------- */
void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        const unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* 53 random bits to a double in [0, 1). */
static double unit_double(uint64_t w) {
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Cut-posterior location draw (Sec. 2.2): x_i ~ Uniform(polygon of county c_i).
 *   county[n]      county id of each event, 0 <= id < n_counties
 *   tri_county[m]  county of each triangle, non-decreasing; every county has
 *                  at least one triangle of positive total area
 *   tri_xy[6 m]    triangle vertices ax, ay, bx, by, cx, cy
 * For event i the Philox block with counter (i, iteration, 0, 0) and key
 * (seed, stream) gives u0, u1, u2 (words 0-2 as 53-bit uniforms).  The
 * triangle is the first k of the county whose running area sum exceeds
 * u0 * (county area), or the county's last triangle if none does; the point is
 *   (1 - sqrt(u1)) A + sqrt(u1)(1 - u2) B + sqrt(u1) u2 C.
 * Areas, sums and the point are evaluated left to right without fused
 * multiply-add.  Returns 0, or -1 on bad arguments.
 */
int oracle_resample(int64_t n, const int32_t* county, int32_t n_counties, int32_t n_tri,
                    const int32_t* tri_county, const double* tri_xy, uint64_t seed,
                    uint64_t stream, uint64_t iteration, double* x_out, double* y_out) {
    if (n < 0 || n_counties < 1 || n_tri < 1) return -1;
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_counties);
    int32_t* last = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_counties);
    double* cum = (double*)malloc(sizeof(double) * (size_t)n_tri);
    if (!first || !last || !cum) {
        free(first); free(last); free(cum);
        return -1;
    }
    for (int32_t c = 0; c < n_counties; ++c) first[c] = -1, last[c] = -1;
    int bad = 0;
    for (int32_t k = 0; k < n_tri; ++k) {
        const int32_t c = tri_county[k];
        if (c < 0 || c >= n_counties || (k > 0 && c < tri_county[k - 1])) { bad = 1; break; }
        const double* v = tri_xy + 6 * (size_t)k;
        double cross = (v[2] - v[0]) * (v[5] - v[1]) - (v[4] - v[0]) * (v[3] - v[1]);
        double area = 0.5 * fabs(cross);
        if (first[c] < 0) {
            first[c] = k;
            cum[k] = area;
        } else {
            cum[k] = cum[k - 1] + area;
        }
        last[c] = k;
    }
    for (int32_t c = 0; c < n_counties && !bad; ++c)
        if (first[c] < 0 || !(cum[last[c]] > 0)) bad = 1;
    for (int64_t i = 0; i < n && !bad; ++i)
        if (county[i] < 0 || county[i] >= n_counties) bad = 1;
    if (bad) {
        free(first); free(last); free(cum);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t c = county[i];
        const uint64_t ctr[4] = {(uint64_t)i, iteration, 0, 0};
        const uint64_t key[2] = {seed, stream};
        uint64_t w[4];
        oracle_philox4x64_10(ctr, key, w);
        const double u0 = unit_double(w[0]), u1 = unit_double(w[1]), u2 = unit_double(w[2]);
        const double target = u0 * cum[last[c]];
        int32_t pick = last[c];
        for (int32_t k = first[c]; k <= last[c]; ++k) {   /* linear scan: first sum above target */
            if (target < cum[k]) { pick = k; break; }
        }
        const double* v = tri_xy + 6 * (size_t)pick;
        const double r1 = sqrt(u1);
        const double w0 = 1.0 - r1;
        const double w1 = r1 * (1.0 - u2);
        const double w2 = r1 * u2;
        x_out[i] = w0 * v[0] + w1 * v[2] + w2 * v[4];
        y_out[i] = w0 * v[1] + w1 * v[3] + w2 * v[5];
    }
    free(first); free(last); free(cum);
    return 0;
}
#endif
