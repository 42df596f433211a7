// C-ABI entry points of libhawkes (declared in include/hawkes.h): context and
// buffer management, argument checks, and the launch sequence of each call.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace hk {
// kernels.cu
__global__ void k_setup(double*, double*, double*, const int32_t*, int32_t, const double*, int64_t,
                        int64_t, int, double*, int32_t*, int32_t*, double*, int*);
__global__ void k_prep(const double*, const double*, const double*, const double*, const double*,
                       const hawkes_params*, int, int, int, int64_t, int64_t, Rec*, double*, double*,
                       int*, double*);
__global__ void k_finalize(const double*, const double*, const int32_t*, const int32_t*,
                           const double*, int64_t, int64_t, int64_t, int64_t, int, int*, int*,
                           double*, double*);
__global__ void k_flushfix(const double*, const double*, const double*, const double*,
                           const double*, const int32_t*, const int32_t*, const double*, int,
                           int64_t, int64_t, int64_t, int64_t, int*, double*, double*, double*);
__global__ void k_rows64(const double*, const double*, const double*, const double*,
                         const int32_t*, const int32_t*, const double*, int, int64_t, int64_t,
                         int64_t, int64_t, int, const int*, int*, double*, double*, double*);
__global__ void k_reduce(const double*, int, const double*, double*, int64_t, double*, int*);
__global__ void k_tri_area(const double*, int32_t, double*, int*);
__global__ void k_tri_county(const int32_t*, int32_t, int32_t, double*, int32_t*, int32_t*, int*);
__global__ void k_tri_check(const int32_t*, int32_t, int32_t, int*);
__global__ void k_resample(const int32_t*, int64_t, const double*, const double*, const int32_t*,
                           const int32_t*, uint64_t, uint64_t, uint64_t, const uint64_t*, double*,
                           double*);
__global__ void k_wait_selftest(int*);
// sweep.cu
cudaError_t sweep_setup_attributes();
int sweep_num_variants();
int sweep_blocks_per_sm(int v);
std::vector<int4> sweep_items(int64_t n, int v);
cudaError_t launch_sweep(hawkes_ctx* c, bool sym, int64_t row_begin, int64_t row_end, bool bgt,
                         bool ll);
cudaError_t launch_sweep_list(hawkes_ctx* c, const int4* items, int nitems, bool bgt, bool ll);
int sweep_variant_rows(int v);
// sweep_spatial.cu
int spatial_build(hawkes_ctx* c);
cudaError_t spatial_launch(hawkes_ctx* c, int model1);
void spatial_free(hawkes_ctx* c);
int spatial_set_window(hawkes_ctx* c, int64_t window);
void spatial_invalidate(hawkes_ctx* c);
}  // namespace hk

using namespace hk;

namespace {

// Restores the caller's current device when a call returns.
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
int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HAWKES_ERR_OOM : HAWKES_ERR_CUDA;
    }
    return HAWKES_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HAWKES_OK : HAWKES_ERR_CUDA; }

#define HK_TRY(expr)                  \
    do {                              \
        int _rc = (expr);             \
        if (_rc != HAWKES_OK) return _rc; \
    } while (0)
#define HK_CUDA(expr) HK_TRY(cuda_status(expr))

// Run `launch` (which enqueues one kernel on c->stream); when profiling, time
// it with a pair of events and add it to kernel class `kind`.
template <typename F>
int timed(hawkes_ctx* c, int kind, F launch) {
    if (c->prof) HK_CUDA(cudaEventRecord(c->pev[0], c->stream));
    launch();
    HK_CUDA(cudaGetLastError());
    if (c->prof) {
        HK_CUDA(cudaEventRecord(c->pev[1], c->stream));
        HK_CUDA(cudaEventSynchronize(c->pev[1]));
        float ms = 0.f;
        HK_CUDA(cudaEventElapsedTime(&ms, c->pev[0], c->pev[1]));
        c->pacc.ms[kind] += ms;
        c->pacc.launches[kind] += 1;
    }
    return HAWKES_OK;
}

int grid_for(hawkes_ctx* c, int64_t items, int per_sm = 8) {
    int64_t g = (items + 255) / 256;
    const int64_t cap = static_cast<int64_t>(c->sms) * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : static_cast<int>(g);
}

void drop_shard_items(hawkes_ctx* c) {
    dfree(c->shard_items);
    c->shard_nitems = 0;
    c->shard_key[0] = c->shard_key[1] = c->shard_key[2] = -1;
}

void free_events(hawkes_ctx* c) {
    dfree(c->t); dfree(c->x); dfree(c->y); dfree(c->s); dfree(c->scale_c); dfree(c->county);
    dfree(c->lo); dfree(c->hi); dfree(c->tb); dfree(c->rec); dfree(c->acc); dfree(c->fixlist);
    dfree(c->items);
    drop_shard_items(c);
    c->nitems = 0;
    c->items_variant = -1;
    dfree(c->rows9);
    c->rows9_cap = 0;
    c->n = c->npad = c->nblk = 0;
}

void free_counties(hawkes_ctx* c) {
    dfree(c->tri_county); dfree(c->tri_xy); dfree(c->tri_cum); dfree(c->cfirst); dfree(c->clast);
    c->n_tri = 0;
    c->counties_ok = false;
}

// Read and clear the latched device error (synchronous).
int take_device_error(hawkes_ctx* c) {
    int err = 0;
    HK_CUDA(cudaMemcpyAsync(&err, c->ctr + CT_ERR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HK_CUDA(cudaStreamSynchronize(c->stream));
    if (err != 0) HK_CUDA(cudaMemsetAsync(c->ctr + CT_ERR, 0, sizeof(int), c->stream));
    return err;
}

bool params_ok(const hawkes_params* p) {
    auto fin = [](double v) { return v == v && v - v == 0.0; };
    return fin(p->mu) && fin(p->tau_x) && fin(p->tau_t) && fin(p->theta) && fin(p->omega) &&
           fin(p->h) && p->mu >= 0 && p->theta >= 0 && p->tau_x > 0 && p->tau_t > 0 &&
           p->omega > 0 && p->h > 0;
}

// (Re)build the symmetric work list for the current events and kernel
// variant (synchronous; never called while a stream is being captured).
int ensure_items(hawkes_ctx* c) {
    if (c->items && c->items_variant == c->variant) return HAWKES_OK;
    dfree(c->items);
    const std::vector<int4> items = sweep_items(c->n, c->variant);
    HK_TRY(dalloc(&c->items, items.size()));
    HK_CUDA(cudaMemcpyAsync(c->items, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, c->stream));
    HK_CUDA(cudaStreamSynchronize(c->stream));
    c->nitems = static_cast<int>(items.size());
    c->items_variant = c->variant;
    return HAWKES_OK;
}

int select_variant(hawkes_ctx* c, int v) {
    if (v < 0 || v >= sweep_num_variants()) return HAWKES_ERR_ARG;
    c->variant = v;
    c->variant_bpsm = sweep_blocks_per_sm(v);
    return c->n ? ensure_items(c) : HAWKES_OK;
}

// Queue the FP32 path's finalisation of rows [rb, re) from the moment sums in
// c->acc: per-row terms (rows near the FP32 floor recomputed in FP64), the
// global reduction, and the FP64 recomputation of the rows whose flushed FP32
// terms could matter to an output.
int enqueue_finalize32(hawkes_ctx* c, int model, int64_t rb, int64_t re, double* d_out,
                       double* d_rows9) {
    HK_TRY(timed(c, HAWKES_K_FINAL, [&] {
        k_finalize<<<c->final_blocks, 256, 0, c->stream>>>(c->acc, c->t, c->lo, c->hi, c->cc, c->n,
                                                           c->npad, rb, re, 1, c->fixlist, c->ctr,
                                                           c->partials, d_rows9);
    }));
    HK_TRY(timed(c, HAWKES_K_ROWS64, [&] {
        k_rows64<<<c->sms, 256, 0, c->stream>>>(c->t, c->x, c->y, c->s, c->lo, c->hi, c->cc, model,
                                                c->n, c->npad, 0, 0, 1, c->fixlist, c->ctr, c->acc,
                                                c->fix7, d_rows9);
    }));
    HK_TRY(timed(c, HAWKES_K_REDUCE, [&] {
        k_reduce<<<1, 256, 0, c->stream>>>(c->partials, c->final_blocks, c->fix7, c->cc, re - rb,
                                           d_out, c->ctr);
    }));
    return timed(c, HAWKES_K_ROWS64, [&] {
        k_flushfix<<<grid_for(c, re - rb, 2), 256, 0, c->stream>>>(
            c->acc, c->t, c->x, c->y, c->s, c->lo, c->hi, c->cc, model, c->n, c->npad, rb, re,
            c->ctr, c->fix7, d_out, d_rows9);
    });
}

// Queue one log-likelihood evaluation over rows [rb, re).  d_params: device
// parameters; d_out: 7 doubles; d_rows9: optional per-row output [9 n].
int enqueue_loglik(hawkes_ctx* c, const hawkes_params* d_params, uint32_t flags, int64_t rb,
                   int64_t re, double* d_out, double* d_rows9) {
    const bool f64 = (flags & HAWKES_F64) != 0;
    const int model = static_cast<int>(flags & kModelBits);
    const bool bgt = (flags & HAWKES_BG_TIME) != 0;
    const bool spatial = (flags & HAWKES_SKIP_SPATIAL) != 0;
    if (spatial && (f64 || bgt || rb != 0 || re != c->n)) return HAWKES_ERR_ARG;
    if (spatial) HK_TRY(spatial_build(c));  // synchronous on first use after set_events
    const int skip = (!f64 && !spatial && (flags & HAWKES_SKIP_UNDERFLOW)) ? 1 : 0;
    const int prep_grid = grid_for(c, c->npad);
    HK_TRY(timed(c, HAWKES_K_PREP, [&] {
        k_prep<<<prep_grid, 256, 0, c->stream>>>(c->t, c->x, c->y, c->s, c->tb, d_params, model,
                                                  (f64 || spatial) ? 0 : 1, skip, c->n, c->npad, c->rec,
                                                  c->acc, c->cc, c->ctr, c->fix7);
    }));
    if (!f64) {
        const bool sym = (rb == 0 && re == c->n);
        cudaError_t se = cudaSuccess;
        HK_TRY(timed(c, HAWKES_K_SWEEP, [&] {
            if (spatial)
                se = spatial_launch(c, (flags & HAWKES_MODEL1) ? 1 : 0);
            else
                launch_sweep(c, sym, rb, re, bgt, (flags & HAWKES_LOGLIK_ONLY) != 0);
        }));
        HK_CUDA(se);
        return enqueue_finalize32(c, model, rb, re, d_out, d_rows9);
    } else {
        const int64_t count = re - rb;
        int g = static_cast<int>(count < static_cast<int64_t>(c->sms) * 16 ? count : c->sms * 16);
        if (g < 1) g = 1;
        HK_TRY(timed(c, HAWKES_K_ROWS64, [&] {
            k_rows64<<<g, 256, 0, c->stream>>>(c->t, c->x, c->y, c->s, c->lo, c->hi, c->cc, model,
                                               c->n, c->npad, rb, count, 0, c->fixlist, c->ctr,
                                               c->acc, c->fix7, d_rows9);
        }));
        HK_TRY(timed(c, HAWKES_K_FINAL, [&] {
            k_finalize<<<c->final_blocks, 256, 0, c->stream>>>(c->acc, c->t, c->lo, c->hi, c->cc,
                                                               c->n, c->npad, rb, re, 0, c->fixlist,
                                                               c->ctr, c->partials, d_rows9);
        }));
    }
    HK_TRY(timed(c, HAWKES_K_REDUCE, [&] {
        k_reduce<<<1, 256, 0, c->stream>>>(c->partials, c->final_blocks, c->fix7, c->cc, re - rb,
                                           d_out, c->ctr);
    }));
    return HAWKES_OK;
}

int sync_loglik(hawkes_ctx* c, const hawkes_params* p, uint32_t flags, int64_t rb, int64_t re,
                double* out7, double* rows_host) {
    if (!params_ok(p)) return HAWKES_ERR_ARG;
    if ((flags & ~kFlagsAll) != 0) return HAWKES_ERR_ARG;
    HK_CUDA(cudaMemcpyAsync(c->params_dev, p, sizeof(hawkes_params), cudaMemcpyHostToDevice,
                            c->stream));
    double* d_rows9 = nullptr;
    if (rows_host) {
        if (c->rows9_cap < c->n) {
            dfree(c->rows9);
            HK_TRY(dalloc(&c->rows9, static_cast<size_t>(9 * c->n)));
            c->rows9_cap = c->n;
        }
        d_rows9 = c->rows9;
    }
    HK_TRY(enqueue_loglik(c, c->params_dev, flags, rb, re, c->out_dev, d_rows9));
    HK_CUDA(cudaMemcpyAsync(c->out_host, c->out_dev, 7 * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    if (rows_host)
        HK_CUDA(cudaMemcpyAsync(rows_host, d_rows9, sizeof(double) * 9 * c->n,
                                cudaMemcpyDeviceToHost, c->stream));
    HK_CUDA(cudaStreamSynchronize(c->stream));
    const int err = take_device_error(c);
    if (err != 0) return err;
    std::memcpy(out7, c->out_host, 7 * sizeof(double));
    return HAWKES_OK;
}

}  // namespace

extern "C" {

const char* hawkes_strerror(int status) {
    switch (status) {
        case HAWKES_OK: return "ok";
        case HAWKES_ERR_ARG: return "invalid argument";
        case HAWKES_ERR_UNSORTED: return "event times not positive and non-decreasing";
        case HAWKES_ERR_CUDA: return "CUDA runtime error";
        case HAWKES_ERR_NONFINITE: return "non-finite result";
        case HAWKES_ERR_TIMEOUT: return "a bounded device wait gave up";
        case HAWKES_ERR_OOM: return "device out of memory";
        case HAWKES_ERR_STATE: return "call out of order";
        case HAWKES_ERR_TOO_LARGE: return "size above the fixed scratch limit of the allocation-free entry point";
        case HAWKES_ERR_IO: return "file could not be written";
        case HAWKES_ERR_BOUNDS: return "a device-side index check of the debug build failed";
        default: return "unknown status";
    }
}

int hawkes_create(hawkes_ctx** out, int device, void* cuda_stream) {
    HK_NVTX("hawkes_create");
    if (!out) return HAWKES_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? HAWKES_ERR_ARG : HAWKES_ERR_CUDA;
    }
    DeviceGuard g(device);
    hawkes_ctx* c = new (std::nothrow) hawkes_ctx();
    if (!c) return HAWKES_ERR_OOM;
    c->device = device;
    int rc = HAWKES_OK;
    do {
        if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            rc = HAWKES_ERR_CUDA;
            break;
        }
        if (cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
                rc = HAWKES_ERR_CUDA;
                break;
            }
            c->own_stream = true;
        }
        if (sweep_setup_attributes() != cudaSuccess) { rc = HAWKES_ERR_CUDA; break; }
        c->variant = 0;
        c->variant_bpsm = sweep_blocks_per_sm(0);
        c->final_blocks = 2 * c->sms;
        if ((rc = dalloc(&c->ctr, CT_COUNT)) != HAWKES_OK) break;
        if ((rc = dalloc(&c->cc, CC_COUNT)) != HAWKES_OK) break;
        if ((rc = dalloc(&c->params_dev, 1)) != HAWKES_OK) break;
        if ((rc = dalloc(&c->out_dev, 8)) != HAWKES_OK) break;
        if ((rc = dalloc(&c->fix7, FIX_DOUBLES)) != HAWKES_OK) break;
        if ((rc = dalloc(&c->partials, static_cast<size_t>(PART_STRIDE * c->final_blocks))) != HAWKES_OK)
            break;
        if (cudaMallocHost(reinterpret_cast<void**>(&c->out_host), 8 * sizeof(double)) != cudaSuccess) {
            rc = HAWKES_ERR_OOM;
            break;
        }
        if (cudaEventCreate(&c->pev[0]) != cudaSuccess || cudaEventCreate(&c->pev[1]) != cudaSuccess) {
            rc = HAWKES_ERR_CUDA;
            break;
        }
        if (cudaMemsetAsync(c->ctr, 0, CT_COUNT * sizeof(int), c->stream) != cudaSuccess ||
            cudaMemsetAsync(c->cc, 0, CC_COUNT * sizeof(double), c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            rc = HAWKES_ERR_CUDA;
            break;
        }
    } while (0);
    if (rc != HAWKES_OK) {
        cudaGetLastError();
        hawkes_destroy(c);
        return rc;
    }
    *out = c;
    return HAWKES_OK;
}

void hawkes_destroy(hawkes_ctx* c) {
    HK_NVTX("hawkes_destroy");
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_events(c);
    free_counties(c);
    spatial_free(c);
    dfree(c->ctr); dfree(c->cc); dfree(c->params_dev); dfree(c->out_dev); dfree(c->fix7);
    dfree(c->partials);
    if (c->out_host) cudaFreeHost(c->out_host);
    for (auto& e : c->pev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

int64_t hawkes_num_events(const hawkes_ctx* c) { return c ? c->n : 0; }

int hawkes_set_events(hawkes_ctx* c, int64_t n, const double* t, const double* x, const double* y,
                      const int32_t* county, int32_t n_counties, const double* county_scale) {
    HK_NVTX("hawkes_set_events");
    if (!c || n < 1 || !t || !county || n_counties < 1 || !county_scale) return HAWKES_ERR_ARG;
    if ((x == nullptr) != (y == nullptr)) return HAWKES_ERR_ARG;
    if (n > (int64_t(1) << 31) - 2 * NPAD_MULT) return HAWKES_ERR_ARG;  // 32-bit event indices
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t npad = (n + NPAD_MULT - 1) / NPAD_MULT * NPAD_MULT;
    int rc = HAWKES_OK;
    auto fail = [&](int r) {
        free_events(c);
        return r;
    };
    if (!(c->t && c->n == n && c->n_counties == n_counties)) {
        // new sizes: (re)allocate; county triangles survive if the county count does
        const bool keep_counties = c->counties_ok && n_counties == c->n_counties;
        free_events(c);
        if (!keep_counties) free_counties(c);
        c->n = n;
        c->npad = npad;
        c->nblk = npad / TB;
        c->n_counties = n_counties;
        if ((rc = dalloc(&c->t, npad)) || (rc = dalloc(&c->x, npad)) || (rc = dalloc(&c->y, npad)) ||
            (rc = dalloc(&c->s, npad)) || (rc = dalloc(&c->scale_c, n_counties)) ||
            (rc = dalloc(&c->county, n)) || (rc = dalloc(&c->lo, npad)) ||
            (rc = dalloc(&c->hi, npad)) || (rc = dalloc(&c->tb, c->nblk)) ||
            (rc = dalloc(&c->rec, npad)) || (rc = dalloc(&c->acc, 6 * npad)) ||
            (rc = dalloc(&c->fixlist, npad)))
            return fail(rc);
    }
    cudaStream_t st = c->stream;
    if (cudaMemcpyAsync(c->t, t, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (x && cudaMemcpyAsync(c->x, x, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (y && cudaMemcpyAsync(c->y, y, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        cudaMemcpyAsync(c->county, county, n * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->scale_c, county_scale, n_counties * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return fail(HAWKES_ERR_CUDA);
    if (cudaMemsetAsync(c->ctr + CT_CEMAX, 0, sizeof(int), st) != cudaSuccess)
        return fail(HAWKES_ERR_CUDA);
    rc = timed(c, HAWKES_K_OTHER, [&] {
        k_setup<<<grid_for(c, npad), 256, 0, st>>>(c->t, c->x, c->y, c->county, n_counties,
                                                   c->scale_c, n, npad, x ? 1 : 0, c->s, c->lo,
                                                   c->hi, c->tb, c->ctr);
    });
    if (rc != HAWKES_OK) return fail(rc);
    const int err = take_device_error(c);
    if (err < 0) return fail(err);
    c->items_variant = -1;
    rc = ensure_items(c);
    if (rc != HAWKES_OK) return fail(rc);
    spatial_invalidate(c);  // the spatial order is rebuilt on its next use
    return HAWKES_OK;
}

int hawkes_set_counties(hawkes_ctx* c, int32_t n_tri, const int32_t* tri_county,
                        const double* tri_xy) {
    HK_NVTX("hawkes_set_counties");
    if (!c || n_tri < 1 || !tri_county || !tri_xy) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    free_counties(c);
    int rc;
    if ((rc = dalloc(&c->tri_county, n_tri)) || (rc = dalloc(&c->tri_xy, 6 * (size_t)n_tri)) ||
        (rc = dalloc(&c->tri_cum, n_tri)) || (rc = dalloc(&c->cfirst, c->n_counties)) ||
        (rc = dalloc(&c->clast, c->n_counties))) {
        free_counties(c);
        return rc;
    }
    c->n_tri = n_tri;
    cudaStream_t st = c->stream;
    if (cudaMemcpyAsync(c->tri_county, tri_county, n_tri * sizeof(int32_t), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(c->tri_xy, tri_xy, 6 * (size_t)n_tri * sizeof(double),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
        free_counties(c);
        return HAWKES_ERR_CUDA;
    }
    rc = timed(c, HAWKES_K_OTHER, [&] {
        k_tri_check<<<grid_for(c, n_tri), 256, 0, st>>>(c->tri_county, n_tri, c->n_counties, c->ctr);
    });
    if (rc == HAWKES_OK) rc = take_device_error(c);
    if (rc == HAWKES_OK)
        rc = timed(c, HAWKES_K_OTHER, [&] {
            k_tri_area<<<grid_for(c, n_tri), 256, 0, st>>>(c->tri_xy, n_tri, c->tri_cum, c->ctr);
        });
    if (rc == HAWKES_OK)
        rc = timed(c, HAWKES_K_OTHER, [&] {
            k_tri_county<<<grid_for(c, c->n_counties), 256, 0, st>>>(
                c->tri_county, n_tri, c->n_counties, c->tri_cum, c->cfirst, c->clast, c->ctr);
        });
    if (rc == HAWKES_OK) rc = take_device_error(c);
    if (rc != HAWKES_OK) {
        free_counties(c);
        return rc;
    }
    c->counties_ok = true;
    return HAWKES_OK;
}

int hawkes_resample_locations(hawkes_ctx* c, uint64_t seed, uint64_t stream, uint64_t iteration) {
    HK_NVTX("hawkes_resample_locations");
    if (!c) return HAWKES_ERR_ARG;
    if (c->n == 0 || !c->counties_ok) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    return timed(c, HAWKES_K_RESAMPLE, [&] {
        k_resample<<<grid_for(c, c->n), 256, 0, c->stream>>>(c->county, c->n, c->tri_xy, c->tri_cum,
                                                             c->cfirst, c->clast, seed, stream,
                                                             iteration, nullptr, c->x, c->y);
    });
}

int hawkes_get_locations(hawkes_ctx* c, double* x, double* y) {
    HK_NVTX("hawkes_get_locations");
    if (!c || !x || !y) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    HK_CUDA(cudaMemcpyAsync(x, c->x, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HK_CUDA(cudaMemcpyAsync(y, c->y, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HK_CUDA(cudaStreamSynchronize(c->stream));
    return HAWKES_OK;
}

int hawkes_loglik_grad(hawkes_ctx* c, const hawkes_params* p, uint32_t flags, int64_t row_begin,
                       int64_t row_end, double* loglik, double* grad) {
    HK_NVTX("hawkes_loglik_grad");
    if (!c || !p || !loglik || !grad) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    if (row_begin < 0 || row_end > c->n || row_begin >= row_end) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    double out[7];
    HK_TRY(sync_loglik(c, p, flags, row_begin, row_end, out, nullptr));
    *loglik = out[0];
    for (int k = 0; k < 6; ++k) grad[k] = out[1 + k];
    return HAWKES_OK;
}

int hawkes_loglik_grad_async(hawkes_ctx* c, const hawkes_params* d_params, uint32_t flags,
                             double* d_out) {
    HK_NVTX("hawkes_loglik_grad_async");
    if (!c || !d_params || !d_out || !aligned8(d_params) || !aligned8(d_out)) return HAWKES_ERR_ARG;
    if ((flags & ~kFlagsAll) != 0) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    return enqueue_loglik(c, d_params, flags, 0, c->n, d_out, nullptr);
}

int hawkes_loglik_rows(hawkes_ctx* c, const hawkes_params* p, uint32_t flags, double* out7,
                       double* rows) {
    HK_NVTX("hawkes_loglik_rows");
    if (!c || !p || !out7 || !rows) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    return sync_loglik(c, p, flags, 0, c->n, out7, rows);
}

int hawkes_check_bounded_wait(hawkes_ctx* c, double* seconds) {
    HK_NVTX("hawkes_check_bounded_wait");
    if (!c) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    const int pending = take_device_error(c);  // do not mistake an earlier error for the test's
    if (pending != HAWKES_OK) return pending;
    HK_CUDA(cudaEventRecord(c->pev[0], c->stream));
    k_wait_selftest<<<1, 32, 0, c->stream>>>(c->ctr);
    HK_CUDA(cudaGetLastError());
    HK_CUDA(cudaEventRecord(c->pev[1], c->stream));
    HK_CUDA(cudaEventSynchronize(c->pev[1]));
    float ms = 0.f;
    HK_CUDA(cudaEventElapsedTime(&ms, c->pev[0], c->pev[1]));
    if (seconds) *seconds = ms / 1000.0;
    const int err = take_device_error(c);
    return err == HAWKES_ERR_TIMEOUT ? HAWKES_OK : (err == HAWKES_OK ? HAWKES_ERR_STATE : err);
}

int hawkes_shard_bounds(int64_t n, int64_t tile_rows, int nshards, int64_t* bounds) {
    if (n < 1 || tile_rows < 1 || nshards < 1 || !bounds) return HAWKES_ERR_ARG;
    const int64_t nI = (n + tile_rows - 1) / tile_rows;
    // pairs (i, j < i) of row tile I: sum of i over its rows [a, b)
    std::vector<double> cum(static_cast<size_t>(nI) + 1, 0.0);
    for (int64_t I = 0; I < nI; ++I) {
        const int64_t a = I * tile_rows, b = std::min(a + tile_rows, n);
        cum[I + 1] = cum[I] + static_cast<double>(b - a) * static_cast<double>(a + b - 1) / 2.0;
    }
    bounds[0] = 0;
    int64_t k = 0;
    for (int g = 1; g < nshards; ++g) {
        const double target = cum[nI] * g / nshards;
        while (k < nI && cum[k] < target) ++k;  // first tile boundary at or past the target
        int64_t pick = k;
        if (pick > 0 && target - cum[pick - 1] < cum[pick] - target) --pick;  // the nearer one
        const int64_t b = std::min(pick * tile_rows, n);
        bounds[g] = b > bounds[g - 1] ? b : bounds[g - 1];
    }
    bounds[nshards] = n;
    return HAWKES_OK;
}

int64_t hawkes_shard_tile_rows(const hawkes_ctx* c) {
    return c ? static_cast<int64_t>(sweep_variant_rows(c->variant)) : HAWKES_ERR_ARG;
}

int hawkes_shard_moments(hawkes_ctx* c, const hawkes_params* d_params, uint32_t flags, int shard,
                         int nshards, double* d_moments) {
    HK_NVTX("hawkes_shard_moments");
    if (!c || !d_params || !d_moments || !aligned8(d_params) || !aligned8(d_moments))
        return HAWKES_ERR_ARG;
    if (nshards < 1 || shard < 0 || shard >= nshards) return HAWKES_ERR_ARG;
    if ((flags & ~kFlagsAll) != 0 || (flags & (HAWKES_F64 | HAWKES_SKIP_SPATIAL)) != 0)
        return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    const int key[3] = {nshards, shard, c->variant};
    if (!(c->shard_items && key[0] == c->shard_key[0] && key[1] == c->shard_key[1] &&
          key[2] == c->shard_key[2])) {
        // this shard's row tiles of the symmetric work list (synchronous)
        drop_shard_items(c);
        const int64_t tr = sweep_variant_rows(c->variant);
        std::vector<int64_t> b(static_cast<size_t>(nshards) + 1);
        HK_TRY(hawkes_shard_bounds(c->n, tr, nshards, b.data()));
        const int64_t I0 = b[shard] / tr, I1 = (b[shard + 1] + tr - 1) / tr;
        std::vector<int4> mine;
        for (const int4& it : sweep_items(c->n, c->variant))
            if (it.x >= I0 && it.x < I1) mine.push_back(it);
        HK_TRY(dalloc(&c->shard_items, mine.size()));
        HK_CUDA(cudaMemcpyAsync(c->shard_items, mine.data(), mine.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, c->stream));
        HK_CUDA(cudaStreamSynchronize(c->stream));
        c->shard_nitems = static_cast<int>(mine.size());
        for (int q = 0; q < 3; ++q) c->shard_key[q] = key[q];
    }
    const int model = static_cast<int>(flags & kModelBits);
    const int skip = (flags & HAWKES_SKIP_UNDERFLOW) ? 1 : 0;
    HK_TRY(timed(c, HAWKES_K_PREP, [&] {
        k_prep<<<grid_for(c, c->npad), 256, 0, c->stream>>>(c->t, c->x, c->y, c->s, c->tb, d_params,
                                                            model, 1, skip, c->n, c->npad, c->rec,
                                                            c->acc, c->cc, c->ctr, c->fix7);
    }));
    cudaError_t se = cudaSuccess;
    HK_TRY(timed(c, HAWKES_K_SWEEP, [&] {
        se = launch_sweep_list(c, c->shard_items, c->shard_nitems, (flags & HAWKES_BG_TIME) != 0,
                               (flags & HAWKES_LOGLIK_ONLY) != 0);
    }));
    HK_CUDA(se);
    HK_CUDA(cudaMemcpy2DAsync(d_moments, c->n * sizeof(double), c->acc, c->npad * sizeof(double),
                              c->n * sizeof(double), 6, cudaMemcpyDeviceToDevice, c->stream));
    return HAWKES_OK;
}

int hawkes_finalize_moments(hawkes_ctx* c, const hawkes_params* d_params, uint32_t flags,
                            const double* d_moments, double* d_out) {
    HK_NVTX("hawkes_finalize_moments");
    if (!c || !d_params || !d_moments || !d_out || !aligned8(d_params) || !aligned8(d_moments) ||
        !aligned8(d_out))
        return HAWKES_ERR_ARG;
    if ((flags & ~kFlagsAll) != 0 || (flags & (HAWKES_F64 | HAWKES_SKIP_SPATIAL)) != 0)
        return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    DeviceGuard g(c->device);
    const int model = static_cast<int>(flags & kModelBits);
    HK_TRY(timed(c, HAWKES_K_PREP, [&] {  // constants and counters (nothing staged)
        k_prep<<<grid_for(c, c->npad), 256, 0, c->stream>>>(c->t, c->x, c->y, c->s, c->tb, d_params,
                                                            model, 0, 0, c->n, c->npad, c->rec,
                                                            c->acc, c->cc, c->ctr, c->fix7);
    }));
    HK_CUDA(cudaMemcpy2DAsync(c->acc, c->npad * sizeof(double), d_moments, c->n * sizeof(double),
                              c->n * sizeof(double), 6, cudaMemcpyDeviceToDevice, c->stream));
    return enqueue_finalize32(c, model, 0, c->n, d_out, nullptr);
}

int hawkes_sweep_variants(void) { return sweep_num_variants(); }

int hawkes_set_sweep_variant(hawkes_ctx* c, int variant) {
    HK_NVTX("hawkes_set_sweep_variant");
    if (!c) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    return select_variant(c, variant);
}

int hawkes_get_sweep_variant(const hawkes_ctx* c) { return c ? c->variant : HAWKES_ERR_ARG; }

int hawkes_tune(hawkes_ctx* c, const hawkes_params* p, uint32_t flags, int reps, int* chosen,
                double* ms) {
    HK_NVTX("hawkes_tune");
    if (!c || !p || reps < 1) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    if (!params_ok(p) ||
        (flags & ~(kFlagsAll & ~static_cast<uint32_t>(HAWKES_F64 | HAWKES_SKIP_SPATIAL))) != 0)
        return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    const bool prof = c->prof;
    const hawkes_profile saved = c->pacc;
    int best = -1;
    double best_ms = 0.0;
    double out7[7];
    for (int v = 0; v < sweep_num_variants(); ++v) {
        HK_TRY(select_variant(c, v));
        HK_TRY(sync_loglik(c, p, flags, 0, c->n, out7, nullptr));  // warm-up
        c->prof = true;
        std::memset(&c->pacc, 0, sizeof(c->pacc));
        for (int r = 0; r < reps; ++r) HK_TRY(sync_loglik(c, p, flags, 0, c->n, out7, nullptr));
        const double t = c->pacc.ms[HAWKES_K_SWEEP] / reps;
        c->prof = prof;
        if (ms) ms[v] = t;
        if (best < 0 || t < best_ms) {
            best = v;
            best_ms = t;
        }
    }
    c->pacc = saved;
    c->prof = prof;
    if (chosen) *chosen = best;
    return select_variant(c, best);
}

int hawkes_profile_enable(hawkes_ctx* c, int on) {
    HK_NVTX("hawkes_profile_enable");
    if (!c) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    c->prof = on != 0;
    if (c->prof) std::memset(&c->pacc, 0, sizeof(c->pacc));
    return HAWKES_OK;
}

int hawkes_profile_read(hawkes_ctx* c, hawkes_profile* out) {
    HK_NVTX("hawkes_profile_read");
    if (!c || !out) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    *out = c->pacc;
    return HAWKES_OK;
}

}  // extern "C"

namespace hk {
int tune_cache_get(const char* path, const char* key, int* variant, int* chunk, int* order,
                   double* ms, int* kc);
int tune_cache_put(const char* path, const char* key, int variant, int chunk, int order, double ms,
                   int kc);
int log2_ceil(double v);
std::string device_key();
}  // namespace hk

int hawkes_tune_cached(hawkes_ctx* c, const hawkes_params* p, uint32_t flags, int reps,
                       const char* cache_path, int* chosen, int* from_cache) {
    HK_NVTX("hawkes_tune_cached");
    using namespace hk;
    if (!c || !p || reps < 1 || !cache_path) return HAWKES_ERR_ARG;
    if (c->n == 0) return HAWKES_ERR_STATE;
    if (!params_ok(p) ||
        (flags & ~(kFlagsAll & ~static_cast<uint32_t>(HAWKES_F64 | HAWKES_SKIP_SPATIAL))) != 0)
        return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    const std::string dk = device_key();
    if (dk.empty()) return HAWKES_ERR_CUDA;
    const std::string key = dk + "single|n<=2^" + std::to_string(log2_ceil(static_cast<double>(c->n))) +
                            "|flags=" + std::to_string(flags);
    int v = -1;
    if (tune_cache_get(cache_path, key.c_str(), &v, nullptr, nullptr, nullptr, nullptr) == 1) {
        HK_TRY(select_variant(c, v));
        if (chosen) *chosen = v;
        if (from_cache) *from_cache = 1;
        return HAWKES_OK;
    }
    std::vector<double> ms(sweep_num_variants());
    HK_TRY(hawkes_tune(c, p, flags, reps, &v, ms.data()));
    if (chosen) *chosen = v;
    if (from_cache) *from_cache = 0;
    return tune_cache_put(cache_path, key.c_str(), v, CHUNK, 0, ms[v], 1);
}

int hawkes_debug_build(void) { return kDebug ? 1 : 0; }

int hawkes_debug_set_item(hawkes_ctx* c, int k, int row_tile, int col_begin, int col_end) {
    HK_NVTX("hawkes_debug_set_item");
    if (!kDebug) return HAWKES_ERR_STATE;
    if (!c || k < 0 || k >= c->nitems || !c->items) return HAWKES_ERR_ARG;
    DeviceGuard g(c->device);
    HK_CUDA(cudaStreamSynchronize(c->stream));
    const int4 it = make_int4(row_tile, col_begin, col_end, 0);
    HK_CUDA(cudaMemcpy(c->items + k, &it, sizeof(int4), cudaMemcpyHostToDevice));
    c->items_variant = -1;  // rebuilt by the next variant selection or event set
    return HAWKES_OK;
}

int hawkes_set_spatial_window(hawkes_ctx* c, int64_t events) {
    HK_NVTX("hawkes_set_spatial_window");
    if (!c || events < TC) return HAWKES_ERR_ARG;
    return spatial_set_window(c, events);
}
