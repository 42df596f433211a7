// hawkes_loglik_grad_noalloc: the FP32 log-likelihood + gradient for callers
// that must not allocate device memory, with every scratch buffer carved out
// of one fixed array that lives in this library's device image.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// wanted, e.g. inside a custom device-memory allocator or a memory-pool
// callback (allocating there would recurse), in an application that reserves
// all device memory up front and accounts for every byte, or in a host thread
// that must never block on the allocator's device-wide synchronisation.  They
// pass device pointers to their own inputs and output; nothing else is
// allocated, freed or requested from any library (PyTorch included).
//
// The scratch array below is a file-scope __device__ variable: every GPU that
// loads this library holds it (about 10 MB) until the process exits.  In host
// code its name is only a host-side stand-in, not a device address, so the
// first call on each device looks up the real address with
// cudaGetSymbolAddress (with that device current) and passes it to the
// kernels.  All calls on a device share the array and it keeps the last
// call's contents; each call clears what must start at zero.  Calls whose
// work overlaps on the GPU (other streams, other host threads) race on it.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace hk {
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
cudaError_t sweep_setup_attributes();
int sweep_blocks_per_sm(int v);
int sweep_variant_rows(int v);
cudaError_t launch_sweep(hawkes_ctx* c, bool sym, int64_t row_begin, int64_t row_end, bool bgt,
                         bool ll);
}  // namespace hk

using namespace hk;

namespace {

// Largest event count the fixed scratch holds (a multiple of NPAD_MULT).
constexpr int64_t kMaxN = HAWKES_NOALLOC_MAX_N;
static_assert(kMaxN % NPAD_MULT == 0, "scratch holds whole row tiles");
constexpr int kMaxFinalBlocks = 512;
constexpr int kMaxItems = 4096;
constexpr int kVariant = 0;  // sweep variant used by this entry point

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// Scratch layout (byte offsets).
constexpr size_t OFF_T = 0;
constexpr size_t OFF_X = OFF_T + align256(kMaxN * sizeof(double));
constexpr size_t OFF_Y = OFF_X + align256(kMaxN * sizeof(double));
constexpr size_t OFF_S = OFF_Y + align256(kMaxN * sizeof(double));
constexpr size_t OFF_LO = OFF_S + align256(kMaxN * sizeof(double));
constexpr size_t OFF_HI = OFF_LO + align256(kMaxN * sizeof(int32_t));
constexpr size_t OFF_TB = OFF_HI + align256(kMaxN * sizeof(int32_t));
constexpr size_t OFF_REC = OFF_TB + align256((kMaxN / TB) * sizeof(double));
constexpr size_t OFF_ACC = OFF_REC + align256(kMaxN * sizeof(Rec));
constexpr size_t OFF_FIX = OFF_ACC + align256(6 * kMaxN * sizeof(double));
constexpr size_t OFF_PART = OFF_FIX + align256(kMaxN * sizeof(int));
constexpr size_t OFF_FIX7 = OFF_PART + align256(PART_STRIDE * kMaxFinalBlocks * sizeof(double));
constexpr size_t OFF_CTR = OFF_FIX7 + align256(FIX_DOUBLES * sizeof(double));
constexpr size_t OFF_CC = OFF_CTR + align256(CT_COUNT * sizeof(int));
constexpr size_t OFF_ITEMS = OFF_CC + align256(CC_COUNT * sizeof(double));
constexpr size_t SCRATCH_BYTES = OFF_ITEMS + align256(kMaxItems * sizeof(int4));

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool done = false;
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
    int bpsm = 1;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Copy the caller's events into the padded scratch arrays, check them, and
// build the tie ranges and block time bases (same rules as hawkes_set_events).
__global__ void k_na_setup(const double* __restrict__ t_in, const double* __restrict__ x_in,
                           const double* __restrict__ y_in, const double* __restrict__ s_in,
                           int64_t n, int64_t npad, double* t, double* x, double* y, double* s,
                           int32_t* lo, int32_t* hi, double* tb, int* ctr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npad;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n) {
            const double te = t_in[e];
            if (!(te > 0.0) || !isfinite(te) || (e + 1 < n && !(te <= t_in[e + 1])))
                set_error(ctr, HAWKES_ERR_UNSORTED);
            const double se = s_in ? s_in[e] : 1.0;
            if (!(se > 0.0) || !isfinite(se) || !isfinite(x_in[e]) || !isfinite(y_in[e]))
                set_error(ctr, HAWKES_ERR_ARG);
            // largest -2 log2 s_j above 0 (the excitation flush bound reads it)
            const float ce = static_cast<float>(-2.0 * log2(se));
            if (ce > 0.f) atomicMax(ctr + CT_CEMAX, __float_as_int(ce));
            t[e] = te;
            x[e] = x_in[e];
            y[e] = y_in[e];
            s[e] = se;
            int64_t a = 0, b = n;  // first index with t >= te
            while (a < b) {
                const int64_t m = (a + b) >> 1;
                if (t_in[m] < te) a = m + 1; else b = m;
            }
            lo[e] = static_cast<int32_t>(a);
            a = 0;
            b = n;  // first index with t > te
            while (a < b) {
                const int64_t m = (a + b) >> 1;
                if (t_in[m] <= te) a = m + 1; else b = m;
            }
            hi[e] = static_cast<int32_t>(a);
        } else {
            t[e] = t_in[n - 1];
            x[e] = 0.0;
            y[e] = 0.0;
            s[e] = 1.0;
            lo[e] = 0;
            hi[e] = 0;
        }
        if (e % TB == 0) tb[e / TB] = t_in[e < n ? e : n - 1];
    }
}

// Symmetric work list (row tile, column tiles [jb, je)), largest row tiles first.
__global__ void k_na_items(int64_t n, int tr, int4* items) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t nI = (n + tr - 1) / tr;
    int k = 0;
    for (int64_t I = nI - 1; I >= 0; --I) {
        const int64_t last = (I + 1) * tr < n ? (I + 1) * tr : n;
        const int nJ = static_cast<int>((last + TC - 1) / TC);
        for (int jb = 0; jb < nJ && k < kMaxItems; jb += CHUNK)
            items[k++] = make_int4(static_cast<int>(I), jb, jb + CHUNK < nJ ? jb + CHUNK : nJ, 0);
    }
}

__global__ void k_na_nan_on_error(const int* ctr, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && ctr[CT_ERR] != 0)
        for (int q = 0; q < 7; ++q) out[q] = nan("");
}

int items_for(int64_t n, int tr) {
    const int64_t nI = (n + tr - 1) / tr;
    int64_t k = 0;
    for (int64_t I = 0; I < nI; ++I) {
        const int64_t last = (I + 1) * tr < n ? (I + 1) * tr : n;
        const int64_t nJ = (last + TC - 1) / TC;
        k += (nJ + CHUNK - 1) / CHUNK;
    }
    return static_cast<int>(k);
}

// First call on a device: resolve the scratch array's device address (with
// that device current) and prepare the sweep kernel's launch attributes.
int device_setup(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= kMaxDevices) return HAWKES_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.done) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return HAWKES_ERR_CUDA;
        }
        if (sweep_setup_attributes() != cudaSuccess ||
            cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return HAWKES_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char*>(p);
        d.bpsm = sweep_blocks_per_sm(kVariant);
        d.done = true;
    }
    *out = &d;
    return HAWKES_OK;
}

}  // namespace

extern "C" int hawkes_loglik_grad_noalloc(const double* d_t, const double* d_x, const double* d_y,
                                          const double* d_s, int64_t n,
                                          const hawkes_params* d_params, uint32_t flags,
                                          double* d_out, void* cuda_stream) {
    if (!d_t || !d_x || !d_y || !d_params || !d_out) return HAWKES_ERR_ARG;
    for (const void* p : {static_cast<const void*>(d_t), static_cast<const void*>(d_x),
                          static_cast<const void*>(d_y), static_cast<const void*>(d_s),
                          static_cast<const void*>(d_params), static_cast<const void*>(d_out)})
        if (!aligned8(p)) return HAWKES_ERR_ARG;  // NULL d_s is aligned
    if ((flags & ~static_cast<uint32_t>(HAWKES_MODEL1 | HAWKES_BG_TIME)) != 0)
        return HAWKES_ERR_ARG;  // FP32 only
    if (n < 1) return HAWKES_ERR_ARG;
    if (n > kMaxN) return HAWKES_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HAWKES_ERR_CUDA;
    }
    DeviceSetup* d = nullptr;
    const int rc = device_setup(dev, &d);
    if (rc != HAWKES_OK) return rc;

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = d->scratch;
    const int tr = sweep_variant_rows(kVariant);
    const int64_t npad = (n + NPAD_MULT - 1) / NPAD_MULT * NPAD_MULT;

    // A context on the stack that points into the scratch array; only the
    // fields the launch helpers read are set.
    hawkes_ctx c;
    c.device = dev;
    c.stream = st;
    c.sms = d->sms;
    c.n = n;
    c.npad = npad;
    c.nblk = npad / TB;
    c.t = reinterpret_cast<double*>(base + OFF_T);
    c.x = reinterpret_cast<double*>(base + OFF_X);
    c.y = reinterpret_cast<double*>(base + OFF_Y);
    c.s = reinterpret_cast<double*>(base + OFF_S);
    c.lo = reinterpret_cast<int32_t*>(base + OFF_LO);
    c.hi = reinterpret_cast<int32_t*>(base + OFF_HI);
    c.tb = reinterpret_cast<double*>(base + OFF_TB);
    c.rec = reinterpret_cast<Rec*>(base + OFF_REC);
    c.acc = reinterpret_cast<double*>(base + OFF_ACC);
    c.fixlist = reinterpret_cast<int*>(base + OFF_FIX);
    c.partials = reinterpret_cast<double*>(base + OFF_PART);
    c.fix7 = reinterpret_cast<double*>(base + OFF_FIX7);
    c.ctr = reinterpret_cast<int*>(base + OFF_CTR);
    c.cc = reinterpret_cast<double*>(base + OFF_CC);
    c.items = reinterpret_cast<int4*>(base + OFF_ITEMS);
    c.nitems = items_for(n, tr);
    c.variant = kVariant;
    c.variant_bpsm = d->bpsm;
    c.final_blocks = 2 * d->sms < kMaxFinalBlocks ? 2 * d->sms : kMaxFinalBlocks;
    if (c.nitems > kMaxItems) return HAWKES_ERR_TOO_LARGE;
    const int model = static_cast<int>(flags & (HAWKES_MODEL1 | HAWKES_BG_TIME));
    int grid = static_cast<int>((npad + 255) / 256);
    if (grid > 8 * c.sms) grid = 8 * c.sms;

    // Counters and the error flag start at zero on every call.
    if (cudaMemsetAsync(c.ctr, 0, CT_COUNT * sizeof(int), st) != cudaSuccess) return HAWKES_ERR_CUDA;
    k_na_setup<<<grid, 256, 0, st>>>(d_t, d_x, d_y, d_s, n, npad, c.t, c.x, c.y, c.s, c.lo, c.hi,
                                     c.tb, c.ctr);
    k_na_items<<<1, 32, 0, st>>>(n, tr, c.items);
    k_prep<<<grid, 256, 0, st>>>(c.t, c.x, c.y, c.s, c.tb, d_params, model, 1, 0, n, npad, c.rec,
                                 c.acc, c.cc, c.ctr, c.fix7);
    if (launch_sweep(&c, true, 0, n, (flags & HAWKES_BG_TIME) != 0, false) != cudaSuccess) return HAWKES_ERR_CUDA;
    k_finalize<<<c.final_blocks, 256, 0, st>>>(c.acc, c.t, c.lo, c.hi, c.cc, n, npad, 0, n, 1,
                                               c.fixlist, c.ctr, c.partials, nullptr);
    k_rows64<<<c.sms, 256, 0, st>>>(c.t, c.x, c.y, c.s, c.lo, c.hi, c.cc, model, n, npad, 0, 0, 1,
                                    c.fixlist, c.ctr, c.acc, c.fix7, nullptr);
    k_reduce<<<1, 256, 0, st>>>(c.partials, c.final_blocks, c.fix7, c.cc, n, d_out, c.ctr);
    k_flushfix<<<c.sms, 256, 0, st>>>(c.acc, c.t, c.x, c.y, c.s, c.lo, c.hi, c.cc, model, n, npad,
                                      0, n, c.ctr, c.fix7, d_out, nullptr);
    k_na_nan_on_error<<<1, 32, 0, st>>>(c.ctr, d_out);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ERR_CUDA;
}
