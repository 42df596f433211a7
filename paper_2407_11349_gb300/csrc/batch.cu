// Batched evaluation: many problems (MCMC chains with their own parameters
// and location draws, and regional subsets of uneven size) in one persistent
// pair-sweep launch, optionally captured with the per-problem O(N) kernels in
// one CUDA graph.  The paper ran its 30 chains as separate cluster jobs
// (Sec. 3.2); here they share one GPU and one work queue.
//
// Chains per CTA: problems whose event times are identical (chains of one data
// set) can be swept kc at a time by the group kernel (sweep_group.cu), which
// forms each pair's time difference once for all kc chains; the other
// problems go through the one-problem-per-item batch kernel.  kc is a tuner
// knob beside the sweep variant, the chunk length and the item order.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

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
__global__ void k_resample(const int32_t*, int64_t, const double*, const double*, const int32_t*,
                           const int32_t*, uint64_t, uint64_t, uint64_t, const uint64_t*, double*,
                           double*);
int sweep_num_variants();
int sweep_blocks_per_sm(int v);
struct GroupDesc;
bool group_kc_supported(int kc);
int group_blocks_per_sm(int kc);
size_t group_tile_bytes(int kc);
cudaError_t group_setup_attributes();
std::vector<int4> group_items(const std::vector<int64_t>& ns, int kc, int chunk);
cudaError_t launch_group_stage(cudaStream_t st, int sms, const GroupDesc& gd,
                               const Rec* const* recs, const double* t, int kc, float4* out);
cudaError_t launch_sweep_group(cudaStream_t st, int kc, int grid, const GroupDesc* groups,
                               int ngroups, const int4* items, int nitems, int* ctr);
std::vector<int4> sweep_items_batch(const std::vector<int64_t>& ns, int v, int chunk, int order);
cudaError_t launch_sweep_batch(cudaStream_t st, int variant, int grid, const ProbDesc* probs,
                               int nprobs, const int4* items, int nitems, int* ctr, bool bgt,
                               bool ll);

__global__ void k_set_u64(uint64_t* dst, uint64_t v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}
int tune_cache_get(const char* path, const char* key, int* variant, int* chunk, int* order,
                   double* ms, int* kc);
int tune_cache_put(const char* path, const char* key, int variant, int chunk, int order, double ms,
                   int kc);
int log2_ceil(double v);
std::string device_key();
}  // namespace hk

using namespace hk;

struct hawkes_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    uint32_t flags = 0;
    std::vector<hawkes_ctx*> probs;
    std::vector<uint64_t> seeds, streams;
    bool resample = false;
    ProbDesc* d_probs = nullptr;
    int4* d_items = nullptr;
    int nitems = 0;
    int variant = 0;
    int chunk = CHUNK;
    int order = 1;
    int grid = 0;
    int* d_ctr = nullptr;        // [2 CT_COUNT]: work cursor, latched error (batch kernel, group kernel)
    uint64_t* d_iter = nullptr;  // iteration read by the resample kernels
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const hawkes_params* g_params = nullptr;  // pointers the graph was captured with
    double* g_out = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // the per-problem O(N) kernels run on NAUX side streams forked from and
    // joined back into `stream` (branches of the captured graph)
    static constexpr int NAUX = 4;
    cudaStream_t aux[NAUX] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[NAUX] = {nullptr, nullptr, nullptr, nullptr};
    // chains per CTA (sweep_group.cu)
    int kc = 1;
    std::vector<std::vector<int>> tclass;  // problems with identical event times, in input order
    std::vector<std::vector<int>> groups;  // groups of kc problems of one class (kc > 1)
    std::vector<int> singles;              // problems in the one-problem batch kernel
    std::vector<GroupDesc> h_groups;
    GroupDesc* d_groups = nullptr;
    int4* d_gitems = nullptr;
    int ngitems = 0;
    float4* d_gtiles = nullptr;
    size_t gtiles_cap = 0;                 // bytes allocated at d_gtiles
    std::vector<size_t> gtile_off;         // per group: first float4 of its tiles
    int ggrid = 0;
};

namespace {

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

int st_of(cudaError_t e) {
    if (e == cudaSuccess) return HAWKES_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HAWKES_ERR_OOM : HAWKES_ERR_CUDA;
}

#define HB_TRY(expr)                       \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != HAWKES_OK) return _rc;  \
    } while (0)
#define HB_CUDA(expr) HB_TRY(st_of(expr))

void drop_graph(hawkes_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->g_params = nullptr;
    b->g_out = nullptr;
}

// Classes of problems whose event times are identical (same n, the same
// doubles): chains of one data set.  Read back once when the batch is made.
int time_classes(hawkes_batch* b) {
    b->tclass.clear();
    std::vector<std::vector<double>> rep_t;  // each class's times
    std::vector<double> t;
    for (size_t p = 0; p < b->probs.size(); ++p) {
        const hawkes_ctx* c = b->probs[p];
        t.resize(static_cast<size_t>(c->n));
        HB_CUDA(cudaMemcpy(t.data(), c->t, t.size() * sizeof(double), cudaMemcpyDeviceToHost));
        size_t k = 0;
        for (; k < rep_t.size(); ++k)
            if (rep_t[k].size() == t.size() &&
                std::memcmp(rep_t[k].data(), t.data(), t.size() * sizeof(double)) == 0)
                break;
        if (k == rep_t.size()) {
            rep_t.push_back(t);
            b->tclass.emplace_back();
        }
        b->tclass[k].push_back(static_cast<int>(p));
    }
    return HAWKES_OK;
}

// Flags the group kernel covers: the space-time background with its full
// gradient, Model 1 or 2, no tile skipping.
bool group_flags_ok(uint32_t flags) {
    return (flags & (HAWKES_BG_TIME | HAWKES_LOGLIK_ONLY | HAWKES_SKIP_UNDERFLOW)) == 0;
}

// Largest class of problems with identical event times.
size_t largest_class(const hawkes_batch* b) {
    size_t m = 0;
    for (const auto& c : b->tclass) m = std::max(m, c.size());
    return m;
}

// Split the problems into groups of b->kc chains with identical times and
// singles, and (kc > 1) build the groups' descriptors, tile buffer and work
// list.
int build_groups(hawkes_batch* b, int chunk) {
    b->groups.clear();
    b->singles.clear();
    b->h_groups.clear();
    b->gtile_off.clear();
    b->ngitems = 0;
    std::vector<char> grouped(b->probs.size(), 0);
    if (b->kc > 1)
        for (const auto& cls : b->tclass)
            for (size_t s = 0; s + b->kc <= cls.size(); s += b->kc) {
                b->groups.emplace_back(cls.begin() + s, cls.begin() + s + b->kc);
                for (int k = 0; k < b->kc; ++k) grouped[cls[s + k]] = 1;
            }
    for (size_t p = 0; p < b->probs.size(); ++p)
        if (!grouped[p]) b->singles.push_back(static_cast<int>(p));
    if (b->groups.empty()) return HAWKES_OK;
    size_t tot = 0;
    std::vector<int64_t> ns;
    for (const auto& g : b->groups) {
        const hawkes_ctx* c0 = b->probs[g[0]];
        b->gtile_off.push_back(tot);
        tot += static_cast<size_t>(c0->npad / TC) * gt_f4(b->kc);
        ns.push_back(c0->n);
    }
    if (tot * sizeof(float4) > b->gtiles_cap) {
        if (b->d_gtiles) cudaFree(b->d_gtiles);
        b->d_gtiles = nullptr;
        b->gtiles_cap = 0;
        HB_CUDA(cudaMalloc(&b->d_gtiles, tot * sizeof(float4)));
        b->gtiles_cap = tot * sizeof(float4);
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const auto& g = b->groups[gi];
        const hawkes_ctx* c0 = b->probs[g[0]];
        GroupDesc d{};
        d.tiles = b->d_gtiles + b->gtile_off[gi];
        d.lo = c0->lo;
        d.tb = c0->tb;
        for (int k = 0; k < b->kc; ++k) {
            d.cc[k] = b->probs[g[k]]->cc;
            d.acc[k] = b->probs[g[k]]->acc;
        }
        d.n = c0->n;
        d.npad = c0->npad;
        b->h_groups.push_back(d);
    }
    const std::vector<int4> items = group_items(ns, b->kc, chunk);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_gitems) cudaFree(b->d_gitems);
    b->d_groups = nullptr;
    b->d_gitems = nullptr;
    HB_CUDA(cudaMalloc(&b->d_groups, b->h_groups.size() * sizeof(GroupDesc)));
    HB_CUDA(cudaMalloc(&b->d_gitems, std::max<size_t>(items.size(), 1) * sizeof(int4)));
    HB_CUDA(cudaMemcpyAsync(b->d_groups, b->h_groups.data(), b->h_groups.size() * sizeof(GroupDesc),
                            cudaMemcpyHostToDevice, b->stream));
    HB_CUDA(cudaMemcpyAsync(b->d_gitems, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, b->stream));
    HB_CUDA(cudaStreamSynchronize(b->stream));
    b->ngitems = static_cast<int>(items.size());
    b->ggrid = b->sms * group_blocks_per_sm(b->kc);
    return HAWKES_OK;
}

int build_items(hawkes_batch* b, int variant, int chunk, int order) {
    HB_TRY(build_groups(b, chunk));
    std::vector<int64_t> ns;
    for (int p : b->singles) ns.push_back(b->probs[p]->n);
    std::vector<int4> items = sweep_items_batch(ns, variant, chunk, order);
    for (int4& it : items) it.w = b->singles[it.w];  // index into all problems
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    HB_CUDA(cudaMalloc(&b->d_items, std::max<size_t>(items.size(), 1) * sizeof(int4)));
    HB_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, b->stream));
    HB_CUDA(cudaStreamSynchronize(b->stream));
    b->nitems = static_cast<int>(items.size());
    b->variant = variant;
    b->chunk = chunk;
    b->order = order;
    b->grid = b->sms * sweep_blocks_per_sm(variant);
    drop_graph(b);  // a captured graph refers to the old work list
    return HAWKES_OK;
}

// Make the side streams wait for the work queued so far on the batch's stream,
// and the batch's stream wait for the side streams.
int fork_side(hawkes_batch* b) {
    HB_CUDA(cudaEventRecord(b->fork_ev, b->stream));
    for (cudaStream_t s : b->aux) HB_CUDA(cudaStreamWaitEvent(s, b->fork_ev, 0));
    return HAWKES_OK;
}
int join_side(hawkes_batch* b) {
    for (int k = 0; k < hawkes_batch::NAUX; ++k) {
        HB_CUDA(cudaEventRecord(b->join_ev[k], b->aux[k]));
        HB_CUDA(cudaStreamWaitEvent(b->stream, b->join_ev[k], 0));
    }
    return HAWKES_OK;
}

// Queue one batched evaluation.  d_params[P], d_out[7 P]; the iteration is read
// from b->d_iter by the resample kernels.  The problems' resample and staging
// kernels, and after the sweep their finalisation, are spread over the side
// streams (problems are independent there); the sweep launches run on the
// batch's stream, which also ends the whole evaluation.
int enqueue(hawkes_batch* b, const hawkes_params* d_params, double* d_out, bool time_sweep) {
    const int model = static_cast<int>(b->flags & kModelBits);
    const bool bgt = (b->flags & HAWKES_BG_TIME) != 0;
    const int skip = (b->flags & HAWKES_SKIP_UNDERFLOW) ? 1 : 0;
    const int P = static_cast<int>(b->probs.size());
    HB_TRY(fork_side(b));
    for (int p = 0; p < P; ++p) {
        cudaStream_t st = b->aux[p % hawkes_batch::NAUX];
        hawkes_ctx* c = b->probs[p];
        int g = static_cast<int>((c->npad + 255) / 256);
        if (g > 8 * b->sms) g = 8 * b->sms;
        if (b->resample)
            k_resample<<<g, 256, 0, st>>>(c->county, c->n, c->tri_xy, c->tri_cum, c->cfirst, c->clast,
                                          b->seeds[p], b->streams[p], 0, b->d_iter, c->x, c->y);
        k_prep<<<g, 256, 0, st>>>(c->t, c->x, c->y, c->s, c->tb, d_params + p, model, 1, skip,
                                  c->n, c->npad, c->rec, c->acc, c->cc, c->ctr, c->fix7);
    }
    HB_TRY(join_side(b));
    cudaStream_t st = b->stream;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Rec* recs[KMAX] = {nullptr, nullptr, nullptr, nullptr};
        for (int k = 0; k < b->kc; ++k) recs[k] = b->probs[b->groups[gi][k]]->rec;
        HB_CUDA(launch_group_stage(st, b->sms, b->h_groups[gi], recs, b->probs[b->groups[gi][0]]->t,
                                   b->kc, b->d_gtiles + b->gtile_off[gi]));
    }
    HB_CUDA(cudaMemsetAsync(b->d_ctr + CT_WORK, 0, sizeof(int), st));
    HB_CUDA(cudaMemsetAsync(b->d_ctr + CT_COUNT + CT_WORK, 0, sizeof(int), st));
    if (time_sweep) HB_CUDA(cudaEventRecord(b->ev[0], st));
    if (b->ngitems > 0)
        HB_CUDA(launch_sweep_group(st, b->kc, b->ggrid, b->d_groups,
                                   static_cast<int>(b->h_groups.size()), b->d_gitems, b->ngitems,
                                   b->d_ctr + CT_COUNT));
    HB_CUDA(launch_sweep_batch(st, b->variant, b->grid, b->d_probs, static_cast<int>(P), b->d_items,
                               b->nitems, b->d_ctr, bgt,
                               (b->flags & HAWKES_LOGLIK_ONLY) != 0));
    if (time_sweep) HB_CUDA(cudaEventRecord(b->ev[1], st));
    HB_TRY(fork_side(b));
    for (int p = 0; p < P; ++p) {
        cudaStream_t st = b->aux[p % hawkes_batch::NAUX];
        hawkes_ctx* c = b->probs[p];
        k_finalize<<<c->final_blocks, 256, 0, st>>>(c->acc, c->t, c->lo, c->hi, c->cc, c->n,
                                                    c->npad, 0, c->n, 1, c->fixlist, c->ctr,
                                                    c->partials, nullptr);
        k_rows64<<<b->sms, 256, 0, st>>>(c->t, c->x, c->y, c->s, c->lo, c->hi, c->cc, model, c->n,
                                         c->npad, 0, 0, 1, c->fixlist, c->ctr, c->acc, c->fix7,
                                         nullptr);
        k_reduce<<<1, 256, 0, st>>>(c->partials, c->final_blocks, c->fix7, c->cc, c->n,
                                    d_out + 7 * p, c->ctr);
        int gf = static_cast<int>((c->n + 255) / 256);
        if (gf > 2 * b->sms) gf = 2 * b->sms;
        k_flushfix<<<gf, 256, 0, st>>>(c->acc, c->t, c->x, c->y, c->s, c->lo, c->hi, c->cc, model,
                                       c->n, c->npad, 0, c->n, c->ctr, c->fix7, d_out + 7 * p,
                                       nullptr);
    }
    HB_CUDA(cudaGetLastError());
    return join_side(b);
}

int latched_errors(hawkes_batch* b) {
    int err = 0, gerr = 0;
    HB_CUDA(cudaMemcpyAsync(&err, b->d_ctr + CT_ERR, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    HB_CUDA(cudaMemcpyAsync(&gerr, b->d_ctr + CT_COUNT + CT_ERR, sizeof(int), cudaMemcpyDeviceToHost,
                            b->stream));
    HB_CUDA(cudaStreamSynchronize(b->stream));
    if (gerr != 0) {
        HB_CUDA(cudaMemsetAsync(b->d_ctr + CT_COUNT + CT_ERR, 0, sizeof(int), b->stream));
        if (err == 0) err = gerr;
    }
    for (auto* c : b->probs) {
        int e = 0;
        HB_CUDA(cudaMemcpyAsync(&e, c->ctr + CT_ERR, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        HB_CUDA(cudaStreamSynchronize(b->stream));
        if (e != 0) {
            HB_CUDA(cudaMemsetAsync(c->ctr + CT_ERR, 0, sizeof(int), b->stream));
            if (err == 0) err = e;
        }
    }
    HB_CUDA(cudaStreamSynchronize(b->stream));
    if (err != 0) HB_CUDA(cudaMemsetAsync(b->d_ctr + CT_ERR, 0, sizeof(int), b->stream));
    return err;
}

}  // namespace

extern "C" {

int hawkes_batch_create(hawkes_batch** out, hawkes_ctx* const* problems, int32_t n_problems,
                        const uint64_t* seeds, const uint64_t* streams, uint32_t flags,
                        void* cuda_stream) {
    HK_NVTX("hawkes_batch_create");
    if (!out) return HAWKES_ERR_ARG;
    *out = nullptr;
    if (!problems || n_problems < 1 ||
        (flags & ~(kFlagsAll & ~static_cast<uint32_t>(HAWKES_F64 | HAWKES_SKIP_SPATIAL))) != 0 ||
        (seeds == nullptr) != (streams == nullptr))
        return HAWKES_ERR_ARG;
    const int dev = problems[0] ? problems[0]->device : -1;
    for (int32_t p = 0; p < n_problems; ++p) {
        const hawkes_ctx* c = problems[p];
        if (!c || c->device != dev) return HAWKES_ERR_ARG;
        if (c->n == 0 || (seeds && !c->counties_ok)) return HAWKES_ERR_STATE;
        for (int32_t q = 0; q < p; ++q)
            if (problems[q] == c) return HAWKES_ERR_ARG;  // one context appears once
    }
    DeviceGuard g(dev);
    hawkes_batch* b = new (std::nothrow) hawkes_batch();
    if (!b) return HAWKES_ERR_OOM;
    b->device = dev;
    b->flags = flags;
    b->probs.assign(problems, problems + n_problems);
    if (seeds) {
        b->seeds.assign(seeds, seeds + n_problems);
        b->streams.assign(streams, streams + n_problems);
        b->resample = true;
    }
    int rc = HAWKES_OK;
    do {
        if ((rc = st_of(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)))) break;
        if (cuda_stream) {
            b->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            if ((rc = st_of(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)))) break;
            b->own_stream = true;
        }
        if ((rc = st_of(cudaEventCreate(&b->ev[0]))) || (rc = st_of(cudaEventCreate(&b->ev[1])))) break;
        if ((rc = st_of(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming)))) break;
        for (int k = 0; k < hawkes_batch::NAUX && rc == HAWKES_OK; ++k) {
            rc = st_of(cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking));
            if (rc == HAWKES_OK) rc = st_of(cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming));
        }
        if (rc) break;
        if ((rc = st_of(cudaMalloc(&b->d_ctr, 2 * CT_COUNT * sizeof(int))))) break;
        if ((rc = st_of(cudaMalloc(&b->d_iter, sizeof(uint64_t))))) break;
        if ((rc = st_of(cudaMemsetAsync(b->d_ctr, 0, 2 * CT_COUNT * sizeof(int), b->stream)))) break;
        if ((rc = st_of(group_setup_attributes()))) break;
        if ((rc = st_of(cudaMemsetAsync(b->d_iter, 0, sizeof(uint64_t), b->stream)))) break;
        std::vector<ProbDesc> descs;
        for (auto* c : b->probs)
            descs.push_back(ProbDesc{c->t, c->rec, c->lo, c->hi, c->tb, c->cc, c->acc, c->n, c->npad});
        if ((rc = st_of(cudaMalloc(&b->d_probs, descs.size() * sizeof(ProbDesc))))) break;
        if ((rc = st_of(cudaMemcpyAsync(b->d_probs, descs.data(), descs.size() * sizeof(ProbDesc),
                                        cudaMemcpyHostToDevice, b->stream))))
            break;
        // the contexts' own queued work must finish before the batch touches their buffers
        for (auto* c : b->probs)
            if ((rc = st_of(cudaStreamSynchronize(c->stream)))) break;
        if (rc) break;
        if ((rc = time_classes(b))) break;
        rc = build_items(b, 0, CHUNK, 1);
    } while (0);
    if (rc != HAWKES_OK) {
        hawkes_batch_destroy(b);
        return rc;
    }
    *out = b;
    return HAWKES_OK;
}

void hawkes_batch_destroy(hawkes_batch* b) {
    HK_NVTX("hawkes_batch_destroy");
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_gitems) cudaFree(b->d_gitems);
    if (b->d_gtiles) cudaFree(b->d_gtiles);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->d_iter) cudaFree(b->d_iter);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : b->aux)
        if (s) cudaStreamSynchronize(s);
    for (int k = 0; k < hawkes_batch::NAUX; ++k) {
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
        if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

int hawkes_batch_run(hawkes_batch* b, const hawkes_params* d_params, uint64_t iteration,
                     double* d_out) {
    HK_NVTX("hawkes_batch_run");
    if (!b || !d_params || !d_out || !aligned8(d_params) || !aligned8(d_out)) return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    k_set_u64<<<1, 32, 0, b->stream>>>(b->d_iter, iteration);
    HB_CUDA(cudaGetLastError());
    if (b->exec && b->g_params == d_params && b->g_out == d_out)
        return st_of(cudaGraphLaunch(b->exec, b->stream));
    return enqueue(b, d_params, d_out, false);
}

int hawkes_batch_capture(hawkes_batch* b, const hawkes_params* d_params, double* d_out) {
    HK_NVTX("hawkes_batch_capture");
    if (!b || !d_params || !d_out || !aligned8(d_params) || !aligned8(d_out)) return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    HB_CUDA(cudaStreamSynchronize(b->stream));
    drop_graph(b);
    HB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue(b, d_params, d_out, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc != HAWKES_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != HAWKES_OK ? rc : HAWKES_ERR_CUDA;
    }
    b->graph = graph;
    if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(b);
        return HAWKES_ERR_CUDA;
    }
    b->g_params = d_params;
    b->g_out = d_out;
    return HAWKES_OK;
}

int hawkes_batch_wait(hawkes_batch* b) {
    HK_NVTX("hawkes_batch_wait");
    if (!b) return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    HB_CUDA(cudaStreamSynchronize(b->stream));
    return latched_errors(b);
}

int hawkes_batch_tune(hawkes_batch* b, const hawkes_params* d_params, double* d_out, int reps,
                      int* variant, int* chunk, int* order, double* best_ms) {
    HK_NVTX("hawkes_batch_tune");
    if (!b || !d_params || !d_out || !aligned8(d_params) || !aligned8(d_out) || reps < 1)
        return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    static const int kChunks[] = {16, 32, 64};
    int bv = -1, bc = 0, bo = 0, bk = 1;
    double bms = 0.0;
    auto time_one = [&](int v, int ch, int o, double* t) -> int {
        HB_TRY(build_items(b, v, ch, o));
        HB_TRY(enqueue(b, d_params, d_out, false));  // warm-up
        double tot = 0.0;
        for (int r = 0; r < reps; ++r) {
            HB_TRY(enqueue(b, d_params, d_out, true));
            HB_CUDA(cudaEventSynchronize(b->ev[1]));
            float ms = 0.f;
            HB_CUDA(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
            tot += ms;
        }
        *t = tot / reps;
        return HAWKES_OK;
    };
    // one problem per CTA: sweep variant x item order x chunk length
    b->kc = 1;
    for (int v = 0; v < sweep_num_variants(); ++v) {
        for (int o = 0; o < 2; ++o) {
            for (int ch : kChunks) {
                double t = 0.0;
                HB_TRY(time_one(v, ch, o, &t));
                if (bv < 0 || t < bms) {
                    bv = v;
                    bc = ch;
                    bo = o;
                    bms = t;
                }
            }
        }
    }
    // several chains per CTA (where chains share their event times): chains
    // per CTA x chunk length, the other problems as found above
    if (group_flags_ok(b->flags)) {
        for (int kc : {2, 4}) {
            if (!group_kc_supported(kc) || largest_class(b) < static_cast<size_t>(kc)) continue;
            b->kc = kc;
            for (int ch : kChunks) {
                double t = 0.0;
                HB_TRY(time_one(bv, ch, bo, &t));
                if (t < bms) {
                    bk = kc;
                    bc = ch;
                    bms = t;
                }
            }
        }
    }
    b->kc = bk;
    HB_TRY(build_items(b, bv, bc, bo));
    HB_CUDA(cudaStreamSynchronize(b->stream));
    if (variant) *variant = bv;
    if (chunk) *chunk = bc;
    if (order) *order = bo;
    if (best_ms) *best_ms = bms;
    return latched_errors(b);
}

int hawkes_batch_set_chains_per_cta(hawkes_batch* b, int chains_per_cta) {
    HK_NVTX("hawkes_batch_set_chains_per_cta");
    if (!b) return HAWKES_ERR_ARG;
    if (chains_per_cta != 1 &&
        (!group_kc_supported(chains_per_cta) || !group_flags_ok(b->flags)))
        return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    HB_CUDA(cudaStreamSynchronize(b->stream));
    const int prev = b->kc;
    b->kc = chains_per_cta;
    const int rc = build_items(b, b->variant, b->chunk, b->order);
    if (rc != HAWKES_OK) {  // e.g. no memory for the group tiles: keep the previous setting
        b->kc = prev;
        (void)build_items(b, b->variant, b->chunk, b->order);
    }
    return rc;
}

int hawkes_batch_get_config(const hawkes_batch* b, int* variant, int* chunk, int* order,
                            int* chains_per_cta, int* n_groups) {
    if (!b) return HAWKES_ERR_ARG;
    if (variant) *variant = b->variant;
    if (chunk) *chunk = b->chunk;
    if (order) *order = b->order;
    if (chains_per_cta) *chains_per_cta = b->kc;
    if (n_groups) *n_groups = static_cast<int>(b->groups.size());
    return HAWKES_OK;
}

int hawkes_batch_set_config(hawkes_batch* b, int variant, int chunk, int order) {
    HK_NVTX("hawkes_batch_set_config");
    if (!b || variant < 0 || variant >= sweep_num_variants() || chunk < 1 || order < 0 ||
        order > 1)
        return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    HB_CUDA(cudaStreamSynchronize(b->stream));
    return build_items(b, variant, chunk, order);
}

}  // extern "C"

int hawkes_batch_tune_cached(hawkes_batch* b, const hawkes_params* d_params, double* d_out,
                             int reps, const char* cache_path, int* variant, int* chunk,
                             int* order, int* from_cache) {
    HK_NVTX("hawkes_batch_tune_cached");
    if (!b || !d_params || !d_out || !aligned8(d_params) || !aligned8(d_out) || reps < 1 ||
        !cache_path)
        return HAWKES_ERR_ARG;
    DeviceGuard g(b->device);
    const std::string dk = device_key();
    if (dk.empty()) return HAWKES_ERR_CUDA;
    double pairs = 0.0;
    for (const hawkes_ctx* c : b->probs) pairs += 0.5 * static_cast<double>(c->n) * (c->n - 1);
    const std::string key = dk + "batch|P=" + std::to_string(b->probs.size()) + "|pairs<=2^" +
                            std::to_string(log2_ceil(pairs > 1.0 ? pairs : 1.0)) +
                            "|flags=" + std::to_string(b->flags);
    int v = -1, ch = 0, o = 0, kc = 1;
    if (tune_cache_get(cache_path, key.c_str(), &v, &ch, &o, nullptr, &kc) == 1 && ch >= 1 &&
        o <= 1 && (kc == 1 || (group_kc_supported(kc) && group_flags_ok(b->flags)))) {
        b->kc = kc;
        HB_TRY(hawkes_batch_set_config(b, v, ch, o));
        if (variant) *variant = v;
        if (chunk) *chunk = ch;
        if (order) *order = o;
        if (from_cache) *from_cache = 1;
        return HAWKES_OK;
    }
    double ms = 0.0;
    HB_TRY(hawkes_batch_tune(b, d_params, d_out, reps, &v, &ch, &o, &ms));
    if (variant) *variant = v;
    if (chunk) *chunk = ch;
    if (order) *order = o;
    if (from_cache) *from_cache = 0;
    return tune_cache_put(cache_path, key.c_str(), v, ch, o, ms, b->kc);
}
