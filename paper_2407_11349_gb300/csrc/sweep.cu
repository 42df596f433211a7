// Host side of the FP32 pair sweep (kernels in sweep_kernel.cuh): kernel
// variants, their work lists, and launch.  This unit instantiates the
// space-time background's kernels; sweep_bgt.cu the time-only background's
// and sweep_ll.cu the log-likelihood-only ones.
#include <algorithm>
#include <vector>

#include "sweep_kernel.cuh"

namespace hk {

static const Variant kVariants[] = HK_SWEEP_VARIANTS(false, false);
static_assert(sizeof(kVariants) / sizeof(kVariants[0]) == kNumVariants, "variant count");

// The kernel family of a call: the time-only background keeps its own kernels
// (with the log-likelihood-only flag it forms every moment and the gradient is
// dropped at finalisation).
static const Variant& variant_of(int v, bool bgt, bool ll) {
    return bgt ? sweep_variants_bgt()[v] : ll ? sweep_variants_ll()[v] : kVariants[v];
}

int sweep_num_variants() { return kNumVariants; }
int sweep_variant_rows(int v) { return kVariants[v].tr; }

cudaError_t sweep_setup_attributes() {
    for (int k = 0; k < 3 * kNumVariants; ++k) {
        const int fam = k / kNumVariants;
        const Variant& v = variant_of(k % kNumVariants, fam == 1, fam == 2);
        for (SweepFn f : {v.win, v.sym, v.batch}) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(v.smem));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int sweep_blocks_per_sm(int v) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kVariants[v].sym, THREADS,
                                                      kVariants[v].smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

// Symmetric work list over problems of sizes ns[] for variant v: items
// (row tile, column tiles [jb, je), problem) in chunks of `chunk` column
// tiles.  order 0: all items longest first (ties: later row tiles first);
// order 1: problem by problem, largest problem first, each problem's items
// longest first, so that the source tiles and accumulators of the problems
// in flight stay in L2 while the tail still ends on the smallest items.
std::vector<int4> sweep_items_batch(const std::vector<int64_t>& ns, int v, int chunk, int order) {
    const int tr = kVariants[v].tr;
    auto longest_first = [](const int4& a, const int4& b) {
        return (a.z - a.y) > (b.z - b.y) || ((a.z - a.y) == (b.z - b.y) && a.x > b.x);
    };
    std::vector<size_t> pidx(ns.size());
    for (size_t p = 0; p < ns.size(); ++p) pidx[p] = p;
    if (order == 1)
        std::stable_sort(pidx.begin(), pidx.end(), [&](size_t a, size_t b) { return ns[a] > ns[b]; });
    std::vector<int4> items;
    for (size_t p : pidx) {
        const int64_t n = ns[p];
        const int64_t nI = (n + tr - 1) / tr;
        const size_t first = items.size();
        for (int64_t I = 0; I < nI; ++I) {
            const int nJ = static_cast<int>((std::min<int64_t>((I + 1) * tr, n) + TC - 1) / TC);
            for (int jb = 0; jb < nJ; jb += chunk)
                items.push_back(make_int4(static_cast<int>(I), jb, std::min(jb + chunk, nJ),
                                          static_cast<int>(p)));
        }
        if (order == 1) std::stable_sort(items.begin() + first, items.end(), longest_first);
    }
    if (order == 0) std::stable_sort(items.begin(), items.end(), longest_first);
    return items;
}

std::vector<int4> sweep_items(int64_t n, int v) { return sweep_items_batch({n}, v, CHUNK, 0); }

static ProbDesc desc_of(const hawkes_ctx* c) {
    return ProbDesc{c->t, c->rec, c->lo, c->hi, c->tb, c->cc, c->acc, c->n, c->npad};
}

// Symmetric sweep of one problem over the work list items[0, nitems) (the
// whole list, or one shard's part of it).
cudaError_t launch_sweep_list(hawkes_ctx* c, const int4* items, int nitems, bool bgt, bool ll) {
    const Variant& v = variant_of(c->variant, bgt, ll);
    const int grid_cap = c->sms * c->variant_bpsm;
    const int grid = nitems < grid_cap ? nitems : grid_cap;
    if (grid <= 0) return cudaSuccess;
    v.sym<<<grid, THREADS, v.smem, c->stream>>>(desc_of(c), nullptr, items, nitems, c->ctr, 0,
                                                c->n, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_sweep(hawkes_ctx* c, bool sym, int64_t row_begin, int64_t row_end, bool bgt,
                         bool ll) {
    const Variant& v = variant_of(c->variant, bgt, ll);
    const int grid_cap = c->sms * c->variant_bpsm;
    const ProbDesc one = desc_of(c);
    if (sym) {
        return launch_sweep_list(c, c->items, c->nitems, bgt, ll);
    } else {
        const int item0 = static_cast<int>(row_begin / v.tr);
        const int nrt = static_cast<int>((row_end + v.tr - 1) / v.tr) - item0;
        const int ncol = static_cast<int>((c->n + TC - 1) / TC);
        const int nch = (ncol + CHUNK - 1) / CHUNK;
        const int nitems = nrt * nch;
        const int grid = nitems < grid_cap ? nitems : grid_cap;
        if (grid <= 0) return cudaSuccess;
        v.win<<<grid, THREADS, v.smem, c->stream>>>(one, nullptr, nullptr, nitems, c->ctr, row_begin,
                                                    row_end, item0, nch);
    }
    return cudaGetLastError();
}

// One persistent launch over the items of many problems; ctr[CT_WORK] must be
// zero when it starts.
cudaError_t launch_sweep_batch(cudaStream_t st, int variant, int grid, const ProbDesc* probs,
                               int nprobs, const int4* items, int nitems, int* ctr, bool bgt,
                               bool ll) {
    const Variant& v = variant_of(variant, bgt, ll);
    if (grid > nitems) grid = nitems;
    if (grid <= 0) return cudaSuccess;
    ProbDesc none{};
    v.batch<<<grid, THREADS, v.smem, st>>>(none, probs, items, nitems, ctr, 0, 0, 0, nprobs);
    return cudaGetLastError();
}

}  // namespace hk
