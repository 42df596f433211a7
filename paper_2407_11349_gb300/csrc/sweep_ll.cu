// Pair-sweep kernels that form the log-likelihood only (HAWKES_LOGLIK_ONLY,
// space-time background), instantiated in a unit of their own so they compile
// in parallel with the other kernel families.
#include "sweep_kernel.cuh"

namespace hk {

static const Variant kVariantsLl[] = HK_SWEEP_VARIANTS(false, true);
static_assert(sizeof(kVariantsLl) / sizeof(kVariantsLl[0]) == kNumVariants, "variant count");

const Variant* sweep_variants_ll() { return kVariantsLl; }

}  // namespace hk
