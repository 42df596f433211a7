// Pair-sweep kernels for the time-only background of eq. 2 (HAWKES_BG_TIME),
// instantiated in a unit of their own so they compile in parallel with the
// default kernels in sweep.cu.
#include "sweep_kernel.cuh"

namespace hk {

static const Variant kVariantsBgt[] = HK_SWEEP_VARIANTS(true, false);
static_assert(sizeof(kVariantsBgt) / sizeof(kVariantsBgt[0]) == kNumVariants, "variant count");

const Variant* sweep_variants_bgt() { return kVariantsBgt; }

}  // namespace hk
