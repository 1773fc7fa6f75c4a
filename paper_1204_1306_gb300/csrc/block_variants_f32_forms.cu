// Explicit instantiations of the block-solver variants (FP32 inner
// iterations, out-of-line / branch-free hops and BiCGStab), compiled
// as their own translation unit so that the variants build in parallel.
#include "block_solve.cuh"

namespace psms {
PSMS_BLOCK_VARIANTS_FORMS(PSMS_BLOCK_INSTANTIATE, Store<float>)
PSMS_BLOCK_VARIANTS_SMEM(PSMS_BLOCK_INSTANTIATE, Store<float>)
}  // namespace psms
