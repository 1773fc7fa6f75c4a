// Explicit instantiations of the block-solver variants (FP32 inner
// iterations, CGNR with inlined hops), compiled
// as their own translation unit so that the variants build in parallel.
#include "block_solve.cuh"

namespace psms {
PSMS_BLOCK_VARIANTS_CG(PSMS_BLOCK_INSTANTIATE, Store<float>)
}  // namespace psms
