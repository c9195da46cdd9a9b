// Explicit instantiation of the persistent batched kernels for the StF32
// population format (compiled with global loads in the L2-coherent
// cache-global mode, see lbm_batch_kernels.cuh).
#include "lbm_batch_kernels.cuh"

template struct lbm::BatchLaunch<lbm::StF32>;
