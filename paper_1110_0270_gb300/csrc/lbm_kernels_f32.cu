// Explicit instantiation of the step, fix-up, state and batched kernels for the
// StF32 population format (one translation unit per format so that the
// build compiles them in parallel).
#include "lbm_batch_kernels.cuh"

template struct lbm::Launch<lbm::StF32>;
template struct lbm::BatchLaunch<lbm::StF32>;
