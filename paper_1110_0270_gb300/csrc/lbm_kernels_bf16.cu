// Explicit instantiation of the step, fix-up and state kernels for the
// StBF16 population format (one translation unit per format so that the
// build compiles them in parallel).
#include "lbm_kernels.cuh"

template struct lbm::Launch<lbm::StBF16>;
