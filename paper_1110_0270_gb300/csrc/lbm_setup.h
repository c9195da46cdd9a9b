// Configuration checks and the layout-independent part of the kernel
// parameters, shared by every entry point that turns an lbm_config into a
// Params block (lbm_create, the allocation-free step).  Defined in
// lbm_abi.cu.
#pragma once

#include "lbm.h"
#include "lbm_params.h"

namespace lbm {

// nullptr when cfg is a valid configuration, else the reason.
const char* check_config(const lbm_config* cfg);

// beta of cfg: cfg->beta, or 1 / (6 nu + 1) when cfg->beta <= 0 (the reading
// nu = c_s^2 (1/beta - 1) / 2 of Section 2 with c_s^2 = 1/3).
double config_beta(const lbm_config* cfg);

// Every Params field that does not depend on where the populations and the
// scratch live: sizes, boundary flags, collision constants (and their FP32
// copies), the median filter's window source and the CTA count of the
// grid-stride kernels (nsm = SMs of the device).  The storage pointers,
// pitch and plane sizes are left to the caller.
void fill_params(const lbm_config* cfg, int nsm, Params& p);

}  // namespace lbm
