// Launch parameters shared by the host ABI and the kernels (plain data).
#pragma once

#include <stdint.h>

#include "lbm.h"

namespace lbm {

// MRT rates divided by the squared row norms of M1 (Section 5):
// e: s_e/36, eps: s_eps/36, q: s_q/12, nu: s_nu/4 with s_nu = 2 beta.
struct MrtRates {
    double e, eps, q, nu;
};
struct MrtRatesF {
    float e, eps, q, nu;
};

// Device counters (one 256-byte block of scratch, zeroed at create).
enum Counter {
    CNT_CAND0 = 0,     // candidate count, step parity 0
    CNT_CAND1 = 1,     // candidate count, step parity 1
    CNT_DIVERGED = 2,  // set to 1 on a non-finite / non-positive density
    CNT_OVERFLOW = 3,  // candidate list overflow
    CNT_NSEL = 4,      // number of sites selected in the last Ehrenfest step
    CNT_NVALID = 5,    // candidates (FP64 Delta S > delta) of the current step
    CNT_DONE = 6,      // CTAs of ehrenfest_eval_select that have finished
    CNT_PROBE = 7,     // samples written by the control-point probe
    CNT_WORDS = 8
};
constexpr int kRedSlots = 1024;  // partial-sum slots (spread the atomics)

enum Stat {
    ST_LIMITED = 0,
    ST_ELBM_SOLVED = 1,
    ST_ELBM_SKIPPED = 2,
    ST_ELBM_FALLBACK = 3,
    ST_ELBM_ITERS = 4,
    ST_ELBM_ITERS_MAX = 5,
    ST_WORDS = 16
};

struct Params {
    void* f;          // population storage base (pitched SoA)
    int64_t plane;    // elements per population plane (ny * pitch)
    int plane32;      // the same as int (Q * plane < 2^31 is enforced)
    int pitch, nx, ny;
    int periodic_x, periodic_y;
    int eq;           // equilibrium kind (LBM_EQ_*)
    double lid_u;     // top wall velocity along +x
    double beta;
    float beta_f, lid_u_f, delta_f;  // FP32 copies (no FP64 conversions per site)
    int topk;
    double delta;
    MrtRates mrt;
    MrtRatesF mrt_f;
    double elbm_eps;
    int elbm_max_iter, elbm_norm, elbm_fallback;
    double elbm_skip_rel;  // near-equilibrium skip: Delta S < 1e-15 + elbm_skip_rel * rho
    // Sections 4.2-4.4 limiters
    double lim_alpha, lim_k, lim_dst, lim_delta0;
    double* red;      // kRedSlots partial sums (+ kRedSlots counts), zero between steps
    double* lim_E;    // the step's E(Delta S) (ensemble limiter)
    float* lim_E_f;   // the same in FP32 (read by the 16/32-bit step kernels)
    float lim_f[4];   // FP32 copies: alpha, k, 1 / Delta S_t, -1 / (2 k)
    int pipe_ctas;    // host side: CTAs of the grid-stride reduction kernels
    double* probe_buf;  // control-point probe: (u_x, u_y) per step, ring of probe_cap
    int probe_site, probe_cap;
    int diffusive;    // Section 8's diffusive Maxwell walls on the edge sites
    double wall_u;    // their top-wall velocity (lid_u; the streaming adds no lid term)
    // scratch
    unsigned* counters;              // CNT_WORDS words
    unsigned long long* stats;       // ST_WORDS words
    int cand_cap;                    // capacity of the candidate list
    void* cand_f;                    // [Q][cand_cap] arithmetic type
    double* cand_ds;                 // [cand_cap] FP64 Delta S (-1: not a candidate)
    int* cand_site;                  // [cand_cap] y * nx + x
    int* cand_sel;                   // [cand_cap] selected flag (Ehrenfest/median)
    void* ds_field;                  // [ny][nx] arithmetic type (median only)
    double median_inv;               // median filter: 1 / (1 - 2 beta) when the
                                     // window's Delta S is taken from the
                                     // post-collision state (no field); 0: field
    double* scratch_d;               // small FP64 reduction scratch
    int cslot;                       // candidate counter used by this step (t & 1)
    int pdl;                         // host side: launch the step kernels with
                                     // programmatic dependent launch
};

}  // namespace lbm
