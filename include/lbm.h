/*
 * lbm.h - C ABI of the GB300 (sm_103a) lattice Boltzmann stream-and-collide
 * library with the add-ons of Brownlee, Levesley, Packwood and Gorban,
 * "Add-ons for Lattice Boltzmann Methods: Regularization, Filtering and
 * Limiters" (arXiv:1110.0270).
 *
 * What one step computes (Section 2, collide then stream): at every site the
 * moments {rho, rho u} = sum_i {1, v_i} f_i, an equilibrium f*, the selected
 * collision F(f), then free flight f_i(x + v_i, t + 1) = F_i(x, t) with
 * half-way bounce-back at walls (Section 8) and the moving-wall term
 * -6 W_i rho_w (v_i . u_wall), rho_w = 1, on links that cross a moving lid.
 *
 * Lattices and numbering:
 *   D1Q3 (Section 6): i = 0, 1, 2  <->  v = -1, 0, +1.
 *   D2Q9 (Section 5's numbering 1..9 shifted to 0..8):
 *     0 rest, 1 E, 2 SE, 3 S, 4 SW, 5 W, 6 NW, 7 N, 8 NE  (y grows north;
 *     the moving lid is the top row y = ny - 1, moving along +x).
 *
 * Collisions (lbm_config.collision):
 *   LBM_LBGK        F = f + 2 beta (f* - f)                  (Eq. CollisionIntegral)
 *   LBM_ELBM        F = f + alpha beta (f* - f), alpha the non-trivial root of
 *                   S(f + alpha (f* - f)) = S(f), entropic f*; parabola root
 *                   finder in FP64 (Section 3.3, Eqs. NewCondition,
 *                   Stopping, ConvergenceTwo)
 *   LBM_EHRENFEST   LBGK, except that among the sites with Delta S > delta the
 *                   k (= topk) largest jump to f* (Section 4, Ehrenfests'
 *                   regularisation); Delta S = sum f ln(f/f*) (Eq. DelS)
 *   LBM_POSITIVITY  LBGK followed by the positivity rule (Section 4, Eq. StrLine)
 *   LBM_MEDIAN      LBGK after the median entropy filter (Section 4.4): where
 *                   Delta S > delta and the median of Delta S over the site and
 *                   its neighbours is smaller, f -> f* + sqrt(med/DeltaS)(f - f*)
 *   LBM_MRT         F = f + M1^-1 C1 M1 (f* - f) (Section 5), C1 = diag(1, s_e,
 *                   s_eps, 1, s_q, 1, s_q, s_nu, s_nu), s_nu = 2 beta
 *
 * Memory and ownership.  The caller provides ONE device allocation of at
 * least lbm_required_bytes() bytes (for example a torch uint8 tensor) to
 * lbm_create(); the library carves the population array and its scratch out
 * of it and never allocates device memory itself.  The allocation must stay
 * alive until lbm_destroy().  The population array is structure-of-arrays,
 * f[i][y][pitch], with pitch = nx rounded up to 32 elements, updated in place
 * with the A-A pattern (every step reads and writes each population once).
 *
 * Streams.  Every call that takes `stream` (a cudaStream_t, NULL = legacy
 * default stream) enqueues its work there and returns without waiting,
 * except where a host output is documented to synchronise that stream.
 *
 * Errors.  Every call returns an lbm_status; no C++ exception crosses the
 * ABI.  On failure lbm_last_error(ctx) describes the cause.  A context whose
 * kernel launch failed with a CUDA error keeps returning LBM_ERR_CUDA.
 *
 * Thread safety.  A context is not thread safe; distinct contexts are
 * independent.  Steps on the same context must not overlap on the GPU.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument or configuration */
    LBM_ERR_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
    LBM_ERR_OOM = 3,      /* the caller's allocation is smaller than required */
    LBM_ERR_DIVERGED = 4, /* a non-finite or non-positive density was seen */
    LBM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
    LBM_ERR_STATE = 6     /* call not valid in the context's current state */
} lbm_status;

enum { LBM_D1Q3 = 1, LBM_D2Q9 = 2 };
enum { LBM_LBGK = 0, LBM_ELBM = 1, LBM_EHRENFEST = 2, LBM_POSITIVITY = 3,
       LBM_MEDIAN = 4, LBM_MRT = 5,
       /* Limiters of Sections 4.2-4.4: the state moves to
        * f* + phi(Delta S) (f - f*) before the LBGK collision. */
       LBM_SMOOTH = 6,           /* phi = 1 / (1 + alpha Delta S^k), Eq. (smoothReg) */
       LBM_DOUBLE_MONOTONIC = 7, /* phi = (1 + (Delta S / Delta S_t)^k)^(-1/(2k)),
                                    Eq. (DoublMonSpec) */
       LBM_ENSEMBLE = 8,         /* Eq. (phiExamp) with E(Delta S) the mean of
                                    the step's finite Delta S over the lattice */
       LBM_THRESHOLD = 9,        /* homothety sqrt(Delta S_t / Delta S) where
                                    Delta S >= Delta S_t = max(Delta S_0, delta),
                                    Delta S_0 from Eq. (EntThresh) on the step's
                                    Delta S distribution, Eq. (entrHom) */
       /* Section 5's "aggressive" MRT A_2 = M_2^-1 C_2 M_2 (D2Q9 only):
        * every moment but the two shear moments relaxes to equilibrium,
        * those at s_nu = 2 beta */
       LBM_MRT2 = 10,            /* F = f - A_2 (f - f*) at every site */
       LBM_MRT_LIMITER = 11,     /* LBGK; the Ehrenfest selection (topk, delta)
                                    gets A_2 instead of f* */
       LBM_ENSEMBLE_LAGGED = 12 }; /* LBM_ENSEMBLE with E(Delta S) the mean over
                                    the previous step's pre-collision state
                                    (accumulated by that step; the first step
                                    after lbm_init / lbm_set_state uses its
                                    own, computed there): no pass over the
                                    state before each step */
/* Equilibria: product of the 1D polynomial equilibria of Section 6 (the
 * paper's D2Q9 choice, Section 8), product of the 1D entropic equilibria
 * (always used by ELBM), or the textbook W_i rho (1 + 3cu + 9/2 (cu)^2 - 3/2 u^2). */
enum { LBM_EQ_POLY_PRODUCT = 0, LBM_EQ_ENTROPIC = 1, LBM_EQ_POLY_STD = 2 };
/* Storage of the populations.  FP64 and FP32 store f; BF16_DEV and FP16_DEV
 * store the deviation f_i - W_i rounded to nearest even, with FP32 math. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_BF16_DEV = 2, LBM_FP16_DEV = 3 };
/* Boundaries: CAVITY = walls on all four sides, the top one moving with
 * lid_u (half-way bounce-back, every site fluid); ENDS = D1Q3 tube closed at
 * both ends; PERIODIC = both directions wrap; CHANNEL = periodic in x, walls
 * at bottom and top (top moving); DIFFUSIVE = Section 8's diffusive Maxwell
 * walls (D2Q9, nx, ny >= 3): the edge sites are wall sites, not collided;
 * at the start of each step a wall site's populations pointing into the
 * fluid become gamma f*_i(u_wall) (f* at unit density, u_wall = (lid_u, 0)
 * on the top wall, 0 elsewhere; gamma returns the mass that arrived), and a
 * corner takes bounce-back for the populations from outside; limiters and
 * median windows see the fluid sites only. */
enum { LBM_BC_CAVITY = 0, LBM_BC_ENDS = 1, LBM_BC_PERIODIC = 2, LBM_BC_CHANNEL = 3, LBM_BC_DIFFUSIVE = 4 };
enum { LBM_NORM_ENTROPIC = 0, LBM_NORM_L1 = 1 };
enum { LBM_FALLBACK_POSITIVITY = 0, LBM_FALLBACK_EHRENFEST = 1 };
/* Element types of caller buffers exchanged with the library. */
enum { LBM_DTYPE_F64 = 0, LBM_DTYPE_F32 = 1 };

typedef struct {
    int lattice;     /* LBM_D1Q3 | LBM_D2Q9 */
    int nx, ny;      /* sites; ny = 1 for D1Q3.  nx, ny >= 1 */
    int collision;   /* LBM_LBGK ... LBM_ENSEMBLE_LAGGED */
    int equilibrium; /* LBM_EQ_*; ignored by LBM_ELBM (always entropic) */
    int precision;   /* LBM_FP64 | LBM_FP32 | LBM_BF16_DEV | LBM_FP16_DEV */
    int bc;          /* LBM_BC_* */
    double beta;     /* over-relaxation coefficient in (0, 1]; if <= 0 it is
                        set from nu as beta = 1 / (6 nu + 1), the reading
                        nu = c_s^2 (1/beta - 1) / 2 with c_s^2 = 1/3 */
    double nu;       /* kinematic viscosity, used only when beta <= 0 */
    double lid_u;    /* velocity of the top wall along +x (0: resting wall) */
    int topk;        /* Ehrenfest: at most this many sites per step (>= 0) */
    double delta;    /* Ehrenfest / median threshold on Delta S (>= 0) */
    double s_e, s_eps, s_q; /* MRT relaxation rates of C1 */
    double elbm_eps;        /* ELBM stopping tolerance (> 0), e.g. 1e-15 */
    int elbm_max_iter;      /* ELBM parabola iterations (>= 1), e.g. 20 */
    int elbm_norm;          /* LBM_NORM_* in the stopping rule */
    int elbm_fallback;      /* rule when no non-trivial root exists */
    /* Sections 4.2-4.4 limiters (appended in ABI version 2) */
    double lim_alpha;       /* alpha of Eqs. (smoothReg), (phiExamp); > 0 */
    double lim_k;           /* k of Eqs. (smoothReg), (phiExamp), (DoublMonSpec); > 0 */
    double lim_dst;         /* Delta S_t of Eq. (DoublMonSpec); > 0 */
    double lim_delta0;      /* delta_0 of Eqs. (LimEntLim), (EntThresh); >= 0 */
} lbm_config;

typedef struct {
    uint64_t steps;            /* steps taken since lbm_init/lbm_set_state */
    uint64_t candidates_last;  /* sites with Delta S > delta in the last step */
    uint64_t limited_total;    /* limiter corrections applied, cumulative
                                  (not counted for LBM_SMOOTH,
                                  LBM_DOUBLE_MONOTONIC, LBM_ENSEMBLE, which act
                                  on every site) */
    uint64_t elbm_solved;      /* ELBM sites that ran the root finder */
    uint64_t elbm_skipped;     /* ELBM sites with Delta S < 1e-15 */
    uint64_t elbm_fallbacks;   /* ELBM sites without a non-trivial root */
    uint64_t elbm_iters_total; /* parabola iterations, summed */
    uint64_t elbm_iters_max;   /* largest iteration count at one site */
    uint64_t diverged;         /* 1 once a non-finite or non-positive rho is seen */
    uint64_t overflow;         /* 1 if a candidate list overflowed (never with
                                  the default capacity of one entry per site) */
    uint64_t screened_last;    /* sites the FP32 screen passed to the FP64
                                  Delta S test in the last step (limiters) */
} lbm_stats;

/* Fills *cfg with defaults: D2Q9 16x16 cavity, LBGK, product polynomial
 * equilibrium, FP32, beta = 0.9, topk = 0, delta = 1e-3, MRT rates
 * (1.64, 1.54, 1.9), elbm_eps = 1e-15, elbm_max_iter = 20, lim_alpha = 1,
 * lim_k = 1, lim_dst = 1e-3, lim_delta0 = 0.01. */
lbm_status lbm_config_default(lbm_config* cfg);

/* MRT relaxation rates of the presets of Sections 5, 7 and 8, written into
 * cfg->s_e, s_eps, s_q with s_nu = 2 beta (beta = cfg->beta, or 1/(6 nu + 1)
 * when cfg->beta <= 0); the other fields are left as they are.  Use with
 * collision = LBM_MRT.
 *   LBM_MRT_PRESET_TRT   two relaxation times (Section 5): s_e = s_eps = s_nu,
 *                        s_q = 8 (2 - s_nu) / (8 - s_nu) (the printed
 *                        "8(2=s_nu)/(8-s_nu)" read with a minus sign)
 *   LBM_MRT_PRESET_MRT   s_e = 1.64, s_eps = 1.54, s_q as for TRT (Section 8)
 *   LBM_MRT_PRESET_MRT1  s_e = 1.64, s_eps = 1.54, s_q = 1.9 (Section 8)
 *   LBM_MRT_PRESET_LL    s_e = 1.64, s_eps = 1.54, s_q = 3 (2 - s_nu) / (3 - s_nu),
 *                        the A_1 rates of Section 7's shear-decay comparison
 * LBM_ERR_ARG for a NULL cfg, an unknown preset or beta outside (0, 1]. */
enum { LBM_MRT_PRESET_TRT = 0, LBM_MRT_PRESET_MRT = 1, LBM_MRT_PRESET_MRT1 = 2, LBM_MRT_PRESET_LL = 3 };
lbm_status lbm_mrt_preset(lbm_config* cfg, int preset);

/* Device bytes needed for cfg (populations + scratch).  Fails with
 * LBM_ERR_ARG for an invalid configuration. */
lbm_status lbm_required_bytes(const lbm_config* cfg, size_t* bytes);

/* Creates a context over the caller's device allocation dev_mem (256-byte
 * aligned, at least lbm_required_bytes) on the current CUDA device.  The
 * populations are undefined until lbm_init or lbm_set_state.  Clears the
 * scratch with a synchronous cudaMemset and captures the kernels of two
 * steps (one A-A period) into a CUDA graph that lbm_step replays, and of 64
 * steps into a second one for long runs (lbm_step uses it while at least 64
 * steps remain). */
lbm_status lbm_create(const lbm_config* cfg, void* dev_mem, size_t bytes, lbm_ctx** out);

/* Releases the host-side context (not the caller's device memory). */
void lbm_destroy(lbm_ctx* ctx);

/* f = f*(rho, u) at every site from HOST arrays rho, ux, uy of nx*ny
 * doubles, row-major [y][x] (uy may be NULL for D1Q3).  The equilibrium is
 * the configured one (entropic for ELBM), evaluated in the storage's
 * arithmetic type (FP64 for FP64 storage, FP32 otherwise) from the inputs
 * rounded to it.  Copies the inputs to device scratch first; synchronises
 * `stream` (the host arrays may be reused on return).  Resets the step
 * counter and statistics. */
lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    void* stream);

/* Same as lbm_init with DEVICE arrays (no synchronisation). */
lbm_status lbm_init_device(lbm_ctx* ctx, const double* rho, const double* ux,
                           const double* uy, void* stream);

/* Loads the pre-collision populations from a dense DEVICE array f[Q][ny][nx]
 * of dtype LBM_DTYPE_F64 or LBM_DTYPE_F32 (rounded to the storage format). */
lbm_status lbm_set_state(lbm_ctx* ctx, const void* f, int dtype, void* stream);

/* Writes the current pre-collision populations to a dense DEVICE array
 * f[Q][ny][nx] of the given dtype (undoing the A-A layout of odd steps). */
lbm_status lbm_get_state(lbm_ctx* ctx, void* f, int dtype, void* stream);

/* Advances nsteps >= 0 steps.  Allocates nothing.  Pairs of steps that start
 * at an even step count replay the context's graph (one launch instead of
 * two to four, which matters for small lattices); the rest, and every step
 * while kernel tracing is on, are launched one by one. */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps, void* stream);

/* Density rho[ny][nx] and velocity u[2][ny][nx] (u_x plane then u_y plane;
 * D1Q3 writes only u_x) of the current state into caller-owned DEVICE
 * buffers of the given dtype.  LBM_DTYPE_F64 outputs are formed in FP64;
 * LBM_DTYPE_F32 outputs of FP32 or 16-bit storage in FP32, with opposite
 * populations subtracted before the sum (exact while they lie within a
 * factor 2 of each other), so that rho u keeps its relative precision. */
lbm_status lbm_macros(lbm_ctx* ctx, void* rho, void* u, int dtype, void* stream);

/* H = sum_x sum_i f_i ln(f_i / W_i) (minus the perfect-mixture entropy of
 * Section 4, summed over the lattice) into *H_total_host (synchronises
 * `stream`), and optionally the FP64 Delta S field dS[ny][nx] (DEVICE,
 * may be NULL), Delta S computed against the configured equilibrium. */
lbm_status lbm_entropy(lbm_ctx* ctx, double* H_total_host, double* dS_dev, void* stream);

/* Enstrophy of Section 8 into *E_host (synchronises `stream`): the sum over
 * sites of the vorticity squared divided by the number of sites, with the
 * vorticity w = d u_y/dx - d u_x/dy of the site velocities by central
 * differences (wrapped in periodic directions, one-sided to the inside
 * neighbour at a wall edge).  D2Q9 only (LBM_ERR_ARG for D1Q3).  Uses the
 * context's scratch; the state is not modified. */
lbm_status lbm_enstrophy(lbm_ctx* ctx, double* E_host, void* stream);

/* Control-point probe (the signal of Section 8's Hopf-bifurcation study):
 * from the next lbm_step on, every step records the velocity (u_x, u_y) of
 * site (x, y) in the state it produced into the caller's DEVICE ring buffer
 * buf of 2*cap doubles (sample k at buf[2 (k mod cap)]), with one extra
 * one-thread launch per step; buf = NULL turns the probe off.  Re-captures
 * the step graph (synchronous).  lbm_probe_count returns into *count the
 * number of samples recorded since lbm_probe_set, lbm_init or lbm_set_state
 * (synchronises `stream`). */
lbm_status lbm_probe_set(lbm_ctx* ctx, int x, int y, double* buf, int cap);
lbm_status lbm_probe_count(lbm_ctx* ctx, uint64_t* count, void* stream);

/* Copies the step counters into *out (synchronises `stream`). */
lbm_status lbm_stats_get(lbm_ctx* ctx, lbm_stats* out, void* stream);

/* Limiter candidates of the most recent step (the collisions with a
 * candidate list: EHRENFEST, MEDIAN, THRESHOLD, MRT_LIMITER; LBM_ERR_STATE
 * otherwise), i.e. the sites whose FP64 Delta S exceeds delta: up to `cap`
 * entries of (Delta S, linear site index y*nx + x, selected flag) into HOST
 * arrays (any may be NULL); *count receives the number of candidates.  The
 * FP64 Delta S of the step's screened sites is evaluated on `stream` by one
 * small kernel (the step itself may have settled them in FP32), then the
 * call synchronises `stream`.  The candidate order is arbitrary.  Uses a host
 * buffer of one entry per screened site. */
lbm_status lbm_last_candidates(lbm_ctx* ctx, double* ds, int32_t* site, int32_t* selected,
                               int cap, int* count, void* stream);

/* ---- Batched form: many independent lattices in one context -------------
 * Instances: D2Q9 cavities, channels or periodic boxes and D1Q3 tubes (ends)
 * or rings, of any size, mixed in one batch; they share the precision of
 * cfgs[0]; size, lattice, boundary, collision (LBM_LBGK ... LBM_MRT), beta,
 * lid, limiter and MRT/ELBM parameters are per instance.
 *
 * Persistent launch: one kernel launch advances every instance of its group
 * several steps.  Its CTAs claim work items - (step, instance, tile) in step
 * order - from a device queue until the queue is drained; an item waits until
 * its instance has completed the previous step (a per-instance step
 * generation), so instances advance independently, without a barrier
 * between steps, and the CTA that completes an instance's step runs that
 * instance's limiter fix-up (Ehrenfest selection, median filter) before
 * publishing it.  Three kernels, on parallel stream branches: the streaming
 * collisions (LBGK, positivity, MRT), the limiters (Ehrenfest, median) and
 * ELBM (its FP64 root finder needs far more registers).
 * graph_steps steps of both are captured once, at creation, into a CUDA
 * graph that lbm_batch_step replays.  Every wait is bounded (wait_ms): one
 * that runs out stops the launch and the next status check returns
 * LBM_ERR_TIMEOUT (the states are then undefined until re-initialised).
 *
 * Memory: one caller device allocation of lbm_batch_required_bytes(_ex)
 * (populations, limiter scratch, descriptors, work queues and step
 * generations); nothing is allocated afterwards. */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* Launch shape and schedule of a batch (the autotuner's knobs). */
enum { LBM_BATCH_ORDER_INSTANCE = 0,     /* an instance's tiles one after another */
       LBM_BATCH_ORDER_INTERLEAVED = 1 }; /* tile j of every instance, then j + 1 */
typedef struct {
    int tile_x;       /* D2Q9 tile width in sites: 16, 32, 64, 128 or 256; the
                         tile is tile_x x (256 / tile_x) sites, one per thread
                         (D1Q3 tiles are 256 sites of the line) */
    int ctas_per_sm;  /* CTAs per SM of each kernel, 0 = as many as fit */
    int chunk;        /* work items claimed per queue access (1 ... 1024) */
    int order;        /* LBM_BATCH_ORDER_* within a step */
    int graph_steps;  /* steps per launch in the replayed graph (1 ... 4096) */
    double wait_ms;   /* limit of one wait for an instance's previous step */
    int tile_rows;    /* tiles per work item, stacked along y (D1Q3: along the
                         line), 1 ... 64 */
} lbm_batch_opts;
/* Defaults: tile 128 x 2, 4 tiles per item, as many CTAs as fit, chunk 4,
 * instance order, 16 steps per graph launch, 1000 ms waits. */
lbm_status lbm_batch_opts_default(lbm_batch_opts* opts);

lbm_status lbm_batch_required_bytes(const lbm_config* cfgs, int n, size_t* bytes);
/* The same for explicit options (NULL: defaults); LBM_ERR_ARG for an invalid
 * batch or option. */
lbm_status lbm_batch_required_bytes_ex(const lbm_config* cfgs, int n, const lbm_batch_opts* opts,
                                       size_t* bytes);
/* Creates the batch over dev_mem (256-byte aligned) on the current device
 * with the default options; copies the descriptors and queues and builds
 * the graph (synchronous). */
lbm_status lbm_batch_create(const lbm_config* cfgs, int n, void* dev_mem, size_t bytes,
                            lbm_batch** out);
lbm_status lbm_batch_create_ex(const lbm_config* cfgs, int n, const lbm_batch_opts* opts, void* dev_mem,
                               size_t bytes, lbm_batch** out);
lbm_status lbm_batch_get_opts(const lbm_batch* b, lbm_batch_opts* opts);
void lbm_batch_destroy(lbm_batch* b);
/* Every instance to the equilibrium of a uniform (rho, u) (entropic for ELBM
 * instances, the configured one otherwise; u_y ignored for D1Q3); resets the
 * step counter. */
lbm_status lbm_batch_init_uniform(lbm_batch* b, double rho, double ux, double uy, void* stream);
/* Per-instance state transfer, dense DEVICE f[Q][ny][nx] as in
 * lbm_set_state / lbm_get_state.  set_state needs an even step count. */
lbm_status lbm_batch_set_state(lbm_batch* b, int instance, const void* f, int dtype, void* stream);
lbm_status lbm_batch_get_state(lbm_batch* b, int instance, void* f, int dtype, void* stream);
/* Advances every instance nsteps steps (graph replays, the remainder as
 * direct launches).  If status is not NULL it receives, per instance,
 * LBM_OK or LBM_ERR_DIVERGED (a non-finite or non-positive density seen
 * since creation or the last init); this synchronises `stream` and returns
 * LBM_ERR_TIMEOUT if a bounded wait ran out since the last check. */
lbm_status lbm_batch_step(lbm_batch* b, int nsteps, int* status, void* stream);
/* Per-collision-group timing: for each collision k = LBM_LBGK ... LBM_MRT,
 * the instances of that collision alone advance nsteps steps in one
 * persistent launch timed with CUDA events on `stream`; ms[k] receives its
 * time in milliseconds (0 for a collision without instances).  Every
 * instance ends nsteps steps further, as after lbm_batch_step.
 * Synchronises `stream`; LBM_ERR_TIMEOUT as lbm_batch_step. */
lbm_status lbm_batch_group_times(lbm_batch* b, int nsteps, double* ms, void* stream);
lbm_status lbm_batch_stats(lbm_batch* b, int instance, lbm_stats* out, void* stream);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Autotuner.  Sweeps one knob at a time from *best (tile width 32, 64, 128,
 * 256; tiles per item 1, 2, 4, 8, 16; CTAs per SM 0, 6, 4, 2; chunk 1, 4, 16;
 * both orders), keeping each value that lowers the objective, and writes the
 * winner to *best and its objective to *best_obj.  Each candidate is a batch
 * of cfgs created over dev_mem (at least lbm_batch_tune_bytes; it is
 * overwritten), started from rest, two steps of warm-up, then `steps` steps
 * of each collision group alone (lbm_batch_group_times) on `stream`
 * (synchronised).  The objective is the mean over the groups of each
 * group's time relative to its time with the starting options (1 = the
 * start), so that every group weighs alike.  Up to cap candidates (options,
 * summed group time per step in ms, objective) go to records (may be NULL)
 * and *nrec receives how many were timed. */
typedef struct {
    lbm_batch_opts opts;
    double ms_per_step;
    double objective;
} lbm_batch_tune_record;
lbm_status lbm_batch_tune_bytes(const lbm_config* cfgs, int n, size_t* bytes);
lbm_status lbm_batch_tune(const lbm_config* cfgs, int n, void* dev_mem, size_t bytes, int steps,
                          lbm_batch_opts* best, lbm_batch_tune_record* records, int cap, int* nrec,
                          double* best_obj, void* stream);

/* Testing support for the bounded waits: sets the step generation of
 * `instance` one step behind the batch, so that the instance's next step
 * waits for a step that is never published and runs into wait_ms
 * (synchronous; LBM_ERR_STATE before the first step). */
lbm_status lbm_batch_debug_hold(lbm_batch* b, int instance, void* stream);

/* ---- Adjoint: reverse-mode gradient ---------------------------------------
 * For the LBGK, Ehrenfest, median-filter and positivity collisions (no
 * diffusive walls): the gradient of a functional J of the state f_T after T
 * steps with respect to the initial populations f_0, the lid velocity
 * (lid_u) and beta.  J defaults to the kinetic energy 1/2 sum_x rho |u|^2;
 * any J is served by passing its gradient dJ/df_T as `seed`.  Per step the
 * adjoint is the transpose of the streaming (walls and moving-lid term
 * included) and of the collision's Jacobian.  Through the limiters the
 * selected branch is differentiated with the selection of each step held
 * fixed: F = f* at the sites the Ehrenfest step selected (Section 4);
 * F = f* + (1 - 2 beta) sqrt(M / C) (f - f*) at the median filter's sites
 * (Section 4.4, Eq. entrHom), through both C = Delta S of the site and
 * M = Delta S of the window site holding the lower median (ties by site
 * index); F = f* + f*_k / (f*_k - f_k) (f - f*) where the positivity rule
 * (Eq. StrLine) binds at population k.  Checkpoint and recompute: the
 * forward pass keeps a dense copy of the state every K steps; the backward
 * pass, segment by segment from the last, recomputes the K states and each
 * site's branch and runs K adjoint steps.  `work` is caller DEVICE memory
 * of lbm_adjoint_required_bytes (256-byte aligned): ceil(T/K) checkpoints,
 * K segment states, K branch records of one int per site (limiters), two
 * adjoint buffers and the final state, dense in the arithmetic type (double
 * for FP64 storage, float otherwise).  Nothing is allocated. */
lbm_status lbm_adjoint_required_bytes(const lbm_config* cfg, int T, int K, size_t* bytes);
/* Advances ctx T steps from its current state (which must be at an even step
 * count) keeping the checkpoints; *J_host (if not NULL) receives the kinetic
 * energy of f_T and then the stream is synchronised. */
lbm_status lbm_adjoint_forward(lbm_ctx* ctx, int T, int K, void* work, size_t work_bytes,
                               double* J_host, void* stream);
/* After lbm_adjoint_forward with the same T, K and work: dJ/df_0 into the
 * dense DEVICE array dJ_df0 [Q][ny][nx] of out_dtype (may be NULL), dJ/dU and
 * dJ/dbeta into the host doubles (may be NULL); seed = dJ/df_T (dense DEVICE
 * array of seed_dtype) or NULL for the kinetic energy.  The context holds
 * f_T again on return (its step counter and statistics are reset).
 * Synchronises the stream. */
lbm_status lbm_adjoint_backward(lbm_ctx* ctx, int T, int K, const void* seed, int seed_dtype,
                                void* dJ_df0, int out_dtype, double* dJ_dU, double* dJ_dbeta,
                                void* work, size_t work_bytes, void* stream);

/* Kernel tracing.  While enabled, every kernel lbm_step launches is
 * bracketed by two CUDA events recorded on the caller's stream (timing
 * events; the first LBM_PROFILE_MAX launches after enabling are kept).
 * Enabling clears the record.  Costs two event records per launch. */
#define LBM_PROFILE_MAX 65536
enum { LBM_KERNEL_STEP = 0, LBM_KERNEL_FIXUP = 1, LBM_KERNEL_KINDS = 2 };
lbm_status lbm_profile_enable(lbm_ctx* ctx, int enable);

/* Waits for the recorded events and returns, per kernel kind (index
 * LBM_KERNEL_STEP: the fused stream-collide kernel; LBM_KERNEL_FIXUP: the
 * limiter kernels around it - after it, FP64 Delta S of the screened sites
 * then the Ehrenfest selection, the median filter or the threshold limiter;
 * before it, the lattice mean of Delta S for LBM_ENSEMBLE), the number of
 * launches and their summed device time in milliseconds (arrays of
 * LBM_KERNEL_KINDS entries), then clears the record. */
lbm_status lbm_profile_read(lbm_ctx* ctx, int* launches, double* ms);

/* ---- Stepping without any device allocation -----------------------------
 * The paper has no counterpart to this call; it serves deployment.  Some
 * callers cannot allocate device memory where they step: a host framework
 * that owns a fixed device pool and hands a plugin only the population
 * buffer, or a time-critical loop that must not call cudaMalloc because it
 * can synchronise the device and stall other streams.  Such a caller cannot
 * provide the scratch that lbm_create needs, and uses this call instead.
 *
 * Runs nsteps (even, >= 0) LBGK steps with the Ehrenfest limiter
 * (cfg->collision must be LBM_EHRENFEST; the other fields as for
 * lbm_create) on the caller's DENSE population array f[Q][ny][nx] (no row
 * padding; natural pre-collision layout on entry and on return; elements in
 * the configured storage format: double, float, or f_i - W_i in bf16/fp16),
 * enqueued on `stream`.  It calls no allocating routine.  Its scratch (step
 * counters and the limiter candidate list) is one file-scope device array of
 * LBM_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds
 * until the process exits.  A lattice whose scratch would not fit,
 * 256 + N (Q b + 16) bytes plus alignment with N = nx * ny and b = 8 in FP64,
 * 4 otherwise (about 645,000 D2Q9 sites in FP32, 381,000 in FP64), is
 * rejected with LBM_ERR_OOM before any GPU work.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array, which keeps the
 * last call's contents (the counters are cleared at the start of each call):
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Returns LBM_ERR_ARG for an invalid
 * configuration (the checks of lbm_create), an odd nsteps, another collision
 * or diffusive walls, LBM_ERR_CUDA when a CUDA call fails.  The call does
 * not wait for its kernels, so it cannot report what they find: a diverged
 * state (non-finite or non-positive density) is not reported, and neither
 * are the limiter statistics; a caller that needs them uses lbm_create and
 * lbm_stats_get. */
#define LBM_NOALLOC_SCRATCH_BYTES (32u << 20)
lbm_status lbm_ehrenfest_step_noalloc(const lbm_config* cfg, void* f, int nsteps, void* stream);

/* ---------------------------------------------------------------------------
 * Measurement support (the paper has no counterpart).  FP64 throughput of the
 * current GPU: *dfma_flops = FP64 fused multiply-add rate in FLOP/s (2 per
 * FMA), *log_per_s = FP64 log() evaluations per second, each from one timed
 * launch after a warm-up launch on `stream` (synchronised).  These are the
 * ceilings of the step kernels bound by the FP64 pipe (the ELBM root solve,
 * FP64 storage).  Either output may be NULL, not both (LBM_ERR_ARG).
 * Allocates and frees 8 bytes of device memory; LBM_ERR_CUDA on failure.
 * ------------------------------------------------------------------------- */
lbm_status lbm_fp64_rates(double* dfma_flops, double* log_per_s, void* stream);

/* Message of the last failure on ctx ("" if none).  Valid until the next call.
 * With ctx NULL: the message of the calling thread's last failed lbm_create
 * ("" after a successful one). */
const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(lbm_status s);
int lbm_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
