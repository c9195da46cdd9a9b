// extern "C" boundary of the GB300 lattice Boltzmann library (declared in
// include/lbm.h).  Owns no device memory: the caller's allocation is carved
// into the population array and the scratch the limiters need.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"
#include "lbm_setup.h"

using namespace lbm;

namespace lbm {
extern template struct Launch<StF64>;
extern template struct Launch<StF32>;
extern template struct Launch<StBF16>;
extern template struct Launch<StF16>;
const char* check_config(const lbm_config* c) {
    if (!c) return "config is NULL";
    if (c->lattice != LBM_D1Q3 && c->lattice != LBM_D2Q9) return "lattice must be LBM_D1Q3 or LBM_D2Q9";
    if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
    if (c->lattice == LBM_D1Q3 && c->ny != 1) return "D1Q3 needs ny == 1";
    if ((long long)c->nx * c->ny > 0x7fffffffLL) return "nx * ny must fit in 31 bits";
    if (c->ny > 65535LL * kBlockY) return "ny too large for the launch grid";
    if ((long long)(c->lattice == LBM_D1Q3 ? 3 : 9) * c->ny * ((c->nx + 31) / 32 * 32) >= 0x7fffffffLL)
        return "Q * ny * pitch must be below 2^31 elements";
    if (c->collision < LBM_LBGK || c->collision > LBM_ENSEMBLE_LAGGED) return "unknown collision";
    if ((c->collision == LBM_MRT2 || c->collision == LBM_MRT_LIMITER) && c->lattice != LBM_D2Q9)
        return "LBM_MRT2 and LBM_MRT_LIMITER need D2Q9";
    if (c->equilibrium < LBM_EQ_POLY_PRODUCT || c->equilibrium > LBM_EQ_POLY_STD) return "unknown equilibrium";
    if (c->precision < LBM_FP64 || c->precision > LBM_FP16_DEV) return "unknown precision";
    if (c->bc < LBM_BC_CAVITY || c->bc > LBM_BC_DIFFUSIVE) return "unknown boundary condition";
    if (c->bc == LBM_BC_DIFFUSIVE && (c->lattice != LBM_D2Q9 || c->nx < 3 || c->ny < 3))
        return "DIFFUSIVE needs D2Q9 with nx, ny >= 3";
    if (c->lattice == LBM_D1Q3 && c->bc == LBM_BC_CHANNEL) return "CHANNEL needs D2Q9";
    double beta = c->beta > 0 ? c->beta : (c->nu > 0 ? 1.0 / (6.0 * c->nu + 1.0) : -1.0);
    if (!(beta > 0.0 && beta <= 1.0)) return "beta must be in (0, 1] (or nu > 0)";
    if (!std::isfinite(c->lid_u)) return "lid_u must be finite";
    if (c->topk < 0) return "topk must be >= 0";
    if (!(c->delta >= 0.0)) return "delta must be >= 0";
    const bool ensemble = c->collision == LBM_ENSEMBLE || c->collision == LBM_ENSEMBLE_LAGGED;
    if (c->collision == LBM_SMOOTH || ensemble) {
        if (!(c->lim_alpha > 0.0 && std::isfinite(c->lim_alpha))) return "lim_alpha must be > 0";
    }
    if (c->collision == LBM_SMOOTH || ensemble || c->collision == LBM_DOUBLE_MONOTONIC) {
        if (!(c->lim_k > 0.0 && std::isfinite(c->lim_k))) return "lim_k must be > 0";
    }
    if (c->collision == LBM_DOUBLE_MONOTONIC && !(c->lim_dst > 0.0)) return "lim_dst must be > 0";
    if (c->collision == LBM_THRESHOLD && !(c->lim_delta0 >= 0.0 && std::isfinite(c->lim_delta0)))
        return "lim_delta0 must be >= 0";
    if (c->collision == LBM_ELBM) {
        if (!(c->elbm_eps > 0.0)) return "elbm_eps must be > 0";
        if (c->elbm_max_iter < 1) return "elbm_max_iter must be >= 1";
        if (c->elbm_norm != LBM_NORM_ENTROPIC && c->elbm_norm != LBM_NORM_L1) return "unknown elbm_norm";
        if (c->elbm_fallback != LBM_FALLBACK_POSITIVITY && c->elbm_fallback != LBM_FALLBACK_EHRENFEST)
            return "unknown elbm_fallback";
    }
    return nullptr;
}


double config_beta(const lbm_config* c) { return c->beta > 0 ? c->beta : 1.0 / (6.0 * c->nu + 1.0); }

void fill_params(const lbm_config* cfg, int nsm, Params& p) {
    p.nx = cfg->nx;
    p.ny = cfg->ny;
    p.periodic_x = cfg->bc == LBM_BC_PERIODIC || cfg->bc == LBM_BC_CHANNEL;
    p.periodic_y = cfg->bc == LBM_BC_PERIODIC;
    p.eq = cfg->equilibrium;
    p.lid_u = (cfg->bc == LBM_BC_CAVITY || cfg->bc == LBM_BC_CHANNEL) ? cfg->lid_u : 0.0;
    p.diffusive = cfg->bc == LBM_BC_DIFFUSIVE;
    p.wall_u = p.diffusive ? cfg->lid_u : 0.0;
    p.beta = config_beta(cfg);
    p.topk = cfg->topk;
    p.delta = cfg->delta;
    p.beta_f = (float)p.beta;
    p.lid_u_f = (float)p.lid_u;
    p.delta_f = (float)cfg->delta;
    const double snu = 2.0 * p.beta;
    p.mrt.e = cfg->s_e / 36.0;
    p.mrt.eps = cfg->s_eps / 36.0;
    p.mrt.q = cfg->s_q / 12.0;
    p.mrt.nu = snu / 4.0;
    p.mrt_f = {(float)p.mrt.e, (float)p.mrt.eps, (float)p.mrt.q, (float)p.mrt.nu};
    p.elbm_eps = cfg->elbm_eps;
    p.elbm_max_iter = cfg->elbm_max_iter;
    p.elbm_norm = cfg->elbm_norm;
    p.elbm_fallback = cfg->elbm_fallback;
    // the rounding of FP32 (or coarser) storage alone leaves Delta S up to
    // 2^-49 rho: below that the state is at equilibrium as far as the
    // storage can tell, and the LBGK step is taken as for Delta S < 1e-15
    p.elbm_skip_rel = cfg->precision == LBM_FP64 ? 0.0 : 0x1p-48;
    p.lim_alpha = cfg->lim_alpha;
    p.lim_k = cfg->lim_k;
    p.lim_dst = cfg->lim_dst;
    p.lim_delta0 = cfg->lim_delta0;
    // the limiter constants in FP32, so the 16/32-bit step kernels convert
    // no FP64 parameter per site (GB300's FP64 pipe is narrow)
    p.lim_f[0] = (float)cfg->lim_alpha;
    p.lim_f[1] = (float)cfg->lim_k;
    p.lim_f[2] = cfg->lim_dst > 0.0 ? (float)(1.0 / cfg->lim_dst) : 0.f;
    p.lim_f[3] = cfg->lim_k > 0.0 ? (float)(-0.5 / cfg->lim_k) : 0.f;
    // median filter: with 1 - 2 beta away from 0 the window's Delta S is
    // recovered from the post-collision state, f - f* = (F - f*) / (1 - 2 beta),
    // and the step writes no Delta S field (median_recon_fixup).  The
    // recovery multiplies the stored rounding of F by 1 / |1 - 2 beta|: up to
    // 16 for FP32 / FP64 storage, up to 4 for the 16-bit formats, whose own
    // rounding is coarser; closer to beta = 1/2 the step writes the field.
    p.median_inv = 0.0;
    if (cfg->collision == LBM_MEDIAN) {
        const bool wide = cfg->precision == LBM_FP64 || cfg->precision == LBM_FP32;
        const double b = cfg->precision == LBM_FP64 ? p.beta : (double)p.beta_f;
        if (std::fabs(1.0 - 2.0 * b) >= (wide ? 1.0 / 16 : 0.25)) p.median_inv = 1.0 / (1.0 - 2.0 * b);
    }
    p.pipe_ctas = 8 * nsm;
}

}  // namespace lbm

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t storage_bytes(int precision) {
    return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
}
size_t math_bytes(int precision) { return precision == LBM_FP64 ? 8 : 4; }

// collisions with a candidate list and a follow-up kernel
bool limiter(int coll) {
    return coll == LBM_EHRENFEST || coll == LBM_MEDIAN || coll == LBM_THRESHOLD || coll == LBM_MRT_LIMITER;
}
// collisions that reduce over the lattice each step
bool reduces(int coll) { return coll == LBM_ENSEMBLE || coll == LBM_THRESHOLD || coll == LBM_ENSEMBLE_LAGGED; }

struct Layout {
    int Q, pitch;
    int64_t plane;
    size_t f_off, f_bytes, cnt_off, cand_f_off, cand_ds_off, cand_site_off, cand_sel_off,
        field_off, red_off, staging_off, total;
    int cand_cap;
};

Layout layout(const lbm_config* c) {
    Layout L;
    L.Q = c->lattice == LBM_D1Q3 ? 3 : 9;
    L.pitch = (c->nx + 31) / 32 * 32;
    L.plane = (int64_t)c->ny * L.pitch;
    const size_t N = (size_t)c->nx * c->ny;
    size_t off = 0;
    L.f_off = off;
    L.f_bytes = align_up((size_t)L.Q * L.plane * storage_bytes(c->precision));
    off += L.f_bytes;
    L.cnt_off = off;
    off += align_up(CNT_WORDS * 4 + ST_WORDS * 8 + 8 * 8);
    L.cand_cap = limiter(c->collision) ? (int)N : 0;
    const size_t cap = (size_t)L.cand_cap;
    L.cand_f_off = off;
    off += align_up(cap * L.Q * math_bytes(c->precision));
    L.cand_ds_off = off;
    off += align_up(cap * 8);
    L.cand_site_off = off;
    off += align_up(cap * 4);
    L.cand_sel_off = off;
    off += align_up(cap * 4);
    L.field_off = off;
    off += c->collision == LBM_MEDIAN ? align_up(N * math_bytes(c->precision)) : 0;
    L.red_off = off;  // kRedSlots sums + kRedSlots counts + E
    off += reduces(c->collision) ? align_up((2 * kRedSlots + 8) * sizeof(double)) : 0;
    L.staging_off = off;
    off += align_up(3 * N * 8);
    L.total = off;
    return L;
}

lbm_status fail(lbm_ctx* ctx, lbm_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(ctx, LBM_ERR_CUDA, m);
}

#define LBM_CK(ctx, expr)                                       \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

template <class Fn>
cudaError_t dispatch(int precision, Fn&& fn) {
    switch (precision) {
        case LBM_FP64: return fn(Launch<StF64>());
        case LBM_FP32: return fn(Launch<StF32>());
        case LBM_BF16_DEV: return fn(Launch<StBF16>());
        case LBM_FP16_DEV: return fn(Launch<StF16>());
    }
    return cudaErrorInvalidValue;
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

// Message of the calling thread's last failed lbm_create (no context exists
// to hold it).
thread_local std::string g_create_error;

// Launches fn() bracketed by a pair of timing events when tracing is on.
template <class Fn>
cudaError_t traced(lbm_ctx* ctx, int kind, cudaStream_t s, Fn&& fn) {
    if (!ctx->profiling || ctx->ev_used >= LBM_PROFILE_MAX) return fn();
    if (ctx->ev.size() < 2 * (ctx->ev_used + 1)) {
        for (int k = 0; k < 2; ++k) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            ctx->ev.push_back(e);
        }
        ctx->ev_kind.push_back(0);
    }
    cudaEvent_t a = ctx->ev[2 * ctx->ev_used], b = ctx->ev[2 * ctx->ev_used + 1];
    cudaError_t err = cudaEventRecord(a, s);
    if (err == cudaSuccess) err = fn();
    if (err == cudaSuccess) err = cudaEventRecord(b, s);
    if (err == cudaSuccess) ctx->ev_kind[ctx->ev_used++] = kind;
    return err;
}

// d g / d coordinate at index i of a line of n values (spacing 1, stride
// between neighbours), as in the enstrophy's definition in include/lbm.h.
__device__ __forceinline__ double line_diff(const double* g, int64_t stride, int i, int n, int periodic) {
    if (n < 2) return 0.0;
    if (periodic) {
        const int ip = i + 1 < n ? i + 1 : 0, im = i > 0 ? i - 1 : n - 1;
        return 0.5 * (g[ip * stride] - g[im * stride]);
    }
    if (i == 0) return g[stride] - g[0];
    if (i == n - 1) return g[(int64_t)i * stride] - g[(int64_t)(i - 1) * stride];
    return 0.5 * (g[(int64_t)(i + 1) * stride] - g[(int64_t)(i - 1) * stride]);
}

// Sum over sites of w^2 (Section 8's enstrophy times the site count) into
// *out, from the FP64 site velocities ux, uy [ny][nx].
__global__ void __launch_bounds__(256) enstrophy_kernel(int nx, int ny, int px, int py, const double* __restrict__ ux,
                                                        const double* __restrict__ uy, double* out) {
    __shared__ double part[8];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (s < (int64_t)nx * ny) {
        const int y = (int)(s / nx), x = (int)(s - (int64_t)y * nx);
        const double w = line_diff(uy + (int64_t)y * nx, 1, x, nx, px) - line_diff(ux + x, nx, y, ny, py);
        e = w * w;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
        if (t != 0.0) atomicAdd(out, t);
    }
}

lbm_status reset_counters(lbm_ctx* ctx, cudaStream_t s) {
    LBM_CK(ctx, cudaMemsetAsync(ctx->p.counters, 0, CNT_WORDS * 4 + ST_WORDS * 8, s));
    return LBM_OK;
}

// The lagged ensemble limiter's E(Delta S) for the first step of a new
// state: the mean over that state itself (the unlagged limiter's pre-pass).
lbm_status initial_mean(lbm_ctx* ctx, cudaStream_t s) {
    if (ctx->cfg.collision != LBM_ENSEMBLE_LAGGED) return LBM_OK;
    Params q = ctx->p;
    q.pdl = 0;
    LBM_CK(ctx, dispatch(ctx->cfg.precision,
                         [&](auto L) { return decltype(L)::prepass(ctx->Q, LBM_ENSEMBLE, false, q, s); }));
    return LBM_OK;
}

}  // namespace

namespace {

// The kernels of one step with counter slot `cslot` and A-A parity `odd`.
cudaError_t enqueue_one_step(lbm_ctx* ctx, bool odd, int cslot, cudaStream_t s) {
    const int coll = ctx->cfg.collision;
    Params q = ctx->p;
    q.cslot = cslot;
    q.pdl = ctx->profiling ? 0 : 1;  // the timing events bracket whole kernels
    cudaError_t e = cudaSuccess;
    if (coll == LBM_ENSEMBLE)  // E(Delta S) of this step's pre-collision state
        e = traced(ctx, LBM_KERNEL_FIXUP, s, [&] {
            return dispatch(ctx->cfg.precision,
                            [&](auto L) { return decltype(L)::prepass(ctx->Q, coll, odd, q, s); });
        });
    if (e == cudaSuccess)
        e = traced(ctx, LBM_KERNEL_STEP, s, [&] {
            return dispatch(ctx->cfg.precision,
                            [&](auto L) { return decltype(L)::step(ctx->Q, coll, odd, q, s); });
        });
    if (e == cudaSuccess && q.diffusive)  // the wall sites of the same step
        e = dispatch(ctx->cfg.precision, [&](auto L) { return decltype(L)::walls(odd, q, s); });
    if (e == cudaSuccess && (limiter(coll) || coll == LBM_ENSEMBLE_LAGGED))
        e = traced(ctx, LBM_KERNEL_FIXUP, s, [&] {
            return dispatch(ctx->cfg.precision,
                            [&](auto L) { return decltype(L)::fixup(ctx->Q, coll, odd, q, s, ctx->nsm); });
        });
    if (e == cudaSuccess && q.probe_buf)  // the control point of the state just produced
        e = dispatch(ctx->cfg.precision, [&](auto L) { return decltype(L)::probe(ctx->Q, !odd, q, s); });
    return e;
}

// Captures `periods` A-A periods (even step with counter slot 0, odd with
// slot 1, repeated) into *graph / *exec on a private stream.
cudaError_t capture_periods(lbm_ctx* ctx, int periods, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaSuccess;
        for (int k = 0; k < periods && e1 == cudaSuccess; ++k) {
            e1 = enqueue_one_step(ctx, false, 0, cap);
            if (e1 == cudaSuccess) e1 = enqueue_one_step(ctx, true, 1, cap);
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        if (e1 != cudaSuccess) e = e1;
        if (e == cudaSuccess) {
            *graph = g;
            e = cudaGraphInstantiate(exec, g, 0);
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(cap);
    return e;
}

// The two-step graph lbm_step replays, and for long runs of small lattices
// (where the host's graph launches, not the GPU, set the pace) one of
// kLongPeriods periods.
constexpr int kLongPeriods = 32;

cudaError_t build_step_graph(lbm_ctx* ctx) {
    cudaError_t e = capture_periods(ctx, 1, &ctx->graph, &ctx->graph_exec);
    if (e == cudaSuccess) e = capture_periods(ctx, kLongPeriods, &ctx->graph_long, &ctx->graph_long_exec);
    return e;
}

}  // namespace

extern "C" {

int lbm_abi_version(void) { return LBM_ABI_VERSION; }

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_ERR_ARG: return "LBM_ERR_ARG";
        case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
        case LBM_ERR_OOM: return "LBM_ERR_OOM";
        case LBM_ERR_DIVERGED: return "LBM_ERR_DIVERGED";
        case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
        case LBM_ERR_STATE: return "LBM_ERR_STATE";
    }
    return "unknown lbm_status";
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

lbm_status lbm_config_default(lbm_config* c) {
    if (!c) return LBM_ERR_ARG;
    std::memset(c, 0, sizeof *c);
    c->lattice = LBM_D2Q9;
    c->nx = c->ny = 16;
    c->collision = LBM_LBGK;
    c->equilibrium = LBM_EQ_POLY_PRODUCT;
    c->precision = LBM_FP32;
    c->bc = LBM_BC_CAVITY;
    c->beta = 0.9;
    c->delta = 1e-3;
    c->s_e = 1.64;
    c->s_eps = 1.54;
    c->s_q = 1.9;
    c->elbm_eps = 1e-15;
    c->elbm_max_iter = 20;
    c->elbm_norm = LBM_NORM_ENTROPIC;
    c->elbm_fallback = LBM_FALLBACK_POSITIVITY;
    c->lim_alpha = 1.0;
    c->lim_k = 1.0;
    c->lim_dst = 1e-3;
    c->lim_delta0 = 0.01;
    return LBM_OK;
}

lbm_status lbm_mrt_preset(lbm_config* cfg, int preset) {
    if (!cfg) return LBM_ERR_ARG;
    const double beta = cfg->beta > 0 ? cfg->beta : (cfg->nu > 0 ? 1.0 / (6.0 * cfg->nu + 1.0) : -1.0);
    if (!(beta > 0.0 && beta <= 1.0)) return LBM_ERR_ARG;
    const double snu = 2.0 * beta;
    // the "magic" relation of Section 5's TRT, s_q = 8 (2 - s_nu) / (8 - s_nu)
    const double sq_trt = 8.0 * (2.0 - snu) / (8.0 - snu);
    switch (preset) {
        case LBM_MRT_PRESET_TRT:
            cfg->s_e = snu;
            cfg->s_eps = snu;
            cfg->s_q = sq_trt;
            return LBM_OK;
        case LBM_MRT_PRESET_MRT:
            cfg->s_e = 1.64;
            cfg->s_eps = 1.54;
            cfg->s_q = sq_trt;
            return LBM_OK;
        case LBM_MRT_PRESET_MRT1:
            cfg->s_e = 1.64;
            cfg->s_eps = 1.54;
            cfg->s_q = 1.9;
            return LBM_OK;
        case LBM_MRT_PRESET_LL:
            cfg->s_e = 1.64;
            cfg->s_eps = 1.54;
            cfg->s_q = 3.0 * (2.0 - snu) / (3.0 - snu);
            return LBM_OK;
    }
    return LBM_ERR_ARG;
}

lbm_status lbm_required_bytes(const lbm_config* cfg, size_t* bytes) {
    if (!bytes || check_config(cfg)) return LBM_ERR_ARG;
    *bytes = layout(cfg).total;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, void* dev_mem, size_t bytes, lbm_ctx** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (check_config(cfg)) return LBM_ERR_ARG;
    if (!dev_mem || ((uintptr_t)dev_mem % kAlign) != 0) return LBM_ERR_ARG;
    Layout L = layout(cfg);
    if (bytes < L.total) return LBM_ERR_OOM;
    lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
    if (!ctx) return LBM_ERR_OOM;
    ctx->cfg = *cfg;
    ctx->cfg.beta = config_beta(cfg);
    ctx->Q = L.Q;
    ctx->base = (char*)dev_mem;
    ctx->bytes = bytes;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        g_create_error = "lbm_create: no current CUDA device";
        delete ctx;
        return LBM_ERR_CUDA;
    }
    Params& p = ctx->p;
    std::memset(&p, 0, sizeof p);
    fill_params(&ctx->cfg, ctx->nsm, p);
    p.f = ctx->base + L.f_off;
    p.plane = L.plane;
    p.plane32 = (int)L.plane;
    p.pitch = L.pitch;
    p.counters = (unsigned*)(ctx->base + L.cnt_off);
    p.stats = (unsigned long long*)(ctx->base + L.cnt_off + CNT_WORDS * 4);
    p.scratch_d = (double*)(ctx->base + L.cnt_off + CNT_WORDS * 4 + ST_WORDS * 8);
    p.cand_cap = L.cand_cap;
    p.cand_f = ctx->base + L.cand_f_off;
    p.cand_ds = (double*)(ctx->base + L.cand_ds_off);
    p.cand_site = (int*)(ctx->base + L.cand_site_off);
    p.cand_sel = (int*)(ctx->base + L.cand_sel_off);
    p.ds_field = ctx->base + L.field_off;
    if (reduces(cfg->collision)) {
        p.red = (double*)(ctx->base + L.red_off);
        p.lim_E = p.red + 2 * kRedSlots;
        p.lim_E_f = (float*)(p.lim_E + 1);
    }
    ctx->staging = (double*)(ctx->base + L.staging_off);
    cudaError_t e = cudaMemset(ctx->base + L.cnt_off, 0, align_up(CNT_WORDS * 4 + ST_WORDS * 8 + 64));
    if (e == cudaSuccess && reduces(cfg->collision))
        e = cudaMemset(ctx->base + L.red_off, 0, (2 * kRedSlots + 8) * sizeof(double));
    const char* where = "cudaMemset of the counters";
    if (e == cudaSuccess) {
        e = build_step_graph(ctx);
        where = "capture of the two-step graph";
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("lbm_create: ") + where + ": " + cudaGetErrorName(e) + " (" +
                         cudaGetErrorString(e) + ")";
        delete ctx;
        return LBM_ERR_CUDA;
    }
    g_create_error.clear();
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* ctx) { delete ctx; }

lbm_status lbm_init_device(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                           void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (!rho || !ux || (ctx->Q == 9 && !uy)) return fail(ctx, LBM_ERR_ARG, "rho, ux (and uy for D2Q9) are required");
    const int eqkind = ctx->cfg.collision == LBM_ELBM ? LBM_EQ_ENTROPIC : ctx->cfg.equilibrium;
    lbm_status st = reset_counters(ctx, S(stream));
    if (st) return st;
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::init(ctx->Q, ctx->p, rho, ux, ctx->Q == 9 ? uy : nullptr, eqkind, S(stream));
           }));
    ctx->parity = 0;
    ctx->t = 0;
    return initial_mean(ctx, S(stream));
}

lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (!rho || !ux || (ctx->Q == 9 && !uy)) return fail(ctx, LBM_ERR_ARG, "rho, ux (and uy for D2Q9) are required");
    const size_t N = (size_t)ctx->cfg.nx * ctx->cfg.ny;
    double* d = ctx->staging;
    LBM_CK(ctx, cudaMemcpyAsync(d, rho, N * 8, cudaMemcpyHostToDevice, S(stream)));
    LBM_CK(ctx, cudaMemcpyAsync(d + N, ux, N * 8, cudaMemcpyHostToDevice, S(stream)));
    if (ctx->Q == 9) LBM_CK(ctx, cudaMemcpyAsync(d + 2 * N, uy, N * 8, cudaMemcpyHostToDevice, S(stream)));
    lbm_status st = lbm_init_device(ctx, d, d + N, d + 2 * N, stream);
    if (st) return st;
    LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* ctx, const void* f, int dtype, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (!f || (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)) return fail(ctx, LBM_ERR_ARG, "bad state buffer or dtype");
    lbm_status st = reset_counters(ctx, S(stream));
    if (st) return st;
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::set_state(ctx->Q, ctx->p, f, dtype, S(stream));
           }));
    ctx->parity = 0;
    ctx->t = 0;
    return initial_mean(ctx, S(stream));
}

lbm_status lbm_get_state(lbm_ctx* ctx, void* f, int dtype, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (!f || (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)) return fail(ctx, LBM_ERR_ARG, "bad state buffer or dtype");
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::get_state(ctx->Q, ctx->p, f, dtype, ctx->parity != 0, S(stream));
           }));
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int nsteps, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(ctx, LBM_ERR_ARG, "nsteps must be >= 0");
    // parity == t & 1 always (both reset together), so the graph, whose
    // steps use counter slots 0 and 1, starts at an even step
    int k = 0;
    const bool use_graph = ctx->graph_exec && !ctx->profiling;
    while (k < nsteps) {
        if (use_graph && ctx->parity == 0 && ctx->graph_long_exec && nsteps - k >= 2 * kLongPeriods) {
            LBM_CK(ctx, cudaGraphLaunch(ctx->graph_long_exec, S(stream)));
            ctx->t += 2 * kLongPeriods;
            k += 2 * kLongPeriods;
            continue;
        }
        if (use_graph && ctx->parity == 0 && nsteps - k >= 2) {
            LBM_CK(ctx, cudaGraphLaunch(ctx->graph_exec, S(stream)));
            ctx->t += 2;
            k += 2;
            continue;
        }
        LBM_CK(ctx, enqueue_one_step(ctx, ctx->parity != 0, (int)(ctx->t & 1), S(stream)));
        ctx->parity ^= 1;
        ctx->t += 1;
        ++k;
    }
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx* ctx, void* rho, void* u, int dtype, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if ((!rho && !u) || (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32)) return fail(ctx, LBM_ERR_ARG, "bad outputs or dtype");
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::macros(ctx->Q, ctx->p, rho, u, dtype, ctx->parity != 0, S(stream));
           }));
    return LBM_OK;
}

lbm_status lbm_entropy(lbm_ctx* ctx, double* H_total_host, double* dS_dev, void* stream) {
    if (!ctx) return LBM_ERR_ARG;
    if (!H_total_host && !dS_dev) return fail(ctx, LBM_ERR_ARG, "no output requested");
    const int eqkind = ctx->cfg.collision == LBM_ELBM ? LBM_EQ_ENTROPIC : ctx->cfg.equilibrium;
    double* H = ctx->p.scratch_d;
    LBM_CK(ctx, cudaMemsetAsync(H, 0, sizeof(double), S(stream)));
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::entropy(ctx->Q, ctx->p, H, dS_dev, ctx->parity != 0, eqkind, S(stream));
           }));
    if (H_total_host) {
        LBM_CK(ctx, cudaMemcpyAsync(H_total_host, H, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
        LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    }
    return LBM_OK;
}

lbm_status lbm_probe_set(lbm_ctx* ctx, int x, int y, double* buf, int cap) {
    if (!ctx) return LBM_ERR_ARG;
    if (buf && (x < 0 || x >= ctx->cfg.nx || y < 0 || y >= ctx->cfg.ny || cap < 1))
        return fail(ctx, LBM_ERR_ARG, "probe site outside the lattice or cap < 1");
    LBM_CK(ctx, cudaDeviceSynchronize());
    ctx->p.probe_buf = buf;
    ctx->p.probe_site = buf ? y * ctx->cfg.nx + x : -1;
    ctx->p.probe_cap = buf ? cap : 0;
    LBM_CK(ctx, cudaMemset(ctx->p.counters + CNT_PROBE, 0, sizeof(unsigned)));
    // the step graphs hold the kernel parameters: capture them again
    ctx->drop_graphs();
    LBM_CK(ctx, build_step_graph(ctx));
    return LBM_OK;
}

lbm_status lbm_probe_count(lbm_ctx* ctx, uint64_t* count, void* stream) {
    if (!ctx || !count) return LBM_ERR_ARG;
    unsigned c = 0;
    LBM_CK(ctx, cudaMemcpyAsync(&c, ctx->p.counters + CNT_PROBE, sizeof c, cudaMemcpyDeviceToHost, S(stream)));
    LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    *count = c;
    return LBM_OK;
}

lbm_status lbm_enstrophy(lbm_ctx* ctx, double* E_host, void* stream) {
    if (!ctx || !E_host) return LBM_ERR_ARG;
    if (ctx->Q != 9) return fail(ctx, LBM_ERR_ARG, "enstrophy needs D2Q9");
    const int64_t N = (int64_t)ctx->cfg.nx * ctx->cfg.ny;
    double* rho = ctx->staging;  // 3N doubles: rho, u_x, u_y
    double* u = ctx->staging + N;
    double* acc = ctx->p.scratch_d + 2;
    LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) {
               return decltype(L)::macros(ctx->Q, ctx->p, rho, u, LBM_DTYPE_F64, ctx->parity != 0, S(stream));
           }));
    LBM_CK(ctx, cudaMemsetAsync(acc, 0, sizeof(double), S(stream)));
    enstrophy_kernel<<<(unsigned)((N + 255) / 256), 256, 0, S(stream)>>>(ctx->cfg.nx, ctx->cfg.ny, ctx->p.periodic_x,
                                                                      ctx->p.periodic_y, u, u + N, acc);
    LBM_CK(ctx, cudaGetLastError());
    double h = 0.0;
    LBM_CK(ctx, cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
    LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    *E_host = h / (double)N;
    return LBM_OK;
}

lbm_status lbm_stats_get(lbm_ctx* ctx, lbm_stats* out, void* stream) {
    if (!ctx || !out) return LBM_ERR_ARG;
    unsigned cnt[CNT_WORDS];
    unsigned long long st[ST_WORDS];
    LBM_CK(ctx, cudaMemcpyAsync(cnt, ctx->p.counters, sizeof cnt, cudaMemcpyDeviceToHost, S(stream)));
    LBM_CK(ctx, cudaMemcpyAsync(st, ctx->p.stats, sizeof st, cudaMemcpyDeviceToHost, S(stream)));
    LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    std::memset(out, 0, sizeof *out);
    out->steps = ctx->t;
    out->candidates_last = (ctx->t > 0 && limiter(ctx->cfg.collision)) ? cnt[CNT_NVALID] : 0;
    out->limited_total = st[ST_LIMITED];
    out->elbm_solved = st[ST_ELBM_SOLVED];
    out->elbm_skipped = st[ST_ELBM_SKIPPED];
    out->elbm_fallbacks = st[ST_ELBM_FALLBACK];
    out->elbm_iters_total = st[ST_ELBM_ITERS];
    out->elbm_iters_max = st[ST_ELBM_ITERS_MAX];
    out->diverged = cnt[CNT_DIVERGED];
    out->overflow = cnt[CNT_OVERFLOW];
    out->screened_last = (ctx->t > 0 && limiter(ctx->cfg.collision)) ? cnt[(ctx->t - 1) & 1] : 0;
    return LBM_OK;
}

lbm_status lbm_last_candidates(lbm_ctx* ctx, double* ds, int32_t* site, int32_t* selected, int cap,
                               int* count, void* stream) {
    if (!ctx || !count || cap < 0) return LBM_ERR_ARG;
    if (!limiter(ctx->cfg.collision)) return fail(ctx, LBM_ERR_STATE, "collision has no candidate list");
    if (ctx->t == 0) {
        *count = 0;
        return LBM_OK;
    }
    unsigned n = 0;
    LBM_CK(ctx, cudaMemcpyAsync(&n, ctx->p.counters + ((ctx->t - 1) & 1), sizeof n, cudaMemcpyDeviceToHost, S(stream)));
    LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    if (n > (unsigned)ctx->p.cand_cap) n = (unsigned)ctx->p.cand_cap;
    // the FP64 Delta S of every screened site (the step's selection may have
    // settled them in FP32); the candidates are those with Delta S > delta
    {
        const Params& p = ctx->p;
        const int Q = ctx->Q;
        LBM_CK(ctx, dispatch(ctx->cfg.precision, [&](auto L) { return decltype(L)::cand_eval(Q, p, n, S(stream)); }));
    }
    std::vector<double> hds(n);
    std::vector<int32_t> hsite(n), hsel(n);
    if (n) {
        LBM_CK(ctx, cudaMemcpyAsync(hds.data(), ctx->p.cand_ds, n * 8, cudaMemcpyDeviceToHost, S(stream)));
        LBM_CK(ctx, cudaMemcpyAsync(hsite.data(), ctx->p.cand_site, n * 4, cudaMemcpyDeviceToHost, S(stream)));
        LBM_CK(ctx, cudaMemcpyAsync(hsel.data(), ctx->p.cand_sel, n * 4, cudaMemcpyDeviceToHost, S(stream)));
        LBM_CK(ctx, cudaStreamSynchronize(S(stream)));
    }
    int m = 0;
    for (unsigned j = 0; j < n; ++j) {
        if (!(hds[j] > ctx->cfg.delta)) continue;
        if (m < cap) {
            if (ds) ds[m] = hds[j];
            if (site) site[m] = hsite[j];
            if (selected) selected[m] = hsel[j];
        }
        ++m;
    }
    *count = m;
    return LBM_OK;
}

lbm_status lbm_profile_enable(lbm_ctx* ctx, int enable) {
    if (!ctx) return LBM_ERR_ARG;
    ctx->profiling = enable != 0;
    ctx->ev_used = 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* ctx, int* launches, double* ms) {
    if (!ctx || !launches || !ms) return LBM_ERR_ARG;
    for (int k = 0; k < LBM_KERNEL_KINDS; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
    }
    for (size_t j = 0; j < ctx->ev_used; ++j) {
        float t = 0.f;
        LBM_CK(ctx, cudaEventSynchronize(ctx->ev[2 * j + 1]));
        LBM_CK(ctx, cudaEventElapsedTime(&t, ctx->ev[2 * j], ctx->ev[2 * j + 1]));
        launches[ctx->ev_kind[j]] += 1;
        ms[ctx->ev_kind[j]] += t;
    }
    ctx->ev_used = 0;
    return LBM_OK;
}

}  // extern "C"
