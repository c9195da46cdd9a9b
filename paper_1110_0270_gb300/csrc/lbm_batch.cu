// Batched form of the step (declared in include/lbm.h): many independent D2Q9
// lattices of different sizes, parameters and collisions advanced together.
// One launch per collision kind covers all instances of that kind; two steps
// (both A-A parities) are captured once into a CUDA graph whose collision
// groups are independent branches, so that the FP64-bound ELBM instances
// overlap the HBM-bound ones.  No device allocation: the caller's block
// holds populations, scratch, descriptors and work lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_batch_kernels.cuh"

using namespace lbm;

namespace lbm {
extern template struct Launch<StF64>;
extern template struct Launch<StF32>;
extern template struct Launch<StBF16>;
extern template struct Launch<StF16>;
extern template struct BatchLaunch<StF64>;
extern template struct BatchLaunch<StF32>;
extern template struct BatchLaunch<StBF16>;
extern template struct BatchLaunch<StF16>;
}  // namespace lbm

namespace {

// Per-instance divergence flags gathered into one array.
__global__ void batch_flags_kernel(const Params* __restrict__ insts, int n, unsigned* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = insts[i].counters[CNT_DIVERGED];
}

constexpr int kKinds = 6;  // LBM_LBGK .. LBM_MRT

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct InstLayout {
    size_t f_off, cnt_off, cand_f_off, cand_ds_off, cand_site_off, cand_sel_off, field_off;
    int pitch;
    int64_t plane;
    int cap;
};

struct BatchLayout {
    std::vector<InstLayout> inst;
    size_t params_off, work_off[kKinds], ids_off[kKinds], flags_off, total;
    int nwork[kKinds], nids[kKinds];
};

const char* check_batch(const lbm_config* cfgs, int n) {
    if (!cfgs || n < 1) return "need at least one instance";
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        if (c->lattice != LBM_D2Q9) return "batched instances are D2Q9";
        if (c->precision != cfgs[0].precision) return "all instances share one precision";
        if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
        if ((long long)9 * c->ny * ((c->nx + 31) / 32 * 32) >= 0x7fffffffLL) return "instance too large";
        if (c->collision < LBM_LBGK || c->collision > LBM_MRT) return "unknown collision";
        if (c->equilibrium < LBM_EQ_POLY_PRODUCT || c->equilibrium > LBM_EQ_POLY_STD) return "unknown equilibrium";
        if (c->precision < LBM_FP64 || c->precision > LBM_FP16_DEV) return "unknown precision";
        if (c->bc != LBM_BC_CAVITY && c->bc != LBM_BC_PERIODIC && c->bc != LBM_BC_CHANNEL)
            return "unsupported boundary for D2Q9";
        double beta = c->beta > 0 ? c->beta : (c->nu > 0 ? 1.0 / (6.0 * c->nu + 1.0) : -1.0);
        if (!(beta > 0.0 && beta <= 1.0)) return "beta must be in (0, 1] (or nu > 0)";
        if (!std::isfinite(c->lid_u) || c->topk < 0 || !(c->delta >= 0.0)) return "bad lid_u, topk or delta";
        if (c->collision == LBM_ELBM && (!(c->elbm_eps > 0) || c->elbm_max_iter < 1)) return "bad ELBM parameters";
    }
    return nullptr;
}

BatchLayout make_layout(const lbm_config* cfgs, int n) {
    BatchLayout B;
    const size_t sb = cfgs[0].precision == LBM_FP64 ? 8 : (cfgs[0].precision == LBM_FP32 ? 4 : 2);
    const size_t tb = cfgs[0].precision == LBM_FP64 ? 8 : 4;
    size_t off = 0;
    std::fill(B.nwork, B.nwork + kKinds, 0);
    std::fill(B.nids, B.nids + kKinds, 0);
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        InstLayout L;
        L.pitch = (c->nx + 31) / 32 * 32;
        L.plane = (int64_t)c->ny * L.pitch;
        const size_t N = (size_t)c->nx * c->ny;
        const bool lim = c->collision == LBM_EHRENFEST || c->collision == LBM_MEDIAN;
        L.cap = lim ? (int)N : 0;
        L.f_off = off;
        off += up256(9 * (size_t)L.plane * sb);
        L.cnt_off = off;
        off += 256;
        L.cand_f_off = off;
        off += up256((size_t)L.cap * 9 * tb);
        L.cand_ds_off = off;
        off += up256((size_t)L.cap * 8);
        L.cand_site_off = off;
        off += up256((size_t)L.cap * 4);
        L.cand_sel_off = off;
        off += up256((size_t)L.cap * 4);
        L.field_off = off;
        off += c->collision == LBM_MEDIAN ? up256(N * tb) : 0;
        B.inst.push_back(L);
        const int tiles = ((c->nx + kBlockX - 1) / kBlockX) * ((c->ny + kBlockY - 1) / kBlockY);
        B.nwork[c->collision] += tiles;
        if (lim) B.nids[c->collision] += 1;
    }
    B.params_off = off;
    off += up256((size_t)n * sizeof(Params));
    for (int k = 0; k < kKinds; ++k) {
        B.work_off[k] = off;
        off += up256((size_t)B.nwork[k] * sizeof(WorkItem));
        B.ids_off[k] = off;
        off += up256((size_t)B.nids[k] * sizeof(int));
    }
    B.flags_off = off;
    off += up256((size_t)n * 4);
    B.total = off;
    return B;
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_config> cfg;
    std::vector<Params> hp;  // host copies of the instance descriptors
    BatchLayout L;
    char* base = nullptr;
    Params* d_params = nullptr;
    WorkItem* d_work[kKinds] = {};
    int* d_ids[kKinds] = {};
    unsigned* d_flags = nullptr;
    int precision = LBM_FP32;
    int parity = 0;
    uint64_t t = 0;
    cudaStream_t s_cap = nullptr;
    cudaStream_t s_kind[kKinds] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kKinds] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
    ~lbm_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (int k = 0; k < kKinds; ++k) {
            if (s_kind[k]) cudaStreamDestroy(s_kind[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (s_cap) cudaStreamDestroy(s_cap);
    }
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}

lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* where) {
    return bfail(b, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorName(e));
}

#define BCK(b, expr)                                         \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, #expr);   \
    } while (0)

template <class Fn>
cudaError_t with_format(int precision, Fn&& fn) {
    switch (precision) {
        case LBM_FP64: return fn(Launch<StF64>(), BatchLaunch<StF64>());
        case LBM_FP32: return fn(Launch<StF32>(), BatchLaunch<StF32>());
        case LBM_BF16_DEV: return fn(Launch<StBF16>(), BatchLaunch<StBF16>());
        case LBM_FP16_DEV: return fn(Launch<StF16>(), BatchLaunch<StF16>());
    }
    return cudaErrorInvalidValue;
}

// One step of every collision group, group k on stream s[k].
cudaError_t enqueue_step(lbm_batch* b, bool odd, int cslot, const cudaStream_t* s) {
    return with_format(b->precision, [&](auto, auto BL) {
        for (int k = 0; k < kKinds; ++k) {
            if (!b->L.nwork[k]) continue;
            cudaError_t e = decltype(BL)::step(k, odd, b->d_params, b->d_work[k], b->L.nwork[k], cslot, s[k]);
            if (e == cudaSuccess)
                e = decltype(BL)::fixup(k, odd, b->d_params, b->d_ids[k], b->L.nids[k], cslot, s[k]);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
}

lbm_status build_graph(lbm_batch* b) {
    BCK(b, cudaStreamCreateWithFlags(&b->s_cap, cudaStreamNonBlocking));
    BCK(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    for (int k = 0; k < kKinds; ++k) {
        BCK(b, cudaStreamCreateWithFlags(&b->s_kind[k], cudaStreamNonBlocking));
        BCK(b, cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming));
    }
    BCK(b, cudaStreamBeginCapture(b->s_cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->ev_fork, b->s_cap);
    for (int k = 0; k < kKinds && e == cudaSuccess; ++k)
        if (b->L.nwork[k]) e = cudaStreamWaitEvent(b->s_kind[k], b->ev_fork, 0);
    // the two parities of the A-A pattern; each group is its own branch
    if (e == cudaSuccess) e = enqueue_step(b, false, 0, b->s_kind);
    if (e == cudaSuccess) e = enqueue_step(b, true, 1, b->s_kind);
    for (int k = 0; k < kKinds && e == cudaSuccess; ++k) {
        if (!b->L.nwork[k]) continue;
        e = cudaEventRecord(b->ev_join[k], b->s_kind[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_cap, b->ev_join[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->s_cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e, "capture of the batched step");
    }
    BCK(b, e2);
    b->graph = g;
    BCK(b, cudaGraphInstantiate(&b->exec, g, 0));
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_required_bytes(const lbm_config* cfgs, int n, size_t* bytes) {
    if (!bytes || check_batch(cfgs, n)) return LBM_ERR_ARG;
    *bytes = make_layout(cfgs, n).total;
    return LBM_OK;
}

lbm_status lbm_batch_create(const lbm_config* cfgs, int n, void* dev_mem, size_t bytes, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (check_batch(cfgs, n)) return LBM_ERR_ARG;
    if (!dev_mem || ((uintptr_t)dev_mem % 256) != 0) return LBM_ERR_ARG;
    BatchLayout L = make_layout(cfgs, n);
    if (bytes < L.total) return LBM_ERR_OOM;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->cfg.assign(cfgs, cfgs + n);
    b->L = L;
    b->base = (char*)dev_mem;
    b->precision = cfgs[0].precision;
    b->d_params = (Params*)(b->base + L.params_off);
    for (int k = 0; k < kKinds; ++k) {
        b->d_work[k] = (WorkItem*)(b->base + L.work_off[k]);
        b->d_ids[k] = (int*)(b->base + L.ids_off[k]);
    }
    b->d_flags = (unsigned*)(b->base + L.flags_off);
    std::vector<WorkItem> work[kKinds];
    std::vector<int> ids[kKinds];
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        const InstLayout& I = L.inst[i];
        Params p;
        std::memset(&p, 0, sizeof p);
        p.f = b->base + I.f_off;
        p.plane = I.plane;
        p.plane32 = (int)I.plane;
        p.pitch = I.pitch;
        p.nx = c->nx;
        p.ny = c->ny;
        p.periodic_x = c->bc == LBM_BC_PERIODIC || c->bc == LBM_BC_CHANNEL;
        p.periodic_y = c->bc == LBM_BC_PERIODIC;
        // ELBM always uses the entropic equilibrium; storing it here makes the
        // uniform initialisation pick the right one
        p.eq = c->collision == LBM_ELBM ? LBM_EQ_ENTROPIC : c->equilibrium;
        p.lid_u = (c->bc == LBM_BC_CAVITY || c->bc == LBM_BC_CHANNEL) ? c->lid_u : 0.0;
        p.beta = c->beta > 0 ? c->beta : 1.0 / (6.0 * c->nu + 1.0);
        p.beta_f = (float)p.beta;
        p.lid_u_f = (float)p.lid_u;
        p.topk = c->topk;
        p.delta = c->delta;
        p.delta_f = (float)c->delta;
        p.mrt.e = c->s_e / 36.0;
        p.mrt.eps = c->s_eps / 36.0;
        p.mrt.q = c->s_q / 12.0;
        p.mrt.nu = 2.0 * p.beta / 4.0;
        p.mrt_f = {(float)p.mrt.e, (float)p.mrt.eps, (float)p.mrt.q, (float)p.mrt.nu};
        p.elbm_eps = c->elbm_eps;
        p.elbm_max_iter = c->elbm_max_iter;
        p.elbm_norm = c->elbm_norm;
        p.elbm_fallback = c->elbm_fallback;
        // the rounding of FP32 (or coarser) storage alone leaves Delta S up to
        // 2^-49 rho: below that the state is at equilibrium as far as the
        // storage can tell, and the LBGK step is taken as for Delta S < 1e-15
        p.elbm_skip_rel = c->precision == LBM_FP64 ? 0.0 : 0x1p-48;
        p.counters = (unsigned*)(b->base + I.cnt_off);
        p.stats = (unsigned long long*)(b->base + I.cnt_off + CNT_WORDS * 4);
        p.scratch_d = (double*)(b->base + I.cnt_off + CNT_WORDS * 4 + ST_WORDS * 8);
        p.cand_cap = I.cap;
        p.cand_f = b->base + I.cand_f_off;
        p.cand_ds = (double*)(b->base + I.cand_ds_off);
        p.cand_site = (int*)(b->base + I.cand_site_off);
        p.cand_sel = (int*)(b->base + I.cand_sel_off);
        p.ds_field = b->base + I.field_off;
        b->hp.push_back(p);
        const int tx = (c->nx + kBlockX - 1) / kBlockX, ty = (c->ny + kBlockY - 1) / kBlockY;
        for (int yy = 0; yy < ty; ++yy)
            for (int xx = 0; xx < tx; ++xx) work[c->collision].push_back(make_int4(i, xx, yy, 0));
        if (c->collision == LBM_EHRENFEST || c->collision == LBM_MEDIAN) ids[c->collision].push_back(i);
    }
    cudaError_t e = cudaMemcpy(b->d_params, b->hp.data(), n * sizeof(Params), cudaMemcpyHostToDevice);
    for (int k = 0; k < kKinds && e == cudaSuccess; ++k) {
        if (!work[k].empty())
            e = cudaMemcpy(b->d_work[k], work[k].data(), work[k].size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !ids[k].empty())
            e = cudaMemcpy(b->d_ids[k], ids[k].data(), ids[k].size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaMemset(b->hp[i].counters, 0, 256);
    if (e != cudaSuccess || build_graph(b) != LBM_OK) {
        delete b;
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) { delete b; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "batch is NULL"; }

lbm_status lbm_batch_set_state(lbm_batch* b, int instance, const void* f, int dtype, void* stream) {
    if (!b || instance < 0 || instance >= (int)b->cfg.size() || !f ||
        (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32))
        return LBM_ERR_ARG;
    if (b->parity != 0) return bfail(b, LBM_ERR_STATE, "set_state needs an even step count");
    const Params& p = b->hp[instance];
    BCK(b, cudaMemsetAsync(p.counters, 0, 256, (cudaStream_t)stream));
    BCK(b, with_format(b->precision, [&](auto LL, auto) {
            return decltype(LL)::set_state(9, p, f, dtype, (cudaStream_t)stream);
        }));
    return LBM_OK;
}

lbm_status lbm_batch_init_uniform(lbm_batch* b, double rho, double ux, double uy, void* stream) {
    if (!b || !(rho > 0.0)) return LBM_ERR_ARG;
    for (size_t i = 0; i < b->cfg.size(); ++i) {
        const Params& p = b->hp[i];
        BCK(b, cudaMemsetAsync(p.counters, 0, 256, (cudaStream_t)stream));
        BCK(b, with_format(b->precision, [&](auto LL, auto) {
                return decltype(LL)::init_uniform(9, p, rho, ux, uy, p.eq, (cudaStream_t)stream);
            }));
    }
    b->parity = 0;
    b->t = 0;
    return LBM_OK;
}

lbm_status lbm_batch_get_state(lbm_batch* b, int instance, void* f, int dtype, void* stream) {
    if (!b || instance < 0 || instance >= (int)b->cfg.size() || !f ||
        (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32))
        return LBM_ERR_ARG;
    const Params& p = b->hp[instance];
    BCK(b, with_format(b->precision, [&](auto LL, auto) {
            return decltype(LL)::get_state(9, p, f, dtype, b->parity != 0, (cudaStream_t)stream);
        }));
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps, int* status, void* stream) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t same[kKinds];
    std::fill(same, same + kKinds, s);
    int k = 0;
    if (nsteps > 0 && b->parity == 1) {  // realign to the graph's even start
        BCK(b, enqueue_step(b, true, (int)(b->t & 1), same));
        b->parity = 0;
        b->t += 1;
        k = 1;
    }
    // parity == t & 1 always, so here t is even: the graph's counter slots 0, 1
    for (; k + 2 <= nsteps; k += 2) {
        BCK(b, cudaGraphLaunch(b->exec, s));
        b->t += 2;
    }
    if (k < nsteps) {
        BCK(b, enqueue_step(b, false, (int)(b->t & 1), same));
        b->parity = 1;
        b->t += 1;
    }
    if (status) {
        const int n = (int)b->cfg.size();
        batch_flags_kernel<<<(n + 255) / 256, 256, 0, s>>>(b->d_params, n, b->d_flags);
        BCK(b, cudaGetLastError());
        std::vector<unsigned> fl(n);
        BCK(b, cudaMemcpyAsync(fl.data(), b->d_flags, n * 4, cudaMemcpyDeviceToHost, s));
        BCK(b, cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) status[i] = fl[i] ? LBM_ERR_DIVERGED : LBM_OK;
    }
    return LBM_OK;
}

lbm_status lbm_batch_stats(lbm_batch* b, int instance, lbm_stats* out, void* stream) {
    if (!b || !out || instance < 0 || instance >= (int)b->cfg.size()) return LBM_ERR_ARG;
    unsigned cnt[CNT_WORDS];
    unsigned long long st[ST_WORDS];
    const Params& p = b->hp[instance];
    BCK(b, cudaMemcpyAsync(cnt, p.counters, sizeof cnt, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    BCK(b, cudaMemcpyAsync(st, p.stats, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    BCK(b, cudaStreamSynchronize((cudaStream_t)stream));
    std::memset(out, 0, sizeof *out);
    const int coll = b->cfg[instance].collision;
    out->steps = b->t;
    out->candidates_last = (coll == LBM_EHRENFEST || coll == LBM_MEDIAN) && b->t ? cnt[CNT_NVALID] : 0;
    out->limited_total = st[ST_LIMITED];
    out->elbm_solved = st[ST_ELBM_SOLVED];
    out->elbm_skipped = st[ST_ELBM_SKIPPED];
    out->elbm_fallbacks = st[ST_ELBM_FALLBACK];
    out->elbm_iters_total = st[ST_ELBM_ITERS];
    out->elbm_iters_max = st[ST_ELBM_ITERS_MAX];
    out->diverged = cnt[CNT_DIVERGED];
    out->overflow = cnt[CNT_OVERFLOW];
    out->screened_last = (b->t > 0 && (coll == LBM_EHRENFEST || coll == LBM_MEDIAN)) ? cnt[(b->t - 1) & 1] : 0;
    return LBM_OK;
}

}  // extern "C"
