// Reverse-mode gradient of a functional of the state after T steps
// (declared in include/lbm.h): checkpoints every K steps in the forward pass,
// and in the backward pass, segment by segment from the last, recomputation
// of the K states and of each step's branch per site (Ehrenfest selection,
// median window site, positivity binding population) followed by K adjoint
// steps (lbm_adjoint_kernels.cuh).  All buffers live in the caller's work
// memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "lbm.h"
#include "lbm_adjoint_kernels.cuh"
#include "lbm_ctx.h"

using namespace lbm;

namespace {

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct AdjLayout {
    size_t acc, fT, lam0, lam1, aux, wbuf, seg, ckpt, total, dense;
    int nseg;
};

bool adj_supported(const lbm_config* c) {
    return (c->collision == LBM_LBGK || c->collision == LBM_EHRENFEST || c->collision == LBM_MEDIAN ||
            c->collision == LBM_POSITIVITY) &&
           c->bc != LBM_BC_DIFFUSIVE;
}

// collisions whose branch per site and step is recorded
bool has_branches(int coll) { return coll == LBM_EHRENFEST || coll == LBM_MEDIAN || coll == LBM_POSITIVITY; }

AdjLayout adj_layout(const lbm_config* c, int T, int K) {
    AdjLayout L;
    const int Q = c->lattice == LBM_D1Q3 ? 3 : 9;
    const size_t N = (size_t)c->nx * c->ny;
    const size_t tb = c->precision == LBM_FP64 ? 8 : 4;
    L.dense = up256((size_t)Q * N * tb);
    L.nseg = T > 0 ? (T + K - 1) / K : 0;
    size_t off = 0;
    L.acc = off;
    off += 256;
    L.fT = off;
    off += L.dense;
    L.lam0 = off;
    off += L.dense;
    L.lam1 = off;
    off += L.dense;
    L.aux = off;
    off += has_branches(c->collision) ? up256((size_t)K * N * sizeof(int)) : 0;
    L.wbuf = off;
    off += c->collision == LBM_MEDIAN ? up256(N * sizeof(double)) : 0;
    L.seg = off;
    off += (size_t)K * L.dense;
    L.ckpt = off;
    off += (size_t)L.nseg * L.dense;
    L.total = off;
    return L;
}

lbm_status afail(lbm_ctx* ctx, lbm_status s, const char* m) {
    ctx->err = m;
    return s;
}

#define ACK(ctx, expr)                                                       \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            ctx->err = std::string(#expr) + ": " + cudaGetErrorName(e_);     \
            return LBM_ERR_CUDA;                                             \
        }                                                                    \
    } while (0)

#define AST(expr)                          \
    do {                                   \
        lbm_status s_ = (expr);            \
        if (s_ != LBM_OK) return s_;       \
    } while (0)

AdjGeo geometry(const lbm_ctx* ctx) {
    AdjGeo g;
    g.nx = ctx->cfg.nx;
    g.ny = ctx->cfg.ny;
    g.periodic_x = ctx->p.periodic_x;
    g.periodic_y = ctx->p.periodic_y;
    g.eq = ctx->cfg.equilibrium;
    g.beta = ctx->p.beta;
    return g;
}

int dtype_of(const lbm_ctx* ctx) { return ctx->cfg.precision == LBM_FP64 ? LBM_DTYPE_F64 : LBM_DTYPE_F32; }

lbm_status check(lbm_ctx* ctx, int T, int K, void* work, size_t bytes) {
    if (!ctx) return LBM_ERR_ARG;
    if (T < 0 || K < 1 || !work || ((uintptr_t)work % 256) != 0)
        return afail(ctx, LBM_ERR_ARG, "adjoint: T >= 0, K >= 1 and 256-byte aligned work needed");
    if (!adj_supported(&ctx->cfg))
        return afail(ctx, LBM_ERR_ARG,
                     "adjoint: collision must be LBM_LBGK, LBM_EHRENFEST, LBM_MEDIAN or LBM_POSITIVITY "
                     "(and no diffusive walls)");
    if (bytes < adj_layout(&ctx->cfg, T, K).total) return afail(ctx, LBM_ERR_OOM, "adjoint: work too small");
    return LBM_OK;
}

template <class T>
lbm_status backward_t(lbm_ctx* ctx, int T_, int K, const void* seed, int seed_dtype, void* dJ_df0,
                      int out_dtype, double* dU, double* dB, char* w, cudaStream_t s) {
    const AdjLayout L = adj_layout(&ctx->cfg, T_, K);
    const int Q = ctx->Q;
    const int64_t N = (int64_t)ctx->cfg.nx * ctx->cfg.ny;
    const AdjGeo g = geometry(ctx);
    double* acc = (double*)(w + L.acc);
    T* fT = (T*)(w + L.fT);
    T* lam[2] = {(T*)(w + L.lam0), (T*)(w + L.lam1)};
    int* aux = (int*)(w + L.aux);
    double* wbuf = (double*)(w + L.wbuf);
    const int coll = ctx->cfg.collision;
    const bool branches = has_branches(coll);
    ACK(ctx, cudaMemsetAsync(acc, 0, 256, s));
    if (!seed) {
        ACK(ctx, AdjLaunch<T>::seed(Q, g, fT, lam[0], acc + 2, s));
    } else if (seed_dtype == LBM_DTYPE_F64) {
        ACK(ctx, AdjLaunch<double>::convert((const double*)seed, lam[0], Q * N, s));
    } else {
        ACK(ctx, AdjLaunch<float>::convert((const float*)seed, lam[0], Q * N, s));
    }
    // One segment: the recomputation of its len pre-collision states and
    // branches from the context's state (just set from the checkpoint:
    // t = 0, even parity), then len adjoint steps from lambda buffer c0.
    auto enqueue_segment = [&](int len, int c0, cudaStream_t st) -> lbm_status {
        if (branches) ACK(ctx, cudaMemsetAsync(aux, 0xff, (size_t)len * N * sizeof(int), st));  // AUX_LBGK
        for (int k = 0; k < len; ++k) {
            const T* fk = (const T*)(w + L.seg + (size_t)k * L.dense);
            AST(lbm_get_state(ctx, (void*)fk, dtype_of(ctx), st));
            AST(lbm_step(ctx, 1, st));
            if (branches)
                ACK(ctx, AdjLaunch<T>::record(Q, ctx->p, coll, (int)((ctx->t - 1) & 1), fk, aux + (size_t)k * N,
                                              ctx->nsm, st));
        }
        int c = c0;
        for (int k = len - 1; k >= 0; --k) {
            ACK(ctx, AdjLaunch<T>::step(Q, g, (const T*)(w + L.seg + (size_t)k * L.dense),
                                        branches ? aux + (size_t)k * N : nullptr, lam[c], lam[c ^ 1], acc, wbuf,
                                        coll == LBM_MEDIAN, st));
            c ^= 1;
        }
        return LBM_OK;
    };
    // Full segments replay a graph of that sequence (about 5 K kernels of a
    // few microseconds each, where separate launches would set the pace),
    // captured on a private stream once per starting lambda buffer; every
    // segment starts from t = 0, so the captured kernels (parities, counter
    // slots) are those of every full segment.  Without a graph (capture not
    // possible) the kernels are launched one by one.
    struct Execs {
        cudaGraphExec_t e[2] = {nullptr, nullptr};
        ~Execs() {
            for (auto x : e)
                if (x) cudaGraphExecDestroy(x);
        }
    } seg_exec;
    auto capture_segment = [&](int c0) -> cudaGraphExec_t {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        cudaGraphExec_t exec = nullptr;
        const uint64_t t0 = ctx->t;
        const int par0 = ctx->parity;
        ctx->t = 0;
        ctx->parity = 0;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const lbm_status st = enqueue_segment(K, c0, cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (st == LBM_OK && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();  // a failed capture leaves the direct launches
        cudaStreamDestroy(cap);
        ctx->t = t0;
        ctx->parity = par0;
        return exec;
    };
    int cur = 0;
    for (int sg = L.nseg - 1; sg >= 0; --sg) {
        const int len = std::min(K, T_ - sg * K);
        AST(lbm_set_state(ctx, w + L.ckpt + (size_t)sg * L.dense, dtype_of(ctx), s));
        cudaGraphExec_t exec = nullptr;
        if (len == K && K > 1) {
            if (!seg_exec.e[cur]) seg_exec.e[cur] = capture_segment(cur);
            exec = seg_exec.e[cur];
        }
        if (exec) {
            ACK(ctx, cudaGraphLaunch(exec, s));
            ctx->t = len;
            ctx->parity = len & 1;
        } else {
            AST(enqueue_segment(len, cur, s));
        }
        if (len & 1) cur ^= 1;
    }
    // the context ends where the forward pass left it
    AST(lbm_set_state(ctx, fT, dtype_of(ctx), s));
    if (dJ_df0) {
        if (out_dtype == LBM_DTYPE_F64)
            ACK(ctx, AdjLaunch<T>::convert(lam[cur], (double*)dJ_df0, Q * N, s));
        else
            ACK(ctx, AdjLaunch<T>::convert(lam[cur], (float*)dJ_df0, Q * N, s));
    }
    double h[2];
    ACK(ctx, cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, s));
    ACK(ctx, cudaStreamSynchronize(s));
    if (dU) *dU = h[0];
    if (dB) *dB = h[1];
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint_required_bytes(const lbm_config* cfg, int T, int K, size_t* bytes) {
    size_t dummy;
    if (!bytes || !cfg || T < 0 || K < 1 || lbm_required_bytes(cfg, &dummy) != LBM_OK || !adj_supported(cfg))
        return LBM_ERR_ARG;
    *bytes = adj_layout(cfg, T, K).total;
    return LBM_OK;
}

lbm_status lbm_adjoint_forward(lbm_ctx* ctx, int T, int K, void* work, size_t work_bytes, double* J_host,
                               void* stream) {
    AST(check(ctx, T, K, work, work_bytes));
    if (ctx->parity != 0) return afail(ctx, LBM_ERR_STATE, "adjoint: start from an even step count");
    const AdjLayout L = adj_layout(&ctx->cfg, T, K);
    char* w = (char*)work;
    cudaStream_t s = (cudaStream_t)stream;
    for (int sg = 0; sg < L.nseg; ++sg) {
        AST(lbm_get_state(ctx, w + L.ckpt + (size_t)sg * L.dense, dtype_of(ctx), s));
        AST(lbm_step(ctx, std::min(K, T - sg * K), s));
    }
    AST(lbm_get_state(ctx, w + L.fT, dtype_of(ctx), s));
    if (J_host) {
        double* acc = (double*)(w + L.acc);
        const AdjGeo g = geometry(ctx);
        ACK(ctx, cudaMemsetAsync(acc, 0, 256, s));
        // the seed kernel also sums J; its lambda output is scratch here
        if (ctx->cfg.precision == LBM_FP64)
            ACK(ctx, AdjLaunch<double>::seed(ctx->Q, g, (const double*)(w + L.fT), (double*)(w + L.lam0), acc + 2, s));
        else
            ACK(ctx, AdjLaunch<float>::seed(ctx->Q, g, (const float*)(w + L.fT), (float*)(w + L.lam0), acc + 2, s));
        ACK(ctx, cudaMemcpyAsync(J_host, acc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
        ACK(ctx, cudaStreamSynchronize(s));
    }
    return LBM_OK;
}

lbm_status lbm_adjoint_backward(lbm_ctx* ctx, int T, int K, const void* seed, int seed_dtype, void* dJ_df0,
                                int out_dtype, double* dJ_dU, double* dJ_dbeta, void* work, size_t work_bytes,
                                void* stream) {
    AST(check(ctx, T, K, work, work_bytes));
    if ((seed && seed_dtype != LBM_DTYPE_F64 && seed_dtype != LBM_DTYPE_F32) ||
        (dJ_df0 && out_dtype != LBM_DTYPE_F64 && out_dtype != LBM_DTYPE_F32))
        return afail(ctx, LBM_ERR_ARG, "adjoint: dtype must be LBM_DTYPE_F64 or LBM_DTYPE_F32");
    if (ctx->cfg.precision == LBM_FP64)
        return backward_t<double>(ctx, T, K, seed, seed_dtype, dJ_df0, out_dtype, dJ_dU, dJ_dbeta, (char*)work,
                                  (cudaStream_t)stream);
    return backward_t<float>(ctx, T, K, seed, seed_dtype, dJ_df0, out_dtype, dJ_dU, dJ_dbeta, (char*)work,
                             (cudaStream_t)stream);
}

}  // extern "C"
