// Batched form of the step (declared in include/lbm.h): many independent
// lattices - D2Q9 cavities, channels and periodic boxes and D1Q3 tubes of
// different sizes, parameters and collisions, one storage format - advanced
// by persistent kernels (lbm_batch_kernels.cuh).  Work queues of
// (instance, tiles) items: queue 0 holds the instances of the streaming
// collisions (LBGK, positivity, MRT), queue 1 the ELBM instances, queue 2 the
// limiters (Ehrenfest, median), queue 3 + k the instances of collision k
// alone (used to time one collision group).  A launch runs a queue for a
// number of steps; the three main queues run on parallel stream branches,
// captured once into a CUDA graph that lbm_batch_step replays.
// No device allocation: the caller's block holds populations, scratch,
// descriptors, queues and the per-instance step generations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_batch_kernels.cuh"
#include "lbm_setup.h"

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

constexpr int kKinds = 6;             // LBM_LBGK .. LBM_MRT
constexpr int kMain = 3;              // streaming, ELBM, limiters
constexpr int kQueues = kMain + kKinds;

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// The kernel (collision set) of collision `coll`.
int set_of(int coll) {
    return coll == LBM_ELBM ? kSetHeavy : ((coll == LBM_EHRENFEST || coll == LBM_MEDIAN) ? kSetLimiter : kSetStream);
}

// The main queue of collision `coll`'s items.
int main_queue(int coll) {
    const int k = set_of(coll);
    return k == kSetStream ? 0 : (k == kSetHeavy ? 1 : 2);
}

int queue_set(int q) {
    if (q < kMain) return q == 0 ? kSetStream : (q == 1 ? kSetHeavy : kSetLimiter);
    return set_of(q - kMain);
}

// Per-instance divergence flags gathered into one array.
__global__ void batch_flags_kernel(const Params* __restrict__ insts, int n, unsigned* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = insts[i].counters[CNT_DIVERGED];
}

// Resets the queues' step base to `base` (the steps every instance has
// completed) before a launch sequence.
__global__ void batch_set_base(BatchSync* s, int nq, unsigned base) {
    const int q = threadIdx.x;
    if (q < nq) {
        s[q].base = base;
        s[q].head = 0ull;
        s[q].exit = 0u;
    }
}

const char* check_opts(const lbm_batch_opts* o) {
    if (!o) return "opts is NULL";
    if (o->tile_x != 16 && o->tile_x != 32 && o->tile_x != 64 && o->tile_x != 128 && o->tile_x != 256)
        return "tile_x must be 16, 32, 64, 128 or 256";
    if (o->ctas_per_sm < 0 || o->ctas_per_sm > 64) return "ctas_per_sm must be in [0, 64]";
    if (o->chunk < 1 || o->chunk > 1024) return "chunk must be in [1, 1024]";
    if (o->order != LBM_BATCH_ORDER_INSTANCE && o->order != LBM_BATCH_ORDER_INTERLEAVED) return "unknown order";
    if (o->graph_steps < 1 || o->graph_steps > 4096) return "graph_steps must be in [1, 4096]";
    if (o->tile_rows < 1 || o->tile_rows > 64) return "tile_rows must be in [1, 64]";
    if (!(o->wait_ms > 0.0) || !std::isfinite(o->wait_ms)) return "wait_ms must be > 0";
    return nullptr;
}

const char* check_batch(const lbm_config* cfgs, int n) {
    if (!cfgs || n < 1) return "need at least one instance";
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        if (const char* e = check_config(c)) return e;
        if (c->precision != cfgs[0].precision) return "all instances share one precision";
        if (c->collision < LBM_LBGK || c->collision > LBM_MRT) return "batched collisions are LBGK ... MRT";
        if (c->lattice == LBM_D2Q9 && c->bc != LBM_BC_CAVITY && c->bc != LBM_BC_PERIODIC && c->bc != LBM_BC_CHANNEL)
            return "a batched D2Q9 instance is a cavity, a channel or periodic";
        if (c->lattice == LBM_D1Q3 && c->bc != LBM_BC_ENDS && c->bc != LBM_BC_PERIODIC)
            return "a batched D1Q3 instance is a tube (ends) or periodic";
    }
    return nullptr;
}

int log2i(int v) {
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

// Work items of one instance per step: rows tiles each.
int items_of(const lbm_config* c, const lbm_batch_opts& o) {
    if (c->lattice == LBM_D1Q3) {
        const int span = kBatchThreads * o.tile_rows;
        return (c->nx + span - 1) / span;
    }
    const int band = (kBatchThreads / o.tile_x) * o.tile_rows;
    return ((c->nx + o.tile_x - 1) / o.tile_x) * ((c->ny + band - 1) / band);
}

struct InstLayout {
    size_t f_off, cnt_off, cand_f_off, cand_ds_off, cand_site_off, cand_sel_off, field_off;
    int Q, pitch, cap, tiles;
    int64_t plane;
};

struct BatchLayout {
    std::vector<InstLayout> inst;
    size_t params_off, items_off[kQueues], sync_off, gen_off, done_off, ntiles_off, flags_off, total;
    int nitems[kQueues];
};

bool in_queue(int q, int coll) { return q < kMain ? main_queue(coll) == q : coll == q - kMain; }

BatchLayout make_layout(const lbm_config* cfgs, int n, const lbm_batch_opts& o) {
    BatchLayout B;
    const int prec = cfgs[0].precision;
    const size_t sb = prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2);
    const size_t tb = prec == LBM_FP64 ? 8 : 4;
    size_t off = 0;
    std::fill(B.nitems, B.nitems + kQueues, 0);
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        InstLayout L;
        L.Q = c->lattice == LBM_D1Q3 ? 3 : 9;
        L.pitch = (c->nx + 31) / 32 * 32;
        L.plane = (int64_t)c->ny * L.pitch;
        const size_t N = (size_t)c->nx * c->ny;
        const bool lim = c->collision == LBM_EHRENFEST || c->collision == LBM_MEDIAN;
        L.cap = lim ? (int)N : 0;
        L.tiles = items_of(c, o);
        L.f_off = off;
        off += up256((size_t)L.Q * (size_t)L.plane * sb);
        L.cnt_off = off;
        off += 256;
        L.cand_f_off = off;
        off += up256((size_t)L.cap * L.Q * tb);
        L.cand_ds_off = off;
        off += up256((size_t)L.cap * 8);
        L.cand_site_off = off;
        off += up256((size_t)L.cap * 4);
        L.cand_sel_off = off;
        off += up256((size_t)L.cap * 4);
        L.field_off = off;
        off += c->collision == LBM_MEDIAN ? up256(N * tb) : 0;
        B.inst.push_back(L);
        for (int q = 0; q < kQueues; ++q)
            if (in_queue(q, c->collision)) B.nitems[q] += L.tiles;
    }
    B.params_off = off;
    off += up256((size_t)n * sizeof(Params));
    for (int q = 0; q < kQueues; ++q) {
        B.items_off[q] = off;
        off += up256((size_t)B.nitems[q] * sizeof(BatchItem));
    }
    B.sync_off = off;
    off += up256(kQueues * sizeof(BatchSync));
    B.gen_off = off;
    off += up256((size_t)n * 4);
    B.done_off = off;
    off += up256((size_t)n * 4);
    B.ntiles_off = off;
    off += up256((size_t)n * 4);
    B.flags_off = off;
    off += up256((size_t)n * 4);
    B.total = off;
    return B;
}

// One step's items of queue q, in the claim order the options ask for.
std::vector<BatchItem> queue_items(const lbm_config* cfgs, int n, const BatchLayout& B, const lbm_batch_opts& o,
                                   int q) {
    std::vector<BatchItem> out;
    auto item = [&](int i, int t) {
        const lbm_config* c = cfgs + i;
        BatchItem it;
        it.inst = i;
        it.code = (c->collision << 4) | B.inst[i].Q;
        if (B.inst[i].Q == 3) {
            it.x0 = t * kBatchThreads * o.tile_rows;
            it.y0 = 0;
        } else {
            const int ntx = (c->nx + o.tile_x - 1) / o.tile_x;
            it.x0 = (t % ntx) * o.tile_x;
            it.y0 = (t / ntx) * (kBatchThreads / o.tile_x) * o.tile_rows;
        }
        return it;
    };
    if (o.order == LBM_BATCH_ORDER_INSTANCE) {
        for (int i = 0; i < n; ++i)
            if (in_queue(q, cfgs[i].collision))
                for (int t = 0; t < B.inst[i].tiles; ++t) out.push_back(item(i, t));
    } else {
        int most = 0;
        for (int i = 0; i < n; ++i)
            if (in_queue(q, cfgs[i].collision)) most = std::max(most, B.inst[i].tiles);
        for (int t = 0; t < most; ++t)
            for (int i = 0; i < n; ++i)
                if (in_queue(q, cfgs[i].collision) && t < B.inst[i].tiles) out.push_back(item(i, t));
    }
    return out;
}

lbm_batch_opts default_opts() {
    lbm_batch_opts o;
    std::memset(&o, 0, sizeof o);
    o.tile_x = 128;
    o.ctas_per_sm = 0;
    o.chunk = 4;
    o.order = LBM_BATCH_ORDER_INSTANCE;
    o.graph_steps = 16;
    o.wait_ms = 1000.0;
    o.tile_rows = 4;
    return o;
}

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

}  // namespace

struct lbm_batch {
    std::vector<lbm_config> cfg;
    std::vector<Params> hp;  // host copies of the instance descriptors
    lbm_batch_opts opts;
    BatchLayout L;
    char* base = nullptr;
    Params* d_params = nullptr;
    BatchItem* d_items[kQueues] = {};
    BatchSync* d_sync = nullptr;
    unsigned* d_gen = nullptr;
    unsigned* d_done = nullptr;
    int* d_ntiles = nullptr;
    unsigned* d_flags = nullptr;
    int grid[3] = {0, 0, 0};  // CTAs of the kernel of each collision set (kSet*)
    int precision = LBM_FP32;
    int parity = 0;
    uint64_t t = 0;
    cudaStream_t s_cap = nullptr;
    cudaStream_t s_branch[kMain] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMain] = {}, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
    ~lbm_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (int k = 0; k < kMain; ++k) {
            if (s_branch[k]) cudaStreamDestroy(s_branch[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_t0) cudaEventDestroy(ev_t0);
        if (ev_t1) cudaEventDestroy(ev_t1);
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

#define BCK(b, expr)                                       \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return bcuda(b, e_, #expr); \
    } while (0)

BatchArgs make_args(const lbm_batch* b, int q, int steps) {
    BatchArgs a;
    a.insts = b->d_params;
    a.items = b->d_items[q];
    a.nitems = b->L.nitems[q];
    a.steps = steps;
    a.sync = b->d_sync + q;
    a.gen = b->d_gen;
    a.done = b->d_done;
    a.ntiles = b->d_ntiles;
    a.tile_log2x = log2i(b->opts.tile_x);
    a.rows = b->opts.tile_rows;
    a.chunk = b->opts.chunk;
    a.wait_ns = (unsigned long long)(b->opts.wait_ms * 1e6);
    return a;
}

cudaError_t launch_queue(lbm_batch* b, int q, int steps, cudaStream_t s) {
    if (b->L.nitems[q] == 0 || steps <= 0) return cudaSuccess;
    const int set = queue_set(q);
    const BatchArgs a = make_args(b, q, steps);
    const int grid = b->grid[set];
    return with_format(b->precision, [&](auto, auto BL) { return decltype(BL)::persistent(set, a, grid, s); });
}

// `steps` steps of every instance: the main queues on parallel branches
// forked from and joined back into s.
cudaError_t enqueue_steps(lbm_batch* b, int steps, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->ev_fork, s);
    for (int q = 0; q < kMain && e == cudaSuccess; ++q) {
        if (!b->L.nitems[q]) continue;
        e = cudaStreamWaitEvent(b->s_branch[q], b->ev_fork, 0);
        if (e == cudaSuccess) e = launch_queue(b, q, steps, b->s_branch[q]);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[q], b->s_branch[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[q], 0);
    }
    return e;
}

lbm_status build_graph(lbm_batch* b) {
    BCK(b, cudaStreamBeginCapture(b->s_cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_steps(b, b->opts.graph_steps, b->s_cap);
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

// Step counters, queues and generations back to step 0.
cudaError_t reset_sync(lbm_batch* b, cudaStream_t s) {
    const int n = (int)b->cfg.size();
    cudaError_t e = cudaMemsetAsync(b->d_sync, 0, kQueues * sizeof(BatchSync), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_gen, 0, (size_t)n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, (size_t)n * 4, s);
    return e;
}

lbm_status create_batch(const lbm_config* cfgs, int n, const lbm_batch_opts& o, void* dev_mem, size_t bytes,
                        lbm_batch** out) {
    BatchLayout L = make_layout(cfgs, n, o);
    if (bytes < L.total) return LBM_ERR_OOM;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->cfg.assign(cfgs, cfgs + n);
    b->opts = o;
    b->L = L;
    b->base = (char*)dev_mem;
    b->precision = cfgs[0].precision;
    b->d_params = (Params*)(b->base + L.params_off);
    for (int q = 0; q < kQueues; ++q) b->d_items[q] = (BatchItem*)(b->base + L.items_off[q]);
    b->d_sync = (BatchSync*)(b->base + L.sync_off);
    b->d_gen = (unsigned*)(b->base + L.gen_off);
    b->d_done = (unsigned*)(b->base + L.done_off);
    b->d_ntiles = (int*)(b->base + L.ntiles_off);
    b->d_flags = (unsigned*)(b->base + L.flags_off);
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete b;
        return LBM_ERR_CUDA;
    }
    std::vector<int> ntiles(n);
    for (int i = 0; i < n; ++i) {
        const lbm_config* c = cfgs + i;
        const InstLayout& I = L.inst[i];
        Params p;
        std::memset(&p, 0, sizeof p);
        fill_params(c, nsm, p);
        p.f = b->base + I.f_off;
        p.plane = I.plane;
        p.plane32 = (int)I.plane;
        p.pitch = I.pitch;
        // ELBM always uses the entropic equilibrium; storing it here makes the
        // uniform initialisation pick the right one
        if (c->collision == LBM_ELBM) p.eq = LBM_EQ_ENTROPIC;
        p.median_inv = 0.0;  // the batched median filter reads the step's Delta S field
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
        ntiles[i] = I.tiles;
    }
    cudaError_t e = cudaMemcpy(b->d_params, b->hp.data(), n * sizeof(Params), cudaMemcpyHostToDevice);
    for (int q = 0; q < kQueues && e == cudaSuccess; ++q) {
        const std::vector<BatchItem> items = queue_items(cfgs, n, L, o, q);
        if (!items.empty())
            e = cudaMemcpy(b->d_items[q], items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ntiles, ntiles.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaMemset(b->hp[i].counters, 0, 256);
    if (e == cudaSuccess) e = reset_sync(b, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    // CTAs of each kernel: as many as fit on an SM, or fewer per the options
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        int per_sm = 0;
        e = with_format(b->precision, [&](auto, auto BL) { return decltype(BL)::occupancy(k, &per_sm); });
        if (per_sm < 1) per_sm = 1;
        if (o.ctas_per_sm > 0) per_sm = std::min(per_sm, o.ctas_per_sm);
        b->grid[k] = per_sm * nsm;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->s_cap, cudaStreamNonBlocking);
    for (int k = 0; k < kMain && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->s_branch[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_t1);
    if (e != cudaSuccess || build_graph(b) != LBM_OK) {
        delete b;
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

// Reads and clears the queues' error flags: LBM_ERR_TIMEOUT if a bounded
// wait ran out since the last check (synchronises s).
lbm_status check_timeouts(lbm_batch* b, cudaStream_t s) {
    BatchSync hs[kQueues];
    BCK(b, cudaMemcpyAsync(hs, b->d_sync, sizeof hs, cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    bool any = false;
    for (int q = 0; q < kQueues; ++q) any |= hs[q].err != 0;
    if (!any) return LBM_OK;
    for (int q = 0; q < kQueues; ++q)
        BCK(b, cudaMemsetAsync(&b->d_sync[q].err, 0, sizeof(unsigned), s));
    BCK(b, cudaStreamSynchronize(s));
    return bfail(b, LBM_ERR_TIMEOUT,
                 "a batched step waited longer than wait_ms for an instance's previous step; "
                 "the states are undefined until lbm_batch_init_uniform or lbm_batch_set_state");
}

}  // namespace

extern "C" {

lbm_status lbm_batch_opts_default(lbm_batch_opts* o) {
    if (!o) return LBM_ERR_ARG;
    *o = default_opts();
    return LBM_OK;
}

lbm_status lbm_batch_required_bytes_ex(const lbm_config* cfgs, int n, const lbm_batch_opts* opts,
                                       size_t* bytes) {
    const lbm_batch_opts o = opts ? *opts : default_opts();
    if (!bytes || check_batch(cfgs, n) || check_opts(&o)) return LBM_ERR_ARG;
    *bytes = make_layout(cfgs, n, o).total;
    return LBM_OK;
}

lbm_status lbm_batch_required_bytes(const lbm_config* cfgs, int n, size_t* bytes) {
    return lbm_batch_required_bytes_ex(cfgs, n, nullptr, bytes);
}

lbm_status lbm_batch_create_ex(const lbm_config* cfgs, int n, const lbm_batch_opts* opts, void* dev_mem,
                               size_t bytes, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    const lbm_batch_opts o = opts ? *opts : default_opts();
    if (check_batch(cfgs, n) || check_opts(&o)) return LBM_ERR_ARG;
    if (!dev_mem || ((uintptr_t)dev_mem % 256) != 0) return LBM_ERR_ARG;
    return create_batch(cfgs, n, o, dev_mem, bytes, out);
}

lbm_status lbm_batch_create(const lbm_config* cfgs, int n, void* dev_mem, size_t bytes, lbm_batch** out) {
    return lbm_batch_create_ex(cfgs, n, nullptr, dev_mem, bytes, out);
}

void lbm_batch_destroy(lbm_batch* b) { delete b; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "batch is NULL"; }

lbm_status lbm_batch_get_opts(const lbm_batch* b, lbm_batch_opts* o) {
    if (!b || !o) return LBM_ERR_ARG;
    *o = b->opts;
    return LBM_OK;
}

lbm_status lbm_batch_set_state(lbm_batch* b, int instance, const void* f, int dtype, void* stream) {
    if (!b || instance < 0 || instance >= (int)b->cfg.size() || !f ||
        (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32))
        return LBM_ERR_ARG;
    if (b->parity != 0) return bfail(b, LBM_ERR_STATE, "set_state needs an even step count");
    const Params& p = b->hp[instance];
    const int Q = b->L.inst[instance].Q;
    BCK(b, cudaMemsetAsync(p.counters, 0, 256, (cudaStream_t)stream));
    BCK(b, with_format(b->precision, [&](auto LL, auto) {
            return decltype(LL)::set_state(Q, p, f, dtype, (cudaStream_t)stream);
        }));
    return LBM_OK;
}

lbm_status lbm_batch_init_uniform(lbm_batch* b, double rho, double ux, double uy, void* stream) {
    if (!b || !(rho > 0.0)) return LBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < b->cfg.size(); ++i) {
        const Params& p = b->hp[i];
        const int Q = b->L.inst[i].Q;
        BCK(b, cudaMemsetAsync(p.counters, 0, 256, s));
        BCK(b, with_format(b->precision, [&](auto LL, auto) {
                return decltype(LL)::init_uniform(Q, p, rho, ux, Q == 9 ? uy : 0.0, p.eq, s);
            }));
    }
    BCK(b, reset_sync(b, s));
    b->parity = 0;
    b->t = 0;
    return LBM_OK;
}

lbm_status lbm_batch_get_state(lbm_batch* b, int instance, void* f, int dtype, void* stream) {
    if (!b || instance < 0 || instance >= (int)b->cfg.size() || !f ||
        (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32))
        return LBM_ERR_ARG;
    const Params& p = b->hp[instance];
    const int Q = b->L.inst[instance].Q;
    BCK(b, with_format(b->precision, [&](auto LL, auto) {
            return decltype(LL)::get_state(Q, p, f, dtype, b->parity != 0, (cudaStream_t)stream);
        }));
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps, int* status, void* stream) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps > 0) {
        // the queues start from the steps every instance has completed; the
        // graph's launches then advance that base themselves
        batch_set_base<<<1, 32, 0, s>>>(b->d_sync, kMain, (unsigned)b->t);
        BCK(b, cudaGetLastError());
        int left = nsteps;
        while (left >= b->opts.graph_steps) {
            BCK(b, cudaGraphLaunch(b->exec, s));
            left -= b->opts.graph_steps;
        }
        if (left) BCK(b, enqueue_steps(b, left, s));
        b->t += (uint64_t)nsteps;
        b->parity = (int)(b->t & 1);
    }
    if (status) {
        const int n = (int)b->cfg.size();
        batch_flags_kernel<<<(n + 255) / 256, 256, 0, s>>>(b->d_params, n, b->d_flags);
        BCK(b, cudaGetLastError());
        std::vector<unsigned> fl(n);
        BCK(b, cudaMemcpyAsync(fl.data(), b->d_flags, n * 4, cudaMemcpyDeviceToHost, s));
        lbm_status st = check_timeouts(b, s);  // synchronises s
        if (st != LBM_OK) return st;
        for (int i = 0; i < n; ++i) status[i] = fl[i] ? LBM_ERR_DIVERGED : LBM_OK;
    }
    return LBM_OK;
}

lbm_status lbm_batch_group_times(lbm_batch* b, int nsteps, double* ms, void* stream) {
    if (!b || nsteps < 1 || !ms) return LBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < kKinds; ++k) {
        ms[k] = 0.0;
        const int q = kMain + k;
        if (!b->L.nitems[q]) continue;
        batch_set_base<<<1, 32, 0, s>>>(b->d_sync + q, 1, (unsigned)b->t);
        BCK(b, cudaGetLastError());
        BCK(b, cudaEventRecord(b->ev_t0, s));
        BCK(b, launch_queue(b, q, nsteps, s));
        BCK(b, cudaEventRecord(b->ev_t1, s));
        BCK(b, cudaEventSynchronize(b->ev_t1));
        float t = 0.f;
        BCK(b, cudaEventElapsedTime(&t, b->ev_t0, b->ev_t1));
        ms[k] = t;
    }
    b->t += (uint64_t)nsteps;
    b->parity = (int)(b->t & 1);
    return check_timeouts(b, s);
}

lbm_status lbm_batch_debug_hold(lbm_batch* b, int instance, void* stream) {
    if (!b || instance < 0 || instance >= (int)b->cfg.size()) return LBM_ERR_ARG;
    if (b->t == 0) return bfail(b, LBM_ERR_STATE, "hold needs at least one step taken");
    const unsigned behind = (unsigned)(b->t - 1);
    BCK(b, cudaMemcpyAsync(b->d_gen + instance, &behind, 4, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    BCK(b, cudaStreamSynchronize((cudaStream_t)stream));
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
    const bool lim = coll == LBM_EHRENFEST || coll == LBM_MEDIAN;
    out->steps = b->t;
    out->candidates_last = lim && b->t ? cnt[CNT_NVALID] : 0;
    out->limited_total = st[ST_LIMITED];
    out->elbm_solved = st[ST_ELBM_SOLVED];
    out->elbm_skipped = st[ST_ELBM_SKIPPED];
    out->elbm_fallbacks = st[ST_ELBM_FALLBACK];
    out->elbm_iters_total = st[ST_ELBM_ITERS];
    out->elbm_iters_max = st[ST_ELBM_ITERS_MAX];
    out->diverged = cnt[CNT_DIVERGED];
    out->overflow = cnt[CNT_OVERFLOW];
    out->screened_last = (b->t > 0 && lim) ? cnt[(b->t - 1) & 1] : 0;
    return LBM_OK;
}

lbm_status lbm_batch_tune_bytes(const lbm_config* cfgs, int n, size_t* bytes) {
    if (!bytes || check_batch(cfgs, n)) return LBM_ERR_ARG;
    size_t most = 0;  // over every tile shape the tuner tries
    for (int tx : {16, 32, 64, 128, 256})
        for (int rows : {1, 2, 4, 8, 16}) {
            lbm_batch_opts o = default_opts();
            o.tile_x = tx;
            o.tile_rows = rows;
            most = std::max(most, make_layout(cfgs, n, o).total);
        }
    *bytes = most;
    return LBM_OK;
}

lbm_status lbm_batch_tune(const lbm_config* cfgs, int n, void* dev_mem, size_t bytes, int steps,
                          lbm_batch_opts* best, lbm_batch_tune_record* records, int cap, int* nrec,
                          double* best_ms, void* stream) {  // best_ms: the objective
    if (!best || steps < 1 || check_batch(cfgs, n) || check_opts(best)) return LBM_ERR_ARG;
    if (!dev_mem || ((uintptr_t)dev_mem % 256) != 0) return LBM_ERR_ARG;
    size_t need = 0;
    if (lbm_batch_tune_bytes(cfgs, n, &need) != LBM_OK) return LBM_ERR_ARG;
    if (bytes < need) return LBM_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    int count = 0;
    // one candidate: a batch over dev_mem at rest, two steps of warm-up, then
    // `steps` steps of each collision group alone, timed with CUDA events on
    // s.  The objective is the mean over the groups of each group's time
    // relative to its time with the starting options: every group weighs
    // alike (the summed time would be set by the slowest group, ELBM, whose
    // FP64 work the launch shape barely changes)
    double g0[kKinds] = {0.0};
    auto time_opts = [&](const lbm_batch_opts& o, double* obj) -> lbm_status {
        lbm_batch* b = nullptr;
        lbm_status st = create_batch(cfgs, n, o, dev_mem, bytes, &b);
        if (st != LBM_OK) return st;
        double g[kKinds] = {0.0};
        st = lbm_batch_init_uniform(b, 1.0, 0.0, 0.0, s);
        if (st == LBM_OK) st = lbm_batch_step(b, 2, nullptr, s);
        if (st == LBM_OK) st = lbm_batch_group_times(b, steps, g, s);
        delete b;
        if (st != LBM_OK) return st;
        if (count == 0)
            for (int k = 0; k < kKinds; ++k) g0[k] = g[k];
        double sum = 0.0, rel = 0.0;
        int groups = 0;
        for (int k = 0; k < kKinds; ++k) {
            sum += g[k];
            if (g0[k] > 0.0) {
                rel += g[k] / g0[k];
                ++groups;
            }
        }
        *obj = groups ? rel / groups : 0.0;
        if (records && count < cap) {
            records[count].opts = o;
            records[count].ms_per_step = sum / steps;
            records[count].objective = *obj;
        }
        ++count;
        return LBM_OK;
    };
    // one knob at a time, each from the best so far: tile shape, tiles per
    // item, CTAs per SM, items per queue access, claim order
    lbm_batch_opts cur = *best;
    double cur_obj = 0.0;
    lbm_status st = time_opts(cur, &cur_obj);
    if (st != LBM_OK) return st;
    auto sweep = [&](auto set, std::initializer_list<int> values) -> lbm_status {
        for (int v : values) {
            lbm_batch_opts o = cur;
            set(o, v);
            if (std::memcmp(&o, &cur, sizeof o) == 0) continue;
            double obj = 0.0;
            lbm_status r = time_opts(o, &obj);
            if (r != LBM_OK) return r;
            if (obj < cur_obj) {
                cur = o;
                cur_obj = obj;
            }
        }
        return LBM_OK;
    };
    if ((st = sweep([](lbm_batch_opts& o, int v) { o.tile_x = v; }, {32, 64, 128, 256})) != LBM_OK) return st;
    if ((st = sweep([](lbm_batch_opts& o, int v) { o.tile_rows = v; }, {1, 2, 4, 8, 16})) != LBM_OK) return st;
    if ((st = sweep([](lbm_batch_opts& o, int v) { o.ctas_per_sm = v; }, {0, 6, 4, 2})) != LBM_OK) return st;
    if ((st = sweep([](lbm_batch_opts& o, int v) { o.chunk = v; }, {1, 4, 16})) != LBM_OK) return st;
    if ((st = sweep([](lbm_batch_opts& o, int v) { o.order = v; },
                    {LBM_BATCH_ORDER_INSTANCE, LBM_BATCH_ORDER_INTERLEAVED})) != LBM_OK)
        return st;
    *best = cur;
    if (best_ms) *best_ms = cur_obj;
    if (nrec) *nrec = count;
    return LBM_OK;
}

}  // extern "C"
