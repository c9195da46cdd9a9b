// Batched form: many independent lattices (instances: D2Q9 cavities,
// channels and periodic boxes, D1Q3 tubes; one storage format) advanced by
// persistent kernels.  One launch covers `steps` steps of every instance of
// its group: its CTAs claim work items - (step, instance, tile) in step order
// - from a device queue until it is drained.  An item waits until its
// instance has completed the previous step (a per-instance step generation),
// so instances advance independently, without a grid-wide barrier between
// steps; the CTA that completes an instance's last tile of a step runs that
// instance's limiter fix-up (Ehrenfest selection, median filter) and then
// publishes the step.  Waits are bounded (a limit in nanoseconds of the GPU's
// global timer): a wait that runs out sets the group's error flag, every CTA
// stops claiming and the host reports LBM_ERR_TIMEOUT.
//
// Progress does not depend on the CTAs being resident at the same time: an
// item only ever waits for items of earlier steps, which running CTAs have
// already claimed, so the oldest unfinished item can always proceed.
//
// Three kernels per storage format, each on its own stream branch: the
// streaming collisions (LBGK, positivity, MRT: no fix-up, few registers,
// many resident CTAs), the limiters (Ehrenfest, median: their fix-ups in
// the kernel) and ELBM (its FP64 root finder needs far more registers).
// A work item is `rows` tiles of one instance (tile_x x 256 / tile_x sites,
// one per thread, for D2Q9; 256 sites of the line for D1Q3): a CTA that
// stays on one instance and step keeps its parameters and skips the wait.
//
// These kernels are compiled in units whose global loads default to the
// L2-coherent cache-global mode: within one launch a CTA reads populations
// and candidate records that CTAs on other SMs wrote in an earlier step.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// One tile of one instance: origin (x0, y0) and code = (collision << 4) | Q.
struct BatchItem {
    int inst, x0, y0, code;
};

// Queue state of one kernel (one launch at a time per stream branch).
struct BatchSync {
    unsigned long long head;  // next queue index of this launch
    unsigned exit;            // CTAs of this launch that have finished
    unsigned err;             // 1: a bounded wait ran out
    unsigned base;            // steps completed by the earlier launches
    unsigned pad[3];
};

struct BatchArgs {
    const Params* insts;
    const BatchItem* items;  // the items of one step, in claim order
    int nitems, steps;
    BatchSync* sync;
    unsigned* gen;     // per instance: steps completed
    unsigned* done;    // per instance: tiles of its current step completed
    const int* ntiles; // per instance: items per step
    int tile_log2x;    // D2Q9 tiles are 2^tile_log2x x (256 >> tile_log2x) sites
    int rows;          // tiles per item (stacked along y; along the line for D1Q3)
    int chunk;         // items claimed per queue access
    unsigned long long wait_ns;  // a bounded wait gives up after this long
};

constexpr int kBatchThreads = 256;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread: waits until *gen >= target.  False when the wait ran out (the
// group's error flag is then set) or another CTA's already had.
__device__ __forceinline__ bool wait_generation(const unsigned* gen, unsigned target, BatchSync* sync,
                                                unsigned long long limit_ns) {
    if (*(const volatile unsigned*)gen >= target) {
        __threadfence();
        return true;
    }
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (*(const volatile unsigned*)gen < target) {
        if (*(volatile unsigned*)&sync->err) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicExch(&sync->err, 1u);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    __threadfence();
    return true;
}

// The item's sites: `rows` tiles, one site per thread in each.
template <int Q, class ST, int COLL>
__device__ __forceinline__ void batch_tile(const Params& sp, const BatchItem& it, int log2x, int rows, bool odd,
                                           int& e_code, int& e_iters) {
    const int tid = threadIdx.x;
    const int th = kBatchThreads >> log2x;  // D2Q9 tile height
    typename ST::T acc = 0;                 // no reduction in the batched collisions
    for (int r = 0; r < rows; ++r) {
        const int x = Q == 9 ? it.x0 + (tid & ((1 << log2x) - 1)) : it.x0 + r * kBatchThreads + tid;
        const int y = Q == 9 ? it.y0 + r * th + (tid >> log2x) : 0;
        if (x < sp.nx && y < sp.ny) {
            if (odd)
                site_update<Q, ST, COLL, true>(sp, x, y, e_code, e_iters, acc);
            else
                site_update<Q, ST, COLL, false>(sp, x, y, e_code, e_iters, acc);
        }
    }
}

// The limiter fix-up of one instance's completed step, by one whole CTA:
// the Ehrenfest step (FP64 Delta S of the screened sites, one 16-lane group
// each, then the k-largest selection) or the median filter (from the Delta S
// field the step wrote).
template <int Q, class ST, int COLL>
__device__ void batch_fixup(const Params& sp, bool odd) {
    if (COLL == LBM_EHRENFEST) {
        __shared__ unsigned s_valid;
        if (threadIdx.x == 0) s_valid = 0;
        __syncthreads();
        unsigned M = sp.counters[sp.cslot];
        if (M > (unsigned)sp.cand_cap) M = (unsigned)sp.cand_cap;
        unsigned n = 0;
        for (unsigned b = 0; b < M; b += kBatchThreads >> 4) {
            const unsigned j = b + (threadIdx.x >> 4);
            const double d = delta_s_group<Q, ST>(sp, j, j < M);
            if (j < M && (threadIdx.x & 15) == 0) {
                const bool c = d > sp.delta;
                sp.cand_ds[j] = c ? d : -1.0;
                n += c;
            }
        }
        if (n) atomicAdd(&s_valid, n);
        __syncthreads();
        if (threadIdx.x == 0) sp.counters[CNT_NVALID] = s_valid;
        if (odd)
            ehrenfest_select_apply<Q, ST, true>(sp, M, s_valid);
        else
            ehrenfest_select_apply<Q, ST, false>(sp, M, s_valid);
    } else if (COLL == LBM_MEDIAN) {
        if (threadIdx.x == 0) sp.counters[CNT_NVALID] = 0u;
        __syncthreads();
        if (odd)
            median_apply<Q, ST, true>(sp, threadIdx.x >> 4, kBatchThreads >> 4);
        else
            median_apply<Q, ST, false>(sp, threadIdx.x >> 4, kBatchThreads >> 4);
    }
}

template <int Q, class ST, int COLL>
__device__ __forceinline__ void batch_item(const Params& sp, const BatchItem& it, int log2x, int rows, bool odd,
                                           bool fix_only) {
    if (!fix_only) {
        int e_code = -1, e_iters = 0;
        batch_tile<Q, ST, COLL>(sp, it, log2x, rows, odd, e_code, e_iters);
        if (COLL == LBM_ELBM) elbm_stats(sp, e_code, e_iters);
    } else {
        batch_fixup<Q, ST, COLL>(sp, odd);
    }
}

// The kernels' collision sets.
enum { kSetStream = 0, kSetLimiter = 1, kSetHeavy = 2 };

// Dispatch on the item's collision and lattice within the kernel's set.
template <class ST, int SET>
__device__ __forceinline__ void batch_dispatch(const Params& sp, const BatchItem& it, int log2x, int rows, bool odd,
                                               bool fix_only) {
    const int coll = it.code >> 4;
    const bool q9 = (it.code & 15) == 9;
#define LBM_BATCH_CASE(C)                                                     \
    case C:                                                                   \
        if (q9)                                                               \
            batch_item<9, ST, C>(sp, it, log2x, rows, odd, fix_only);         \
        else                                                                  \
            batch_item<3, ST, C>(sp, it, log2x, rows, odd, fix_only);         \
        break;
    if constexpr (SET == kSetHeavy) {
        switch (coll) { LBM_BATCH_CASE(LBM_ELBM) }
    } else if constexpr (SET == kSetLimiter) {
        switch (coll) {
            LBM_BATCH_CASE(LBM_EHRENFEST)
            LBM_BATCH_CASE(LBM_MEDIAN)
        }
    } else {
        switch (coll) {
            LBM_BATCH_CASE(LBM_LBGK)
            LBM_BATCH_CASE(LBM_POSITIVITY)
            LBM_BATCH_CASE(LBM_MRT)
        }
    }
#undef LBM_BATCH_CASE
}

// Resident CTAs per SM each kernel is compiled for (0: no register cap), in
// the 16/32-bit formats: the streaming set six (40 registers), the limiters
// five (48; at 40 they spilled over 1 KB, mostly on the fix-up paths); ELBM
// and FP64 storage uncapped.
template <class ST, int SET>
constexpr int kBatchMinBlocks = sizeof(typename ST::T) == 8 ? 0 : (SET == kSetStream ? 6 : (SET == kSetLimiter ? 5 : 0));

// Completion of a run of `count` items of one instance and step (all
// threads): their stores are made visible, the instance's item counter
// advances, and the CTA that completes the step runs the fix-up (sp holds
// that instance's parameters) and publishes the step.
template <class ST, int SET>
__device__ __forceinline__ void batch_complete(const BatchArgs& a, const Params& sp, const BatchItem& it,
                                               unsigned step, unsigned count, int* s_flag, unsigned* s_ready) {
    __threadfence();  // the run's stores are visible device-wide
    __syncthreads();
    if (threadIdx.x == 0)
        *s_flag = atomicAdd(&a.done[it.inst], count) + count == (unsigned)a.ntiles[it.inst];
    __syncthreads();
    if (*s_flag) {
        __threadfence();
        if (threadIdx.x == 0) sp.counters[(step & 1u) ^ 1u] = 0u;  // the next step's list starts empty
        batch_dispatch<ST, SET>(sp, it, a.tile_log2x, a.rows, (step & 1u) != 0, true);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            a.done[it.inst] = 0u;
            __threadfence();
            atomicExch(&a.gen[it.inst], step + 1u);
            *s_ready = step + 1u;
        }
    }
    __syncthreads();
}

template <class ST, int SET>
__global__ void __launch_bounds__(kBatchThreads, kBatchMinBlocks<ST, SET>) batch_persistent(BatchArgs a) {
    __shared__ Params sp;
    __shared__ unsigned long long s_idx;
    __shared__ int s_flag, s_inst;
    __shared__ unsigned s_base, s_ready;  // s_ready: steps of s_inst known complete
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_base = *(volatile unsigned*)&a.sync->base;
        s_inst = -1;
        s_ready = 0u;
    }
    __syncthreads();
    const unsigned base = s_base;
    const unsigned long long total = (unsigned long long)a.nitems * (unsigned long long)a.steps;
    bool failed = false;
    // a run of processed items of one instance and step whose completion is
    // not yet counted; it is counted before any wait, so that no CTA waits
    // while holding uncounted work
    BatchItem run_it = {0, 0, 0, 0};
    unsigned run_step = 0u, run_n = 0u;
    while (!failed) {
        if (tid == 0) s_idx = atomicAdd(&a.sync->head, (unsigned long long)a.chunk);
        __syncthreads();
        const unsigned long long first = s_idx;
        __syncthreads();  // s_idx read before it is rewritten
        if (first >= total) break;
        const unsigned long long last = first + a.chunk < total ? first + a.chunk : total;
        for (unsigned long long idx = first; idx < last; ++idx) {
            const unsigned s = (unsigned)(idx / (unsigned long long)a.nitems);
            const BatchItem it = a.items[idx - (unsigned long long)s * a.nitems];
            const unsigned step = base + s;
            if (run_n && (it.inst != run_it.inst || step != run_step)) {
                batch_complete<ST, SET>(a, sp, run_it, run_step, run_n, &s_flag, &s_ready);
                run_n = 0u;
            }
            const bool same = it.inst == s_inst;  // read before thread 0 rewrites it
            __syncthreads();
            // the instance's previous step (and its fix-up) is complete
            if (tid == 0) {
                s_flag = 1;
                if (!(same && s_ready >= step)) {
                    s_flag = wait_generation(&a.gen[it.inst], step, a.sync, a.wait_ns);
                    s_ready = step;
                }
                s_inst = it.inst;
            }
            if (!same) {
                const int* src = (const int*)(a.insts + it.inst);
                int* d = (int*)&sp;
                for (int k = tid; k < (int)(sizeof(Params) / 4); k += kBatchThreads) d[k] = src[k];
            }
            __syncthreads();
            if (!s_flag) {
                failed = true;
                break;
            }
            if (tid == 0) sp.cslot = (int)(step & 1u);
            __syncthreads();
            batch_dispatch<ST, SET>(sp, it, a.tile_log2x, a.rows, (step & 1u) != 0, false);
            run_it = it;
            run_step = step;
            ++run_n;
        }
        if (run_n && !failed) {
            batch_complete<ST, SET>(a, sp, run_it, run_step, run_n, &s_flag, &s_ready);
            run_n = 0u;
        }
        __syncthreads();
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&a.sync->exit, 1u) == gridDim.x - 1) {
            // the last CTA out resets the queue for the next launch
            a.sync->head = 0ull;
            a.sync->exit = 0u;
            a.sync->base = base + (unsigned)a.steps;
            __threadfence();
        }
    }
}

template <class ST>
struct BatchLaunch {
    // CTAs of one kernel (set: kSet*) that fit on one SM, and the launch.
    static cudaError_t occupancy(int set, int* per_sm);
    static cudaError_t persistent(int set, const BatchArgs& a, int grid, cudaStream_t s);
};

template <class ST>
using BatchKernel = void (*)(BatchArgs);

template <class ST>
BatchKernel<ST> batch_kernel(int set) {
    return set == kSetHeavy ? batch_persistent<ST, kSetHeavy>
                            : (set == kSetLimiter ? batch_persistent<ST, kSetLimiter> : batch_persistent<ST, kSetStream>);
}

template <class ST>
cudaError_t BatchLaunch<ST>::occupancy(int set, int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<ST>(set), kBatchThreads, 0);
}

template <class ST>
cudaError_t BatchLaunch<ST>::persistent(int set, const BatchArgs& a, int grid, cudaStream_t s) {
    batch_kernel<ST>(set)<<<grid, kBatchThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbm
