// Batched form: many independent lattices (instances) advanced together.
// Each launch covers every instance of one collision kind; a CTA takes one
// (instance, tile) work item, copies that instance's Params to shared memory
// and runs the single-lattice site update on its 128 x 2 tile.  The limiter
// follow-up runs one CTA per instance.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// (instance, tile x, tile y, unused)
using WorkItem = int4;

__device__ __forceinline__ void load_params(Params& dst, const Params* __restrict__ insts, int inst,
                                            int cslot) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    const int* src = (const int*)(insts + inst);
    int* d = (int*)&dst;
    for (int k = tid; k < (int)(sizeof(Params) / 4); k += nthreads) d[k] = src[k];
    __syncthreads();
    if (tid == 0) dst.cslot = cslot;
    __syncthreads();
}

template <int Q, class ST, int COLL, bool ODD>
__global__ void __launch_bounds__(kBlockX* kBlockY)
    batch_step_kernel(const Params* __restrict__ insts, const WorkItem* __restrict__ work, int cslot) {
    __shared__ Params sp;
    const WorkItem w = work[blockIdx.x];
    load_params(sp, insts, w.x, cslot);
    constexpr bool kLimiter = (COLL == LBM_EHRENFEST || COLL == LBM_MEDIAN);
    if (kLimiter && w.y == 0 && w.z == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        sp.counters[cslot ^ 1] = 0u;
        sp.counters[CNT_NVALID] = 0u;
    }
    const int x = w.y * kBlockX + threadIdx.x;
    const int y = w.z * kBlockY + threadIdx.y;
    int e_code = -1, e_iters = 0;
    typename ST::T acc = 0;  // no reduction in the batched collisions
    if (x < sp.nx && y < sp.ny) site_update<Q, ST, COLL, ODD>(sp, x, y, e_code, e_iters, acc);
    if (COLL == LBM_ELBM) elbm_stats(sp, e_code, e_iters);
}

// One CTA per Ehrenfest instance: FP64 Delta S of its screened sites, then
// the k-largest selection and the rewrite to f*.
template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256)
    batch_ehrenfest_kernel(const Params* __restrict__ insts, const int* __restrict__ ids, int cslot) {
    using T = typename ST::T;
    __shared__ Params sp;
    __shared__ unsigned s_valid;
    load_params(sp, insts, ids[blockIdx.x], cslot);
    if (threadIdx.x == 0) s_valid = 0;
    __syncthreads();
    unsigned M = sp.counters[cslot];
    if (M > (unsigned)sp.cand_cap) M = (unsigned)sp.cand_cap;
    unsigned n = 0;
    const unsigned groups = blockDim.x >> 4;
    for (unsigned base = 0; base < M; base += groups) {
        const unsigned j = base + (threadIdx.x >> 4);
        const double d = delta_s_group<Q, ST>(sp, j, j < M);
        if (j < M && (threadIdx.x & 15) == 0) {
            const bool c = d > sp.delta;
            sp.cand_ds[j] = c ? d : -1.0;
            n += c;
        }
    }
    if (n) atomicAdd(&s_valid, n);
    __syncthreads();
    if (threadIdx.x == 0 && s_valid) atomicAdd(&sp.counters[CNT_NVALID], s_valid);
    ehrenfest_select_apply<Q, ST, ODD>(sp, M, s_valid);
}

// One CTA per median-filter instance.
template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256)
    batch_median_kernel(const Params* __restrict__ insts, const int* __restrict__ ids, int cslot) {
    __shared__ Params sp;
    load_params(sp, insts, ids[blockIdx.x], cslot);
    median_apply<Q, ST, ODD>(sp, threadIdx.x >> 4, blockDim.x >> 4);
}

template <class ST>
struct BatchLaunch {
    static cudaError_t step(int coll, bool odd, const Params* insts, const WorkItem* work, int nwork,
                            int cslot, cudaStream_t s);
    static cudaError_t fixup(int coll, bool odd, const Params* insts, const int* ids, int nids,
                             int cslot, cudaStream_t s);
};

template <class ST, int COLL>
cudaError_t batch_step_c(bool odd, const Params* insts, const WorkItem* work, int nwork, int cslot,
                         cudaStream_t s) {
    dim3 b(kBlockX, kBlockY);
    if (odd)
        batch_step_kernel<9, ST, COLL, true><<<nwork, b, 0, s>>>(insts, work, cslot);
    else
        batch_step_kernel<9, ST, COLL, false><<<nwork, b, 0, s>>>(insts, work, cslot);
    return cudaGetLastError();
}

template <class ST>
cudaError_t BatchLaunch<ST>::step(int coll, bool odd, const Params* insts, const WorkItem* work,
                                  int nwork, int cslot, cudaStream_t s) {
    if (nwork <= 0) return cudaSuccess;
    switch (coll) {
        case LBM_LBGK: return batch_step_c<ST, LBM_LBGK>(odd, insts, work, nwork, cslot, s);
        case LBM_ELBM: return batch_step_c<ST, LBM_ELBM>(odd, insts, work, nwork, cslot, s);
        case LBM_EHRENFEST: return batch_step_c<ST, LBM_EHRENFEST>(odd, insts, work, nwork, cslot, s);
        case LBM_POSITIVITY: return batch_step_c<ST, LBM_POSITIVITY>(odd, insts, work, nwork, cslot, s);
        case LBM_MEDIAN: return batch_step_c<ST, LBM_MEDIAN>(odd, insts, work, nwork, cslot, s);
        case LBM_MRT: return batch_step_c<ST, LBM_MRT>(odd, insts, work, nwork, cslot, s);
    }
    return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t BatchLaunch<ST>::fixup(int coll, bool odd, const Params* insts, const int* ids, int nids,
                                   int cslot, cudaStream_t s) {
    if (nids <= 0) return cudaSuccess;
    if (coll == LBM_EHRENFEST) {
        if (odd)
            batch_ehrenfest_kernel<9, ST, true><<<nids, 256, 0, s>>>(insts, ids, cslot);
        else
            batch_ehrenfest_kernel<9, ST, false><<<nids, 256, 0, s>>>(insts, ids, cslot);
    } else if (coll == LBM_MEDIAN) {
        if (odd)
            batch_median_kernel<9, ST, true><<<nids, 256, 0, s>>>(insts, ids, cslot);
        else
            batch_median_kernel<9, ST, false><<<nids, 256, 0, s>>>(insts, ids, cslot);
    } else {
        return cudaSuccess;
    }
    return cudaGetLastError();
}

}  // namespace lbm
