// lbm_ehrenfest_step_noalloc: the LBGK + Ehrenfest step for callers that
// cannot allocate device memory.  Its scratch (step counters and the limiter
// candidate list) lives in a file-scope device array of this library instead
// of a caller allocation; the caller passes only the populations.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_setup.h"

using namespace lbm;

namespace lbm {
extern template struct Launch<StF64>;
extern template struct Launch<StF32>;
extern template struct Launch<StBF16>;
extern template struct Launch<StF16>;
}  // namespace lbm

namespace {

// Shared scratch of every call on a device; held by each GPU that loads the
// library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

constexpr size_t kCounterBytes = 256;  // counters + statistics, zeroed per call
constexpr int kMaxDevices = 64;

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Bytes of scratch a lattice of N sites needs: counters plus one candidate
// entry per site (populations in the arithmetic type, FP64 Delta S, site
// index, selected flag), so the list can never overflow.
size_t scratch_need(int Q, size_t N, int precision) {
    const size_t tb = precision == LBM_FP64 ? 8 : 4;
    return kCounterBytes + up256(N * Q * tb) + up256(N * 8) + up256(N * 4) + up256(N * 4);
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress; the host-side name is only a stand-in).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_ehrenfest_step_noalloc(const lbm_config* cfg, void* f, int nsteps,
                                                 void* stream) {
    if (!cfg || !f || nsteps < 0 || (nsteps & 1)) return LBM_ERR_ARG;
    // the checks of lbm_create, then what this entry point does not cover:
    // other collisions and the diffusive walls (their wall kernel)
    if (check_config(cfg)) return LBM_ERR_ARG;
    if (cfg->collision != LBM_EHRENFEST || cfg->bc == LBM_BC_DIFFUSIVE) return LBM_ERR_ARG;
    const int Q = cfg->lattice == LBM_D1Q3 ? 3 : 9;
    const size_t N = (size_t)cfg->nx * cfg->ny;
    if (scratch_need(Q, N, cfg->precision) > (size_t)LBM_NOALLOC_SCRATCH_BYTES) return LBM_ERR_OOM;

    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LBM_ERR_CUDA;
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;

    // the parameters lbm_create derives from cfg; the layout is the caller's
    // dense one: pitch = nx, one plane of ny * nx per direction
    Params p;
    std::memset(&p, 0, sizeof p);
    fill_params(cfg, nsm, p);
    p.f = f;
    p.plane = (int64_t)N;
    p.plane32 = (int)N;
    p.pitch = cfg->nx;
    char* s = (char*)scratch;
    p.counters = (unsigned*)s;
    p.stats = (unsigned long long*)(s + CNT_WORDS * 4);
    p.scratch_d = (double*)(s + CNT_WORDS * 4 + ST_WORDS * 8);
    const size_t tb = cfg->precision == LBM_FP64 ? 8 : 4;
    size_t off = kCounterBytes;
    p.cand_cap = (int)N;
    p.cand_f = s + off;
    off += up256(N * Q * tb);
    p.cand_ds = (double*)(s + off);
    off += up256(N * 8);
    p.cand_site = (int*)(s + off);
    off += up256(N * 4);
    p.cand_sel = (int*)(s + off);

    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the counters start at zero
    if (cudaMemsetAsync(s, 0, kCounterBytes, st) != cudaSuccess) return LBM_ERR_CUDA;
    for (int k = 0; k < nsteps; ++k) {
        Params q = p;
        q.cslot = k & 1;
        const bool odd = (k & 1) != 0;
        cudaError_t e;
        switch (cfg->precision) {
            case LBM_FP64:
                e = Launch<StF64>::step(Q, LBM_EHRENFEST, odd, q, st);
                if (e == cudaSuccess) e = Launch<StF64>::fixup(Q, LBM_EHRENFEST, odd, q, st, nsm);
                break;
            case LBM_FP32:
                e = Launch<StF32>::step(Q, LBM_EHRENFEST, odd, q, st);
                if (e == cudaSuccess) e = Launch<StF32>::fixup(Q, LBM_EHRENFEST, odd, q, st, nsm);
                break;
            case LBM_BF16_DEV:
                e = Launch<StBF16>::step(Q, LBM_EHRENFEST, odd, q, st);
                if (e == cudaSuccess) e = Launch<StBF16>::fixup(Q, LBM_EHRENFEST, odd, q, st, nsm);
                break;
            default:
                e = Launch<StF16>::step(Q, LBM_EHRENFEST, odd, q, st);
                if (e == cudaSuccess) e = Launch<StF16>::fixup(Q, LBM_EHRENFEST, odd, q, st, nsm);
                break;
        }
        if (e != cudaSuccess) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
