// Host-side state of an lbm_ctx, shared by the translation units of the
// C ABI (lbm_abi.cu, lbm_adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_params.h"

struct lbm_ctx {
    lbm_config cfg;
    int Q = 0;
    lbm::Params p;
    char* base = nullptr;
    size_t bytes = 0;
    int parity = 0;   // 0: natural layout; 1: after an even (in-place) step
    uint64_t t = 0;   // steps since init / set_state
    int nsm = 1;
    int device = 0;
    double* staging = nullptr;  // 3 * N doubles for lbm_init
    std::string err;
    // kernel tracing (lbm_profile_enable)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // pairs (start, end)
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    // two steps (both A-A parities) captured once at creation and replayed,
    // and the same repeated (long runs of small lattices)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph_long = nullptr;
    cudaGraphExec_t graph_long_exec = nullptr;
    void drop_graphs() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        if (graph_long_exec) cudaGraphExecDestroy(graph_long_exec);
        if (graph_long) cudaGraphDestroy(graph_long);
        graph = graph_long = nullptr;
        graph_exec = graph_long_exec = nullptr;
    }
    ~lbm_ctx() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        drop_graphs();
    }
};

