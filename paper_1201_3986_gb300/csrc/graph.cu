// CUDA-graph capture of a batched evaluation (the schedule and the persistent
// evaluator) or of a loop of time steps: one executable graph with fixed
// device pointers, replayed with a single launch.
#include "qdvm_internal.cuh"

#define QDVM_GRAPH_MAGIC 0x51445647u  // "QDVG"

struct qdvm_graph_s {
    uint32_t magic;
    cudaGraphExec_t exec;
};

namespace {

// Captures the stream work of fn(stream) into an executable graph.
template <typename Fn>
qdvm_status capture(qdvm_graph_t* out, Fn fn) {
    if (!out) return qdvm_fail(QDVM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cudaStream_t s = nullptr;
    QDVM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return qdvm_cuda_status(e, "cudaStreamBeginCapture");
    }
    qdvm_status st = fn(s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (st != QDVM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return qdvm_cuda_status(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return qdvm_cuda_status(e, "cudaGraphInstantiate");
    qdvm_graph_s* h = new (std::nothrow) qdvm_graph_s();
    if (!h) {
        cudaGraphExecDestroy(exec);
        return qdvm_fail(QDVM_ERR_OOM, "host allocation");
    }
    h->magic = QDVM_GRAPH_MAGIC;
    h->exec = exec;
    *out = h;
    return QDVM_OK;
}

}  // namespace

extern "C" qdvm_status qdvm_graph_capture_batched(qdvm_graph_t* out, const qdvm_plan_t* plans, int n_plans,
                                                  int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                                  const void* f, void* Q, double* moments, int prec, void* ws,
                                                  size_t ws_bytes) {
    return capture(out, [&](cudaStream_t s) {
        return qdvm_eval_batched(plans, n_plans, n_cells, cell_plan, cell_offset, f, Q, moments, prec, ws, ws_bytes, s);
    });
}

extern "C" qdvm_status qdvm_graph_capture_rk2(qdvm_graph_t* out, const qdvm_plan_t* plans, int n_plans, int n_cells,
                                              const int* cell_plan, const int64_t* cell_offset, int64_t n_elems,
                                              void* f, double dt, int n_steps, double* moments, int prec, void* ws,
                                              size_t ws_bytes) {
    return capture(out, [&](cudaStream_t s) {
        return qdvm_rk2_batched(plans, n_plans, n_cells, cell_plan, cell_offset, n_elems, f, dt, n_steps, moments, prec,
                                ws, ws_bytes, s);
    });
}

extern "C" qdvm_status qdvm_graph_launch(qdvm_graph_t g, void* stream) {
    if (!g || g->magic != QDVM_GRAPH_MAGIC) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad graph handle");
    QDVM_CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_graph_destroy(qdvm_graph_t g) {
    if (!g) return QDVM_OK;
    if (g->magic != QDVM_GRAPH_MAGIC) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad graph handle");
    cudaGraphExecDestroy(g->exec);
    g->magic = 0;
    delete g;
    return QDVM_OK;
}
