// Allocation-free variant of the batched 2D evaluator.
//
// Some callers cannot allocate device memory at all: a solver that owns a
// fixed device-memory budget and hands the library only its own arrays, a
// plug-in called from inside another framework's time loop where any
// cudaMalloc would synchronise the device in the middle of a step, or an
// embedding whose memory manager forbids foreign allocations.  They still
// pass f, Q, the cell layout and the moments array, but no workspace.  The
// only scratch the batched 2D evaluator needs (its atomic work counter and
// the cost-ordered cell list) then lives in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
#include <mutex>

#include "qdvm_internal.cuh"

// Scratch layout (the same as the caller-provided workspace of
// qdvm_eval_batched for the 2D on-chip evaluator): the work counter in the
// first 256 bytes, then one int per cell for the schedule.  256 KB + 256 B.
static __device__ __align__(256) int g_batch_scratch[64 + QDVM_NOALLOC_MAX_CELLS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_batch_scratch for the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with that device current.  It is looked up again on
// every call made outside a stream capture (a lookup allocates nothing), so
// a device reset between calls cannot leave a stale address behind; during a
// capture the address that the last call outside a capture found is used.
qdvm_status scratch_address(cudaStream_t stream, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qdvm_cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return qdvm_fail(QDVM_ERR_UNSUPPORTED, "device ordinal out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing(stream, &cs);
    if (qe != cudaSuccess) cudaGetLastError();  // a refused query (a capture elsewhere) leaves no error behind
    const bool capturing = qe != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!capturing) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess || !p) return qdvm_cuda_status(e, "cudaGetSymbolAddress(g_batch_scratch)");
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return qdvm_fail(QDVM_ERR_INVALID_ARG,
                         "qdvm_eval_batched_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_scratch_ptr[dev];
    return QDVM_OK;
}

}  // namespace

extern "C" qdvm_status qdvm_eval_batched_noalloc(const qdvm_plan_t* plans, int n_plans, int n_cells,
                                                 const int* cell_plan, const int64_t* cell_offset, const void* f,
                                                 void* Q, double* moments, int prec, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (n_cells > QDVM_NOALLOC_MAX_CELLS)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "qdvm_eval_batched_noalloc: n_cells exceeds QDVM_NOALLOC_MAX_CELLS "
                                               "(65536); split the batch or use qdvm_eval_batched with a workspace");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!plans || n_plans < 1 || n_plans > QDVM_MAX_BATCH_PLANS)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_plans must be in [1, QDVM_MAX_BATCH_PLANS]");
    BatchDev b;
    for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b.p[i] = PlanDev();
    b.n_plans = n_plans;
    for (int i = 0; i < n_plans; ++i) {
        if (!qdvm_plan_ok(plans[i])) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle in batch");
        if (plans[i]->d != 2 || !fused2d_supported(plans[i]->N, plans[i]->Ntilde, prec))
            return qdvm_fail(QDVM_ERR_UNSUPPORTED,
                             "qdvm_eval_batched_noalloc covers the on-chip 2D evaluator only (d = 2, N <= 64)");
        b.p[i] = plan_dev(plans[i]);
    }
    if (n_cells == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f || !Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (f == Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must not alias Q");
    void* scratch = nullptr;
    qdvm_status s = scratch_address(static_cast<cudaStream_t>(stream), &scratch);
    if (s != QDVM_OK) return s;
    // The schedule kernel zeroes the work counter at the start of every call;
    // the order list is rewritten in full.
    return fused2d_eval_batched(b, plans[0]->tune, n_cells, cell_plan, cell_offset, f, Q, moments, prec, scratch,
                                static_cast<cudaStream_t>(stream));
}
