// C ABI entry points: argument checks and dispatch to the engines.
#include <algorithm>
#include <vector>

#include "qdvm_internal.cuh"

namespace {

bool prec_ok(int prec) { return prec == QDVM_F64 || prec == QDVM_F32 || prec == QDVM_F32_KAHAN; }

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

qdvm_status build_batch(const qdvm_plan_t* plans, int n_plans, BatchDev* b, int* d_out) {
    if (!plans || n_plans < 1 || n_plans > QDVM_MAX_BATCH_PLANS)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_plans must be in [1, QDVM_MAX_BATCH_PLANS]");
    b->n_plans = n_plans;
    int d = -1;
    for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b->p[i] = PlanDev();
    for (int i = 0; i < n_plans; ++i) {
        if (!qdvm_plan_ok(plans[i])) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle in batch");
        if (d >= 0 && plans[i]->d != d) return qdvm_fail(QDVM_ERR_INVALID_ARG, "plans of a batch must share d");
        d = plans[i]->d;
        b->p[i] = plan_dev(plans[i]);
    }
    *d_out = d;
    return QDVM_OK;
}

// 3D forward with the loss as an FFT convolution (tuning loss_fft = 1)
bool use_fast3d(int mode, const BatchDev& b, const qdvm_tuning& t, int prec) {
    return t.loss_fft && b.p[0].d == 3 && fast3d_supported(mode, b, prec);
}

// workspace of one mode: the 3D FFT-loss evaluator or the line engine
size_t mode_workspace(int mode, const BatchDev& b, int n_cells, int prec, bool single, const qdvm_tuning& t) {
    return use_fast3d(mode, b, t, prec) ? fast3d_workspace(mode, b, n_cells, prec, single, t.line_chunks)
                                        : engine_workspace(mode, b, n_cells, prec, single, t.line_chunks);
}

}  // namespace

BatchDev single_batch(const qdvm_plan_s* p) {
    BatchDev b;
    for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b.p[i] = PlanDev();
    b.n_plans = 1;
    b.p[0] = plan_dev(p);
    return b;
}

extern "C" qdvm_status qdvm_eval_workspace(qdvm_plan_t p, int prec, size_t* bytes) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!prec_ok(prec) || !bytes) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision or NULL bytes");
    const BatchDev b = single_batch(p);
    const size_t der = std::max(mode_workspace(QDVM_MODE_JVP, b, 1, prec, true, p->tune),
                                mode_workspace(QDVM_MODE_VJP, b, 1, prec, true, p->tune));
    if (p->d == 2 && fused2d_supported(p->N, p->Ntilde, prec)) {
        *bytes = std::max(fused2d_single_workspace(p, prec), der);
        return QDVM_OK;
    }
    *bytes = std::max(mode_workspace(QDVM_MODE_FWD, b, 1, prec, true, p->tune), der);
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_eval(qdvm_plan_t p, const void* f, void* Q, int prec, void* ws, size_t ws_bytes,
                                 void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!f || !Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f and Q must be device pointers");
    if (f == Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must not alias Q");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->d == 2 && fused2d_supported(p->N, p->Ntilde, prec)) return fused2d_eval_single(p, f, Q, prec, ws, ws_bytes, st);
    const BatchDev b = single_batch(p);
    if (use_fast3d(QDVM_MODE_FWD, b, p->tune, prec))
        return fast3d_run(QDVM_MODE_FWD, b, 1, nullptr, nullptr, f, nullptr, Q, nullptr, prec, ws, ws_bytes, true,
                          p->tune.line_chunks, st);
    return engine_run(QDVM_MODE_FWD, b, 1, nullptr, nullptr, f, nullptr, Q, nullptr, prec, ws, ws_bytes,
                      true, p->tune.line_chunks, st);
}

static bool all_fused2d(const qdvm_plan_t* plans, int n_plans, int d, int prec) {
    bool ok = d == 2;
    for (int i = 0; i < n_plans && ok; ++i) ok = fused2d_supported(plans[i]->N, plans[i]->Ntilde, prec);
    return ok;
}

extern "C" qdvm_status qdvm_batched_workspace(const qdvm_plan_t* plans, int n_plans, int n_cells, int prec,
                                              size_t* bytes) {
    if (n_cells < 0 || !bytes || !prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad n_cells, prec or NULL bytes");
    BatchDev b;
    int d = 0;
    qdvm_status s = build_batch(plans, n_plans, &b, &d);
    if (s != QDVM_OK) return s;
    const qdvm_tuning& tu = plans[0]->tune;
    const size_t der = std::max(mode_workspace(QDVM_MODE_JVP, b, n_cells, prec, false, tu),
                                mode_workspace(QDVM_MODE_VJP, b, n_cells, prec, false, tu));
    const size_t fwd = all_fused2d(plans, n_plans, d, prec) ? 256 + round256((size_t)std::max(n_cells, 1) * sizeof(int))
                                                            : mode_workspace(QDVM_MODE_FWD, b, n_cells, prec, false, tu);
    *bytes = std::max(fwd, der);
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_eval_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                         const int64_t* cell_offset, const void* f, void* Q, double* moments, int prec,
                                         void* ws, size_t ws_bytes, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (!prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    BatchDev b;
    int d = 0;
    qdvm_status s = build_batch(plans, n_plans, &b, &d);
    if (s != QDVM_OK) return s;
    if (n_cells == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f || !Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (f == Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must not alias Q");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (all_fused2d(plans, n_plans, d, prec)) {
        // the on-chip evaluator needs the work counter and the cell schedule
        if (!ws || ws_bytes < 256 + round256((size_t)n_cells * sizeof(int)))
            return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_eval_batched");
        return fused2d_eval_batched(b, plans[0]->tune, n_cells, cell_plan, cell_offset, f, Q, moments, prec, ws, st);
    }
    // the 3D evaluator and the engine check their own layouts against ws_bytes
    if (use_fast3d(QDVM_MODE_FWD, b, plans[0]->tune, prec))
        return fast3d_run(QDVM_MODE_FWD, b, n_cells, cell_plan, cell_offset, f, nullptr, Q, moments, prec, ws, ws_bytes,
                          false, plans[0]->tune.line_chunks, st);
    return engine_run(QDVM_MODE_FWD, b, n_cells, cell_plan, cell_offset, f, nullptr, Q, moments, prec, ws, ws_bytes,
                      false, plans[0]->tune.line_chunks, st);
}

extern "C" qdvm_status qdvm_moments(qdvm_plan_t p, const void* Q, int prec, double* m, void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!prec_ok(prec) || !Q || !m) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision or NULL pointer");
    return moments_launch(p->d, p->N, p->L, Q, prec, m, static_cast<cudaStream_t>(stream));
}

static qdvm_status derivative_single(int mode, qdvm_plan_t p, const void* f, const void* a, void* out, int prec,
                                     void* ws, size_t ws_bytes, void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!f || !a || !out) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (out == f || out == a) return qdvm_fail(QDVM_ERR_INVALID_ARG, "the output must not alias an input");
    const BatchDev b = single_batch(p);
    if (use_fast3d(mode, b, p->tune, prec))
        return fast3d_run(mode, b, 1, nullptr, nullptr, f, a, out, nullptr, prec, ws, ws_bytes, true, p->tune.line_chunks,
                          static_cast<cudaStream_t>(stream));
    return engine_run(mode, b, 1, nullptr, nullptr, f, a, out, nullptr, prec, ws, ws_bytes, true,
                      p->tune.line_chunks, static_cast<cudaStream_t>(stream));
}

static qdvm_status derivative_batched(int mode, const qdvm_plan_t* plans, int n_plans, int n_cells,
                                      const int* cell_plan, const int64_t* cell_offset, const void* f, const void* a,
                                      void* out, int prec, void* ws, size_t ws_bytes, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (!prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    BatchDev b;
    int d = 0;
    qdvm_status s = build_batch(plans, n_plans, &b, &d);
    if (s != QDVM_OK) return s;
    if (n_cells == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f || !a || !out) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (out == f || out == a) return qdvm_fail(QDVM_ERR_INVALID_ARG, "the output must not alias an input");
    if (use_fast3d(mode, b, plans[0]->tune, prec))
        return fast3d_run(mode, b, n_cells, cell_plan, cell_offset, f, a, out, nullptr, prec, ws, ws_bytes, false,
                          plans[0]->tune.line_chunks, static_cast<cudaStream_t>(stream));
    return engine_run(mode, b, n_cells, cell_plan, cell_offset, f, a, out, nullptr, prec, ws, ws_bytes, false,
                      plans[0]->tune.line_chunks, static_cast<cudaStream_t>(stream));
}

extern "C" qdvm_status qdvm_jvp(qdvm_plan_t p, const void* f, const void* df, void* dQ, int prec, void* ws,
                                size_t ws_bytes, void* stream) {
    return derivative_single(QDVM_MODE_JVP, p, f, df, dQ, prec, ws, ws_bytes, stream);
}

extern "C" qdvm_status qdvm_vjp(qdvm_plan_t p, const void* f, const void* g, void* grad, int prec, void* ws,
                                size_t ws_bytes, void* stream) {
    return derivative_single(QDVM_MODE_VJP, p, f, g, grad, prec, ws, ws_bytes, stream);
}

extern "C" qdvm_status qdvm_jvp_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                        const int64_t* cell_offset, const void* f, const void* df, void* dQ, int prec,
                                        void* ws, size_t ws_bytes, void* stream) {
    return derivative_batched(QDVM_MODE_JVP, plans, n_plans, n_cells, cell_plan, cell_offset, f, df, dQ, prec, ws,
                              ws_bytes, stream);
}

extern "C" qdvm_status qdvm_vjp_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                        const int64_t* cell_offset, const void* f, const void* g, void* grad, int prec,
                                        void* ws, size_t ws_bytes, void* stream) {
    return derivative_batched(QDVM_MODE_VJP, plans, n_plans, n_cells, cell_plan, cell_offset, f, g, grad, prec, ws,
                              ws_bytes, stream);
}

extern "C" qdvm_status qdvm_tune_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                         const int64_t* cell_offset, const void* f, void* Q, int prec, void* ws,
                                         size_t ws_bytes, void* stream, qdvm_tuning* best) {
    if (!prec_ok(prec)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    BatchDev b;
    int d = 0;
    qdvm_status s = build_batch(plans, n_plans, &b, &d);
    if (s != QDVM_OK) return s;
    if (n_cells <= 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "nothing to tune (n_cells <= 0)");
    const qdvm_tuning saved = plans[0]->tune;
    std::vector<qdvm_tuning> cand;
    if (all_fused2d(plans, n_plans, d, prec)) {
        for (int th : {256, 512})
            for (int dj : {0, 1, 2}) cand.push_back(qdvm_tuning{th, dj, saved.line_chunks, 0, saved.scan_j});
        // FFT loss; the gain windows by DIRECT gathers (scan_j = 0) or by the
        // SCAN engine from window half-length scan_j up
        for (int th : {256, 512})
            for (int sj : {0, 2, 3, 4, 5, 7})
                cand.push_back(qdvm_tuning{th, saved.direct_j, saved.line_chunks, 1, sj});
        // FFT loss carrying one axis window too: W_(1,0) with the other
        // windows by DIRECT gathers (scan_j = 0), or W_(0,1) with the SCAN
        // engine walking the pairs from window half-length scan_j up
        for (int th : {256, 512})
            for (int sj : {0, 5, 7, 10, 14})
                cand.push_back(qdvm_tuning{th, saved.direct_j, saved.line_chunks, 2, sj});
        // FFT loss and the FFT window engine for the pairs from window
        // half-length scan_j up, the other windows by DIRECT gathers
        for (int th : {256, 512})
            for (int sj : {5, 7, 10, 14})
                cand.push_back(qdvm_tuning{th, saved.direct_j, saved.line_chunks, 3, sj});
    } else {
        const qdvm_tuning fft{saved.threads, saved.direct_j, 0, 1, saved.scan_j};
        const bool f3 = use_fast3d(QDVM_MODE_FWD, b, fft, prec);
        for (int c : {0, 1, 2, 3, 4, 6, 8, 12, 16}) {
            if (engine_workspace(QDVM_MODE_FWD, b, n_cells, prec, false, c) <= ws_bytes)
                cand.push_back(qdvm_tuning{saved.threads, saved.direct_j, c, 0, saved.scan_j});
            if (f3 && fast3d_workspace(QDVM_MODE_FWD, b, n_cells, prec, false, c) <= ws_bytes)
                cand.push_back(qdvm_tuning{saved.threads, saved.direct_j, c, 1, saved.scan_j});
        }
    }
    if (cand.empty()) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for every candidate");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    QDVM_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return qdvm_cuda_status(ce, "cudaEventCreate");
    }
    qdvm_status rs = QDVM_OK;
    // median of three timed runs after a warm-up, with the plans' current
    // tunings; rs records a failure
    auto time_batch = [&]() -> float {
        float times[3] = {0.f, 0.f, 0.f};
        for (int rep = 0; rep < 4 && rs == QDVM_OK; ++rep) {
            cudaEventRecord(e0, st);
            rs = qdvm_eval_batched(plans, n_plans, n_cells, cell_plan, cell_offset, f, Q, nullptr, prec, ws, ws_bytes,
                                   stream);
            cudaEventRecord(e1, st);
            if (rs != QDVM_OK) break;
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                rs = qdvm_cuda_status(ce, "tuning run");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) times[rep - 1] = ms;  // first run warms up
        }
        std::sort(times, times + 3);
        return times[1];
    };
    float best_ms = 1e30f;
    qdvm_tuning best_t = saved;
    for (const qdvm_tuning& t : cand) {
        for (int i = 0; i < n_plans; ++i) plans[i]->tune = t;
        const float ms = time_batch();
        if (rs != QDVM_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_t = t;
        }
    }
    // per-plan refinement of the 2D launch parameters: each cell runs with
    // its plan's direct_j, loss_fft and scan_j (the block size is plans[0]'s),
    // so, the block size fixed, every plan in turn tries the candidates of
    // that size with the others at their best so far
    std::vector<qdvm_tuning> per(n_plans, best_t);
    if (rs == QDVM_OK && n_plans > 1 && all_fused2d(plans, n_plans, d, prec)) {
        for (int i = 0; i < n_plans; ++i) {
            for (int k = 0; k < n_plans; ++k) plans[k]->tune = per[k];
            for (const qdvm_tuning& t : cand) {
                if (t.threads != best_t.threads) continue;
                plans[i]->tune = t;
                const float ms = time_batch();
                if (rs != QDVM_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    per[i] = t;
                }
            }
            if (rs != QDVM_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < n_plans; ++i) plans[i]->tune = rs == QDVM_OK ? per[i] : saved;
    if (rs != QDVM_OK) return rs;
    if (best) *best = per[0];
    return QDVM_OK;
}
