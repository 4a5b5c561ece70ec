// C ABI entry points: argument checks and dispatch to the engines.
#include <algorithm>

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
    const size_t der = std::max(engine_workspace(QDVM_MODE_JVP, b, 1, prec, true),
                                engine_workspace(QDVM_MODE_VJP, b, 1, prec, true));
    if (p->d == 2 && fused2d_supported(p->N, p->Ntilde, prec)) {
        *bytes = std::max(fused2d_single_workspace(p, prec), der);
        return QDVM_OK;
    }
    *bytes = std::max(engine_workspace(QDVM_MODE_FWD, b, 1, prec, true), der);
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
    return engine_run(QDVM_MODE_FWD, single_batch(p), 1, nullptr, nullptr, f, nullptr, Q, nullptr, prec, ws, ws_bytes,
                      true, st);
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
    const size_t der = std::max(engine_workspace(QDVM_MODE_JVP, b, n_cells, prec, false),
                                engine_workspace(QDVM_MODE_VJP, b, n_cells, prec, false));
    const size_t fwd = all_fused2d(plans, n_plans, d, prec) ? 256 + round256((size_t)std::max(n_cells, 1) * sizeof(int))
                                                            : engine_workspace(QDVM_MODE_FWD, b, n_cells, prec, false);
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
    size_t need = 0;
    s = qdvm_batched_workspace(plans, n_plans, n_cells, prec, &need);
    if (s != QDVM_OK) return s;
    if (!ws || ws_bytes < need) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_eval_batched");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int maxN = 0, maxH = 0;
    for (int i = 0; i < n_plans; ++i) {
        maxN = std::max(maxN, plans[i]->N);
        maxH = std::max(maxH, plans[i]->Ntilde);
    }
    if (all_fused2d(plans, n_plans, d, prec))
        return fused2d_eval_batched(b, maxN, maxH, n_cells, cell_plan, cell_offset, f, Q, moments, prec, ws, st);
    return engine_run(QDVM_MODE_FWD, b, n_cells, cell_plan, cell_offset, f, nullptr, Q, moments, prec, ws, ws_bytes,
                      false, st);
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
    return engine_run(mode, single_batch(p), 1, nullptr, nullptr, f, a, out, nullptr, prec, ws, ws_bytes, true,
                      static_cast<cudaStream_t>(stream));
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
    return engine_run(mode, b, n_cells, cell_plan, cell_offset, f, a, out, nullptr, prec, ws, ws_bytes, false,
                      static_cast<cudaStream_t>(stream));
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
