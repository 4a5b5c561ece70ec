// Space-homogeneous time stepping df/dt = Q(f) of every cell of a batch with
// the second-order total-variation-diminishing Runge-Kutta method that
// Section 4 uses for its runs (the Shu-Osher form):
//   f1      = f + dt Q(f)
//   f_{n+1} = (f + f1 + dt Q(f1)) / 2
// A stage is one batched evaluation (whatever engine the plans' tuning
// selects) and one elementwise kernel.  Everything is stream-ordered, so a
// loop of steps can be captured into one CUDA graph.
#include <algorithm>
#include <cmath>

#include "qdvm_internal.cuh"

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st);

namespace {

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

// f1 = f + dt q
template <typename T>
__global__ void k_rk2_stage1(int64_t n, const T* __restrict__ f, const T* __restrict__ q, T dt, T* __restrict__ f1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f1[i] = f[i] + dt * q[i];
}

// f = (f + f1 + dt q) / 2
template <typename T>
__global__ void k_rk2_stage2(int64_t n, T* __restrict__ f, const T* __restrict__ f1, const T* __restrict__ q, T dt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = T(0.5) * (f[i] + (f1[i] + dt * q[i]));
}

struct Rk2Layout {
    size_t eval, off_f1, off_q, total;
};

qdvm_status rk2_layout(const qdvm_plan_t* plans, int n_plans, int n_cells, int64_t n_elems, int prec, Rk2Layout* g) {
    size_t eval = 0;
    qdvm_status s = qdvm_batched_workspace(plans, n_plans, n_cells, prec, &eval);
    if (s != QDVM_OK) return s;
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    g->eval = r256(eval);
    g->off_f1 = g->eval;
    g->off_q = g->off_f1 + r256((size_t)n_elems * es);
    g->total = g->off_q + r256((size_t)n_elems * es);
    return QDVM_OK;
}

template <typename T>
void launch_stage(int which, int64_t n, T* f, T* f1, const T* q, double dt, cudaStream_t st) {
    const int grid = std::max(1, std::min((int)((n + 255) / 256), 8 * qdvm_num_sms()));
    if (which == 1) k_rk2_stage1<T><<<grid, 256, 0, st>>>(n, f, q, (T)dt, f1);
    else k_rk2_stage2<T><<<grid, 256, 0, st>>>(n, f, f1, q, (T)dt);
}

}  // namespace

extern "C" qdvm_status qdvm_rk2_workspace(const qdvm_plan_t* plans, int n_plans, int n_cells, int64_t n_elems,
                                          int prec, size_t* bytes) {
    if (!bytes || n_cells < 0 || n_elems < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad n_cells, n_elems or NULL bytes");
    Rk2Layout g;
    qdvm_status s = rk2_layout(plans, n_plans, n_cells, n_elems, prec, &g);
    if (s != QDVM_OK) return s;
    *bytes = g.total;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_rk2_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                        const int64_t* cell_offset, int64_t n_elems, void* f, double dt, int n_steps,
                                        double* moments, int prec, void* ws, size_t ws_bytes, void* stream) {
    if (n_cells < 0 || n_elems < 0 || n_steps < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "negative n_cells, n_elems or n_steps");
    if (!std::isfinite(dt)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "dt must be finite");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    Rk2Layout g;
    qdvm_status s = rk2_layout(plans, n_plans, n_cells, n_elems, prec, &g);
    if (s != QDVM_OK) return s;
    if (n_cells == 0 || n_elems == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (!ws || ws_bytes < g.total) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_rk2_batched");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(ws);
    void* f1 = base + g.off_f1;
    void* q = base + g.off_q;
    for (int k = 0; k < n_steps; ++k) {
        s = qdvm_eval_batched(plans, n_plans, n_cells, cell_plan, cell_offset, f, q, nullptr, prec, ws, g.eval, st);
        if (s != QDVM_OK) return s;
        if (prec == QDVM_F64)
            launch_stage<double>(1, n_elems, static_cast<double*>(f), static_cast<double*>(f1), static_cast<double*>(q), dt, st);
        else
            launch_stage<float>(1, n_elems, static_cast<float*>(f), static_cast<float*>(f1), static_cast<float*>(q), dt, st);
        QDVM_LAUNCH_CHECK("rk2 stage 1");
        s = qdvm_eval_batched(plans, n_plans, n_cells, cell_plan, cell_offset, f1, q, nullptr, prec, ws, g.eval, st);
        if (s != QDVM_OK) return s;
        if (prec == QDVM_F64)
            launch_stage<double>(2, n_elems, static_cast<double*>(f), static_cast<double*>(f1), static_cast<double*>(q), dt, st);
        else
            launch_stage<float>(2, n_elems, static_cast<float*>(f), static_cast<float*>(f1), static_cast<float*>(q), dt, st);
        QDVM_LAUNCH_CHECK("rk2 stage 2");
    }
    if (moments) {
        BatchDev b;
        for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b.p[i] = PlanDev();
        b.n_plans = n_plans;
        for (int i = 0; i < n_plans; ++i) b.p[i] = plan_dev(plans[i]);
        return moments_batched_launch(b, n_cells, cell_plan, cell_offset, f, prec, moments, st);
    }
    return QDVM_OK;
}

// One cell (the same scheme with qdvm_eval, which spreads a single cell's
// lines over the whole GPU): workspace = evaluator workspace, f1, Q.
namespace {

qdvm_status rk2_single_layout(qdvm_plan_t p, int prec, Rk2Layout* g) {
    size_t eval = 0;
    qdvm_status s = qdvm_eval_workspace(p, prec, &eval);
    if (s != QDVM_OK) return s;
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    const size_t n = (size_t)p->N * p->N * (p->d == 3 ? p->N : 1);
    g->eval = r256(eval);
    g->off_f1 = g->eval;
    g->off_q = g->off_f1 + r256(n * es);
    g->total = g->off_q + r256(n * es);
    return QDVM_OK;
}

}  // namespace

extern "C" qdvm_status qdvm_rk2_workspace_single(qdvm_plan_t p, int prec, size_t* bytes) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!bytes) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL bytes");
    Rk2Layout g;
    qdvm_status s = rk2_single_layout(p, prec, &g);
    if (s != QDVM_OK) return s;
    *bytes = g.total;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_rk2(qdvm_plan_t p, void* f, double dt, int n_steps, int prec, void* ws, size_t ws_bytes,
                                void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (n_steps < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "negative n_steps");
    if (!std::isfinite(dt)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "dt must be finite");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!f) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must be a device pointer");
    Rk2Layout g;
    qdvm_status s = rk2_single_layout(p, prec, &g);
    if (s != QDVM_OK) return s;
    if (!ws || ws_bytes < g.total) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_rk2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)p->N * p->N * (p->d == 3 ? p->N : 1);
    char* base = static_cast<char*>(ws);
    void* f1 = base + g.off_f1;
    void* q = base + g.off_q;
    for (int k = 0; k < n_steps; ++k) {
        s = qdvm_eval(p, f, q, prec, ws, g.eval, st);
        if (s != QDVM_OK) return s;
        if (prec == QDVM_F64)
            launch_stage<double>(1, n, static_cast<double*>(f), static_cast<double*>(f1), static_cast<double*>(q), dt, st);
        else
            launch_stage<float>(1, n, static_cast<float*>(f), static_cast<float*>(f1), static_cast<float*>(q), dt, st);
        QDVM_LAUNCH_CHECK("rk2 stage 1");
        s = qdvm_eval(p, f1, q, prec, ws, g.eval, st);
        if (s != QDVM_OK) return s;
        if (prec == QDVM_F64)
            launch_stage<double>(2, n, static_cast<double*>(f), static_cast<double*>(f1), static_cast<double*>(q), dt, st);
        else
            launch_stage<float>(2, n, static_cast<float*>(f), static_cast<float*>(f1), static_cast<float*>(q), dt, st);
        QDVM_LAUNCH_CHECK("rk2 stage 2");
    }
    return QDVM_OK;
}
