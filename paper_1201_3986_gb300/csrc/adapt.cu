// Space-dependent truncation: the paper notes (end of Section 3.3) that Nbar
// can vary from cell to cell, with fewer directions where the distribution
// is close to equilibrium.  Two stream-ordered kernels make that choice on
// the device, before the batched evaluation:
//   1. the distance of every cell to the Maxwellian with its own discrete
//      moments, eps = sum |f - M[f]| / sum |f| (to about 1e-7);
//   2. the plan of every cell: level = number of (ascending) thresholds
//      that eps reaches, plan = level_plan[base][level].
#include <algorithm>
#include <cmath>

#include "qdvm_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct LevelTable {
    int n_base, n_levels;
    double thr[QDVM_MAX_LEVELS - 1];
    int plan[QDVM_MAX_BATCH_PLANS * QDVM_MAX_LEVELS];
};

// Block sums of K compensated FP32 partials (s + c per thread), in a fixed
// order: TwoSum shuffles within each warp, then thread 0 adds the warps'
// results in FP64 into out[0..K).  Ends with a barrier.
template <int K>
__device__ void block_sum(const float (&s)[K], const float (&c)[K], double* red, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float a = s[i], e = c[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float b = __shfl_down_sync(0xffffffffu, a, o), eb = __shfl_down_sync(0xffffffffu, e, o);
            const float t = a + b, bp = t - a;
            e += eb + ((a - (t - bp)) + (b - bp));
            a = t;
        }
        if (lane == 0) red[wid * K + i] = (double)a + (double)e;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < K; ++i) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[w * K + i];
            out[i] = t;
        }
    __syncthreads();
}

constexpr int kMaxN = 256;

// One block per cell (grid-stride over cells).  Warps walk rows of the cell
// (lanes along the last axis: coalesced), so a point's coordinates cost one
// division per row.  The Maxwellian is separable on the grid,
// M(v) = rho (2 pi T)^(-d/2) prod_a g_a(v_a), so only d N exponentials per
// cell are evaluated (an FP32 table in shared memory).  Per-point arithmetic
// is FP32 with compensated (Neumaier) sums, since FP64 issues at a small
// fraction of the FP32 rate; the warp results are added and the per-cell
// scalars (rho, u, T) formed in FP64 by one thread.  The indicator is thus
// accurate to about 1e-7.
template <typename T>
__global__ void k_equilibrium_distance(BatchDev B, int n_cells, const int* __restrict__ cell_plan,
                                       const int64_t* __restrict__ cell_offset, const T* __restrict__ f,
                                       double* __restrict__ eps) {
    __shared__ double red[32 * 5];
    __shared__ double tot[5];
    __shared__ float par[5];  // u0, u1, u2, 1 / (2T), norm; par[4] < 0: undefined
    __shared__ float vt[kMaxN];
    __shared__ float gt[3][kMaxN];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        const int pi = cell_plan[cell];
        if (pi < 0 || pi >= B.n_plans) {
            if (threadIdx.x == 0) eps[cell] = INFINITY;
            continue;
        }
        int d = 2, N = 1;
        double L = 1.0;
#pragma unroll
        for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
            if (q == pi) {
                d = B.p[q].d;
                N = B.p[q].N;
                L = B.p[q].L;
            }
        const double h = 2.0 * L / N;
        const int rows = d == 3 ? N * N : N;
        const T* fc = f + cell_offset[cell];
        for (int j = threadIdx.x; j < N; j += blockDim.x) vt[j] = (float)(-L + (double)j * h);
        __syncthreads();
        // pass 1: sum f, sum f v, sum f |v|^2
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, mc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int r = wid; r < rows; r += nw) {
            const int j0 = d == 3 ? r / N : r, j1 = d == 3 ? r - j0 * N : 0;
            const float a0 = vt[j0], a1 = d == 3 ? vt[j1] : 0.f, a01 = a0 * a0 + a1 * a1;
            for (int x = lane; x < N; x += 32) {
                const float fv = (float)fc[(int64_t)r * N + x], a2 = vt[x];
                comp_add<float, true>(m[0], mc[0], fv);
                comp_add<float, true>(m[1], mc[1], fv * a0);
                comp_add<float, true>(m[2], mc[2], fv * (d == 3 ? a1 : a2));
                if (d == 3) comp_add<float, true>(m[3], mc[3], fv * a2);
                comp_add<float, true>(m[4], mc[4], fv * (a01 + a2 * a2));
            }
        }
        block_sum<5>(m, mc, red, tot);
        if (threadIdx.x == 0) {
            const double hd = d == 3 ? h * h * h : h * h;
            const double rho = hd * tot[0];
            double u[3] = {0.0, 0.0, 0.0}, u2 = 0.0;
            for (int a = 0; a < d; ++a) {
                u[a] = rho != 0.0 ? hd * tot[1 + a] / rho : 0.0;
                u2 += u[a] * u[a];
            }
            const double Tt = rho != 0.0 ? (hd * tot[4] / rho - u2) / d : 0.0;
            const bool ok = rho > 0.0 && Tt > 0.0 && isfinite(rho) && isfinite(Tt);
            for (int a = 0; a < 3; ++a) par[a] = (float)u[a];
            par[3] = ok ? (float)(0.5 / Tt) : 0.f;
            par[4] = ok ? (float)(rho * pow(2.0 * kPi * Tt, -0.5 * d)) : -1.f;
        }
        __syncthreads();
        const bool ok = par[4] >= 0.f;
        // pass 2: sum |f - M|, sum |f|
        float s[2] = {0.f, 0.f}, sc[2] = {0.f, 0.f};
        if (ok) {
            for (int i = threadIdx.x; i < d * N; i += blockDim.x) {
                const int a = i / N, j = i - a * N;
                const float w = vt[j] - par[a];
                gt[a][j] = expf(-w * w * par[3]) * (a == 0 ? par[4] : 1.f);
            }
            __syncthreads();
            const float* g2 = d == 3 ? gt[2] : gt[1];
            for (int r = wid; r < rows; r += nw) {
                const int j0 = d == 3 ? r / N : r, j1 = d == 3 ? r - j0 * N : 0;
                const float row = gt[0][j0] * (d == 3 ? gt[1][j1] : 1.f);
                for (int x = lane; x < N; x += 32) {
                    const float fv = (float)fc[(int64_t)r * N + x];
                    comp_add<float, true>(s[0], sc[0], fabsf(fv - row * g2[x]));
                    comp_add<float, true>(s[1], sc[1], fabsf(fv));
                }
            }
        }
        block_sum<2>(s, sc, red, tot);
        if (threadIdx.x == 0) eps[cell] = ok && tot[1] > 0.0 ? tot[0] / tot[1] : INFINITY;
    }
}

__global__ void k_select_levels(int n_cells, const double* __restrict__ eps, const int* __restrict__ cell_base,
                                LevelTable t, int* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const int b = cell_base[c];
        if (b < 0 || b >= t.n_base) {
            out[c] = -1;
            continue;
        }
        const double e = eps[c];
        int level = 0;
        for (int k = 0; k < t.n_levels - 1; ++k) level += !(e < t.thr[k]);  // NaN counts as far
        out[c] = t.plan[b * t.n_levels + level];
    }
}

}  // namespace

extern "C" qdvm_status qdvm_equilibrium_distance(const qdvm_plan_t* plans, int n_plans, int n_cells,
                                                 const int* cell_plan, const int64_t* cell_offset, const void* f,
                                                 int prec, double* eps, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!plans || n_plans < 1 || n_plans > QDVM_MAX_BATCH_PLANS)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_plans must be in [1, QDVM_MAX_BATCH_PLANS]");
    BatchDev b;
    for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b.p[i] = PlanDev();
    b.n_plans = n_plans;
    for (int i = 0; i < n_plans; ++i) {
        if (!qdvm_plan_ok(plans[i])) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
        b.p[i] = plan_dev(plans[i]);
    }
    if (n_cells == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f || !eps) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = std::max(1, std::min(n_cells, 65535));
    if (prec == QDVM_F64)
        k_equilibrium_distance<double><<<grid, 256, 0, st>>>(b, n_cells, cell_plan, cell_offset,
                                                              static_cast<const double*>(f), eps);
    else
        k_equilibrium_distance<float><<<grid, 256, 0, st>>>(b, n_cells, cell_plan, cell_offset,
                                                             static_cast<const float*>(f), eps);
    QDVM_LAUNCH_CHECK("equilibrium distance launch");
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_select_levels(int n_cells, const double* eps, const int* cell_base, int n_base,
                                          int n_levels, const double* thresholds, const int* level_plan,
                                          int* cell_plan_out, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (n_base < 1 || n_base > QDVM_MAX_BATCH_PLANS) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_base out of range");
    if (n_levels < 1 || n_levels > QDVM_MAX_LEVELS) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_levels out of range");
    if (n_levels > 1 && !thresholds) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL thresholds");
    if (!level_plan) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL level_plan");
    LevelTable t{};
    t.n_base = n_base;
    t.n_levels = n_levels;
    for (int k = 0; k + 1 < n_levels; ++k) {
        if (!std::isfinite(thresholds[k]) || (k > 0 && !(thresholds[k] > thresholds[k - 1])))
            return qdvm_fail(QDVM_ERR_INVALID_ARG, "thresholds must be finite and strictly increasing");
        t.thr[k] = thresholds[k];
    }
    for (int i = 0; i < n_base * n_levels; ++i) {
        if (level_plan[i] < 0 || level_plan[i] >= QDVM_MAX_BATCH_PLANS)
            return qdvm_fail(QDVM_ERR_INVALID_ARG, "level_plan entry out of range");
        t.plan[i] = level_plan[i];
    }
    if (n_cells == 0) return QDVM_OK;
    if (!eps || !cell_base || !cell_plan_out) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = std::max(1, std::min((n_cells + 255) / 256, 4 * qdvm_num_sms()));
    k_select_levels<<<grid, 256, 0, st>>>(n_cells, eps, cell_base, t, cell_plan_out);
    QDVM_LAUNCH_CHECK("select levels launch");
    return QDVM_OK;
}
