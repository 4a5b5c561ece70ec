// Direct evaluation of the restricted DVM operator, one thread per output
// point, term by term: k = j e for the lines e of A_m (0 < |j| <= J_e), l in
// the offset list of e (e^perp ∩ [-Ntilde, Ntilde]^d, eq. (decDVM)), weight
// c_e.  Two boundaries:
//   periodic: the operator of eq. (DR) -- the same Q as the fast paths,
//             computed without the line/plane decomposition;
//   box:      D^tr of Section 2.3 -- a term counts only when i + k, i + l and
//             i + k + l all lie in the grid.  D^tr conserves mass, momentum
//             and energy exactly, but is not a convolution (the box test
//             couples k and l), so it has no fast form.
// Cost: one term (3 loads, 2 products) per (point, k, l).
#include <algorithm>

#include "qdvm_internal.cuh"

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st);

namespace {

constexpr int kThreadsD = 128;

// coordinate x + s: wrapped onto [0, N) (|s| < N) or -1 outside the box
template <bool BOX>
__device__ __forceinline__ int shift(int x, int s, int N) {
    int y = x + s;
    if (BOX) return (y < 0 || y >= N) ? -1 : y;
    y += y < 0 ? N : 0;
    y -= y >= N ? N : 0;
    return y;
}

template <typename T, bool KAHAN, bool BOX>
__global__ void __launch_bounds__(kThreadsD) k_direct(BatchDev B, int n_cells, const int* __restrict__ cell_plan,
                                                      const int64_t* __restrict__ cell_offset,
                                                      const T* __restrict__ f, T* __restrict__ Q) {
    for (int cell = blockIdx.y; cell < n_cells; cell += gridDim.y) {
        const int pi = cell_plan[cell];
        if (pi < 0 || pi >= B.n_plans) continue;
        PlanDev P;
#pragma unroll
        for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
            if (q == pi) P = B.p[q];
        const int N = P.N, d = P.d;
        const int total = d == 3 ? N * N * N : N * N;
        const T* fc = f + cell_offset[cell];
        T* qc = Q + cell_offset[cell];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
            // coordinates (axis 0 slowest); in 2D axis 2 is unused
            int c0, c1, c2;
            if (d == 3) {
                c0 = i / (N * N);
                c1 = (i / N) % N;
                c2 = i % N;
            } else {
                c0 = i / N;
                c1 = i % N;
                c2 = 0;
            }
            const T fi = fc[i];
            T acc = T(0), cmp = T(0);
            for (int li = 0; li < P.n_lines; ++li) {
                const int4 e = __ldg(P.lines + li);
                const T c = (T)__ldg(P.c + li);
                const int ps = __ldg(P.plane_start + li), pe = __ldg(P.plane_start + li + 1);
                for (int j = -e.w; j <= e.w; ++j) {
                    if (j == 0) continue;
                    const int k0 = shift<BOX>(c0, j * e.x, N), k1 = shift<BOX>(c1, j * e.y, N);
                    const int k2 = d == 3 ? shift<BOX>(c2, j * e.z, N) : 0;
                    if (BOX && (k0 < 0 || k1 < 0 || k2 < 0)) continue;
                    const int ik = d == 3 ? (k0 * N + k1) * N + k2 : k0 * N + k1;
                    const T fk = __ldg(fc + ik);
                    for (int t = ps; t < pe; ++t) {
                        const char4 l = __ldg(P.plane + t);
                        const int l0 = shift<BOX>(c0, l.x, N), l1 = shift<BOX>(c1, l.y, N);
                        const int l2 = d == 3 ? shift<BOX>(c2, l.z, N) : 0;
                        const int m0 = shift<BOX>(k0, l.x, N), m1 = shift<BOX>(k1, l.y, N);
                        const int m2 = d == 3 ? shift<BOX>(k2, l.z, N) : 0;
                        if (BOX && (l0 < 0 || l1 < 0 || l2 < 0 || m0 < 0 || m1 < 0 || m2 < 0)) continue;
                        const int il = d == 3 ? (l0 * N + l1) * N + l2 : l0 * N + l1;
                        const int ikl = d == 3 ? (m0 * N + m1) * N + m2 : m0 * N + m1;
                        comp_add<T, KAHAN>(acc, cmp, c * (fk * __ldg(fc + il) - fi * __ldg(fc + ikl)));
                    }
                }
            }
            qc[i] = KAHAN ? acc + cmp : acc;
        }
    }
}

template <typename T, bool KAHAN>
void launch(bool box, const BatchDev& b, int n_cells, int max_total, const int* cp, const int64_t* co, const void* f,
            void* Q, cudaStream_t st) {
    dim3 grid((max_total + kThreadsD - 1) / kThreadsD, std::max(1, std::min(n_cells, 65535)));
    if (box)
        k_direct<T, KAHAN, true><<<grid, kThreadsD, 0, st>>>(b, n_cells, cp, co, static_cast<const T*>(f),
                                                               static_cast<T*>(Q));
    else
        k_direct<T, KAHAN, false><<<grid, kThreadsD, 0, st>>>(b, n_cells, cp, co, static_cast<const T*>(f),
                                                                static_cast<T*>(Q));
}

__global__ void k_direct_single_init(int* cp, int64_t* co) {
    *cp = 0;
    *co = 0;
}

}  // namespace

extern "C" qdvm_status qdvm_eval_direct_batched(const qdvm_plan_t* plans, int n_plans, int n_cells,
                                                const int* cell_plan, const int64_t* cell_offset, const void* f,
                                                void* Q, double* moments, int prec, int boundary, void* stream) {
    if (n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_cells < 0");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (boundary != QDVM_BOUNDARY_PERIODIC && boundary != QDVM_BOUNDARY_BOX)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "boundary must be QDVM_BOUNDARY_PERIODIC or QDVM_BOUNDARY_BOX");
    if (!plans || n_plans < 1 || n_plans > QDVM_MAX_BATCH_PLANS)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "n_plans must be in [1, QDVM_MAX_BATCH_PLANS]");
    BatchDev b;
    for (int i = 0; i < QDVM_MAX_BATCH_PLANS; ++i) b.p[i] = PlanDev();
    b.n_plans = n_plans;
    int max_total = 1;
    for (int i = 0; i < n_plans; ++i) {
        if (!qdvm_plan_ok(plans[i])) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
        b.p[i] = plan_dev(plans[i]);
        const int n = plans[i]->N;
        max_total = std::max(max_total, plans[i]->d == 3 ? n * n * n : n * n);
    }
    if (n_cells == 0) return QDVM_OK;
    if (!cell_plan || !cell_offset || !f || !Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (f == Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must not alias Q");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool box = boundary == QDVM_BOUNDARY_BOX;
    if (prec == QDVM_F64) launch<double, false>(box, b, n_cells, max_total, cell_plan, cell_offset, f, Q, st);
    else if (prec == QDVM_F32_KAHAN) launch<float, true>(box, b, n_cells, max_total, cell_plan, cell_offset, f, Q, st);
    else launch<float, false>(box, b, n_cells, max_total, cell_plan, cell_offset, f, Q, st);
    QDVM_LAUNCH_CHECK("direct evaluation launch");
    if (moments) return moments_batched_launch(b, n_cells, cell_plan, cell_offset, Q, prec, moments, st);
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_eval_direct_workspace(size_t* bytes) {
    if (!bytes) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL bytes");
    *bytes = 256;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_eval_direct(qdvm_plan_t p, const void* f, void* Q, int prec, int boundary, void* ws,
                                        size_t ws_bytes, void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!ws || ws_bytes < 256) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_eval_direct");
    int* cp = static_cast<int*>(ws);
    int64_t* co = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + 128);
    k_direct_single_init<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(cp, co);
    QDVM_LAUNCH_CHECK("direct single init");
    const qdvm_plan_t plans[1] = {p};
    return qdvm_eval_direct_batched(plans, 1, 1, cp, co, f, Q, nullptr, prec, boundary, stream);
}
