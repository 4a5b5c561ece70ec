// Batch scheduling (cells ordered by decreasing cost, for the persistent
// evaluators) and the FP64 moment reduction of Section 2.1
// (h^d sum_i Q_i phi(v_i), phi = 1, v, |v|^2).
#include <algorithm>

#include "qdvm_internal.cuh"

namespace {

// Single block of 1024 threads (32 warps): order = cells grouped by plan,
// plans by decreasing cost (N^d x lines), cells ascending within a plan;
// cells with an out-of-range plan index are left out and the tail of order
// is filled with -1.  Also resets the work counter of the persistent
// kernels.  Two passes over cell_plan, whatever the number of plans: first
// the cells of every plan (one warp ballot per plan and 32 cells), then, per
// chunk of 1024 cells, each cell's place = its plan's next free place + the
// plan's cells in the chunk's earlier warps + its rank among its warp's
// cells of that plan.
__global__ void __launch_bounds__(1024) k_schedule(BatchDev B, int n_cells, const int* __restrict__ cell_plan,
                                                   int* __restrict__ order, int* __restrict__ counter) {
    constexpr int NP = QDVM_MAX_BATCH_PLANS;
    __shared__ int s_wc[32][NP];  // per warp and plan: cells (pass 1: all chunks; pass 2: this chunk, then places)
    __shared__ int s_base[NP];    // each plan's next free place in order
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, np = B.n_plans;
    const unsigned lt = (1u << lane) - 1u;
    int cnt = 0;  // lane r < np: cells of plan r seen by this warp
    for (int c0 = 0; c0 < n_cells; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int q = i < n_cells ? cell_plan[i] : -1;
        for (int r = 0; r < np; ++r) {
            const unsigned m = __ballot_sync(0xffffffffu, q == r);
            if (lane == r) cnt += __popc(m);
        }
    }
    if (lane < NP) s_wc[wid][lane] = cnt;
    __syncthreads();
    if (wid < np) {  // warp r: the cells of plan r over all warps
        int v = s_wc[lane][wid];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_base[wid] = v;  // the count for now
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double cost[NP];
        int rank_plan[NP];
        for (int q = 0; q < np; ++q) {
            double nd = 1.0;
            for (int a = 0; a < B.p[q].d; ++a) nd *= B.p[q].N;
            cost[q] = nd * (double)B.p[q].n_lines;
            rank_plan[q] = q;
        }
        for (int i = 1; i < np; ++i)  // insertion sort, stable, descending
            for (int j = i; j > 0 && cost[rank_plan[j]] > cost[rank_plan[j - 1]]; --j) {
                const int t = rank_plan[j];
                rank_plan[j] = rank_plan[j - 1];
                rank_plan[j - 1] = t;
            }
        int base = 0;
        for (int k = 0; k < np; ++k) {
            const int q = rank_plan[k], c = s_base[q];
            s_base[q] = base;
            base += c;
        }
        s_total = base;
        *counter = 0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < n_cells; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int q = i < n_cells ? cell_plan[i] : -1;
        int rank = 0;
        for (int r = 0; r < np; ++r) {
            const unsigned m = __ballot_sync(0xffffffffu, q == r);
            if (q == r) rank = __popc(m & lt);
            if (lane == r) s_wc[wid][r] = __popc(m);
        }
        __syncthreads();
        if (wid < np) {  // warp r: exclusive scan of plan r's counts over the warps
            const int v = s_wc[lane][wid];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int b = s_base[wid];
            s_wc[lane][wid] = b + incl - v;
            __syncwarp();
            if (lane == 31) s_base[wid] = b + incl;
        }
        __syncthreads();
        if (q >= 0 && q < np) order[s_wc[wid][q] + rank] = i;
        __syncthreads();
    }
    for (int i = s_total + threadIdx.x; i < n_cells; i += blockDim.x) order[i] = -1;
}

template <typename T>
__global__ void k_moments(int d, int N, double L, const T* __restrict__ Q, double* __restrict__ m) {
    __shared__ double red[32 * 5];
    const double h = 2.0 * L / N;
    int64_t total = (int64_t)N * N;
    if (d == 3) total *= N;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const double q = (double)Q[i];
        int64_t r = i;
        double v2 = 0.0;
        double v[3];
        for (int a = d - 1; a >= 0; --a) {
            v[a] = -L + (double)(r % N) * h;
            r /= N;
        }
        acc[0] += q;
        for (int a = 0; a < d; ++a) {
            acc[1 + a] += q * v[a];
            v2 += v[a] * v[a];
        }
        acc[d + 1] += q * v2;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
        if (lane == 0) red[wid * 5 + i] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double hd = h * h;
        if (d == 3) hd *= h;
        for (int i = 0; i < d + 2; ++i) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * 5 + i];
            m[i] = hd * s;
        }
    }
}

// One block per cell: FP64 moments of the stored Q of that cell.
template <typename T>
__global__ void k_moments_batched(BatchDev B, int n_cells, const int* __restrict__ cell_plan,
                                  const int64_t* __restrict__ cell_offset, const T* __restrict__ Q,
                                  double* __restrict__ m) {
    __shared__ double red[32 * 5];
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        const int pi = cell_plan[cell];
        if (pi < 0 || pi >= B.n_plans) continue;
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
        int64_t total = (int64_t)N * N;
        if (d == 3) total *= N;
        const T* q = Q + cell_offset[cell];
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
            const double qv = (double)q[i];
            int64_t r = i;
            double v[3], v2 = 0.0;
            for (int a = d - 1; a >= 0; --a) {
                v[a] = -L + (double)(r % N) * h;
                r /= N;
            }
            acc[0] += qv;
            for (int a = 0; a < d; ++a) {
                acc[1 + a] += qv * v[a];
                v2 += v[a] * v[a];
            }
            acc[d + 1] += qv * v2;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
            if (lane == 0) red[wid * 5 + i] = acc[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double hd = h * h;
            if (d == 3) hd *= h;
            for (int i = 0; i < d + 2; ++i) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += red[w * 5 + i];
                m[(size_t)cell * (d + 2) + i] = hd * s;
            }
        }
        __syncthreads();
    }
}

}  // namespace

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st) {
    const int grid = std::max(1, std::min(n_cells, 65535));
    if (prec == QDVM_F64)
        k_moments_batched<double><<<grid, 256, 0, st>>>(b, n_cells, cell_plan, cell_offset,
                                                         static_cast<const double*>(Q), m);
    else
        k_moments_batched<float><<<grid, 256, 0, st>>>(b, n_cells, cell_plan, cell_offset,
                                                        static_cast<const float*>(Q), m);
    QDVM_LAUNCH_CHECK("batched moments launch");
    return QDVM_OK;
}

qdvm_status schedule_launch(const BatchDev& b, int n_cells, const int* cell_plan, int* order, int* counter,
                            cudaStream_t st) {
    k_schedule<<<1, 1024, 0, st>>>(b, n_cells, cell_plan, order, counter);
    QDVM_LAUNCH_CHECK("schedule launch");
    return QDVM_OK;
}

qdvm_status moments_launch(int d, int N, double L, const void* Q, int prec, double* m, cudaStream_t st) {
    if (prec == QDVM_F64)
        k_moments<double><<<1, 256, 0, st>>>(d, N, L, static_cast<const double*>(Q), m);
    else
        k_moments<float><<<1, 256, 0, st>>>(d, N, L, static_cast<const float*>(Q), m);
    QDVM_LAUNCH_CHECK("moments launch");
    return QDVM_OK;
}
