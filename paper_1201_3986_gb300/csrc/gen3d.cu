// 3D evaluation of the restricted periodized DVM operator (eq. (decD)):
//   Q_i = sum_e c_e [ W_e(i) P_e(i) - f_i V_e(i) ],
//   W_e(i) = sum_{0<|j|<=J_e} f(i + j e)                  (alpha_p, eq. (decDVM))
//   P_e(i) = sum_{l in e^perp, 0<|l|_inf<=Ntilde} f(i + l)  (alpha'_p: the plane
//            polygon, listed per line in the plan)
//   V_e(i) = sum_{0<|j|<=J_e} P_e(i + j e)                 (beta(L,L), eq. (betaKL))
//
// Work item = (cell, chunk of lines).  The CTA copies its cell into shared
// memory with a periodic halo of width H = Ntilde along the slowest axis (so z
// offsets need no modulo; y and x wrap with one compare each) -- or into a
// global scratch copy when the cell does not fit on chip (FP64, N = 32).
// Each thread owns z-columns of ZC points at fixed (y, x): one plane offset
// costs one address computation and ZC loads, and a warp reads 32
// consecutive x, i.e. 32 distinct banks.  Per line: (A) P_e for every point,
// written with its z-halo images to a per-CTA scratch buffer; barrier;
// (B) W_e from the cell, V_e from the P buffer, and the gain/loss term added
// to the item's accumulator (the output cell itself when one item covers all
// lines, otherwise a partial slot summed afterwards in a fixed order).
#include <algorithm>

#include "qdvm_internal.cuh"

namespace {

constexpr int kThreads3 = 512;

__device__ __forceinline__ int wrapc(int v, int N) {
    v += v < 0 ? N : 0;
    v -= v >= N ? N : 0;
    return v;
}

template <typename T, bool KAHAN, int ZC>
__device__ __forceinline__ void gen3d_body(const PlanDev& P, const int lb, const int le, const T* __restrict__ fcell,
                                           T* fz /* (N+2H) N^2, smem or global */, T* __restrict__ Pz,
                                           T* __restrict__ acc, T* __restrict__ cmp) {
    const int N = P.N, H = P.Ntilde, N2 = N * N, N3 = N2 * N;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int n_units = (N / ZC) * N2;

    for (int p = tid; p < (N + 2 * H) * N2; p += NT) {
        const int zz = p / N2;
        const int r = p - zz * N2;
        fz[p] = fcell[wrapc(zz - H, N) * N2 + r];
    }
    for (int i = tid; i < N3; i += NT) {
        acc[i] = T(0);
        if (KAHAN) cmp[i] = T(0);
    }
    __syncthreads();

    for (int li = lb; li < le; ++li) {
        const int4 e = P.lines[li];
        const T c = (T)P.c[li];
        const int ps = P.plane_start[li], pn = P.plane_start[li + 1] - ps;
        const char4* __restrict__ pl = P.plane + ps;
        // (A) plane sums
        for (int u = tid; u < n_units; u += NT) {
            const int zb = u / N2;
            const int r = u - zb * N2;
            const int y = r / N, x = r - (r / N) * N, z0 = zb * ZC;
            T s[ZC];
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) s[zc] = T(0);
            for (int t = 0; t < pn; ++t) {
                const char4 l = pl[t];
                const int o = (z0 + l.x + H) * N2 + wrapc(y + l.y, N) * N + wrapc(x + l.z, N);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) s[zc] += fz[o + zc * N2];
            }
            T* dst = Pz + (z0 + H) * N2 + r;
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) {
                const int z = z0 + zc;
                dst[zc * N2] = s[zc];
                if (z < H) dst[zc * N2 + N3] = s[zc];
                if (z >= N - H) dst[zc * N2 - N3] = s[zc];
            }
        }
        __syncthreads();
        // (B) line windows of f and P, gain/loss assembly
        const int J = e.w;
        for (int u = tid; u < n_units; u += NT) {
            const int zb = u / N2;
            const int r = u - zb * N2;
            const int y = r / N, x = r - (r / N) * N, z0 = zb * ZC;
            T W[ZC], V[ZC];
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) {
                W[zc] = T(0);
                V[zc] = T(0);
            }
            for (int j = 1; j <= J; ++j) {
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    const int o = (z0 + sg * j * e.x + H) * N2 + wrapc(y + sg * j * e.y, N) * N + wrapc(x + sg * j * e.z, N);
#pragma unroll
                    for (int zc = 0; zc < ZC; ++zc) {
                        W[zc] += fz[o + zc * N2];
                        V[zc] += Pz[o + zc * N2];
                    }
                }
            }
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) {
                const int i = (z0 + zc) * N2 + r;
                const int ip = (z0 + zc + H) * N2 + r;
                const T t = c * (W[zc] * Pz[ip] - fz[ip] * V[zc]);
                if (KAHAN) {
                    T a = acc[i], cc = cmp[i];
                    comp_add<T, true>(a, cc, t);
                    acc[i] = a;
                    cmp[i] = cc;
                } else {
                    acc[i] += t;
                }
            }
        }
        __syncthreads();
    }
    if (KAHAN) {
        for (int i = tid; i < N3; i += NT) acc[i] = acc[i] + cmp[i];
    }
}

struct Gen3Layout {
    int C;             // chunks (items) per cell
    int grid;          // CTAs
    int zc;            // z-column length
    bool smem_f;       // cell on chip
    size_t smem;       // dynamic shared memory
    size_t scr_stride; // bytes of scratch per CTA
    size_t part_stride;// elements per partial slot
    size_t off_scr, off_part, total;
};

template <typename T, bool KAHAN, int ZC, bool SMEM_F>
__global__ void __launch_bounds__(kThreads3) k_gen3d(BatchDev B, int n_cells, int C, const int* __restrict__ cell_plan,
                                                     const int64_t* __restrict__ cell_offset,
                                                     const int* __restrict__ order, int* counter,
                                                     const T* __restrict__ f, T* __restrict__ Q, T* __restrict__ part,
                                                     size_t part_stride, char* scratch, size_t scr_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_cell;
    __shared__ PlanDev s_plan;
    const int n_items = n_cells * C;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            int cell = -1;
            if (it < n_items) cell = order[it / C];
            s_item = cell >= 0 ? it : -1;
            s_cell = cell;
            if (cell >= 0) {
                const int pi = cell_plan[cell];
#pragma unroll
                for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
                    if (q == pi) s_plan = B.p[q];
            }
        }
        __syncthreads();
        const int item = s_item, cell = s_cell;
        if (item < 0) break;
        const PlanDev P = s_plan;
        const int chunk = item % C;
        const int lpc = (P.n_lines + C - 1) / C;
        const int lb = min(chunk * lpc, P.n_lines), le = min(lb + lpc, P.n_lines);
        const int N = P.N, H = P.Ntilde;
        const size_t N2 = (size_t)N * N, N3 = N2 * N, fzn = (size_t)(N + 2 * H) * N2;
        const int64_t off = cell_offset[cell];
        T* acc = C == 1 ? Q + off : part + ((size_t)cell * C + chunk) * part_stride;
        T* scr = reinterpret_cast<T*>(scratch + (size_t)blockIdx.x * scr_stride);
        T* Pz = scr;
        T* cmp = scr + fzn;
        T* fz = SMEM_F ? reinterpret_cast<T*>(smem_raw) : cmp + (KAHAN ? N3 : 0);
        gen3d_body<T, KAHAN, ZC>(P, lb, le, f + off, fz, Pz, acc, cmp);
        __syncthreads();
    }
}

template <typename T, bool KAHAN>
__global__ void k_reduce_chunks(BatchDev B, int n_cells, int C, const int* __restrict__ cell_plan,
                                const int64_t* __restrict__ cell_offset, const T* __restrict__ part,
                                size_t part_stride, T* __restrict__ Q) {
    for (int cell = blockIdx.y; cell < n_cells; cell += gridDim.y) {
        const int pi = cell_plan[cell];
        if (pi < 0 || pi >= B.n_plans) continue;
        int N = 0;
#pragma unroll
        for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
            if (q == pi) N = B.p[q].N;
        const int64_t n = (int64_t)N * N * N;
        const int64_t off = cell_offset[cell];
        const T* src = part + (size_t)cell * C * part_stride;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            T s = T(0), c = T(0);
            for (int k = 0; k < C; ++k) comp_add<T, KAHAN>(s, c, src[(size_t)k * part_stride + i]);
            Q[off + i] = KAHAN ? s + c : s;
        }
    }
}

__global__ void k_single_init(int* counter, int* order, int* cell_plan, int64_t* cell_offset) {
    *counter = 0;
    *order = 0;
    *cell_plan = 0;
    *cell_offset = 0;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T, bool KAHAN, int ZC, bool SMEM_F>
int occupancy(size_t smem) {
    cudaFuncSetAttribute(k_gen3d<T, KAHAN, ZC, SMEM_F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gen3d<T, KAHAN, ZC, SMEM_F>, kThreads3, smem);
    return std::max(per, 1);
}

template <typename T, bool KAHAN>
int occupancy_rt(int zc, bool smem_f, size_t smem) {
    if (smem_f) {
        if (zc == 8) return occupancy<T, KAHAN, 8, true>(smem);
        if (zc == 4) return occupancy<T, KAHAN, 4, true>(smem);
        return occupancy<T, KAHAN, 1, true>(smem);
    }
    if (zc == 8) return occupancy<T, KAHAN, 8, false>(smem);
    if (zc == 4) return occupancy<T, KAHAN, 4, false>(smem);
    return occupancy<T, KAHAN, 1, false>(smem);
}

Gen3Layout make_layout(const BatchDev& b, int n_cells, int prec, bool single) {
    Gen3Layout g{};
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    const bool kahan = prec == QDVM_F32_KAHAN;
    int maxN = 0, maxLines = 0, zc = 8;
    size_t fzn = 0, n3 = 0;
    for (int i = 0; i < b.n_plans; ++i) {
        const int N = b.p[i].N, H = b.p[i].Ntilde;
        maxN = std::max(maxN, N);
        maxLines = std::max(maxLines, b.p[i].n_lines);
        fzn = std::max(fzn, (size_t)(N + 2 * H) * N * N);
        n3 = std::max(n3, (size_t)N * N * N);
        while (zc > 1 && N % zc) zc /= 2;
    }
    if (zc == 2) zc = 1;
    g.zc = zc;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g.smem_f = fzn * es + 4096 <= (size_t)optin;
    g.smem = g.smem_f ? fzn * es : 0;
    int per = 1;
    if (prec == QDVM_F64)
        per = occupancy_rt<double, false>(zc, g.smem_f, g.smem);
    else if (kahan)
        per = occupancy_rt<float, true>(zc, g.smem_f, g.smem);
    else
        per = occupancy_rt<float, false>(zc, g.smem_f, g.smem);
    const int slots = per * qdvm_num_sms();
    if (single)
        g.C = std::max(1, std::min(maxLines, slots));
    else
        g.C = std::max(1, std::min(maxLines, (4 * slots + std::max(n_cells, 1) - 1) / std::max(n_cells, 1)));
    if (!single && n_cells >= 2 * slots) g.C = 1;
    const long items = (long)std::max(n_cells, 1) * g.C;
    g.grid = (int)std::max(1L, std::min(items, (long)slots));
    g.scr_stride = a256((fzn + (kahan ? n3 : 0) + (g.smem_f ? 0 : fzn)) * es);
    g.part_stride = g.C > 1 ? n3 : 0;
    g.off_scr = 256 + a256((size_t)std::max(n_cells, 1) * sizeof(int)) + 256;  // counter, order, single-cell tables
    g.off_part = g.off_scr + (size_t)g.grid * g.scr_stride;
    g.total = g.off_part + (g.C > 1 ? a256((size_t)std::max(n_cells, 1) * g.C * n3 * es) : 0);
    return g;
}

template <typename T, bool KAHAN, int ZC, bool SMEM_F>
void launch_main(const Gen3Layout& g, const BatchDev& b, int n_cells, const int* cell_plan,
                 const int64_t* cell_offset, const int* order, int* counter, const T* f, T* Q, T* part, char* scr,
                 cudaStream_t st) {
    cudaFuncSetAttribute(k_gen3d<T, KAHAN, ZC, SMEM_F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    k_gen3d<T, KAHAN, ZC, SMEM_F><<<g.grid, kThreads3, g.smem, st>>>(b, n_cells, g.C, cell_plan, cell_offset, order,
                                                                      counter, f, Q, part, g.part_stride, scr,
                                                                      g.scr_stride);
}

template <typename T, bool KAHAN>
qdvm_status run(const Gen3Layout& g, const BatchDev& b, int n_cells, const int* cell_plan,
                const int64_t* cell_offset, const int* order, int* counter, const void* fv, void* Qv, char* base,
                cudaStream_t st) {
    const T* f = static_cast<const T*>(fv);
    T* Q = static_cast<T*>(Qv);
    T* part = reinterpret_cast<T*>(base + g.off_part);
    char* scr = base + g.off_scr;
    if (g.smem_f) {
        if (g.zc == 8) launch_main<T, KAHAN, 8, true>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
        else if (g.zc == 4) launch_main<T, KAHAN, 4, true>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
        else launch_main<T, KAHAN, 1, true>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
    } else {
        if (g.zc == 8) launch_main<T, KAHAN, 8, false>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
        else if (g.zc == 4) launch_main<T, KAHAN, 4, false>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
        else launch_main<T, KAHAN, 1, false>(g, b, n_cells, cell_plan, cell_offset, order, counter, f, Q, part, scr, st);
    }
    QDVM_LAUNCH_CHECK("gen3d launch");
    if (g.C > 1) {
        dim3 grid(8, std::max(1, std::min(n_cells, 65535)));
        k_reduce_chunks<T, KAHAN><<<grid, 256, 0, st>>>(b, n_cells, g.C, cell_plan, cell_offset, part, g.part_stride, Q);
        QDVM_LAUNCH_CHECK("gen3d reduce launch");
    }
    return QDVM_OK;
}

}  // namespace

int gen3d_supported(const qdvm_plan_s* p, int prec) {
    (void)prec;
    return p->d == 3;
}

size_t gen3d_workspace(const BatchDev& b, int n_cells, int prec, bool single) {
    return make_layout(b, single ? 1 : n_cells, prec, single).total;
}

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st);

qdvm_status gen3d_eval(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                       const void* f, void* Q, double* moments, int prec, void* ws, size_t ws_bytes, bool single,
                       cudaStream_t st) {
    const int nc = single ? 1 : n_cells;
    const Gen3Layout g = make_layout(b, nc, prec, single);
    if (!ws || ws_bytes < g.total) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for the 3D engine");
    char* base = static_cast<char*>(ws);
    int* counter = reinterpret_cast<int*>(base);
    int* order = reinterpret_cast<int*>(base + 256);
    if (single) {
        char* tab = base + 256 + a256(sizeof(int));
        int* cp = reinterpret_cast<int*>(tab);
        int64_t* co = reinterpret_cast<int64_t*>(tab + 128);
        k_single_init<<<1, 1, 0, st>>>(counter, order, cp, co);
        QDVM_LAUNCH_CHECK("gen3d single init");
        cell_plan = cp;
        cell_offset = co;
    } else {
        qdvm_status s = schedule_launch(b, nc, cell_plan, order, counter, st);
        if (s != QDVM_OK) return s;
    }
    qdvm_status s;
    if (prec == QDVM_F64)
        s = run<double, false>(g, b, nc, cell_plan, cell_offset, order, counter, f, Q, base, st);
    else if (prec == QDVM_F32_KAHAN)
        s = run<float, true>(g, b, nc, cell_plan, cell_offset, order, counter, f, Q, base, st);
    else
        s = run<float, false>(g, b, nc, cell_plan, cell_offset, order, counter, f, Q, base, st);
    if (s != QDVM_OK) return s;
    if (moments) return moments_batched_launch(b, nc, cell_plan, cell_offset, Q, prec, moments, st);
    return QDVM_OK;
}
