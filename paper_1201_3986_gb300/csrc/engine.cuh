// Generic line/plane engine for the restricted periodized DVM operator and
// its derivatives, any d in {2, 3}, any supported N.
//
// Per line e of A_m (eq. (decDVM)) the operator needs
//   Omega_e x (i) = sum_{0<|j|<=J_e} x(i + j e)               (line window)
//   Pi_e x (i)    = sum_{l in e^perp, 0<|l|_inf<=Ntilde} x(i + l) (plane polygon;
//                   in 2D the segment along e^perp)
// and assembles, with W = Omega f, P = Pi f, V = Omega P (eq. (decD)):
//   forward  Q    += c_e [ W P - f V ]
//   JVP      dQ   += c_e [ Omega(d) P + W Pi(d) - d V - f Omega(Pi(d)) ]
//   VJP      grad += c_e [ Omega(g P) - g V + Pi( g W - Omega(g f) ) ]
// (Omega and Pi are symmetric on the torus, so the VJP is the transpose of
// the JVP).
//
// Layout: every field is stored with a periodic halo of width H = Ntilde
// along axis 0 (padded index (a0 + H) * S + rest, S = N^(d-1)), so axis-0
// offsets need no modulo; the other axes wrap with one compare.  Threads own
// columns of ZC consecutive axis-0 points at a fixed rest index: one offset
// costs one address computation and ZC loads, and a warp reads consecutive
// rest indices (distinct banks).  The field a plane sum reads is staged in
// shared memory when it fits (STAGE), otherwise read from the CTA's global
// scratch copy.  Between the phase that writes a field and the phase that
// reads it at shifted points there is a CTA barrier.
//
// Work item = (cell, chunk of lines); each CTA loops over items taken from
// an atomic counter (cells pre-ordered by cost).  The item accumulates into
// the output cell (one chunk per cell) or into a partial slot that a second
// kernel sums over chunks in a fixed order.
#pragma once

#include "qdvm_internal.cuh"

namespace eng {

enum Mode { FWD = 0, JVP = 1, VJP = 2 };
constexpr int kThreads = 512;

__device__ __forceinline__ int wrapc(int v, int N) {
    v += v < 0 ? N : 0;
    v -= v >= N ? N : 0;
    return v;
}

// rest-index offset of a displacement (d1, d2) from rest coordinates (y, x)
template <int D>
__device__ __forceinline__ int rest_off(int y, int x, int d1, int d2, int N) {
    if (D == 3) return wrapc(y + d1, N) * N + wrapc(x + d2, N);
    return wrapc(x + d1, N);
}

template <typename T, int D, int ZC>
__device__ __forceinline__ void psum(const T* src, const char4* __restrict__ pl, int pn, int z0, int y, int x, int N,
                                     int H, int S, T (&s)[ZC]) {
#pragma unroll
    for (int zc = 0; zc < ZC; ++zc) s[zc] = T(0);
    for (int t = 0; t < pn; ++t) {
        const char4 l = pl[t];
        const int o = (z0 + l.x + H) * S + rest_off<D>(y, x, l.y, l.z, N);
#pragma unroll
        for (int zc = 0; zc < ZC; ++zc) s[zc] += src[o + zc * S];
    }
}

template <typename T, int D, int ZC>
__device__ __forceinline__ void lwin(const T* src, int4 e, int z0, int y, int x, int N, int H, int S, T (&w)[ZC]) {
#pragma unroll
    for (int zc = 0; zc < ZC; ++zc) w[zc] = T(0);
    for (int j = 1; j <= e.w; ++j) {
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            const int o = (z0 + sg * j * e.x + H) * S + rest_off<D>(y, x, sg * j * e.y, sg * j * e.z, N);
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) w[zc] += src[o + zc * S];
        }
    }
}

template <typename T, int ZC>
__device__ __forceinline__ void store_pad(T* dst, int z0, int r, int N, int H, int S, const T (&v)[ZC]) {
#pragma unroll
    for (int zc = 0; zc < ZC; ++zc) {
        const int z = z0 + zc;
        const int p = (z + H) * S + r;
        dst[p] = v[zc];
        if (z < H) dst[p + N * S] = v[zc];
        if (z >= N - H) dst[p - N * S] = v[zc];
    }
}

template <typename T>
__device__ __forceinline__ void fill_pad(T* dst, const T* __restrict__ src, int N, int H, int S) {
    const int padn = (N + 2 * H) * S;
    for (int p = threadIdx.x; p < padn; p += blockDim.x) {
        const int zz = p / S;
        dst[p] = src[wrapc(zz - H, N) * S + (p - zz * S)];
    }
}

template <typename T>
__device__ __forceinline__ void copy_field(T* dst, const T* src, int n) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) dst[p] = src[p];
}

template <typename T, bool KAHAN>
__device__ __forceinline__ void acc_add(T* acc, T* cmp, int i, T t) {
    if (KAHAN) {
        T a = acc[i], c = cmp[i];
        comp_add<T, true>(a, c, t);
        acc[i] = a;
        cmp[i] = c;
    } else {
        acc[i] += t;
    }
}

// Number of (N+2H) N^(d-1) fields in a CTA's global scratch.
__host__ __device__ inline int n_fields(int mode, bool stage) {
    if (mode == FWD) return stage ? 1 : 2;  // P (+ f)
    if (mode == JVP) return 4;              // f, d, P, Pi(d)
    return 6;                               // f, g, g f, P, g P, X
}

template <typename T, bool KAHAN, int D, int ZC, bool STAGE, int MODE>
__device__ void item_body(const PlanDev& P, int lb, int le, const T* __restrict__ fcell, const T* __restrict__ acell,
                          T* stage, T* fld, T* acc, T* cmp) {
    const int N = P.N, H = P.Ntilde;
    const int S = D == 3 ? N * N : N, NN = S * N, PADN = (N + 2 * H) * S;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int n_units = (N / ZC) * S;

    T *Fp, *Dp = nullptr, *GFp = nullptr, *Pb, *Qb = nullptr, *Xb = nullptr;
    if (MODE == FWD) {
        Pb = fld;
        Fp = STAGE ? stage : fld + PADN;
    } else if (MODE == JVP) {
        Fp = fld;
        Dp = fld + PADN;
        Pb = fld + 2 * PADN;
        Qb = fld + 3 * PADN;
    } else {
        Fp = fld;
        Dp = fld + PADN;
        GFp = fld + 2 * PADN;
        Pb = fld + 3 * PADN;
        Qb = fld + 4 * PADN;
        Xb = fld + 5 * PADN;
    }
    fill_pad(Fp, fcell, N, H, S);
    if (MODE != FWD) fill_pad(Dp, acell, N, H, S);
    for (int i = tid; i < NN; i += NT) {
        acc[i] = T(0);
        if (KAHAN) cmp[i] = T(0);
    }
    __syncthreads();
    if (MODE == VJP) {
        for (int p = tid; p < PADN; p += NT) GFp[p] = Dp[p] * Fp[p];
        __syncthreads();
    }

    for (int li = lb; li < le; ++li) {
        const int4 e = P.lines[li];
        const T c = (T)P.c[li];
        const int ps = P.plane_start[li], pn = P.plane_start[li + 1] - ps;
        const char4* __restrict__ pl = P.plane + ps;

        if (MODE == FWD) {
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                T s[ZC];
                psum<T, D, ZC>(Fp, pl, pn, zb * ZC, y, x, N, H, S, s);
                store_pad<T, ZC>(Pb, zb * ZC, r, N, H, S, s);
            }
            __syncthreads();
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                const int z0 = zb * ZC;
                T W[ZC], V[ZC];
                lwin<T, D, ZC>(Fp, e, z0, y, x, N, H, S, W);
                lwin<T, D, ZC>(Pb, e, z0, y, x, N, H, S, V);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) {
                    const int ip = (z0 + zc + H) * S + r;
                    acc_add<T, KAHAN>(acc, cmp, (z0 + zc) * S + r, c * (W[zc] * Pb[ip] - Fp[ip] * V[zc]));
                }
            }
            __syncthreads();
        } else if (MODE == JVP) {
            const T* src = Fp;
            if (STAGE) {
                copy_field(stage, Fp, PADN);
                __syncthreads();
                src = stage;
            }
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                T s[ZC];
                psum<T, D, ZC>(src, pl, pn, zb * ZC, y, x, N, H, S, s);
                store_pad<T, ZC>(Pb, zb * ZC, r, N, H, S, s);
            }
            __syncthreads();
            const T* srcd = Dp;
            if (STAGE) {
                copy_field(stage, Dp, PADN);
                __syncthreads();
                srcd = stage;
            }
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                T s[ZC];
                psum<T, D, ZC>(srcd, pl, pn, zb * ZC, y, x, N, H, S, s);
                store_pad<T, ZC>(Qb, zb * ZC, r, N, H, S, s);
            }
            __syncthreads();
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                const int z0 = zb * ZC;
                T Wd[ZC], W[ZC], V[ZC], Vd[ZC];
                lwin<T, D, ZC>(srcd, e, z0, y, x, N, H, S, Wd);
                lwin<T, D, ZC>(Fp, e, z0, y, x, N, H, S, W);
                lwin<T, D, ZC>(Pb, e, z0, y, x, N, H, S, V);
                lwin<T, D, ZC>(Qb, e, z0, y, x, N, H, S, Vd);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) {
                    const int ip = (z0 + zc + H) * S + r;
                    const T t = c * (Wd[zc] * Pb[ip] + W[zc] * Qb[ip] - Dp[ip] * V[zc] - Fp[ip] * Vd[zc]);
                    acc_add<T, KAHAN>(acc, cmp, (z0 + zc) * S + r, t);
                }
            }
            __syncthreads();
        } else {  // VJP
            const T* src = Fp;
            if (STAGE) {
                copy_field(stage, Fp, PADN);
                __syncthreads();
                src = stage;
            }
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                const int z0 = zb * ZC;
                T Pv[ZC], W[ZC], Y[ZC], A[ZC], X[ZC];
                psum<T, D, ZC>(src, pl, pn, z0, y, x, N, H, S, Pv);
                lwin<T, D, ZC>(src, e, z0, y, x, N, H, S, W);
                lwin<T, D, ZC>(GFp, e, z0, y, x, N, H, S, Y);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) {
                    const T g = Dp[(z0 + zc + H) * S + r];
                    A[zc] = g * Pv[zc];
                    X[zc] = g * W[zc] - Y[zc];
                }
                store_pad<T, ZC>(Pb, z0, r, N, H, S, Pv);
                store_pad<T, ZC>(Qb, z0, r, N, H, S, A);
                store_pad<T, ZC>(Xb, z0, r, N, H, S, X);
            }
            __syncthreads();
            const T* srcx = Xb;
            if (STAGE) {
                copy_field(stage, Xb, PADN);
                __syncthreads();
                srcx = stage;
            }
            for (int u = tid; u < n_units; u += NT) {
                const int zb = u / S, r = u - zb * S, y = D == 3 ? r / N : 0, x = D == 3 ? r - y * N : r;
                const int z0 = zb * ZC;
                T PX[ZC], V[ZC], OA[ZC];
                psum<T, D, ZC>(srcx, pl, pn, z0, y, x, N, H, S, PX);
                lwin<T, D, ZC>(Pb, e, z0, y, x, N, H, S, V);
                lwin<T, D, ZC>(Qb, e, z0, y, x, N, H, S, OA);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) {
                    const T g = Dp[(z0 + zc + H) * S + r];
                    acc_add<T, KAHAN>(acc, cmp, (z0 + zc) * S + r, c * (OA[zc] - g * V[zc] + PX[zc]));
                }
            }
            __syncthreads();
        }
    }
    if (KAHAN) {
        for (int i = tid; i < NN; i += NT) acc[i] = acc[i] + cmp[i];
    }
}

template <typename T, bool KAHAN, int D, int ZC, bool STAGE, int MODE>
__global__ void __launch_bounds__(kThreads) k_engine(BatchDev B, int n_cells, int C, const int* __restrict__ cell_plan,
                                                    const int64_t* __restrict__ cell_offset,
                                                    const int* __restrict__ order, int* counter,
                                                    const T* __restrict__ f, const T* __restrict__ aux,
                                                    T* __restrict__ out, T* __restrict__ part, size_t part_stride,
                                                    char* scratch, size_t scr_stride) {
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
        const size_t S = D == 3 ? (size_t)N * N : (size_t)N;
        const size_t padn = (size_t)(N + 2 * H) * S;
        const int64_t off = cell_offset[cell];
        T* acc = C == 1 ? out + off : part + ((size_t)cell * C + chunk) * part_stride;
        T* fld = reinterpret_cast<T*>(scratch + (size_t)blockIdx.x * scr_stride);
        T* cmp = fld + n_fields(MODE, STAGE) * padn;
        T* stage = STAGE ? reinterpret_cast<T*>(smem_raw) : nullptr;
        item_body<T, KAHAN, D, ZC, STAGE, MODE>(P, lb, le, f + off, aux ? aux + off : nullptr, stage, fld, acc, cmp);
        __syncthreads();
    }
}

// Sum of the chunk partials of every cell, fixed order.
template <typename T, bool KAHAN>
__global__ void k_reduce_chunks(BatchDev B, int n_cells, int C, const int* __restrict__ cell_plan,
                                const int64_t* __restrict__ cell_offset, const T* __restrict__ part,
                                size_t part_stride, T* __restrict__ out) {
    for (int cell = blockIdx.y; cell < n_cells; cell += gridDim.y) {
        const int pi = cell_plan[cell];
        if (pi < 0 || pi >= B.n_plans) continue;
        int N = 0, d = 2;
#pragma unroll
        for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
            if (q == pi) {
                N = B.p[q].N;
                d = B.p[q].d;
            }
        const int64_t n = d == 3 ? (int64_t)N * N * N : (int64_t)N * N;
        const int64_t off = cell_offset[cell];
        const T* src = part + (size_t)cell * C * part_stride;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            T s = T(0), c = T(0);
            for (int k = 0; k < C; ++k) comp_add<T, KAHAN>(s, c, src[(size_t)k * part_stride + i]);
            out[off + i] = KAHAN ? s + c : s;
        }
    }
}

// Host side -----------------------------------------------------------------

struct Layout {
    int C, grid, zc, mode, d;
    bool stage;
    size_t smem, scr_stride, part_stride, off_scr, off_part, total;
};

// Launch / occupancy of the engine for one mode (engine_fwd.cu, engine_jvp.cu,
// engine_vjp.cu).
#define QDVM_ENGINE_DECL(sfx)                                                                                  \
    qdvm_status launch_##sfx(const Layout& g, const BatchDev& b, int n_cells, const int* cp, const int64_t* co, \
                             const int* order, int* counter, const void* f, const void* aux, void* out,         \
                             char* base, int prec, cudaStream_t st);                                            \
    int occupancy_##sfx(int prec, int d, int zc, bool stage, size_t smem);
QDVM_ENGINE_DECL(fwd)
QDVM_ENGINE_DECL(jvp)
QDVM_ENGINE_DECL(vjp)
#undef QDVM_ENGINE_DECL

}  // namespace eng
