// Fused 2D evaluation of the restricted periodized DVM operator, one cell per
// CTA, everything on chip.
//
// For a pair of orthogonal lines {e, e^perp} (Remark 3.4(3): in 2D the lines
// of A_m come in such pairs, with c_e = c_{e^perp} for the unit and
// Heintz-Panferov weights), eq. (decD) contributes
//     2 c_e [ W_e(i) W_{e^perp}(i) - f_i V_e(i) ],
//     W_e(i)  = sum_{0<|j|<=J} f(i + j e)            (alpha_p of eq. (decDVM))
//     P(i)    = W_{e^perp}(i)                        (alpha'_p: e^perp ∩ box)
//     V_e(i)  = sum_{0<|j|<=J} P(i + j e)            (beta(L,L) of eq. (betaKL))
// with J = floor(Ntilde / |e|_inf) for both lines.
//
// Layout: the cell is copied into shared memory with a periodic halo of width
// 2H (H = Ntilde) on every side (padded row stride congruent to N mod 32, see
// pad2d_stride), so every window gather is base + j*step without any modulo,
// and a warp of 32 consecutive points reads 32 distinct banks for every
// direction.  Pairs with J = 1 read V_e straight from the cell at
// i +- e +- e^perp (|e +- e^perp|_inf <= 2|e|_inf <= 2H) with no barrier.  Each thread owns the points tid + k*blockDim.x and keeps their
// accumulators in registers for all pairs; P goes through shared memory
// (with its halo images) because V gathers it along e.
//
// With the loss as one FFT convolution per cell (fftloss_body), the pairs
// only sum the gain 2 c_e W_e W_{e^perp}, and the two windows of a pair come
// from one of two line-sum engines: DIRECT gathers (2J loads per point and
// line) or SCAN, segmented running sums along the orbits of e and e^perp on
// the torus (scan_walks), chosen per pair by the tuning threshold scan_j.
#pragma once

#include <algorithm>

#include "fft.cuh"
#include "qdvm_internal.cuh"

namespace {

// Deterministic block reduction of NV doubles per thread; result in out[] of
// thread 0.  Uses a fixed tree (shuffle-down, then warps in order).
template <int NV>
__device__ __forceinline__ void block_reduce_fixed(double (&v)[NV], double* red /* smem, 32*NV */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[wid * NV + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * NV + i];
            v[i] = s;
        }
    }
    __syncthreads();
}

// The FP64 moments of a cell, h^2 sum_i Q_i phi(v_i) for phi = 1, v_0, v_1,
// |v|^2 with v = -L + (y, x) h, from the integer-weighted sums
// M = sum q (1, y, x, y^2 + x^2):
//   m_0 = h^2 M0,  m_1 = h^2 (h M1 - L M0),  m_2 = h^2 (h M2 - L M0),
//   m_3 = h^2 (h^2 M3 - 2 L h (M1 + M2) + 2 L^2 M0).
// A thread sums its points in the kernel's type.  In FP32 the sums are
// compensated (each product split exactly by an fma, each sum by TwoSum),
// which is as accurate as FP64 arithmetic while keeping off the FP64 pipe
// (1/64 of the FP32 rate on this part).  In FP32 the warps also combine
// their lanes' (sum, compensation) pairs by TwoSum; one warp then adds the
// warps' pairs in FP64, and the combination above is FP64.  In FP64 the
// block reduction is a plain FP64 tree.
template <typename T>
struct CellMoments {
    T s[4], c[4];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 4; ++i) s[i] = c[i] = T(0);
    }
    __device__ __forceinline__ void add(const T q, const int y, const int x) {
        if constexpr (sizeof(T) == 4) {
            const float w[3] = {(float)y, (float)x, (float)(y * y + x * x)};  // exact integers
            comp_add<float, true>(s[0], c[0], q);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float p = q * w[i];
                c[i + 1] += fmaf(q, w[i], -p);  // the product's rounding error
                comp_add<float, true>(s[i + 1], c[i + 1], p);
            }
        } else {
            s[0] += q;
            s[1] += q * y;
            s[2] += q * x;
            s[3] += q * (double)(y * y + x * x);
        }
    }
    // SUB > 0: the block holds several cells, SUB threads each; red is the
    // group's own part of the reduction buffer and only a group with store
    // writes mom (every group reaches the barrier).
    template <int SUB = 0>
    __device__ __forceinline__ void finish(double* red, const double h, const double L, double* mom,
                                           const bool store = true) {
        double m[4];
        static_assert(SUB == 0 || sizeof(T) == 4, "sub-block moments in FP32 only");
        const int tl = SUB ? (int)(threadIdx.x % SUB) : (int)threadIdx.x;
        if constexpr (sizeof(T) == 4) {
            const int lane = tl & 31, wid = tl >> 5, nw = (SUB ? SUB : (int)blockDim.x) >> 5;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_down_sync(0xffffffffu, s[i], o);
                    const float c2 = __shfl_down_sync(0xffffffffu, c[i], o);
                    c[i] += c2;
                    comp_add<float, true>(s[i], c[i], s2);
                }
            }
            float* rf = reinterpret_cast<float*>(red);  // (sum, compensation) of warp w, moment i at 2 (4 w + i)
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    rf[2 * (4 * wid + i)] = s[i];
                    rf[2 * (4 * wid + i) + 1] = c[i];
                }
            }
            __syncthreads();
            // warp 0 alone reads red from here; every body runs barriers
            // (the cell copy's) before it writes red again for its next cell
            if (wid != 0) return;
            // lane l takes the pairs 4 w + i = l and l + 32 (i = l % 4, up
            // to 16 warps), then the lanes of one moment are added in FP64
            double v = 0.0;
            if (lane < 4 * nw) v = (double)rf[2 * lane] + (double)rf[2 * lane + 1];
            if (lane + 32 < 4 * nw) v += (double)rf[2 * (lane + 32)] + (double)rf[2 * (lane + 32) + 1];
#pragma unroll
            for (int o = 16; o >= 4; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
#pragma unroll
            for (int i = 0; i < 4; ++i) m[i] = __shfl_sync(0xffffffffu, v, i);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) m[i] = (double)s[i] + (double)c[i];
            block_reduce_fixed<4>(m, red);
        }
        if (tl == 0 && store) {
            const double h2 = h * h;
            mom[0] = h2 * m[0];
            mom[1] = h2 * (h * m[1] - L * m[0]);
            mom[2] = h2 * (h * m[2] - L * m[0]);
            mom[3] = h2 * (h * h * m[3] - 2.0 * L * h * (m[1] + m[2]) + 2.0 * L * L * m[0]);
        }
    }
};

// 2 c_e of pair pr in the kernel's type (FP32 kernels read the plan's FP32
// copy: no FP64 arithmetic per pair).
template <typename T>
__device__ __forceinline__ T pair_weight(const double* __restrict__ pair_c, const float* __restrict__ pair_c2f,
                                         const int pr) {
    if constexpr (sizeof(T) == 4) return pair_c2f[pr];
    else return 2.0 * pair_c[pr];
}

// One cell, pairs [pb, pe).  Writes Q (or a partial sum of Q) to qcell and,
// when mom != nullptr, the FP64 moments of the stored values to mom[0..3].
template <typename T, bool KAHAN, int PPT>
__device__ __forceinline__ void fused2d_body(const int N, const int H, const int4* __restrict__ pairs,
                                             const double* __restrict__ pair_c, const float* __restrict__ pair_c2f,
                                             const int pb, const int pe,
                                             const double h, const double L, const T* __restrict__ fcell,
                                             T* __restrict__ qcell, double* __restrict__ mom, T* __restrict__ sF,
                                             T* __restrict__ sP, double* red, const int jd) {
    const int RS = pad2d_stride(N, H), RF = pad2d_rows_f(N, H), HF = 2 * H;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int NN = N * N;
    // P buffer viewed in the f buffer's coordinates (P rows start H rows and
    // H columns later than f rows)
    T* const sPf = sP - (H * RS + H);

    // periodic fill of the padded cell, rows/cols [-2H, N+2H)
    for (int p = tid; p < RF * RF; p += NT) {
        const int py = p / RF, px = p - py * RF;
        int sy = py - HF, sx = px - HF;
        sy += sy < 0 ? N : 0;
        sy -= sy >= N ? N : 0;
        sx += sx < 0 ? N : 0;
        sx -= sx >= N ? N : 0;
        sF[py * RS + px] = fcell[sy * N + sx];
    }

    // per owned point: padded address (low 16 bits) and the mask of its halo
    // images (bits 16..24), or -1 when the slot is past the end of the cell
    int pk[PPT];
    T acc[PPT], cmp[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int idx = tid + k * NT;
        const int y = idx / N, x = idx - (idx / N) * N;
        int v = -1;
        if (idx < NN) {
            // image (dy, dx) of point (y, x) lies in the padded window iff the
            // shifted coordinates stay in [-H, N+H)
            const bool oy[3] = {y >= N - H, true, y < H};
            const bool ox[3] = {x >= N - H, true, x < H};
            unsigned msk = 0;
#pragma unroll
            for (int b = 0; b < 9; ++b)
                if (b != 4 && oy[b / 3] && ox[b % 3]) msk |= 1u << b;
            v = (y + HF) * RS + x + HF + (int)(msk << 16);
        }
        pk[k] = v;
        acc[k] = T(0);
        cmp[k] = T(0);
    }
    __syncthreads();

    for (int pr = pb; pr < pe; ++pr) {
        const int4 e = pairs[pr];
        const T c2 = pair_weight<T>(pair_c, pair_c2f, pr);
        const int se = e.x * RS + e.y;   // +e       (axis 0 = rows, axis 1 = columns)
        const int sp = -e.y * RS + e.x;  // +e^perp = (-e1, e0)
        const int J = e.z;
        if (J <= jd) {
            // short windows: V_e(i) = sum_{j,j'} f(i + j e + j' e^perp) read
            // directly from the cell ((2J)^2 loads, |j e + j' e^perp|_inf <= 2H)
            // -- no P buffer, no barrier
            if (J == 1) {
                const int d1 = se + sp, d2 = se - sp;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (pk[k] >= 0) {
                        const int a = pk[k] & 0xFFFF;
                        const T w = sF[a + se] + sF[a - se];
                        const T pp = sF[a + sp] + sF[a - sp];
                        const T v = (sF[a + d1] + sF[a - d1]) + (sF[a + d2] + sF[a - d2]);
                        const T t = c2 * w * pp - c2 * sF[a] * v;
                        comp_add<T, KAHAN>(acc[k], cmp[k], t);
                    }
                }
            } else {  // J == 2
                const int se2 = 2 * se, sp2 = 2 * sp;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (pk[k] >= 0) {
                        const int a = pk[k] & 0xFFFF;
                        const T w = (sF[a + se] + sF[a - se]) + (sF[a + se2] + sF[a - se2]);
                        const T pp = (sF[a + sp] + sF[a - sp]) + (sF[a + sp2] + sF[a - sp2]);
                        T v = T(0);
#pragma unroll
                        for (int j = 1; j <= 2; ++j) {
#pragma unroll
                            for (int jp = 1; jp <= 2; ++jp) {
                                const int d1 = j * se + jp * sp, d2 = j * se - jp * sp;
                                v += (sF[a + d1] + sF[a - d1]) + (sF[a + d2] + sF[a - d2]);
                            }
                        }
                        const T t = c2 * w * pp - c2 * sF[a] * v;
                        comp_add<T, KAHAN>(acc[k], cmp[k], t);
                    }
                }
            }
            continue;
        }
        // (A) W_e and P = W_{e^perp}; j outside, points inside: PPT independent
        // accumulator pairs per thread
        T W[PPT], Pv[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            W[k] = T(0);
            Pv[k] = T(0);
        }
        for (int j = 1; j <= J; ++j) {
            const int o = j * se, q = j * sp;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (pk[k] >= 0) {
                    const int a = pk[k] & 0xFFFF;
                    W[k] += sF[a + o] + sF[a - o];
                    Pv[k] += sF[a + q] + sF[a - q];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (pk[k] >= 0) {
                const int a = pk[k] & 0xFFFF;
                sPf[a] = Pv[k];
                unsigned msk = (unsigned)pk[k] >> 16;
                while (msk) {
                    const int b = __ffs(msk) - 1;
                    msk &= msk - 1;
                    sPf[a + (b / 3 - 1) * N * RS + (b % 3 - 1) * N] = Pv[k];
                }
                W[k] = c2 * W[k] * Pv[k];  // gain, 2 c_e W_e W_{e^perp}
                Pv[k] = T(0);
            }
        }
        __syncthreads();
        // (B) V_e = window of P along e; loss 2 c_e f V_e
        for (int j = 1; j <= J; ++j) {
            const int o = j * se;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (pk[k] >= 0) {
                    const int a = pk[k] & 0xFFFF;
                    Pv[k] += sPf[a + o] + sPf[a - o];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (pk[k] >= 0) {
                const int a = pk[k] & 0xFFFF;
                const T t = W[k] - c2 * sF[a] * Pv[k];
                comp_add<T, KAHAN>(acc[k], cmp[k], t);
            }
        }
        __syncthreads();
    }

    CellMoments<T> cm;
    cm.init();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int idx = tid + k * NT;
        if (idx < NN) {
            const T q = KAHAN ? acc[k] + cmp[k] : acc[k];
            qcell[idx] = q;
            if (mom) cm.add(q, idx / N, idx - (idx / N) * N);
        }
    }
    if (mom) cm.finish(red, h, L, mom);
}

// Cell body specialised for a compile-time N and H = Ntilde (the common cell
// sizes with the default truncation).  Thread t owns column x = t mod N and
// rows y0 + k R (R = rows per step), so its k-th point sits k*R*stride words
// after its first: one address add per window offset serves all of the
// thread's points, each gather being a load with an immediate offset.
template <int N, int H>
struct Geo2 {
    static constexpr int HF = 2 * H;
    static constexpr int W = N + 4 * H;
    static constexpr int RS = W + (((N % 32) - (W % 32) + 32) % 32);
};

template <typename T, bool KAHAN, int N, int H, int NT>
__device__ __forceinline__ void fixed_body(const int4* __restrict__ pairs, const double* __restrict__ pair_c,
                                           const float* __restrict__ pair_c2f, const int pb, const int pe, const double h, const double L,
                                           const T* __restrict__ fcell, T* __restrict__ qcell,
                                           double* __restrict__ mom, T* __restrict__ sF, T* __restrict__ sP,
                                           double* red, const int jd) {
    using G = Geo2<N, H>;
    constexpr int RS = G::RS, HF = G::HF, WF = G::W;
    constexpr int R = (NT / N < N) ? NT / N : N;  // rows per step
    constexpr int PPT = (N + R - 1) / R;          // points per thread
    constexpr int ACT = R * N;                    // threads that own points
    constexpr int DK = R * RS;                    // address step between a thread's points
    constexpr bool PARTIAL = (N % R) != 0;
    static_assert(pad2d_rows_f(N, H) == WF, "layout");
    const int tid = threadIdx.x;
    T* const sPf = sP - (H * RS + H);

    for (int p = tid; p < WF * WF; p += NT) {
        const int py = p / WF, px = p - py * WF;
        int sy = py - HF, sx = px - HF;
        sy += sy < 0 ? N : 0;
        sy -= sy >= N ? N : 0;
        sx += sx < 0 ? N : 0;
        sx -= sx >= N ? N : 0;
        sF[py * RS + px] = fcell[sy * N + sx];
    }
    const bool active = tid < ACT;
    const int x = tid % N, y0 = tid / N;
    const int a0 = (y0 + HF) * RS + x + HF;
    const bool last_ok = !PARTIAL || (y0 + (PPT - 1) * R < N);
    const int ax = x < H ? N : (x >= N - H ? -N : 0);  // column image offset of P
    T acc[PPT], cmp[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        acc[k] = T(0);
        cmp[k] = T(0);
    }
    __syncthreads();

    for (int pr = pb; pr < pe; ++pr) {
        const int4 e = pairs[pr];
        const T c2 = pair_weight<T>(pair_c, pair_c2f, pr);
        const int se = e.x * RS + e.y;
        const int sp = -e.y * RS + e.x;
        const int J = e.z;
        if (J <= jd) {
            if (active) {
                T w[PPT], pp[PPT], v[PPT];
#pragma unroll
                for (int k = 0; k < PPT; ++k) w[k] = pp[k] = v[k] = T(0);
                const T* b;
#define QDVM_GATHER(arr, off)                                                           \
    b = sF + a0 + (off);                                                                \
    _Pragma("unroll") for (int k = 0; k < PPT; ++k) if (k < PPT - 1 || last_ok) arr[k] += b[k * DK];
                for (int j = 1; j <= J; ++j) {
                    QDVM_GATHER(w, j * se)
                    QDVM_GATHER(w, -j * se)
                    QDVM_GATHER(pp, j * sp)
                    QDVM_GATHER(pp, -j * sp)
                    for (int jp = 1; jp <= J; ++jp) {
                        QDVM_GATHER(v, j * se + jp * sp)
                        QDVM_GATHER(v, -j * se - jp * sp)
                        QDVM_GATHER(v, j * se - jp * sp)
                        QDVM_GATHER(v, -j * se + jp * sp)
                    }
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (k < PPT - 1 || last_ok) {
                        const T t = c2 * w[k] * pp[k] - c2 * sF[a0 + k * DK] * v[k];
                        comp_add<T, KAHAN>(acc[k], cmp[k], t);
                    }
                }
            }
            continue;
        }
        // (A) W_e and P = W_{e^perp} into registers and the P buffer
        T W[PPT], Pv[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) W[k] = Pv[k] = T(0);
        if (active) {
            const T* b;
            for (int j = 1; j <= J; ++j) {
                QDVM_GATHER(W, j * se)
                QDVM_GATHER(W, -j * se)
                QDVM_GATHER(Pv, j * sp)
                QDVM_GATHER(Pv, -j * sp)
            }
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (k < PPT - 1 || last_ok) {
                    const int y = y0 + k * R;
                    const int a = a0 + k * DK;
                    const int ay = y < H ? N * RS : (y >= N - H ? -N * RS : 0);
                    sPf[a] = Pv[k];
                    if (ay) sPf[a + ay] = Pv[k];
                    if (ax) sPf[a + ax] = Pv[k];
                    if (ay && ax) sPf[a + ay + ax] = Pv[k];
                    W[k] = c2 * W[k] * Pv[k];
                    Pv[k] = T(0);
                }
            }
        }
        __syncthreads();
        // (B) V_e = window of P along e
        if (active) {
            const T* b;
            for (int j = 1; j <= J; ++j) {
                b = sPf + a0 + j * se;
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (k < PPT - 1 || last_ok) Pv[k] += b[k * DK];
                b = sPf + a0 - j * se;
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (k < PPT - 1 || last_ok) Pv[k] += b[k * DK];
            }
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (k < PPT - 1 || last_ok) {
                    const T t = W[k] - c2 * sF[a0 + k * DK] * Pv[k];
                    comp_add<T, KAHAN>(acc[k], cmp[k], t);
                }
            }
        }
        __syncthreads();
    }
#undef QDVM_GATHER

    CellMoments<T> cm;
    cm.init();
    if (active) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (k < PPT - 1 || last_ok) {
                const int y = y0 + k * R;
                const T q = KAHAN ? acc[k] + cmp[k] : acc[k];
                qcell[y * N + x] = q;
                if (mom) cm.add(q, y, x);
            }
        }
    }
    if (mom) cm.finish(red, h, L, mom);
}

// ------------------------------------------------------------------------
// Loss as one convolution (the paper's remark that the loss part is a plain
// convolution): sum_e c_e V_e(i) = sum_m K(m) f(i + m) = (K * f)(i), K the
// weighted displacement histogram of the terms (plan table, transformed).
// An on-chip 2D FFT (Stockham, mixed radix 4/6/8, ping-pong between two
// N x (N+1) complex buffers) gives K * f for the whole cell; the pair loop
// then only sums the gain 2 c_e W_e W_{e^perp} -- no P buffer, no barrier.

// One Stockham pass of radix R over all N lines (rows, or columns with
// COLS), NS = product of the radices already applied.  Butterfly b works on
// line b % N, so a warp touches consecutive lines (row stride LD = N + 1
// complex: no bank conflicts on columns or rows).
// KH = 1: multiply each output by the real factor kh at its mode (row-major
// N x N), used on the last forward pass to apply the loss kernel's transform;
// KH = 2: by the complex factor kh + i dw[row frequency] instead; KH = 3: by
// kh + i dw[column frequency].
// SUB > 0: the block works on several cells at once, SUB threads per cell;
// each group transforms its own buffers (the barriers stay block-wide).
template <typename C, int N, int LD, int R, int NS, bool INV, bool COLS, int KH = 0, int SUB = 0>
__device__ __forceinline__ void fft_pass(const C* __restrict__ src, C* __restrict__ dst, const C* __restrict__ tw,
                                         const decltype(C::x)* __restrict__ kh = nullptr,
                                         const decltype(C::x)* __restrict__ dw = nullptr) {
    constexpr int NB = N / R;
    const int t0 = SUB ? (int)(threadIdx.x % SUB) : (int)threadIdx.x;
    const int nt = SUB ? SUB : (int)blockDim.x;
    for (int b = t0; b < N * NB; b += nt) {
        const int line = b % N, j = b / N;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * NB;
            v[r] = src[COLS ? e * LD + line : line * LD + e];
        }
        const int jm = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C w = tw[(jm * (N / (NS * R)) * r) % N];
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
        dft_small<R, INV>(v);
        const int idxD = (j / NS) * NS * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = idxD + r * NS;
            if constexpr (KH == 1) {
                const auto k = kh[COLS ? e * N + line : line * N + e];
                v[r].x *= k;
                v[r].y *= k;
            } else if constexpr (KH == 2 || KH == 3) {
                const auto k = kh[COLS ? e * N + line : line * N + e];
                const auto dd = dw[(KH == 2) == COLS ? e : line];
                const auto re = v[r].x * k - v[r].y * dd;
                v[r].y = v[r].x * dd + v[r].y * k;
                v[r].x = re;
            }
            dst[COLS ? e * LD + line : line * LD + e] = v[r];
        }
    }
}

template <typename C, int N, int LD, bool INV, bool COLS, int KH, int SUB, int NS, int R, int... Rs>
__device__ __forceinline__ C* fft_passes(C* a, C* b, const C* tw, const decltype(C::x)* kh,
                                         const decltype(C::x)* dw) {
    fft_pass<C, N, LD, R, NS, INV, COLS, sizeof...(Rs) == 0 ? KH : 0, SUB>(a, b, tw, kh, dw);
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0)
        return fft_passes<C, N, LD, INV, COLS, KH, SUB, NS * R, Rs...>(b, a, tw, kh, dw);
    else
        return b;
}

// All N line transforms of length N; returns the buffer holding the result.
// KH: the last pass also multiplies by kh (1) or kh + i dw (2, 3) (see fft_pass).
template <typename C, int N, int LD, bool INV, bool COLS, int KH = 0, int SUB = 0>
__device__ __forceinline__ C* fft_lines(C* a, C* b, const C* tw, const decltype(C::x)* kh = nullptr,
                                        const decltype(C::x)* dw = nullptr) {
    if constexpr (N == 64) return fft_passes<C, N, LD, INV, COLS, KH, SUB, 1, 8, 8>(a, b, tw, kh, dw);
    else if constexpr (N == 48) return fft_passes<C, N, LD, INV, COLS, KH, SUB, 1, 6, 8>(a, b, tw, kh, dw);
    else if constexpr (N == 32) return fft_passes<C, N, LD, INV, COLS, KH, SUB, 1, 4, 8>(a, b, tw, kh, dw);
    else return fft_passes<C, N, LD, INV, COLS, KH, SUB, 1, 4, 4>(a, b, tw, kh, dw);  // N == 16
}

// The first pass (NS = 1, no twiddles) of a transform that reads a stored
// spectrum src and multiplies each input by mul(row frequency, column
// frequency) before the butterflies; dst receives the pass's output.
template <typename C, int N, int LD, int R, bool INV, bool COLS, typename Mul>
__device__ __forceinline__ void fft_pass_mul(const C* __restrict__ src, C* __restrict__ dst, Mul mul) {
    constexpr int NB = N / R;
    for (int b = threadIdx.x; b < N * NB; b += blockDim.x) {
        const int line = b % N, j = b / N;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * NB;
            v[r] = cmul(src[COLS ? e * LD + line : line * LD + e], COLS ? mul(e, line) : mul(line, e));
        }
        dft_small<R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j * R + r;
            dst[COLS ? e * LD + line : line * LD + e] = v[r];
        }
    }
}

template <typename C, int N, int LD, int R, int... Rs, typename Mul>
__device__ __forceinline__ C* icols_from(const C* F, C* A, C* B, const C* tw, Mul mul) {
    fft_pass_mul<C, N, LD, R, true, true>(F, A, mul);
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0)
        return fft_passes<C, N, LD, true, true, 0, 0, R, Rs...>(A, B, tw, nullptr, nullptr);
    else
        return A;
}

// The inverse 2D transform of mul(xi) * F (F a stored spectrum, left
// unchanged) through the buffers A and B: the first column pass reads F
// and writes A, the other passes ping-pong.  With an even number of passes
// in all, the result is always in B.
template <typename C, int N, int LD, typename Mul>
__device__ __forceinline__ C* ifft2_from(const C* F, C* A, C* B, const C* tw, Mul mul) {
    C* r;
    if constexpr (N == 64) r = icols_from<C, N, LD, 8, 8>(F, A, B, tw, mul);
    else if constexpr (N == 48) r = icols_from<C, N, LD, 6, 8>(F, A, B, tw, mul);
    else if constexpr (N == 32) r = icols_from<C, N, LD, 4, 8>(F, A, B, tw, mul);
    else r = icols_from<C, N, LD, 4, 4>(F, A, B, tw, mul);  // N == 16
    return fft_lines<C, N, LD, true, false>(r, r == A ? B : A, tw);
}

// The points a thread owns in the FFT body.  By default rows y0 + k R of
// column x (R = NT / N rows per step, the last point predicated off where R
// does not divide N).  For 48^2 cells on 256 threads, where that would leave
// 16 threads idle and some warps one point short, each thread owns a 3 x 3
// tile of points 16 apart instead: (y0 + 16 a, x + 16 b), y0, x < 16,
// 256 x 9 = 48^2.  A warp then covers two rows of 16 consecutive points,
// which with a row stride of 16 (mod 32) words hit distinct banks.  With VEC
// (FP32 cells of 32^2 and 64^2) a thread owns pairs of neighbouring points
// (y0 + m R, x + c), x even, c = 0, 1 (point k = 2 m + c), so that every
// gather reads the two values of a pair with one 8-byte load; a warp's 32
// pairs are 64 consecutive points of a row, or two rows of 32.  STAIR (VEC
// with an even number NP >= 4 of pairs per thread): the pairs of a thread
// climb the diagonal instead, pair m at (y0 + m, x + m + c), y0 = NP g for
// the thread's row group g, so that they lie on two lines of direction
// (1,1), which the diagonal pair's window walks as a running sum.  Their
// columns reach XR = NP - 1 past the row's end (read from the cell's
// halo, taken modulo N for the FFT buffers and the output).
template <int N, int NT, bool VEC = false>
struct PointMap {
    static constexpr bool TILE = !VEC && N == 48 && NT == 256;
    static constexpr int XW = VEC ? N / 2 : N;  // threads per row
    static constexpr int R = TILE ? 16 : ((NT / XW < N) ? NT / XW : N);
    static constexpr int PPT = TILE ? 9 : (VEC ? 2 : 1) * ((N + R - 1) / R);
    static constexpr int ACT = TILE ? NT : R * XW;  // threads that own points
    static constexpr bool PARTIAL = !TILE && (N % R) != 0;
    static constexpr bool STAIR = VEC && N % R == 0 && N / R >= 4 && (N / R) % 2 == 0;
    static constexpr int XR = STAIR ? N / R - 1 : 0;
    __host__ __device__ static constexpr int dy(int k) {
        return TILE ? (k / 3) * 16 : (STAIR ? k / 2 : (VEC ? (k / 2) * R : k * R));
    }
    __host__ __device__ static constexpr int dx(int k) {
        return TILE ? (k % 3) * 16 : (STAIR ? k / 2 + k % 2 : (VEC ? k % 2 : 0));
    }
    __device__ static int x0(int tid) { return TILE ? tid % 16 : (VEC ? 2 * (tid % XW) : tid % N); }
    __device__ static int y0(int tid) { return TILE ? tid / 16 : (STAIR ? (tid / XW) * (N / R) : tid / XW); }
};

// Layouts of the FFT body.  Without the SCAN engine: the cell with a
// periodic halo of width H (all the direct gathers need), then two
// N x (N+1) complex FFT buffers.  With it: a running-sum segment reaches
// (S - 1 + 2J)|e|_inf <= 4H rows or columns across, so the cell carries a
// 2H halo, followed by the two N x N window fields; the FFT buffers of the
// loss phase alias both (a cell of 64^2 FP32 fits twice per SM either way).
// XR > 0 (the STAIR point map): XR more halo columns on the right, and an
// odd row stride, so that a step along (1,1), RS + 1 words, keeps the
// parity of an address and all pairs of a thread share one alignment.
template <int N, int H, bool SCAN, int XR = 0>
struct GeoF {
    static constexpr int HW = SCAN ? 2 * H : H;  // halo width of the cell copy
    static constexpr int W = N + 2 * HW;         // rows (and columns without XR)
    static constexpr int RS = XR ? ((W + XR) | 1) : W + (((N % 32) - (W % 32) + 32) % 32);
    static constexpr int LD = N + 1;
};

template <typename T, int N, int H, bool SCAN, int XR = 0>
__host__ __device__ constexpr size_t cell_bytes() {
    return ((size_t)GeoF<N, H, SCAN, XR>::W * GeoF<N, H, SCAN, XR>::RS * sizeof(T) + 15) / 16 * 16;
}
// the extra halo columns of the FFT body's cell for NT threads (no SCAN)
template <typename T, int N, int NT>
__host__ __device__ constexpr int body_xr() {
    return PointMap<N, NT, sizeof(T) == 4 && (N == 32 || N == 64)>::XR;
}

// floor(a / D) from the plan's magic number m = ceil(2^32 / D) (m = 0 for
// D = 1), exact for the small non-negative a of the strip enumeration.
__device__ __forceinline__ int strip_div(const int a, const unsigned m) {
    return m ? (int)__umulhi((unsigned)a, m) : a;
}

// Scan engine, one piece of direction v = (v0, v1), v0 > 0 (plan table
// pair_scan: da = (v0, v1, S, npg), db = (lo, ng, magic npg, magic v0)):
// piece uu starts on row y (one of the first v0 rows of strip k, rows
// [k S v0, (k + 1) S v0)) at column x = lo + (uu mod npg) and takes up to S
// steps of v, carrying the running sum R = sum_{|j| <= J} f(. + j v) (the
// window W_v plus the centre): the first sum costs 2J + 1 loads, each further
// step one load ahead and one behind.  R is stored at the points of the
// piece that lie in the cell (out, N x N row-major); the others, left or
// right of the cell, only carry the sum.  Consecutive pieces start at
// consecutive columns of one row, so a warp's loads and stores hit distinct
// banks at every step.  The loads stay inside the cell's 2H halo because the
// plan keeps (S - 1 + J)|v1| <= 2H and J v0 <= H.
template <typename T, int N, int H>
__device__ __forceinline__ void strip_walk(const T* __restrict__ sF, T* __restrict__ out, const int4 da,
                                           const int4 db, const int J, const int uu) {
    using G = GeoF<N, H, true>;
    constexpr int RS = G::RS, HW = G::HW;
    const int v0 = da.x, v1 = da.y, S = da.z, npg = da.w;
    const int g = strip_div(uu, (unsigned)db.z);
    const int k = strip_div(g, (unsigned)db.w);
    const int y = k * S * v0 + (g - k * v0);
    const int x = db.x + (uu - g * npg);
    const int steps = min(S, strip_div(N - 1 - y, (unsigned)db.w) + 1);
    const int sv = v0 * RS + v1, ov = v0 * N + v1;
    const T* c = sF + (y + HW) * RS + (x + HW);
    T R0 = c[0], R1 = T(0);
#pragma unroll 4
    for (int j = 1; j <= J; ++j) {
        R0 += c[j * sv];
        R1 += c[-j * sv];
    }
    T R = R0 + R1;
    T* o = out + (y * N + x);
    int xc = x;
    if ((unsigned)xc < (unsigned)N) *o = R;
    const T* lead = c + (J + 1) * sv;
    const T* trail = c - J * sv;
#pragma unroll 4
    for (int t = 1; t < steps; ++t) {
        R += *lead - *trail;
        lead += sv;
        trail += sv;
        o += ov;
        xc += v1;
        if ((unsigned)xc < (unsigned)N) *o = R;
    }
}

// SCAN: pairs with J >= scan_j take the SCAN engine (the caller instantiates
// SCAN = true only when some pair of the cell does); the others, and every
// pair when !SCAN, gather their windows directly.
// FWIN (without SCAN): the FFT window engine.  The spectrum fhat of the cell
// stays in the cell's place while every pair with J >= scan_j takes one
// inverse transform of fhat (D_J(e.xi) + i D_J(e^perp.xi)), which returns
// W_e + i W_{e^perp} (both real: f is real and the window transforms even),
// and the loss takes one of fhat Ktilde; the cell is copied afterwards for
// the direct gathers of the remaining pairs.
// SUB > 0 (small FP32 cells, see cell_groups): the block evaluates several cells
// at once, SUB = NT threads each with their own shared memory; store is
// false for a group without a cell of its own (it runs on another group's
// data so that every barrier is reached, and writes nothing).
template <typename T, bool KAHAN, int N, int H, int NT, bool SCAN, int SUB = 0>
__device__ __forceinline__ void fftloss_body(const PlanDev& P, const int pb, const int pe, const T* __restrict__ fcell,
                                             T* __restrict__ qcell, double* __restrict__ mom, unsigned char* smem,
                                             double* red, const bool do_loss, const int scan_j, const bool wfft,
                                             const bool fwin = false, const bool store = true) {
    using C = typename Cplx<T>::type;
    // FP32 cells of 32^2 and 64^2 without SCAN: pairs of neighbouring points
    // per thread, gathered with 8-byte loads (PointMap)
    constexpr bool VEC = !SCAN && sizeof(T) == 4 && (N == 32 || N == 64);
    using PM = PointMap<N, NT, VEC>;
    constexpr int PPT = PM::PPT, XR = PM::XR;
    using G = GeoF<N, H, SCAN, XR>;
    constexpr int W = G::W, RS = G::RS, HW = G::HW, LD = G::LD;
    // the parity of a0 (x, y0 and, with an even stride, RS are even; with
    // STAIR, RS is odd and a0 = (y0 + HW) RS + x + HW is even)
    constexpr int A0P = PM::STAIR ? 0 : (HW & 1);
    static_assert(SUB == 0 || (SUB == NT && !SCAN), "a sub-block body is the plain FFT body");
    const int tid = SUB ? (int)(threadIdx.x % SUB) : (int)threadIdx.x;
    // with VEC: the cell shifted by one word, sS[i] = sF[i + 1], so that a
    // pair of points whose gather address is odd loads its two values with
    // one aligned 8-byte load from sS.  VEC without the FFT window engine
    // (late): the cell and sS are written after the loss transform, from the
    // f values each thread holds in registers, so that they alias the FFT
    // buffers (sF and A at 0, sS at the cell's size, B at N LD complex;
    // body_smem).  Otherwise the FFT buffers follow the cell, and sS (VEC)
    // takes their place once the loss transform is done.
    constexpr size_t CB = cell_bytes<T, N, H, SCAN, XR>();
    const bool late = VEC && !fwin;
    T* sF = reinterpret_cast<T*>(smem);
    T* sRe = reinterpret_cast<T*>(smem + CB);
    T* sRp = sRe + N * N;
    C* A = reinterpret_cast<C*>((SCAN || late) ? smem : smem + CB);
    C* B = A + N * LD;
    T* sS = late ? reinterpret_cast<T*>(smem + CB) : reinterpret_cast<T*>(A);
    static_assert(!VEC || W * RS <= 4 * N * LD, "the shifted cell fits in the FFT buffers");
    static_assert(!VEC || (N * N) % NT == 0, "the cell's points split evenly over the threads");
    static_assert(!VEC || (PM::STAIR ? RS % 2 == 1 : (RS % 2 == 0 && (PM::R * RS) % 2 == 0)),
                  "the strides keep the pairs of a thread at one alignment");
    static_assert(2 * HW + XR < N, "one periodic image per axis");
    const C* tw;
    const T* kh;
    if constexpr (sizeof(T) == 8) {
        tw = reinterpret_cast<const C*>(P.tw);
        kh = reinterpret_cast<const T*>(P.khat);
    } else {
        tw = reinterpret_cast<const C*>(P.tw_f);
        kh = reinterpret_cast<const T*>(P.khat_f);
    }

    const bool active = tid < PM::ACT;
    const int x = PM::x0(tid), y0 = PM::y0(tid);  // the thread's first point; point k at + (dy(k), dx(k))
    const int a0 = (y0 + HW) * RS + x + HW;
    // the column of point k in [0, N) (a STAIR run may pass the row's end)
    auto colk = [&](const int k) {
        const int c = x + PM::dx(k);
        return (PM::STAIR && c >= N) ? c - N : c;
    };
    const bool last_ok = !PM::PARTIAL || (y0 + PM::dy(PPT - 1) < N);
    T acc[PPT], cmp[PPT];

    // VEC: add the values at +-off from every owned pair to arr.  The
    // address of pair m, a0 + off + dy RS + dx, has the parity of A0P + off
    // for every m: even, an aligned 8-byte load from the cell; odd, from sS.
    auto vgather = [&](T (&arr)[PPT], const int off) {
        if constexpr (VEC) {
            const bool al = ((A0P + off) & 1) == 0;
            const T* bp = al ? sF + a0 + off : sS + a0 + off - 1;
            const T* bm = al ? sF + a0 - off : sS + a0 - off - 1;
#pragma unroll
            for (int m = 0; m < PPT / 2; ++m) {
                const C u = *reinterpret_cast<const C*>(bp + PM::dy(2 * m) * RS + PM::dx(2 * m));
                const C v = *reinterpret_cast<const C*>(bm + PM::dy(2 * m) * RS + PM::dx(2 * m));
                arr[2 * m] += u.x + v.x;
                arr[2 * m + 1] += u.y + v.y;
            }
        }
    };

    // the direct gathers of the gain's two windows, 2 c_e W_e W_{e^perp}
    auto gain_direct = [&](const int4 e, const T c2) {
        const int se = e.x * RS + e.y;
        const int sp = -e.y * RS + e.x;
        T w[PPT], pp[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) w[k] = pp[k] = T(0);
        if constexpr (VEC) {
            for (int j = 1; j <= e.z; ++j) {
                vgather(w, j * se);
                vgather(pp, j * sp);
            }
        } else {
            const T* b;
            for (int j = 1; j <= e.z; ++j) {
#define QDVM_GATHER(arr, off)                                                                \
    b = sF + a0 + (off);                                                                     \
    _Pragma("unroll") for (int k = 0; k < PPT; ++k) if (k < PPT - 1 || last_ok) arr[k] += b[PM::dy(k) * RS + PM::dx(k)];
                QDVM_GATHER(w, j * se)
                QDVM_GATHER(w, -j * se)
                QDVM_GATHER(pp, j * sp)
                QDVM_GATHER(pp, -j * sp)
#undef QDVM_GATHER
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k)
            if (k < PPT - 1 || last_ok) comp_add<T, KAHAN>(acc[k], cmp[k], c2 * w[k] * pp[k]);
    };
    // STAIR: the gain of the diagonal pair (|e_1| = |e_2| = 1, J = H).  The
    // thread's pairs P_0 .. P_{NP-1} lie on one run along (1,1), P_i the
    // pair at a0 + i (RS + 1), so their windows along (1,1) come from one
    // running sum, R_0 = P_{-H} + ... + P_H, R_m = R_{m-1} + P_{m+H} - P_{m-1-H},
    // W_m = R_m - P_m: 2H + 2NP - 1 loads where direct gathers take 2H NP.
    // The window along (1,-1) is gathered directly.
    auto gain_diag = [&](const T c2) {
        if constexpr (PM::STAIR) {
            constexpr int NP = PPT / 2, D = RS + 1;
            T w[PPT], pp[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) w[k] = pp[k] = T(0);
            for (int j = 1; j <= H; ++j) vgather(pp, j * (RS - 1));
            auto ld = [&](const int i) { return *reinterpret_cast<const C*>(sF + a0 + i * D); };  // a0 even
            T rx = T(0), ry = T(0);
#pragma unroll
            for (int i = -H; i <= H; ++i) {
                const C u = ld(i);
                rx += u.x;
                ry += u.y;
                if (i >= 0 && i < NP) {
                    w[2 * i] -= u.x;
                    w[2 * i + 1] -= u.y;
                }
            }
            w[0] += rx;
            w[1] += ry;
#pragma unroll
            for (int m = 1; m < NP; ++m) {
                const C a = ld(m + H), b = ld(m - 1 - H);
                rx += a.x - b.x;
                ry += a.y - b.y;
                if (m + H < NP) {
                    w[2 * (m + H)] -= a.x;
                    w[2 * (m + H) + 1] -= a.y;
                }
                w[2 * m] += rx;
                w[2 * m + 1] += ry;
            }
#pragma unroll
            for (int k = 0; k < PPT; ++k) comp_add<T, KAHAN>(acc[k], cmp[k], c2 * w[k] * pp[k]);
        }
    };
    // DIRECT gathers for pair e, or the running sum for the diagonal pair
    auto gain_pair = [&](const int4 e, const T c2) {
        if (PM::STAIR && abs(e.x) == 1 && abs(e.y) == 1 && e.z == H) gain_diag(c2);
        else gain_direct(e, c2);
    };
    // the loss -f (K * f) from the FFT buffers A, B (K's transform in kh);
    // fk(k) gives f at the k-th owned point.  With dw (the axis window's
    // transform, scaled by a power of two s to the size of Ktilde) the
    // spectrum is multiplied by Ktilde + i s D instead, and the returned
    // buffer holds K * f + i s W_(1,0): both are real, so one inverse
    // transform carries the two, and with parts of one size the rounding of
    // each stays relative to itself.
    auto loss_fft = [&](auto fk, const T* dw) {
        C* r = fft_lines<C, N, LD, false, false, 0, SUB>(A, B, tw);
        if (dw)  // times Ktilde + i s D: D at the row frequency (W_(1,0)), with SCAN at the column one (W_(0,1))
            r = fft_lines<C, N, LD, false, true, SCAN ? 3 : 2, SUB>(r, r == A ? B : A, tw, kh, dw);
        else
            r = fft_lines<C, N, LD, false, true, 1, SUB>(r, r == A ? B : A, tw, kh);  // times Ktilde
        r = fft_lines<C, N, LD, true, true, 0, SUB>(r, r == A ? B : A, tw);
        r = fft_lines<C, N, LD, true, false, 0, SUB>(r, r == A ? B : A, tw);
        if (active) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (k < PPT - 1 || last_ok) acc[k] = -fk(k) * r[(y0 + PM::dy(k)) * LD + colk(k)].x;
            }
        }
        return static_cast<const C*>(r);
    };
    // the gain of the axis pair {(1,0), (0,1)} (J = H) with s W_(1,0) from
    // the loss transform's imaginary part rw and W_(0,1) by direct gathers
    // along the row; c2 arrives divided by s (exact: s is a power of two)
    auto gain_axis = [&](const C* rw, const T c2) {
        T w[PPT], pp[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            w[k] = (k < PPT - 1 || last_ok) ? rw[(y0 + PM::dy(k)) * LD + colk(k)].y : T(0);
            pp[k] = T(0);
        }
        for (int j = 1; j <= H; ++j) {
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (k < PPT - 1 || last_ok) pp[k] += sF[a0 + PM::dy(k) * RS + PM::dx(k) + j];
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (k < PPT - 1 || last_ok) pp[k] += sF[a0 + PM::dy(k) * RS + PM::dx(k) - j];
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k)
            if (k < PPT - 1 || last_ok) comp_add<T, KAHAN>(acc[k], cmp[k], c2 * w[k] * pp[k]);
    };
    // The cell copy with its periodic halo of width HW, XR more columns on
    // the right (2 HW + XR < N, so a point has at most one image per axis),
    // and optionally the FFT input: the N^2
    // points are read once; consecutive threads take consecutive points, so
    // a warp's loads are coalesced and its stores hit distinct banks.
    auto fill_cell = [&](const bool fft_in) {
        auto put = [&](const int y, const int x, const T v) {
            const int a = (y + HW) * RS + x + HW;
            const int dy = y < HW ? N * RS : (y >= N - HW ? -N * RS : 0);
            const int dx = x < HW + XR ? N : (x >= N - HW ? -N : 0);
            sF[a] = v;
            if (dy) sF[a + dy] = v;
            if (dx) sF[a + dx] = v;
            if (dy && dx) sF[a + dy + dx] = v;
            if (fft_in) A[y * LD + x] = C{v, T(0)};
        };
#pragma unroll 4
        for (int i = tid; i < N * N; i += NT) put(i / N, i % N, __ldcs(fcell + i));
    };
    // late: the cell and sS from the values fv[r] of the points tid + r NT
    // (every image a of a point also goes to sS[a - 1]; a = 0, possible for
    // a corner image only, has no place in sS and is never read from there)
    constexpr int NFV = VEC ? N * N / NT : 1;
    auto fill_late = [&](const T (&fv)[NFV]) {
#pragma unroll
        for (int r = 0; r < NFV; ++r) {
            const int i = tid + r * NT, y = i / N, x = i % N;
            const int a = (y + HW) * RS + x + HW;
            const int dy = y < HW ? N * RS : (y >= N - HW ? -N * RS : 0);
            const int dx = x < HW + XR ? N : (x >= N - HW ? -N : 0);
            const T v = fv[r];
            sF[a] = v;
            sS[a - 1] = v;
            if (dy) {
                sF[a + dy] = v;
                sS[a + dy - 1] = v;
            }
            if (dx) {
                sF[a + dx] = v;
                sS[a + dx - 1] = v;
            }
            if (dy && dx) {
                sF[a + dy + dx] = v;
                if (a + dy + dx > 0) sS[a + dy + dx - 1] = v;
            }
        }
    };

    if constexpr (!SCAN) {
        if (SUB == 0 && fwin) {
            // fhat: f into A, forward transform (an even number of passes:
            // the result is in A), then into the cell's place F
            const T* djt;
            if constexpr (sizeof(T) == 8) djt = P.dj;
            else djt = P.dj_f;
            C* F = reinterpret_cast<C*>(smem);
            static_assert((size_t)N * LD * sizeof(C) <= cell_bytes<T, N, H, false, XR>(), "fhat fits in the cell's place");
            for (int i = tid; i < N * N; i += NT) A[(i / N) * LD + (i % N)] = C{fcell[i], T(0)};
            __syncthreads();
            C* r = fft_lines<C, N, LD, false, false>(A, B, tw);
            r = fft_lines<C, N, LD, false, true>(r, r == A ? B : A, tw);
            for (int i = tid; i < N * LD; i += NT) F[i] = r[i];
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                acc[k] = T(0);
                cmp[k] = T(0);
            }
            for (int pr = pb; pr < pe; ++pr) {
                const int4 e = P.pairs[pr];
                if (e.z < scan_j) continue;
                const T c2 = pair_weight<T>(P.pair_c, P.pair_c2f, pr);
                const T* dje = djt + e.z * N;
                // e and e^perp = (-e1, e0) reduced to [0, N): every product below is non-negative
                const int e0 = (e.x % N + N) % N, e1 = (e.y % N + N) % N, n1 = (N - e1) % N;
                const C* q = ifft2_from<C, N, LD>(F, A, B, tw, [&](const int ky, const int kx) {
                    return C{dje[(e0 * ky + e1 * kx) % N], dje[(n1 * ky + e0 * kx) % N]};
                });
                if (active) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (k < PPT - 1 || last_ok) {
                            const C w = q[(y0 + PM::dy(k)) * LD + colk(k)];
                            comp_add<T, KAHAN>(acc[k], cmp[k], c2 * w.x * w.y);
                        }
                    }
                }
                __syncthreads();
            }
            // the loss, then the cell in F's place for the other pairs
            const C* q = nullptr;
            if (do_loss)
                q = ifft2_from<C, N, LD>(F, A, B, tw,
                                         [&](const int ky, const int kx) { return C{kh[ky * N + kx], T(0)}; });
            fill_cell(false);
            __syncthreads();
            if (do_loss && active) {
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (k < PPT - 1 || last_ok)
                        comp_add<T, KAHAN>(acc[k], cmp[k],
                                           -sF[a0 + PM::dy(k) * RS + PM::dx(k)] * q[(y0 + PM::dy(k)) * LD + colk(k)].x);
            }
            if constexpr (VEC) {
                __syncthreads();  // the loss result is read: the FFT buffers take the shifted cell
                for (int i = tid; i < W * RS - 1; i += NT) sS[i] = sF[i + 1];
                __syncthreads();
            }
            if (active)
                for (int pr = pb; pr < pe; ++pr) {
                    const int4 e = P.pairs[pr];
                    if (e.z < scan_j) gain_pair(e, pair_weight<T>(P.pair_c, P.pair_c2f, pr));
                }
        } else {
        // VEC (late): f into registers and the FFT input; the cell follows
        // the transform.  Otherwise the cell and the FFT input at once.
        T fv[NFV];
        if constexpr (VEC) {
#pragma unroll
            for (int r = 0; r < NFV; ++r) {
                const int i = tid + r * NT;
                fv[r] = __ldcs(fcell + i);
                if (do_loss) A[(i / N) * LD + i % N] = C{fv[r], T(0)};
            }
        } else {
            fill_cell(do_loss);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            acc[k] = T(0);
            cmp[k] = T(0);
        }
        // the first pair is the axis pair (lines in order of |e|_inf): with
        // wfft its W_(1,0) comes out of the loss transform
        bool wax = false;
        if (wfft && do_loss && pb < pe) {
            const int4 e0 = P.pairs[pb];
            wax = abs(e0.x) + abs(e0.y) == 1 && e0.z == H;
        }
        const T* dw = nullptr;
        if (wax) {
            if constexpr (sizeof(T) == 8) dw = P.dwin;
            else dw = P.dwin_f;
        }
        // VEC: the loss leaves the transform as -(K * f), to be multiplied by
        // f at the owned points once the cell is in place
        const C* rw = nullptr;
        if (do_loss)
            rw = loss_fft([&](int k) { return VEC ? T(1) : sF[a0 + PM::dy(k) * RS + PM::dx(k)]; }, dw);
        if constexpr (VEC) {
            // s W_(1,0) leaves the FFT buffers before they take the cell and sS
            T wx[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) wx[k] = (wax && active) ? rw[(y0 + PM::dy(k)) * LD + colk(k)].y : T(0);
            __syncthreads();
            fill_late(fv);
            __syncthreads();
            if (do_loss && active) {
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (k < PPT - 1 || last_ok) acc[k] *= sF[a0 + PM::dy(k) * RS + PM::dx(k)];
            }
            if (active) {
                int pr = pb;
                if (wax) {
                    // W_(0,1) along the row for both points of a pair from
                    // the segment x - H .. x + H + 1 (H + 1 aligned 8-byte
                    // loads, from sS when a0 - H is odd), the centres left out:
                    // W(x) = v[0] + A + v[H+1] + B, W(x+1) = A + v[H] + B + v[2H+1]
                    // with A, B the sums of v[1..H-1] and v[H+2..2H]
                    const T c2 = pair_weight<T>(P.pair_c, P.pair_c2f, pr++) * dw[N];  // dw[N] = 1 / s
                    const T* sb = ((A0P - H) & 1) ? sS + a0 - H - 1 : sF + a0 - H;
                    T pp[PPT];
#pragma unroll
                    for (int m = 0; m < PPT / 2; ++m) {
                        const C* b = reinterpret_cast<const C*>(sb + PM::dy(2 * m) * RS + PM::dx(2 * m));
                        T v[2 * H + 2];
#pragma unroll
                        for (int t = 0; t <= H; ++t) {
                            const C u = b[t];
                            v[2 * t] = u.x;
                            v[2 * t + 1] = u.y;
                        }
                        T A = T(0), Bs = T(0);
#pragma unroll
                        for (int k = 1; k < H; ++k) A += v[k];
#pragma unroll
                        for (int k = H + 2; k <= 2 * H; ++k) Bs += v[k];
                        pp[2 * m] = (v[0] + A) + (v[H + 1] + Bs);
                        pp[2 * m + 1] = (A + v[H]) + (Bs + v[2 * H + 1]);
                    }
#pragma unroll
                    for (int k = 0; k < PPT; ++k) comp_add<T, KAHAN>(acc[k], cmp[k], c2 * wx[k] * pp[k]);
                }
                for (; pr < pe; ++pr) gain_pair(P.pairs[pr], pair_weight<T>(P.pair_c, P.pair_c2f, pr));
            }
        } else if (active) {
            int pr = pb;
            if (wax) gain_axis(rw, pair_weight<T>(P.pair_c, P.pair_c2f, pr++) * dw[N]);  // dw[N] = 1 / s
            for (; pr < pe; ++pr) gain_direct(P.pairs[pr], pair_weight<T>(P.pair_c, P.pair_c2f, pr));
        }
        }
    } else {
        // the FFT buffers occupy the cell's place: the loss reads f at the
        // owned points from global memory, the cell is copied after it
        const int h0 = y0 * N + x;
        if (do_loss)
            for (int i = tid; i < N * N; i += NT) A[(i / N) * LD + (i % N)] = C{fcell[i], T(0)};
        static_assert(2 * HW < N, "one periodic image per axis");
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            acc[k] = T(0);
            cmp[k] = T(0);
        }
        // the first pair is the axis pair (lines in order of |e|_inf): with
        // wfft its horizontal window W_(0,1), which the strips do not walk,
        // comes out of the loss transform (scaled by s); it waits in the
        // window field of its own direction, which that pair leaves unused
        bool wax = false;
        if (wfft && do_loss && pb < pe) {
            const int4 e0 = P.pairs[pb];
            wax = abs(e0.x) + abs(e0.y) == 1 && e0.z == H;
        }
        const T* dw = nullptr;
        if (wax) {
            if constexpr (sizeof(T) == 8) dw = P.dwin;
            else dw = P.dwin_f;
        }
        __syncthreads();
        if (do_loss) {
            // the transform ping-pongs an even number of passes (four line
            // transforms of equal pass count), so its result is in A, which
            // ends before the window fields: the window moves there directly
            static_assert((size_t)N * LD * sizeof(C) <= cell_bytes<T, N, H, true>(), "A below the window fields");
            const C* r = loss_fft([&](int k) { return fcell[(y0 + PM::dy(k)) * N + x + PM::dx(k)]; }, dw);
            if (wax && active) {
                T* wf = (P.pairs[pb].w & 1) ? sRp : sRe;  // the unwalked direction's field
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    if (k < PPT - 1 || last_ok)
                        wf[h0 + PM::dy(k) * N + PM::dx(k)] = r[(y0 + PM::dy(k)) * LD + colk(k)].y;
            }
            __syncthreads();
        }
        fill_cell(false);
        __syncthreads();
        bool pending = false;  // window fields still being read by the previous scanned pair
        for (int pr = pb; pr < pe; ++pr) {
            const int4 e = P.pairs[pr];
            const T c2 = pair_weight<T>(P.pair_c, P.pair_c2f, pr);
            const int walked = e.z >= scan_j ? e.w : 0;  // bit d: direction d (e, e^perp) walked in strips
            if (walked) {
                if (pending) __syncthreads();
                const int4* sd = P.pair_scan + 4 * pr;
                const int n0 = (walked & 1) ? __ldg(&sd[1].y) * __ldg(&sd[0].w) : 0;
                const int n1 = (walked & 2) ? __ldg(&sd[3].y) * __ldg(&sd[2].w) : 0;
                for (int u = tid; u < n0 + n1; u += NT) {
                    const int d = u >= n0;
                    strip_walk<T, N, H>(sF, d ? sRp : sRe, __ldg(sd + 2 * d), __ldg(sd + 2 * d + 1), e.z,
                                        d ? u - n0 : u);
                }
                __syncthreads();
                if (active) {
                    // the unwalked (horizontal) window: from the loss transform
                    // for the axis pair with wax (c2 divided by s, exact), else
                    // gathered along the row
                    const bool from_fft = wax && pr == pb;
                    const T cw = from_fft ? c2 * dw[N] : c2;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (k < PPT - 1 || last_ok) {
                            const int a = a0 + PM::dy(k) * RS + PM::dx(k);
                            const int hk = h0 + PM::dy(k) * N + PM::dx(k);
                            const T fk = sF[a];
                            T wv[2];
#pragma unroll
                            for (int d = 0; d < 2; ++d) {
                                if ((walked >> d) & 1) {
                                    wv[d] = (d ? sRp : sRe)[hk] - fk;
                                } else if (from_fft) {
                                    wv[d] = (d ? sRp : sRe)[hk];
                                } else {
                                    T sum = T(0);
                                    for (int j = 1; j <= e.z; ++j) sum += sF[a + j] + sF[a - j];
                                    wv[d] = sum;
                                }
                            }
                            comp_add<T, KAHAN>(acc[k], cmp[k], cw * wv[0] * wv[1]);
                        }
                    }
                }
                pending = true;
            } else if (active) {
                gain_direct(e, c2);
            }
        }
    }

    CellMoments<T> cm;
    cm.init();
    if (active) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (k < PPT - 1 || last_ok) {
                const int y = y0 + PM::dy(k), xk = colk(k);
                const T q = KAHAN ? acc[k] + cmp[k] : acc[k];
                if (store) __stcs(qcell + y * N + xk, q);
                if (mom) cm.add(q, y, xk);
            }
        }
    }
    if (mom) cm.template finish<SUB>(red, P.h, P.L, mom, store);
}

// elements of the f buffer; the P buffer follows it
__host__ __device__ inline size_t buf_f_elems(int N, int H) {
    return (size_t)pad2d_rows_f(N, H) * (size_t)pad2d_stride(N, H);
}
__host__ __device__ inline size_t buf_p_elems(int N, int H) {
    return (size_t)pad2d_rows_p(N, H) * (size_t)pad2d_stride(N, H);
}

// Points per thread instantiated for a CTA of NT threads (cells up to 64^2).
template <int NT>
__host__ __device__ constexpr int ppt_max() { return NT == 256 ? 16 : 8; }
__host__ __device__ inline int ppt_pick(int NT, int need) {
    if (NT == 256) return need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 9 ? 9 : 16;
    return need <= 1 ? 1 : need <= 2 ? 2 : need <= 5 ? 5 : 8;
}

// One cell with the smallest body that covers it (no predicated-off slots).
template <typename T, bool KAHAN, int NT>
__device__ __forceinline__ void run_cell(const PlanDev& P, int pb, int pe, const T* f, T* q, double* mom, T* sF, T* sP,
                                         double* red, int jd, int fft, int sj, bool do_loss) {
    // the common cell sizes with the default truncation floor(N/(3+sqrt 2))
#define QDVM_FIXED(NN, HH)                                                                                        \
    if (P.N == NN && P.Ntilde == HH) {                                                                            \
        if (fft && P.khat) {                                                                                      \
            unsigned char* sm = reinterpret_cast<unsigned char*>(sF);                                             \
            if (fft == 3)                                                                                         \
                fftloss_body<T, KAHAN, NN, HH, NT, false>(P, pb, pe, f, q, mom, sm, red, do_loss, sj > 0 ? sj : 65, \
                                                          false, true);                                           \
            else if (sj > 0 && sj <= HH)                                                                          \
                fftloss_body<T, KAHAN, NN, HH, NT, true>(P, pb, pe, f, q, mom, sm, red, do_loss, sj, fft == 2);   \
            else                                                                                                  \
                fftloss_body<T, KAHAN, NN, HH, NT, false>(P, pb, pe, f, q, mom, sm, red, do_loss, 0, fft == 2);   \
        } else {                                                                                                  \
            fixed_body<T, KAHAN, NN, HH, NT>(P.pairs, P.pair_c, P.pair_c2f, pb, pe, P.h, P.L, f, q, mom, sF, sP, \
                                             red, jd);                                                            \
        }                                                                                                         \
        return;                                                                                                   \
    }
    QDVM_FIXED(64, 14)
    QDVM_FIXED(48, 10)
    QDVM_FIXED(32, 7)
    QDVM_FIXED(16, 3)
#undef QDVM_FIXED
    const int k = ppt_pick(NT, (P.N * P.N + NT - 1) / NT);
#define QDVM_BODY(K)                                                                                          \
    fused2d_body<T, KAHAN, K>(P.N, P.Ntilde, P.pairs, P.pair_c, P.pair_c2f, pb, pe, P.h, P.L, f, q, mom, sF, sP, \
                              red, jd);                                                                          \
    return
    if (NT == 256) {
        if (k == 1) { QDVM_BODY(1); }
        if (k == 2) { QDVM_BODY(2); }
        if (k == 4) { QDVM_BODY(4); }
        if (k == 9) { QDVM_BODY(9); }
        QDVM_BODY(ppt_max<NT>());
    } else {
        if (k == 1) { QDVM_BODY(1); }
        if (k == 2) { QDVM_BODY(2); }
        if (k == 5) { QDVM_BODY(5); }
        QDVM_BODY(ppt_max<NT>());
    }
#undef QDVM_BODY
}

template <typename T, bool KAHAN, int NT>
__global__ void __launch_bounds__(NT, 2) k_fused2d_single(PlanDev P, const T* __restrict__ f, T* __restrict__ out,
                                                          int pairs_per_cta, size_t slot_stride, int jd, int fft,
                                                          int sj) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32 * 4];
    T* sF = reinterpret_cast<T*>(smem_raw);
    T* sP = sF + buf_f_elems(P.N, P.Ntilde);
    const int pb = blockIdx.x * pairs_per_cta;
    const int pe = min(pb + pairs_per_cta, P.n_pairs);
    run_cell<T, KAHAN, NT>(P, pb, pe, f, out + blockIdx.x * slot_stride, nullptr, sF, sP, red, jd, fft, sj,
                           blockIdx.x == 0);
}

// Deterministic sum of S partial results (fixed order s = 0..S-1).
template <typename T, bool KAHAN>
__global__ void k_reduce_partials(const T* __restrict__ part, int S, int n, T* __restrict__ Q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = T(0), c = T(0);
    for (int k = 0; k < S; ++k) comp_add<T, KAHAN>(s, c, part[(size_t)k * n + i]);
    Q[i] = KAHAN ? s + c : s;
}

// Small cells in FP32 with the plain FFT body (loss_fft 1 or 2, no SCAN) on
// 256 threads go several at a time: four 16^2 cells of 64 threads each, two
// 32^2 cells of 128.  A lone 16^2 cell keeps only 64 of 256 threads busy in
// its FFT passes (a lone 32^2 cell 128 in its radix-8 passes), and each of
// its ~13 barriers serves one cell; the cells of a group share them.
// cell_groups returns the group size, 0 for one cell at a time.
template <typename T, int NT>
__host__ __device__ constexpr int cell_groups(const int N, const int Nt, const bool khat, const int fft, const int sj) {
    if (!(NT == 256 && sizeof(T) == 4 && khat && (fft == 1 || fft == 2) && !(sj > 0 && sj <= Nt))) return 0;
    return (N == 16 && Nt == 3) ? 4 : ((N == 32 && Nt == 7) ? 2 : 0);
}
// Shared memory of the FFT body (fftloss_body) of an N^2 cell on NT threads
// for the tuning fft (loss_fft) and sj (scan_j): with SCAN the cell with a
// 2H halo and the two window fields, the FFT buffers aliasing them; with
// paired points (FP32, 32^2 and 64^2) and no FFT window engine the larger of
// the cell with its shifted copy and the FFT buffers, which alias; else the
// cell followed by the FFT buffers (also with the FFT window engine, fft = 3,
// whose threshold sj is).
template <typename T, int N, int H, int NT>
__host__ __device__ constexpr size_t body_smem(const int fft, const int sj) {
    constexpr size_t fftb = 2 * (size_t)N * (N + 1) * sizeof(typename Cplx<T>::type);
    constexpr size_t cb = cell_bytes<T, N, H, false, body_xr<T, N, NT>()>();
    constexpr size_t cs = cell_bytes<T, N, H, true>() + 2 * (size_t)N * N * sizeof(T);
    constexpr bool vec = sizeof(T) == 4 && (N == 32 || N == 64);
    if (fft == 3) return cb + fftb;  // sj is the FFT window threshold here
    if (sj > 0 && sj <= H) return cs > fftb ? cs : fftb;
    if (vec) return 2 * cb > fftb ? 2 * cb : fftb;
    return cb + fftb;
}
// shared memory of one cell of a group of NT threads, 128-byte aligned
template <typename T, int N, int H, int NT>
__host__ __device__ constexpr size_t group_cell_bytes() {
    return (body_smem<T, N, H, NT>(2, 0) + 127) / 128 * 128;
}
template <typename T>
__host__ __device__ constexpr size_t group_smem_bytes(const int G) {
    return G == 4 ? 4 * group_cell_bytes<T, 16, 3, 64>() : (G == 2 ? 2 * group_cell_bytes<T, 32, 7, 128>() : 0);
}

// One pass of the group body: thread group g (NT / G threads) evaluates cell
// cg when mine, else runs on cell `fallback` and stores nothing.  A cell of
// a groupable plan always goes through this body, whichever group takes it,
// so its moments come out of the same reduction.
template <typename T, bool KAHAN, int NT, int N, int H, int G>
__device__ __forceinline__ void group_pass(const PlanDev& P, const int cg, const bool mine, const int fallback,
                                           const int64_t* __restrict__ cell_offset, const T* __restrict__ f,
                                           T* __restrict__ Q, double* __restrict__ moments, unsigned char* smem_raw,
                                           double* red) {
    constexpr int SUBT = NT / G;
    const int g = threadIdx.x / SUBT;
    const int src = mine ? cg : fallback;
    const int64_t offg = cell_offset[src];
    fftloss_body<T, KAHAN, N, H, SUBT, false, SUBT>(P, 0, P.n_pairs, f + offg, Q + offg,
                                                    moments ? moments + (size_t)src * 4 : nullptr,
                                                    smem_raw + g * group_cell_bytes<T, N, H, SUBT>(), red + g * (128 / G),
                                                    true, 0, P.tfft == 2, false, mine);
    __syncthreads();
}

// A group of G cells of plan P (index pi): thread group g takes the first
// cell (g = 0) or the g-th drawn one when it is of the same plan.  Drawn
// cells of another plan then run one at a time: through their own group
// body when their plan is groupable (group 0 takes the cell), else through
// the one-cell body.
template <typename T, bool KAHAN, int NT, int N, int H, int G>
__device__ __forceinline__ void run_cell_group(const BatchDev& B, const PlanDev& P, const int cell, const int pi,
                                               const int* more, PlanDev* s_plan, const int* __restrict__ cell_plan,
                                               const int64_t* __restrict__ cell_offset, const T* __restrict__ f,
                                               T* __restrict__ Q, double* __restrict__ moments,
                                               unsigned char* smem_raw, double* red) {
    constexpr int SUBT = NT / G;
    const int g = threadIdx.x / SUBT;
    const int cg = g == 0 ? cell : more[g - 1];
    group_pass<T, KAHAN, NT, N, H, G>(P, cg, cg >= 0 && cell_plan[cg] == pi, cell, cell_offset, f, Q, moments,
                                      smem_raw, red);
    for (int k = 0; k < G - 1; ++k) {
        const int ck = more[k];
        if (ck < 0 || cell_plan[ck] == pi) continue;
        if (threadIdx.x == 0) {
            const int pk = cell_plan[ck];
#pragma unroll
            for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
                if (q == pk) *s_plan = B.p[q];
        }
        __syncthreads();
        const PlanDev Pk = *s_plan;
        const int Gk = cell_groups<T, NT>(Pk.N, Pk.Ntilde, Pk.khat != nullptr, Pk.tfft, Pk.tsj);
        if (Gk == 4) {
            group_pass<T, KAHAN, NT, 16, 3, 4>(Pk, ck, threadIdx.x < NT / 4, ck, cell_offset, f, Q, moments, smem_raw,
                                               red);
        } else if (Gk == 2) {
            group_pass<T, KAHAN, NT, 32, 7, 2>(Pk, ck, threadIdx.x < NT / 2, ck, cell_offset, f, Q, moments, smem_raw,
                                               red);
        } else {
            const int64_t offk = cell_offset[ck];
            T* sFk = reinterpret_cast<T*>(smem_raw);
            T* sPk = sFk + buf_f_elems(Pk.N, Pk.Ntilde);
            run_cell<T, KAHAN, NT>(Pk, 0, Pk.n_pairs, f + offk, Q + offk, moments ? moments + (size_t)ck * 4 : nullptr,
                                   sFk, sPk, red, Pk.tjd, Pk.tfft, Pk.tsj, true);
            __syncthreads();
        }
    }
}

template <typename T, bool KAHAN, int NT>
__global__ void __launch_bounds__(NT, 2) k_fused2d_batched(BatchDev B, int n_cells, const int* __restrict__ cell_plan,
                                                           const int64_t* __restrict__ cell_offset,
                                                           const int* __restrict__ order, int* counter,
                                                           const T* __restrict__ f, T* __restrict__ Q,
                                                           double* __restrict__ moments) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32 * 4];
    __shared__ int s_cell, s_pi, s_more[3];
    __shared__ PlanDev s_plan;
    for (;;) {
        if (threadIdx.x == 0) {
            const int c = atomicAdd(counter, 1);
            s_cell = c < n_cells ? order[c] : -1;
            s_more[0] = s_more[1] = s_more[2] = -1;
            if (s_cell >= 0) {
                const int pi = cell_plan[s_cell];
                s_pi = pi;
#pragma unroll
                for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
                    if (q == pi) s_plan = B.p[q];
                // the schedule lists cells plan by plan, so the next entries
                // are almost always cells of the same plan
                const int G = cell_groups<T, NT>(s_plan.N, s_plan.Ntilde, s_plan.khat != nullptr, s_plan.tfft,
                                                 s_plan.tsj);
                if (G > 1) {
                    const int c2 = atomicAdd(counter, G - 1);
                    for (int k = 0; k < G - 1; ++k) s_more[k] = c2 + k < n_cells ? order[c2 + k] : -1;
                }
            }
        }
        __syncthreads();
        const int cell = s_cell;
        if (cell < 0) break;
        const PlanDev P = s_plan;
        if constexpr (NT == 256 && sizeof(T) == 4) {
            const int G = cell_groups<T, NT>(P.N, P.Ntilde, P.khat != nullptr, P.tfft, P.tsj);
            if (G == 4) {
                run_cell_group<T, KAHAN, NT, 16, 3, 4>(B, P, cell, s_pi, s_more, &s_plan, cell_plan, cell_offset, f, Q,
                                                       moments, smem_raw, red);
                continue;
            }
            if (G == 2) {
                run_cell_group<T, KAHAN, NT, 32, 7, 2>(B, P, cell, s_pi, s_more, &s_plan, cell_plan, cell_offset, f, Q,
                                                       moments, smem_raw, red);
                continue;
            }
        }
        const int64_t off = cell_offset[cell];
        T* sF = reinterpret_cast<T*>(smem_raw);
        T* sP = sF + buf_f_elems(P.N, P.Ntilde);
        // the cell's plan's own direct_j, loss_fft and scan_j
        run_cell<T, KAHAN, NT>(P, 0, P.n_pairs, f + off, Q + off, moments ? moments + (size_t)cell * 4 : nullptr, sF,
                               sP, red, P.tjd, P.tfft, P.tsj, true);
        __syncthreads();
    }
}

template <typename T, bool KAHAN, int NT>
qdvm_status launch_single_t(const qdvm_plan_s* p, const T* f, T* Q, T* part, int S, int ppc, size_t smem, int jd,
                            int fft, int sj, cudaStream_t st) {
    cudaFuncSetAttribute(k_fused2d_single<T, KAHAN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const PlanDev P = plan_dev(p);
    const int n = p->N * p->N;
    if (S == 1) {
        k_fused2d_single<T, KAHAN, NT><<<1, NT, smem, st>>>(P, f, Q, ppc, 0, jd, fft, sj);
    } else {
        k_fused2d_single<T, KAHAN, NT><<<S, NT, smem, st>>>(P, f, part, ppc, (size_t)n, jd, fft, sj);
        k_reduce_partials<T, KAHAN><<<(n + 255) / 256, 256, 0, st>>>(part, S, n, Q);
    }
    QDVM_LAUNCH_CHECK("fused2d single-cell launch");
    return QDVM_OK;
}

template <typename T, bool KAHAN>
qdvm_status dispatch_single(const qdvm_plan_s* p, const void* f, void* Q, void* ws, int S, int ppc, size_t smem,
                            cudaStream_t st) {
    const T* fi = static_cast<const T*>(f);
    T* qo = static_cast<T*>(Q);
    T* part = static_cast<T*>(ws);
    const int jd = p->tune.direct_j, fft = p->tune.loss_fft, sj = p->tune.scan_j;
    if (p->tune.threads == 512)
        return launch_single_t<T, KAHAN, 512>(p, fi, qo, part, S, ppc, smem, jd, fft, sj, st);
    return launch_single_t<T, KAHAN, 256>(p, fi, qo, part, S, ppc, smem, jd, fft, sj, st);
}

inline void split_pairs(int n_pairs, int max_ctas, int* S, int* ppc) {
    int s = std::max(1, std::min(n_pairs, max_ctas));
    int per = (n_pairs + s - 1) / s;
    *ppc = per;
    *S = (n_pairs + per - 1) / per;
}

template <typename T, bool KAHAN, int NT>
qdvm_status launch_batched_t(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                             const int* order, int* counter, const T* f, T* Q, double* moments, size_t smem,
                             cudaStream_t st) {
    auto k = k_fused2d_batched<T, KAHAN, NT>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem);
    per_sm = std::max(per_sm, 1);
    const int grid = std::max(1, std::min(n_cells, per_sm * qdvm_num_sms()));
    k<<<grid, NT, smem, st>>>(b, n_cells, cell_plan, cell_offset, order, counter, f, Q, moments);
    QDVM_LAUNCH_CHECK("fused2d batched launch");
    return QDVM_OK;
}

template <typename T, bool KAHAN>
qdvm_status dispatch_batched(const BatchDev& b, const qdvm_tuning& tu, int n_cells, const int* cell_plan,
                             const int64_t* cell_offset, const int* order, int* counter, const void* f, void* Q,
                             double* moments, size_t smem, cudaStream_t st) {
    const T* fi = static_cast<const T*>(f);
    T* qo = static_cast<T*>(Q);
    if (tu.threads == 512)
        return launch_batched_t<T, KAHAN, 512>(b, n_cells, cell_plan, cell_offset, order, counter, fi, qo, moments,
                                               smem, st);
    return launch_batched_t<T, KAHAN, 256>(b, n_cells, cell_plan, cell_offset, order, counter, fi, qo, moments, smem,
                                           st);
}


}  // namespace

// Per-precision entry points, one translation unit each (fused2d_f64.cu,
// fused2d_f32.cu, fused2d_f32k.cu), so that the instantiations compile in
// parallel.
#define QDVM_FUSED2D_DECLARE(sfx)                                                                                  \
    qdvm_status fused2d_single_##sfx(const qdvm_plan_s* p, const void* f, void* Q, void* ws, int S, int ppc,      \
                                     size_t smem, cudaStream_t st);                                                \
    qdvm_status fused2d_batched_##sfx(const BatchDev& b, const qdvm_tuning& tu, int n_cells, const int* cell_plan, \
                                      const int64_t* cell_offset, const int* order, int* counter, const void* f,   \
                                      void* Q, double* moments, size_t smem, cudaStream_t st);
QDVM_FUSED2D_DECLARE(f64)
QDVM_FUSED2D_DECLARE(f32)
QDVM_FUSED2D_DECLARE(f32k)
#undef QDVM_FUSED2D_DECLARE

#define QDVM_FUSED2D_INSTANTIATE(sfx, T, KAHAN)                                                                    \
    qdvm_status fused2d_single_##sfx(const qdvm_plan_s* p, const void* f, void* Q, void* ws, int S, int ppc,      \
                                     size_t smem, cudaStream_t st) {                                               \
        return dispatch_single<T, KAHAN>(p, f, Q, ws, S, ppc, smem, st);                                           \
    }                                                                                                              \
    qdvm_status fused2d_batched_##sfx(const BatchDev& b, const qdvm_tuning& tu, int n_cells, const int* cell_plan, \
                                      const int64_t* cell_offset, const int* order, int* counter, const void* f,   \
                                      void* Q, double* moments, size_t smem, cudaStream_t st) {                    \
        return dispatch_batched<T, KAHAN>(b, tu, n_cells, cell_plan, cell_offset, order, counter, f, Q, moments,   \
                                          smem, st);                                                               \
    }
