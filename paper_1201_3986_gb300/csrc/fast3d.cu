// 3D evaluation (forward, JVP, VJP) with the loss as one convolution per
// cell (eq. (decD): the loss terms of all lines form one convolution).
//
// The loss part sum_e c_e f V_e equals f (K * f) with K the weighted
// displacement histogram of all (k, l) terms (its transform is the plan's
// Ktilde, factorised line by line).  A work item (cell, chunk of lines)
// therefore only sums the gain c_e W_e P_e of its lines; the first chunk of
// a cell also evaluates K * f with a 3D Stockham FFT (mixed radix 4/8) over
// the CTA's global scratch.  Without V there is no P buffer and no barrier
// per line: each thread owns z-columns of 8 points at a fixed (y, x), runs
// the item's lines for one column at a time and keeps the sums in
// registers.  The cell sits in shared memory with a periodic halo of Ntilde
// along z; y and x wrap with a mask (N = 16 or 32, a power of two; the
// halo is Ntilde < N / 2 planes on each side).
#include <algorithm>

#include "fft.cuh"
#include "engine.cuh"
#include "qdvm_internal.cuh"

namespace {

// Threads per CTA: the cell occupies most of the shared memory (one CTA
// per SM), so 32^3 cells run 1024 threads (32 warps to hide latency, 64
// registers each); 16^3 cells have 512 units of 8 points.
__host__ __device__ constexpr int f3_threads(int N) { return N >= 32 ? 1024 : 512; }

// One Stockham pass of radix R along AXIS (0 = z, 1 = y, 2 = x) over all N^2
// lines of an N^3 complex array in global memory.  Consecutive threads take
// consecutive addresses: along x they share a line, along y and z they take
// neighbouring lines.
template <typename C, int N, int R, int NS, bool INV, int AXIS>
__device__ __forceinline__ void fft3_pass(const C* __restrict__ src, C* __restrict__ dst, const C* __restrict__ tw) {
    constexpr int NB = N / R, NL = N * N;
    constexpr int ST = AXIS == 2 ? 1 : (AXIS == 1 ? N : NL);
    for (int b = threadIdx.x; b < NL * NB; b += blockDim.x) {
        int line, j;
        if (AXIS == 2) {
            line = b / NB;
            j = b - line * NB;
        } else {
            line = b % NL;
            j = b / NL;
        }
        const int base = AXIS == 2 ? line * N : (AXIS == 1 ? (line / N) * NL + (line % N) : line);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[base + (j + r * NB) * ST];
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
        for (int r = 0; r < R; ++r) dst[base + (idxD + r * NS) * ST] = v[r];
    }
}

template <typename C, int N, bool INV, int AXIS, int NS, int R, int... Rs>
__device__ __forceinline__ C* fft3_passes(C* a, C* b, const C* tw) {
    fft3_pass<C, N, R, NS, INV, AXIS>(a, b, tw);
    __syncthreads();
    if constexpr (sizeof...(Rs) > 0)
        return fft3_passes<C, N, INV, AXIS, NS * R, Rs...>(b, a, tw);
    else
        return b;
}

template <typename C, int N, bool INV, int AXIS>
__device__ __forceinline__ C* fft3_axis(C* a, C* b, const C* tw) {
    if constexpr (N == 32) return fft3_passes<C, N, INV, AXIS, 1, 4, 8>(a, b, tw);
    else return fft3_passes<C, N, INV, AXIS, 1, 4, 4>(a, b, tw);  // N == 16
}

template <typename T, bool KAHAN, int N>
__device__ void fast3d_item(const PlanDev& P, const int lb, const int le, const bool do_loss,
                            const T* __restrict__ fcell, T* __restrict__ fz, typename Cplx<T>::type* A,
                            typename Cplx<T>::type* B, T* __restrict__ dst) {
    using C = typename Cplx<T>::type;
    constexpr int N2 = N * N, N3 = N2 * N, ZC = 8, NU = (N / ZC) * N2, M = N - 1;
    const int NT = blockDim.x, tid = threadIdx.x, H = P.Ntilde;

    for (int p = tid; p < (N + 2 * H) * N2; p += NT) {
        const int zz = p / N2;
        fz[p] = fcell[((zz - H + N) & M) * N2 + (p - zz * N2)];
    }
    if (do_loss)
        for (int i = tid; i < N3; i += NT) A[i] = C{fcell[i], T(0)};
    __syncthreads();

    const C* conv = nullptr;
    if (do_loss) {
        const C* tw;
        const T* kh;
        if constexpr (sizeof(T) == 8) {
            tw = reinterpret_cast<const C*>(P.tw);
            kh = reinterpret_cast<const T*>(P.khat);
        } else {
            tw = reinterpret_cast<const C*>(P.tw_f);
            kh = reinterpret_cast<const T*>(P.khat_f);
        }
        C* r = fft3_axis<C, N, false, 2>(A, B, tw);
        r = fft3_axis<C, N, false, 1>(r, r == A ? B : A, tw);
        r = fft3_axis<C, N, false, 0>(r, r == A ? B : A, tw);
        for (int i = tid; i < N3; i += NT) {
            const T k = kh[i];
            r[i].x *= k;
            r[i].y *= k;
        }
        __syncthreads();
        r = fft3_axis<C, N, true, 0>(r, r == A ? B : A, tw);
        r = fft3_axis<C, N, true, 1>(r, r == A ? B : A, tw);
        r = fft3_axis<C, N, true, 2>(r, r == A ? B : A, tw);
        conv = r;
    }

    for (int u = tid; u < NU; u += NT) {
        const int zb = u / N2, rr = u - zb * N2, y = rr / N, x = rr - (rr / N) * N, z0 = zb * ZC;
        T acc[ZC], cmp[ZC];
#pragma unroll
        for (int zc = 0; zc < ZC; ++zc) {
            // the loss, - f (K * f), starts the sum
            acc[zc] = do_loss ? -fz[(z0 + zc + H) * N2 + rr] * conv[(z0 + zc) * N2 + rr].x : T(0);
            cmp[zc] = T(0);
        }
        for (int li = lb; li < le; ++li) {
            const int4 e = P.lines[li];
            const T c = (T)P.c[li];
            const int ps = P.plane_start[li], pn = P.plane_start[li + 1] - ps;
            const char4* __restrict__ pl = P.plane + ps;
            T s[ZC], w[ZC];
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) s[zc] = w[zc] = T(0);
            for (int t = 0; t < pn; ++t) {
                const char4 l = __ldg(pl + t);
                const T* b = fz + (z0 + l.x + H) * N2 + ((y + l.y) & M) * N + ((x + l.z) & M);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) s[zc] += b[zc * N2];
            }
            for (int j = 1; j <= e.w; ++j) {
                const T* bp = fz + (z0 + j * e.x + H) * N2 + ((y + j * e.y) & M) * N + ((x + j * e.z) & M);
                const T* bm = fz + (z0 - j * e.x + H) * N2 + ((y - j * e.y) & M) * N + ((x - j * e.z) & M);
#pragma unroll
                for (int zc = 0; zc < ZC; ++zc) w[zc] += bp[zc * N2] + bm[zc * N2];
            }
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) comp_add<T, KAHAN>(acc[zc], cmp[zc], c * w[zc] * s[zc]);
        }
#pragma unroll
        for (int zc = 0; zc < ZC; ++zc) dst[(z0 + zc) * N2 + rr] = KAHAN ? acc[zc] + cmp[zc] : acc[zc];
    }
}

template <typename T, bool KAHAN, int N>
__global__ void __launch_bounds__(f3_threads(N), 1) k_fast3d(BatchDev Bt, int n_cells, int Cn, const int* __restrict__ cell_plan,
                                                       const int64_t* __restrict__ cell_offset,
                                                       const int* __restrict__ order, int* counter,
                                                       const T* __restrict__ f, const T* __restrict__ /*aux*/,
                                                       T* __restrict__ out, T* __restrict__ part, size_t part_stride,
                                                       char* scratch, size_t scr_stride) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_cell;
    __shared__ PlanDev s_plan;
    const int n_items = n_cells * Cn;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            int cell = -1;
            if (it < n_items) cell = order[it / Cn];
            s_item = cell >= 0 ? it : -1;
            s_cell = cell;
            if (cell >= 0) {
                const int pi = cell_plan[cell];
#pragma unroll
                for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
                    if (q == pi) s_plan = Bt.p[q];
            }
        }
        __syncthreads();
        const int item = s_item, cell = s_cell;
        if (item < 0) break;
        const PlanDev P = s_plan;
        const int chunk = item % Cn;
        const int lpc = (P.n_lines + Cn - 1) / Cn;
        const int lb = min(chunk * lpc, P.n_lines), le = min(lb + lpc, P.n_lines);
        const int64_t off = cell_offset[cell];
        T* dst = Cn == 1 ? out + off : part + ((size_t)cell * Cn + chunk) * part_stride;
        C* A = reinterpret_cast<C*>(scratch + (size_t)blockIdx.x * scr_stride);
        C* B = A + N * N * N;
        fast3d_item<T, KAHAN, N>(P, lb, le, chunk == 0, f + off, reinterpret_cast<T*>(smem_raw), A, B, dst);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- row form
// Gain via the row tables of the plan (plan_rows.cu).  For each line class
// the cell is re-indexed in the class coordinates q = (alpha, beta, gamma),
// point = M q mod N, and stored as g[(beta N + gamma) SA + a] for every
// a < SA with a = alpha (mod N), so that a run of up to QDVM_ROW_MAX + 7
// points starting at any alpha < N is contiguous.  SA is odd: the 32 lanes
// of a warp, which differ in gamma (and, for N = 16, in beta), hit 32
// distinct banks.
template <int N>
__host__ __device__ constexpr int rows_sa() {
    return (N + QDVM_ROW_MAX + 6) | 1;
}

// The loss convolution of one or two real fields at once: with A = x1 + i x2
// on entry, the FFT times the real Ktilde, transformed back, holds K * x1 in
// the real and K * x2 in the imaginary part (3D FFT over the CTA's scratch A,
// B; the caller fills A and synchronises).
template <typename T, int N>
__device__ const typename Cplx<T>::type* loss_conv(const PlanDev& P, typename Cplx<T>::type* A,
                                                   typename Cplx<T>::type* B) {
    using C = typename Cplx<T>::type;
    constexpr int N3 = N * N * N;
    const C* tw;
    const T* kh;
    if constexpr (sizeof(T) == 8) {
        tw = reinterpret_cast<const C*>(P.tw);
        kh = reinterpret_cast<const T*>(P.khat);
    } else {
        tw = reinterpret_cast<const C*>(P.tw_f);
        kh = reinterpret_cast<const T*>(P.khat_f);
    }
    C* r = fft3_axis<C, N, false, 2>(A, B, tw);
    r = fft3_axis<C, N, false, 1>(r, r == A ? B : A, tw);
    r = fft3_axis<C, N, false, 0>(r, r == A ? B : A, tw);
    for (int i = threadIdx.x; i < N3; i += blockDim.x) {
        const T k = kh[i];
        r[i].x *= k;
        r[i].y *= k;
    }
    __syncthreads();
    r = fft3_axis<C, N, true, 0>(r, r == A ? B : A, tw);
    r = fft3_axis<C, N, true, 1>(r, r == A ? B : A, tw);
    r = fft3_axis<C, N, true, 2>(r, r == A ? B : A, tw);
    return r;
}

// Window stride of the global class-coordinate copy: alpha runs of 8 from
// any alpha < N.
template <int N>
__host__ __device__ constexpr int rows_sw() {
    return N + 7;
}

// The same in the CTA's global scratch for line-window taps, gamma fastest
// (a warp's 32 gammas share cache lines): gw[(beta SW + alpha) N + gamma],
// alpha < 7 repeated after N - 1.  Read back with plain loads after a CTA
// barrier.
template <typename T, int N>
__device__ __forceinline__ void relayout_glob(const int (&Mi)[9], const T* __restrict__ src, T* gw) {
    constexpr int N2 = N * N, N3 = N2 * N, M = N - 1, SW = rows_sw<N>();
    for (int p = threadIdx.x; p < N3; p += blockDim.x) {
        const int p0 = p / N2, p1 = (p / N) & M, p2 = p & M;
        const int al = (Mi[0] * p0 + Mi[1] * p1 + Mi[2] * p2) & M;
        const int be = (Mi[3] * p0 + Mi[4] * p1 + Mi[5] * p2) & M;
        const int ga = (Mi[6] * p0 + Mi[7] * p1 + Mi[8] * p2) & M;
        const T v = src[p];
        T* d = gw + (be * SW + al) * N + ga;
        d[0] = v;
        if (al < SW - N) d[N2] = v;
    }
}

// Pairwise sum of v[LO, HI).
template <int LO, int HI, typename T, int K>
__device__ __forceinline__ T tree_sum(const T (&v)[K]) {
    if constexpr (HI - LO == 1) return v[LO];
    else return tree_sum<LO, (LO + HI) / 2>(v) + tree_sum<(LO + HI) / 2, HI>(v);
}

// c_e of row-form line li in the kernel's type (FP32 kernels read the
// plan's FP32 copy: no FP64 conversion per line).
template <typename T>
__device__ __forceinline__ T line_weight(const PlanDev& P, const int li) {
    if constexpr (sizeof(T) == 4) return __ldg(P.rc_f + li);
    else return __ldg(P.rc + li);
}

// Start of a row run in the class-coordinate cell: row offsets (dalpha,
// dbeta, dgamma) from the unit at (a0, be, ga).
template <int N, typename T>
__device__ __forceinline__ const T* row_base(const T* g, int be, int ga, int a0, uchar4 w) {
    constexpr int M = N - 1, SA = rows_sa<N>();
    return g + (((be + w.y) & M) * N + ((ga + w.z) & M)) * SA + ((a0 + w.x) & M);
}

// One row of length LEN for the 8 points a0 .. a0 + 7: LEN + 7 loads; the
// first window is added to P0 and the window increments to D (the window at
// point k is P0 + D[0] + ... + D[k-1]).  The next row's start is computed
// while the loads are in flight and returned.
template <int LEN, int N, typename T>
__device__ __forceinline__ const T* row_run(const T* __restrict__ b, T& P0, T (&D)[7], const T* g, int be, int ga,
                                            int a0, uchar4 wn) {
    T v[LEN + 7];
#pragma unroll
    for (int t = 0; t < LEN + 7; ++t) v[t] = b[t];
    const T* bn = row_base<N>(g, be, ga, a0, wn);
    P0 += tree_sum<0, LEN>(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) D[k - 1] += v[LEN - 1 + k] - v[k - 1];
    return bn;
}

template <int N, typename T>
__device__ __forceinline__ const T* row_dispatch(int len, const T* b, T& P0, T (&D)[7], const T* g, int be, int ga,
                                                 int a0, uchar4 wn) {
    switch (len) {
        case 1: return row_run<1, N>(b, P0, D, g, be, ga, a0, wn);
        case 2: return row_run<2, N>(b, P0, D, g, be, ga, a0, wn);
        case 3: return row_run<3, N>(b, P0, D, g, be, ga, a0, wn);
        case 4: return row_run<4, N>(b, P0, D, g, be, ga, a0, wn);
        case 5: return row_run<5, N>(b, P0, D, g, be, ga, a0, wn);
        case 6: return row_run<6, N>(b, P0, D, g, be, ga, a0, wn);
        case 7: return row_run<7, N>(b, P0, D, g, be, ga, a0, wn);
        case 8: return row_run<8, N>(b, P0, D, g, be, ga, a0, wn);
        case 9: return row_run<9, N>(b, P0, D, g, be, ga, a0, wn);
        case 10: return row_run<10, N>(b, P0, D, g, be, ga, a0, wn);
        case 11: return row_run<11, N>(b, P0, D, g, be, ga, a0, wn);
        case 12: return row_run<12, N>(b, P0, D, g, be, ga, a0, wn);
        case 13: return row_run<13, N>(b, P0, D, g, be, ga, a0, wn);
        case 14: return row_run<14, N>(b, P0, D, g, be, ga, a0, wn);
        default: return row_run<15, N>(b, P0, D, g, be, ga, a0, wn);
    }
}

// Plane sums of one line, rows [rs, re), for the unit (a0, be, ga):
// P0 and D as in row_run.  Row descriptors are fetched two rows ahead and
// row starts one row ahead.
template <int N, typename T>
__device__ __forceinline__ void plane_rows(const uchar4* __restrict__ rows, int rs, int re, const T* g, int be,
                                           int ga, int a0, T& P0, T (&D)[7]) {
    if (rs >= re) return;
    uchar4 w0 = __ldg(rows + rs);
    uchar4 w1 = __ldg(rows + min(rs + 1, re - 1));
    const T* b = row_base<N>(g, be, ga, a0, w0);
    for (int r = rs; r < re; ++r) {
        const uchar4 w2 = __ldg(rows + min(r + 2, re - 1));
        b = row_dispatch<N>(w0.w, b, P0, D, g, be, ga, a0, w1);
        w0 = w1;
        w1 = w2;
    }
}

// Prefix form of the class-coordinate cell (forward and JVP): for every
// (beta, gamma) line, S[(beta N + gamma) SP + a] = sum_{t < a} g_t with g_t
// the cell value at alpha = t mod N, a <= SP - 1.  A run of LEN points
// starting at alpha = s sums to S[s + LEN] - S[s], whatever LEN, so the 8
// windows of a unit (a0 .. a0 + 7) of one row cost 16 loads and no dispatch
// on the length.  SP is odd (a warp's lanes, consecutive gamma, hit distinct
// banks) and covers s <= N - 1, LEN <= QDVM_ROW_MAX, plus the 7 further
// points of a unit.
template <int N>
__host__ __device__ constexpr int rows_sp() {
    return (N + QDVM_ROW_MAX + 8) | 1;
}

// The cell src in prefix form: the class-coordinate values at a + 1 for
// every a < SP - 1 with a = alpha (mod N), then one thread per (beta, gamma)
// line accumulates them in place (S[0] = 0).  Ends with a barrier.
template <typename T, int N>
__device__ __forceinline__ void relayout_prefix(const int (&Mi)[9], const T* __restrict__ src, T* __restrict__ S) {
    constexpr int N2 = N * N, N3 = N2 * N, M = N - 1, SP = rows_sp<N>();
    for (int p = threadIdx.x; p < N3; p += blockDim.x) {
        const int p0 = p / N2, p1 = (p / N) & M, p2 = p & M;
        const int al = (Mi[0] * p0 + Mi[1] * p1 + Mi[2] * p2) & M;
        const int be = (Mi[3] * p0 + Mi[4] * p1 + Mi[5] * p2) & M;
        const int ga = (Mi[6] * p0 + Mi[7] * p1 + Mi[8] * p2) & M;
        const T v = src[p];
        T* d = S + (be * N + ga) * SP + 1;
        for (int a = al; a < SP - 1; a += N) d[a] = v;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < N2; l += blockDim.x) {
        T* d = S + l * SP;
        T run = T(0);
        d[0] = run;
#pragma unroll 8
        for (int a = 1; a < SP; ++a) {
            run += d[a];
            d[a] = run;
        }
    }
    __syncthreads();
}

// One row (dalpha, dbeta, dgamma, LEN) of the unit (a0, be, ga) in prefix
// form: P[k] += S[lo + k + LEN] - S[lo + k].
template <int N, typename T>
__device__ __forceinline__ void prefix_row(const T* S, const int be, const int ga, const int a0, const uchar4 w,
                                           T (&P)[8]) {
    constexpr int M = N - 1, SP = rows_sp<N>();
    const T* lo = S + (((be + w.y) & M) * N + ((ga + w.z) & M)) * SP + ((a0 + w.x) & M);
    const T* hi = lo + w.w;
    T a[8], b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = lo[k];
        b[k] = hi[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) P[k] += b[k] - a[k];
}

// The forward and JVP sums over the lines [ls, lend) of one class for the
// thread's units of 8 consecutive alpha points, added at the points' cell
// indices p = M q (mod N).  Plane sums come from the rows of S in prefix
// form; the first nc rows of every line are the class's central row
// {a u : 0 < |a| <= A} (A > 0), summed once per unit and taken as the start
// of each line's plane sums.  Line windows come from S (WG false: a value is
// the difference of neighbouring prefix entries) or from the global copy gw
// (WG true).
template <typename T, bool KAHAN, int N, bool WG>
__device__ void class_units_prefix(const PlanDev& P, const int (&Mm)[9], int ls, int lend, const int A, const int nc,
                                   const T* __restrict__ S, const T* gw, T* __restrict__ dst, T* __restrict__ comp) {
    constexpr int N2 = N * N, M = N - 1, SP = rows_sp<N>(), SW = rows_sw<N>(), NU = (N / 8) * N2;
    for (int u = threadIdx.x; u < NU; u += blockDim.x) {
        const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
        T acc[8], cmp[8], C[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = cmp[t] = C[t] = T(0);
        if (A > 0) {  // the central row {a u : 0 < |a| <= A}: [-A, -1] and [1, A] along alpha
            prefix_row<N>(S, be, ga, a0, make_uchar4((unsigned char)((N - A) & M), 0, 0, (unsigned char)A), C);
            prefix_row<N>(S, be, ga, a0, make_uchar4(1, 0, 0, (unsigned char)A), C);
        }
        int4 e = __ldg(P.rline + ls);
        T cd = line_weight<T>(P, ls);
        int rs = __ldg(P.rrow_start + ls);
        for (int li = ls; li < lend; ++li) {
            const int re = __ldg(P.rrow_start + li + 1);
            const int ln = min(li + 1, lend - 1);
            const int4 e_n = __ldg(P.rline + ln);
            const T c_n = line_weight<T>(P, ln);
            T Pk[8], W[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                Pk[t] = C[t];
                W[t] = T(0);
            }
            for (int r = rs + nc; r < re; ++r) prefix_row<N>(S, be, ga, a0, __ldg(P.rrow + r), Pk);
            for (int j = 1; j <= e.w; ++j) {
                if (WG) {
                    const T* bp = gw + (((be + j * e.y) & M) * SW + ((a0 + j * e.x) & M)) * N + ((ga + j * e.z) & M);
                    const T* bm = gw + (((be - j * e.y) & M) * SW + ((a0 - j * e.x) & M)) * N + ((ga - j * e.z) & M);
#pragma unroll
                    for (int t = 0; t < 8; ++t) W[t] += bp[t * N] + bm[t * N];
                } else {
                    const T* bp = S + (((be + j * e.y) & M) * N + ((ga + j * e.z) & M)) * SP + ((a0 + j * e.x) & M);
                    const T* bm = S + (((be - j * e.y) & M) * N + ((ga - j * e.z) & M)) * SP + ((a0 - j * e.x) & M);
                    T xp[9], xm[9];
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        xp[t] = bp[t];
                        xm[t] = bm[t];
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) W[t] += (xp[t + 1] - xp[t]) + (xm[t + 1] - xm[t]);
                }
            }
            const T c = cd;
#pragma unroll
            for (int t = 0; t < 8; ++t) comp_add<T, KAHAN>(acc[t], cmp[t], c * W[t] * Pk[t]);
            e = e_n;
            cd = c_n;
            rs = re;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int al = a0 + t;
            const int o0 = (Mm[0] * al + Mm[1] * be + Mm[2] * ga) & M;
            const int o1 = (Mm[3] * al + Mm[4] * be + Mm[5] * ga) & M;
            const int o2 = (Mm[6] * al + Mm[7] * be + Mm[8] * ga) & M;
            const int o = o0 * N2 + o1 * N + o2;
            if (KAHAN) {
                T s = dst[o], cc = comp[o];
                comp_add<T, true>(s, cc, acc[t] + cmp[t]);
                dst[o] = s;
                comp[o] = cc;
            } else {
                dst[o] += acc[t];
            }
        }
    }
}

// VJP with cotangent gc (the transpose of the JVP; Omega_e and Pi_e are
// symmetric on the torus): loss part -[g (K * f) + K * (g f)], gain part
// sum_e c [Omega_e(g P_e(f)) + Pi_e(g W_e(f))].  Both gain terms apply a
// stencil to a per-line product, so each line materialises its product over
// the cell.  Pass A: rows of f in shared memory, X = g P_e(f) to the global
// window copy, then the windows Omega_e(X).  Pass B: windows of f from the
// global window copy, Y = g W_e(f) into shared memory, then the rows Pi_e(Y).
// Class sums go to a compact class-coordinate field acc[(beta N + alpha) N +
// gamma] (gamma fastest: a warp's accesses are coalesced) and are added at
// the cell indices once per class.
template <typename T, int N>
__device__ __forceinline__ void relayout_compact(const int (&Mi)[9], const T* __restrict__ src, T* dstc) {
    constexpr int N2 = N * N, N3 = N2 * N, M = N - 1;
    for (int p = threadIdx.x; p < N3; p += blockDim.x) {
        const int p0 = p / N2, p1 = (p / N) & M, p2 = p & M;
        const int al = (Mi[0] * p0 + Mi[1] * p1 + Mi[2] * p2) & M;
        const int be = (Mi[3] * p0 + Mi[4] * p1 + Mi[5] * p2) & M;
        const int ga = (Mi[6] * p0 + Mi[7] * p1 + Mi[8] * p2) & M;
        dstc[(be * N + al) * N + ga] = src[p];
    }
}

// 8 values of a compact field at alpha = a0 .. a0 + 7 (stride N)
template <int N, typename T>
__device__ __forceinline__ void load8(const T* p, T (&v)[8]) {
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = p[t * N];
}

template <int N, typename T, bool KAHAN>
__device__ __forceinline__ void acc8(T* acc, T* cmp, const T (&x)[8], T c) {
    T a[8];
    load8<N>(acc, a);
    if (KAHAN) {
        T k[8];
        load8<N>(cmp, k);
#pragma unroll
        for (int t = 0; t < 8; ++t) comp_add<T, true>(a[t], k[t], c * x[t]);
#pragma unroll
        for (int t = 0; t < 8; ++t) cmp[t * N] = k[t];
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t] += c * x[t];
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t * N] = a[t];
}

template <typename T, bool KAHAN, int N>
__device__ void vjp_class(const PlanDev& P, const int (&Mm)[9], const int (&Mi)[9], int ls, int lend,
                          const T* __restrict__ fcell, const T* __restrict__ gcell, T* __restrict__ g, T* gwf, T* X,
                          T* gC, T* accC, T* cmpC, T* __restrict__ dst, T* __restrict__ comp) {
    constexpr int N2 = N * N, N3 = N2 * N, M = N - 1, SA = rows_sa<N>(), SW = rows_sw<N>(), NU = (N / 8) * N2;
    const int NT = blockDim.x, tid = threadIdx.x;
    relayout_glob<T, N>(Mi, fcell, gwf);
    relayout_compact<T, N>(Mi, gcell, gC);
    for (int i = tid; i < N3; i += NT) {
        accC[i] = T(0);
        if (KAHAN) cmpC[i] = T(0);
    }
    // pass A reads the plane rows of f from its prefix form (one per class);
    // pass B writes each line's product Y in the direct row layout over it
    relayout_prefix<T, N>(Mi, fcell, g);  // ends with a barrier
    // pass A: X = g P_e(f), then Omega_e(X)
    for (int li = ls; li < lend; ++li) {
        const int rs = __ldg(P.rrow_start + li), re = __ldg(P.rrow_start + li + 1);
        for (int u = tid; u < NU; u += NT) {
            const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
            T Pk[8], gv[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) Pk[t] = T(0);
            for (int r = rs; r < re; ++r) prefix_row<N>(g, be, ga, a0, __ldg(P.rrow + r), Pk);
            load8<N>(gC + (be * N + a0) * N + ga, gv);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                T* xp = X + (be * SW + a0 + t) * N + ga;
                const T x = gv[t] * Pk[t];
                xp[0] = x;
                if (a0 + t < SW - N) xp[N2] = x;
            }
        }
        __syncthreads();
        const int4 e = __ldg(P.rline + li);
        const T c = line_weight<T>(P, li);
        for (int u = tid; u < NU; u += NT) {
            const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
            T W[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) W[t] = T(0);
            for (int j = 1; j <= e.w; ++j) {
                const T* bp = X + (((be + j * e.y) & M) * SW + ((a0 + j * e.x) & M)) * N + ((ga + j * e.z) & M);
                const T* bm = X + (((be - j * e.y) & M) * SW + ((a0 - j * e.x) & M)) * N + ((ga - j * e.z) & M);
#pragma unroll
                for (int t = 0; t < 8; ++t) W[t] += bp[t * N] + bm[t * N];
            }
            const int ci = (be * N + a0) * N + ga;
            acc8<N, T, KAHAN>(accC + ci, cmpC + ci, W, c);
        }
        __syncthreads();
    }
    // pass B: Y = g W_e(f) into shared memory, then Pi_e(Y)
    for (int li = ls; li < lend; ++li) {
        const int4 e = __ldg(P.rline + li);
        const T c = line_weight<T>(P, li);
        for (int u = tid; u < NU; u += NT) {
            const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
            T W[8], gv[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) W[t] = T(0);
            for (int j = 1; j <= e.w; ++j) {
                const T* bp = gwf + (((be + j * e.y) & M) * SW + ((a0 + j * e.x) & M)) * N + ((ga + j * e.z) & M);
                const T* bm = gwf + (((be - j * e.y) & M) * SW + ((a0 - j * e.x) & M)) * N + ((ga - j * e.z) & M);
#pragma unroll
                for (int t = 0; t < 8; ++t) W[t] += bp[t * N] + bm[t * N];
            }
            load8<N>(gC + (be * N + a0) * N + ga, gv);
            T* yp = g + (be * N + ga) * SA;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const T y = gv[t] * W[t];
                for (int a = a0 + t; a < SA; a += N) yp[a] = y;
            }
        }
        __syncthreads();
        const int rs = __ldg(P.rrow_start + li), re = __ldg(P.rrow_start + li + 1);
        for (int u = tid; u < NU; u += NT) {
            const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
            T P0 = T(0), D[7], Pv[8];
#pragma unroll
            for (int t = 0; t < 7; ++t) D[t] = T(0);
            plane_rows<N>(P.rrow, rs, re, g, be, ga, a0, P0, D);
            Pv[0] = P0;
#pragma unroll
            for (int t = 1; t < 8; ++t) Pv[t] = Pv[t - 1] + D[t - 1];
            const int ci = (be * N + a0) * N + ga;
            acc8<N, T, KAHAN>(accC + ci, cmpC + ci, Pv, c);
        }
        __syncthreads();
    }
    // class sums to the cell indices p = M q (mod N)
    for (int u = tid; u < NU; u += NT) {
        const int ga = u & M, be = (u / N) & M, a0 = (u / N2) * 8;
        const int ci = (be * N + a0) * N + ga;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int al = a0 + t;
            const int o = ((Mm[0] * al + Mm[1] * be + Mm[2] * ga) & M) * N2 +
                          ((Mm[3] * al + Mm[4] * be + Mm[5] * ga) & M) * N + ((Mm[6] * al + Mm[7] * be + Mm[8] * ga) & M);
            if (KAHAN) {
                T s = dst[o], cc = comp[o];
                comp_add<T, true>(s, cc, accC[ci + t * N] + cmpC[ci + t * N]);
                dst[o] = s;
                comp[o] = cc;
            } else {
                dst[o] += accC[ci + t * N];
            }
        }
    }
    __syncthreads();
}

enum { F3_FWD = 0, F3_JVP = 1, F3_VJP = 2 };

// One work item: the loss part (first chunk) or zero, then for every class
// with lines in [lb, le) the class sums.  Forward: sum c W_e(f) P_e(f).
// JVP with tangent d: loss -d (K * f) - f (K * d), gain
// sum c [W_e(d) P_e(f) + W_e(f) P_e(d)] as two passes (plane rows of f with
// windows of d, then rows of d with windows of f).
template <typename T, bool KAHAN, int N, int MODE>
__device__ void rows3d_item(const PlanDev& P, const int lb, const int le, const bool do_loss,
                            const T* __restrict__ fcell, const T* __restrict__ acell, T* __restrict__ g,
                            typename Cplx<T>::type* A, typename Cplx<T>::type* B, T* __restrict__ comp, T* gw,
                            T* __restrict__ dst) {
    using C = typename Cplx<T>::type;
    constexpr int N3 = N * N * N, NW = N * rows_sw<N>() * N;
    const int NT = blockDim.x, tid = threadIdx.x;

    if (do_loss) {
        // forward: K * f; JVP: K * f and K * d; VJP: K * f and K * (g f)
        for (int i = tid; i < N3; i += NT) {
            const T im = MODE == F3_JVP ? acell[i] : (MODE == F3_VJP ? acell[i] * fcell[i] : T(0));
            A[i] = C{fcell[i], im};
        }
        __syncthreads();
        const C* conv = loss_conv<T, N>(P, A, B);
        for (int i = tid; i < N3; i += NT) {
            const C k = conv[i];
            if (MODE == F3_JVP) dst[i] = -acell[i] * k.x - fcell[i] * k.y;
            else if (MODE == F3_VJP) dst[i] = -(acell[i] * k.x + k.y);
            else dst[i] = -fcell[i] * k.x;
        }
    } else {
        for (int i = tid; i < N3; i += NT) dst[i] = T(0);
    }
    if (KAHAN)
        for (int i = tid; i < N3; i += NT) comp[i] = T(0);
    __syncthreads();

    if (MODE == F3_VJP) {
        // scratch after the window copy gw: X (window layout), g, acc and
        // its compensation in compact class coordinates
        T* X = gw + NW;
        T* gC = X + NW;
        T* accC = gC + N3;
        T* cmpC = accC + N3;
        for (int k = 0; k < P.n_rclass; ++k) {
            const int* cdp = P.rclass + k * QDVM_RCLASS_INTS;
            const int ls = max(__ldg(cdp + 18), lb), lend = min(__ldg(cdp + 19), le);
            if (ls >= lend) continue;
            int Mm[9], Mi[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                Mm[t] = __ldg(cdp + t);
                Mi[t] = __ldg(cdp + 9 + t);
            }
            vjp_class<T, KAHAN, N>(P, Mm, Mi, ls, lend, fcell, acell, g, gw, X, gC, accC, cmpC, dst, comp);
        }
    }
    constexpr int passes = MODE == F3_JVP ? 2 : (MODE == F3_FWD ? 1 : 0);
    for (int pass = 0; pass < passes; ++pass) {
        const T* rsrc = pass ? acell : fcell;
        const T* wsrc = pass ? fcell : acell;
        for (int k = 0; k < P.n_rclass; ++k) {
            const int* cdp = P.rclass + k * QDVM_RCLASS_INTS;
            const int ls = max(__ldg(cdp + 18), lb), lend = min(__ldg(cdp + 19), le);
            if (ls >= lend) continue;
            int Mm[9], Mi[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                Mm[t] = __ldg(cdp + t);
                Mi[t] = __ldg(cdp + 9 + t);
            }
            if (MODE == F3_JVP) relayout_glob<T, N>(Mi, wsrc, gw);
            relayout_prefix<T, N>(Mi, rsrc, g);  // ends with a barrier
            // the shared central row: A = floor(Ntilde / |u|_inf), u = (Mm[0], Mm[3], Mm[6])
            const int un = max(abs(Mm[0]), max(abs(Mm[3]), abs(Mm[6])));
            const int A = P.Ntilde / un;
            class_units_prefix<T, KAHAN, N, MODE == F3_JVP>(P, Mm, ls, lend, A, A > 0 ? 2 : 0, g, gw, dst, comp);
            __syncthreads();
        }
    }
    if (KAHAN) {
        for (int i = tid; i < N3; i += NT) dst[i] = dst[i] + comp[i];
    }
}

template <typename T, bool KAHAN, int N, int MODE>
__global__ void __launch_bounds__(f3_threads(N), 1) k_rows3d(BatchDev Bt, int n_cells, int Cn, const int* __restrict__ cell_plan,
                                                       const int64_t* __restrict__ cell_offset,
                                                       const int* __restrict__ order, int* counter,
                                                       const T* __restrict__ f, const T* __restrict__ aux,
                                                       T* __restrict__ out, T* __restrict__ part, size_t part_stride,
                                                       char* scratch, size_t scr_stride) {
    using C = typename Cplx<T>::type;
    constexpr int N3 = N * N * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_cell;
    __shared__ PlanDev s_plan;
    const int n_items = n_cells * Cn;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            int cell = -1;
            if (it < n_items) cell = order[it / Cn];
            s_item = cell >= 0 ? it : -1;
            s_cell = cell;
            if (cell >= 0) {
                const int pi = cell_plan[cell];
#pragma unroll
                for (int q = 0; q < QDVM_MAX_BATCH_PLANS; ++q)
                    if (q == pi) s_plan = Bt.p[q];
            }
        }
        __syncthreads();
        const int item = s_item, cell = s_cell;
        if (item < 0) break;
        const PlanDev P = s_plan;
        const int chunk = item % Cn;
        const int lpc = (P.n_lines + Cn - 1) / Cn;
        const int lb = min(chunk * lpc, P.n_lines), le = min(lb + lpc, P.n_lines);
        const int64_t off = cell_offset[cell];
        T* dst = Cn == 1 ? out + off : part + ((size_t)cell * Cn + chunk) * part_stride;
        // scratch: FFT buffers A, B (complex N^3 each), compensation (N^3),
        // window copy (JVP)
        C* A = reinterpret_cast<C*>(scratch + (size_t)blockIdx.x * scr_stride);
        C* B = A + N3;
        T* comp = reinterpret_cast<T*>(B + N3);
        T* gw = comp + N3;
        rows3d_item<T, KAHAN, N, MODE>(P, lb, le, chunk == 0, f + off, aux ? aux + off : nullptr,
                                       reinterpret_cast<T*>(smem_raw), A, B, comp, gw, dst);
        __syncthreads();
    }
}

__global__ void k_fast3d_single_init(int* counter, int* order, int* cell_plan, int64_t* cell_offset) {
    *counter = 0;
    *order = 0;
    *cell_plan = 0;
    *cell_offset = 0;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct F3Layout {
    int N, C, grid, mode;
    bool rows;
    size_t smem, scr_stride, part_stride, off_scr, off_part, total;
};

template <typename T>
using F3Kernel = void (*)(BatchDev, int, int, const int*, const int64_t*, const int*, int*, const T*, const T*, T*, T*,
                          size_t, char*, size_t);

// the kernel for a layout: point-by-point plane sums (forward only) or the
// row form, forward or JVP
template <typename T, bool KAHAN, int N>
F3Kernel<T> f3_kernel(bool rows, int mode) {
    if (!rows) return k_fast3d<T, KAHAN, N>;
    if (mode == F3_VJP) return k_rows3d<T, KAHAN, N, F3_VJP>;
    return mode == F3_JVP ? k_rows3d<T, KAHAN, N, F3_JVP> : k_rows3d<T, KAHAN, N, F3_FWD>;
}

template <typename T, bool KAHAN>
F3Kernel<T> f3_kernel_n(int N, bool rows, int mode) {
    return N == 32 ? f3_kernel<T, KAHAN, 32>(rows, mode) : f3_kernel<T, KAHAN, 16>(rows, mode);
}

template <typename T>
int f3_occupancy(F3Kernel<T> k, int threads, size_t smem) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem);
    return per > 0 ? per : 1;
}

int f3_occ(int N, int prec, size_t smem, bool rows, int mode) {
    const int nt = f3_threads(N);
    if (prec == QDVM_F64) return f3_occupancy<double>(f3_kernel_n<double, false>(N, rows, mode), nt, smem);
    if (prec == QDVM_F32_KAHAN) return f3_occupancy<float>(f3_kernel_n<float, true>(N, rows, mode), nt, smem);
    return f3_occupancy<float>(f3_kernel_n<float, false>(N, rows, mode), nt, smem);
}

// 0 unless every plan is 3D with the same N in {16, 32}, has the loss
// transform, and the re-indexed cell (row form, when every plan has row
// tables) or the haloed cell (point-by-point plane sums, forward only) fits
// in shared memory.
int f3_size(const BatchDev& b, int prec, int mode, size_t* smem, bool* rows) {
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    const int N = b.p[0].N;
    int H = 0;
    bool r = true;
    if (N != 16 && N != 32) return 0;
    for (int i = 0; i < b.n_plans; ++i) {
        const PlanDev& p = b.p[i];
        if (p.d != 3 || p.N != N || !p.khat || !p.khat_f || !p.tw || !p.tw_f) return 0;
        H = std::max(H, p.Ntilde);
        r = r && p.n_rclass > 0;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the VJP's row layout (stride rows_sa) and the forward / JVP prefix form (rows_sp)
    const size_t sa = (size_t)(N == 32 ? std::max(rows_sa<32>(), rows_sp<32>()) : std::max(rows_sa<16>(), rows_sp<16>()));
    const size_t s_rows = (size_t)N * N * sa * es, s_dir = (size_t)(N + 2 * H) * N * N * es;
    r = r && s_rows + 1024 <= (size_t)optin;
    if (mode != F3_FWD && !r) return 0;
    const size_t s = r ? s_rows : s_dir;
    if (s + 1024 > (size_t)optin) return 0;
    if (smem) *smem = s;
    if (rows) *rows = r;
    return N;
}

F3Layout f3_layout(const BatchDev& b, int mode, int n_cells, int prec, bool single, int chunks) {
    F3Layout g{};
    g.mode = mode;
    g.N = f3_size(b, prec, mode, &g.smem, &g.rows);
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    const size_t n3 = (size_t)g.N * g.N * g.N;
    int maxLines = 1;
    for (int i = 0; i < b.n_plans; ++i) maxLines = std::max(maxLines, b.p[i].n_lines);
    const int slots = g.N ? f3_occ(g.N, prec, g.smem, g.rows, mode) * qdvm_num_sms() : 1;
    const int nc = std::max(n_cells, 1);
    if (single)
        g.C = std::max(1, std::min(maxLines, slots));
    else
        g.C = std::max(1, std::min(maxLines, (4 * slots + nc - 1) / nc));
    if (!single && nc >= 2 * slots) g.C = 1;
    if (chunks > 0) g.C = std::max(1, std::min(maxLines, chunks));
    g.grid = (int)std::max(1L, std::min((long)nc * g.C, (long)slots));
    // two complex N^3 FFT buffers, the compensation field (row form), the
    // window copy in class coordinates (JVP, VJP) and for the VJP the product
    // X in window layout plus g, acc, compensation in compact layout
    const size_t sw = (size_t)g.N * (g.N == 32 ? rows_sw<32>() : rows_sw<16>()) * g.N;
    size_t fields = 2 * n3 * 2 + (g.rows ? n3 : 0);
    if (mode == F3_JVP) fields += sw;
    if (mode == F3_VJP) fields += 2 * sw + 3 * n3;
    g.scr_stride = a256(fields * es);
    g.part_stride = g.C > 1 ? n3 : 0;
    g.off_scr = 256 + a256((size_t)nc * sizeof(int)) + 256;  // counter, order, single-cell tables
    g.off_part = g.off_scr + (size_t)g.grid * g.scr_stride;
    g.total = g.off_part + (g.C > 1 ? a256((size_t)nc * g.C * n3 * es) : 0);
    return g;
}

template <typename T, bool KAHAN>
void f3_launch(const F3Layout& g, const BatchDev& b, int n_cells, const int* cp, const int64_t* co, const int* order,
               int* counter, const void* f, const void* aux, void* out, char* base, cudaStream_t st) {
    const F3Kernel<T> k = f3_kernel_n<T, KAHAN>(g.N, g.rows, g.mode);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    k<<<g.grid, f3_threads(g.N), g.smem, st>>>(b, n_cells, g.C, cp, co, order, counter, static_cast<const T*>(f),
                                           static_cast<const T*>(aux), static_cast<T*>(out),
                                           reinterpret_cast<T*>(base + g.off_part), g.part_stride, base + g.off_scr,
                                           g.scr_stride);
}

template <typename T, bool KAHAN>
void f3_reduce(const F3Layout& g, const BatchDev& b, int n_cells, const int* cp, const int64_t* co, char* base,
               void* out, cudaStream_t st) {
    dim3 grid(8, std::max(1, std::min(n_cells, 65535)));
    eng::k_reduce_chunks<T, KAHAN><<<grid, 256, 0, st>>>(b, n_cells, g.C, cp, co,
                                                          reinterpret_cast<const T*>(base + g.off_part), g.part_stride,
                                                          static_cast<T*>(out));
}

int f3_mode(int qdvm_mode) {
    return qdvm_mode == QDVM_MODE_JVP ? F3_JVP : (qdvm_mode == QDVM_MODE_VJP ? F3_VJP : F3_FWD);
}

}  // namespace

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st);

bool fast3d_supported(int mode, const BatchDev& b, int prec) {
    if (mode != QDVM_MODE_FWD && mode != QDVM_MODE_JVP && mode != QDVM_MODE_VJP) return false;
    return f3_size(b, prec, f3_mode(mode), nullptr, nullptr) != 0;
}

size_t fast3d_workspace(int mode, const BatchDev& b, int n_cells, int prec, bool single, int chunks) {
    return f3_layout(b, f3_mode(mode), single ? 1 : n_cells, prec, single, chunks).total;
}

qdvm_status fast3d_run(int mode, const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                       const void* f, const void* aux, void* out, double* moments, int prec, void* ws,
                       size_t ws_bytes, bool single, int chunks, cudaStream_t st) {
    const int nc = single ? 1 : n_cells;
    if (mode != QDVM_MODE_FWD && mode != QDVM_MODE_JVP && mode != QDVM_MODE_VJP)
        return qdvm_fail(QDVM_ERR_UNSUPPORTED, "unknown mode for the 3D FFT-loss evaluator");
    if (mode != QDVM_MODE_FWD && !aux) return qdvm_fail(QDVM_ERR_INVALID_ARG, "JVP / VJP without a tangent or cotangent");
    const F3Layout g = f3_layout(b, f3_mode(mode), nc, prec, single, chunks);
    if (!g.N) return qdvm_fail(QDVM_ERR_INVALID_ARG, "the 3D FFT-loss evaluator does not support this batch");
    if (!ws || ws_bytes < g.total) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for the 3D evaluator");
    char* base = static_cast<char*>(ws);
    int* counter = reinterpret_cast<int*>(base);
    int* order = reinterpret_cast<int*>(base + 256);
    if (single) {
        char* tab = base + 256 + 256;
        int* cp = reinterpret_cast<int*>(tab);
        int64_t* co = reinterpret_cast<int64_t*>(tab + 128);
        k_fast3d_single_init<<<1, 1, 0, st>>>(counter, order, cp, co);
        QDVM_LAUNCH_CHECK("3D evaluator single init");
        cell_plan = cp;
        cell_offset = co;
    } else {
        qdvm_status s = schedule_launch(b, nc, cell_plan, order, counter, st);
        if (s != QDVM_OK) return s;
    }
    if (prec == QDVM_F64) f3_launch<double, false>(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, st);
    else if (prec == QDVM_F32_KAHAN) f3_launch<float, true>(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, st);
    else f3_launch<float, false>(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, st);
    QDVM_LAUNCH_CHECK("3D evaluator launch");
    if (g.C > 1) {
        if (prec == QDVM_F64) f3_reduce<double, false>(g, b, nc, cell_plan, cell_offset, base, out, st);
        else if (prec == QDVM_F32_KAHAN) f3_reduce<float, true>(g, b, nc, cell_plan, cell_offset, base, out, st);
        else f3_reduce<float, false>(g, b, nc, cell_plan, cell_offset, base, out, st);
        QDVM_LAUNCH_CHECK("3D evaluator reduce launch");
    }
    if (moments) return moments_batched_launch(b, nc, cell_plan, cell_offset, out, prec, moments, st);
    return QDVM_OK;
}
