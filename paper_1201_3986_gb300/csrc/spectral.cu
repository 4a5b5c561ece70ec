// The pseudo-spectral route of Section 3.1: Q through the Fourier modes,
//     Qhat_I = sum_{K + L = I} beta~(K, L) fhat_K fhat_L          (eq. (sysDiff))
//     beta~(K, L) = beta(K, L) - beta(L, L),
//     beta(K, L)  = sum_{(k, l)} Gamma(k) e_K(k) e_L(l)            (eq. (betaKL))
// with fhat_I = N^{-d} sum_i f_i e_{-I}(i), Q_i = sum_I Qhat_I e_I(i) and
// e_K(k) = exp(2 pi i K.k / N).  It costs O(N^{2d}) per cell and a dense
// N^d x N^d table: a second evaluation of the same operator, independent of
// the line sums of the fast evaluators (it shares only the plan's lines).
//
// The table: the pair set is symmetric under k -> -k and l -> -l separately
// (the box, orthogonality, the line restriction and Gamma are), so beta is
// real and, grouping the pairs by the line e of k (eq. (decDVM)),
//     beta(K, L) = sum_e D_e(K) P_e(L),
//     D_e(K) = c_e sum_{0<|j|<=J_e} cos(2 pi j K.e / N),
//     P_e(L) = sum_{l in e^perp, 0<|l|_inf<=Ntilde} cos(2 pi L.l / N),
// a product of an (N^d x #lines) and a (#lines x N^d) matrix, formed here in
// FP64 by a tiled kernel.
#include <algorithm>

#include "qdvm_internal.cuh"

namespace {

template <typename T>
struct Cx {
    T x, y;
};

// cos(2 pi t / N) for t in [0, N)
__device__ __forceinline__ double cos2pi(int t, int N) { return cospi(2.0 * (double)t / (double)N); }

// Multi-index of the flat mode K (row-major, last axis fastest).
__device__ __forceinline__ void unflat(int K, int d, int N, int k[3]) {
    k[2] = 0;
    for (int a = d - 1; a >= 0; --a) {
        k[a] = K % N;
        K /= N;
    }
}

// D_e(K) and P_e(K) for every line e (blockIdx.y) and mode K.
__global__ void k_spec_lines(int d, int N, int M, const int4* __restrict__ lines, const double* __restrict__ c,
                             const int* __restrict__ plane_start, const char4* __restrict__ plane,
                             double* __restrict__ D, double* __restrict__ P) {
    __shared__ double cs[256];
    for (int t = threadIdx.x; t < N; t += blockDim.x) cs[t] = cos2pi(t, N);
    __syncthreads();
    const int e = blockIdx.y;
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= M) return;
    int k[3];
    unflat(K, d, N, k);
    const int4 v = lines[e];
    int dot = (k[0] * v.x + k[1] * v.y + k[2] * v.z) % N;
    dot += dot < 0 ? N : 0;
    double s = 0.0;
    for (int j = 1; j <= v.w; ++j) s += cs[(j * dot) % N];
    D[(size_t)e * M + K] = 2.0 * c[e] * s;
    double p = 0.0;
    for (int q = plane_start[e]; q < plane_start[e + 1]; ++q) {
        const char4 l = plane[q];
        int t = (k[0] * l.x + k[1] * l.y + k[2] * l.z) % N;
        t += t < 0 ? N : 0;
        p += cs[t];
    }
    P[(size_t)e * M + K] = p;
}

// beta(L, L) = sum_e D_e(L) P_e(L)
__global__ void k_spec_diag(int M, int n_lines, const double* __restrict__ D, const double* __restrict__ P,
                            double* __restrict__ diag) {
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= M) return;
    double s = 0.0;
    for (int e = 0; e < n_lines; ++e) s += D[(size_t)e * M + L] * P[(size_t)e * M + L];
    diag[L] = s;
}

// table[K M + L] = sum_e D_e(K) P_e(L) - beta(L, L), 64 x 64 tiles of
// (K, L), 16 lines per shared-memory stage; thread (tx, ty) owns rows
// K = K0 + ty + 16 r and columns L = L0 + tx + 16 s (r, s < 4), so a warp's
// stores are 16 consecutive L of two rows.
template <typename TO>
__global__ void __launch_bounds__(256) k_spec_beta(int M, int n_lines, const double* __restrict__ D,
                                                   const double* __restrict__ P, const double* __restrict__ diag,
                                                   TO* __restrict__ table) {
    constexpr int TB = 64, LC = 16;
    __shared__ double Ds[LC][TB], Ps[LC][TB];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int K0 = blockIdx.y * TB, L0 = blockIdx.x * TB;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = 0.0;
    for (int e0 = 0; e0 < n_lines; e0 += LC) {
        for (int i = threadIdx.x; i < LC * TB; i += 256) {
            const int le = i / TB, col = i % TB, e = e0 + le;
            const bool ok = e < n_lines;
            Ds[le][col] = ok && K0 + col < M ? D[(size_t)e * M + K0 + col] : 0.0;
            Ps[le][col] = ok && L0 + col < M ? P[(size_t)e * M + L0 + col] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int le = 0; le < LC; ++le) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = Ds[le][ty + 16 * r];
#pragma unroll
            for (int s = 0; s < 4; ++s) b[s] = Ps[le][tx + 16 * s];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int K = K0 + ty + 16 * r;
        if (K >= M) continue;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int L = L0 + tx + 16 * s;
            if (L < M) table[(size_t)K * M + L] = (TO)(acc[r][s] - diag[L]);
        }
    }
}

// One DFT pass along one axis (stride S between neighbours on the axis) of
// n_cells arrays of M modes, one output per thread:
//     out[k] = scale sum_n in[n] exp(sign 2 pi i k n / N).
// IN_REAL: the input is real (the cells' f); OUT_REAL: only the real part is
// written (Q).
template <typename T, bool IN_REAL, bool OUT_REAL>
__global__ void k_dft_pass(int N, int S, int M, int n_cells, const void* __restrict__ in, void* __restrict__ out,
                           int sign, T scale) {
    __shared__ T cw[256], sw[256];
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)t / (double)N, &s, &c);
        cw[t] = (T)c;
        sw[t] = (T)(sign * s);
    }
    __syncthreads();
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (size_t)n_cells * M) return;
    const size_t cell = g / M;
    const int idx = (int)(g - cell * M);
    const int k = (idx / S) % N;
    const size_t base = cell * M + (idx - k * S);
    T re = T(0), im = T(0);
    int t = 0;  // k n mod N
    for (int n = 0; n < N; ++n) {
        T xr, xi;
        if constexpr (IN_REAL) {
            xr = static_cast<const T*>(in)[base + (size_t)n * S];
            xi = T(0);
        } else {
            const Cx<T> z = static_cast<const Cx<T>*>(in)[base + (size_t)n * S];
            xr = z.x;
            xi = z.y;
        }
        re += xr * cw[t] - xi * sw[t];
        im += xr * sw[t] + xi * cw[t];
        t += k;
        t -= t >= N ? N : 0;
    }
    if constexpr (OUT_REAL) {
        static_cast<T*>(out)[g] = scale * re;
    } else {
        static_cast<Cx<T>*>(out)[g] = Cx<T>{scale * re, scale * im};
    }
}

// Qhat_c(I) = sum_K beta~(K, I - K) fhat_c(K) fhat_c(I - K) for CB cells per
// CTA (their spectra in shared memory, 128 KB: one CTA per SM), one mode I
// per thread, CTAs of up to 1024 threads (32 warps to hide the L2 latency of
// the table loads; smaller when the batch would leave SMs idle).  For a fixed K the threads of a warp read consecutive
// table entries (L = I - K runs along the last axis).
template <typename T, bool KAHAN, int CB, int DIM>
__global__ void __launch_bounds__(1024) k_spec_conv(int N, int M, int n_cells, const T* __restrict__ table,
                                                   const Cx<T>* __restrict__ fh, Cx<T>* __restrict__ qh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T>* s = reinterpret_cast<Cx<T>*>(smem_raw);
    const int c0 = blockIdx.y * CB;
    for (int i = threadIdx.x; i < CB * M; i += blockDim.x) {
        const int cb = i / M, K = i - cb * M;
        s[i] = c0 + cb < n_cells ? fh[(size_t)(c0 + cb) * M + K] : Cx<T>{T(0), T(0)};
    }
    __syncthreads();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= M) return;
    int ii[3];
    unflat(I, DIM, N, ii);
    T ar[CB], ai[CB], cr[CB], ci[CB];
#pragma unroll
    for (int b = 0; b < CB; ++b) ar[b] = ai[b] = cr[b] = ci[b] = T(0);
    auto term = [&](int K, int L, T bt) {
#pragma unroll
        for (int b = 0; b < CB; ++b) {
            const Cx<T> z = s[b * M + K], y = s[b * M + L];
            comp_add<T, KAHAN>(ar[b], cr[b], bt * (z.x * y.x - z.y * y.y));
            comp_add<T, KAHAN>(ai[b], ci[b], bt * (z.x * y.y + z.y * y.x));
        }
    };
    // one row of K (the last axis), K = Kb + t and L = Lb + l_t with l_t
    // running down from l (mod N): the table loads of 8 consecutive terms
    // are issued before their arithmetic (L2 latency)
    auto row = [&](const int Kb, const int Lb, int l) {
        int t = 0;
        for (; t + 8 <= N; t += 8) {
            T bt[8];
            int Ls[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                Ls[u] = Lb + l;
                bt[u] = table[(size_t)(Kb + t + u) * M + Ls[u]];
                l = l == 0 ? N - 1 : l - 1;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) term(Kb + t + u, Ls[u], bt[u]);
        }
        for (; t < N; ++t) {
            term(Kb + t, Lb + l, table[(size_t)(Kb + t) * M + Lb + l]);
            l = l == 0 ? N - 1 : l - 1;
        }
    };
    for (int k0 = 0; k0 < N; ++k0) {
        int l0 = ii[0] - k0;
        l0 += l0 < 0 ? N : 0;
        if constexpr (DIM == 2) {
            row(k0 * N, l0 * N, ii[1]);
        } else {
            for (int k1 = 0; k1 < N; ++k1) {
                int l1 = ii[1] - k1;
                l1 += l1 < 0 ? N : 0;
                row((k0 * N + k1) * N, (l0 * N + l1) * N, ii[2]);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < CB; ++b)
        if (c0 + b < n_cells)
            qh[(size_t)(c0 + b) * M + I] = KAHAN ? Cx<T>{ar[b] + cr[b], ai[b] + ci[b]} : Cx<T>{ar[b], ai[b]};
}

bool spectral_supported(const qdvm_plan_s* p) { return (p->d == 2 && p->N <= 64) || (p->d == 3 && p->N <= 16); }

size_t modes(const qdvm_plan_s* p) { return p->d == 2 ? (size_t)p->N * p->N : (size_t)p->N * p->N * p->N; }

// Cells per CTA of the spectral sum: the spectra of CB cells in 128 KB.
template <typename T>
constexpr int conv_cb() {
    return sizeof(T) == 8 ? 2 : 4;
}

template <typename T, bool KAHAN>
qdvm_status launch_spectral(const qdvm_plan_s* p, const T* table, int n_cells, const T* f, T* Q, void* ws,
                            cudaStream_t st) {
    const int N = p->N, d = p->d, M = (int)modes(p);
    using C = Cx<T>;
    C* A = static_cast<C*>(ws);
    C* B = A + (size_t)n_cells * M;
    const size_t tot = (size_t)n_cells * M;
    const int nb = (int)((tot + 255) / 256);
    // forward: f (real) -> A along the last axis, then the other axes
    int S = 1;
    k_dft_pass<T, true, false><<<nb, 256, 0, st>>>(N, S, M, n_cells, f, A, -1, T(1.0 / M));
    C* cur = A;
    C* oth = B;
    for (int a = d - 2; a >= 0; --a) {
        S *= N;
        k_dft_pass<T, false, false><<<nb, 256, 0, st>>>(N, S, M, n_cells, cur, oth, -1, T(1));
        std::swap(cur, oth);
    }
    // the spectral sum: cur (fhat) -> oth (Qhat)
    constexpr int CB = conv_cb<T>();
    const size_t smem = (size_t)CB * M * sizeof(C);
    // the largest CTA (up to 1024 threads) that still gives every SM a CTA
    const int groups = (n_cells + CB - 1) / CB;
    int nt = std::min(1024, (M + 31) / 32 * 32);
    while (nt > 256 && (long long)((M + nt - 1) / nt) * groups < qdvm_num_sms()) nt /= 2;
    dim3 grid((M + nt - 1) / nt, groups);
    if (d == 2) {
        auto k = k_spec_conv<T, KAHAN, CB, 2>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, nt, smem, st>>>(N, M, n_cells, table, cur, oth);
    } else {
        auto k = k_spec_conv<T, KAHAN, CB, 3>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, nt, smem, st>>>(N, M, n_cells, table, cur, oth);
    }
    std::swap(cur, oth);
    // inverse: Qhat -> Q (real), last axis first
    S = 1;
    for (int a = d - 1; a >= 1; --a) {
        k_dft_pass<T, false, false><<<nb, 256, 0, st>>>(N, S, M, n_cells, cur, oth, +1, T(1));
        std::swap(cur, oth);
        S *= N;
    }
    k_dft_pass<T, false, true><<<nb, 256, 0, st>>>(N, S, M, n_cells, cur, Q, +1, T(1));
    QDVM_LAUNCH_CHECK("spectral evaluation");
    return QDVM_OK;
}

}  // namespace

extern "C" qdvm_status qdvm_spectral_table_entries(qdvm_plan_t p, size_t* n) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!n) return qdvm_fail(QDVM_ERR_INVALID_ARG, "n is NULL");
    if (!spectral_supported(p))
        return qdvm_fail(QDVM_ERR_UNSUPPORTED, "spectral route: d = 2 with N <= 64 or d = 3 with N <= 16");
    *n = modes(p) * modes(p);
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_spectral_table(qdvm_plan_t p, void* table, int prec, void* stream) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!spectral_supported(p))
        return qdvm_fail(QDVM_ERR_UNSUPPORTED, "spectral route: d = 2 with N <= 64 or d = 3 with N <= 16");
    if (!table) return qdvm_fail(QDVM_ERR_INVALID_ARG, "table is NULL");
    const int M = (int)modes(p), A = p->n_lines;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *D = nullptr, *P = nullptr, *diag = nullptr;
    cudaError_t e;
    auto done = [&](qdvm_status s) {
        cudaFree(D);
        cudaFree(P);
        cudaFree(diag);
        return s;
    };
    if ((e = cudaMalloc(&D, (size_t)A * M * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&P, (size_t)A * M * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&diag, (size_t)M * sizeof(double))) != cudaSuccess)
        return done(qdvm_cuda_status(e, "spectral table temporaries"));
    k_spec_lines<<<dim3((M + 255) / 256, A), 256, 0, st>>>(p->d, p->N, M, p->d_lines, p->d_c, p->d_plane_start,
                                                           p->d_plane, D, P);
    k_spec_diag<<<(M + 255) / 256, 256, 0, st>>>(M, A, D, P, diag);
    dim3 grid((M + 63) / 64, (M + 63) / 64);
    if (prec == QDVM_F64)
        k_spec_beta<double><<<grid, 256, 0, st>>>(M, A, D, P, diag, static_cast<double*>(table));
    else
        k_spec_beta<float><<<grid, 256, 0, st>>>(M, A, D, P, diag, static_cast<float*>(table));
    if ((e = cudaGetLastError()) != cudaSuccess) return done(qdvm_cuda_status(e, "spectral table kernels"));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(qdvm_cuda_status(e, "spectral table"));
    return done(QDVM_OK);
}

extern "C" qdvm_status qdvm_spectral_workspace(qdvm_plan_t p, int n_cells, int prec, size_t* bytes) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!bytes || n_cells < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "bytes is NULL or n_cells < 0");
    if (prec != QDVM_F64 && prec != QDVM_F32 && prec != QDVM_F32_KAHAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "bad precision");
    if (!spectral_supported(p))
        return qdvm_fail(QDVM_ERR_UNSUPPORTED, "spectral route: d = 2 with N <= 64 or d = 3 with N <= 16");
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    *bytes = 2 * (size_t)n_cells * modes(p) * 2 * es;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_eval_spectral(qdvm_plan_t p, const void* table, int n_cells, const void* f, void* Q,
                                          int prec, void* ws, size_t ws_bytes, void* stream) {
    size_t need = 0;
    qdvm_status s = qdvm_spectral_workspace(p, n_cells, prec, &need);
    if (s != QDVM_OK) return s;
    if (n_cells == 0) return QDVM_OK;
    if (!table || !f || !Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL device array");
    if (f == Q) return qdvm_fail(QDVM_ERR_INVALID_ARG, "f must not alias Q");
    if (!ws || ws_bytes < need) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_eval_spectral");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (prec) {
        case QDVM_F64:
            return launch_spectral<double, false>(p, static_cast<const double*>(table), n_cells,
                                                  static_cast<const double*>(f), static_cast<double*>(Q), ws, st);
        case QDVM_F32:
            return launch_spectral<float, false>(p, static_cast<const float*>(table), n_cells,
                                                 static_cast<const float*>(f), static_cast<float*>(Q), ws, st);
        default:
            return launch_spectral<float, true>(p, static_cast<const float*>(table), n_cells,
                                                static_cast<const float*>(f), static_cast<float*>(Q), ws, st);
    }
}
