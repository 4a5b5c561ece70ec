// Plan construction: the line set A_m of Section 3.2 (Farey-type series
// F^1 / F^2, lines through 0 in [-m, m]^d), the window half-lengths
// J_e = floor(Ntilde / |e|_inf), the decoupled weights c_e of eq. (decoup),
// the 2D pairing e <-> e^perp of Remark 3.4(3) and the 3D plane lists
// e^perp ∩ [-Ntilde, Ntilde]^3 of eq. (decDVM).  Every table is computed by a
// kernel; the host only sizes allocations.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "qdvm_internal.cuh"

// ------------------------------------------------------------ error state

static thread_local std::string g_last_error;

void qdvm_set_error(const std::string& msg) { g_last_error = msg; }

qdvm_status qdvm_fail(qdvm_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

qdvm_status qdvm_cuda_status(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return QDVM_ERR_OOM;
    return QDVM_ERR_CUDA;
}

bool qdvm_plan_ok(const qdvm_plan_s* p) { return p != nullptr && p->magic == QDVM_PLAN_MAGIC; }

extern "C" const char* qdvm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* qdvm_status_string(qdvm_status s) {
    switch (s) {
        case QDVM_OK: return "ok";
        case QDVM_ERR_INVALID_ARG: return "invalid argument";
        case QDVM_ERR_UNSUPPORTED: return "unsupported configuration";
        case QDVM_ERR_OOM: return "out of device memory";
        case QDVM_ERR_CUDA: return "CUDA error";
        case QDVM_ERR_TIMEOUT: return "timeout";
        case QDVM_ERR_BAD_PLAN: return "bad plan handle";
    }
    return "unknown status";
}

extern "C" const char* qdvm_version(void) { return "qdvm 0.1 (sm_103a)"; }

int qdvm_num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    return n;
}

// ------------------------------------------------------------ device helpers

__device__ __forceinline__ int iabs(int x) { return x < 0 ? -x : x; }

__device__ __forceinline__ int gcd_dev(int a, int b) {
    a = iabs(a);
    b = iabs(b);
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Candidate number idx of the lexicographic enumeration of [-n, n]^d
// (first axis slowest).
__device__ __forceinline__ void cand_vec(int idx, int d, int n, int v[3]) {
    int w = 2 * n + 1;
    v[0] = v[1] = v[2] = 0;
    for (int a = d - 1; a >= 0; --a) {
        v[a] = idx % w - n;
        idx /= w;
    }
}

// True if v is a canonical primitive direction on the shell |v|_inf == n.
__device__ __forceinline__ bool is_line_rep(const int v[3], int d, int n) {
    int linf = 0, g = 0, first = 0;
    for (int a = 0; a < d; ++a) {
        linf = max(linf, iabs(v[a]));
        g = gcd_dev(g, v[a]);
        if (first == 0) first = v[a];
    }
    return linf == n && g == 1 && first > 0;
}

// Block-wide exclusive scan of one int per thread (blockDim multiple of 32,
// at most 1024).  Returns the exclusive prefix; *total gets the block sum.
__device__ int block_exclusive_scan(int x, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    int base = wid > 0 ? warp_sums[wid - 1] : 0;
    int tot = warp_sums[nw - 1];
    __syncthreads();
    *total = tot;
    return base + incl - x;
}

// One block per shell n = blockIdx.x + 1: number of line representatives.
__global__ void k_shell_count(int d, int* counts) {
    const int n = blockIdx.x + 1;
    int w = 2 * n + 1, total = w * w;
    if (d == 3) total *= w;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int v[3];
        cand_vec(i, d, n, v);
        local += is_line_rep(v, d, n) ? 1 : 0;
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = cnt;
}

// One block per shell: write the representatives of the shell in
// lexicographic order at offsets[shell].
__global__ void k_shell_emit(int d, const int* offsets, int4* lines) {
    const int n = blockIdx.x + 1;
    int w = 2 * n + 1, total = w * w;
    if (d == 3) total *= w;
    int base = offsets[blockIdx.x];
    for (int c0 = 0; c0 < total; c0 += blockDim.x) {
        int i = c0 + threadIdx.x;
        int v[3] = {0, 0, 0};
        bool ok = false;
        if (i < total) {
            cand_vec(i, d, n, v);
            ok = is_line_rep(v, d, n);
        }
        int tot;
        int r = block_exclusive_scan(ok ? 1 : 0, &tot);
        if (ok) lines[base + r] = make_int4(v[0], v[1], v[2], 0);
        base += tot;
    }
}

// J_e and c_e per line.
__global__ void k_line_tables(int d, int n_lines, int Ntilde, int kernel, double h, int4* lines, double* c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_lines) return;
    int4 e = lines[i];
    int linf = max(iabs(e.x), max(iabs(e.y), iabs(e.z)));
    e.w = Ntilde / linf;
    lines[i] = e;
    double w = 1.0;
    if (kernel == QDVM_KERNEL_HP) {
        double hp = 1.0;
        for (int a = 0; a < 2 * d - 1; ++a) hp *= h;
        double n2 = (double)e.x * e.x + (double)e.y * e.y + (double)e.z * e.z;
        w = hp * sqrt(n2);
    }
    c[i] = w;
}

// 2D: keep e when it precedes its canonical partner e^perp = (-e1, e0)
// lexicographically (both lie on the same shell |.|_inf).  Single block.
__global__ void k_pairs(int n_lines, const int4* lines, const double* c, int4* pairs, double* pair_c, int cap,
                        int* n_out) {
    int base = 0;
    for (int c0 = 0; c0 < n_lines; c0 += blockDim.x) {
        int i = c0 + threadIdx.x;
        bool keep = false;
        int4 e = make_int4(0, 0, 0, 0);
        if (i < n_lines) {
            e = lines[i];
            int p0 = -e.y, p1 = e.x;
            if (p0 < 0 || (p0 == 0 && p1 < 0)) {
                p0 = -p0;
                p1 = -p1;
            }
            keep = (e.x < p0) || (e.x == p0 && e.y < p1);
        }
        int tot;
        int r = block_exclusive_scan(keep ? 1 : 0, &tot);
        if (keep && base + r < cap) {
            pairs[base + r] = make_int4(e.x, e.y, e.w, 0);
            pair_c[base + r] = c[i];
        }
        base += tot;
    }
    if (threadIdx.x == 0) *n_out = base;
}

// Tables of the running-sum (scan) line-sum engine of the 2D evaluator, one
// thread per pair {e, e^perp}.  A direction v = (v0, v1) with v0 != 0 (sign
// chosen so that v0 > 0) is walked in strips of S v0 rows: a piece starts on
// one of the first v0 rows of a strip, at any column x in [lo, lo + npg),
// and advances S steps of v (fewer in the last strip, so that it ends inside
// the cell), carrying the running window sum R = sum_{|j| <= J} f(. + j v).
// Every point of the cell lies on exactly one piece; pieces that start left
// of the cell (lo < 0) or leave it on the right write only their points
// inside it.  Reads reach (S - 1 + J)|v1| columns beyond the cell, which the
// evaluator's 2H halo allows when (S - 1 + J)|v1| <= 2H.  The horizontal
// direction (v0 = 0) is not walked.
//   scan[4 i + 2 d]     = (v0, v1, S, npg)      d = 0: v = e, d = 1: v = e^perp
//   scan[4 i + 2 d + 1] = (lo, ng, magic(npg), magic(v0))
// with ng the number of start rows and magic(D) = ceil(2^32 / D) (0 for
// D = 1), so that floor(a / D) = umulhi(a, magic(D)) for the small a used.
//   pairs[i].w = bit d set when direction d is walked.
// S (at most 32 per direction) minimises a per-thread cost model of a
// 256-thread CTA: the pieces of both directions dealt out to the threads in
// rounds, a round costing the longest piece (its first window, 2J + 1 loads
// and adds, a set-up, and about 10 instructions per further step).
__host__ __device__ inline unsigned div_magic_of(int D) { return D <= 1 ? 0u : 0xFFFFFFFFu / (unsigned)D + 1u; }

__device__ void strip_desc(int v0, int v1, int J, int N, int H, int S, int4* a, int4* b) {
    const int m = abs(v1);
    const int npg = N + (S - 1) * m;
    const int kf = N / (S * v0);
    const int ng = kf * v0 + min(v0, N - kf * S * v0);
    *a = make_int4(v0, v1, S, npg);
    *b = make_int4(v1 > 0 ? -(S - 1) * v1 : 0, ng, (int)div_magic_of(npg), (int)div_magic_of(v0));
}

__global__ void k_pair_scan(int n_pairs, int N, int H, int4* pairs, int4* scan) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pairs) return;
    int4 e = pairs[i];
    const int J = e.z;
    int v[2][2] = {{e.x, e.y}, {-e.y, e.x}};
    int smax[2];
    for (int d = 0; d < 2; ++d) {
        if (v[d][0] < 0) {
            v[d][0] = -v[d][0];
            v[d][1] = -v[d][1];
        }
        const int m = abs(v[d][1]);
        smax[d] = 0;
        if (v[d][0] == 0 || J < 1 || J * v[d][0] > H) continue;  // horizontal: not walked
        const int s = m ? (2 * H) / m - J + 1 : 32;
        smax[d] = max(0, min(s, min(32, (N + v[d][0] - 1) / v[d][0])));
    }
    // cost of direction d with S steps: (pieces, per-piece cost)
    auto pieces = [&](int d, int S) -> long long {
        int4 a, b;
        strip_desc(v[d][0], v[d][1], J, N, H, S, &a, &b);
        return (long long)a.w * b.y;
    };
    int best[2] = {0, 0};
    double best_cost = -1.0;
    for (int s0 = (smax[0] ? 1 : 0); s0 <= smax[0]; ++s0)
        for (int s1 = (smax[1] ? 1 : 0); s1 <= smax[1]; ++s1) {
            double work = 0.0, cmax = 0.0;
            long long np = 0;
            const int ss[2] = {s0, s1};
            for (int d = 0; d < 2; ++d) {
                if (!ss[d]) continue;
                const double c = 4 * J + 20 + 10.0 * ss[d];  // first window, set-up, steps
                const long long n = pieces(d, ss[d]);
                np += n;
                work += (double)n * c;
                cmax = fmax(cmax, c);
            }
            // rounds of pieces over the threads times the longest piece, the
            // total work breaking ties
            const double cost = (double)((np + 255) / 256) * cmax + 1e-3 * work;
            if (best_cost < 0.0 || cost < best_cost) {
                best_cost = cost;
                best[0] = s0;
                best[1] = s1;
            }
        }
    int mask = 0;
    for (int d = 0; d < 2; ++d) {
        int4 a = make_int4(0, 0, 0, 0), b = make_int4(0, 0, 0, 0);
        if (best[d]) {
            strip_desc(v[d][0], v[d][1], J, N, H, best[d], &a, &b);
            mask |= 1 << d;
        }
        scan[4 * i + 2 * d] = a;
        scan[4 * i + 2 * d + 1] = b;
    }
    e.w = mask;
    pairs[i] = e;
}

// 2 c_e per pair rounded to FP32, the weight the FP32 evaluators apply.
__global__ void k_pair_c2f(int n_pairs, const double* __restrict__ pair_c, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pairs) out[i] = (float)(2.0 * pair_c[i]);
}

// Size of e^perp ∩ [-Nt, Nt]^d \ {0} per line (one block per line).
__global__ void k_plane_count(int d, int n_lines, const int4* lines, int Nt, int* counts) {
    const int4 e = lines[blockIdx.x];
    const int w = 2 * Nt + 1, total = d == 3 ? w * w * w : w * w;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int v[3];
        cand_vec(i, d, Nt, v);
        bool nz = v[0] | v[1] | v[2];
        local += (nz && v[0] * e.x + v[1] * e.y + v[2] * e.z == 0) ? 1 : 0;
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = cnt;
}

// The plane list of each line in lexicographic order of l (one block per line).
__global__ void k_plane_emit(int d, int n_lines, const int4* lines, int Nt, const int* start, char4* plane) {
    const int4 e = lines[blockIdx.x];
    const int w = 2 * Nt + 1, total = d == 3 ? w * w * w : w * w;
    int base = start[blockIdx.x];
    for (int c0 = 0; c0 < total; c0 += blockDim.x) {
        int i = c0 + threadIdx.x;
        int v[3] = {0, 0, 0};
        bool ok = false;
        if (i < total) {
            cand_vec(i, d, Nt, v);
            bool nz = v[0] | v[1] | v[2];
            ok = nz && (v[0] * e.x + v[1] * e.y + v[2] * e.z == 0);
        }
        int tot;
        int r = block_exclusive_scan(ok ? 1 : 0, &tot);
        if (ok) plane[base + r] = make_char4((signed char)v[0], (signed char)v[1], (signed char)v[2], 0);
        base += tot;
    }
}

// K(m) = sum over lines e, 0<|j|<=J_e, l in the plane list of e, of c_e
// [j e + l = m mod N] (2D), one thread per m, lines in order: the loss
// sum_e c_e V_e(i) is the correlation sum_m K(m) f(i + m).
__global__ void k_loss_kernel2d(int n_lines, const int4* lines, const double* c, const int* plane_start,
                                const char4* plane, int N, double* K) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N * N) return;
    const int m0 = m / N, m1 = m - (m / N) * N;
    double acc = 0.0;
    for (int li = 0; li < n_lines; ++li) {
        const int4 e = lines[li];
        int hits = 0;
        for (int t = plane_start[li]; t < plane_start[li + 1]; ++t) {
            const char4 l = plane[t];
            for (int j = -e.w; j <= e.w; ++j) {
                if (j == 0) continue;
                int a0 = (j * e.x + l.x) % N, a1 = (j * e.y + l.y) % N;
                a0 += a0 < 0 ? N : 0;
                a1 += a1 < 0 ? N : 0;
                hits += (a0 == m0 && a1 == m1) ? 1 : 0;
            }
        }
        acc += c[li] * (double)hits;
    }
    K[m] = acc;
}

// Ktilde(xi) = sum_m K(m) cos(2 pi (m.xi mod N) / N) / N^2 (exact integer
// phases), in FP64 and rounded to FP32.
__global__ void k_khat2d(int N, const double* K, double* kh, float* khf) {
    const int xi = blockIdx.x * blockDim.x + threadIdx.x;
    if (xi >= N * N) return;
    const int x0 = xi / N, x1 = xi - (xi / N) * N;
    double acc = 0.0;
    for (int m = 0; m < N * N; ++m) {
        const double k = K[m];
        if (k == 0.0) continue;
        const int t = ((m / N) * x0 + (m - (m / N) * N) * x1) % N;
        acc += k * cospi(2.0 * t / N);
    }
    acc /= (double)N * (double)N;
    kh[xi] = acc;
    khf[xi] = (float)acc;
}

__global__ void k_twiddles(int N, double2* tw, float2* twf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double s, c;
    sincospi(2.0 * t / N, &s, &c);
    tw[t] = make_double2(c, -s);
    twf[t] = make_float2((float)c, (float)-s);
}

// The axis window's transform D(t) = 2 sum_{j=1..J} cos(2 pi j t / N) / N^2,
// t < N, phases reduced exactly modulo N, times s = the power of two nearest
// Ktilde(0) / D(0) (the two parts of one inverse transform then have one
// size); entry N holds 1 / s.  One thread per t.
__global__ void k_dwin(int N, int J, const double* kh, double* dw, float* dwf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > N) return;
    const double d0 = 2.0 * J / ((double)N * (double)N);
    const int es = kh[0] > 0.0 ? (int)lround(log2(kh[0] / d0)) : 0;
    double v;
    if (t == N) {
        v = ldexp(1.0, -es);
    } else {
        double acc = 0.0;
        for (int j = 1; j <= J; ++j) acc += 2.0 * cospi(2.0 * ((j * t) % N) / N);
        v = ldexp(acc / ((double)N * (double)N), es);
    }
    dw[t] = v;
    dwf[t] = (float)v;
}

// Transforms of the line windows for the FFT window engine of the 2D
// evaluator: dj[J N + t] = sum_{0<|j|<=J} cos(2 pi j t / N) / N^2 for
// J = 0..H, t < N (row 0 zero), phases reduced exactly modulo N.  With
// m = e.xi mod N, fhat(xi) dj[J N + m] is the transform of W_e (the window
// of half-length J along e) including the inverse transform's 1 / N^2.
// One thread per (J, t).
__global__ void k_djtab(int N, int H, double* dj, float* djf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (H + 1) * N) return;
    const int J = i / N, t = i - J * N;
    double acc = 0.0;
    for (int j = 1; j <= J; ++j) acc += 2.0 * cospi(2.0 * ((j * t) % N) / N);
    const double v = acc / ((double)N * (double)N);
    dj[i] = v;
    djf[i] = (float)v;
}

// Ktilde(xi) = sum_e c_e D_e(xi) Lambda_e(xi) / N^d with
// D_e = 2 sum_{j=1..J_e} cos(2 pi j (e.xi) / N) (the line factor) and
// Lambda_e = sum_{l in plane list} cos(2 pi (l.xi) / N) (the e^perp factor):
// the transform of the loss kernel K factorises line by line (the kernel
// modes of eq. (decDVM) on the diagonal K = L).  Fixed summation order,
// phases reduced exactly modulo N.  One thread per xi.
__global__ void k_khat_factored(int d, int N, int n_lines, const int4* lines, const double* c,
                                const int* plane_start, const char4* plane, double* kh, float* khf) {
    __shared__ double ct[64];
    for (int t = threadIdx.x; t < N; t += blockDim.x) ct[t] = cospi(2.0 * t / N);
    __syncthreads();
    int total = N * N;
    if (d == 3) total *= N;
    const int xi = blockIdx.x * blockDim.x + threadIdx.x;
    if (xi >= total) return;
    int x[3] = {0, 0, 0};
    int r = xi;
    for (int a = d - 1; a >= 0; --a) {
        x[a] = r % N;
        r /= N;
    }
    double acc = 0.0;
    for (int li = 0; li < n_lines; ++li) {
        const int4 e = lines[li];
        int ed = (e.x * x[0] + e.y * x[1] + e.z * x[2]) % N;
        ed += ed < 0 ? N : 0;
        double D = 0.0;
        for (int j = 1; j <= e.w; ++j) D += ct[(j * ed) % N];
        double lam = 0.0;
        for (int t = plane_start[li]; t < plane_start[li + 1]; ++t) {
            const char4 l = plane[t];
            int ph = (l.x * x[0] + l.y * x[1] + l.z * x[2]) % N;
            ph += ph < 0 ? N : 0;
            lam += ct[ph];
        }
        acc += c[li] * 2.0 * D * lam;
    }
    acc /= (double)total;
    kh[xi] = acc;
    khf[xi] = (float)acc;
}

// ------------------------------------------------------------ plan lifecycle

static void plan_free(qdvm_plan_s* p) {
    if (!p) return;
    cudaFree(p->d_lines);
    cudaFree(p->d_c);
    cudaFree(p->d_pairs);
    cudaFree(p->d_pair_c);
    cudaFree(p->d_pair_scan);
    cudaFree(p->d_pair_c2f);
    cudaFree(p->d_plane_start);
    cudaFree(p->d_plane);
    cudaFree(p->d_khat);
    cudaFree(p->d_khat_f);
    cudaFree(p->d_tw);
    cudaFree(p->d_tw_f);
    cudaFree(p->d_dwin);
    cudaFree(p->d_dwin_f);
    cudaFree(p->d_dj);
    cudaFree(p->d_dj_f);
    cudaFree(p->d_rclass);
    cudaFree(p->d_rline);
    cudaFree(p->d_rc);
    cudaFree(p->d_rc_f);
    cudaFree(p->d_rrow_start);
    cudaFree(p->d_rrow);
    p->magic = 0;
    delete p;
}

int qdvm_default_ntilde(int N) { return (int)floor((double)N / (3.0 + sqrt(2.0))); }

static qdvm_status build_tables(qdvm_plan_s* p) {
    const int d = p->d, m = p->m;
    int* d_counts = nullptr;
    int* d_offsets = nullptr;
    int* d_tmp = nullptr;
    qdvm_status st = QDVM_OK;
    std::vector<int> counts(m), offsets(m);
    auto fail = [&](qdvm_status s) {
        cudaFree(d_counts);
        cudaFree(d_offsets);
        cudaFree(d_tmp);
        return s;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&d_counts, m * sizeof(int))) != cudaSuccess) return fail(qdvm_cuda_status(e, "plan counts"));
    if ((e = cudaMalloc(&d_offsets, m * sizeof(int))) != cudaSuccess) return fail(qdvm_cuda_status(e, "plan offsets"));
    k_shell_count<<<m, 256>>>(d, d_counts);
    if ((e = cudaMemcpy(counts.data(), d_counts, m * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "k_shell_count"));
    int total = 0;
    for (int i = 0; i < m; ++i) {
        offsets[i] = total;
        total += counts[i];
    }
    p->n_lines = total;
    if ((e = cudaMemcpy(d_offsets, offsets.data(), m * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "plan offsets upload"));
    if ((e = cudaMalloc(&p->d_lines, total * sizeof(int4))) != cudaSuccess) return fail(qdvm_cuda_status(e, "lines"));
    if ((e = cudaMalloc(&p->d_c, total * sizeof(double))) != cudaSuccess) return fail(qdvm_cuda_status(e, "c"));
    k_shell_emit<<<m, 256>>>(d, d_offsets, p->d_lines);
    k_line_tables<<<(total + 255) / 256, 256>>>(d, total, p->Ntilde, p->kernel, p->h, p->d_lines, p->d_c);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(qdvm_cuda_status(e, "line tables"));

    p->h_lines.resize(total);
    p->h_c.resize(total);
    if ((e = cudaMemcpy(p->h_lines.data(), p->d_lines, total * sizeof(int4), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "lines readback"));
    if ((e = cudaMemcpy(p->h_c.data(), p->d_c, total * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "c readback"));

    if (d == 2) {
        int np = total / 2;
        if ((e = cudaMalloc(&p->d_pairs, np * sizeof(int4))) != cudaSuccess) return fail(qdvm_cuda_status(e, "pairs"));
        if ((e = cudaMalloc(&p->d_pair_c, np * sizeof(double))) != cudaSuccess)
            return fail(qdvm_cuda_status(e, "pair c"));
        if ((e = cudaMalloc(&d_tmp, sizeof(int))) != cudaSuccess) return fail(qdvm_cuda_status(e, "tmp"));
        k_pairs<<<1, 1024>>>(total, p->d_lines, p->d_c, p->d_pairs, p->d_pair_c, np, d_tmp);
        int got = -1;
        if ((e = cudaMemcpy(&got, d_tmp, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return fail(qdvm_cuda_status(e, "k_pairs"));
        if (got != np || 2 * np != total) return fail(qdvm_fail(QDVM_ERR_CUDA, "2D line pairing is inconsistent"));
        p->n_pairs = np;
        cudaFree(d_tmp);
        d_tmp = nullptr;
        if ((e = cudaMalloc(&p->d_pair_scan, 4 * np * sizeof(int4))) != cudaSuccess)
            return fail(qdvm_cuda_status(e, "pair scan table"));
        k_pair_scan<<<(np + 127) / 128, 128>>>(np, p->N, p->Ntilde, p->d_pairs, p->d_pair_scan);
        if ((e = cudaMalloc(&p->d_pair_c2f, np * sizeof(float))) != cudaSuccess)
            return fail(qdvm_cuda_status(e, "pair weights"));
        k_pair_c2f<<<(np + 127) / 128, 128>>>(np, p->d_pair_c, p->d_pair_c2f);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(qdvm_cuda_status(e, "k_pair_scan"));
    }
    // plane lists e^perp ∩ [-Ntilde, Ntilde]^d \ {0} (in 2D: the segment along e^perp)
    if ((e = cudaMalloc(&d_tmp, total * sizeof(int))) != cudaSuccess) return fail(qdvm_cuda_status(e, "plane counts"));
    k_plane_count<<<total, 256>>>(d, total, p->d_lines, p->Ntilde, d_tmp);
    std::vector<int> pc(total);
    if ((e = cudaMemcpy(pc.data(), d_tmp, total * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "k_plane_count"));
    p->h_plane_start.assign(total + 1, 0);
    int64_t terms = 0;
    int mx = 0;
    for (int i = 0; i < total; ++i) {
        p->h_plane_start[i + 1] = p->h_plane_start[i] + pc[i];
        terms += (int64_t)(2 * p->h_lines[i].w) * pc[i];
        mx = pc[i] > mx ? pc[i] : mx;
    }
    p->n_plane = p->h_plane_start[total];
    p->max_plane = mx;
    p->n_terms = terms;
    if ((e = cudaMalloc(&p->d_plane_start, (total + 1) * sizeof(int))) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "plane start"));
    if ((e = cudaMalloc(&p->d_plane, (size_t)std::max(p->n_plane, 1) * sizeof(char4))) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "plane"));
    if ((e = cudaMemcpy(p->d_plane_start, p->h_plane_start.data(), (total + 1) * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(qdvm_cuda_status(e, "plane start upload"));
    k_plane_emit<<<total, 256>>>(d, total, p->d_lines, p->Ntilde, p->d_plane_start, p->d_plane);
    if (d == 3 && p->N <= 32) {
        const int N = p->N, n3 = N * N * N;
        if ((e = cudaMalloc(&p->d_khat, n3 * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_khat_f, n3 * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_tw, N * sizeof(double2))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_tw_f, N * sizeof(float2))) != cudaSuccess)
            return fail(qdvm_cuda_status(e, "3D loss kernel tables"));
        k_khat_factored<<<(n3 + 127) / 128, 128>>>(3, N, total, p->d_lines, p->d_c, p->d_plane_start, p->d_plane,
                                                   p->d_khat, p->d_khat_f);
        k_twiddles<<<(N + 63) / 64, 64>>>(N, p->d_tw, p->d_tw_f);
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(qdvm_cuda_status(e, "3D loss kernel tables"));
        const qdvm_status rs = build_row_tables(p);
        if (rs != QDVM_OK) return fail(rs);
    }
    if (d == 2 && p->N <= 64) {
        const int N = p->N, n2 = N * N;
        double* dK = nullptr;
        if ((e = cudaMalloc(&dK, n2 * sizeof(double))) != cudaSuccess) return fail(qdvm_cuda_status(e, "K"));
        if ((e = cudaMalloc(&p->d_khat, n2 * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_khat_f, n2 * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_tw, N * sizeof(double2))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_tw_f, N * sizeof(float2))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_dwin, (N + 1) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_dwin_f, (N + 1) * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_dj, (p->Ntilde + 1) * N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&p->d_dj_f, (p->Ntilde + 1) * N * sizeof(float))) != cudaSuccess) {
            cudaFree(dK);
            return fail(qdvm_cuda_status(e, "loss kernel tables"));
        }
        k_loss_kernel2d<<<(n2 + 127) / 128, 128>>>(total, p->d_lines, p->d_c, p->d_plane_start, p->d_plane, N, dK);
        k_khat2d<<<(n2 + 127) / 128, 128>>>(N, dK, p->d_khat, p->d_khat_f);
        k_twiddles<<<(N + 63) / 64, 64>>>(N, p->d_tw, p->d_tw_f);
        k_dwin<<<(N + 64) / 64, 64>>>(N, p->Ntilde, p->d_khat, p->d_dwin, p->d_dwin_f);
        k_djtab<<<((p->Ntilde + 1) * N + 127) / 128, 128>>>(N, p->Ntilde, p->d_dj, p->d_dj_f);
        e = cudaDeviceSynchronize();
        cudaFree(dK);
        if (e != cudaSuccess) return fail(qdvm_cuda_status(e, "loss kernel tables"));
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(qdvm_cuda_status(e, "plan build"));
    return fail(st);
}

extern "C" qdvm_status qdvm_plan_create_ex(qdvm_plan_t* out, int d, int N, int Nbar, int Ntilde, double L,
                                           int kernel, int engine) {
    if (!out) return qdvm_fail(QDVM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (d != 2 && d != 3) return qdvm_fail(QDVM_ERR_INVALID_ARG, "d must be 2 or 3");
    if (N < 4 || (d == 2 && N > 256) || (d == 3 && N > 64))
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "N out of range (2D: 4..256, 3D: 4..64)");
    if (Nbar < 1) return qdvm_fail(QDVM_ERR_INVALID_ARG, "Nbar must be >= 1");
    if (!(L > 0.0) || !isfinite(L)) return qdvm_fail(QDVM_ERR_INVALID_ARG, "L must be positive and finite");
    if (kernel != QDVM_KERNEL_UNIT && kernel != QDVM_KERNEL_HP)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "unknown kernel");
    if (engine < QDVM_ENGINE_AUTO || engine > QDVM_ENGINE_SCAN)
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "unknown engine");
    int Nt = Ntilde < 0 ? qdvm_default_ntilde(N) : Ntilde;
    if (Nt < 1 || 2 * Nt >= N) return qdvm_fail(QDVM_ERR_INVALID_ARG, "Ntilde must satisfy 1 <= Ntilde, 2 Ntilde < N");

    qdvm_plan_s* p = new (std::nothrow) qdvm_plan_s();
    if (!p) return qdvm_fail(QDVM_ERR_OOM, "host allocation");
    p->magic = QDVM_PLAN_MAGIC;
    p->d = d;
    p->N = N;
    p->Nbar = Nbar;
    p->Ntilde = Nt;
    p->m = Nbar < Nt ? Nbar : Nt;
    p->kernel = kernel;
    p->engine = engine;
    p->L = L;
    p->h = 2.0 * L / N;
    p->tune.threads = 256;
    p->tune.direct_j = 2;
    p->tune.line_chunks = 0;
    p->tune.loss_fft = 0;
    // the engine only sets the initial choice; qdvm_tune_batched may change it
    p->tune.scan_j = engine == QDVM_ENGINE_SCAN ? 1 : engine == QDVM_ENGINE_DIRECT ? 0 : QDVM_SCAN_J_DEFAULT;
    cudaGetDevice(&p->device);
    qdvm_status s = build_tables(p);
    if (s != QDVM_OK) {
        plan_free(p);
        return s;
    }
    *out = p;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_create(qdvm_plan_t* out, int d, int N, int Nbar, double L, int kernel) {
    return qdvm_plan_create_ex(out, d, N, Nbar, -1, L, kernel, QDVM_ENGINE_AUTO);
}

extern "C" qdvm_status qdvm_plan_destroy(qdvm_plan_t plan) {
    if (!plan) return QDVM_OK;
    if (!qdvm_plan_ok(plan)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    plan_free(plan);
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_info(qdvm_plan_t p, int* d, int* N, int* Ntilde, int* m, int* n_lines,
                                      int64_t* n_terms) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (d) *d = p->d;
    if (N) *N = p->N;
    if (Ntilde) *Ntilde = p->Ntilde;
    if (m) *m = p->m;
    if (n_lines) *n_lines = p->n_lines;
    if (n_terms) *n_terms = p->n_terms;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_row_info(qdvm_plan_t p, int* n_classes, int* n_rows) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (n_classes) *n_classes = p->n_rclass;
    if (n_rows) *n_rows = p->n_rclass ? p->n_rrow : 0;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_lines(qdvm_plan_t p, int* dirs, int* J, double* c) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    for (int i = 0; i < p->n_lines; ++i) {
        const int4 e = p->h_lines[i];
        if (dirs) {
            dirs[3 * i + 0] = e.x;
            dirs[3 * i + 1] = e.y;
            dirs[3 * i + 2] = e.z;
        }
        if (J) J[i] = e.w;
        if (c) c[i] = p->h_c[i];
    }
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_get_tuning(qdvm_plan_t p, qdvm_tuning* t) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!t) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL tuning");
    *t = p->tune;
    return QDVM_OK;
}

extern "C" qdvm_status qdvm_plan_set_tuning(qdvm_plan_t p, const qdvm_tuning* t) {
    if (!qdvm_plan_ok(p)) return qdvm_fail(QDVM_ERR_BAD_PLAN, "bad plan handle");
    if (!t) return qdvm_fail(QDVM_ERR_INVALID_ARG, "NULL tuning");
    if (t->threads != 256 && t->threads != 512) return qdvm_fail(QDVM_ERR_INVALID_ARG, "threads must be 256 or 512");
    if (t->direct_j < 0 || t->direct_j > 2) return qdvm_fail(QDVM_ERR_INVALID_ARG, "direct_j must be 0, 1 or 2");
    if (t->line_chunks < 0) return qdvm_fail(QDVM_ERR_INVALID_ARG, "line_chunks must be >= 0");
    if (t->loss_fft < 0 || t->loss_fft > 3) return qdvm_fail(QDVM_ERR_INVALID_ARG, "loss_fft must be 0, 1, 2 or 3");
    if (t->scan_j < 0 || t->scan_j > 64) return qdvm_fail(QDVM_ERR_INVALID_ARG, "scan_j must be in [0, 64]");
    p->tune = *t;
    return QDVM_OK;
}
