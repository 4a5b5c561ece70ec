// Internal definitions shared by the qdvm CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qdvm.h"

#define QDVM_PLAN_MAGIC 0x51445650u  // "QDVP"
#define QDVM_RCLASS_INTS 20           // ints per row class: M, M^-1, first line, end line
#define QDVM_ROW_MAX 15               // longest polygon row (2 Ntilde + 1 with Ntilde <= 7)

// Plan object behind the opaque qdvm_plan_t.
struct qdvm_plan_s {
    uint32_t magic;
    int d, N, Nbar, Ntilde, m, kernel, engine;
    double L, h;
    int n_lines;     // lines of A_m
    int n_pairs;     // 2D: pairs {e, e^perp}
    int n_plane;     // 3D: total entries of the plane offset lists
    int max_plane;   // 3D: largest plane list
    int64_t n_terms; // (k, l) terms per output point
    int device;
    qdvm_tuning tune;  // launch parameters (set by qdvm_plan_set_tuning / qdvm_tune_batched)
    // device tables (owned)
    int4* d_lines;        // (e0, e1, e2, J)
    double* d_c;          // c_e
    int4* d_pairs;        // 2D: (e0, e1, J, S), one per pair
    double* d_pair_c;     // 2D: c_e (= c_{e^perp})
    float* d_pair_c2f;    // 2D: 2 c_e rounded to FP32 (the FP32 kernels' pair weight)
    int4* d_pair_scan;    // 2D: strip descriptors of e and e^perp, 4 per pair (scan engine; walked directions in d_pairs[].w)
    int* d_plane_start;   // 3D: n_lines + 1 offsets into d_plane
    char4* d_plane;       // (l0, l1, l2, 0), l in e^perp, 0 < |l|_inf <= Ntilde
    // 2D with N <= 64 and 3D with N <= 32: the loss as one convolution,
    // loss_i = f_i (K * f)_i with K(m) = sum_e c_e #{(j, l): j e + l = m};
    // Ktilde(xi) = sum_m K(m) cos(2 pi m.xi / N) / N^d (real: K is
    // symmetric), and the N-th roots of unity exp(-2 pi i t / N) for the FFTs.
    double* d_khat;
    float* d_khat_f;
    double2* d_tw;
    float2* d_tw_f;
    // 2D with N <= 64: the transform of the axis window (j e, 0 < |j| <= J,
    // e = (1, 0), J = Ntilde) at row frequency t < N,
    // s D(t) = s sum_{0<|j|<=J} cos(2 pi j t / N) / N^2, so that one inverse
    // FFT of fhat (Ktilde + i s D) returns the loss convolution and s W_(1,0);
    // s is a power of two of the size of Ktilde(0) / D(0), entry N is 1 / s
    double* d_dwin;
    float* d_dwin_f;
    // 2D with N <= 64: the window transforms of every half-length J <= Ntilde,
    // dj[J N + t] = sum_{0<|j|<=J} cos(2 pi j t / N) / N^2 (the FFT window
    // engine multiplies fhat by dj[J N + (e.xi mod N)] + i dj[J N + (e^perp.xi mod N)])
    double* d_dj;
    float* d_dj_f;
    // 3D, N in {16, 32}, Ntilde <= 7: the plane polygons as rows along an
    // in-plane lattice vector u, lines grouped into classes of a common u
    // (plan_rows.cu).  Lines are listed class by class.
    int n_rclass;          // 0: no row tables
    int n_rrow;
    int* d_rclass;         // per class: M (3x3, columns u, w2, w3), M^-1, first and end line
    int4* d_rline;         // per line: e in class coordinates (mod N), J
    double* d_rc;          // c_e
    float* d_rc_f;         // c_e rounded to FP32 (the FP32 kernels' line weight)
    int* d_rrow_start;     // n_lines + 1 offsets into d_rrow
    uchar4* d_rrow;        // per row: start (alpha, beta, gamma) mod N, length
    // host copies
    std::vector<int4> h_lines;
    std::vector<double> h_c;
    std::vector<int> h_plane_start;
};

// Plain-data view of a plan for kernels (passed by value).
struct PlanDev {
    int d, N, Ntilde, n_lines, n_pairs;
    double h, L;
    const int4* lines;
    const double* c;
    const int4* pairs;
    const double* pair_c;
    const float* pair_c2f;
    const int4* pair_scan;
    const int* plane_start;
    const char4* plane;
    const double* khat;
    const float* khat_f;
    const double2* tw;
    const float2* tw_f;
    const double* dwin;
    const float* dwin_f;
    const double* dj;
    const float* dj_f;
    int n_rclass;
    const int* rclass;
    const int4* rline;
    const double* rc;
    const float* rc_f;
    const int* rrow_start;
    const uchar4* rrow;
    // the plan's own launch parameters (direct_j, loss_fft, scan_j): a
    // batched 2D launch takes them per cell from the cell's plan
    int tjd, tfft, tsj;
};

struct BatchDev {
    int n_plans;
    PlanDev p[QDVM_MAX_BATCH_PLANS];
};

inline PlanDev plan_dev(const qdvm_plan_s* p) {
    PlanDev v;
    v.d = p->d;
    v.N = p->N;
    v.Ntilde = p->Ntilde;
    v.n_lines = p->n_lines;
    v.n_pairs = p->n_pairs;
    v.h = p->h;
    v.L = p->L;
    v.lines = p->d_lines;
    v.c = p->d_c;
    v.pairs = p->d_pairs;
    v.pair_c = p->d_pair_c;
    v.pair_c2f = p->d_pair_c2f;
    v.pair_scan = p->d_pair_scan;
    v.plane_start = p->d_plane_start;
    v.plane = p->d_plane;
    v.khat = p->d_khat;
    v.khat_f = p->d_khat_f;
    v.tw = p->d_tw;
    v.tw_f = p->d_tw_f;
    v.dwin = p->d_dwin;
    v.dwin_f = p->d_dwin_f;
    v.dj = p->d_dj;
    v.dj_f = p->d_dj_f;
    v.n_rclass = p->n_rclass;
    v.rclass = p->d_rclass;
    v.rline = p->d_rline;
    v.rc = p->d_rc;
    v.rc_f = p->d_rc_f;
    v.rrow_start = p->d_rrow_start;
    v.rrow = p->d_rrow;
    v.tjd = p->tune.direct_j;
    v.tfft = p->tune.loss_fft;
    v.tsj = p->tune.scan_j;
    return v;
}

// ------------------------------------------------------------ error state
void qdvm_set_error(const std::string& msg);
qdvm_status qdvm_fail(qdvm_status s, const std::string& msg);
qdvm_status qdvm_cuda_status(cudaError_t e, const char* where);
bool qdvm_plan_ok(const qdvm_plan_s* p);

#define QDVM_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) return qdvm_cuda_status(_e, #expr);                 \
    } while (0)

#define QDVM_LAUNCH_CHECK(where)                                                   \
    do {                                                                           \
        cudaError_t _e = cudaGetLastError();                                       \
        if (_e != cudaSuccess) return qdvm_cuda_status(_e, where);                 \
    } while (0)

// Compensated accumulation s + c += x (Neumaier's TwoSum form of Kahan
// summation) when KAHAN, plain s += x otherwise.
template <typename T, bool KAHAN>
__device__ __forceinline__ void comp_add(T& s, T& c, T x) {
    if (KAHAN) {
        T t = s + x;
        T bp = t - s;
        T err = (s - (t - bp)) + (x - bp);
        c += err;
        s = t;
    } else {
        s += x;
    }
}

// ------------------------------------------------------------ 2D fused engine
// Padded on-chip layout of a 2D cell.  The f buffer holds rows/cols
// [-2H, N+2H) with the periodic halo replicated (H = Ntilde): a pair with
// J = 1 reads f at i +- e +- e^perp, up to 2H away.  The P buffer holds rows
// [-H, N+H) on the same row stride, so a point's P address is its f address
// minus H*(stride+1).  The stride is congruent to N modulo 32 so that a warp
// of 32 consecutive points never hits the same bank twice, even when it
// straddles two rows (N = 16, 48).
__host__ __device__ constexpr int pad2d_stride(int N, int H) {
    return N + 4 * H + (((N % 32) - ((N + 4 * H) % 32) + 32) % 32);
}
__host__ __device__ constexpr int pad2d_rows_f(int N, int H) { return N + 4 * H; }
__host__ __device__ constexpr int pad2d_rows_p(int N, int H) { return N + 2 * H; }

size_t fused2d_smem_bytes(int N, int H, int prec, int fft);
int fused2d_supported(int N, int H, int prec);

qdvm_status fused2d_eval_single(const qdvm_plan_s* p, const void* f, void* Q, int prec, void* ws,
                                size_t ws_bytes, cudaStream_t st);
size_t fused2d_single_workspace(const qdvm_plan_s* p, int prec);
qdvm_status fused2d_eval_batched(const BatchDev& b, const qdvm_tuning& tu, int n_cells, const int* cell_plan,
                                 const int64_t* cell_offset, const void* f, void* Q, double* moments, int prec,
                                 void* ws, cudaStream_t st);

qdvm_status moments_launch(int d, int N, double L, const void* Q, int prec, double* m, cudaStream_t st);
qdvm_status schedule_launch(const BatchDev& b, int n_cells, const int* cell_plan, int* order, int* counter,
                            cudaStream_t st);

int qdvm_num_sms();

// ------------------------------------------------------------ generic engine
// mode: 0 forward, 1 JVP (aux = tangent), 2 VJP (aux = cotangent)
enum { QDVM_MODE_FWD = 0, QDVM_MODE_JVP = 1, QDVM_MODE_VJP = 2 };
// chunks: lines-per-cell split (0 = automatic)
size_t engine_workspace(int mode, const BatchDev& b, int n_cells, int prec, bool single, int chunks);
qdvm_status engine_run(int mode, const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                       const void* f, const void* aux, void* out, double* moments, int prec, void* ws,
                       size_t ws_bytes, bool single, int chunks, cudaStream_t st);

// ------------------------------------------------------------ 3D FFT-loss evaluator
// 3D batches whose plans share N in {16, 32}: the loss as one FFT
// convolution per cell, the gain per line with register accumulation (row
// form of the plane sums where the plans carry row tables).  mode: forward,
// JVP (aux = tangent) or VJP (aux = cotangent); the derivatives need the row
// form.
bool fast3d_supported(int mode, const BatchDev& b, int prec);
qdvm_status build_row_tables(qdvm_plan_s* p);
size_t fast3d_workspace(int mode, const BatchDev& b, int n_cells, int prec, bool single, int chunks);
qdvm_status fast3d_run(int mode, const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                       const void* f, const void* aux, void* out, double* moments, int prec, void* ws,
                       size_t ws_bytes, bool single, int chunks, cudaStream_t st);
