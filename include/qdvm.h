/*
 * qdvm.h -- C ABI of the GB300 (sm_103a) fast summation library for the
 * periodized, direction-restricted discrete-velocity Boltzmann operator.
 *
 * Operator (Mouhot, Pareschi, Rey, "Convolutive decomposition and fast
 * summation methods for discrete-velocity approximations of the Boltzmann
 * equation"):
 *
 *   Q_i = sum_{e in A_m} c_e [ W_e(i) P_e(i) - f_i V_e(i) ]           eq. (decD)
 *   W_e(i) = sum_{0<|j|<=J_e} f_{i+je}              (k in eZ: alpha_p)  eq. (decDVM)
 *   P_e(i) = sum_{l in e^perp, 0<|l|_inf<=Ntilde} f_{i+l}  (alpha'_p)   eq. (decDVM)
 *   V_e(i) = sum_{0<|j|<=J_e} P_e(i+je)             (the beta(L,L) part) eq. (betaKL)
 *
 * which equals, term by term, eq. (DR) of Section 2.3 restricted to the
 * pairs (k, l), k.l = 0, whose k lies on a line e with |e|_inf <= m:
 *   Q_i = sum Gamma_{k,l} [f_{i+k} f_{i+l} - f_i f_{i+k+l}],
 *   Gamma_{k,l} = a(k) = c_e (decoupled kernel of eq. (decoup), b = 1).
 * Here m = min(Nbar, Ntilde), J_e = floor(Ntilde / |e|_inf), A_m is the set
 * of lines through 0 with a primitive direction in [-m, m]^d (the Farey-type
 * sets A^1, A^2 of Section 3.2), and
 *   c_e = 1                       (QDVM_KERNEL_UNIT, constant kernel),
 *   c_e = h^(2d-1) |e|_2          (QDVM_KERNEL_HP: a(k) = h^(2d-1)|k|/gcd(k),
 *                                  2D Maxwell molecules / 3D hard spheres).
 *
 * Grid: N points per axis on the periodic box [-L, L)^d, h = 2L/N, node j at
 * v_j = -L + j h; indices are taken modulo N.  Arrays are row-major N^d with
 * the last axis fastest.  Default Ntilde = floor(N / (3 + sqrt 2)) (Section 4).
 *
 * Conventions for every entry point:
 *   - Array pointers are DEVICE pointers owned by the caller unless a
 *     parameter says "host".  f is read only and must not alias any output.
 *   - prec selects the arithmetic: QDVM_F64 (f, Q are double), QDVM_F32 or
 *     QDVM_F32_KAHAN (f, Q are float; KAHAN compensates the sum over
 *     directions).  Moments are always double.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Evaluation entry points enqueue kernels only: they allocate nothing,
 *     never synchronise the host and may be captured in a CUDA graph.
 *   - workspace is caller-owned device memory of at least the size that the
 *     matching *_workspace query returns (may be NULL when that size is 0).
 *   - Errors are returned as qdvm_status, never by aborting.  A launch error
 *     is reported as QDVM_ERR_CUDA; qdvm_last_error() gives details for the
 *     calling host thread.
 */
#ifndef QDVM_H
#define QDVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qdvm_plan_s* qdvm_plan_t;
typedef struct qdvm_graph_s* qdvm_graph_t;

typedef enum {
    QDVM_OK = 0,
    QDVM_ERR_INVALID_ARG = 1,
    QDVM_ERR_UNSUPPORTED = 2,
    QDVM_ERR_OOM = 3,
    QDVM_ERR_CUDA = 4,
    QDVM_ERR_TIMEOUT = 5,
    QDVM_ERR_BAD_PLAN = 6
} qdvm_status;

enum { QDVM_KERNEL_UNIT = 0, QDVM_KERNEL_HP = 1 };
enum { QDVM_F64 = 0, QDVM_F32 = 1, QDVM_F32_KAHAN = 2 };
/* Line-sum engines of the on-chip 2D evaluator (the windows W_e, the alpha_p
 * factors of eq. (decDVM)).  DIRECT: each window gathered term by term from
 * an on-chip copy of the cell (2J loads per point and line).  SCAN: segmented
 * running sums along the orbits of e on the torus (the lattice lines of
 * Section 3.2): a thread walks S consecutive points of a line, adding the
 * entering and subtracting the leaving value (2 loads per point and line
 * after the first window).  The engine given to qdvm_plan_create_ex sets
 * the initial qdvm_tuning.scan_j (DIRECT: 0, SCAN: 1, AUTO:
 * QDVM_SCAN_J_DEFAULT, i.e. DIRECT until qdvm_tune_batched measures
 * otherwise).  Measured on GB300: SCAN halves the shared-memory traffic of
 * a pair but adds integer work, so it pays for long windows (J >= 7) and in
 * the single-cell FP64 evaluation; batched FP32 evaluations with Nbar = 8 are
 * fastest with DIRECT.  A third engine serves one window: with
 * qdvm_tuning.loss_fft = 2 the axis window W_(1,0) is the convolution of f
 * with its window, taken from the same inverse FFT as the loss (see
 * qdvm_tuning). */
enum { QDVM_ENGINE_AUTO = 0, QDVM_ENGINE_DIRECT = 1, QDVM_ENGINE_SCAN = 2 };
#define QDVM_SCAN_J_DEFAULT 0

/* Maximum number of distinct plans in one batched call. */
#define QDVM_MAX_BATCH_PLANS 16

/* Launch parameters of the evaluators.  They change speed, never the set of
 * terms summed; results agree to rounding (and bit for bit on integer data).
 *   threads     CTA size of the on-chip 2D evaluator: 256 or 512.
 *   direct_j    2D pairs with window half-length J <= direct_j (0, 1 or 2)
 *               read V_e straight from the cell ((2J)^2 loads, no barrier);
 *               longer windows go through the on-chip P buffer.
 *   line_chunks generic (3D) engine: chunks of lines per cell, each a work
 *               item summed afterwards in a fixed order; 0 = automatic.
 *   loss_fft    1: the loss part sum_e c_e f V_e is evaluated as one
 *               convolution per cell, f (K * f) with K the weighted
 *               displacement histogram of the terms, by an on-chip 2D FFT
 *               (mixed radix 4/6/8; cells of 16, 32, 48 or 64 points per axis
 *               with the default truncation); the lines then only sum the
 *               gain.  Rounding differs from the direct sums (no longer
 *               bit-exact on integer data).  0: direct sums.
 *               2: as 1, and in the on-chip 2D evaluator the same inverse
 *               transform also returns one window sum of the axis pair
 *               {(1,0), (0,1)} (the spectrum is multiplied by Ktilde + i D
 *               with D the window's real transform): W_(1,0) with DIRECT
 *               gathers (scan_j = 0 or above the cell's Ntilde), so that
 *               pair gathers only along (0,1); W_(0,1) with the SCAN engine,
 *               which walks the other axis.
 *               3: as 1, and in the on-chip 2D evaluator the pairs with
 *               J >= scan_j take their windows from the FFT window engine:
 *               the cell's spectrum fhat stays on chip and each such pair
 *               takes one inverse transform of fhat (D_J(e.xi) +
 *               i D_J(e^perp.xi)), which returns W_e + i W_{e^perp}
 *               (Section 3.2, eq. (decDVM): each direction term as a
 *               convolution); the other pairs gather directly (scan_j = 0:
 *               DIRECT for every pair).  Elsewhere 2 and 3 act as 1.
 *   scan_j      with loss_fft >= 1 in the on-chip 2D evaluator (cells of 16,
 *               32, 48 or 64 points per axis with the default truncation):
 *               pairs {e, e^perp} with J >= scan_j compute their windows
 *               with the SCAN engine (running sums along strips of the
 *               lattice lines; the horizontal window (0,1) is gathered, or
 *               taken from the loss transform with loss_fft = 2), the others
 *               with DIRECT gathers; 0 = DIRECT for every pair.
 *               0 <= scan_j <= 64.  Ignored elsewhere. */
typedef struct {
    int threads;
    int direct_j;
    int line_chunks;
    int loss_fft;
    int scan_j;
} qdvm_tuning;

/* ------------------------------------------------------------------ plans */

/* Build a plan: enumerate the lines of A_m on the GPU (Section 3.2, sets A^1 /
 * A^2; Remark 3.4(1)), their window lengths J_e and weights c_e, the 2D
 * pairing e <-> e^perp (Remark 3.4(3)) and the 3D plane offset lists of
 * e^perp inside [-Ntilde, Ntilde]^3 (eq. (decDVM), alpha'_p).
 *   out     host pointer receiving the plan (owned by the caller, release
 *           with qdvm_plan_destroy).
 *   d       2 or 3.
 *   N       points per axis; 2D: 4 <= N <= 256, 3D: 4 <= N <= 64.
 *   Nbar    Farey order >= 1; values above Ntilde are clamped (m = Ntilde is
 *           the unrestricted operator, eq. (DR)).
 *   Ntilde  truncation (|k|_inf, |l|_inf <= Ntilde); -1 selects the default
 *           floor(N/(3+sqrt 2)); must satisfy 1 <= Ntilde and 2 Ntilde < N.
 *   L       half-width of the box, > 0 (h = 2L/N).
 *   kernel  QDVM_KERNEL_UNIT or QDVM_KERNEL_HP.
 *   engine  QDVM_ENGINE_*.
 * Synchronises the current device once (plan creation is not a hot path).
 * Errors: INVALID_ARG for out-of-range arguments, OOM, CUDA. */
qdvm_status qdvm_plan_create(qdvm_plan_t* out, int d, int N, int Nbar, double L, int kernel);
qdvm_status qdvm_plan_create_ex(qdvm_plan_t* out, int d, int N, int Nbar, int Ntilde, double L,
                                int kernel, int engine);

/* Release a plan and its device tables.  NULL is accepted. */
qdvm_status qdvm_plan_destroy(qdvm_plan_t plan);

/* Plan facts (any pointer may be NULL): dimension, N, Ntilde, m = min(Nbar,
 * Ntilde), number of lines in A_m, number of (k, l) terms per output point
 * (the direct-sum cost). */
qdvm_status qdvm_plan_info(qdvm_plan_t plan, int* d, int* N, int* Ntilde, int* m, int* n_lines,
                           int64_t* n_terms);

/* Row decomposition of the 3D plane polygons (3D plans with N = 16 or 32
 * and Ntilde <= 7; the offset sets {l in e^perp, 0 < |l|_inf <= Ntilde} of
 * eq. (decDVM), alpha'_p, written as rows along an in-plane lattice
 * vector): the number of line classes
 * sharing that vector and the total number of rows.  Both are 0 for other
 * plans, whose 3D evaluation sums the polygons point by point.  Any pointer
 * may be NULL. */
qdvm_status qdvm_plan_row_info(qdvm_plan_t plan, int* n_classes, int* n_rows);

/* Copy the line table to HOST arrays of n_lines entries: dirs (3 ints per
 * line, unused components 0, first non-zero component positive, ordered by
 * |e|_inf then lexicographically), J (window half-length), c (weight). */
qdvm_status qdvm_plan_lines(qdvm_plan_t plan, int* dirs, int* J, double* c);

/* Read / set a plan's launch parameters (defaults: 256, 2, 0, 0).  A batched
 * call uses the parameters of plans[0].  Errors: BAD_PLAN, INVALID_ARG. */
qdvm_status qdvm_plan_get_tuning(qdvm_plan_t plan, qdvm_tuning* t);
qdvm_status qdvm_plan_set_tuning(qdvm_plan_t plan, const qdvm_tuning* t);

/* Bytes of workspace that qdvm_eval, qdvm_jvp and qdvm_vjp need for this plan
 * and precision (0 is a valid answer).  Errors: BAD_PLAN, INVALID_ARG,
 * UNSUPPORTED (no engine for this plan and precision). */
qdvm_status qdvm_eval_workspace(qdvm_plan_t plan, int prec, size_t* bytes);

/* Bytes of workspace that the batched entry points (eval, jvp, vjp) need for
 * n_cells cells over these plans at this precision. */
qdvm_status qdvm_batched_workspace(const qdvm_plan_t* plans, int n_plans, int n_cells, int prec, size_t* bytes);

/* ------------------------------------------------------------- evaluation */

/* Q = Q(f) for one cell (eq. (decD); the path: W_e, P_e, V_e and the gain /
 * loss assembly of every line, fused on chip).  f and Q hold N^d elements of
 * the precision's type.  Deterministic: lines are summed in a fixed order. */
qdvm_status qdvm_eval(qdvm_plan_t plan, const void* f, void* Q, int prec, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Batched evaluation of many independent cells (space-inhomogeneous
 * setting; Section 3.3 notes the decomposition is fully parallel) in one
 * persistent launch.  All plans must have the same d.
 *   plans       HOST array of n_plans plans (n_plans <= QDVM_MAX_BATCH_PLANS).
 *   cell_plan   DEVICE int[n_cells]: plan index of each cell.
 *   cell_offset DEVICE int64[n_cells]: element offset of each cell in f / Q.
 *   f, Q        DEVICE arrays holding the cells back to back.
 *   moments     DEVICE double[n_cells * (d+2)] or NULL: per cell
 *               h^d sum_i Q_i phi(v_i), phi = 1, v_0..v_{d-1}, |v|^2
 *               (Section 2.1), reduced from the stored Q with FP64
 *               accuracy (on-chip 2D evaluator in FP32: per-thread partials
 *               in compensated FP32, exact products by fma, combined across
 *               each warp by TwoSum, then added across the warps in FP64).
 * Cells are scheduled largest first through an atomic work counter kept in
 * the workspace (size from qdvm_batched_workspace); results do not depend on
 * the schedule.  Cells whose plan index is out of range are skipped (their
 * outputs are left untouched).  Overlapping calls that share a workspace
 * race.  n_cells == 0 is a no-op.  Launch parameters: in the on-chip 2D
 * evaluator every cell runs with its own plan's direct_j, loss_fft and
 * scan_j, and the block size is plans[0]'s; elsewhere plans[0]'s tuning
 * applies to the whole batch. */
qdvm_status qdvm_eval_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                              const int64_t* cell_offset, const void* f, void* Q, double* moments,
                              int prec, void* workspace, size_t workspace_bytes, void* stream);

/* Autotuner: time every candidate launch configuration of
 * qdvm_eval_batched on this batch (CUDA events on `stream`, synchronises the
 * host; not for a hot path) and keep the fastest in every plan of the batch.
 * For the on-chip 2D evaluator with several plans, the block size chosen,
 * each plan in turn then tries the candidates with that block size while
 * the others keep their best so far, so plans may end with different
 * direct_j, loss_fft and scan_j.  *best (may be NULL) receives plans[0]'s
 * tuning.  Arguments as for qdvm_eval_batched; Q is overwritten.
 * Candidates that would need more workspace than given are skipped. */
qdvm_status qdvm_tune_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                              const int64_t* cell_offset, const void* f, void* Q, int prec, void* workspace,
                              size_t workspace_bytes, void* stream, qdvm_tuning* best);

/* Capture one qdvm_eval_batched call (same arguments, all pointers fixed)
 * into an executable CUDA graph; qdvm_graph_launch replays it on a stream
 * (one launch per step), qdvm_graph_destroy releases it.  Capture itself
 * launches nothing; the graph owns no device memory (the workspace stays the
 * caller's and must outlive the graph). */
qdvm_status qdvm_graph_capture_batched(qdvm_graph_t* out, const qdvm_plan_t* plans, int n_plans, int n_cells,
                                       const int* cell_plan, const int64_t* cell_offset, const void* f, void* Q,
                                       double* moments, int prec, void* workspace, size_t workspace_bytes);
qdvm_status qdvm_graph_launch(qdvm_graph_t graph, void* stream);
qdvm_status qdvm_graph_destroy(qdvm_graph_t graph);

/* Space-homogeneous time stepping df/dt = Q(f) of every cell of a batch by
 * the second-order total-variation-diminishing Runge-Kutta scheme of
 * Section 4, in the Shu-Osher form
 *   f1 = f + dt Q(f),   f <- (f + f1 + dt Q(f1)) / 2,
 * repeated n_steps times, in place on f.  f: device, n_elems values of the
 * given precision, the cells laid out as for qdvm_eval_batched (n_elems =
 * total number of values).  Each Q evaluation is a qdvm_eval_batched call
 * with the plans' tuning.  moments: device, n_cells x (d + 2) doubles, or
 * NULL; receives the FP64 moments h^d sum f phi of the final f.  The
 * workspace (size from qdvm_rk2_workspace) holds the evaluator's workspace,
 * f1 and Q; it is the caller's.  Stream-ordered, no host synchronisation,
 * capturable (qdvm_graph_capture_rk2).  Errors: INVALID_ARG for negative
 * counts, a non-finite dt, NULL arrays or a small workspace; the
 * evaluator's errors otherwise. */
qdvm_status qdvm_rk2_workspace(const qdvm_plan_t* plans, int n_plans, int n_cells, int64_t n_elems, int prec,
                               size_t* bytes);
qdvm_status qdvm_rk2_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                             const int64_t* cell_offset, int64_t n_elems, void* f, double dt, int n_steps,
                             double* moments, int prec, void* workspace, size_t workspace_bytes, void* stream);

/* The same time stepping for one cell f (device, N^d values), with
 * qdvm_eval for each Q evaluation (a single cell's lines spread over the
 * whole GPU).  Workspace from qdvm_rk2_workspace_single.  Same errors. */
qdvm_status qdvm_rk2_workspace_single(qdvm_plan_t plan, int prec, size_t* bytes);
qdvm_status qdvm_rk2(qdvm_plan_t plan, void* f, double dt, int n_steps, int prec, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Space-dependent truncation (Section 3.3: Nbar may vary from cell to cell,
 * with fewer directions where the distribution is close to equilibrium).
 *
 * qdvm_equilibrium_distance: for every cell of a batch (layout as for
 * qdvm_eval_batched; each cell's plan gives N, d and L), the distance to
 * the Maxwellian with the cell's own discrete moments (per-point sums in
 * FP32 with compensation, reduced in FP64: accurate to about 1e-7):
 *   rho = h^d sum f, u = h^d sum f v / rho, T = (h^d sum f |v|^2 / rho - |u|^2) / d,
 *   M(v) = rho (2 pi T)^(-d/2) exp(-|v - u|^2 / (2 T)),
 *   eps = sum |f - M| / sum |f|     (v_j = -L + j h, h = 2L/N),
 * written to eps (device, n_cells doubles); +inf where rho <= 0, T <= 0 or
 * sum |f| = 0, and for cells whose plan index is out of range.
 *
 * qdvm_select_levels: cell_plan_out[c] = level_plan[cell_base[c] * n_levels
 * + level] with level = number of thresholds t_k (n_levels - 1 of them,
 * finite, strictly increasing, HOST array) such that eps[c] >= t_k (NaN
 * counts as beyond every threshold).  level_plan: HOST array of n_base x
 * n_levels plan indices (< QDVM_MAX_BATCH_PLANS) into the plans array the
 * caller then passes to qdvm_eval_batched with cell_plan_out.  Cells whose
 * base index is outside [0, n_base) get -1 (skipped by the evaluator).
 * eps, cell_base, cell_plan_out: device.  Both calls are stream-ordered and
 * capturable (the host tables are copied into the launch).  Errors:
 * INVALID_ARG for bad counts, tables or NULL arrays. */
#define QDVM_MAX_LEVELS 8
qdvm_status qdvm_equilibrium_distance(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                      const int64_t* cell_offset, const void* f, int prec, double* eps, void* stream);
qdvm_status qdvm_select_levels(int n_cells, const double* eps, const int* cell_base, int n_base, int n_levels,
                               const double* thresholds, const int* level_plan, int* cell_plan_out, void* stream);

/* Direct term-by-term evaluation, one thread per output point: every
 * (k, l) of the restricted operator (k = j e for e in A_m, 0 < |j| <= J_e;
 * l in the offset list of e, eq. (decDVM); weight c_e), with
 *   QDVM_BOUNDARY_PERIODIC: the periodised operator of eq. (DR) -- the Q of
 *     qdvm_eval computed without the line/plane decomposition;
 *   QDVM_BOUNDARY_BOX: the box-truncated operator D^tr of Section 2.3 -- a
 *     term counts only when i + k, i + l and i + k + l all lie in the grid.
 *     D^tr conserves mass, momentum and energy exactly for any f; the box
 *     couples k and l, so it has no fast (convolution) form.
 * Cost: one term per (point, k, l); use the fast paths for the periodised
 * operator.  Batched layout as for qdvm_eval_batched; moments (device,
 * n_cells x (d + 2), or NULL) receive the FP64 moments of the result.  The
 * single-cell call needs a 256-byte device workspace
 * (qdvm_eval_direct_workspace).  Errors: INVALID_ARG for a bad boundary,
 * precision, counts or NULL arrays. */
#define QDVM_BOUNDARY_PERIODIC 0
#define QDVM_BOUNDARY_BOX 1
qdvm_status qdvm_eval_direct_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                     const int64_t* cell_offset, const void* f, void* Q, double* moments, int prec,
                                     int boundary, void* stream);
qdvm_status qdvm_eval_direct_workspace(size_t* bytes);
qdvm_status qdvm_eval_direct(qdvm_plan_t plan, const void* f, void* Q, int prec, int boundary, void* workspace,
                             size_t workspace_bytes, void* stream);

/* Pseudo-spectral evaluation (Section 3.1): Q through its Fourier modes,
 *   Qhat_I = sum_{K + L = I} beta~(K, L) fhat_K fhat_L               (eq. (sysDiff))
 *   beta~(K, L) = beta(K, L) - beta(L, L),
 *   beta(K, L)  = sum_{(k, l)} Gamma(k) e_K(k) e_L(l)                 (eq. (betaKL))
 * with fhat_I = N^-d sum_i f_i e_{-I}(i), Q_i = sum_I Qhat_I e_I(i), e_K(k) =
 * exp(2 pi i K.k / N), over the (k, l) pairs of the plan (lines of A_m).
 * O(N^{2d}) work per cell and a dense N^d x N^d table: a second, Fourier-side
 * evaluation of the operator of qdvm_eval, independent of its line sums, for
 * checking, not for speed.  Supported plans: d = 2 with N <= 64, d = 3 with
 * N <= 16; others return QDVM_ERR_UNSUPPORTED.
 *
 * qdvm_spectral_table_entries: *n = N^{2d}, the entries of the table.
 * qdvm_spectral_table: fills table[K * N^d + L] = beta~(K, L) (modes K, L
 *   flat row-major in [0, N)^d).  beta is real (the pair set is symmetric in
 *   k and in l); it is formed in FP64 as sum_e D_e(K) P_e(L) over the lines e
 *   (D_e the weighted cosine sum of the window of e, P_e that of the offset
 *   list of e^perp) and stored as double (QDVM_F64) or float (QDVM_F32,
 *   QDVM_F32_KAHAN).  table: caller-owned DEVICE memory of
 *   qdvm_spectral_table_entries elements.  A set-up call: it allocates
 *   temporaries (2 x lines x N^d doubles) and synchronises the stream.
 * qdvm_spectral_workspace: bytes of workspace for n_cells cells (two complex
 *   spectra per cell).
 * qdvm_eval_spectral: Q of n_cells cells stored back to back (N^d elements
 *   each, row-major) from f, through two batched DFTs and the sum of eq.
 *   (sysDiff) (F32_KAHAN: compensated sums).  table from qdvm_spectral_table
 *   in the same precision; f, Q, workspace: DEVICE; f must not alias Q.
 *   Stream-ordered, allocates nothing.  Errors: BAD_PLAN, UNSUPPORTED,
 *   INVALID_ARG (precision, NULL arrays, workspace too small). */
qdvm_status qdvm_spectral_table_entries(qdvm_plan_t plan, size_t* n);
qdvm_status qdvm_spectral_table(qdvm_plan_t plan, void* table, int prec, void* stream);
qdvm_status qdvm_spectral_workspace(qdvm_plan_t plan, int n_cells, int prec, size_t* bytes);
qdvm_status qdvm_eval_spectral(qdvm_plan_t plan, const void* table, int n_cells, const void* f, void* Q, int prec,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Capture qdvm_rk2_batched (n_steps steps, all pointers fixed) into an
 * executable graph for qdvm_graph_launch: one launch runs the whole loop. */
qdvm_status qdvm_graph_capture_rk2(qdvm_graph_t* out, const qdvm_plan_t* plans, int n_plans, int n_cells,
                                   const int* cell_plan, const int64_t* cell_offset, int64_t n_elems, void* f,
                                   double dt, int n_steps, double* moments, int prec, void* workspace,
                                   size_t workspace_bytes);

/* Largest batch accepted by qdvm_eval_batched_noalloc. */
#define QDVM_NOALLOC_MAX_CELLS 65536

/* Allocation-free batched 2D evaluation.  The paper has no counterpart: this
 * is an interface for callers that cannot allocate device memory -- a solver
 * that owns a fixed device-memory budget and passes the library only its own
 * arrays, or a plug-in called inside another framework's time loop, where a
 * cudaMalloc would synchronise the device mid-step.  Same arguments and
 * results as qdvm_eval_batched, without the workspace: the work counter and
 * the cell schedule live in a 256 KB array inside the library that every GPU
 * loading the library keeps until the process exits.
 *   - Only the on-chip 2D evaluator (all plans d = 2, N <= 64) is covered;
 *     other plans return QDVM_ERR_UNSUPPORTED.
 *   - n_cells <= QDVM_NOALLOC_MAX_CELLS, else QDVM_ERR_INVALID_ARG (nothing
 *     is launched).
 *   - Allocates nothing (no cudaMalloc / cudaFree / allocating library call).
 *   - Every call made outside a stream capture looks up the array's device
 *     address (cudaGetSymbolAddress) for the current device, so a device
 *     reset between calls is harmless; a call made during a capture uses the
 *     address found by the last call outside one.  Make the first call on a
 *     device before any stream capture (else QDVM_ERR_INVALID_ARG).
 *   - All calls share the array (the counter is reset by every call), so
 *     calls that overlap on the GPU -- on different streams, or from
 *     different host threads -- race; serialise them. */
qdvm_status qdvm_eval_batched_noalloc(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                                      const int64_t* cell_offset, const void* f, void* Q, double* moments, int prec,
                                      void* stream);

/* Directional derivative dQ = Q'(f) df (Q is quadratic in f, eq. (DR)):
 *   dQ = sum_e c_e [ W_e[df] P_e[f] + W_e[f] P_e[df] - df V_e[f] - f V_e[df] ]. */
qdvm_status qdvm_jvp(qdvm_plan_t plan, const void* f, const void* df, void* dQ, int prec, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Vector-Jacobian product grad = Q'(f)^T g.  The window and plane operators
 * are symmetric on the torus, so
 *   grad = sum_e c_e [ W_e[g P_e] - g V_e + P_e[ g W_e - W_e[g f] ] ]
 * with W_e[x], P_e[x] the line window and plane sum of x. */
qdvm_status qdvm_vjp(qdvm_plan_t plan, const void* f, const void* g, void* grad, int prec, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Batched JVP / VJP with the same cell layout as qdvm_eval_batched. */
qdvm_status qdvm_jvp_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                             const int64_t* cell_offset, const void* f, const void* df, void* dQ, int prec,
                             void* workspace, size_t workspace_bytes, void* stream);
qdvm_status qdvm_vjp_batched(const qdvm_plan_t* plans, int n_plans, int n_cells, const int* cell_plan,
                             const int64_t* cell_offset, const void* f, const void* g, void* grad, int prec,
                             void* workspace, size_t workspace_bytes, void* stream);

/* Moments of one cell: m[0..d+1] = h^d sum_i Q_i phi(v_i), phi = 1, v, |v|^2
 * (Section 2.1), FP64 reduction of Q (double or float per prec).  m is a
 * DEVICE array of d+2 doubles. */
qdvm_status qdvm_moments(qdvm_plan_t plan, const void* Q, int prec, double* m, void* stream);

/* --------------------------------------------------------------- utility */

const char* qdvm_status_string(qdvm_status s);
/* Detail of the last error on the calling host thread ("" if none). */
const char* qdvm_last_error(void);
/* Library version string. */
const char* qdvm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QDVM_H */
