/*
 * qdvm_oracle.c -- plain, slow CPU oracle (FP64) for the periodized,
 * direction-restricted discrete-velocity collision operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package entry's smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It
 * shares no code, header, table or helper with the CUDA implementation.
 *
 * What it computes (Mouhot, Pareschi, Rey, "Convolutive decomposition and
 * fast summation methods for discrete-velocity approximations of the
 * Boltzmann equation"):
 *
 *   Q_i = sum_{k,l} Gamma_{k,l} [ f_{i+k} f_{i+l} - f_i f_{i+k+l} ]
 *        eq. (DR), Section 2.3: the periodized operator truncated to
 *        |k|_inf, |l|_inf <= Ntilde; indices are taken modulo N (torus).
 *   Gamma_{k,l} = 1(k.l = 0) a(k) b(l),  b = 1
 *        eq. (decoup), Section 3.2 (decoupling of kernel and weights).
 *   a(k) = h^(2d-1) |k| / gcd(k)     ("hp": hard spheres in 3D, h^5 |k|/gcd;
 *                                       Maxwell molecules in 2D, h^3 |k|/gcd)
 *   a(k) = 1                          ("unit": constant kernel)
 *        Section 3.2, the weights quoted after eq. (decoup).
 *   Restriction: only k whose line e(k) = k/gcd(k) satisfies |e|_inf <= m
 *        are kept (the directions of the Farey-type set A_m); l ranges over
 *        all of e(k)^perp inside the box.  eq. (decDVM), Section 3.2.  With
 *        m >= Ntilde every line is kept and the sum is eq. (DR) itself.
 *   Terms with k = 0 or l = 0 are left out: each such term is identically
 *   zero (f_i f_{i+l} - f_i f_{i+l} = 0), and a(0) is not defined.
 *
 * Each sum is accumulated with Neumaier's compensated summation.  Loops run
 * over output points with OpenMP; every output point is summed by one thread
 * in a fixed term order, so results do not depend on the thread count
 * (except oracle_vjp, whose per-thread partial gradients are combined in
 * thread order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_D 3

/* ---------------------------------------------------------------- helpers */

typedef struct {
    double s, c;
} nsum_t; /* Neumaier accumulator: value = s + c */

static inline void nsum_add(nsum_t* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double nsum_value(const nsum_t* a) { return a->s + a->c; }

static long gcd2(long a, long b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) {
        long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static long gcd_vec(const int* v, int d) {
    long g = 0;
    for (int a = 0; a < d; ++a) g = gcd2(g, v[a]);
    return g;
}

static int linf_vec(const int* v, int d) {
    int n = 0;
    for (int a = 0; a < d; ++a) {
        int x = v[a] < 0 ? -v[a] : v[a];
        if (x > n) n = x;
    }
    return n;
}

static inline int wrap(int x, int N) {
    int r = x % N;
    return r < 0 ? r + N : r;
}

/* Advance a d-digit odometer over [-R, R]^d in lexicographic order (first
 * axis slowest).  Returns 0 when it wraps around. */
static int odometer_next(int* v, int d, int R) {
    for (int a = d - 1; a >= 0; --a) {
        if (v[a] < R) {
            v[a]++;
            return 1;
        }
        v[a] = -R;
    }
    return 0;
}

/* ------------------------------------------------------------ public API */

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Default truncation: Ntilde = floor(N / (3 + sqrt 2)), the no-aliasing
 * choice of Section 4 read with N = number of grid points per axis (the only
 * reading that reproduces the stated values 1, 3, 7, 14 for N = 8..64). */
int oracle_default_ntilde(int N) { return (int)floor((double)N / (3.0 + sqrt(2.0))); }

/* Lines through 0 with direction in [-m, m]^d: primitive integer vectors
 * (gcd of the components = 1), one per +- pair (first non-zero component
 * positive), listed by |e|_inf and then lexicographically.  Section 3.2,
 * the sets A^1 and A^2.  Writes min(count, cap) vectors (d ints each) into
 * out (may be NULL) and returns the count. */
int oracle_lines(int d, int m, int* out, int cap) {
    if (d < 1 || d > ORACLE_MAX_D || m < 0) return -1;
    int count = 0;
    for (int n = 1; n <= m; ++n) {
        int v[ORACLE_MAX_D];
        for (int a = 0; a < d; ++a) v[a] = -n;
        do {
            if (linf_vec(v, d) != n) continue;
            if (gcd_vec(v, d) != 1) continue;
            int first = 0;
            for (int a = 0; a < d; ++a)
                if (v[a] != 0) {
                    first = v[a];
                    break;
                }
            if (first <= 0) continue;
            if (out && count < cap)
                for (int a = 0; a < d; ++a) out[count * d + a] = v[a];
            count++;
        } while (odometer_next(v, d, n));
    }
    return count;
}

typedef struct {
    int k[ORACLE_MAX_D];
    int l[ORACLE_MAX_D];
    double w;
} term_t;

/* Weight a(k) of the decoupled kernel (b = 1). */
static double weight_a(const int* k, int d, int kernel, double h) {
    if (kernel == 0) return 1.0;
    long g = gcd_vec(k, d);
    double n2 = 0.0;
    for (int a = 0; a < d; ++a) n2 += (double)k[a] * (double)k[a];
    return pow(h, 2 * d - 1) * sqrt(n2) / (double)g;
}

/* All (k, l) with k, l in [-Nt, Nt]^d \ {0}, k.l = 0 and |k/gcd(k)|_inf <= m,
 * in lexicographic order of (k, l). */
static int build_terms(int d, int Nt, int m, int kernel, double h, term_t** out) {
    size_t cap = 1024, n = 0;
    term_t* t = (term_t*)malloc(cap * sizeof(term_t));
    if (!t) return -1;
    int k[ORACLE_MAX_D], l[ORACLE_MAX_D];
    for (int a = 0; a < d; ++a) k[a] = -Nt;
    do {
        if (linf_vec(k, d) == 0) continue;
        long g = gcd_vec(k, d);
        int e[ORACLE_MAX_D];
        for (int a = 0; a < d; ++a) e[a] = (int)(k[a] / g);
        if (linf_vec(e, d) > m) continue;
        double w = weight_a(k, d, kernel, h);
        for (int a = 0; a < d; ++a) l[a] = -Nt;
        do {
            if (linf_vec(l, d) == 0) continue;
            long dot = 0;
            for (int a = 0; a < d; ++a) dot += (long)k[a] * l[a];
            if (dot != 0) continue;
            if (n == cap) {
                cap *= 2;
                term_t* nt = (term_t*)realloc(t, cap * sizeof(term_t));
                if (!nt) {
                    free(t);
                    return -1;
                }
                t = nt;
            }
            memset(&t[n], 0, sizeof(term_t));
            for (int a = 0; a < d; ++a) {
                t[n].k[a] = k[a];
                t[n].l[a] = l[a];
            }
            t[n].w = w;
            n++;
        } while (odometer_next(l, d, Nt));
    } while (odometer_next(k, d, Nt));
    *out = t;
    return (int)n;
}

/* Number of (k, l) terms per output point. */
int oracle_terms_count(int d, int Ntilde, int m) {
    term_t* t = NULL;
    int n = build_terms(d, Ntilde, m, 0, 1.0, &t);
    free(t);
    return n;
}

static void unflatten(int64_t idx, int d, int N, int* c) {
    for (int a = d - 1; a >= 0; --a) {
        c[a] = (int)(idx % N);
        idx /= N;
    }
}

static int64_t flat_shift(const int* c, const int* s1, const int* s2, int d, int N) {
    int64_t r = 0;
    for (int a = 0; a < d; ++a) {
        int x = c[a] + (s1 ? s1[a] : 0) + (s2 ? s2[a] : 0);
        r = r * N + wrap(x, N);
    }
    return r;
}

static int check_args(int d, int N, int Ntilde, int m) {
    if (d < 2 || d > ORACLE_MAX_D) return -1;
    if (N < 1 || Ntilde < 1 || m < 0) return -1;
    return 0;
}

/* Q (and optionally gain, loss, scale = sum |terms|) at the listed flat
 * output indices (all N^d points if idx == NULL, in which case n_idx is
 * ignored and outputs have N^d entries).  Returns 0 on success. */
int oracle_q_points(int d, int N, int Ntilde, int m, int kernel, double h, const double* f,
                    const int64_t* idx, int64_t n_idx, double* Q, double* gain, double* loss,
                    double* scale) {
    if (check_args(d, N, Ntilde, m)) return -1;
    term_t* T = NULL;
    int nt = build_terms(d, Ntilde, m, kernel, h, &T);
    if (nt < 0) return -2;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
    int64_t n_out = idx ? n_idx : total;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        int c[ORACLE_MAX_D];
        unflatten(i, d, N, c);
        nsum_t q = {0, 0}, g = {0, 0}, lo = {0, 0}, sc = {0, 0};
        double fi = f[i];
        for (int t = 0; t < nt; ++t) {
            double a = f[flat_shift(c, T[t].k, NULL, d, N)];
            double b = f[flat_shift(c, T[t].l, NULL, d, N)];
            double e = f[flat_shift(c, T[t].k, T[t].l, d, N)];
            double gain_t = T[t].w * a * b;
            double loss_t = T[t].w * fi * e;
            nsum_add(&q, gain_t);
            nsum_add(&q, -loss_t);
            nsum_add(&g, gain_t);
            nsum_add(&lo, loss_t);
            nsum_add(&sc, fabs(gain_t));
            nsum_add(&sc, fabs(loss_t));
        }
        Q[o] = nsum_value(&q);
        if (gain) gain[o] = nsum_value(&g);
        if (loss) loss[o] = nsum_value(&lo);
        if (scale) scale[o] = nsum_value(&sc);
    }
    free(T);
    return 0;
}

int oracle_q(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, double* Q,
             double* gain, double* loss, double* scale) {
    return oracle_q_points(d, N, Ntilde, m, kernel, h, f, NULL, 0, Q, gain, loss, scale);
}

/* Flat index of c + s1 + s2 inside the box [0, N)^d, or -1 outside. */
static int64_t flat_box(const int* c, const int* s1, const int* s2, int d, int N) {
    int64_t r = 0;
    for (int a = 0; a < d; ++a) {
        int x = c[a] + (s1 ? s1[a] : 0) + (s2 ? s2[a] : 0);
        if (x < 0 || x >= N) return -1;
        r = r * N + x;
    }
    return r;
}

/* The box-truncated operator D^tr of Section 2.3 with the same terms as Q
 * (k, l in [-Ntilde, Ntilde]^d, k.l = 0, k's line in A_m, weight a(k)):
 * no periodisation, a term counts only when i + k, i + l and i + k + l all
 * lie in the grid.  Q and scale (sum of |terms|) at every point. */
int oracle_dtr(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, double* Q,
               double* scale) {
    if (check_args(d, N, Ntilde, m)) return -1;
    term_t* T = NULL;
    int nt = build_terms(d, Ntilde, m, kernel, h, &T);
    if (nt < 0) return -2;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < total; ++i) {
        int c[ORACLE_MAX_D];
        unflatten(i, d, N, c);
        nsum_t q = {0, 0}, sc = {0, 0};
        double fi = f[i];
        for (int t = 0; t < nt; ++t) {
            int64_t ik = flat_box(c, T[t].k, NULL, d, N);
            int64_t il = flat_box(c, T[t].l, NULL, d, N);
            int64_t ikl = flat_box(c, T[t].k, T[t].l, d, N);
            if (ik < 0 || il < 0 || ikl < 0) continue;
            double gain_t = T[t].w * f[ik] * f[il];
            double loss_t = T[t].w * fi * f[ikl];
            nsum_add(&q, gain_t);
            nsum_add(&q, -loss_t);
            nsum_add(&sc, fabs(gain_t));
            nsum_add(&sc, fabs(loss_t));
        }
        Q[i] = nsum_value(&q);
        if (scale) scale[i] = nsum_value(&sc);
    }
    free(T);
    return 0;
}

/* Directional derivative of Q at f along df (Q is quadratic in f):
 *   dQ_i = sum Gamma [df_{i+k} f_{i+l} + f_{i+k} df_{i+l}
 *                     - df_i f_{i+k+l} - f_i df_{i+k+l}],
 * at the listed flat indices (all points if idx == NULL).  scale (may be
 * NULL) receives the sum of the absolute values of the four products. */
int oracle_jvp_points(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, const double* df,
                      const int64_t* idx, int64_t n_idx, double* dQ, double* scale) {
    if (check_args(d, N, Ntilde, m)) return -1;
    term_t* T = NULL;
    int nt = build_terms(d, Ntilde, m, kernel, h, &T);
    if (nt < 0) return -2;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
    int64_t n_out = idx ? n_idx : total;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        int c[ORACLE_MAX_D];
        unflatten(i, d, N, c);
        nsum_t s = {0, 0}, sc = {0, 0};
        for (int t = 0; t < nt; ++t) {
            int64_t ia = flat_shift(c, T[t].k, NULL, d, N);
            int64_t ib = flat_shift(c, T[t].l, NULL, d, N);
            int64_t ie = flat_shift(c, T[t].k, T[t].l, d, N);
            double w = T[t].w;
            double p1 = w * df[ia] * f[ib], p2 = w * f[ia] * df[ib];
            double p3 = w * df[i] * f[ie], p4 = w * f[i] * df[ie];
            nsum_add(&s, p1);
            nsum_add(&s, p2);
            nsum_add(&s, -p3);
            nsum_add(&s, -p4);
            nsum_add(&sc, fabs(p1) + fabs(p2));
            nsum_add(&sc, fabs(p3) + fabs(p4));
        }
        dQ[o] = nsum_value(&s);
        if (scale) scale[o] = nsum_value(&sc);
    }
    free(T);
    return 0;
}

int oracle_jvp(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, const double* df,
               double* dQ) {
    return oracle_jvp_points(d, N, Ntilde, m, kernel, h, f, df, NULL, 0, dQ, NULL);
}

/* Transpose of the Jacobian applied to g, by scattering the four partial
 * derivatives of every term:
 *   grad[i+k] += w g_i f_{i+l},   grad[i+l]   += w g_i f_{i+k},
 *   grad[i]   -= w g_i f_{i+k+l}, grad[i+k+l] -= w g_i f_i.
 * scale (may be NULL) receives the scattered absolute values. */
int oracle_vjp_scale(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, const double* g,
                     double* grad, double* scale) {
    if (check_args(d, N, Ntilde, m)) return -1;
    term_t* T = NULL;
    int nt = build_terms(d, Ntilde, m, kernel, h, &T);
    if (nt < 0) return -2;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
    int nthr = oracle_max_threads();
    nsum_t* part = (nsum_t*)calloc((size_t)nthr * (size_t)total * 2, sizeof(nsum_t));
    if (!part) {
        free(T);
        return -2;
    }
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        nsum_t* acc = part + (size_t)tid * (size_t)total * 2;
        nsum_t* sca = acc + total;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < total; ++i) {
            int c[ORACLE_MAX_D];
            unflatten(i, d, N, c);
            for (int t = 0; t < nt; ++t) {
                int64_t ia = flat_shift(c, T[t].k, NULL, d, N);
                int64_t ib = flat_shift(c, T[t].l, NULL, d, N);
                int64_t ie = flat_shift(c, T[t].k, T[t].l, d, N);
                double wg = T[t].w * g[i];
                double pa = wg * f[ib], pb = wg * f[ia], pi = wg * f[ie], pe = wg * f[i];
                nsum_add(&acc[ia], pa);
                nsum_add(&acc[ib], pb);
                nsum_add(&acc[i], -pi);
                nsum_add(&acc[ie], -pe);
                nsum_add(&sca[ia], fabs(pa));
                nsum_add(&sca[ib], fabs(pb));
                nsum_add(&sca[i], fabs(pi));
                nsum_add(&sca[ie], fabs(pe));
            }
        }
    }
    for (int64_t i = 0; i < total; ++i) {
        nsum_t s = {0, 0}, sc = {0, 0};
        for (int t = 0; t < nthr; ++t) {
            const nsum_t* acc = part + (size_t)t * (size_t)total * 2;
            nsum_add(&s, acc[i].s);
            nsum_add(&s, acc[i].c);
            nsum_add(&sc, acc[total + i].s);
            nsum_add(&sc, acc[total + i].c);
        }
        grad[i] = nsum_value(&s);
        if (scale) scale[i] = nsum_value(&sc);
    }
    free(part);
    free(T);
    return 0;
}

int oracle_vjp(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, const double* g,
               double* grad) {
    return oracle_vjp_scale(d, N, Ntilde, m, kernel, h, f, g, grad, NULL);
}

/* The same transpose at selected points, summed as a gather: point p
 * receives, from every term (k, l), the derivative of the terms in which f_p
 * appears:
 *   grad_p = sum Gamma [ g_{p-k} f_{p-k+l} + g_{p-l} f_{p-l+k}
 *                        - g_p f_{p+k+l} - g_{p-k-l} f_{p-k-l} ]. */
int oracle_vjp_points(int d, int N, int Ntilde, int m, int kernel, double h, const double* f, const double* g,
                      const int64_t* idx, int64_t n_idx, double* grad, double* scale) {
    if (check_args(d, N, Ntilde, m)) return -1;
    term_t* T = NULL;
    int nt = build_terms(d, Ntilde, m, kernel, h, &T);
    if (nt < 0) return -2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t o = 0; o < n_idx; ++o) {
        int64_t p = idx[o];
        int c[ORACLE_MAX_D];
        unflatten(p, d, N, c);
        nsum_t s = {0, 0}, sc = {0, 0};
        for (int t = 0; t < nt; ++t) {
            int mk[ORACLE_MAX_D], ml[ORACLE_MAX_D];
            for (int a = 0; a < d; ++a) {
                mk[a] = -T[t].k[a];
                ml[a] = -T[t].l[a];
            }
            double w = T[t].w;
            double t1 = w * g[flat_shift(c, mk, NULL, d, N)] * f[flat_shift(c, mk, T[t].l, d, N)];
            double t2 = w * g[flat_shift(c, ml, NULL, d, N)] * f[flat_shift(c, ml, T[t].k, d, N)];
            double t3 = w * g[p] * f[flat_shift(c, T[t].k, T[t].l, d, N)];
            double t4 = w * g[flat_shift(c, mk, ml, d, N)] * f[flat_shift(c, mk, ml, d, N)];
            nsum_add(&s, t1);
            nsum_add(&s, t2);
            nsum_add(&s, -t3);
            nsum_add(&s, -t4);
            nsum_add(&sc, fabs(t1) + fabs(t2));
            nsum_add(&sc, fabs(t3) + fabs(t4));
        }
        grad[o] = nsum_value(&s);
        if (scale) scale[o] = nsum_value(&sc);
    }
    free(T);
    return 0;
}

/* Velocity moments h^d sum_i Q_i phi(v_i) for phi = 1, v_0, ..., v_{d-1},
 * |v|^2 (conservation of mass, momentum and energy, Section 2.1), with
 * v_j = -L + j h per axis.  m_out has d + 2 entries. */
int oracle_moments(int d, int N, double L, const double* Q, double* m_out) {
    if (d < 1 || d > ORACLE_MAX_D || N < 1) return -1;
    double h = 2.0 * L / N;
    int64_t total = 1;
    for (int a = 0; a < d; ++a) total *= N;
    nsum_t acc[ORACLE_MAX_D + 2];
    memset(acc, 0, sizeof(acc));
    for (int64_t i = 0; i < total; ++i) {
        int c[ORACLE_MAX_D];
        unflatten(i, d, N, c);
        double v2 = 0.0;
        nsum_add(&acc[0], Q[i]);
        for (int a = 0; a < d; ++a) {
            double v = -L + c[a] * h;
            nsum_add(&acc[1 + a], Q[i] * v);
            v2 += v * v;
        }
        nsum_add(&acc[d + 1], Q[i] * v2);
    }
    double hd = pow(h, d);
    for (int a = 0; a < d + 2; ++a) m_out[a] = hd * nsum_value(&acc[a]);
    return 0;
}
