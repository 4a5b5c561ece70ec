// Host side of the plan: the 3D plane polygons e^perp ∩ [-Ntilde, Ntilde]^3
// (the offsets l of the plane sums P_e, alpha'_p in eq. (decDVM)) as rows
// along an in-plane lattice vector, with the lines grouped by that vector.
//
// For a line e pick a primitive u in e^perp and a v with u x v = ±e, so that
// (u, v) is a basis of the plane lattice e^perp ∩ Z^3.  Every polygon point
// is l = a u + b v, and for fixed b the admissible a form an interval (the
// polygon is convex); the row b = 0 is split at the excluded l = 0.  Lines
// sharing u form a class.  For a class the evaluator re-indexes the cell in
// the coordinates (alpha, beta, gamma) of a unimodular basis (u, w2, w3) of
// Z^3 — a bijection of the torus Z_N^3 — so that every row is a contiguous
// run along alpha and a thread that owns 8 consecutive alpha points reads a
// row of length n once (n + 7 loads) instead of 8 n times.
//
// u is chosen per line among short vectors to minimise the loads of its
// rows other than the central one (see below), allowing 15% over the best
// choice so that few classes cover all lines (greedy).
//
// The row b = 0 of every line of a class is the same set {a u : 0 < |a| <= A},
// A = floor(Ntilde / |u|_inf): the line window of u itself.  When A >= 1 each
// line lists these two segments first, so that an evaluator may sum them
// once per class (A follows from u, the first column of the class matrix).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <map>
#include <vector>

#include "qdvm_internal.cuh"

namespace {

using V3 = std::array<int, 3>;

int dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
V3 cross(const V3& a, const V3& b) {
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
int det3(const V3& a, const V3& b, const V3& c) { return dot(a, cross(b, c)); }
V3 neg(const V3& a) { return {-a[0], -a[1], -a[2]}; }
int inf_norm(const V3& a) { return std::max(std::abs(a[0]), std::max(std::abs(a[1]), std::abs(a[2]))); }
int l1_norm(const V3& a) { return std::abs(a[0]) + std::abs(a[1]) + std::abs(a[2]); }
int gcd(int a, int b) {
    a = std::abs(a);
    b = std::abs(b);
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

struct Seg {
    int b, a0, a1;
};

struct Option {
    int cost = 0, ui = -1;
    V3 v{};
    std::vector<Seg> segs;
};

// Primitive vectors of [-3, 3]^3 up to sign (first non-zero entry positive),
// shortest first.
std::vector<V3> small_vectors() {
    std::vector<V3> out;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) {
                const V3 u{x, y, z};
                if (!x && !y && !z) continue;
                if (gcd(gcd(x, y), z) != 1) continue;
                const int first = x ? x : (y ? y : z);
                if (first < 0) continue;
                out.push_back(u);
            }
    std::sort(out.begin(), out.end(), [](const V3& a, const V3& b) {
        const int na = inf_norm(a), nb = inf_norm(b);
        if (na != nb) return na < nb;
        const int la = l1_norm(a), lb = l1_norm(b);
        if (la != lb) return la < lb;
        return a < b;
    });
    return out;
}

// Rows of the polygon pts (sorted shortest first) along u; false when no
// v with u x v = ±e lies in the polygon.
bool rows_for(const V3& e, const V3& u, const std::vector<V3>& pts, Option* o) {
    const int ee = dot(e, e);
    int s = 0;
    for (const V3& l : pts) {
        const V3 c = cross(u, l);
        if (c == e) s = 1;
        else if (c == neg(e)) s = -1;
        if (s) {
            o->v = l;
            break;
        }
    }
    if (!s) return false;
    const int k = u[0] ? 0 : (u[1] ? 1 : 2);
    std::map<int, std::vector<int>> rows;
    for (const V3& l : pts) {
        const int bn = dot(cross(u, l), e) * s;
        if (bn % ee) return false;
        const int b = bn / ee;
        const V3 r{l[0] - b * o->v[0], l[1] - b * o->v[1], l[2] - b * o->v[2]};
        if (r[k] % u[k]) return false;
        const int a = r[k] / u[k];
        if (r[0] != a * u[0] || r[1] != a * u[1] || r[2] != a * u[2]) return false;
        rows[b].push_back(a);
    }
    o->segs.clear();
    o->cost = 0;
    for (auto& kv : rows) {
        std::vector<int>& aa = kv.second;
        std::sort(aa.begin(), aa.end());
        size_t i = 0;
        while (i < aa.size()) {
            size_t j = i;
            while (j + 1 < aa.size() && aa[j + 1] == aa[j] + 1) ++j;
            o->segs.push_back(Seg{kv.first, aa[i], aa[j]});
            // the central row b = 0 is summed once per class, not per line
            if (kv.first != 0) o->cost += (aa[j] - aa[i] + 1) + 7 + 10;
            i = j + 1;
        }
    }
    return true;
}

// (w2, w3) with det(u, w2, w3) = 1; w3 a coordinate axis, the last axis
// preferred (then neighbouring gamma are neighbouring addresses).
bool complete_basis(const V3& u, V3* w2, V3* w3) {
    const V3 axes[3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}};
    std::vector<V3> cand;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) cand.push_back(V3{x, y, z});
    std::sort(cand.begin(), cand.end(), [](const V3& a, const V3& b) {
        const int la = l1_norm(a), lb = l1_norm(b);
        return la != lb ? la < lb : a < b;
    });
    for (const V3& ax : axes)
        for (const V3& w : cand) {
            const int d = det3(u, w, ax);
            if (d == 1 || d == -1) {
                *w2 = d == 1 ? w : neg(w);
                *w3 = ax;
                return true;
            }
        }
    return false;
}

int mod(int a, int N) { return ((a % N) + N) % N; }

}  // namespace

// Builds the row tables of a 3D plan (N = 16 or 32, Ntilde <= 7).  On any
// inconsistency the plan keeps n_rclass = 0 and the evaluator uses the
// point-by-point plane sums.
qdvm_status build_row_tables(qdvm_plan_s* p) {
    p->n_rclass = 0;
    const int N = p->N, Nt = p->Ntilde, n = p->n_lines;
    if (p->d != 3 || (N != 16 && N != 32) || Nt > 7 || n < 1) return QDVM_OK;
    const std::vector<V3> small = small_vectors();
    std::vector<V3> box;
    for (int x = -Nt; x <= Nt; ++x)
        for (int y = -Nt; y <= Nt; ++y)
            for (int z = -Nt; z <= Nt; ++z)
                if (x || y || z) box.push_back(V3{x, y, z});
    std::sort(box.begin(), box.end(), [](const V3& a, const V3& b) {
        const int na = inf_norm(a), nb = inf_norm(b);
        return na != nb ? na < nb : a < b;
    });

    // options per line
    std::vector<std::vector<Option>> opts(n);
    std::vector<int> best(n, 0);
    for (int i = 0; i < n; ++i) {
        const int4 q = p->h_lines[i];
        const V3 e{q.x, q.y, q.z};
        std::vector<V3> pts;
        for (const V3& l : box)
            if (dot(l, e) == 0) pts.push_back(l);
        for (int ui = 0; ui < (int)small.size(); ++ui) {
            if (dot(small[ui], e) != 0) continue;
            Option o;
            o.ui = ui;
            if (rows_for(e, small[ui], pts, &o)) opts[i].push_back(o);
        }
        if (opts[i].empty()) return QDVM_OK;
        int b = opts[i][0].cost;
        for (const Option& o : opts[i]) b = std::min(b, o.cost);
        best[i] = b;
    }
    auto ok = [&](int i, const Option& o) { return 100 * o.cost <= 115 * best[i]; };

    // greedy cover of the lines by classes of a common u
    std::vector<char> done(n, 0);
    int left = n;
    std::vector<int> cls_u;
    std::vector<std::vector<int>> cls_lines;
    while (left > 0) {
        std::vector<int> cnt(small.size(), 0);
        for (int i = 0; i < n; ++i)
            if (!done[i])
                for (const Option& o : opts[i])
                    if (ok(i, o)) ++cnt[o.ui];
        const int ui = (int)(std::max_element(cnt.begin(), cnt.end()) - cnt.begin());
        if (cnt[ui] == 0) return QDVM_OK;
        std::vector<int> got;
        for (int i = 0; i < n; ++i)
            if (!done[i])
                for (const Option& o : opts[i])
                    if (o.ui == ui && ok(i, o)) {
                        got.push_back(i);
                        done[i] = 1;
                        --left;
                        break;
                    }
        cls_u.push_back(ui);
        cls_lines.push_back(got);
    }

    // class tables
    const int nc = (int)cls_u.size();
    std::vector<int> hcls((size_t)nc * QDVM_RCLASS_INTS);
    std::vector<int4> hline;
    std::vector<double> hc;
    std::vector<int> hrs(1, 0);
    std::vector<uchar4> hrow;
    for (int k = 0; k < nc; ++k) {
        const V3 u = small[cls_u[k]];
        V3 w2, w3;
        if (!complete_basis(u, &w2, &w3)) return QDVM_OK;
        const int M[3][3] = {{u[0], w2[0], w3[0]}, {u[1], w2[1], w3[1]}, {u[2], w2[2], w3[2]}};
        // inverse of a determinant-1 integer matrix: its adjugate
        int Mi[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
                Mi[r][c] = M[r1][c1] * M[r2][c2] - M[r1][c2] * M[r2][c1];
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                int s = 0;
                for (int t = 0; t < 3; ++t) s += Mi[r][t] * M[t][c];
                if (s != (r == c ? 1 : 0)) return QDVM_OK;
            }
        int* cd = &hcls[(size_t)k * QDVM_RCLASS_INTS];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                cd[3 * r + c] = M[r][c];
                cd[9 + 3 * r + c] = Mi[r][c];
            }
        cd[18] = (int)hline.size();
        // the central row b = 0 of every line: [-A, -1] and [1, A]
        const int A = Nt / inf_norm(u);
        for (int i : cls_lines[k]) {
            const Option* o = nullptr;
            for (const Option& q : opts[i])
                if (q.ui == cls_u[k] && ok(i, q)) {
                    o = &q;
                    break;
                }
            const int4 q = p->h_lines[i];
            const V3 e{q.x, q.y, q.z};
            V3 ep, vp;
            for (int r = 0; r < 3; ++r) {
                ep[r] = Mi[r][0] * e[0] + Mi[r][1] * e[1] + Mi[r][2] * e[2];
                vp[r] = Mi[r][0] * o->v[0] + Mi[r][1] * o->v[1] + Mi[r][2] * o->v[2];
            }
            hline.push_back(make_int4(mod(ep[0], N), mod(ep[1], N), mod(ep[2], N), q.w));
            hc.push_back(p->h_c[i]);
            // central segments first, then the other rows in order of b
            std::vector<Seg> segs;
            for (const Seg& s : o->segs)
                if (s.b == 0) segs.push_back(s);
            const bool has_central = segs.size() == 2 && segs[0].a0 == -A && segs[0].a1 == -1 && segs[1].a0 == 1 &&
                                     segs[1].a1 == A;
            if (A >= 1 ? !has_central : !segs.empty()) return QDVM_OK;
            for (const Seg& s : o->segs)
                if (s.b != 0) segs.push_back(s);
            for (const Seg& s : segs) {
                const int len = s.a1 - s.a0 + 1;
                if (len < 1 || len > QDVM_ROW_MAX) return QDVM_OK;
                hrow.push_back(make_uchar4((unsigned char)mod(s.a0 + s.b * vp[0], N),
                                           (unsigned char)mod(s.b * vp[1], N), (unsigned char)mod(s.b * vp[2], N),
                                           (unsigned char)len));
            }
            hrs.push_back((int)hrow.size());
        }
        cd[19] = (int)hline.size();
    }

    std::vector<float> hcf(hc.size());  // the FP32 kernels' copy of the weights
    for (size_t i = 0; i < hc.size(); ++i) hcf[i] = (float)hc[i];
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_rclass, hcls.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rline, hline.size() * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rc, hc.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rc_f, hc.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rrow_start, hrs.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_rrow, hrow.size() * sizeof(uchar4))) != cudaSuccess)
        return qdvm_cuda_status(e, "row tables");
    if ((e = cudaMemcpy(p->d_rclass, hcls.data(), hcls.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_rline, hline.data(), hline.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_rc, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_rc_f, hcf.data(), hcf.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_rrow_start, hrs.data(), hrs.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->d_rrow, hrow.data(), hrow.size() * sizeof(uchar4), cudaMemcpyHostToDevice)) != cudaSuccess)
        return qdvm_cuda_status(e, "row tables upload");
    p->n_rclass = nc;
    p->n_rrow = (int)hrow.size();
    return QDVM_OK;
}
