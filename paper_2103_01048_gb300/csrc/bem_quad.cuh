// Quadrature rules and the analytic triangle integrals shared by the P0 and
// P1 Galerkin assembly on the GPU (regular rules, collapsed Gauss rules,
// graded outer rules of the vertex-sharing patterns, the closed-form inner
// integrals of the singular entries).
#pragma once
#include "bem.cuh"
#include <algorithm>
#include <cmath>
#include <vector>

namespace pbfmm {

// ---------------------------------------------------------------------------
// quadrature rules
// ---------------------------------------------------------------------------
// regular rules, barycentric (l0, l1, l2) and weight (sum 1): the interior
// degree-2 3-point rule and Dunavant's degree-4 6-point rule
static inline void regular_rule(int nq, std::vector<double>& L, std::vector<double>& W) {
    L.clear(); W.clear();
    if (nq == 3) {
        const double a = 2.0 / 3.0, b = 1.0 / 6.0;
        double pts[3][3] = {{a, b, b}, {b, a, b}, {b, b, a}};
        for (auto& p : pts) { L.insert(L.end(), p, p + 3); W.push_back(1.0 / 3.0); }
    } else if (nq == 6) {
        const double a1 = 0.445948490915965, w1 = 0.223381589678011;
        const double a2 = 0.091576213509771, w2 = 0.109951743655322;
        for (int k = 0; k < 3; ++k) {
            double p[3] = {a1, a1, a1};
            p[k] = 1.0 - 2.0 * a1;
            L.insert(L.end(), p, p + 3); W.push_back(w1);
        }
        for (int k = 0; k < 3; ++k) {
            double p[3] = {a2, a2, a2};
            p[k] = 1.0 - 2.0 * a2;
            L.insert(L.end(), p, p + 3); W.push_back(w2);
        }
    } else {
        throw Error(PB_EINVAL, "nquad must be 3 or 6");
    }
}

// Gauss-Legendre on [0,1] (Newton on the Legendre recurrence)
static inline void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n); w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

// collapsed Gauss rule on the reference triangle (l1, l2, weight), weights sum to 1
// singular entries: 4x4 collapsed rules; the singular part of the outer rule
// is graded 5 levels deep in FP64 and 4 in FP32, the smooth Yukawa remainder
// 2 levels; FP64 up to kSingFp64MaxTris triangles unless chosen otherwise
constexpr int kSingOuterN = 4, kSingInnerN = 4;
constexpr int kSingDepth64 = 5, kSingDepth32 = 4, kSingRemDepth = 2;
constexpr long long kSingFp64MaxTris = 262144;

static inline void collapsed_rule(int n, std::vector<double>& out) {
    std::vector<double> x, w;
    gauss01(n, x, w);
    out.clear();
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            out.push_back(x[i] * (1.0 - x[j]));
            out.push_back(x[i] * x[j]);
            out.push_back(2.0 * x[i] * w[i] * w[j]);
        }
}

// ---------------------------------------------------------------------------
// singular Galerkin entries (identical or vertex-sharing pairs)
// Inner integrals: analytic for 1/r (uniform-density triangle potential,
// Wilton et al. 1984) and for (x-y).n/r^3 (solid angle, Van Oosterom &
// Strackee 1983); bounded Yukawa remainders by a collapsed Gauss rule.
// Outer integral: collapsed Gauss rule on a subdivision of T_i refined
// geometrically toward the part of T_i that T_j shares (its whole boundary,
// the common edge or the common vertex). That part depends only on which
// local vertices the two triangles share, so the graded outer rules of the
// eight sharing patterns are built once on the host in the reference frame
// of T_i (x = v0 + l1 (v1 - v0) + l2 (v2 - v0)) and every pair reads its
// pattern's points. The smooth Yukawa remainder takes a shallower rule.
// ---------------------------------------------------------------------------
template <typename T> struct V3 { T x, y, z; };
template <typename T> __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T> __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T> __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T> __device__ __forceinline__ T len(V3<T> a) { return sqrt(dot(a, a)); }

// int_T 1/|x-y| dA_y
template <typename T>
__device__ T pot_uniform_triangle(V3<T> x, const V3<T>* v) {
    const T skip = sizeof(T) == 8 ? T(1e-14) : T(1e-7);
    V3<T> n = cross(v[1] - v[0], v[2] - v[0]);
    n = (T(1) / len(n)) * n;
    T h = dot(x - v[0], n);
    T ah = fabs(h);
    V3<T> xp = x - h * n;                    // projection on the plane
    T scale = len(v[1] - v[0]) + len(v[2] - v[0]);
    T total = 0;
    for (int e = 0; e < 3; ++e) {
        V3<T> p = v[e], q = v[(e + 1) % 3];
        V3<T> t = q - p;
        t = (T(1) / len(t)) * t;
        V3<T> m = cross(t, n);                // in-plane, outward
        T d0 = dot(p - xp, m);                // signed distance to the edge line
        if (fabs(d0) <= skip * scale) continue;
        T s0 = dot(p - xp, t), s1 = dot(q - xp, t);
        T r0 = len(x - p), r1 = len(x - q);
        T w2 = d0 * d0 + h * h;
        T f1 = s1 >= 0 ? r1 + s1 : w2 / (r1 - s1);
        T f0 = s0 >= 0 ? r0 + s0 : w2 / (r0 - s0);
        total += d0 * log(f1 / f0);
        if (ah > 0) total -= ah * (atan(d0 * s1 / (w2 + ah * r1)) - atan(d0 * s0 / (w2 + ah * r0)));
    }
    return total;
}

// int_T (x-y).n_y/|x-y|^3 dA_y = signed solid angle of T seen from x
template <typename T>
__device__ T solid_angle(V3<T> x, const V3<T>* v) {
    V3<T> a = v[0] - x, b = v[1] - x, c = v[2] - x;
    T la = len(a), lb = len(b), lc = len(c);
    T num = dot(a, cross(b, c));
    T den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
    return T(-2) * atan2(num, den);
}

// g(t) = e^-t (1 + t) - 1: the Yukawa double-layer kernel minus the Laplace
// one is (x-y).n g(kr) / r^3. Below t = 1/4 the Taylor series
// sum_{n>=2} (-1)^n (1 - n) t^n / n! avoids the cancellation of the closed form.
template <typename T>
__device__ __forceinline__ T yukawa_dl_factor(T t) {
    if (t < T(0.25)) {
        T s = T(-1.0 / 43545600.0);
        s = s * t + T(1.0 / 3991680.0);
        s = s * t + T(-1.0 / 403200.0);
        s = s * t + T(1.0 / 45360.0);
        s = s * t + T(-1.0 / 5760.0);
        s = s * t + T(1.0 / 840.0);
        s = s * t + T(-1.0 / 144.0);
        s = s * t + T(1.0 / 30.0);
        s = s * t + T(-1.0 / 8.0);
        s = s * t + T(1.0 / 3.0);
        s = s * t + T(-0.5);
        return s * t * t;
    }
    return expm1(-t) + t * exp(-t);
}

constexpr int kNumPat = 8;     // 0 identical, 1..3 edge (v_k, v_k+1), 4..6 vertex k, 7 none
struct SingRule {
    int s_off[kNumPat + 1];    // singular-part outer points of pattern p: [s_off[p], s_off[p+1])
    int r_off[kNumPat + 1];    // remainder outer points
    int in_off;                // kSingInnerN^2 inner points of the remainder
};

// Is the reference-frame point (l1, l2) on the part of T_i shared with T_j?
// Subdivision vertices are dyadic rationals, so the tests are exact.
static inline bool on_shared(int pat, double l1, double l2) {
    switch (pat) {
    case 0: return l1 == 0.0 || l2 == 0.0 || l1 + l2 == 1.0;   // identical: the boundary
    case 1: return l2 == 0.0;                                  // edge v0 v1
    case 2: return l1 + l2 == 1.0;                             // edge v1 v2
    case 3: return l1 == 0.0;                                  // edge v2 v0
    case 4: return l1 == 0.0 && l2 == 0.0;                     // vertex v0
    case 5: return l1 == 1.0 && l2 == 0.0;                     // vertex v1
    case 6: return l1 == 0.0 && l2 == 1.0;                     // vertex v2
    default: return false;
    }
}

// Graded outer rule of one sharing pattern: leaves of the midpoint subdivision
// of the reference triangle, split while one of its vertices is on the shared
// part and fewer than `depth` levels deep, each carrying the collapsed rule
// scaled by its area fraction. Appends (l1, l2, w) with sum w = 1.
static inline void graded_rule(int pat, int depth, const std::vector<double>& rule, std::vector<double>& out) {
    struct Sub { double v[3][2]; int d; };
    std::vector<Sub> st{{{{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}}, 0}};
    while (!st.empty()) {
        Sub s = st.back();
        st.pop_back();
        bool touch = false;
        for (int a = 0; a < 3; ++a) touch = touch || on_shared(pat, s.v[a][0], s.v[a][1]);
        if (touch && s.d < depth) {
            double m[3][2];   // midpoints of v0v1, v1v2, v2v0
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 2; ++c) m[a][c] = 0.5 * (s.v[a][c] + s.v[(a + 1) % 3][c]);
            auto push = [&](const double* p, const double* q, const double* r) {
                st.push_back({{{p[0], p[1]}, {q[0], q[1]}, {r[0], r[1]}}, s.d + 1});
            };
            push(s.v[0], m[0], m[2]);
            push(m[0], s.v[1], m[1]);
            push(m[2], m[1], s.v[2]);
            push(m[1], m[2], m[0]);
            continue;
        }
        const double e1[2] = {s.v[1][0] - s.v[0][0], s.v[1][1] - s.v[0][1]};
        const double e2[2] = {s.v[2][0] - s.v[0][0], s.v[2][1] - s.v[0][1]};
        const double frac = std::fabs(e1[0] * e2[1] - e1[1] * e2[0]);
        for (size_t k = 0; k < rule.size(); k += 3) {
            out.push_back(s.v[0][0] + rule[k] * e1[0] + rule[k + 1] * e2[0]);
            out.push_back(s.v[0][1] + rule[k] * e1[1] + rule[k + 1] * e2[1]);
            out.push_back(rule[k + 2] * frac);
        }
    }
}


// All points of the singular rules (l1, l2, w triples): the graded outer
// rules of every pattern for the singular part (`depth` levels) and for the
// smooth Yukawa remainder (at most kSingRemDepth levels), then the inner
// collapsed rule of the remainder.
static inline SingRule make_sing_rule(int depth, std::vector<double>& pts) {
    std::vector<double> ro, ri;
    collapsed_rule(kSingOuterN, ro);
    collapsed_rule(kSingInnerN, ri);
    SingRule R;
    pts.clear();
    for (int pat = 0; pat <= kNumPat; ++pat) {
        R.s_off[pat] = (int)(pts.size() / 3);
        if (pat < kNumPat) graded_rule(pat, depth, ro, pts);
    }
    for (int pat = 0; pat <= kNumPat; ++pat) {
        R.r_off[pat] = (int)(pts.size() / 3);
        if (pat < kNumPat) graded_rule(pat, std::min(depth, kSingRemDepth), ro, pts);
    }
    R.in_off = (int)(pts.size() / 3);
    pts.insert(pts.end(), ri.begin(), ri.end());
    return R;
}

}  // namespace pbfmm
