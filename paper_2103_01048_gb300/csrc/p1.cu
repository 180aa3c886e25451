// P1 (continuous piecewise-linear) Galerkin BEM on the GPU: the direct
// formulation (Eq. direct) and the two derivative formulations, interior
// (Eq. juffer) and exterior (Eq. lu), with the mass-lumped preconditioner
// (Sec. "Matrix conditioning of two derivative formulations").
//
// Mat-vec, as Eq. bempp_fmm_matvec with P1 trial/test functions:
//   P1   quadrature-point densities from the vertex values: monopole
//        w psi (psi = dphi/dn), dipole w phi, and for the hypersingular
//        operators the surface-curl density w curl(phi) (3 components) and
//        w phi n (3 components);
//   G    FMM passes: one paired Laplace+Yukawa pass with monopoles and
//        dipoles (V and K), one paired pass with target-normal derivatives
//        (K', derivative formulations only), three paired passes of the
//        curl components and three Yukawa passes of the phi n components
//        (W_Y - W_L in the integrated-by-parts form
//          <W u, v> = int int g curl u . curl v (+ kappa^2 n.n' g_Y u v));
//   C, S the G entries of vertex-sharing triangle pairs replaced by their
//        singular values: per pair a 3x3 block per kernel of the singular
//        integral minus the same block under the regular product rule,
//        assembled once (K' blocks are transposed K blocks, W blocks follow
//        from the V blocks and the curls);
//   P2^T per triangle the three test integrals, then per vertex a
//        fixed-order sum over its triangles;
// then the identity terms (the P1 mass matrix) and the lumped-mass
// preconditioner.
#include "bem.cuh"
#include "bem_quad.cuh"
#include <algorithm>
#include <cmath>
#include <vector>

namespace pbfmm {

constexpr double kInv4PiP = 0.07957747154594767;

struct RegRule {        // regular rule: barycentrics and weights (sum 1)
    int nq;
    double l[6][3];
    double w[6];
};

static RegRule make_reg_rule(int nq) {
    std::vector<double> L, W;
    regular_rule(nq, L, W);
    RegRule r;
    r.nq = nq;
    for (int k = 0; k < nq; ++k) {
        for (int a = 0; a < 3; ++a) r.l[k][a] = L[3 * k + a];
        r.w[k] = W[k];
    }
    return r;
}

// ---------------------------------------------------------------------------
// linear-density inner integrals over a flat triangle v[0..2] at x:
//   sl3[b] = int lambda_b(y) / |x - y| dA_y,
//   dl3[b] = int lambda_b(y) (x - y).n / |x - y|^3 dA_y,
// around the projection p of x on the plane (height h): lambda_b(y) =
// lambda_b(p) + grad lambda_b . (y - p); the uniform parts are the closed
// forms of the P0 entries (Wilton et al.; the solid angle), the vector
// moments int (y - p)/R and int (y - p)/R^3 become edge integrals by the
// divergence theorem in the plane (int R ds and int 1/R ds in closed form).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void tri_lin(V3<T> x, const V3<T>* v, bool same, T* sl3, T* dl3) {
    const T skip = sizeof(T) == 8 ? T(1e-14) : T(1e-7);
    const V3<T> e1 = v[1] - v[0], e2 = v[2] - v[0];
    V3<T> n = cross(e1, e2);
    const T twoA = len(n);
    n = (T(1) / twoA) * n;
    const T h = dot(x - v[0], n);
    const T ah = fabs(h);
    const V3<T> p = x - h * n;
    const T scale = len(e1) + len(e2);
    T sl0 = 0;
    V3<T> I1 = {0, 0, 0}, J1 = {0, 0, 0};
    for (int e = 0; e < 3; ++e) {
        const V3<T> pa = v[e], pb = v[(e + 1) % 3];
        V3<T> t = pb - pa;
        t = (T(1) / len(t)) * t;
        const V3<T> m = cross(t, n);               // in-plane, outward
        const T d0 = dot(pa - p, m);
        const T s0 = dot(pa - p, t), s1 = dot(pb - p, t);
        const T r0 = len(x - pa), r1 = len(x - pb);
        const T w2 = d0 * d0 + h * h;
        T intR = T(0.5) * (s1 * r1 - s0 * r0);
        if (w2 > skip * skip * scale * scale) {
            const T f1 = s1 >= 0 ? r1 + s1 : w2 / (r1 - s1);
            const T f0 = s0 >= 0 ? r0 + s0 : w2 / (r0 - s0);
            const T lg = log(f1 / f0);
            intR += T(0.5) * w2 * lg;
            J1 = J1 + lg * m;
            if (fabs(d0) > skip * scale) {
                sl0 += d0 * lg;
                if (ah > 0) sl0 -= ah * (atan(d0 * s1 / (w2 + ah * r1)) - atan(d0 * s0 / (w2 + ah * r0)));
            }
        }
        I1 = I1 + intR * m;
    }
    const T om = (same || !(ah > 0)) ? T(0) : solid_angle(x, v);
    for (int b = 0; b < 3; ++b) {
        const V3<T> A = v[(b + 1) % 3], C = v[(b + 2) % 3];
        const T lam = dot(cross(A - p, C - p), n) / twoA;
        const V3<T> g = (T(1) / twoA) * cross(n, C - A);
        sl3[b] = lam * sl0 + dot(g, I1);
        dl3[b] = same ? T(0) : lam * om - h * dot(g, J1);
    }
}

// ---------------------------------------------------------------------------
// singular P1 blocks of the vertex-sharing pairs, minus their regular-rule
// part: D[e][op][a][b], op = V_L, K_L, V_Y, K_Y, a the test vertex of T_i,
// b the trial vertex of T_j (CSR entry e = (i, j)).  One warp per pair; the
// graded outer rules of the sharing patterns as for the P0 entries.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_singular_p1(long long nadj, int nt, const double* __restrict__ V,
                                                     const int* __restrict__ F, const int* __restrict__ adj_off,
                                                     const int* __restrict__ adj_ids, T kappa, SingRule R,
                                                     const T* __restrict__ pts, RegRule rr, double* __restrict__ D) {
    const int lane = threadIdx.x & 31;
    const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
    for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < nadj; e += nw) {
        int lo = 0, hi = nt;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (adj_off[mid] <= e) lo = mid; else hi = mid;
        }
        const int i = lo, j = adj_ids[e];
        int fi[3], fj[3];
        for (int k = 0; k < 3; ++k) { fi[k] = F[3 * i + k]; fj[k] = F[3 * j + k]; }
        int shared = 0, mask = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (fi[a] == fj[b]) { ++shared; mask |= 1 << a; }
        int pat;
        if (i == j || shared == 3) pat = 0;
        else if (shared == 2) pat = mask == 3 ? 1 : (mask == 6 ? 2 : 3);
        else if (shared == 1) pat = 4 + (mask == 1 ? 0 : (mask == 2 ? 1 : 2));
        else pat = 7;
        const double ox = V[3 * fi[0]], oy = V[3 * fi[0] + 1], oz = V[3 * fi[0] + 2];
        auto rel = [&](int vv) -> V3<T> {
            return {(T)(V[3 * vv] - ox), (T)(V[3 * vv + 1] - oy), (T)(V[3 * vv + 2] - oz)};
        };
        const V3<T> E1 = rel(fi[1]), E2 = rel(fi[2]);
        const V3<T> Tj[3] = {rel(fj[0]), rel(fj[1]), rel(fj[2])};
        V3<T> nj = cross(Tj[1] - Tj[0], Tj[2] - Tj[0]);
        const T aj = T(0.5) * len(nj);
        nj = (T(1) / (T(2) * aj)) * nj;
        const T ai = T(0.5) * len(cross(E1, E2));
        const bool same = pat == 0;
        // accumulators divided by |T_i| / (4 pi) (singular parts) and by
        // |T_i| |T_j| / (4 pi) (Yukawa remainders)
        T sl[3][3] = {}, dl[3][3] = {}, rs[3][3] = {}, rd[3][3] = {};
        for (int k = R.s_off[pat] + lane; k < R.s_off[pat + 1]; k += 32) {
            const T l1 = pts[3 * k], l2 = pts[3 * k + 1], w = pts[3 * k + 2];
            const V3<T> x = l1 * E1 + l2 * E2;
            const T la[3] = {T(1) - l1 - l2, l1, l2};
            T s3[3], d3[3];
            tri_lin(x, Tj, same, s3, d3);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    sl[a][b] += w * la[a] * s3[b];
                    dl[a][b] += w * la[a] * d3[b];
                }
        }
        if (kappa > 0) {
            for (int k = R.r_off[pat] + lane; k < R.r_off[pat + 1]; k += 32) {
                const T l1 = pts[3 * k], l2 = pts[3 * k + 1], w = pts[3 * k + 2];
                const V3<T> x = l1 * E1 + l2 * E2;
                const T la[3] = {T(1) - l1 - l2, l1, l2};
                T s3[3] = {0, 0, 0}, d3[3] = {0, 0, 0};
                for (int m = 0; m < kSingInnerN * kSingInnerN; ++m) {
                    const T m1 = pts[3 * (R.in_off + m)], m2 = pts[3 * (R.in_off + m) + 1];
                    const T wm = pts[3 * (R.in_off + m) + 2];
                    const T lb[3] = {T(1) - m1 - m2, m1, m2};
                    const V3<T> y = (lb[0] * Tj[0]) + (m1 * Tj[1]) + (m2 * Tj[2]);
                    const V3<T> dv = x - y;
                    const T r = len(dv);
                    T fs, fd = 0;
                    if (r > (T)1e-30) {
                        const T t = kappa * r;
                        fs = expm1(-t) / r;
                        if (!same) fd = dot(dv, nj) * yukawa_dl_factor(t) / (r * r * r);
                    } else {
                        fs = -kappa;
                    }
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        s3[b] += wm * lb[b] * fs;
                        d3[b] += wm * lb[b] * fd;
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        rs[a][b] += w * la[a] * s3[b];
                        rd[a][b] += w * la[a] * d3[b];
                    }
            }
        }
        // minus the regular product rule of the same pair (what the FMM and
        // the point sums include for it), in the same scaling
        for (int q = lane; q < rr.nq * rr.nq; q += 32) {
            const int qa = q / rr.nq, qb = q % rr.nq;
            // a point paired with itself (identical triangles) is excluded by
            // the point sums; here x and y are built in different frames, so
            // their rounded difference is not exactly zero: skip by index
            if (same && qa == qb) continue;
            const V3<T> x = (T)rr.l[qa][1] * E1 + (T)rr.l[qa][2] * E2;
            const V3<T> y = ((T)rr.l[qb][0] * Tj[0]) + ((T)rr.l[qb][1] * Tj[1]) + ((T)rr.l[qb][2] * Tj[2]);
            const V3<T> dv = x - y;
            const T r = len(dv);
            if (!(r > T(0))) continue;
            const T w = (T)(rr.w[qa] * rr.w[qb]);
            const T rn = dot(dv, nj);
            const T t = kappa * r;
            const T gL = T(1) / r, kL = rn / (r * r * r);
            const T gR = expm1(-t) / r, kR = rn * yukawa_dl_factor(t) / (r * r * r);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T ww = w * (T)rr.l[qa][a] * (T)rr.l[qb][b];
                    sl[a][b] -= ww * aj * gL;
                    dl[a][b] -= ww * aj * kL;
                    rs[a][b] -= ww * gR;
                    rd[a][b] -= ww * kR;
                }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                for (int o = 16; o > 0; o >>= 1) {
                    sl[a][b] += __shfl_xor_sync(0xffffffffu, sl[a][b], o);
                    dl[a][b] += __shfl_xor_sync(0xffffffffu, dl[a][b], o);
                    rs[a][b] += __shfl_xor_sync(0xffffffffu, rs[a][b], o);
                    rd[a][b] += __shfl_xor_sync(0xffffffffu, rd[a][b], o);
                }
        if (lane == 0) {
            double* out = D + e * 36;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double vl = kInv4PiP * (double)ai * (double)sl[a][b];
                    const double kl = same ? 0.0 : kInv4PiP * (double)ai * (double)dl[a][b];
                    out[0 * 9 + 3 * a + b] = vl;
                    out[1 * 9 + 3 * a + b] = kl;
                    out[2 * 9 + 3 * a + b] = vl + kInv4PiP * (double)ai * (double)aj * (double)rs[a][b];
                    out[3 * 9 + 3 * a + b] =
                        same ? 0.0 : kl + kInv4PiP * (double)ai * (double)aj * (double)rd[a][b];
                }
        }
    }
}

// ---------------------------------------------------------------------------
// formulation coefficients
// ---------------------------------------------------------------------------
struct Form {
    double sL, sY;            // monopole scales of the V/K pass: qL = sL w psi, qY = sY w psi
    double r0L, r0Y;          // row 0 potential = r0L pL + r0Y pY
    double r1L, r1Y;          // row 1 part of the V/K pass (direct formulation)
    double kpL, kpY;          // row 1: kpL K'_L psi + kpY K'_Y psi
    double cw;                // row 1: cw (W_Y - W_L) phi
    double m00, m10, m11;     // identity terms: row 0 m00 M phi; row 1 m10 M phi + m11 M psi
    double kL0, kY0, vL0, vY0;   // singular blocks in row 0: (kL0 K_L + kY0 K_Y) phi + (vL0 V_L + vY0 V_Y) psi
    double kL1, kY1, vL1, vY1;   // and in row 1 (direct formulation)
    double kappa;
    int deriv;
};

static Form make_form(int formulation, double eps_in, double eps_out, double kappa) {
    const double e12 = eps_in / eps_out, e21 = eps_out / eps_in;
    Form f{};
    f.kappa = kappa;
    if (formulation == PB_FORM_DIRECT) {
        f.sL = -1; f.sY = -e12;
        f.r0L = 1; f.r0Y = 0; f.r1L = 0; f.r1Y = -1;
        f.m00 = 0.5; f.m10 = 0.5; f.m11 = 0;
        f.kL0 = 1; f.vL0 = -1; f.kY1 = -1; f.vY1 = e12;
        f.deriv = 0;
    } else if (formulation == PB_FORM_EXTERIOR) {
        f.sL = -e21; f.sY = -1;
        f.r0L = e12; f.r0Y = -1;
        f.kpL = -1; f.kpY = e12; f.cw = e12;
        f.m00 = 0.5 * (1 + e12); f.m11 = 0.5 * (1 + e12);
        f.kL0 = e12; f.kY0 = -1; f.vL0 = -1; f.vY0 = 1;
        f.deriv = 1;
    } else {
        f.sL = -1; f.sY = -e12;
        f.r0L = 1; f.r0Y = -e21;
        f.kpL = -1; f.kpY = e12; f.cw = 1;
        f.m00 = 0.5 * (1 + e21); f.m11 = 0.5 * (1 + e12);
        f.kL0 = 1; f.kY0 = -e21; f.vL0 = -1; f.vY0 = 1;
        f.deriv = 1;
    }
    return f;
}

// quadrature-point densities from the vertex values x = [phi; psi]
template <typename T>
__global__ void k_p1_dens(int nt, int nq, int nv, const int* __restrict__ F, const double* __restrict__ x,
                          const double* __restrict__ rule, const T* __restrict__ qw, const double* __restrict__ nrm,
                          const double* __restrict__ curl, double sL, double sY, int deriv, T* __restrict__ qL,
                          T* __restrict__ qY, T* __restrict__ dip, T* __restrict__ mono, T* __restrict__ c0,
                          T* __restrict__ c1, T* __restrict__ c2, T* __restrict__ n0, T* __restrict__ n1,
                          T* __restrict__ n2) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= (long long)nt * nq) return;
    const int t = (int)(b / nq), k = (int)(b % nq);
    const int f0 = F[3 * t], f1 = F[3 * t + 1], f2 = F[3 * t + 2];
    const double l0 = rule[4 * k], l1 = rule[4 * k + 1], l2 = rule[4 * k + 2];
    const double w = (double)qw[b];
    const double ph = l0 * x[f0] + l1 * x[f1] + l2 * x[f2];
    const double ps = l0 * x[nv + f0] + l1 * x[nv + f1] + l2 * x[nv + f2];
    qL[b] = (T)(sL * w * ps);
    qY[b] = (T)(sY * w * ps);
    dip[b] = (T)(w * ph);
    if (!deriv) return;
    mono[b] = (T)(w * ps);
    const double* cv = curl + 9 * (long long)t;
    const double p0 = x[f0], p1 = x[f1], p2 = x[f2];
    c0[b] = (T)(w * (p0 * cv[0] + p1 * cv[3] + p2 * cv[6]));
    c1[b] = (T)(w * (p0 * cv[1] + p1 * cv[4] + p2 * cv[7]));
    c2[b] = (T)(w * (p0 * cv[2] + p1 * cv[5] + p2 * cv[8]));
    n0[b] = (T)(w * ph * nrm[3 * t]);
    n1[b] = (T)(w * ph * nrm[3 * t + 1]);
    n2[b] = (T)(w * ph * nrm[3 * t + 2]);
}

// FMM outputs read by the local kernel
template <typename T>
struct P1Pots {
    const T *pL, *pY;                 // V/K pass
    const T *dnL, *dnY;               // K' pass (derivative formulations)
    const T *AL[3], *AY[3];           // single layers of the curl components
    const T *B[3];                    // Yukawa single layers of the phi n components
};

// Per triangle t and local vertex a: the two block rows' test integrals
// loc[t][a][0..1] (FMM part, singular corrections, identity terms).
template <typename T>
__global__ void k_p1_local(int nt, int nq, int nv, const int* __restrict__ F, const double* __restrict__ x,
                           const double* __restrict__ rule, const T* __restrict__ qw, const double* __restrict__ nrm,
                           const double* __restrict__ area, const double* __restrict__ curl, P1Pots<T> P, Form fm,
                           const int* __restrict__ adj_off, const int* __restrict__ adj_ids,
                           const int* __restrict__ adj_tr, const double* __restrict__ D, double* __restrict__ loc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int ft[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    const double* cv = curl + 9 * (long long)t;
    const double nt0 = nrm[3 * t], nt1 = nrm[3 * t + 1], nt2 = nrm[3 * t + 2];
    const T k2 = (T)(fm.kappa * fm.kappa);
    // FMM part in the arithmetic of the FMM
    T r0[3] = {0, 0, 0}, r1[3] = {0, 0, 0};
    for (int k = 0; k < nq; ++k) {
        const long long b = (long long)t * nq + k;
        const T w = qw[b];
        const T p0 = (T)fm.r0L * P.pL[b] + (T)fm.r0Y * P.pY[b];
        T p1 = (T)fm.r1L * P.pL[b] + (T)fm.r1Y * P.pY[b];
        T wc[3] = {0, 0, 0}, nb = 0;
        if (fm.deriv) {
            p1 += (T)fm.kpL * P.dnL[b] + (T)fm.kpY * P.dnY[b];
            for (int c = 0; c < 3; ++c) wc[c] = P.AY[c][b] - P.AL[c][b];
            nb = (T)nt0 * P.B[0][b] + (T)nt1 * P.B[1][b] + (T)nt2 * P.B[2][b];
        }
        for (int a = 0; a < 3; ++a) {
            const T la = (T)rule[4 * k + a];
            r0[a] += w * la * p0;
            r1[a] += w * la * p1;
            if (fm.deriv)
                r1[a] += (T)fm.cw * w * ((T)cv[3 * a] * wc[0] + (T)cv[3 * a + 1] * wc[1] + (T)cv[3 * a + 2] * wc[2] +
                                         k2 * la * nb);
        }
    }
    double R0[3], R1[3];
    for (int a = 0; a < 3; ++a) { R0[a] = (double)r0[a]; R1[a] = (double)r1[a]; }
    // singular corrections of the vertex-sharing pairs (FP64)
    for (int e = adj_off[t]; e < adj_off[t + 1]; ++e) {
        const int s = adj_ids[e];
        const int fs[3] = {F[3 * s], F[3 * s + 1], F[3 * s + 2]};
        double phs[3], pss[3];
        for (int b = 0; b < 3; ++b) { phs[b] = x[fs[b]]; pss[b] = x[nv + fs[b]]; }
        const double* De = D + (long long)e * 36;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const int ab = 3 * a + b;
                R0[a] += (fm.kL0 * De[9 + ab] + fm.kY0 * De[27 + ab]) * phs[b] +
                         (fm.vL0 * De[ab] + fm.vY0 * De[18 + ab]) * pss[b];
                R1[a] += (fm.kL1 * De[9 + ab] + fm.kY1 * De[27 + ab]) * phs[b] +
                         (fm.vL1 * De[ab] + fm.vY1 * De[18 + ab]) * pss[b];
            }
        if (fm.deriv) {
            // K' blocks: the transposed K blocks of the pair (s, t)
            const double* Dt = D + (long long)adj_tr[e] * 36;
            double sumL = 0, sumY = 0;
            for (int q = 0; q < 9; ++q) { sumL += De[q]; sumY += De[18 + q]; }
            const double* cs = curl + 9 * (long long)s;
            const double nn = nt0 * nrm[3 * s] + nt1 * nrm[3 * s + 1] + nt2 * nrm[3 * s + 2];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const int ba = 3 * b + a;
                    R1[a] += (fm.kpL * Dt[9 + ba] + fm.kpY * Dt[27 + ba]) * pss[b];
                    const double cc = cv[3 * a] * cs[3 * b] + cv[3 * a + 1] * cs[3 * b + 1] + cv[3 * a + 2] * cs[3 * b + 2];
                    R1[a] += fm.cw * (cc * (sumY - sumL) + fm.kappa * fm.kappa * nn * De[18 + 3 * a + b]) * phs[b];
                }
        }
    }
    // identity terms: the P1 mass matrix |T| (1 + delta_ab) / 12
    const double m = area[t] / 12.0;
    const double ph[3] = {x[ft[0]], x[ft[1]], x[ft[2]]};
    const double ps[3] = {x[nv + ft[0]], x[nv + ft[1]], x[nv + ft[2]]};
    const double sph = ph[0] + ph[1] + ph[2], sps = ps[0] + ps[1] + ps[2];
    for (int a = 0; a < 3; ++a) {
        const double Mph = m * (sph + ph[a]), Mps = m * (sps + ps[a]);
        R0[a] += fm.m00 * Mph;
        R1[a] += fm.m10 * Mph + fm.m11 * Mps;
        loc[6LL * t + 2 * a] = R0[a];
        loc[6LL * t + 2 * a + 1] = R1[a];
    }
}

// per vertex: the sum over its triangles in a fixed order, then the
// lumped-mass preconditioner
__global__ void k_p1_gather(int nv, const int* __restrict__ vt_off, const int* __restrict__ vt_ent,
                            const double* __restrict__ loc, const double* __restrict__ lmass, int precond,
                            double* __restrict__ y) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s0 = 0.0, s1 = 0.0;
    for (int e = vt_off[v]; e < vt_off[v + 1]; ++e) {
        const int ta = vt_ent[e];
        s0 += loc[2LL * ta];
        s1 += loc[2LL * ta + 1];
    }
    if (precond) {
        const double inv = 1.0 / lmass[v];
        s0 *= inv;
        s1 *= inv;
    }
    y[v] = s0;
    y[nv + v] = s1;
}

// Coulomb field of the charges at the quadrature points and its normal
// derivative, FP64: f = sum_k q_k / (4 pi eps |x - r_k|), df/dn_x
__global__ void k_coulomb_dn(long long np, const double* __restrict__ qp, const double* __restrict__ qn, int na,
                             const double4* __restrict__ atoms, double inv_eps, double* __restrict__ f,
                             double* __restrict__ dfdn) {
    __shared__ double4 s[256];
    const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double x = 0, y = 0, z = 0, nx = 0, ny = 0, nz = 0;
    if (a < np) {
        x = qp[3 * a]; y = qp[3 * a + 1]; z = qp[3 * a + 2];
        nx = qn[3 * a]; ny = qn[3 * a + 1]; nz = qn[3 * a + 2];
    }
    double acc = 0.0, accd = 0.0;
    for (int k0 = 0; k0 < na; k0 += 256) {
        __syncthreads();
        if (k0 + threadIdx.x < na) s[threadIdx.x] = atoms[k0 + threadIdx.x];
        __syncthreads();
        const int cnt = min(256, na - k0);
        for (int k = 0; k < cnt; ++k) {
            const double dx = x - s[k].x, dy = y - s[k].y, dz = z - s[k].z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0) {
                const double ri = rsqrt(r2);
                acc += s[k].w * ri;
                accd -= s[k].w * (dx * nx + dy * ny + dz * nz) * ri * ri * ri;
            }
        }
    }
    if (a < np) {
        f[a] = acc * kInv4PiP * inv_eps;
        dfdn[a] = accd * kInv4PiP * inv_eps;
    }
}

// right-hand side test integrals per triangle and local vertex
__global__ void k_p1_rhs_local(int nt, int nq, const double* __restrict__ rule, const double* __restrict__ qw,
                               const double* __restrict__ f, const double* __restrict__ dfdn, int deriv,
                               double* __restrict__ loc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double r0[3] = {0, 0, 0}, r1[3] = {0, 0, 0};
    for (int k = 0; k < nq; ++k) {
        const long long b = (long long)t * nq + k;
        for (int a = 0; a < 3; ++a) {
            r0[a] += qw[b] * rule[4 * k + a] * f[b];
            if (deriv) r1[a] += qw[b] * rule[4 * k + a] * dfdn[b];
        }
    }
    for (int a = 0; a < 3; ++a) {
        loc[6LL * t + 2 * a] = r0[a];
        loc[6LL * t + 2 * a + 1] = r1[a];
    }
}

// interior surface fields at the quadrature points (reaction potential):
// monopole w dphi_1/dn and dipole -w phi_1 (dphi_1/dn = s * second block)
__global__ void k_p1_reac_points(int nt, int nq, int nv, const int* __restrict__ F, const double* __restrict__ x,
                                 const double* __restrict__ rule, const double* __restrict__ qw, double s,
                                 double* __restrict__ mono, double* __restrict__ dip) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= (long long)nt * nq) return;
    const int t = (int)(b / nq), k = (int)(b % nq);
    const int f0 = F[3 * t], f1 = F[3 * t + 1], f2 = F[3 * t + 2];
    const double l0 = rule[4 * k], l1 = rule[4 * k + 1], l2 = rule[4 * k + 2];
    mono[b] = qw[b] * s * (l0 * x[nv + f0] + l1 * x[nv + f1] + l2 * x[nv + f2]);
    dip[b] = -qw[b] * (l0 * x[f0] + l1 * x[f1] + l2 * x[f2]);
}

// phi_reac at the atoms from point densities (Eq. phi_reac), FP64, atoms x
// point ranges with partial sums (summed in a fixed order)
__global__ void k_phi_reac_pts(int na, const double4* __restrict__ atoms, long long np, const double* __restrict__ qp,
                               const double* __restrict__ qn, const double* __restrict__ mono,
                               const double* __restrict__ dip, int nsplit, double* __restrict__ partial) {
    __shared__ double s_p[128][4];
    __shared__ double s_n[128][3];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int split = blockIdx.y;
    const long long b_lo = np * split / nsplit, b_hi = np * (split + 1) / nsplit;
    double px = 0, py = 0, pz = 0;
    if (k < na) { px = atoms[k].x; py = atoms[k].y; pz = atoms[k].z; }
    double acc = 0.0;
    for (long long b0 = b_lo; b0 < b_hi; b0 += 128) {
        __syncthreads();
        const long long b = b0 + threadIdx.x;
        if (b < b_hi) {
            s_p[threadIdx.x][0] = qp[3 * b];
            s_p[threadIdx.x][1] = qp[3 * b + 1];
            s_p[threadIdx.x][2] = qp[3 * b + 2];
            s_p[threadIdx.x][3] = mono[b];
            s_n[threadIdx.x][0] = dip[b] * qn[3 * b];
            s_n[threadIdx.x][1] = dip[b] * qn[3 * b + 1];
            s_n[threadIdx.x][2] = dip[b] * qn[3 * b + 2];
        }
        __syncthreads();
        const int cnt = (int)min((long long)128, b_hi - b0);
        for (int m = 0; m < cnt; ++m) {
            const double dx = px - s_p[m][0], dy = py - s_p[m][1], dz = pz - s_p[m][2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double rinv = r2 > 0 ? rsqrt(r2) : 0.0;
            acc += rinv * s_p[m][3] + (dx * s_n[m][0] + dy * s_n[m][1] + dz * s_n[m][2]) * rinv * rinv * rinv;
        }
    }
    if (k < na) partial[(long long)split * na + k] = acc;
}

__global__ void k_phi_reac_pts_sum(int na, int nsplit, const double* __restrict__ partial, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += partial[(long long)q * na + k];
    out[k] = s * kInv4PiP;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void ensure_adj_transpose(pb_mesh* M);

// vertex incidence, lumped mass, hat-function curls, regular rule
void p1_setup(pb_mesh* M) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nv = (int)M->nv;
    std::vector<double> V(3 * (size_t)nv);
    std::vector<int> F(3 * (size_t)nt);
    PB_CUDA(cudaMemcpyAsync(V.data(), M->verts.p, V.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(F.data(), M->tris.p, F.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    std::vector<int> off(nv + 1, 0), ent(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) off[F[3 * t + a] + 1]++;
    for (int v = 0; v < nv; ++v) off[v + 1] += off[v];
    std::vector<int> fill(off.begin(), off.end() - 1);
    std::vector<double> lm(nv, 0.0), cu(9 * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        const double* p[3] = {&V[3 * F[3 * t]], &V[3 * F[3 * t + 1]], &V[3 * F[3 * t + 2]]};
        const double e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
        const double e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double twoA = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int a = 0; a < 3; ++a) {
            const int v = F[3 * t + a];
            ent[fill[v]++] = 3 * t + a;          // triangles in ascending order per vertex
            lm[v] += twoA / 6.0;                 // |T| / 3
            // surface curl of the hat function: (v_{a+1} - v_{a+2}) / (2 |T|)
            const double* q1 = p[(a + 1) % 3];
            const double* q2 = p[(a + 2) % 3];
            for (int k = 0; k < 3; ++k) cu[9 * (size_t)t + 3 * a + k] = (q1[k] - q2[k]) / twoA;
        }
    }
    const RegRule rr = make_reg_rule(M->nq);
    std::vector<double> rule(4 * M->nq);
    for (int k = 0; k < M->nq; ++k) {
        for (int a = 0; a < 3; ++a) rule[4 * k + a] = rr.l[k][a];
        rule[4 * k + 3] = rr.w[k];
    }
    M->vt_off.alloc(nv + 1, st);
    M->vt_ent.alloc(ent.size(), st);
    M->lmass.alloc(nv, st);
    M->curl.alloc(cu.size(), st);
    M->rule.alloc(rule.size(), st);
    PB_CUDA(cudaMemcpyAsync(M->vt_off.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(M->vt_ent.p, ent.data(), ent.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(M->lmass.p, lm.data(), lm.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(M->curl.p, cu.data(), cu.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(M->rule.p, rule.data(), rule.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaStreamSynchronize(st));
}

static void ensure_singular_p1(pb_mesh* M, double kappa) {
    const int mode = M->ctx->singular ? M->ctx->singular : (M->nt <= kSingFp64MaxTris ? 1 : 2);
    if (M->kappa_D1 == kappa && M->sing_mode1 == mode) return;
    cudaStream_t st = M->ctx->stream;
    ensure_adj_transpose(M);
    std::vector<double> pts;
    const SingRule R = make_sing_rule(mode == 1 ? kSingDepth64 : kSingDepth32, pts);
    const RegRule rr = make_reg_rule(M->nq);
    M->D1.alloc(36 * (size_t)std::max<int64_t>(M->nadj, 1), st);
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    const int blocks = (int)std::min<long long>(div_up(M->nadj, 8), 152LL * 64);
    if (mode == 1) {
        DBuf<double> rule;
        rule.alloc(pts.size(), st);
        PB_CUDA(cudaMemcpyAsync(rule.p, pts.data(), pts.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        k_singular_p1<double><<<blocks, 256, 0, st>>>(M->nadj, (int)M->nt, M->verts.p, M->tris.p, M->adj_off.p,
                                                      M->adj_ids.p, kappa, R, rule.p, rr, M->D1.p);
        PB_CHECK_LAUNCH();
        PB_CUDA(cudaStreamSynchronize(st));
    } else {
        std::vector<float> pf(pts.begin(), pts.end());
        DBuf<float> rule;
        rule.alloc(pf.size(), st);
        PB_CUDA(cudaMemcpyAsync(rule.p, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        k_singular_p1<float><<<blocks, 256, 0, st>>>(M->nadj, (int)M->nt, M->verts.p, M->tris.p, M->adj_off.p,
                                                     M->adj_ids.p, (float)kappa, R, rule.p, rr, M->D1.p);
        PB_CHECK_LAUNCH();
        PB_CUDA(cudaStreamSynchronize(st));
    }
    M->kappa_D1 = kappa;
    M->sing_mode1 = mode;
}

void ensure_singular_p1_public(pb_mesh* M, double kappa) { ensure_singular_p1(M, kappa); }

template <typename T>
static void matvec_p1_t(pb_mesh* M, const Form& fm, const double* x, double* y, int precond) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq, nv = (int)M->nv;
    const long long np = (long long)nt * nq;
    const bool fp32 = std::is_same<T, float>::value;
    const int prec = fp32 ? PB_MIXED : PB_FP64;
    const T* qw = fp32 ? (const T*)M->qw_f.p : (const T*)M->qw_d.p;
    const T* qn = fp32 ? (const T*)M->qn_f.p : (const T*)M->qn_d.p;
    DBuf<T> qL, qY, dip, pL, pY;
    qL.alloc(np, st); qY.alloc(np, st); dip.alloc(np, st); pL.alloc(np, st); pY.alloc(np, st);
    DBuf<T> mono, c[3], nphi[3], dnL, dnY, AL[3], AY[3], B[3], junkL, junkY;
    if (fm.deriv) {
        mono.alloc(np, st); dnL.alloc(np, st); dnY.alloc(np, st); junkL.alloc(np, st); junkY.alloc(np, st);
        for (int k = 0; k < 3; ++k) {
            c[k].alloc(np, st); nphi[k].alloc(np, st);
            AL[k].alloc(np, st); AY[k].alloc(np, st); B[k].alloc(np, st);
        }
    }
    {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        k_p1_dens<T><<<div_up(np, 256), 256, 0, st>>>(nt, nq, nv, M->tris.p, x, M->rule.p, qw, M->nrm.p, M->curl.p,
                                                      fm.sL, fm.sY, fm.deriv, qL.p, qY.p, dip.p, mono.p, c[0].p,
                                                      c[1].p, c[2].p, nphi[0].p, nphi[1].p, nphi[2].p);
        PB_CHECK_LAUNCH();
    }
    fmm_apply_pair_impl(M->tree, fm.kappa, M->p, prec, qL.p, qY.p, dip.p, qn, nullptr, pL.p, pY.p, nullptr, nullptr);
    P1Pots<T> P{};
    P.pL = pL.p;
    P.pY = pY.p;
    if (fm.deriv) {
        fmm_apply_pair_impl(M->tree, fm.kappa, M->p, prec, mono.p, mono.p, nullptr, nullptr, qn, junkL.p, junkY.p,
                            dnL.p, dnY.p);
        for (int k = 0; k < 3; ++k) {
            fmm_apply_pair_impl(M->tree, fm.kappa, M->p, prec, c[k].p, c[k].p, nullptr, nullptr, nullptr, AL[k].p,
                                AY[k].p, nullptr, nullptr);
            fmm_apply_impl(M->tree, FMM_YUKAWA, fm.kappa, M->p, prec, nphi[k].p, nullptr, nullptr, nullptr, B[k].p,
                           nullptr);
            P.AL[k] = AL[k].p;
            P.AY[k] = AY[k].p;
            P.B[k] = B[k].p;
        }
        P.dnL = dnL.p;
        P.dnY = dnY.p;
    }
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    DBuf<double> loc;
    loc.alloc(6LL * nt, st);
    k_p1_local<T><<<div_up(nt, 128), 128, 0, st>>>(nt, nq, nv, M->tris.p, x, M->rule.p, qw, M->nrm.p, M->area.p,
                                                   M->curl.p, P, fm, M->adj_off.p, M->adj_ids.p, M->adj_tr.p,
                                                   M->D1.p, loc.p);
    PB_CHECK_LAUNCH();
    k_p1_gather<<<div_up(nv, 128), 128, 0, st>>>(nv, M->vt_off.p, M->vt_ent.p, loc.p, M->lmass.p, precond, y);
    PB_CHECK_LAUNCH();
}

void matvec_p1(pb_mesh* M, double eps_in, double eps_out, double kappa, int precision, int formulation,
               const double* x, double* y, int precond) {
    ensure_singular_p1(M, kappa);
    const Form fm = make_form(formulation, eps_in, eps_out, kappa);
    if (precision == PB_FP64) matvec_p1_t<double>(M, fm, x, y, precond);
    else matvec_p1_t<float>(M, fm, x, y, precond);
}

// preconditioned right-hand side of the formulation, b [2 nv]
void rhs_p1(pb_mesh* M, pb_result* R, double* b) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq, nv = (int)M->nv;
    const long long np = (long long)nt * nq;
    const bool deriv = R->formulation != PB_FORM_DIRECT;
    // the interior formulations scale the Coulomb field by 1/eps_in, the
    // exterior one by 1/eps_out (Eq. juffer, Eq. lu)
    const double eps = R->formulation == PB_FORM_EXTERIOR ? R->eps_out : R->eps_in;
    DBuf<double> f, dfdn, loc;
    f.alloc(np, st); dfdn.alloc(np, st); loc.alloc(6LL * nt, st);
    k_coulomb_dn<<<div_up(np, 256), 256, 0, st>>>(np, M->qp_d.p, M->qn_d.p, (int)R->na, (const double4*)R->atoms.p,
                                                  1.0 / eps, f.p, dfdn.p);
    PB_CHECK_LAUNCH();
    k_p1_rhs_local<<<div_up(nt, 128), 128, 0, st>>>(nt, nq, M->rule.p, M->qw_d.p, f.p, dfdn.p, deriv ? 1 : 0, loc.p);
    PB_CHECK_LAUNCH();
    k_p1_gather<<<div_up(nv, 128), 128, 0, st>>>(nv, M->vt_off.p, M->vt_ent.p, loc.p, M->lmass.p, 1, b);
    PB_CHECK_LAUNCH();
}

// Eq. phi_reac at the atoms from the P1 solution (interior fields)
void reaction_potential_p1(pb_mesh* M, pb_result* R, double* phir) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq, nv = (int)M->nv;
    const long long np = (long long)nt * nq;
    const double s = R->formulation == PB_FORM_EXTERIOR ? R->eps_out / R->eps_in : 1.0;
    DBuf<double> mono, dip;
    mono.alloc(np, st); dip.alloc(np, st);
    k_p1_reac_points<<<div_up(np, 256), 256, 0, st>>>(nt, nq, nv, M->tris.p, R->x.p, M->rule.p, M->qw_d.p, s, mono.p,
                                                      dip.p);
    PB_CHECK_LAUNCH();
    const int tiles = div_up(R->na, 128);
    const int nsplit = (int)std::max<long long>(1, std::min<long long>(div_up(2 * M->ctx->sm_count, tiles),
                                                                      div_up(np, 128)));
    DBuf<double> part;
    part.alloc((size_t)nsplit * R->na, st);
    k_phi_reac_pts<<<dim3(tiles, nsplit), 128, 0, st>>>((int)R->na, (const double4*)R->atoms.p, np, M->qp_d.p,
                                                        M->qn_d.p, mono.p, dip.p, nsplit, part.p);
    PB_CHECK_LAUNCH();
    k_phi_reac_pts_sum<<<tiles, 128, 0, st>>>((int)R->na, nsplit, part.p, phir);
    PB_CHECK_LAUNCH();
}

}  // namespace pbfmm
