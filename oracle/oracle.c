/*
 * Plain CPU oracle for the FMM-BEM hot path (test infrastructure only).
 *
 * Nothing in the product path may link or call this file: it is compiled into
 * oracle/_oracle.so and loaded only by tests/, bench.py's cpu_baseline leg and
 * __graft_entry__.smoke() to check the CUDA path.
 *
 * Everything is FP64, written as the plain definition with no blocking, no
 * fusion and no reordering beyond what the definition states.  OpenMP only
 * splits independent targets / matrix rows across cores.
 *
 * Contents
 *   or_direct_sum        direct N-body sums of the Laplace and Yukawa single-
 *                        and double-layer kernels (the sum the FMM
 *                        approximates, Eq. nbody_sum; kernels from
 *                        Eq. single_double and Eq. adj_hyp).
 *   or_tri_sl, or_tri_dl analytic inner integrals over a flat triangle of 1/r
 *                        (uniform-density potential) and of (x-y).n_y/r^3
 *                        (signed solid angle); used for the singular Galerkin
 *                        entries (Sec. "An introduction to Bempp").
 *   or_assemble_p0       dense P0 Galerkin matrices of V_L, K_L, V_Y, K_Y
 *                        (Sec. "An introduction to Bempp": A_ij = int psi_i
 *                        int g phi_j), regular product rule for disjoint
 *                        triangle pairs, semi-analytic rule for identical or
 *                        vertex-sharing pairs.
 *   or_tri_lin           linear-density versions of or_tri_sl / or_tri_dl
 *                        (one value per barycentric coordinate).
 *   or_assemble_p1       dense P1 Galerkin matrices of V, K and the
 *                        hypersingular W (Eq. adj_hyp) of both kernels for
 *                        the derivative formulations (Eq. juffer, Eq. lu).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

enum { OR_LAPLACE = 0, OR_YUKAWA = 1 };

/* ------------------------------------------------------------------ */
/* Direct sums                                                          */
/* ------------------------------------------------------------------ */

/*
 * out[i]    = sum_j  g(x_i, y_j) q_j + dg/dn_y(x_i, y_j) d_j
 * out_dn[i] = sum_j  dg/dn_x(x_i, y_j) q_j + d2g/dn_x dn_y(x_i, y_j) d_j
 * with g_L = 1/(4 pi r), g_Y = exp(-kappa r)/(4 pi r), r = |x - y|; pairs with
 * r == 0 contribute nothing.  q, d, sn, tn, out_dn may be NULL (d needs sn,
 * out_dn needs tn).  Coordinates are AoS [n][3].
 */
void or_direct_sum(int kernel, double kappa,
                   long ns, const double *sxyz, const double *q,
                   const double *d, const double *sn,
                   long nt, const double *txyz, const double *tn,
                   double *out, double *out_dn)
{
    const double k4pi = 1.0 / (4.0 * OR_PI);
    const double kap = (kernel == OR_YUKAWA) ? kappa : 0.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < nt; ++i) {
        const double x0 = txyz[3 * i], x1 = txyz[3 * i + 1], x2 = txyz[3 * i + 2];
        double nx0 = 0, nx1 = 0, nx2 = 0;
        if (tn) { nx0 = tn[3 * i]; nx1 = tn[3 * i + 1]; nx2 = tn[3 * i + 2]; }
        double acc = 0.0, acc_dn = 0.0;
        for (long j = 0; j < ns; ++j) {
            const double r0 = x0 - sxyz[3 * j];
            const double r1 = x1 - sxyz[3 * j + 1];
            const double r2 = x2 - sxyz[3 * j + 2];
            const double rr = r0 * r0 + r1 * r1 + r2 * r2;
            if (rr == 0.0) continue;
            const double r = sqrt(rr);
            const double e = exp(-kap * r);          /* 1 for Laplace */
            const double g = e * k4pi / r;
            /* f(r) = e (1 + kappa r) / (4 pi r^3): dg/dn_y = f (x-y).n_y */
            const double f = e * (1.0 + kap * r) * k4pi / (rr * r);
            if (q) acc += g * q[j];
            double rny = 0.0;
            if (d) {
                rny = r0 * sn[3 * j] + r1 * sn[3 * j + 1] + r2 * sn[3 * j + 2];
                acc += f * rny * d[j];
            }
            if (out_dn) {
                const double rnx = r0 * nx0 + r1 * nx1 + r2 * nx2;
                if (q) acc_dn += -f * rnx * q[j];
                if (d) {
                    const double nn = nx0 * sn[3 * j] + nx1 * sn[3 * j + 1] + nx2 * sn[3 * j + 2];
                    const double h = e * k4pi / (rr * r);
                    const double c3 = kap * kap * rr + 3.0 * kap * r + 3.0;
                    acc_dn += h * ((1.0 + kap * r) * nn - c3 * rnx * rny / rr) * d[j];
                }
            }
        }
        out[i] = acc;
        if (out_dn) out_dn[i] = acc_dn;
    }
}

/* ------------------------------------------------------------------ */
/* Analytic integrals over a flat triangle                              */
/* ------------------------------------------------------------------ */

static void sub3(const double *a, const double *b, double *c)
{ c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b)
{ return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* R + s computed without cancellation when s < 0: R + s = R0^2 / (R - s). */
static double r_plus_s(double R, double s, double R02)
{
    return (s >= 0.0) ? (R + s) : (R02 / (R - s));
}

/*
 * int_T 1/|x - y| dA_y for the flat triangle T = (v0, v1, v2): the potential
 * of a unit uniform surface density (closed form of Wilton et al. 1984, edge
 * by edge: P0 ln((R+ + s+)/(R- + s-)) - |d| [atan(..) - atan(..)]).
 */
double or_tri_sl(const double *x, const double *v0, const double *v1, const double *v2)
{
    double e1[3], e2[3], n[3], t[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
    const double nn = norm3(n);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    sub3(x, v0, t);
    const double d = dot3(t, n);
    const double ad = fabs(d);
    const double rho[3] = { x[0] - d * n[0], x[1] - d * n[1], x[2] - d * n[2] };
    const double *V[3] = { v0, v1, v2 };
    double phi = 0.0;
    double scale = norm3(e1) + norm3(e2);
    for (int k = 0; k < 3; ++k) {
        const double *a = V[k], *b = V[(k + 1) % 3];
        double L[3], l[3], m[3], ar[3], br[3], xa[3], xb[3];
        sub3(b, a, L);
        const double len = norm3(L);
        l[0] = L[0] / len; l[1] = L[1] / len; l[2] = L[2] / len;
        cross3(l, n, m);                  /* outward in-plane edge normal */
        sub3(a, rho, ar); sub3(b, rho, br);
        const double P0 = dot3(ar, m);
        const double sm = dot3(ar, l), sp = dot3(br, l);
        sub3(x, a, xa); sub3(x, b, xb);
        const double Rm = norm3(xa), Rp = norm3(xb);
        const double R02 = P0 * P0 + d * d;
        double term = 0.0;
        if (fabs(P0) > 1e-14 * scale) {
            term += P0 * log(r_plus_s(Rp, sp, R02) / r_plus_s(Rm, sm, R02));
            if (ad > 0.0)
                term -= ad * (atan(P0 * sp / (R02 + ad * Rp)) - atan(P0 * sm / (R02 + ad * Rm)));
        }
        phi += term;
    }
    return phi;
}

/*
 * int_T (x - y).n_y / |x - y|^3 dA_y for the flat triangle T with normal
 * n_y = (v1-v0)x(v2-v0)/|..|: the signed solid angle under which T is seen
 * from x (Van Oosterom & Strackee 1983), positive on the +n side.
 */
double or_tri_dl(const double *x, const double *v0, const double *v1, const double *v2)
{
    double a[3], b[3], c[3], bc[3];
    sub3(v0, x, a); sub3(v1, x, b); sub3(v2, x, c);
    cross3(b, c, bc);
    const double num = dot3(a, bc);
    const double la = norm3(a), lb = norm3(b), lc = norm3(c);
    const double den = la * lb * lc + dot3(a, b) * lc + dot3(a, c) * lb + dot3(b, c) * la;
    return -2.0 * atan2(num, den);
}

/* ------------------------------------------------------------------ */
/* Quadrature helpers                                                   */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
static void gauss_legendre01(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2; p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-15) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * pp * pp);   /* = 2/((1-z^2)P'^2) / 2 */
    }
}

/*
 * Collapsed (Duffy) Gauss-Legendre rule on the reference triangle:
 * lambda1 = u (1 - w), lambda2 = u w, weight 2 u W_u W_w (weights sum to 1).
 * Writes n*n barycentric pairs (l1, l2) and weights.
 */
static void triangle_rule(int n, double *l1, double *l2, double *wt)
{
    double *x = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    gauss_legendre01(n, x, w);
    int k = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j, ++k) {
            l1[k] = x[i] * (1.0 - x[j]);
            l2[k] = x[i] * x[j];
            wt[k] = 2.0 * x[i] * w[i] * w[j];
        }
    free(x); free(w);
}

/* Regular rules for the quadrature points (barycentric l0, l1, l2, weight). */
static int regular_rule(int nq, double *L /* [nq][3] */, double *W)
{
    if (nq == 1) {
        L[0] = L[1] = L[2] = 1.0 / 3.0; W[0] = 1.0; return 0;
    }
    if (nq == 3) {      /* interior degree-2 rule (2/3, 1/6, 1/6) */
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) L[3 * k + c] = (c == k) ? 2.0 / 3.0 : 1.0 / 6.0;
            W[k] = 1.0 / 3.0;
        }
        return 0;
    }
    if (nq == 6) {      /* Dunavant degree-4 rule */
        const double a = 0.445948490915965, wa = 0.223381589678011;
        const double b = 0.091576213509771, wb = 0.109951743655322;
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) L[3 * k + c] = (c == k) ? 1.0 - 2.0 * a : a;
            W[k] = wa;
            for (int c = 0; c < 3; ++c) L[3 * (k + 3) + c] = (c == k) ? 1.0 - 2.0 * b : b;
            W[k + 3] = wb;
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Dense P0 Galerkin assembly                                           */
/* ------------------------------------------------------------------ */

typedef struct { double v[3][3]; } tri_t;

static void tri_point(const tri_t *T, double l1, double l2, double *p)
{
    const double l0 = 1.0 - l1 - l2;
    for (int c = 0; c < 3; ++c) p[c] = l0 * T->v[0][c] + l1 * T->v[1][c] + l2 * T->v[2][c];
}

static double tri_area_normal(const tri_t *T, double *n)
{
    double e1[3], e2[3];
    sub3(T->v[1], T->v[0], e1); sub3(T->v[2], T->v[0], e2); cross3(e1, e2, n);
    double a = norm3(n);
    n[0] /= a; n[1] /= a; n[2] /= a;
    return 0.5 * a;
}

/*
 * Inner integrals over triangle Tj at point x (Tj's normal nj):
 *   out[0] = int g_L,  out[1] = int dg_L/dn_y,
 *   out[2] = int g_Y,  out[3] = int dg_Y/dn_y.
 * The 1/r and (x-y).n/r^3 parts are analytic; the Yukawa remainders
 * (e^{-kr}-1)/r and (x-y).n [e^{-kr}(1+kr)-1]/r^3 are bounded and use the
 * inner collapsed Gauss rule (ni points, li1/li2/wi).
 */
static void inner_integrals(const double *x, const tri_t *Tj, const double *nj, double areaj,
                            int identical, double kappa, int ni,
                            const double *li1, const double *li2, const double *wi,
                            double *out)
{
    const double k4pi = 1.0 / (4.0 * OR_PI);
    const double sl = or_tri_sl(x, Tj->v[0], Tj->v[1], Tj->v[2]);
    const double dl = identical ? 0.0 : or_tri_dl(x, Tj->v[0], Tj->v[1], Tj->v[2]);
    double rem_sl = 0.0, rem_dl = 0.0;
    for (int k = 0; k < ni; ++k) {
        double y[3];
        tri_point(Tj, li1[k], li2[k], y);
        double rv[3];
        sub3(x, y, rv);
        const double r = norm3(rv);
        const double s = kappa * r;
        double fsl, fdl;
        if (r < 1e-300) {
            fsl = -kappa; fdl = 0.0;
        } else {
            fsl = expm1(-s) / r;
            fdl = dot3(rv, nj) * (expm1(-s) + s * exp(-s)) / (r * r * r);
        }
        rem_sl += wi[k] * fsl;
        rem_dl += wi[k] * fdl;
    }
    out[0] = k4pi * sl;
    out[1] = k4pi * dl;
    out[2] = k4pi * (sl + areaj * rem_sl);
    out[3] = identical ? 0.0 : k4pi * (dl + areaj * rem_dl);
}

/* midpoint subdivision of a triangle into its 4 children */
static void split4(const tri_t *T, tri_t *ch)
{
    double m01[3], m12[3], m20[3];
    for (int c = 0; c < 3; ++c) {
        m01[c] = 0.5 * (T->v[0][c] + T->v[1][c]);
        m12[c] = 0.5 * (T->v[1][c] + T->v[2][c]);
        m20[c] = 0.5 * (T->v[2][c] + T->v[0][c]);
    }
    for (int c = 0; c < 3; ++c) {
        ch[0].v[0][c] = T->v[0][c]; ch[0].v[1][c] = m01[c];      ch[0].v[2][c] = m20[c];
        ch[1].v[0][c] = m01[c];     ch[1].v[1][c] = T->v[1][c];  ch[1].v[2][c] = m12[c];
        ch[2].v[0][c] = m20[c];     ch[2].v[1][c] = m12[c];      ch[2].v[2][c] = T->v[2][c];
        ch[3].v[0][c] = m12[c];     ch[3].v[1][c] = m20[c];      ch[3].v[2][c] = m01[c];
    }
}

/* distance from point p to segment [a, b] */
static double point_segment(const double *p, const double *a, const double *b)
{
    double ab[3], ap[3];
    sub3(b, a, ab); sub3(p, a, ap);
    double t = dot3(ap, ab) / dot3(ab, ab);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double q[3] = { a[0] + t * ab[0] - p[0], a[1] + t * ab[1] - p[1], a[2] + t * ab[2] - p[2] };
    return norm3(q);
}

/* does a vertex of S lie on an edge of Tj (where the outer integrand is
   not smooth)? */
static int touches_edges(const tri_t *S, const tri_t *Tj, double tol)
{
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 3; ++e)
            if (point_segment(S->v[a], Tj->v[e], Tj->v[(e + 1) % 3]) < tol) return 1;
    return 0;
}

typedef struct {
    const tri_t *Tj; const double *nj; double areaj; int identical; double kappa;
    int no; const double *lo1, *lo2, *wo;
    int ni; const double *li1, *li2, *wi;
    double tol;
} outer_ctx;

/* outer integral of the inner integrals over S, refined geometrically
   (graded) toward the edges of Tj up to `depth` more levels */
static void outer_graded(const outer_ctx *C, const tri_t *S, int depth, double *acc)
{
    if (depth > 0 && touches_edges(S, C->Tj, C->tol)) {
        tri_t ch[4];
        split4(S, ch);
        for (int i = 0; i < 4; ++i) outer_graded(C, &ch[i], depth - 1, acc);
        return;
    }
    double dummy[3];
    const double as = tri_area_normal(S, dummy);
    for (int k = 0; k < C->no; ++k) {
        double x[3], in[4];
        tri_point(S, C->lo1[k], C->lo2[k], x);
        inner_integrals(x, C->Tj, C->nj, C->areaj, C->identical, C->kappa, C->ni, C->li1, C->li2, C->wi, in);
        const double w = C->wo[k] * as;
        for (int m = 0; m < 4; ++m) acc[m] += w * in[m];
    }
}

/*
 * Dense P0 Galerkin matrices, row-major [nt][nt]:
 *   VL_ij = int_Ti int_Tj g_L,  KL_ij = int_Ti int_Tj dg_L/dn_y, and the
 *   Yukawa pair VY, KY.
 * Disjoint pairs (no shared vertex): product of the nq-point regular rule on
 * both triangles (the G entries of Eq. bempp_fmm_matvec).  Identical or
 * vertex-sharing pairs: outer collapsed Gauss rule (n_outer^2 points per
 * sub-triangle) of the inner integrals above on a geometrically graded
 * subdivision of Ti: sub-triangles touching an edge of Tj (where the inner
 * integral stops being smooth) are split again, L_outer levels deep.
 */
int or_assemble_p0(long nv, const double *verts, long nt, const int *tris,
                   int nq, double kappa, int L_outer, int n_outer, int n_inner,
                   double *VL, double *KL, double *VY, double *KY)
{
    double RL[6 * 3], RW[6];
    if (regular_rule(nq, RL, RW) != 0) return -1;
    (void)nv;
    tri_t *T = malloc(sizeof(tri_t) * nt);
    double *N = malloc(sizeof(double) * 3 * nt), *A = malloc(sizeof(double) * nt);
    double *Q = malloc(sizeof(double) * 3 * nq * nt);
    for (long i = 0; i < nt; ++i) {
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) T[i].v[a][c] = verts[3 * tris[3 * i + a] + c];
        A[i] = tri_area_normal(&T[i], N + 3 * i);
        for (int k = 0; k < nq; ++k)
            for (int c = 0; c < 3; ++c)
                Q[(i * nq + k) * 3 + c] = RL[3 * k] * T[i].v[0][c] + RL[3 * k + 1] * T[i].v[1][c]
                                          + RL[3 * k + 2] * T[i].v[2][c];
    }
    const int no = n_outer * n_outer, ni = n_inner * n_inner;
    double *lo1 = malloc(sizeof(double) * no), *lo2 = malloc(sizeof(double) * no), *wo = malloc(sizeof(double) * no);
    double *li1 = malloc(sizeof(double) * ni), *li2 = malloc(sizeof(double) * ni), *wi = malloc(sizeof(double) * ni);
    triangle_rule(n_outer, lo1, lo2, wo);
    triangle_rule(n_inner, li1, li2, wi);
    const double k4pi = 1.0 / (4.0 * OR_PI);

#pragma omp parallel
    {
#pragma omp for schedule(dynamic, 4)
        for (long i = 0; i < nt; ++i) {
            for (long j = 0; j < nt; ++j) {
                int shared = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        if (tris[3 * i + a] == tris[3 * j + b]) shared++;
                double vl = 0, kl = 0, vy = 0, ky = 0;
                if (shared == 0) {
                    for (int a = 0; a < nq; ++a) {
                        const double *x = Q + (i * nq + a) * 3;
                        for (int b = 0; b < nq; ++b) {
                            const double *y = Q + (j * nq + b) * 3;
                            double rv[3];
                            sub3(x, y, rv);
                            const double r = norm3(rv);
                            const double w = RW[a] * A[i] * RW[b] * A[j];
                            const double rn = dot3(rv, N + 3 * j);
                            const double e = exp(-kappa * r);
                            vl += w * k4pi / r;
                            kl += w * k4pi * rn / (r * r * r);
                            vy += w * k4pi * e / r;
                            ky += w * k4pi * e * (1.0 + kappa * r) * rn / (r * r * r);
                        }
                    }
                } else {
                    outer_ctx C = { &T[j], N + 3 * j, A[j], shared == 3, kappa,
                                    no, lo1, lo2, wo, ni, li1, li2, wi,
                                    1e-10 * sqrt(A[j]) };
                    double acc[4] = { 0, 0, 0, 0 };
                    outer_graded(&C, &T[i], L_outer, acc);
                    vl = acc[0]; kl = acc[1]; vy = acc[2]; ky = acc[3];
                }
                VL[i * nt + j] = vl; KL[i * nt + j] = kl;
                VY[i * nt + j] = vy; KY[i * nt + j] = ky;
            }
        }
    }
    free(T); free(N); free(A); free(Q);
    free(lo1); free(lo2); free(wo); free(li1); free(li2); free(wi);
    return 0;
}

/* Triangle rule export so the Python side can build points with the same rule. */
int or_regular_rule(int nq, double *L, double *W) { return regular_rule(nq, L, W); }
void or_triangle_rule(int n, double *l1, double *l2, double *w) { triangle_rule(n, l1, l2, w); }

/* ------------------------------------------------------------------ */
/* P1 (continuous piecewise-linear) Galerkin assembly                   */
/* ------------------------------------------------------------------ */

/*
 * Linear-density inner integrals over the flat triangle T = (v0, v1, v2)
 * at the point x, for the three barycentric coordinates lambda_b of T:
 *   sl3[b] = int_T lambda_b(y) / |x - y| dA_y
 *   dl3[b] = int_T lambda_b(y) (x - y).n / |x - y|^3 dA_y
 * Written around the projection p of x on T's plane (height h = (x-v0).n):
 * lambda_b(y) = lambda_b(p) + grad lambda_b . (y - p), so each integral is
 * lambda_b(p) times the uniform-density one (or_tri_sl, or_tri_dl) plus
 * grad lambda_b dotted with a vector moment, turned into edge integrals by
 * the divergence theorem in the plane (R = |x - y|, m_e the outward in-plane
 * normal of edge e):
 *   int_T (y - p)/R dA     =  sum_e m_e int_e R ds
 *   int_T (y - p) h/R^3 dA = -h sum_e m_e int_e 1/R ds
 * with int R ds = (s R + R0^2 ln(s + R))/2 and int 1/R ds = ln(s + R)
 * along the edge (s the coordinate along it from the foot of p, R0 the
 * distance of x from the edge line).
 */
void or_tri_lin(const double *x, const double *v0, const double *v1, const double *v2, double *sl3, double *dl3)
{
    double e1[3], e2[3], n[3], t[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2); cross3(e1, e2, n);
    const double twoA = norm3(n);
    n[0] /= twoA; n[1] /= twoA; n[2] /= twoA;
    sub3(x, v0, t);
    const double h = dot3(t, n);
    const double p[3] = { x[0] - h * n[0], x[1] - h * n[1], x[2] - h * n[2] };
    const double *V[3] = { v0, v1, v2 };
    const double scale = norm3(e1) + norm3(e2);
    /* barycentric coordinates of p and gradients of lambda_b (in-plane) */
    double lam[3], grad[3][3];
    for (int b = 0; b < 3; ++b) {
        const double *a = V[(b + 1) % 3], *c = V[(b + 2) % 3];
        double ac[3], ap[3], cr[3];
        sub3(c, a, ac); sub3(p, a, ap);
        cross3(ac, ap, cr);
        lam[b] = dot3(cr, n) / twoA;           /* signed area of (a, c, p) / area of T */
        cross3(n, ac, grad[b]);                /* n x (v_{b+2} - v_{b+1}) / (2A) */
        for (int k = 0; k < 3; ++k) grad[b][k] /= twoA;
    }
    /* vector moments I1 = int (y - p)/R dA, J1 = int (y - p)/R^3 dA */
    double I1[3] = { 0, 0, 0 }, J1[3] = { 0, 0, 0 };
    for (int k = 0; k < 3; ++k) {
        const double *a = V[k], *b = V[(k + 1) % 3];
        double L[3], l[3], m[3], ap[3], bp[3], xa[3], xb[3];
        sub3(b, a, L);
        const double len = norm3(L);
        l[0] = L[0] / len; l[1] = L[1] / len; l[2] = L[2] / len;
        cross3(l, n, m);                        /* outward in-plane edge normal */
        sub3(a, p, ap); sub3(b, p, bp);
        const double P0 = dot3(ap, m);
        const double sm = dot3(ap, l), sp = dot3(bp, l);
        sub3(x, a, xa); sub3(x, b, xb);
        const double Rm = norm3(xa), Rp = norm3(xb);
        const double R02 = P0 * P0 + h * h;
        double intR = 0.5 * (sp * Rp - sm * Rm);
        double intInvR = 0.0;
        if (R02 > 1e-28 * scale * scale) {
            const double lg = log(r_plus_s(Rp, sp, R02) / r_plus_s(Rm, sm, R02));
            intR += 0.5 * R02 * lg;
            intInvR = lg;
        }
        for (int c = 0; c < 3; ++c) {
            I1[c] += m[c] * intR;
            J1[c] += m[c] * intInvR;
        }
    }
    const double sl0 = or_tri_sl(x, v0, v1, v2);
    const double dl0 = (fabs(h) > 0.0) ? or_tri_dl(x, v0, v1, v2) : 0.0;
    for (int b = 0; b < 3; ++b) {
        sl3[b] = lam[b] * sl0 + dot3(grad[b], I1);
        dl3[b] = lam[b] * dl0 - h * dot3(grad[b], J1);
    }
}

/* surface curl of the hat function of local vertex a on triangle T:
   n x grad lambda_a = (v_{a+1} - v_{a+2}) / (2 |T|) */
static void hat_curl(const tri_t *T, double area, int a, double *c)
{
    const double *p = T->v[(a + 1) % 3], *q = T->v[(a + 2) % 3];
    for (int k = 0; k < 3; ++k) c[k] = (p[k] - q[k]) / (2.0 * area);
}

/* inner linear-density integrals of the four kernels at x over Tj:
   out[op][b], op = V_L, K_L, V_Y, K_Y (including 1/(4 pi)) */
static void inner_lin(const double *x, const tri_t *Tj, const double *nj, double areaj, int identical,
                      double kappa, int ni, const double *li1, const double *li2, const double *wi,
                      double out[4][3])
{
    const double k4pi = 1.0 / (4.0 * OR_PI);
    double sl[3], dl[3];
    or_tri_lin(x, Tj->v[0], Tj->v[1], Tj->v[2], sl, dl);
    if (identical) dl[0] = dl[1] = dl[2] = 0.0;
    double rs[3] = { 0, 0, 0 }, rd[3] = { 0, 0, 0 };
    for (int k = 0; k < ni; ++k) {
        double y[3], rv[3];
        tri_point(Tj, li1[k], li2[k], y);
        sub3(x, y, rv);
        const double r = norm3(rv);
        const double s = kappa * r;
        double fsl, fdl;
        if (r < 1e-300) {
            fsl = -kappa; fdl = 0.0;
        } else {
            fsl = expm1(-s) / r;
            fdl = dot3(rv, nj) * (expm1(-s) + s * exp(-s)) / (r * r * r);
        }
        const double lb[3] = { 1.0 - li1[k] - li2[k], li1[k], li2[k] };
        for (int b = 0; b < 3; ++b) {
            rs[b] += wi[k] * lb[b] * fsl;
            rd[b] += wi[k] * lb[b] * fdl;
        }
    }
    for (int b = 0; b < 3; ++b) {
        out[0][b] = k4pi * sl[b];
        out[1][b] = k4pi * dl[b];
        out[2][b] = k4pi * (sl[b] + areaj * rs[b]);
        out[3][b] = identical ? 0.0 : k4pi * (dl[b] + areaj * rd[b]);
    }
}

typedef struct {
    const tri_t *Tj; const double *nj; double areaj; int identical; double kappa;
    int no; const double *lo1, *lo2, *wo;
    int ni; const double *li1, *li2, *wi;
    double tol;
} outer_lin_ctx;

/* acc[op][a][b] += int_S lambda_a^{Ti}(x) inner_lin(x)[op][b]; S a piece of
   Ti (graded toward the edges of Tj), Ti's barycentric coordinates of x
   from (Ti, S) */
static void outer_graded_lin(const outer_lin_ctx *C, const tri_t *Ti, const tri_t *S, int depth,
                             double acc[4][3][3])
{
    if (depth > 0 && touches_edges(S, C->Tj, C->tol)) {
        tri_t ch[4];
        split4(S, ch);
        for (int i = 0; i < 4; ++i) outer_graded_lin(C, Ti, &ch[i], depth - 1, acc);
        return;
    }
    double ni_[3];
    const double as = tri_area_normal(S, ni_);
    const double ai = tri_area_normal(Ti, ni_);
    for (int k = 0; k < C->no; ++k) {
        double x[3], in[4][3];
        tri_point(S, C->lo1[k], C->lo2[k], x);
        inner_lin(x, C->Tj, C->nj, C->areaj, C->identical, C->kappa, C->ni, C->li1, C->li2, C->wi, in);
        /* barycentric coordinates of x in Ti (areas of the sub-triangles) */
        double la[3];
        for (int a = 0; a < 3; ++a) {
            double u[3], w[3], cr[3];
            sub3(Ti->v[(a + 1) % 3], x, u); sub3(Ti->v[(a + 2) % 3], x, w);
            cross3(u, w, cr);
            la[a] = dot3(cr, ni_) / (2.0 * ai);
        }
        const double wgt = C->wo[k] * as;
        for (int op = 0; op < 4; ++op)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc[op][a][b] += wgt * la[a] * in[op][b];
    }
}

/*
 * Dense P1 Galerkin matrices [nv][nv], row = test vertex, column = trial
 * vertex (hat functions phi_i):
 *   VL_ij = int int phi_i(x) g_L phi_j(y),  KL_ij = ... dg_L/dn_y ...,
 *   VY, KY the Yukawa pair,
 *   WL_ij = int int g_L curl phi_i(x) . curl phi_j(y)
 *   WY_ij = int int g_Y [curl phi_i . curl phi_j + kappa^2 (n_x.n_y) phi_i phi_j]
 * (the hypersingular operators of Eq. adj_hyp in the integrated-by-parts
 * form that holds for continuous trial and test functions on a closed
 * surface; curl phi = n x grad phi is constant on each triangle).  Triangle
 * pairs without a shared vertex use the product of the nq-point regular rule;
 * identical or vertex-sharing pairs the graded outer rule of the analytic
 * linear-density inner integrals (as or_assemble_p0).  One row per thread:
 * every (Ti, Tj) block is computed once for each vertex of Ti.
 */
int or_assemble_p1(long nv, const double *verts, long nt, const int *tris,
                   int nq, double kappa, int L_outer, int n_outer, int n_inner,
                   double *VL, double *KL, double *VY, double *KY, double *WL, double *WY)
{
    double RL[6 * 3], RW[6];
    if (regular_rule(nq, RL, RW) != 0) return -1;
    tri_t *T = malloc(sizeof(tri_t) * nt);
    double *N = malloc(sizeof(double) * 3 * nt), *A = malloc(sizeof(double) * nt);
    double *Q = malloc(sizeof(double) * 3 * nq * nt);
    for (long i = 0; i < nt; ++i) {
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) T[i].v[a][c] = verts[3 * tris[3 * i + a] + c];
        A[i] = tri_area_normal(&T[i], N + 3 * i);
        for (int k = 0; k < nq; ++k)
            for (int c = 0; c < 3; ++c)
                Q[(i * nq + k) * 3 + c] = RL[3 * k] * T[i].v[0][c] + RL[3 * k + 1] * T[i].v[1][c]
                                          + RL[3 * k + 2] * T[i].v[2][c];
    }
    /* vertex -> incident triangles */
    long *vcnt = calloc((size_t)nv + 1, sizeof(long));
    for (long i = 0; i < nt; ++i)
        for (int a = 0; a < 3; ++a) vcnt[tris[3 * i + a] + 1]++;
    for (long v = 0; v < nv; ++v) vcnt[v + 1] += vcnt[v];
    long *vtri = malloc(sizeof(long) * 3 * (size_t)nt), *vfill = calloc((size_t)nv, sizeof(long));
    for (long i = 0; i < nt; ++i)
        for (int a = 0; a < 3; ++a) {
            const long v = tris[3 * i + a];
            vtri[vcnt[v] + vfill[v]++] = i;
        }
    const int no = n_outer * n_outer, ni = n_inner * n_inner;
    double *lo1 = malloc(sizeof(double) * no), *lo2 = malloc(sizeof(double) * no), *wo = malloc(sizeof(double) * no);
    double *li1 = malloc(sizeof(double) * ni), *li2 = malloc(sizeof(double) * ni), *wi = malloc(sizeof(double) * ni);
    triangle_rule(n_outer, lo1, lo2, wo);
    triangle_rule(n_inner, li1, li2, wi);
    const double k4pi = 1.0 / (4.0 * OR_PI);
    memset(VL, 0, sizeof(double) * nv * nv); memset(KL, 0, sizeof(double) * nv * nv);
    memset(VY, 0, sizeof(double) * nv * nv); memset(KY, 0, sizeof(double) * nv * nv);
    memset(WL, 0, sizeof(double) * nv * nv); memset(WY, 0, sizeof(double) * nv * nv);

#pragma omp parallel for schedule(dynamic, 2)
    for (long v = 0; v < nv; ++v) {
        for (long e = vcnt[v]; e < vcnt[v + 1]; ++e) {
            const long i = vtri[e];
            int a = 0;
            while (tris[3 * i + a] != v) ++a;
            double ca[3];
            hat_curl(&T[i], A[i], a, ca);
            for (long j = 0; j < nt; ++j) {
                int shared = 0;
                for (int s = 0; s < 3; ++s)
                    for (int t = 0; t < 3; ++t)
                        if (tris[3 * i + s] == tris[3 * j + t]) shared++;
                double blk[4][3][3];
                memset(blk, 0, sizeof(blk));
                if (shared == 0) {
                    for (int qa = 0; qa < nq; ++qa) {
                        const double *x = Q + (i * nq + qa) * 3;
                        for (int qb = 0; qb < nq; ++qb) {
                            const double *y = Q + (j * nq + qb) * 3;
                            double rv[3];
                            sub3(x, y, rv);
                            const double r = norm3(rv);
                            const double w = RW[qa] * A[i] * RW[qb] * A[j];
                            const double rn = dot3(rv, N + 3 * j);
                            const double ek = exp(-kappa * r);
                            const double kk[4] = { k4pi / r, k4pi * rn / (r * r * r), k4pi * ek / r,
                                                   k4pi * ek * (1.0 + kappa * r) * rn / (r * r * r) };
                            for (int op = 0; op < 4; ++op)
                                for (int aa = 0; aa < 3; ++aa)
                                    for (int b = 0; b < 3; ++b)
                                        blk[op][aa][b] += w * RL[3 * qa + aa] * RL[3 * qb + b] * kk[op];
                        }
                    }
                } else {
                    outer_lin_ctx C = { &T[j], N + 3 * j, A[j], shared == 3, kappa,
                                        no, lo1, lo2, wo, ni, li1, li2, wi, 1e-10 * sqrt(A[j]) };
                    outer_graded_lin(&C, &T[i], &T[i], L_outer, blk);
                }
                /* P0 sums of the single layers: the curl-curl term */
                double vl0 = 0.0, vy0 = 0.0;
                for (int aa = 0; aa < 3; ++aa)
                    for (int b = 0; b < 3; ++b) { vl0 += blk[0][aa][b]; vy0 += blk[2][aa][b]; }
                const double nn = dot3(N + 3 * i, N + 3 * j);
                for (int b = 0; b < 3; ++b) {
                    const long col = tris[3 * j + b];
                    double cb[3];
                    hat_curl(&T[j], A[j], b, cb);
                    const double cc = dot3(ca, cb);
                    VL[v * nv + col] += blk[0][a][b];
                    KL[v * nv + col] += blk[1][a][b];
                    VY[v * nv + col] += blk[2][a][b];
                    KY[v * nv + col] += blk[3][a][b];
                    WL[v * nv + col] += cc * vl0;
                    WY[v * nv + col] += cc * vy0 + kappa * kappa * nn * blk[2][a][b];
                }
            }
        }
    }
    free(T); free(N); free(A); free(Q); free(vcnt); free(vtri); free(vfill);
    free(lo1); free(lo2); free(wo); free(li1); free(li2); free(wi);
    return 0;
}

/*
 * P1 block of one triangle pair (test triangle Ti = vertices ti[0..2],
 * trial Tj), for op = V_L, K_L, V_Y, K_Y and local test / trial vertices a,
 * b: out[op*9 + 3a + b] = int_Ti lambda_a int_Tj lambda_b k.  With
 * `minus_regular`, the same block under the nq x nq regular product rule
 * (pairs at distance 0 excluded) is subtracted: what the singular quadrature
 * adds to a point-sum (FMM) evaluation of the pair.  Identical or
 * vertex-sharing pairs use the graded outer rule of or_assemble_p1.
 */
int or_pair_p1(const double *verts, const int *ti, const int *tj, int nq, double kappa,
               int L_outer, int n_outer, int n_inner, int minus_regular, double *out)
{
    double RL[6 * 3], RW[6];
    if (regular_rule(nq, RL, RW) != 0) return -1;
    tri_t Ti, Tj;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) { Ti.v[a][c] = verts[3 * ti[a] + c]; Tj.v[a][c] = verts[3 * tj[a] + c]; }
    double ni[3], nj[3];
    const double ai = tri_area_normal(&Ti, ni), aj = tri_area_normal(&Tj, nj);
    int shared = 0;
    for (int s = 0; s < 3; ++s)
        for (int t = 0; t < 3; ++t)
            if (ti[s] == tj[t]) shared++;
    const int no = n_outer * n_outer, ni_ = n_inner * n_inner;
    double lo1[64], lo2[64], wo[64], li1[64], li2[64], wi[64];
    if (no > 64 || ni_ > 64) return -1;
    triangle_rule(n_outer, lo1, lo2, wo);
    triangle_rule(n_inner, li1, li2, wi);
    double blk[4][3][3];
    memset(blk, 0, sizeof(blk));
    outer_lin_ctx C = { &Tj, nj, aj, shared == 3, kappa, no, lo1, lo2, wo, ni_, li1, li2, wi, 1e-10 * sqrt(aj) };
    outer_graded_lin(&C, &Ti, &Ti, shared ? L_outer : 0, blk);
    if (minus_regular) {
        const double k4pi = 1.0 / (4.0 * OR_PI);
        for (int qa = 0; qa < nq; ++qa) {
            double x[3], y[3], rv[3];
            for (int c = 0; c < 3; ++c)
                x[c] = RL[3 * qa] * Ti.v[0][c] + RL[3 * qa + 1] * Ti.v[1][c] + RL[3 * qa + 2] * Ti.v[2][c];
            for (int qb = 0; qb < nq; ++qb) {
                for (int c = 0; c < 3; ++c)
                    y[c] = RL[3 * qb] * Tj.v[0][c] + RL[3 * qb + 1] * Tj.v[1][c] + RL[3 * qb + 2] * Tj.v[2][c];
                sub3(x, y, rv);
                const double r = norm3(rv);
                if (r == 0.0) continue;
                const double w = RW[qa] * ai * RW[qb] * aj;
                const double rn = dot3(rv, nj);
                const double ek = exp(-kappa * r);
                const double kk[4] = { k4pi / r, k4pi * rn / (r * r * r), k4pi * ek / r,
                                       k4pi * ek * (1.0 + kappa * r) * rn / (r * r * r) };
                for (int op = 0; op < 4; ++op)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) blk[op][a][b] -= w * RL[3 * qa + a] * RL[3 * qb + b] * kk[op];
            }
        }
    }
    for (int op = 0; op < 4; ++op)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) out[op * 9 + 3 * a + b] = blk[op][a][b];
    return 0;
}

/*
 * P0 corrections of the given triangle pairs (i[k], j[k]), k < npairs:
 * out[4k + op] = (semi-analytic Galerkin entry of Ti x Tj) - (the same entry
 * under the nq x nq regular product rule, pairs at distance 0 excluded),
 * op = V_L, K_L, V_Y, K_Y.  The entries are those of or_assemble_p0 (graded
 * outer rule L_outer levels deep for vertex-sharing pairs).  For a
 * matrix-free mat-vec: the point sums hold the regular-rule part of every
 * pair, the corrections swap it for the singular value.  OpenMP over pairs.
 */
int or_corrections_p0(long nv, const double *verts, long nt, const int *tris, long npairs, const long *pi,
                      const long *pj, int nq, double kappa, int L_outer, int n_outer, int n_inner, double *out)
{
    double RL[6 * 3], RW[6];
    if (regular_rule(nq, RL, RW) != 0) return -1;
    (void)nv; (void)nt;
    const int no = n_outer * n_outer, ni = n_inner * n_inner;
    double lo1[64], lo2[64], wo[64], li1[64], li2[64], wi[64];
    if (no > 64 || ni > 64) return -1;
    triangle_rule(n_outer, lo1, lo2, wo);
    triangle_rule(n_inner, li1, li2, wi);
    const double k4pi = 1.0 / (4.0 * OR_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < npairs; ++k) {
        const long i = pi[k], j = pj[k];
        tri_t Ti, Tj;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                Ti.v[a][c] = verts[3 * tris[3 * i + a] + c];
                Tj.v[a][c] = verts[3 * tris[3 * j + a] + c];
            }
        double ni_[3], nj[3];
        const double ai = tri_area_normal(&Ti, ni_), aj = tri_area_normal(&Tj, nj);
        int shared = 0;
        for (int s = 0; s < 3; ++s)
            for (int t = 0; t < 3; ++t)
                if (tris[3 * i + s] == tris[3 * j + t]) shared++;
        double acc[4] = { 0, 0, 0, 0 };
        outer_ctx C = { &Tj, nj, aj, shared == 3, kappa, no, lo1, lo2, wo, ni, li1, li2, wi,
                        1e-10 * sqrt(aj) };
        outer_graded(&C, &Ti, shared ? L_outer : 0, acc);
        for (int qa = 0; qa < nq; ++qa) {
            double x[3], y[3], rv[3];
            for (int c = 0; c < 3; ++c)
                x[c] = RL[3 * qa] * Ti.v[0][c] + RL[3 * qa + 1] * Ti.v[1][c] + RL[3 * qa + 2] * Ti.v[2][c];
            for (int qb = 0; qb < nq; ++qb) {
                for (int c = 0; c < 3; ++c)
                    y[c] = RL[3 * qb] * Tj.v[0][c] + RL[3 * qb + 1] * Tj.v[1][c] + RL[3 * qb + 2] * Tj.v[2][c];
                sub3(x, y, rv);
                const double r = norm3(rv);
                if (r == 0.0) continue;
                const double w = RW[qa] * ai * RW[qb] * aj;
                const double rn = dot3(rv, nj);
                const double ek = exp(-kappa * r);
                acc[0] -= w * k4pi / r;
                acc[1] -= w * k4pi * rn / (r * r * r);
                acc[2] -= w * k4pi * ek / r;
                acc[3] -= w * k4pi * ek * (1.0 + kappa * r) * rn / (r * r * r);
            }
        }
        for (int op = 0; op < 4; ++op) out[4 * k + op] = acc[op];
    }
    return 0;
}
