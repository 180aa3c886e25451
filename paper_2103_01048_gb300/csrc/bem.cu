// Galerkin BEM of the direct formulation on the GPU.
//
// Mat-vec (Eq. bempp_fmm_matvec): A x = P2^T (G - C) P1 x + S x, with
//   P1  quadrature-point densities from the P0 coefficients,
//   G   applied by one Laplace and one Yukawa FMM pass that carry the
//       single-layer (monopole) and double-layer (dipole) sources together,
//   C   the G entries of identical / vertex-sharing triangle pairs, removed
//       on the fly,
//   S   the singular Galerkin entries of those pairs (assembled once),
// combined into the 2x2 block system of Eq. direct, then the block-diagonal
// preconditioner (per element the 2x2 matrix of diagonal entries).
// Solve: full GMRES in FP64 (classical Gram-Schmidt twice), Givens rotations
// on the device.  RHS (charge -> surface), reaction potential (Eq. phi_reac,
// surface -> charge) and the FP64 energy sum (Eq. energy).
#include "bem.cuh"
#include "bem_quad.cuh"
#include <cub/cub.cuh>
#include <algorithm>
#include <cmath>
#include <functional>

namespace pbfmm {

void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn);
void fmm_apply_pair_impl(fmm_tree* Tr, double kappa, int p, int precision, const void* qL, const void* qY,
                         const void* dip, const void* src_n, const void* tgt_n, void* outL, void* outY, void* dnL,
                         void* dnY);
void build_tree(fmm_tree* T, const float* src, const float* tgt);

constexpr double kInv4PiB = 0.07957747154594767;
constexpr double kKcal = 332.0637;     // kcal A / (mol e^2)

// ---------------------------------------------------------------------------
// geometry, quadrature points
// ---------------------------------------------------------------------------
__global__ void k_geometry(int nt, int nv, const double* __restrict__ V, const int* __restrict__ F, int nq,
                           const double* __restrict__ rl, const double* __restrict__ rw, double* nrm, double* area,
                           double* qp_d, double* qn_d, double* qw_d, float* qp_f, float* qn_f, float* qw_f, int* bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int f0 = F[3 * i], f1 = F[3 * i + 1], f2 = F[3 * i + 2];
    if (f0 < 0 || f1 < 0 || f2 < 0 || f0 >= nv || f1 >= nv || f2 >= nv || f0 == f1 || f1 == f2 || f0 == f2) {
        atomicExch(bad, 1);
        f0 = f1 = f2 = 0;
    }
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) { a[k] = V[3 * f0 + k]; b[k] = V[3 * f1 + k]; c[k] = V[3 * f2 + k]; }
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double inv = nn > 0 ? 1.0 / nn : 0.0;
    for (int k = 0; k < 3; ++k) nrm[3 * i + k] = n[k] * inv;
    area[i] = 0.5 * nn;
    for (int q = 0; q < nq; ++q) {
        long long pidx = (long long)i * nq + q;
        for (int k = 0; k < 3; ++k) {
            double x = rl[3 * q] * a[k] + rl[3 * q + 1] * b[k] + rl[3 * q + 2] * c[k];
            qp_d[3 * pidx + k] = x;
            qp_f[3 * pidx + k] = (float)x;
            qn_d[3 * pidx + k] = n[k] * inv;
            qn_f[3 * pidx + k] = (float)(n[k] * inv);
        }
        qw_d[pidx] = rw[q] * 0.5 * nn;
        qw_f[pidx] = (float)(rw[q] * 0.5 * nn);
    }
}

// vertex -> triangle incidence
__global__ void k_vcount(int nt, const int* F, int* cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    for (int k = 0; k < 3; ++k) atomicAdd(cnt + F[3 * i + k], 1);
}
__global__ void k_vfill(int nt, const int* F, const int* off, int* cur, int* ids) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    for (int k = 0; k < 3; ++k) {
        int v = F[3 * i + k];
        ids[off[v] + atomicAdd(cur + v, 1)] = i;
    }
}

constexpr int kAdjCap = 128;

// triangles sharing a vertex with triangle i (self included), ascending;
// pass 0 counts, pass 1 writes
__global__ void k_adjacency(int nt, const int* F, const int* voff, const int* vids, int pass, int* cnt,
                            const int* off, int* ids, int* overflow) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int buf[kAdjCap];
    int n = 0;
    for (int k = 0; k < 3; ++k) {
        int v = F[3 * i + k];
        for (int e = voff[v]; e < voff[v + 1]; ++e) {
            int t = vids[e];
            bool dup = false;
            for (int m = 0; m < n; ++m) dup |= (buf[m] == t);
            if (!dup) {
                if (n >= kAdjCap) { atomicExch(overflow, 1); break; }
                buf[n++] = t;
            }
        }
    }
    for (int a = 1; a < n; ++a) {
        int v = buf[a], b = a - 1;
        while (b >= 0 && buf[b] > v) { buf[b + 1] = buf[b]; --b; }
        buf[b + 1] = v;
    }
    if (pass == 0) cnt[i] = n;
    else for (int m = 0; m < n; ++m) ids[off[i] + m] = buf[m];
}

template <typename T>
__global__ void __launch_bounds__(256) k_singular(long long nadj, int nt, const double* __restrict__ V,
                                                  const int* __restrict__ F, const int* __restrict__ adj_off,
                                                  const int* __restrict__ adj_ids, T kappa, SingRule R,
                                                  const T* __restrict__ pts, double* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
    for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < nadj; e += nw) {
        int lo = 0, hi = nt;               // row: adj_off[lo] <= e < adj_off[lo + 1]
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
        else if (shared == 2) pat = mask == 3 ? 1 : (mask == 6 ? 2 : 3);   // {0,1}, {1,2}, {2,0}
        else if (shared == 1) pat = 4 + (mask == 1 ? 0 : (mask == 2 ? 1 : 2));
        else pat = 7;
        // local frame at v0 of T_i: differences in FP64, then T
        const double ox = V[3 * fi[0]], oy = V[3 * fi[0] + 1], oz = V[3 * fi[0] + 2];
        auto rel = [&](int v) -> V3<T> {
            return {(T)(V[3 * v] - ox), (T)(V[3 * v + 1] - oy), (T)(V[3 * v + 2] - oz)};
        };
        const V3<T> E1 = rel(fi[1]), E2 = rel(fi[2]);
        V3<T> Tj[3] = {rel(fj[0]), rel(fj[1]), rel(fj[2])};
        V3<T> nj = cross(Tj[1] - Tj[0], Tj[2] - Tj[0]);
        const T aj = T(0.5) * len(nj);
        nj = (T(1) / (T(2) * aj)) * nj;
        const T ai = T(0.5) * len(cross(E1, E2));
        const bool same = pat == 0;
        T vl = 0, kl = 0, rs = 0, rd = 0;
        for (int k = R.s_off[pat] + lane; k < R.s_off[pat + 1]; k += 32) {
            const T l1 = pts[3 * k], l2 = pts[3 * k + 1], w = pts[3 * k + 2];
            const V3<T> x = l1 * E1 + l2 * E2;
            vl += w * pot_uniform_triangle(x, Tj);
            if (!same) kl += w * solid_angle(x, Tj);
        }
        if (kappa > 0) {
            for (int k = R.r_off[pat] + lane; k < R.r_off[pat + 1]; k += 32) {
                const T l1 = pts[3 * k], l2 = pts[3 * k + 1], w = pts[3 * k + 2];
                const V3<T> x = l1 * E1 + l2 * E2;
                T s = 0, d = 0;
                for (int m = 0; m < kSingInnerN * kSingInnerN; ++m) {
                    const T m1 = pts[3 * (R.in_off + m)], m2 = pts[3 * (R.in_off + m) + 1];
                    const T wm = pts[3 * (R.in_off + m) + 2];
                    const V3<T> y = ((T(1) - m1 - m2) * Tj[0]) + (m1 * Tj[1]) + (m2 * Tj[2]);
                    const V3<T> dv = x - y;
                    const T r = len(dv);
                    if (r > (T)1e-30) {
                        const T t = kappa * r;
                        s += wm * expm1(-t) / r;
                        if (!same) d += wm * dot(dv, nj) * yukawa_dl_factor(t) / (r * r * r);
                    } else {
                        s -= wm * kappa;
                    }
                }
                rs += w * s;
                rd += w * d;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            vl += __shfl_xor_sync(0xffffffffu, vl, o);
            kl += __shfl_xor_sync(0xffffffffu, kl, o);
            rs += __shfl_xor_sync(0xffffffffu, rs, o);
            rd += __shfl_xor_sync(0xffffffffu, rd, o);
        }
        if (lane == 0) {
            const double VLi = (double)ai * (double)vl, KLi = same ? 0.0 : (double)ai * (double)kl;
            S[4 * e + 0] = kInv4PiB * VLi;
            S[4 * e + 1] = kInv4PiB * KLi;
            S[4 * e + 2] = kInv4PiB * (VLi + (double)ai * (double)aj * (double)rs);
            S[4 * e + 3] = kInv4PiB * (same ? 0.0 : KLi + (double)ai * (double)aj * (double)rd);
        }
    }
}

__global__ void k_to_float(long long n, const double* a, float* b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// mat-vec pieces
// ---------------------------------------------------------------------------
// P1: quadrature-point densities of both FMM passes from x = [phi; dphi]
//   Laplace: q = -w dphi, d = w phi;  Yukawa: q = (eps1/eps2) w dphi, d = -w phi.
// The paired apply shares the dipole density, so the Yukawa pass takes
// (-q, -d) = ((eps1/eps2) qL, dL) and its potential is negated in the combine.
template <typename T>
__global__ void k_p1(int nt, int nq, const double* __restrict__ x, const T* __restrict__ qw, double er,
                     T* qL, T* dL, T* qYn) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= (long long)nt * nq) return;
    int i = (int)(a / nq);
    T w = qw[a];
    T phi = (T)x[i], dphi = (T)x[nt + i];
    qL[a] = -w * dphi;
    dL[a] = w * phi;
    qYn[a] = -(T)er * w * dphi;
}

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <typename T> __device__ __forceinline__ T ex(T x);
template <> __device__ __forceinline__ float ex<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double ex<double>(double x) { return exp(x); }

// P2^T (pot - C) + S x + M/2 phi, then the 2x2 block-diagonal preconditioner
// (if precond).  One thread per triangle.
template <typename T>
__global__ void k_combine(int nt, int nq, const double* __restrict__ x, const T* __restrict__ potL,
                          const T* __restrict__ potYn, const T* __restrict__ qp, const T* __restrict__ qn,
                          const T* __restrict__ qw, const int* __restrict__ adj_off, const int* __restrict__ adj_ids,
                          const T* __restrict__ S, const double* __restrict__ area, double er, double kappa_d,
                          int precond, double* __restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const T kappa = (T)kappa_d;
    const T c4 = (T)kInv4PiB;
    T r1 = 0, r2 = 0;
    for (int a = 0; a < nq; ++a) {
        long long pa = (long long)i * nq + a;
        T wa = qw[pa];
        T xa = qp[3 * pa], ya = qp[3 * pa + 1], za = qp[3 * pa + 2];
        T cL = 0, cY = 0;      // C: G entries of adjacent pairs, removed
        for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
            int j = adj_ids[e];
            T phi = (T)x[j], dphi = (T)x[nt + j];
            for (int b = 0; b < nq; ++b) {
                long long pb = (long long)j * nq + b;
                if (pb == pa) continue;
                T dx = xa - qp[3 * pb], dy = ya - qp[3 * pb + 1], dz = za - qp[3 * pb + 2];
                T r2s = dx * dx + dy * dy + dz * dz;
                if (r2s <= T(0)) continue;
                T rinv = rsq<T>(r2s);
                T r = r2s * rinv;
                T rn = (dx * qn[3 * pb] + dy * qn[3 * pb + 1] + dz * qn[3 * pb + 2]) * rinv * rinv * rinv;
                T wb = qw[pb];
                cL += wb * (rinv * (-dphi) + rn * phi);
                T e1 = ex<T>(-kappa * r);
                cY += wb * (e1 * rinv * ((T)er * dphi) - e1 * (T(1) + kappa * r) * rn * phi);
            }
        }
        r1 += wa * (potL[pa] - c4 * cL);
        r2 += wa * (-potYn[pa] - c4 * cY);
    }
    double R1 = (double)r1, R2 = (double)r2;
    double phi_i = x[i];
    double d11 = 0.5 * area[i], d12 = 0, d21 = 0.5 * area[i], d22 = 0;
    for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
        int j = adj_ids[e];
        double vl = S[4 * (long long)e], kl = S[4 * (long long)e + 1], vy = S[4 * (long long)e + 2],
               ky = S[4 * (long long)e + 3];
        double phi = x[j], dphi = x[nt + j];
        R1 += kl * phi - vl * dphi;
        R2 += -ky * phi + er * vy * dphi;
        if (j == i) { d11 += kl; d12 = -vl; d21 -= ky; d22 = er * vy; }
    }
    R1 += 0.5 * area[i] * phi_i;
    R2 += 0.5 * area[i] * phi_i;
    if (precond) {
        double det = d11 * d22 - d12 * d21;
        double a1 = (d22 * R1 - d12 * R2) / det;
        double a2 = (-d21 * R1 + d11 * R2) / det;
        R1 = a1;
        R2 = a2;
    }
    y[i] = R1;
    y[nt + i] = R2;
}

// Coulomb potential of the charges at the quadrature points, FP64:
//   f(x_a) = sum_k q_k / (4 pi eps1 |x_a - r_k|)           (RHS of Eq. direct)
__global__ void k_coulomb(long long np, const double* __restrict__ qp, int na, const double4* __restrict__ atoms,
                          double inv_eps, double* __restrict__ f) {
    __shared__ double4 s[256];
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double x = 0, y = 0, z = 0;
    if (a < np) { x = qp[3 * a]; y = qp[3 * a + 1]; z = qp[3 * a + 2]; }
    double acc = 0.0;
    for (int k0 = 0; k0 < na; k0 += 256) {
        __syncthreads();
        if (k0 + threadIdx.x < na) s[threadIdx.x] = atoms[k0 + threadIdx.x];
        __syncthreads();
        int cnt = min(256, na - k0);
        for (int k = 0; k < cnt; ++k) {
            double dx = x - s[k].x, dy = y - s[k].y, dz = z - s[k].z;
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0) acc += s[k].w * rsqrt(r2);
        }
    }
    if (a < np) f[a] = acc * kInv4PiB * inv_eps;
}

// b_i = sum_{a in T_i} w_a f_a, then [b; 0] through the preconditioner
__global__ void k_rhs(int nt, int nq, const double* __restrict__ f, const double* __restrict__ qw,
                      const int* __restrict__ adj_off, const int* __restrict__ adj_ids, const double* __restrict__ S,
                      const double* __restrict__ area, double er, int precond, double* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double s = 0.0;
    for (int a = 0; a < nq; ++a) s += qw[(long long)i * nq + a] * f[(long long)i * nq + a];
    double R1 = s, R2 = 0.0;
    if (precond) {
        double d11 = 0.5 * area[i], d12 = 0, d21 = 0.5 * area[i], d22 = 0;
        for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
            if (adj_ids[e] != i) continue;
            d11 += S[4 * (long long)e + 1]; d12 = -S[4 * (long long)e];
            d21 -= S[4 * (long long)e + 3]; d22 = er * S[4 * (long long)e + 2];
        }
        double det = d11 * d22 - d12 * d21;
        double a1 = (d22 * R1 - d12 * R2) / det, a2 = (-d21 * R1 + d11 * R2) / det;
        R1 = a1; R2 = a2;
    }
    b[i] = R1;
    b[nt + i] = R2;
}

// phi_reac(r_k) = -K_L[phi](r_k) + V_L[dphi](r_k)   (Eq. phi_reac), FP64;
// one block per 128 atoms, quadrature points staged in shared memory
// Grid: (atom tiles of 128, nsplit ranges of quadrature points); writes the
// partial sum of range `split` to partial[split][atom] (summed in a fixed
// order by k_phi_reac_sum).
__global__ void k_phi_reac(int na, const double4* __restrict__ atoms, long long np, int nq, int nt,
                           const double* __restrict__ qp, const double* __restrict__ qn, const double* __restrict__ qw,
                           const double* __restrict__ x, int nsplit, double* __restrict__ partial) {
    __shared__ double s_p[128][4];
    __shared__ double s_n[128][4];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int split = blockIdx.y;
    const long long b_lo = np * split / nsplit, b_hi = np * (split + 1) / nsplit;
    double px = 0, py = 0, pz = 0;
    if (k < na) { px = atoms[k].x; py = atoms[k].y; pz = atoms[k].z; }
    double acc = 0.0;
    for (long long b0 = b_lo; b0 < b_hi; b0 += 128) {
        __syncthreads();
        long long b = b0 + threadIdx.x;
        if (b < b_hi) {
            int t = (int)(b / nq);
            double w = qw[b];
            s_p[threadIdx.x][0] = qp[3 * b]; s_p[threadIdx.x][1] = qp[3 * b + 1]; s_p[threadIdx.x][2] = qp[3 * b + 2];
            s_p[threadIdx.x][3] = w * x[nt + t];                 // monopole w dphi
            double d = -w * x[t];                                // dipole -w phi
            s_n[threadIdx.x][0] = d * qn[3 * b]; s_n[threadIdx.x][1] = d * qn[3 * b + 1];
            s_n[threadIdx.x][2] = d * qn[3 * b + 2];
        }
        __syncthreads();
        int cnt = (int)min((long long)128, b_hi - b0);
        for (int m = 0; m < cnt; ++m) {
            double dx = px - s_p[m][0], dy = py - s_p[m][1], dz = pz - s_p[m][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rinv = r2 > 0 ? rsqrt(r2) : 0.0;
            acc += rinv * s_p[m][3] + (dx * s_n[m][0] + dy * s_n[m][1] + dz * s_n[m][2]) * rinv * rinv * rinv;
        }
    }
    if (k < na) partial[(long long)split * na + k] = acc;
}

__global__ void k_phi_reac_sum(int na, int nsplit, const double* __restrict__ partial, double* __restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += partial[(long long)q * na + k];
    out[k] = s * kInv4PiB;
}

// dG = 1/2 sum q phi_reac * 4 pi C, FP64 with a fixed reduction order
__global__ void k_energy(int na, const double4* __restrict__ atoms, const double* __restrict__ phir, double* out) {
    __shared__ double red[1024];
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        double v = atoms[k].w * phir[k] - c;     // Kahan
        double t = s + v;
        c = (t - s) - v;
        s = t;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * red[0] * 4.0 * M_PI * kKcal;
}

// ---------------------------------------------------------------------------
// FP64 GMRES kernels
// ---------------------------------------------------------------------------
constexpr int kDotBlocks = 304;

// partial[blk][k] = sum over the block's rows of V[k][i] w[i], k < nk
__global__ void k_dots(long long n, const double* __restrict__ V, long long ld, int nk, const double* __restrict__ w,
                       double* __restrict__ partial, int kmax) {
    __shared__ double red[256];
    long long chunk = (n + gridDim.x - 1) / gridDim.x;
    long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int k = 0; k < nk; ++k) {
        double s = 0.0;
        const double* v = V + (long long)k * ld;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += v[i] * w[i];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * kmax + k] = red[0];
        __syncthreads();
    }
}

__global__ void k_dots_reduce(int nblk, int nk, const double* __restrict__ partial, int kmax, double* __restrict__ h,
                              int accumulate) {
    int k = threadIdx.x + blockIdx.x * blockDim.x;
    if (k >= nk) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(long long)b * kmax + k];
    h[k] = accumulate ? h[k] + s : s;
}

// w -= sum_k h[k] V[k]
__global__ void k_update(long long n, const double* __restrict__ V, long long ld, int nk, const double* __restrict__ h,
                         double* __restrict__ w) {
    extern __shared__ double sh[];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) sh[k] = h[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < nk; ++k) s -= sh[k] * V[(long long)k * ld + i];
        w[i] = s;
    }
}

// out = w / nrm  (nrm = sqrt(*nrm2)); used for V[j+1]
__global__ void k_scale(long long n, const double* __restrict__ w, const double* __restrict__ nrm2, double* __restrict__ out) {
    double inv = 1.0 / sqrt(*nrm2);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
}

// Hessenberg column j (h[0..j], h[j+1] = ||w||^2 on input) -> Givens update.
// H is column-major [kmax+1][kmax]; g, cs, sn of length kmax+1.
__global__ void k_givens(int j, int kmax, const double* __restrict__ h, const double* __restrict__ nrm2,
                         double* H, double* cs, double* sn, double* g, double* resid) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (long long)j * (kmax + 1);
    for (int k = 0; k <= j; ++k) col[k] = h[k];
    col[j + 1] = sqrt(*nrm2);
    for (int k = 0; k < j; ++k) {
        double a = col[k], b = col[k + 1];
        col[k] = cs[k] * a + sn[k] * b;
        col[k + 1] = -sn[k] * a + cs[k] * b;
    }
    double a = col[j], b = col[j + 1];
    double r = hypot(a, b);
    double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    resid[0] = fabs(g[j + 1]);
}

__global__ void k_backsolve(int m, int kmax, const double* __restrict__ H, const double* __restrict__ g, double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = m - 1; k >= 0; --k) {
        double s = g[k];
        for (int c = k + 1; c < m; ++c) s -= H[(long long)c * (kmax + 1) + k] * y[c];
        y[k] = s / H[(long long)k * (kmax + 1) + k];
    }
}

// x += sum_k y[k] V[k]
__global__ void k_axpy_basis(long long n, const double* __restrict__ V, long long ld, int m, const double* __restrict__ y,
                             double* __restrict__ x) {
    extern __shared__ double sh[];
    for (int k = threadIdx.x; k < m; k += blockDim.x) sh[k] = y[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int k = 0; k < m; ++k) s += sh[k] * V[(long long)k * ld + i];
        x[i] = s;
    }
}

__global__ void k_set_g0(const double* nrm2, double* g) { g[0] = sqrt(*nrm2); }

__global__ void k_vadd(int n, const double* a, double* b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] += a[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void ensure_singular(pb_mesh* M, double kappa) {
    const int mode = M->ctx->singular ? M->ctx->singular : (M->nt <= kSingFp64MaxTris ? 1 : 2);
    if (M->kappa_S == kappa && M->sing_mode == mode) return;
    cudaStream_t st = M->ctx->stream;
    const int depth = mode == 1 ? kSingDepth64 : kSingDepth32;
    std::vector<double> pts;
    const SingRule R = make_sing_rule(depth, pts);
    M->S_d.alloc(4 * M->nadj, st);
    M->S_f.alloc(4 * M->nadj, st);
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    const int blocks = (int)std::min<long long>(div_up(M->nadj, 8), 152LL * 64);   // 8 warps per block
    if (mode == 1) {
        DBuf<double> rule;
        rule.alloc(pts.size(), st);
        PB_CUDA(cudaMemcpyAsync(rule.p, pts.data(), pts.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        k_singular<double><<<blocks, 256, 0, st>>>(M->nadj, (int)M->nt, M->verts.p, M->tris.p, M->adj_off.p,
                                                   M->adj_ids.p, kappa, R, rule.p, M->S_d.p);
        PB_CHECK_LAUNCH();
    } else {
        std::vector<float> pf(pts.begin(), pts.end());
        DBuf<float> rule;
        rule.alloc(pf.size(), st);
        PB_CUDA(cudaMemcpyAsync(rule.p, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        k_singular<float><<<blocks, 256, 0, st>>>(M->nadj, (int)M->nt, M->verts.p, M->tris.p, M->adj_off.p,
                                                  M->adj_ids.p, (float)kappa, R, rule.p, M->S_d.p);
        PB_CHECK_LAUNCH();
    }
    k_to_float<<<div_up(4 * M->nadj, 256), 256, 0, st>>>(4 * M->nadj, M->S_d.p, M->S_f.p);
    PB_CHECK_LAUNCH();
    M->kappa_S = kappa;
    M->sing_mode = mode;
}

void ensure_singular_public(pb_mesh* M, double kappa) { ensure_singular(M, kappa); }

void mesh_setup(pb_mesh* M, const double* verts, const int* tris) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nv = (int)M->nv, nq = M->nq;
    M->verts.alloc(3 * nv, st);
    M->tris.alloc(3 * nt, st);
    PB_CUDA(cudaMemcpyAsync(M->verts.p, verts, 3 * nv * sizeof(double), cudaMemcpyDefault, st));
    PB_CUDA(cudaMemcpyAsync(M->tris.p, tris, 3 * nt * sizeof(int), cudaMemcpyDefault, st));
    std::vector<double> L, W;
    regular_rule(nq, L, W);
    DBuf<double> rl, rw;
    rl.alloc(L.size(), st); rw.alloc(W.size(), st);
    PB_CUDA(cudaMemcpyAsync(rl.p, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(rw.p, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    const long long np = (long long)nt * nq;
    M->nrm.alloc(3 * nt, st); M->area.alloc(nt, st);
    M->qp_d.alloc(3 * np, st); M->qn_d.alloc(3 * np, st); M->qw_d.alloc(np, st);
    M->qp_f.alloc(3 * np, st); M->qn_f.alloc(3 * np, st); M->qw_f.alloc(np, st);
    DBuf<int> bad;
    bad.alloc(1, st);
    bad.zero(st);
    k_geometry<<<div_up(nt, 128), 128, 0, st>>>(nt, nv, M->verts.p, M->tris.p, nq, rl.p, rw.p, M->nrm.p, M->area.p,
                                                M->qp_d.p, M->qn_d.p, M->qw_d.p, M->qp_f.p, M->qn_f.p, M->qw_f.p, bad.p);
    PB_CHECK_LAUNCH();
    int hbad = 0;
    PB_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    PB_REQUIRE(!hbad, PB_EMESH, "pb_mesh_setup: triangle with an invalid or repeated vertex index");
    {   // degenerate triangles: area < 1e-12 * mean
        std::vector<double> ar(nt);
        PB_CUDA(cudaMemcpyAsync(ar.data(), M->area.p, nt * sizeof(double), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        double mean = 0;
        for (double a : ar) mean += a;
        mean /= nt;
        for (double a : ar) PB_REQUIRE(a >= 1e-12 * mean && a > 0, PB_EMESH, "pb_mesh_setup: degenerate triangle");
    }
    // adjacency through the vertex -> triangle incidence
    DBuf<int> vcnt, voff, vcur, vids;
    vcnt.alloc(nv + 1, st); vcnt.zero(st);
    voff.alloc(nv + 1, st); vcur.alloc(nv, st); vcur.zero(st);
    vids.alloc(3 * nt, st);
    k_vcount<<<div_up(nt, 256), 256, 0, st>>>(nt, M->tris.p, vcnt.p);
    PB_CHECK_LAUNCH();
    {
        size_t tmp = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tmp, vcnt.p, voff.p, nv + 1, st);
        DBuf<char> t;
        t.alloc(std::max<size_t>(tmp, 1), st);
        cub::DeviceScan::ExclusiveSum(t.p, tmp, vcnt.p, voff.p, nv + 1, st);
    }
    k_vfill<<<div_up(nt, 256), 256, 0, st>>>(nt, M->tris.p, voff.p, vcur.p, vids.p);
    PB_CHECK_LAUNCH();
    DBuf<int> acnt, ovf;
    acnt.alloc(nt + 1, st); acnt.zero(st);
    ovf.alloc(1, st); ovf.zero(st);
    M->adj_off.alloc(nt + 1, st);
    k_adjacency<<<div_up(nt, 128), 128, 0, st>>>(nt, M->tris.p, voff.p, vids.p, 0, acnt.p, nullptr, nullptr, ovf.p);
    PB_CHECK_LAUNCH();
    {
        size_t tmp = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tmp, acnt.p, M->adj_off.p, nt + 1, st);
        DBuf<char> t;
        t.alloc(std::max<size_t>(tmp, 1), st);
        cub::DeviceScan::ExclusiveSum(t.p, tmp, acnt.p, M->adj_off.p, nt + 1, st);
    }
    int last = 0, hovf = 0;
    PB_CUDA(cudaMemcpyAsync(&last, M->adj_off.p + nt, sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    PB_REQUIRE(!hovf, PB_EMESH, "pb_mesh_setup: a triangle has more than 128 vertex neighbours");
    M->nadj = last;
    M->adj_ids.alloc(std::max(last, 1), st);
    k_adjacency<<<div_up(nt, 128), 128, 0, st>>>(nt, M->tris.p, voff.p, vids.p, 1, nullptr, M->adj_off.p,
                                                 M->adj_ids.p, ovf.p);
    PB_CHECK_LAUNCH();
    M->nunk = M->basis == PB_P1 ? M->nv : M->nt;
    if (M->basis == PB_P1) p1_setup(M);
    // FMM tree over the quadrature points
    M->tree = new fmm_tree();
    M->tree->ctx = M->ctx;
    M->tree->ns = np;
    M->tree->nt = np;
    M->tree->same = true;
    M->tree->ncrit = M->ncrit;
    build_tree(M->tree, M->qp_f.p, nullptr);
    PB_CUDA(cudaStreamSynchronize(st));
}

// y = A x (precond = 0) or P^{-1} A x (precond = 1), x, y FP64 device [2 nt]
template <typename T>
static void matvec_t(pb_mesh* M, double eps_in, double eps_out, double kappa, const double* x, double* y, int precond) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    const double er = eps_in / eps_out;
    const int prec = std::is_same<T, float>::value ? PB_MIXED : PB_FP64;
    DBuf<T> qL, dL, qYn, pL, pYn;
    qL.alloc(np, st); dL.alloc(np, st); qYn.alloc(np, st); pL.alloc(np, st); pYn.alloc(np, st);
    const T* qw = std::is_same<T, float>::value ? (const T*)M->qw_f.p : (const T*)M->qw_d.p;
    const T* qp = std::is_same<T, float>::value ? (const T*)M->qp_f.p : (const T*)M->qp_d.p;
    const T* qn = std::is_same<T, float>::value ? (const T*)M->qn_f.p : (const T*)M->qn_d.p;
    const T* S = std::is_same<T, float>::value ? (const T*)M->S_f.p : (const T*)M->S_d.p;
    {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        k_p1<T><<<div_up(np, 256), 256, 0, st>>>(nt, nq, x, qw, er, qL.p, dL.p, qYn.p);
        PB_CHECK_LAUNCH();
    }
    fmm_apply_pair_impl(M->tree, kappa, M->p, prec, qL.p, qYn.p, dL.p, qn, nullptr, pL.p, pYn.p, nullptr, nullptr);
    {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        // S in FP64 for the combine (both paths): the singular entries are exact data
        k_combine<T><<<div_up(nt, 128), 128, 0, st>>>(nt, nq, x, pL.p, pYn.p, qp, qn, qw, M->adj_off.p, M->adj_ids.p,
                                                      (const T*)S, M->area.p, er, kappa, precond, y);
        PB_CHECK_LAUNCH();
    }
}

void mesh_matvec(pb_mesh* M, double eps_in, double eps_out, double kappa, int precision, const double* x, double* y,
                 int precond, int formulation) {
    if (M->basis == PB_P1) {
        matvec_p1(M, eps_in, eps_out, kappa, precision, formulation, x, y, precond);
        return;
    }
    PB_REQUIRE(formulation == PB_FORM_DIRECT, PB_EINVAL, "the derivative formulations need a PB_P1 mesh");
    ensure_singular(M, kappa);
    if (precision == PB_FP64) matvec_t<double>(M, eps_in, eps_out, kappa, x, y, precond);
    else matvec_t<float>(M, eps_in, eps_out, kappa, x, y, precond);
}

template <typename T>
static T read_scalar(const T* d, cudaStream_t st) {
    T h;
    PB_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    return h;
}

// Full GMRES (x0 = 0, left preconditioned, CGS2), FP64.  `matvec(v, w)`
// writes w = P^{-1} A v for device vectors of length 2 nt.
int gmres(pb_mesh* M, const std::function<void(const double*, double*)>& matvec, const double* b,
          DBuf<double>& x, double tol, int max_iter, int* iterations, double* residual) {
    cudaStream_t st = M->ctx->stream;
    const long long n = 2 * M->nunk;
    const int kmax = std::max(1, max_iter);
    DBuf<double> V, w, partial, h, h2, H, cs, sn, g, nrm2, resid, yv;
    V.alloc((size_t)(kmax + 1) * n, st);
    w.alloc(n, st);
    partial.alloc((size_t)kDotBlocks * (kmax + 1), st);
    h.alloc(kmax + 2, st);
    h2.alloc(kmax + 2, st);
    H.alloc((size_t)(kmax + 1) * kmax, st);
    cs.alloc(kmax + 1, st); sn.alloc(kmax + 1, st); g.alloc(kmax + 2, st);
    nrm2.alloc(1, st); resid.alloc(1, st); yv.alloc(kmax + 1, st);
    g.zero(st);
    x.alloc(n, st);
    x.zero(st);
    const int nb = std::min<long long>(kDotBlocks, (n + 255) / 256);
    auto dots = [&](const double* Vb, int nk, const double* vec, double* out, int acc) {
        k_dots<<<nb, 256, 0, st>>>(n, Vb, n, nk, vec, partial.p, kmax + 1);
        PB_CHECK_LAUNCH();
        k_dots_reduce<<<div_up(nk, 128), 128, 0, st>>>(nb, nk, partial.p, kmax + 1, out, acc);
        PB_CHECK_LAUNCH();
    };
    const int ub = std::min<long long>(4 * M->ctx->sm_count, (n + 255) / 256);
    // r0 = P^{-1} b (b is already preconditioned), beta = ||r0||
    dots(b, 1, b, nrm2.p, 0);
    double beta = std::sqrt(read_scalar(nrm2.p, st));
    if (beta == 0.0) { *iterations = 0; *residual = 0.0; return PB_OK; }
    k_scale<<<ub, 256, 0, st>>>(n, b, nrm2.p, V.p);
    k_set_g0<<<1, 1, 0, st>>>(nrm2.p, g.p);
    PB_CHECK_LAUNCH();
    int j = 0;
    double rel = 1.0;
    int status = PB_ENOCONV;
    for (j = 0; j < kmax; ++j) {
        matvec(V.p + (long long)j * n, w.p);
        PhaseTimer ph(M->ctx, PB_PH_GMRES);
        // CGS2: two passes of classical Gram-Schmidt
        dots(V.p, j + 1, w.p, h.p, 0);
        k_update<<<ub, 256, (j + 1) * sizeof(double), st>>>(n, V.p, n, j + 1, h.p, w.p);
        PB_CHECK_LAUNCH();
        dots(V.p, j + 1, w.p, h2.p, 0);
        k_update<<<ub, 256, (j + 1) * sizeof(double), st>>>(n, V.p, n, j + 1, h2.p, w.p);
        PB_CHECK_LAUNCH();
        k_vadd<<<div_up(j + 1, 128), 128, 0, st>>>(j + 1, h2.p, h.p);
        PB_CHECK_LAUNCH();
        dots(w.p, 1, w.p, nrm2.p, 0);
        k_givens<<<1, 1, 0, st>>>(j, kmax, h.p, nrm2.p, H.p, cs.p, sn.p, g.p, resid.p);
        PB_CHECK_LAUNCH();
        k_scale<<<ub, 256, 0, st>>>(n, w.p, nrm2.p, V.p + (long long)(j + 1) * n);
        PB_CHECK_LAUNCH();
        rel = read_scalar(resid.p, st) / beta;
        if (rel <= tol) { ++j; status = PB_OK; break; }
    }
    int m = std::min(j, kmax);
    k_backsolve<<<1, 1, 0, st>>>(m, kmax, H.p, g.p, yv.p);
    k_axpy_basis<<<ub, 256, m * sizeof(double), st>>>(n, V.p, n, m, yv.p, x.p);
    PB_CHECK_LAUNCH();
    PB_CUDA(cudaStreamSynchronize(st));
    *iterations = m;
    *residual = rel;
    return status;
}

// ---------------------------------------------------------------------------
// charge <-> surface couplings through the FMM (large atom counts)
// ---------------------------------------------------------------------------
__global__ void k_atoms_split(int na, const double4* __restrict__ atoms, double qscale, float* __restrict__ xyz,
                              float* __restrict__ qf, double* __restrict__ qd) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    double4 a = atoms[k];
    xyz[3 * k] = (float)a.x; xyz[3 * k + 1] = (float)a.y; xyz[3 * k + 2] = (float)a.z;
    qf[k] = (float)(a.w * qscale);
    qd[k] = a.w * qscale;
}

// surface densities of the reaction potential: monopole w dphi, dipole -w phi
template <typename T>
__global__ void k_reac_densities(long long np, int nq, int nt, const double* __restrict__ qw,
                                 const double* __restrict__ x, T* __restrict__ mono, T* __restrict__ dip) {
    long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= np) return;
    int t = (int)(b / nq);
    mono[b] = (T)(qw[b] * x[nt + t]);
    dip[b] = (T)(-qw[b] * x[t]);
}

template <typename T>
__global__ void k_to_double(long long n, const T* __restrict__ a, double* __restrict__ b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

bool use_fmm_coupling(const pb_mesh* M, const pb_result* R) {
    const int mode = M->ctx->coupling;
    if (mode == 1) return false;
    if (mode == 2) return true;
    return (double)R->na * (double)M->nt * M->nq > 4e9;
}

// the two coupling trees of a result (atoms as targets / as sources)
void ensure_coupling_trees(pb_mesh* M, pb_result* R) {
    if (R->tree_qa) return;
    cudaStream_t st = M->ctx->stream;
    const long long np = M->nt * M->nq;
    R->atoms_f.alloc(3 * R->na, st);
    R->q_f.alloc(R->na, st);
    R->q_d.alloc(R->na, st);
    k_atoms_split<<<div_up(R->na, 128), 128, 0, st>>>((int)R->na, (const double4*)R->atoms.p, 1.0 / R->eps_in,
                                                      R->atoms_f.p, R->q_f.p, R->q_d.p);
    PB_CHECK_LAUNCH();
    R->tree_qa = new fmm_tree();       // sources = quadrature points, targets = atoms
    R->tree_qa->ctx = M->ctx;
    R->tree_qa->ns = np; R->tree_qa->nt = R->na; R->tree_qa->same = false; R->tree_qa->ncrit = M->ncrit;
    build_tree(R->tree_qa, M->qp_f.p, R->atoms_f.p);
    R->tree_aq = new fmm_tree();       // sources = atoms, targets = quadrature points
    R->tree_aq->ctx = M->ctx;
    R->tree_aq->ns = R->na; R->tree_aq->nt = np; R->tree_aq->same = false; R->tree_aq->ncrit = M->ncrit;
    build_tree(R->tree_aq, R->atoms_f.p, M->qp_f.p);
}

// f(x_a) = sum_k q_k / (4 pi eps1 |x_a - r_k|) at every quadrature point
void coulomb_at_points(pb_mesh* M, pb_result* R, double* f) {
    cudaStream_t st = M->ctx->stream;
    const long long np = M->nt * M->nq;
    if (!use_fmm_coupling(M, R)) {
        k_coulomb<<<div_up(np, 256), 256, 0, st>>>(np, M->qp_d.p, (int)R->na, (const double4*)R->atoms.p,
                                                   1.0 / R->eps_in, f);
        PB_CHECK_LAUNCH();
        return;
    }
    ensure_coupling_trees(M, R);
    if (R->precision == PB_FP64) {
        fmm_apply_impl(R->tree_aq, FMM_LAPLACE, 0.0, M->p, PB_FP64, R->q_d.p, nullptr, nullptr, nullptr, f, nullptr);
    } else {
        DBuf<float> ff;
        ff.alloc(np, st);
        fmm_apply_impl(R->tree_aq, FMM_LAPLACE, 0.0, M->p, PB_MIXED, R->q_f.p, nullptr, nullptr, nullptr, ff.p,
                       nullptr);
        k_to_double<float><<<div_up(np, 256), 256, 0, st>>>(np, ff.p, f);
        PB_CHECK_LAUNCH();
    }
}

// phi_reac at every atom (Eq. phi_reac)
static void reaction_potential(pb_mesh* M, pb_result* R, double* phir) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    if (!use_fmm_coupling(M, R)) {
        // split the points so that the grid has at least two CTAs per SM
        const int tiles = (int)div_up(R->na, 128);
        const int nsplit = (int)std::max<long long>(1, std::min<long long>(div_up(2 * M->ctx->sm_count, tiles),
                                                                          div_up(np, 128)));
        DBuf<double> part;
        part.alloc((size_t)nsplit * R->na, st);
        k_phi_reac<<<dim3(tiles, nsplit), 128, 0, st>>>((int)R->na, (const double4*)R->atoms.p, np, nq, nt,
                                                        M->qp_d.p, M->qn_d.p, M->qw_d.p, R->x.p, nsplit, part.p);
        PB_CHECK_LAUNCH();
        k_phi_reac_sum<<<tiles, 128, 0, st>>>((int)R->na, nsplit, part.p, phir);
        PB_CHECK_LAUNCH();
        return;
    }
    ensure_coupling_trees(M, R);
    if (R->precision == PB_FP64) {
        DBuf<double> mono, dip;
        mono.alloc(np, st); dip.alloc(np, st);
        k_reac_densities<double><<<div_up(np, 256), 256, 0, st>>>(np, nq, nt, M->qw_d.p, R->x.p, mono.p, dip.p);
        PB_CHECK_LAUNCH();
        fmm_apply_impl(R->tree_qa, FMM_LAPLACE, 0.0, M->p, PB_FP64, mono.p, dip.p, M->qn_d.p, nullptr, phir,
                       nullptr);
    } else {
        DBuf<float> mono, dip, pf;
        mono.alloc(np, st); dip.alloc(np, st); pf.alloc(R->na, st);
        k_reac_densities<float><<<div_up(np, 256), 256, 0, st>>>(np, nq, nt, M->qw_d.p, R->x.p, mono.p, dip.p);
        PB_CHECK_LAUNCH();
        fmm_apply_impl(R->tree_qa, FMM_LAPLACE, 0.0, M->p, PB_MIXED, mono.p, dip.p, M->qn_f.p, nullptr, pf.p,
                       nullptr);
        k_to_double<float><<<div_up(R->na, 256), 256, 0, st>>>(R->na, pf.p, phir);
        PB_CHECK_LAUNCH();
    }
}

// The preconditioned mat-vec of a solve as a CUDA graph replayed on the
// context stream: captured on a private stream through a context copy once
// an uncaptured mat-vec with the same parameters has filled the caches
// (operators, singular entries); false when no graph is available, then the
// caller launches the kernels itself.
static bool matvec_graph(pb_mesh* M, pb_result* R) {
    pb_ctx* ctx = M->ctx;
    const double key[9] = {R->eps_in, R->eps_out, R->kappa, (double)R->precision,
                           (double)(ctx->deterministic + 2 * ctx->overlap), (double)ctx->singular,
                           (double)(uintptr_t)M->S_d.p, (double)(uintptr_t)M->D1.p, (double)R->formulation};
    const bool same = std::equal(key, key + 9, M->mv_key);
    if (same && M->mv_exec) return true;
    if (!same || !M->mv_warm) {
        // first solve with these parameters: run uncaptured, capture next time
        std::copy(key, key + 9, M->mv_key);
        M->mv_warm = false;
        if (M->mv_exec) { cudaGraphExecDestroy(M->mv_exec); M->mv_exec = nullptr; }
        if (M->mv_graph) { cudaGraphDestroy(M->mv_graph); M->mv_graph = nullptr; }
        return false;
    }
    const long long n = 2 * M->nunk;
    M->mv_in.alloc(n, ctx->stream);
    M->mv_out.alloc(n, ctx->stream);
    M->mv_in.zero(ctx->stream);
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
    pb_ctx sub;
    sub.device = ctx->device;
    sub.sm_count = ctx->sm_count;
    sub.dev_err = ctx->dev_err;
    sub.profile = false;
    sub.coupling = ctx->coupling;
    sub.deterministic = ctx->deterministic;
    sub.singular = ctx->singular;
    sub.overlap = ctx->overlap;
    sub.aux = ctx->aux;                 // joins the capture through the fork event
    sub.ev_fork = ctx->ev_fork;
    sub.ev_join = ctx->ev_join;
    PB_CUDA(cudaStreamCreateWithFlags(&sub.stream, cudaStreamNonBlocking));
    pb_ctx* saved_tree = M->tree->ctx;
    M->ctx = &sub;
    M->tree->ctx = &sub;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(sub.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        try {
            mesh_matvec(M, R->eps_in, R->eps_out, R->kappa, R->precision, M->mv_in.p, M->mv_out.p, 1,
                        R->formulation);
        } catch (const Error&) {
            ok = false;
        }
        ok = (cudaStreamEndCapture(sub.stream, &graph) == cudaSuccess) && ok;
    }
    M->ctx = ctx;
    M->tree->ctx = saved_tree;
    if (ok) ok = cudaGraphInstantiate(&M->mv_exec, graph, 0) == cudaSuccess;
    if (ok) {
        M->mv_graph = graph;
    } else {
        if (graph) cudaGraphDestroy(graph);
        M->mv_exec = nullptr;
        cudaGetLastError();
    }
    cudaStreamSynchronize(sub.stream);
    cudaStreamDestroy(sub.stream);
    return ok;
}

int solve(pb_mesh* M, pb_result* R, double tol, int max_iter) {
    cudaStream_t st = M->ctx->stream;
    PB_REQUIRE(M->basis == PB_P1 || R->formulation == PB_FORM_DIRECT, PB_EINVAL,
               "the derivative formulations need a PB_P1 mesh");
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    DBuf<double> f, b;
    b.alloc(2 * M->nunk, st);
    if (M->basis == PB_P1) {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        rhs_p1(M, R, b.p);
    } else {
        ensure_singular(M, R->kappa);
        f.alloc(np, st);
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        coulomb_at_points(M, R, f.p);
        k_rhs<<<div_up(nt, 128), 128, 0, st>>>(nt, nq, f.p, M->qw_d.p, M->adj_off.p, M->adj_ids.p, M->S_d.p,
                                               M->area.p, R->eps_in / R->eps_out, 1, b.p);
        PB_CHECK_LAUNCH();
    }
    const bool graph = matvec_graph(M, R);
    const long long n = 2 * M->nunk;
    auto mv = [&](const double* v, double* w) {
        if (graph) {
            PB_CUDA(cudaMemcpyAsync(M->mv_in.p, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            PB_CUDA(cudaGraphLaunch(M->mv_exec, st));
            PB_CUDA(cudaMemcpyAsync(w, M->mv_out.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            mesh_matvec(M, R->eps_in, R->eps_out, R->kappa, R->precision, v, w, 1, R->formulation);
        }
    };
    int status = gmres(M, mv, b.p, R->x, tol, max_iter, &R->iterations, &R->residual);
    if (!graph) M->mv_warm = true;
    R->status = status;
    return status;
}

void reaction_energy(pb_result* R, double* phir_host, double* dG) {
    pb_mesh* M = R->mesh;
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    DBuf<double> phir, e;
    phir.alloc(std::max<int64_t>(R->na, 1), st);
    e.alloc(1, st);
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    (void)np;
    if (M->basis == PB_P1) reaction_potential_p1(M, R, phir.p);
    else reaction_potential(M, R, phir.p);
    k_energy<<<1, 1024, 0, st>>>((int)R->na, (const double4*)R->atoms.p, phir.p, e.p);
    PB_CHECK_LAUNCH();
    if (phir_host) PB_CUDA(cudaMemcpyAsync(phir_host, phir.p, R->na * sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(dG, e.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
}

}  // namespace pbfmm
