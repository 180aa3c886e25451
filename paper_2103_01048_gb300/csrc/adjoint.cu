// Gradients of the polar solvation energy by an adjoint solve.
//
// With u = A^{-1} B q the solution of Eq. direct (B: charges -> right-hand
// side, the Coulomb term of Eq. direct integrated against the test functions)
// and phi_reac = E u (Eq. phi_reac evaluated at the atoms), the energy of
// Eq. energy is E(q, x) = 1/2 q^T E A^{-1} B q.  With the adjoint solution
// lambda = A^{-T} E^T q:
//   dE/dq_k = 1/2 [phi_reac(r_k) + psi(r_k)],
//   dE/dr_k = 1/2 q_k [grad phi_reac(r_k) + grad psi(r_k)],
//   psi(r) = sum_a w_a lambda_phi(tri(a)) g_L(x_a, r) / eps1,
// the surface held fixed (the mesh does not move with the atoms), all times
// 4 pi * 332.0637 for kcal/mol.
//
// A^T goes through the same FMM split: the single layer is symmetric and
// the transpose of the double layer is the adjoint double layer K' (target
// normal derivative of a monopole field, Eq. adj_hyp), so each adjoint
// mat-vec is one Laplace and one Yukawa FMM pass with monopole sources and
// both outputs (potential and target-normal derivative), the C correction of
// the same pairs, the transposed singular entries S^T, and the transposed
// block preconditioner.
#include "bem.cuh"
#include <cmath>

namespace pbfmm {

constexpr double kInv4PiA = 0.07957747154594767;
constexpr double kKcalA = 332.0637;

template <typename T> __device__ __forceinline__ T rsqrt_a(T x);
template <> __device__ __forceinline__ float rsqrt_a<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_a<double>(double x) { return rsqrt(x); }
template <typename T> __device__ __forceinline__ T exp_a(T x);
template <> __device__ __forceinline__ float exp_a<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double exp_a<double>(double x) { return exp(x); }

// adjacency transpose: for entry e = (i, j) the index of (j, i) in row j
__global__ void k_adj_transpose(int nt, const int* __restrict__ off, const int* __restrict__ ids, int* __restrict__ tr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    for (int e = off[i]; e < off[i + 1]; ++e) {
        int j = ids[e];
        int lo = off[j], hi = off[j + 1];
        while (lo < hi) {
            int m = (lo + hi) >> 1;
            if (ids[m] < i) lo = m + 1;
            else hi = m;
        }
        tr[e] = lo;
    }
}

// 2x2 diagonal block of triangle i: [[d11, d12], [d21, d22]]
__device__ __forceinline__ void diag_block(int i, const int* adj_off, const int* adj_ids, const double* S,
                                           const double* area, double er, double& d11, double& d12, double& d21,
                                           double& d22) {
    d11 = 0.5 * area[i]; d12 = 0.0; d21 = 0.5 * area[i]; d22 = 0.0;
    for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
        if (adj_ids[e] != i) continue;
        d11 += S[4 * (long long)e + 1];
        d12 = -S[4 * (long long)e];
        d21 -= S[4 * (long long)e + 3];
        d22 = er * S[4 * (long long)e + 2];
    }
}

// adjoint right-hand side E^T q, then the transposed preconditioner:
//   c_phi,i  = -sum_{a in T_i} w_a sum_k q_k dg_L/dn_y(r_k, x_a)
//   c_dphi,i =  sum_{a in T_i} w_a sum_k q_k g_L(r_k, x_a)
__global__ void k_adj_rhs(int nt, int nq, const double* __restrict__ qp, const double* __restrict__ qn,
                          const double* __restrict__ qw, int na, const double4* __restrict__ atoms,
                          const int* __restrict__ adj_off, const int* __restrict__ adj_ids, const double* __restrict__ S,
                          const double* __restrict__ area, double er, double* __restrict__ c) {
    __shared__ double4 s_a[128];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double cphi = 0.0, cdphi = 0.0;
    for (int k0 = 0; k0 < na; k0 += 128) {
        __syncthreads();
        if (k0 + threadIdx.x < na) s_a[threadIdx.x] = atoms[k0 + threadIdx.x];
        __syncthreads();
        if (i >= nt) continue;
        int cnt = min(128, na - k0);
        for (int a = 0; a < nq; ++a) {
            long long pa = (long long)i * nq + a;
            double x = qp[3 * pa], y = qp[3 * pa + 1], z = qp[3 * pa + 2];
            double nx = qn[3 * pa], ny = qn[3 * pa + 1], nz = qn[3 * pa + 2], w = qw[pa];
            double sp = 0.0, sd = 0.0;
            for (int k = 0; k < cnt; ++k) {
                double dx = s_a[k].x - x, dy = s_a[k].y - y, dz = s_a[k].z - z;
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= 0) continue;
                double ri = rsqrt(r2);
                sp += s_a[k].w * ri;
                sd += s_a[k].w * (dx * nx + dy * ny + dz * nz) * ri * ri * ri;
            }
            cdphi += w * sp * kInv4PiA;
            cphi -= w * sd * kInv4PiA;
        }
    }
    if (i >= nt) return;
    double d11, d12, d21, d22;
    diag_block(i, adj_off, adj_ids, S, area, er, d11, d12, d21, d22);
    // transposed block [[d11, d21], [d12, d22]]
    double det = d11 * d22 - d12 * d21;
    c[i] = (d22 * cphi - d21 * cdphi) / det;
    c[nt + i] = (-d12 * cphi + d11 * cdphi) / det;
}

// the same right-hand side from FMM outputs at the quadrature points:
// pot = sum_k q_k g(x_a, r_k), dn = its n_a-derivative (charges as sources)
__global__ void k_adj_rhs_fmm(int nt, int nq, const double* __restrict__ qw, const float* __restrict__ pot,
                              const float* __restrict__ dn, double qscale, const int* __restrict__ adj_off,
                              const int* __restrict__ adj_ids, const double* __restrict__ S,
                              const double* __restrict__ area, double er, double* __restrict__ c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double cphi = 0.0, cdphi = 0.0;
    for (int a = 0; a < nq; ++a) {
        long long pa = (long long)i * nq + a;
        cdphi += qw[pa] * (double)pot[pa] * qscale;
        cphi -= qw[pa] * (double)dn[pa] * qscale;
    }
    double d11, d12, d21, d22;
    diag_block(i, adj_off, adj_ids, S, area, er, d11, d12, d21, d22);
    double det = d11 * d22 - d12 * d21;
    c[i] = (d22 * cphi - d21 * cdphi) / det;
    c[nt + i] = (-d12 * cphi + d11 * cdphi) / det;
}

template <typename T>
__global__ void k_p1_adj(int nt, int nq, const double* __restrict__ lam, const T* __restrict__ qw, T* mL, T* mY) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= (long long)nt * nq) return;
    int i = (int)(a / nq);
    mL[a] = qw[a] * (T)lam[i];
    mY[a] = qw[a] * (T)lam[nt + i];
}

// y = D^{-T} (A^T lam):  FMM outputs (potential and target-normal derivative
// of the monopole fields of w*lam_phi (Laplace) and w*lam_dphi (Yukawa)),
// minus C, plus S^T and the mass term.
template <typename T>
__global__ void k_combine_adj(int nt, int nq, const double* __restrict__ lam, const T* __restrict__ pL,
                              const T* __restrict__ dL, const T* __restrict__ pY, const T* __restrict__ dY,
                              const T* __restrict__ qp, const T* __restrict__ qn, const T* __restrict__ qw,
                              const int* __restrict__ adj_off, const int* __restrict__ adj_ids,
                              const int* __restrict__ adj_tr, const double* __restrict__ S,
                              const double* __restrict__ area, double er, double kappa_d, double* __restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const T kappa = (T)kappa_d;
    const T c4 = (T)kInv4PiA;
    T sdL = 0, spL = 0, sdY = 0, spY = 0;
    for (int a = 0; a < nq; ++a) {
        long long pa = (long long)i * nq + a;
        T wa = qw[pa];
        T xa = qp[3 * pa], ya = qp[3 * pa + 1], za = qp[3 * pa + 2];
        T nxa = qn[3 * pa], nya = qn[3 * pa + 1], nza = qn[3 * pa + 2];
        T cpL = 0, cdL = 0, cpY = 0, cdY = 0;
        for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
            int j = adj_ids[e];
            T l1 = (T)lam[j], l2 = (T)lam[nt + j];
            for (int b = 0; b < nq; ++b) {
                long long pb = (long long)j * nq + b;
                if (pb == pa) continue;
                T dx = xa - qp[3 * pb], dy = ya - qp[3 * pb + 1], dz = za - qp[3 * pb + 2];
                T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= T(0)) continue;
                T ri = rsqrt_a<T>(r2);
                T r = r2 * ri;
                T rn = (dx * nxa + dy * nya + dz * nza) * ri * ri * ri;     // (x_a - x_b).n_a / r^3
                T wb = qw[pb];
                cpL += wb * l1 * ri;
                cdL -= wb * l1 * rn;
                T e1 = exp_a<T>(-kappa * r);
                cpY += wb * l2 * e1 * ri;
                cdY -= wb * l2 * e1 * (T(1) + kappa * r) * rn;
            }
        }
        spL += wa * (pL[pa] - c4 * cpL);
        sdL += wa * (dL[pa] - c4 * cdL);
        spY += wa * (pY[pa] - c4 * cpY);
        sdY += wa * (dY[pa] - c4 * cdY);
    }
    double l1i = lam[i], l2i = lam[nt + i];
    double Yphi = 0.5 * area[i] * (l1i + l2i) + (double)sdL - (double)sdY;
    double Ydphi = -(double)spL + er * (double)spY;
    for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
        int j = adj_ids[e];
        long long et = adj_tr[e];                 // entry (j, i)
        double vl = S[4 * et], kl = S[4 * et + 1], vy = S[4 * et + 2], ky = S[4 * et + 3];
        double l1 = lam[j], l2 = lam[nt + j];
        Yphi += kl * l1 - ky * l2;
        Ydphi += -vl * l1 + er * vy * l2;
    }
    double d11, d12, d21, d22;
    diag_block(i, adj_off, adj_ids, S, area, er, d11, d12, d21, d22);
    double det = d11 * d22 - d12 * d21;
    y[i] = (d22 * Yphi - d21 * Ydphi) / det;
    y[nt + i] = (-d12 * Yphi + d11 * Ydphi) / det;
}

// per atom: phi_reac, grad phi_reac (forward solution x) and psi, grad psi
// (adjoint solution), then dE/dq and dE/dr in kcal/mol units
__global__ void k_atom_grad(int na, const double4* __restrict__ atoms, long long np, int nq, int nt,
                            const double* __restrict__ qp, const double* __restrict__ qn, const double* __restrict__ qw,
                            const double* __restrict__ x, const double* __restrict__ lam, double inv_eps,
                            double* __restrict__ dEdq, double* __restrict__ dEdx) {
    __shared__ double s_p[128][3], s_n[128][3], s_v[128][3];   // v: (w dphi, -w phi, w lam_phi / eps1)
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double px = 0, py = 0, pz = 0;
    if (k < na) { px = atoms[k].x; py = atoms[k].y; pz = atoms[k].z; }
    double f = 0, fx = 0, fy = 0, fz = 0;       // phi_reac + psi and its gradient
    for (long long b0 = 0; b0 < np; b0 += 128) {
        __syncthreads();
        long long b = b0 + threadIdx.x;
        if (b < np) {
            int t = (int)(b / nq);
            double w = qw[b];
            for (int c = 0; c < 3; ++c) { s_p[threadIdx.x][c] = qp[3 * b + c]; s_n[threadIdx.x][c] = qn[3 * b + c]; }
            s_v[threadIdx.x][0] = w * x[nt + t];
            s_v[threadIdx.x][1] = -w * x[t];
            s_v[threadIdx.x][2] = w * lam[t] * inv_eps;
        }
        __syncthreads();
        int cnt = (int)min((long long)128, np - b0);
        for (int m = 0; m < cnt; ++m) {
            double dx = px - s_p[m][0], dy = py - s_p[m][1], dz = pz - s_p[m][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 <= 0) continue;
            double ri = rsqrt(r2), ri3 = ri * ri * ri;
            double mono = s_v[m][0] + s_v[m][2];          // monopole sources (reaction + adjoint)
            double dip = s_v[m][1];                       // dipole source of the reaction field
            double rn = dx * s_n[m][0] + dy * s_n[m][1] + dz * s_n[m][2];
            f += mono * ri + dip * rn * ri3;
            // grad of g: -(d) / r^3;  grad of (d.n)/r^3: n / r^3 - 3 d (d.n) / r^5
            double gm = -mono * ri3;
            double c5 = 3.0 * rn * ri3 * ri * ri;
            fx += gm * dx + dip * (s_n[m][0] * ri3 - c5 * dx);
            fy += gm * dy + dip * (s_n[m][1] * ri3 - c5 * dy);
            fz += gm * dz + dip * (s_n[m][2] * ri3 - c5 * dz);
        }
    }
    if (k >= na) return;
    const double u = 0.5 * kInv4PiA * 4.0 * M_PI * kKcalA;    // 1/2 * 1/(4 pi) * 4 pi C
    dEdq[k] = u * f;
    const double qk = atoms[k].w;
    dEdx[3 * k] = u * qk * fx;
    dEdx[3 * k + 1] = u * qk * fy;
    dEdx[3 * k + 2] = u * qk * fz;
}

void ensure_adj_transpose(pb_mesh* M) {
    if (M->adj_tr.p) return;
    cudaStream_t st = M->ctx->stream;
    M->adj_tr.alloc(std::max<int64_t>(M->nadj, 1), st);
    k_adj_transpose<<<div_up(M->nt, 128), 128, 0, st>>>((int)M->nt, M->adj_off.p, M->adj_ids.p, M->adj_tr.p);
    PB_CHECK_LAUNCH();
}

template <typename T>
static void adj_matvec_t(pb_mesh* M, const pb_result* R, const double* lam, double* y) {
    cudaStream_t st = M->ctx->stream;
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    const bool f32 = std::is_same<T, float>::value;
    const int prec = f32 ? PB_MIXED : PB_FP64;
    const T* qw = f32 ? (const T*)M->qw_f.p : (const T*)M->qw_d.p;
    const T* qp = f32 ? (const T*)M->qp_f.p : (const T*)M->qp_d.p;
    const T* qn = f32 ? (const T*)M->qn_f.p : (const T*)M->qn_d.p;
    DBuf<T> mL, mY, pL, dL, pY, dY;
    mL.alloc(np, st); mY.alloc(np, st); pL.alloc(np, st); dL.alloc(np, st); pY.alloc(np, st); dY.alloc(np, st);
    {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        k_p1_adj<T><<<div_up(np, 256), 256, 0, st>>>(nt, nq, lam, qw, mL.p, mY.p);
        PB_CHECK_LAUNCH();
    }
    fmm_apply_pair_impl(M->tree, R->kappa, M->p, prec, mL.p, mY.p, nullptr, nullptr, qn, pL.p, pY.p, dL.p, dY.p);
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    k_combine_adj<T><<<div_up(nt, 128), 128, 0, st>>>(nt, nq, lam, pL.p, dL.p, pY.p, dY.p, qp, qn, qw, M->adj_off.p,
                                                      M->adj_ids.p, M->adj_tr.p, M->S_d.p, M->area.p,
                                                      R->eps_in / R->eps_out, R->kappa, y);
    PB_CHECK_LAUNCH();
}

// y = P^{-T} A^T lam (precond = 1 always)
void adjoint_matvec(pb_mesh* M, const pb_result* R, const double* lam, double* y) {
    ensure_singular_public(M, R->kappa);
    ensure_adj_transpose(M);
    if (R->precision == PB_FP64) adj_matvec_t<double>(M, R, lam, y);
    else adj_matvec_t<float>(M, R, lam, y);
}

bool use_fmm_coupling(const pb_mesh* M, const pb_result* R);
void ensure_coupling_trees(pb_mesh* M, pb_result* R);

int energy_gradient(pb_result* R, double tol, int max_iter, double* dEdq_host, double* dEdx_host) {
    pb_mesh* M = R->mesh;
    cudaStream_t st = M->ctx->stream;
    ensure_singular_public(M, R->kappa);
    ensure_adj_transpose(M);
    const int nt = (int)M->nt, nq = M->nq;
    const long long np = (long long)nt * nq;
    DBuf<double> c, gq, gx;
    c.alloc(2 * nt, st);
    if (use_fmm_coupling(M, R)) {
        // charges (scaled by 1/eps1 in q_f; undone below) -> potential and
        // normal derivative at the quadrature points
        ensure_coupling_trees(M, R);
        DBuf<float> pot, dn;
        pot.alloc(np, st); dn.alloc(np, st);
        fmm_apply_impl(R->tree_aq, FMM_LAPLACE, 0.0, M->p, PB_MIXED, R->q_f.p, nullptr, nullptr, M->qn_f.p, pot.p,
                       dn.p);
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        k_adj_rhs_fmm<<<div_up(nt, 128), 128, 0, st>>>(nt, nq, M->qw_d.p, pot.p, dn.p, R->eps_in, M->adj_off.p,
                                                       M->adj_ids.p, M->S_d.p, M->area.p, R->eps_in / R->eps_out, c.p);
        PB_CHECK_LAUNCH();
    } else {
        PhaseTimer ph(M->ctx, PB_PH_BEM);
        k_adj_rhs<<<div_up(nt, 128), 128, 0, st>>>(nt, nq, M->qp_d.p, M->qn_d.p, M->qw_d.p, (int)R->na,
                                                   (const double4*)R->atoms.p, M->adj_off.p, M->adj_ids.p, M->S_d.p,
                                                   M->area.p, R->eps_in / R->eps_out, c.p);
        PB_CHECK_LAUNCH();
    }
    auto mv = [&](const double* v, double* w) { adjoint_matvec(M, R, v, w); };
    int status = gmres(M, mv, c.p, R->lambda, tol, max_iter, &R->adj_iterations, &R->adj_residual);
    gq.alloc(R->na, st);
    gx.alloc(3 * R->na, st);
    PhaseTimer ph(M->ctx, PB_PH_BEM);
    k_atom_grad<<<div_up(R->na, 128), 128, 0, st>>>((int)R->na, (const double4*)R->atoms.p, np, nq, nt, M->qp_d.p,
                                                    M->qn_d.p, M->qw_d.p, R->x.p, R->lambda.p, 1.0 / R->eps_in, gq.p,
                                                    gx.p);
    PB_CHECK_LAUNCH();
    if (dEdq_host) PB_CUDA(cudaMemcpyAsync(dEdq_host, gq.p, R->na * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dEdx_host) PB_CUDA(cudaMemcpyAsync(dEdx_host, gx.p, 3 * R->na * sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    return status;
}

}  // namespace pbfmm
