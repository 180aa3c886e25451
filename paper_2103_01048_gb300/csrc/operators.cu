// Precomputation of the KIFMM translation operators (the "invariant
// matrices" the paper pre-computes and caches, Sec. "Fast multipole method"
// and the assembly-time discussion of the performance study).
//
// For each level l (box half-width r_l = R / 2^l), all in FP64 on the GPU:
//   UC2UE_l = pinv(K(upward check, upward equivalent))      [Eq. multipole_local]
//   DC2DE_l = pinv(K(downward check, downward equivalent))
//   M2M_l[c] = UC2UE_{l-1} K(parent upward check, child-c upward equivalent)
//   L2L_l[c] = DC2DE_l K(child-c downward check, parent downward equivalent)
//   M2L_l[o] = DC2DE_l K(downward check of B, upward equivalent of the box at offset o)
// The pseudo-inverses have norms ~1e6-1e7, so a product with one of them
// computed in FP32 loses every digit; folded into the translations above
// (in FP64) the operators have norms of order 1-100 and are stored in FP32.
// UC2UE / DC2DE themselves are needed where raw check potentials are
// converted (P2M at leaves, P2L of X lists): in FP64 for the all-FP64 path,
// and for the FP32 path in factored form, pinv = V D V^T K^T with
// K^T K = V diag(mu) V^T (Householder tridiagonalisation and implicit
// symmetric QR, FP64, on the host) and
// D = diag(1 / (mu + lam)): W1 = D V^T K^T and W2 = V are well scaled, and the
// FP32 rounding of W1 x is amplified only along eigenvectors of small mu,
// whose equivalent densities produce correspondingly small fields away from
// the surfaces (the part of the potential the FMM uses).
// The paper says only "solve the linear systems"; the regularised solve used
// here is Tikhonov: pinv(K) = (K^T K + lam I)^{-1} K^T with
// lam = (1e-7 ||K||_F)^2, by a Cholesky factorisation (FP64 path) or the
// eigendecomposition above (FP32 path).
#include "fmm.cuh"
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace pbfmm {

constexpr double kInv4Pi = 0.07957747154594767;   // 1/(4 pi)

__global__ void k_kernel_matrix(int ne, int kernel, double kappa, const double* __restrict__ surf,
                                double tcx, double tcy, double tcz, double ts,
                                double scx, double scy, double scz, double ss, double* __restrict__ out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ne * ne) return;
    int i = idx / ne, j = idx % ne;
    double dx = (tcx + ts * surf[3 * i]) - (scx + ss * surf[3 * j]);
    double dy = (tcy + ts * surf[3 * i + 1]) - (scy + ss * surf[3 * j + 1]);
    double dz = (tcz + ts * surf[3 * i + 2]) - (scz + ss * surf[3 * j + 2]);
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double g = kInv4Pi / r;
    if (kernel == FMM_YUKAWA) g *= exp(-kappa * r);
    out[idx] = g;
}

__global__ void k_sumsq(int n, const double* a, double* out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * a[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// G = K^T K + lam I,  lam = eps^2 * sumsq(K)
__global__ void k_gram(int n, const double* __restrict__ K, const double* sumsq, double eps2, double* __restrict__ G) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int i = idx / n, j = idx % n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += K[k * n + i] * K[k * n + j];
    if (i == j) s += eps2 * sumsq[0];
    G[idx] = s;
}

// In-place lower Cholesky factor of G (one CTA).
__global__ void k_cholesky(int n, double* G) {
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            double d = G[k * n + k];
            piv = sqrt(d > 0.0 ? d : 1e-300);
            G[k * n + k] = piv;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) G[i * n + k] /= piv;
        __syncthreads();
        int m = n - k - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int i = k + 1 + t / m, j = k + 1 + t % m;
            if (j <= i) G[i * n + j] -= G[i * n + k] * G[j * n + k];
        }
        __syncthreads();
    }
}

// X = G^{-1} K^T with G = L L^T: column j of X solves G x = (row j of K)^T.
__global__ void k_chol_solve(int n, const double* __restrict__ L, const double* __restrict__ K, double* __restrict__ X) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int k = 0; k < n; ++k) {                 // L y = b
        double s = K[j * n + k];
        for (int m = 0; m < k; ++m) s -= L[k * n + m] * X[m * n + j];
        X[k * n + j] = s / L[k * n + k];
    }
    for (int k = n - 1; k >= 0; --k) {            // L^T x = y
        double s = X[k * n + j];
        for (int m = k + 1; m < n; ++m) s -= L[m * n + k] * X[m * n + j];
        X[k * n + j] = s / L[k * n + k];
    }
}

// Symmetric eigendecomposition A = V diag(w) V^T (A n x n, row-major,
// overwritten; V[k * n + j] = component k of eigenvector j) in two stages:
//  1. Householder tridiagonalisation Q^T A Q = T: reflection k maps the part
//     of column k below the diagonal onto its first entry; the trailing
//     block is updated as S - v w^T - w v^T with p = beta S v,
//     w = p - (beta / 2)(v . p) v; Q^T = H_{n-3} ... H_0 is accumulated.
//  2. Implicit symmetric QR steps with the Wilkinson shift (the eigenvalue
//     of the trailing 2 x 2 block of the unreduced part nearer its last
//     diagonal entry) on T, chasing the bulge with Givens rotations that
//     are applied to the rows of Q^T as well; off-diagonal entries below
//     eps (|d_i| + |d_i+1|) are set to zero and split the problem.
// O(n^3) in all with unit-stride inner loops.
static void sym_eig(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
    std::vector<double> d(n, 0.0), e(std::max(n - 1, 1), 0.0), Zt((size_t)n * n, 0.0), vv(n), pv(n), wv(n);
    for (int i = 0; i < n; ++i) Zt[(size_t)i * n + i] = 1.0;
    // 1. tridiagonalisation
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;                  // trailing size
        const double* row = &A[(size_t)k * n + k + 1];   // column k below the diagonal (symmetric)
        double xn = 0.0;
        for (int i = 0; i < m; ++i) xn += row[i] * row[i];
        xn = std::sqrt(xn);
        d[k] = A[(size_t)k * n + k];
        if (xn == 0.0) { e[k] = 0.0; continue; }
        const double alpha = row[0] > 0 ? -xn : xn;
        for (int i = 0; i < m; ++i) vv[i] = row[i];
        vv[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < m; ++i) vn2 += vv[i] * vv[i];
        e[k] = alpha;
        if (vn2 == 0.0) continue;
        const double beta = 2.0 / vn2;
        // p = beta S v, S = A[k+1.., k+1..]
        for (int i = 0; i < m; ++i) {
            const double* Si = &A[(size_t)(k + 1 + i) * n + k + 1];
            double acc = 0.0;
            for (int j = 0; j < m; ++j) acc += Si[j] * vv[j];
            pv[i] = beta * acc;
        }
        double vp = 0.0;
        for (int i = 0; i < m; ++i) vp += vv[i] * pv[i];
        const double K = 0.5 * beta * vp;
        for (int i = 0; i < m; ++i) wv[i] = pv[i] - K * vv[i];
        for (int i = 0; i < m; ++i) {
            double* Si = &A[(size_t)(k + 1 + i) * n + k + 1];
            const double vi = vv[i], wi = wv[i];
            for (int j = 0; j < m; ++j) Si[j] -= vi * wv[j] + wi * vv[j];
        }
        // Q^T <- H_k Q^T: rows k+1 .. n-1 of Zt
        for (int j = 0; j < n; ++j) pv[j] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double* Zi = &Zt[(size_t)(k + 1 + i) * n];
            const double vi = vv[i];
            for (int j = 0; j < n; ++j) pv[j] += vi * Zi[j];
        }
        for (int i = 0; i < m; ++i) {
            double* Zi = &Zt[(size_t)(k + 1 + i) * n];
            const double f = beta * vv[i];
            for (int j = 0; j < n; ++j) Zi[j] -= f * pv[j];
        }
    }
    if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
        e[n - 2] = A[(size_t)(n - 1) * n + n - 2];
    }
    d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
    // 2. implicit symmetric QR with Wilkinson shifts
    const double eps = 2.220446049250313e-16;
    auto small = [&](int i) { return std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1])); };
    int hi = n - 1, guard = 0;
    while (hi > 0 && guard < 60 * n) {
        if (small(hi - 1)) { e[hi - 1] = 0.0; --hi; continue; }
        int lo = hi - 1;
        while (lo > 0 && !small(lo - 1)) --lo;
        ++guard;
        // shift: eigenvalue of [[d_{hi-1}, e_{hi-1}], [e_{hi-1}, d_hi]] nearer d_hi
        const double b = e[hi - 1], delta = 0.5 * (d[hi - 1] - d[hi]);
        const double den = delta + (delta >= 0 ? 1.0 : -1.0) * std::hypot(delta, b);
        const double mu = d[hi] - b * b / den;
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = std::hypot(x, z);
            const double c = r > 0 ? x / r : 1.0, sn = r > 0 ? z / r : 0.0;
            if (k > lo) e[k - 1] = r;
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk + 2.0 * c * sn * ek + sn * sn * dk1;
            d[k + 1] = sn * sn * dk - 2.0 * c * sn * ek + c * c * dk1;
            e[k] = c * sn * (dk1 - dk) + (c * c - sn * sn) * ek;
            if (k + 1 < hi) {
                z = sn * e[k + 1];               // bulge at (k + 2, k)
                e[k + 1] *= c;
                x = e[k];
            }
            double* Zk = &Zt[(size_t)k * n];
            double* Zk1 = &Zt[(size_t)(k + 1) * n];
            for (int j = 0; j < n; ++j) {
                const double a0 = Zk[j], a1 = Zk1[j];
                Zk[j] = c * a0 + sn * a1;
                Zk1[j] = -sn * a0 + c * a1;
            }
        }
    }
    w = d;
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) V[(size_t)k * n + j] = Zt[(size_t)j * n + k];
}

// Factored Tikhonov pseudo-inverse of K(check surface at scale tscale,
// equivalent surface at scale sscale), both centred at the origin:
// W1 = D V^T K^T and W2 = V, written padded to npad x npad in FP32.
static void factored_pinv(int n, int npad, int kernel, double kappa, const std::vector<double>& surf, double tscale,
                          double sscale, float* W1, float* W2) {
    std::vector<double> K((size_t)n * n), G((size_t)n * n, 0.0), V, mu, KV((size_t)n * n, 0.0);
    double fro = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double dx = tscale * surf[3 * i] - sscale * surf[3 * j];
            const double dy = tscale * surf[3 * i + 1] - sscale * surf[3 * j + 1];
            const double dz = tscale * surf[3 * i + 2] - sscale * surf[3 * j + 2];
            const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            double g = kInv4Pi / r;
            if (kernel == FMM_YUKAWA) g *= std::exp(-kappa * r);
            K[(size_t)i * n + j] = g;
            fro += g * g;
        }
    // G = K^T K (upper triangle by rows of K, then mirrored)
    for (int k = 0; k < n; ++k) {
        const double* Kk = &K[(size_t)k * n];
        for (int i = 0; i < n; ++i) {
            const double a = Kk[i];
            double* Gi = &G[(size_t)i * n];
            for (int j = i; j < n; ++j) Gi[j] += a * Kk[j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) G[(size_t)i * n + j] = G[(size_t)j * n + i];
    sym_eig(n, G, V, mu);
    const double lam = 1e-14 * fro;
    // KV = K V
    for (int i = 0; i < n; ++i) {
        double* KVi = &KV[(size_t)i * n];
        for (int k = 0; k < n; ++k) {
            const double a = K[(size_t)i * n + k];
            const double* Vk = &V[(size_t)k * n];
            for (int j = 0; j < n; ++j) KVi[j] += a * Vk[j];
        }
    }
    std::fill(W1, W1 + (size_t)npad * npad, 0.f);
    std::fill(W2, W2 + (size_t)npad * npad, 0.f);
    for (int j = 0; j < n; ++j) {
        const double dj = 1.0 / (std::max(mu[j], 0.0) + lam);
        for (int i = 0; i < n; ++i) W1[(size_t)j * npad + i] = (float)(dj * KV[(size_t)i * n + j]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) W2[(size_t)i * npad + j] = (float)V[(size_t)i * n + j];
}

__global__ void k_store_padded(int n, int npad, const double* __restrict__ src, float* __restrict__ dst_f,
                               double* __restrict__ dst_d) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npad * npad) return;
    int i = idx / npad, j = idx % npad;
    double v = (i < n && j < n) ? src[i * n + j] : 0.0;
    if (dst_f) dst_f[idx] = (float)v;
    if (dst_d) dst_d[idx] = v;
}

// Translation operators of one level in one launch: for every z (M2L: the
// 343 relative offsets, the 27 near ones skipped; M2M / L2L: the 8 child
// octants) C_z = P K_z with P the level's pseudo-inverse (n x n, FP64) and
// K_z[k][j] = g(t_z + ts u_k, s_z + ss u_j) generated on the fly from the
// unit surface u.  Tiled FP64 GEMM: 64 x 64 outputs per CTA, 4 x 4 per thread,
// 16-wide K steps through shared memory; written padded to npad x npad (FP32
// and, if dst_d, FP64) at dst + z * npad^2.
enum { OPB_M2L = 0, OPB_M2M = 1, OPB_L2L = 2 };
constexpr int kOpTile = 64, kOpK = 16;

__global__ void __launch_bounds__(256) k_build_ops(int n, int npad, int mode, int kernel, double kappa,
                                                   const double* __restrict__ surf, const double* __restrict__ P,
                                                   double r, double ts, double ss, float* __restrict__ dst_f,
                                                   double* __restrict__ dst_d) {
    const int z = blockIdx.z;
    double tc[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
    if (mode == OPB_M2L) {
        const int ox = z / 49 - 3, oy = (z / 7) % 7 - 3, oz = z % 7 - 3;
        if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) return;   // near offsets: no operator
        sc[0] = 2 * r * ox; sc[1] = 2 * r * oy; sc[2] = 2 * r * oz;
    } else {
        const double cc[3] = {((z >> 2) & 1) ? r : -r, ((z >> 1) & 1) ? r : -r, (z & 1) ? r : -r};
        for (int a = 0; a < 3; ++a) (mode == OPB_M2M ? sc : tc)[a] = cc[a];
    }
    __shared__ double sA[kOpTile][kOpK + 1];
    __shared__ double sB[kOpK][kOpTile + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * kOpTile, j0 = blockIdx.x * kOpTile;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += kOpK) {
        for (int e = threadIdx.x; e < kOpTile * kOpK; e += 256) {
            const int ii = e / kOpK, kk = e % kOpK;
            const int i = i0 + ii, k = k0 + kk;
            sA[ii][kk] = (i < n && k < n) ? P[(size_t)i * n + k] : 0.0;
        }
        for (int e = threadIdx.x; e < kOpK * kOpTile; e += 256) {
            const int kk = e / kOpTile, jj = e % kOpTile;
            const int k = k0 + kk, j = j0 + jj;
            double g = 0.0;
            if (k < n && j < n) {
                const double dx = (tc[0] + ts * surf[3 * k]) - (sc[0] + ss * surf[3 * j]);
                const double dy = (tc[1] + ts * surf[3 * k + 1]) - (sc[1] + ss * surf[3 * j + 1]);
                const double dz = (tc[2] + ts * surf[3 * k + 2]) - (sc[2] + ss * surf[3 * j + 2]);
                const double rr = sqrt(dx * dx + dy * dy + dz * dz);
                g = kInv4Pi / rr;
                if (kernel == FMM_YUKAWA) g *= exp(-kappa * rr);
            }
            sB[kk][jj] = g;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kOpK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = sA[ty + 16 * u][kk];
                b[u] = sB[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
    const size_t m2 = (size_t)npad * npad;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i < n && j < n) {
                dst_f[(size_t)z * m2 + (size_t)i * npad + j] = (float)acc[u][v];
                if (dst_d) dst_d[(size_t)z * m2 + (size_t)i * npad + j] = acc[u][v];
            }
        }
}

static void build_ops(cudaStream_t st, int n, int npad, int mode, int kernel, double kappa, const double* surf,
                      const double* P, double r, double ts, double ss, float* dst_f, double* dst_d) {
    const int nz = mode == OPB_M2L ? kNumOffsets : 8;
    dim3 grid(div_up(n, kOpTile), div_up(n, kOpTile), nz);
    k_build_ops<<<grid, 256, 0, st>>>(n, npad, mode, kernel, kappa, surf, P, r, ts, ss, dst_f, dst_d);
    PB_CHECK_LAUNCH();
}

namespace {

struct Builder {
    cudaStream_t st;
    int n, kernel;
    double kappa;
    const double* surf;
    DBuf<double> A, B, C, G, ss;
    Builder(cudaStream_t s, int ne, int k, double kap, const double* su) : st(s), n(ne), kernel(k), kappa(kap), surf(su) {
        A.alloc((size_t)n * n, st); B.alloc((size_t)n * n, st); C.alloc((size_t)n * n, st);
        G.alloc((size_t)n * n, st); ss.alloc(1, st);
    }
    void kmat(double* out, const double tc[3], double ts, const double sc[3], double sscale) {
        k_kernel_matrix<<<div_up((long long)n * n, 256), 256, 0, st>>>(n, kernel, kappa, surf, tc[0], tc[1], tc[2], ts,
                                                                      sc[0], sc[1], sc[2], sscale, out);
        PB_CHECK_LAUNCH();
    }
    // out = pinv(Kin)  (Kin is destroyed)
    void pinv(const double* Kin, double* out) {
        k_sumsq<<<1, 1024, 0, st>>>(n * n, Kin, ss.p);
        k_gram<<<div_up((long long)n * n, 256), 256, 0, st>>>(n, Kin, ss.p, 1e-14, G.p);
        k_cholesky<<<1, 1024, 0, st>>>(n, G.p);
        k_chol_solve<<<div_up(n, 64), 64, 0, st>>>(n, G.p, Kin, out);
        PB_CHECK_LAUNCH();
    }
    void store(const double* src, float* f, double* d, int npad) {
        k_store_padded<<<div_up((long long)npad * npad, 256), 256, 0, st>>>(n, npad, src, f, d);
        PB_CHECK_LAUNCH();
    }
};

}  // namespace

void pack_m2l_tc(Operators& O, cudaStream_t st);

std::shared_ptr<Operators> get_operators(fmm_tree* T, int kernel, double kappa, int p, bool need_fp64) {
    auto key = std::make_tuple(kernel, kernel == FMM_YUKAWA ? kappa : 0.0, p, T->nlev);
    auto it = T->ops.find(key);
    if (it != T->ops.end() && (!need_fp64 || it->second->have_d)) return it->second;
    // another tree of the context with the same box sizes may hold the set
    const auto gkey = std::make_tuple(kernel, kernel == FMM_YUKAWA ? kappa : 0.0, p, T->R, T->nlev);
    {
        auto g = T->ctx->op_cache.find(gkey);
        if (g != T->ctx->op_cache.end()) {
            auto sp = std::static_pointer_cast<Operators>(g->second.lock());
            if (sp && (!need_fp64 || sp->have_d)) {
                T->ops[key] = sp;
                return sp;
            }
        }
    }
    cudaStream_t st = T->ctx->stream;
    auto O = std::make_shared<Operators>();
    O->kernel = kernel;
    O->kappa = kappa;
    O->p = p;
    O->ne = surface_count(p);
    O->npad = pad32(O->ne);
    O->nlev = T->nlev;
    const int n = O->ne, np = O->npad, L = T->nlev;
    // unit surface: boundary points of the p x p x p grid on [-1, 1]^3
    std::vector<double> s;
    std::vector<float> sf;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                if (i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1) {
                    double x = -1.0 + 2.0 * i / (p - 1), y = -1.0 + 2.0 * j / (p - 1), z = -1.0 + 2.0 * k / (p - 1);
                    s.push_back(x); s.push_back(y); s.push_back(z);
                    sf.push_back((float)x); sf.push_back((float)y); sf.push_back((float)z); sf.push_back(0.f);
                }
            }
    O->surf.alloc(s.size(), st);
    O->surf_f.alloc(sf.size(), st);
    PB_CUDA(cudaMemcpyAsync(O->surf.p, s.data(), s.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(O->surf_f.p, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    const size_t m2 = (size_t)np * np;
    O->uc2ue_d.alloc(L * m2, st); O->dc2de_d.alloc(L * m2, st);
    O->m2m.alloc(L * 8 * m2, st); O->l2l.alloc(L * 8 * m2, st);
    O->m2l.alloc(L * (size_t)kNumOffsets * m2, st);
    O->m2m.zero(st); O->l2l.zero(st); O->m2l.zero(st);
    if (need_fp64) {
        O->m2m_d.alloc(L * 8 * m2, st); O->l2l_d.alloc(L * 8 * m2, st);
        O->m2l_d.alloc(L * (size_t)kNumOffsets * m2, st);
        O->m2m_d.zero(st); O->l2l_d.zero(st); O->m2l_d.zero(st);
        O->have_d = true;
    }
    Builder Bd(st, n, kernel, kappa, O->surf.p);
    DBuf<double> uc2ue_prev, dc;
    uc2ue_prev.alloc((size_t)n * n, st);
    dc.alloc((size_t)n * n, st);
    const double zero[3] = {0, 0, 0};
    for (int l = 0; l < L; ++l) {
        const double r = std::ldexp(T->R, -l);
        // UC2UE_l, DC2DE_l
        Bd.kmat(Bd.A.p, zero, kAlphaOuter * r, zero, kAlphaInner * r);
        Bd.pinv(Bd.A.p, Bd.B.p);
        Bd.store(Bd.B.p, nullptr, O->uc2ue_d.p + l * m2, np);
        // DC2DE_l (kept in Bd.G's sibling buffer `dc`)
        Bd.kmat(Bd.A.p, zero, kAlphaInner * r, zero, kAlphaOuter * r);
        Bd.pinv(Bd.A.p, dc.p);
        Bd.store(dc.p, nullptr, O->dc2de_d.p + l * m2, np);
        if (l > 0) {
            // M2M_l[c] = UC2UE_{l-1} K(parent uc, child-c ue); parent half-width 2r
            build_ops(st, n, np, OPB_M2M, kernel, kappa, O->surf.p, uc2ue_prev.p, r, kAlphaOuter * 2 * r,
                      kAlphaInner * r, O->m2m.p + (size_t)l * 8 * m2, need_fp64 ? O->m2m_d.p + (size_t)l * 8 * m2 : nullptr);
            // L2L_l[c] = DC2DE_l K(child-c dc, parent de)
            build_ops(st, n, np, OPB_L2L, kernel, kappa, O->surf.p, dc.p, r, kAlphaInner * r, kAlphaOuter * 2 * r,
                      O->l2l.p + (size_t)l * 8 * m2, need_fp64 ? O->l2l_d.p + (size_t)l * 8 * m2 : nullptr);
        }
        PB_CUDA(cudaMemcpyAsync(uc2ue_prev.p, Bd.B.p, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // M2L_l[o] = DC2DE_l K(dc of B, ue of the box at offset o); the
        // Laplace operators do not depend on the level (1/r scales as 2^l,
        // the regularised pseudo-inverse as 2^-l): levels below take level 2's
        if (l > 2 && kernel == FMM_LAPLACE) {
            const size_t blk = (size_t)kNumOffsets * m2;
            PB_CUDA(cudaMemcpyAsync(O->m2l.p + l * blk, O->m2l.p + 2 * blk, blk * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
            if (need_fp64)
                PB_CUDA(cudaMemcpyAsync(O->m2l_d.p + l * blk, O->m2l_d.p + 2 * blk, blk * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st));
        } else if (l >= 2) {
            build_ops(st, n, np, OPB_M2L, kernel, kappa, O->surf.p, dc.p, r, kAlphaInner * r, kAlphaInner * r,
                      O->m2l.p + (size_t)l * kNumOffsets * m2,
                      need_fp64 ? O->m2l_d.p + (size_t)l * kNumOffsets * m2 : nullptr);
        }
        PB_CHECK_LAUNCH();
    }
    // factored UC2UE / DC2DE for the FP32 path: one host job per level and
    // direction, spread over the host cores
    {
        std::vector<float> w1((size_t)2 * L * m2), w2((size_t)2 * L * m2);
        std::atomic<int> next(0);
        // Laplace: K scales as 2^l with the level, so the eigenvectors are the
        // same and W1 scales as 2^-l (exact in FP32): decompose level 0 only
        const int njobs = kernel == FMM_LAPLACE ? 2 : 2 * L;
        auto work = [&]() {
            for (int job; (job = next.fetch_add(1)) < njobs;) {
                const int l = job / 2;
                const bool up = (job % 2) == 0;
                const double r = std::ldexp(T->R, -l);
                factored_pinv(n, np, kernel, kappa, s, (up ? kAlphaOuter : kAlphaInner) * r,
                              (up ? kAlphaInner : kAlphaOuter) * r, w1.data() + (size_t)job * m2,
                              w2.data() + (size_t)job * m2);
            }
        };
        const int nth = std::max(1, std::min<int>(njobs, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
        for (int job = njobs; job < 2 * L; ++job) {
            const int l = job / 2;
            const float sc = std::ldexp(1.0f, -l);
            for (size_t e = 0; e < m2; ++e) {
                w1[(size_t)job * m2 + e] = sc * w1[(size_t)(job % 2) * m2 + e];
                w2[(size_t)job * m2 + e] = w2[(size_t)(job % 2) * m2 + e];
            }
        }
        // [job = 2 l + (0 up, 1 down)] -> [level] per direction
        std::vector<float> u1((size_t)L * m2), u2((size_t)L * m2), d1((size_t)L * m2), d2((size_t)L * m2);
        for (int l = 0; l < L; ++l) {
            std::copy_n(w1.data() + (size_t)(2 * l) * m2, m2, u1.data() + (size_t)l * m2);
            std::copy_n(w2.data() + (size_t)(2 * l) * m2, m2, u2.data() + (size_t)l * m2);
            std::copy_n(w1.data() + (size_t)(2 * l + 1) * m2, m2, d1.data() + (size_t)l * m2);
            std::copy_n(w2.data() + (size_t)(2 * l + 1) * m2, m2, d2.data() + (size_t)l * m2);
        }
        O->uc2ue_w1.alloc(L * m2, st); O->uc2ue_w2.alloc(L * m2, st);
        O->dc2de_w1.alloc(L * m2, st); O->dc2de_w2.alloc(L * m2, st);
        PB_CUDA(cudaMemcpyAsync(O->uc2ue_w1.p, u1.data(), L * m2 * sizeof(float), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(O->uc2ue_w2.p, u2.data(), L * m2 * sizeof(float), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(O->dc2de_w1.p, d1.data(), L * m2 * sizeof(float), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(O->dc2de_w2.p, d2.data(), L * m2 * sizeof(float), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaStreamSynchronize(st));    // the host vectors go out of scope
    }
    pack_m2l_tc(*O, st);
    PB_CUDA(cudaStreamSynchronize(st));
    T->ops[key] = O;
    auto& cache = T->ctx->op_cache;
    for (auto g = cache.begin(); g != cache.end();) g = g->second.expired() ? cache.erase(g) : std::next(g);
    cache[gkey] = std::static_pointer_cast<void>(O);
    return O;
}

}  // namespace pbfmm

// test hook (include/pbfmm_testing.h): the host eigensolver of the factored
// pseudo-inverses; no GPU involved
extern "C" int pbfmm_test_sym_eig(int n, const double* A, double* w, double* V) {
    if (n < 1 || !A || !w || !V) return PB_EINVAL;
    std::vector<double> a(A, A + (size_t)n * n), vv, ww;
    pbfmm::sym_eig(n, a, vv, ww);
    std::copy(ww.begin(), ww.end(), w);
    std::copy(vv.begin(), vv.end(), V);
    return PB_OK;
}
