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
// K^T K = V diag(mu) V^T (cyclic Jacobi, FP64, on the host) and
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

__global__ void k_matmul(int n, const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int i = idx / n, j = idx % n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
    C[idx] = s;
}

// Symmetric eigendecomposition A = V diag(w) V^T by the cyclic Jacobi method
// (plane rotations that annihilate one off-diagonal entry each, with the
// rotation angle from theta = (a_qq - a_pp) / (2 a_pq), t = sgn(theta) /
// (|theta| + sqrt(theta^2 + 1))). A (n x n, row-major) is overwritten.
static void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int i = 0; i < n; ++i) {
            dg += A[(size_t)i * n + i] * A[(size_t)i * n + i];
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        }
        if (off <= 1e-32 * dg) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                if (std::fabs(apq) <= 1e-18 * std::sqrt(std::fabs(app * aqq))) {
                    A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                    continue;
                }
                const double th = (aqq - app) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Factored Tikhonov pseudo-inverse of K(check surface at scale tscale,
// equivalent surface at scale sscale), both centred at the origin:
// W1 = D V^T K^T and W2 = V, written padded to npad x npad in FP32.
static void factored_pinv(int n, int npad, int kernel, double kappa, const std::vector<double>& surf, double tscale,
                          double sscale, float* W1, float* W2) {
    std::vector<double> K((size_t)n * n), G((size_t)n * n), V, mu;
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
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a += K[(size_t)k * n + i] * K[(size_t)k * n + j];
            G[(size_t)i * n + j] = G[(size_t)j * n + i] = a;
        }
    jacobi_eig(n, G, V, mu);
    const double lam = 1e-14 * fro;
    std::fill(W1, W1 + (size_t)npad * npad, 0.f);
    std::fill(W2, W2 + (size_t)npad * npad, 0.f);
    for (int j = 0; j < n; ++j) {
        const double d = 1.0 / (std::max(mu[j], 0.0) + lam);
        for (int i = 0; i < n; ++i) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a += K[(size_t)i * n + k] * V[(size_t)k * n + j];
            W1[(size_t)j * npad + i] = (float)(d * a);
        }
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
            for (int c = 0; c < 8; ++c) {
                const double cc[3] = {((c >> 2) & 1) ? r : -r, ((c >> 1) & 1) ? r : -r, (c & 1) ? r : -r};
                // M2M_l[c] = UC2UE_{l-1} K(parent uc, child ue); parent half-width 2r
                Bd.kmat(Bd.C.p, zero, kAlphaOuter * 2 * r, cc, kAlphaInner * r);
                k_matmul<<<div_up((long long)n * n, 256), 256, 0, st>>>(n, uc2ue_prev.p, Bd.C.p, Bd.A.p);
                Bd.store(Bd.A.p, O->m2m.p + ((size_t)l * 8 + c) * m2,
                         need_fp64 ? O->m2m_d.p + ((size_t)l * 8 + c) * m2 : nullptr, np);
                // L2L_l[c] = DC2DE_l K(child dc, parent de)
                Bd.kmat(Bd.C.p, cc, kAlphaInner * r, zero, kAlphaOuter * 2 * r);
                k_matmul<<<div_up((long long)n * n, 256), 256, 0, st>>>(n, dc.p, Bd.C.p, Bd.A.p);
                Bd.store(Bd.A.p, O->l2l.p + ((size_t)l * 8 + c) * m2,
                         need_fp64 ? O->l2l_d.p + ((size_t)l * 8 + c) * m2 : nullptr, np);
            }
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
            for (int o = 0; o < kNumOffsets; ++o) {
                int ox = o / 49 - 3, oy = (o / 7) % 7 - 3, oz = o % 7 - 3;
                if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
                const double sc[3] = {2 * r * ox, 2 * r * oy, 2 * r * oz};
                Bd.kmat(Bd.C.p, zero, kAlphaInner * r, sc, kAlphaInner * r);
                k_matmul<<<div_up((long long)n * n, 256), 256, 0, st>>>(n, dc.p, Bd.C.p, Bd.A.p);
                Bd.store(Bd.A.p, O->m2l.p + ((size_t)l * kNumOffsets + o) * m2,
                         need_fp64 ? O->m2l_d.p + ((size_t)l * kNumOffsets + o) * m2 : nullptr, np);
            }
        }
        PB_CHECK_LAUNCH();
    }
    // factored UC2UE / DC2DE for the FP32 path: one host job per level and
    // direction, spread over the host cores
    {
        std::vector<float> w1((size_t)2 * L * m2), w2((size_t)2 * L * m2);
        std::atomic<int> next(0);
        auto work = [&]() {
            for (int job; (job = next.fetch_add(1)) < 2 * L;) {
                const int l = job / 2;
                const bool up = (job % 2) == 0;
                const double r = std::ldexp(T->R, -l);
                factored_pinv(n, np, kernel, kappa, s, (up ? kAlphaOuter : kAlphaInner) * r,
                              (up ? kAlphaInner : kAlphaOuter) * r, w1.data() + (size_t)job * m2,
                              w2.data() + (size_t)job * m2);
            }
        };
        const int nth = std::max(1, std::min<int>(2 * L, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
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
    return O;
}

}  // namespace pbfmm
