// Batched solves of many systems and an ncrit autotuner.
//
// pb_solve_batch runs the GMRES iterations of several meshes in lockstep:
// each system gets its own CUDA stream, its preconditioned mat-vec (P1, the
// Laplace and Yukawa FMM passes, the fused Galerkin glue) is captured once
// as a CUDA graph and replayed every iteration, and one host synchronisation
// per iteration reads all the residuals.  Small systems therefore overlap
// on the GPU instead of running one after another, and the ~60 launches of
// a mat-vec cost one graph launch.
#include "bem.cuh"
#include <algorithm>
#include <cmath>
#include <memory>

namespace pbfmm {

void check_device_error(pb_ctx* ctx);
void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn);
void build_tree(fmm_tree* T, const float* src, const float* tgt);

// kernels of bem.cu reused here
__global__ void k_coulomb(long long np, const double* __restrict__ qp, int na, const double4* __restrict__ atoms,
                          double inv_eps, double* __restrict__ f);
__global__ void k_rhs(int nt, int nq, const double* __restrict__ f, const double* __restrict__ qw,
                      const int* __restrict__ adj_off, const int* __restrict__ adj_ids, const double* __restrict__ S,
                      const double* __restrict__ area, double er, int precond, double* __restrict__ b);
__global__ void k_dots(long long n, const double* __restrict__ V, long long ld, int nk, const double* __restrict__ w,
                       double* __restrict__ partial, int kmax);
__global__ void k_dots_reduce(int nblk, int nk, const double* __restrict__ partial, int kmax, double* __restrict__ h,
                              int accumulate);
__global__ void k_update(long long n, const double* __restrict__ V, long long ld, int nk, const double* __restrict__ h,
                         double* __restrict__ w);
__global__ void k_scale(long long n, const double* __restrict__ w, const double* __restrict__ nrm2,
                        double* __restrict__ out);
__global__ void k_givens(int j, int kmax, const double* __restrict__ h, const double* __restrict__ nrm2, double* H,
                         double* cs, double* sn, double* g, double* resid);
__global__ void k_backsolve(int m, int kmax, const double* __restrict__ H, const double* __restrict__ g, double* y);
__global__ void k_axpy_basis(long long n, const double* __restrict__ V, long long ld, int m,
                             const double* __restrict__ y, double* __restrict__ x);
__global__ void k_set_g0(const double* nrm2, double* g);
__global__ void k_vadd(int n, const double* a, double* b);

constexpr int kDotBlocksB = 304;
void coulomb_at_points(pb_mesh* M, pb_result* R, double* f);

struct BatchSystem {
    pb_mesh* M = nullptr;
    pb_result* R = nullptr;
    pb_ctx sub;                       // per-system context (own stream)
    pb_ctx* saved_mesh_ctx = nullptr;
    pb_ctx* saved_tree_ctx = nullptr;
    long long n = 0;
    int kmax = 0, nb = 0, ub = 0;
    DBuf<double> V, w, partial, h, h2, H, cs, sn, g, nrm2, resid, yv, xin, xout, b, f;
    double* host = nullptr;           // pinned: [0] residual, [1] ||b||^2
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double beta = 0.0;
    int j = 0;
    bool active = true;
    int status = PB_ENOCONV;
    ~BatchSystem() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (host) cudaFreeHost(host);
    }
};

static void batch_dots(BatchSystem& S, const double* Vb, int nk, const double* vec, double* out, int acc) {
    cudaStream_t st = S.sub.stream;
    k_dots<<<S.nb, 256, 0, st>>>(S.n, Vb, S.n, nk, vec, S.partial.p, S.kmax + 1);
    PB_CHECK_LAUNCH();
    k_dots_reduce<<<div_up(nk, 128), 128, 0, st>>>(S.nb, nk, S.partial.p, S.kmax + 1, out, acc);
    PB_CHECK_LAUNCH();
}

void solve_batch(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, pb_result** results, double tol, int max_iter,
                 int* status) {
    // Every persistent buffer is allocated on the context stream (which
    // outlives the batch); the per-system streams only run work and the
    // graphs' own temporaries.
    cudaStream_t main = ctx->stream;
    std::vector<std::unique_ptr<BatchSystem>> sys(nsys);
    struct Restore {
        std::vector<std::unique_ptr<BatchSystem>>* s;
        cudaStream_t main;
        ~Restore() {
            for (auto& p : *s) {
                if (!p) continue;
                cudaStream_t st = p->sub.stream;
                if (st) cudaStreamSynchronize(st);
                if (p->saved_mesh_ctx) p->M->ctx = p->saved_mesh_ctx;
                if (p->saved_tree_ctx) p->M->tree->ctx = p->saved_tree_ctx;
                p.reset();                      // frees on the context stream
                if (st) cudaStreamDestroy(st);
            }
            cudaStreamSynchronize(main);
        }
    } restore{&sys, main};
    // phase 0, on the context stream: singular entries, operators (warm
    // mat-vec), right-hand sides, Krylov storage
    for (int s = 0; s < nsys; ++s) {
        auto S = std::make_unique<BatchSystem>();
        S->M = meshes[s];
        S->R = results[s];
        pb_mesh* M = S->M;
        pb_result* R = S->R;
        ensure_singular_public(M, R->kappa);
        const int nt = (int)M->nt, nq = M->nq;
        const long long np = (long long)nt * nq;
        S->n = 2LL * nt;
        S->kmax = max_iter;
        S->nb = (int)std::min<long long>(kDotBlocksB, (S->n + 255) / 256);
        S->ub = (int)std::min<long long>(4LL * ctx->sm_count, (S->n + 255) / 256);
        S->V.alloc((size_t)(S->kmax + 1) * S->n, main);
        S->partial.alloc((size_t)kDotBlocksB * (S->kmax + 1), main);
        S->h.alloc(S->kmax + 2, main); S->h2.alloc(S->kmax + 2, main);
        S->H.alloc((size_t)(S->kmax + 1) * S->kmax, main);
        S->cs.alloc(S->kmax + 1, main); S->sn.alloc(S->kmax + 1, main); S->g.alloc(S->kmax + 2, main);
        S->nrm2.alloc(1, main); S->resid.alloc(1, main); S->yv.alloc(S->kmax + 1, main);
        S->xin.alloc(S->n, main); S->xout.alloc(S->n, main); S->b.alloc(S->n, main); S->f.alloc(np, main);
        S->g.zero(main);
        S->xin.zero(main);
        R->x.alloc(S->n, main);
        R->x.zero(main);
        coulomb_at_points(M, R, S->f.p);
        k_rhs<<<div_up(nt, 128), 128, 0, main>>>(nt, nq, S->f.p, M->qw_d.p, M->adj_off.p, M->adj_ids.p, M->S_d.p,
                                                 M->area.p, R->eps_in / R->eps_out, 1, S->b.p);
        PB_CHECK_LAUNCH();
        mesh_matvec(M, R->eps_in, R->eps_out, R->kappa, R->precision, S->xin.p, S->xout.p, 1);
        PB_CUDA(cudaMallocHost((void**)&S->host, 2 * sizeof(double)));
        sys[s] = std::move(S);
    }
    PB_CUDA(cudaStreamSynchronize(main));
    // phase 1: one stream per system, mat-vec captured as a graph
    for (auto& Sp : sys) {
        BatchSystem& S = *Sp;
        S.sub.device = ctx->device;
        S.sub.sm_count = ctx->sm_count;
        S.sub.dev_err = ctx->dev_err;
        S.sub.profile = false;
        S.sub.coupling = ctx->coupling;
        S.sub.deterministic = ctx->deterministic;
        S.sub.singular = ctx->singular;
        S.sub.overlap = 0;              // systems already run side by side on their own streams
        PB_CUDA(cudaStreamCreateWithFlags(&S.sub.stream, cudaStreamNonBlocking));
        S.saved_mesh_ctx = S.M->ctx;
        S.saved_tree_ctx = S.M->tree->ctx;
        S.M->ctx = &S.sub;
        S.M->tree->ctx = &S.sub;
        cudaStream_t st = S.sub.stream;
        pb_result* R = S.R;
        PB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        mesh_matvec(S.M, R->eps_in, R->eps_out, R->kappa, R->precision, S.xin.p, S.xout.p, 1);
        PB_CUDA(cudaStreamEndCapture(st, &S.graph));
        PB_CUDA(cudaGraphInstantiate(&S.exec, S.graph, 0));
        // r0 = P^{-1} b, beta = ||r0||
        batch_dots(S, S.b.p, 1, S.b.p, S.nrm2.p, 0);
        PB_CUDA(cudaMemcpyAsync(S.host + 1, S.nrm2.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        k_scale<<<S.ub, 256, 0, st>>>(S.n, S.b.p, S.nrm2.p, S.V.p);
        k_set_g0<<<1, 1, 0, st>>>(S.nrm2.p, S.g.p);
        PB_CHECK_LAUNCH();
    }
    for (auto& Sp : sys) {
        PB_CUDA(cudaStreamSynchronize(Sp->sub.stream));
        Sp->beta = std::sqrt(Sp->host[1]);
        if (Sp->beta == 0.0) { Sp->active = false; Sp->status = PB_OK; Sp->j = 0; }
    }
    // lockstep GMRES iterations (CGS2), one host synchronisation per iteration
    for (int j = 0; j < max_iter; ++j) {
        bool any = false;
        for (auto& Sp : sys) {
            BatchSystem& S = *Sp;
            if (!S.active) continue;
            any = true;
            cudaStream_t st = S.sub.stream;
            PB_CUDA(cudaMemcpyAsync(S.xin.p, S.V.p + (long long)j * S.n, S.n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
            PB_CUDA(cudaGraphLaunch(S.exec, st));
            batch_dots(S, S.V.p, j + 1, S.xout.p, S.h.p, 0);
            k_update<<<S.ub, 256, (j + 1) * sizeof(double), st>>>(S.n, S.V.p, S.n, j + 1, S.h.p, S.xout.p);
            PB_CHECK_LAUNCH();
            batch_dots(S, S.V.p, j + 1, S.xout.p, S.h2.p, 0);
            k_update<<<S.ub, 256, (j + 1) * sizeof(double), st>>>(S.n, S.V.p, S.n, j + 1, S.h2.p, S.xout.p);
            PB_CHECK_LAUNCH();
            k_vadd<<<div_up(j + 1, 128), 128, 0, st>>>(j + 1, S.h2.p, S.h.p);
            PB_CHECK_LAUNCH();
            batch_dots(S, S.xout.p, 1, S.xout.p, S.nrm2.p, 0);
            k_givens<<<1, 1, 0, st>>>(j, S.kmax, S.h.p, S.nrm2.p, S.H.p, S.cs.p, S.sn.p, S.g.p, S.resid.p);
            PB_CHECK_LAUNCH();
            k_scale<<<S.ub, 256, 0, st>>>(S.n, S.xout.p, S.nrm2.p, S.V.p + (long long)(j + 1) * S.n);
            PB_CHECK_LAUNCH();
            PB_CUDA(cudaMemcpyAsync(S.host, S.resid.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        if (!any) break;
        for (auto& Sp : sys) {
            BatchSystem& S = *Sp;
            if (!S.active) continue;
            PB_CUDA(cudaStreamSynchronize(S.sub.stream));
            S.j = j + 1;
            double rel = S.host[0] / S.beta;
            S.R->residual = rel;
            if (rel <= tol) { S.active = false; S.status = PB_OK; }
        }
    }
    for (int s = 0; s < nsys; ++s) {
        BatchSystem& S = *sys[s];
        cudaStream_t st = S.sub.stream;
        int m = S.j;
        if (m > 0) {
            k_backsolve<<<1, 1, 0, st>>>(m, S.kmax, S.H.p, S.g.p, S.yv.p);
            k_axpy_basis<<<S.ub, 256, m * sizeof(double), st>>>(S.n, S.V.p, S.n, m, S.yv.p, S.R->x.p);
            PB_CHECK_LAUNCH();
        }
        S.R->iterations = m;
        S.R->status = S.status;
        if (m == 0) S.R->residual = 0.0;
        status[s] = S.status;
    }
    for (auto& Sp : sys) PB_CUDA(cudaStreamSynchronize(Sp->sub.stream));
}

__global__ void k_fill(long long n, float v, float* a) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// time one Laplace + one Yukawa SL+DL apply for each candidate ncrit
void tune_ncrit(pb_ctx* ctx, const float* xyz_dev, long long n, int p, const int* cand, int ncand, int* best,
                double* best_ms) {
    cudaStream_t st = ctx->stream;
    DBuf<float> q, nrm, out;
    q.alloc(n, st); nrm.alloc(3 * n, st); out.alloc(n, st);
    k_fill<<<div_up(n, 256), 256, 0, st>>>(n, 1.0f, q.p);
    k_fill<<<div_up(3 * n, 256), 256, 0, st>>>(3 * n, 0.57735026f, nrm.p);
    PB_CHECK_LAUNCH();
    cudaEvent_t a, b;
    PB_CUDA(cudaEventCreate(&a));
    PB_CUDA(cudaEventCreate(&b));
    double bestv = 1e300;
    int bestc = cand[0];
    for (int c = 0; c < ncand; ++c) {
        fmm_tree T;
        T.ctx = ctx;
        T.ns = n;
        T.nt = n;
        T.same = true;
        T.ncrit = cand[c];
        build_tree(&T, xyz_dev, nullptr);
        auto run = [&]() {
            fmm_apply_impl(&T, FMM_LAPLACE, 0.0, p, PB_MIXED, q.p, q.p, nrm.p, nullptr, out.p, nullptr);
            fmm_apply_impl(&T, FMM_YUKAWA, 0.125, p, PB_MIXED, q.p, q.p, nrm.p, nullptr, out.p, nullptr);
        };
        run();
        PB_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f, tot = 0.f;
        for (int r = 0; r < 3; ++r) {
            PB_CUDA(cudaEventRecord(a, st));
            run();
            PB_CUDA(cudaEventRecord(b, st));
            PB_CUDA(cudaEventSynchronize(b));
            PB_CUDA(cudaEventElapsedTime(&ms, a, b));
            tot += ms;
        }
        if (tot / 3 < bestv) { bestv = tot / 3; bestc = cand[c]; }
        PB_CUDA(cudaStreamSynchronize(st));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *best = bestc;
    if (best_ms) *best_ms = bestv;
}

}  // namespace pbfmm
