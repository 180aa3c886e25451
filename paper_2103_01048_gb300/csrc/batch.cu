// Batched solves of many systems and an ncrit autotuner.
//
// pb_solve_batch runs the GMRES iterations of several meshes in lockstep,
// and one lockstep iteration of ALL active systems is one CUDA graph: for
// every system, on its own stream (branches of the graph), the copy of the
// current Krylov vector, the preconditioned mat-vec (P1, the Laplace and
// Yukawa FMM passes, the fused Galerkin glue), the two classical
// Gram-Schmidt passes, the Givens update with the device-side convergence
// test, and the next basis vector.  The Arnoldi kernels read the iteration
// index from device memory, so the same graph is replayed every iteration;
// a system that converges marks itself done on the device and its Arnoldi
// kernels return at once.  The host launches the graph, reads the systems'
// done flags (one synchronisation per iteration) and, once a quarter of the
// systems in the graph have converged, re-captures it without them, so their
// mat-vecs stop too.
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

// Arnoldi step kernels with the iteration index j in device memory (the
// graph of one lockstep iteration is replayed for every j); each returns at
// once when its system is done.
struct BatchDev {
    int j;          // current iteration
    int done;       // 1: converged or out of iterations
    int m;          // iterations taken (valid once done)
    int pad;
    double resid;   // |g[j+1]| of the last completed iteration
};

__global__ void k_b_copy_in(long long n, const double* __restrict__ V, const BatchDev* __restrict__ d,
                            double* __restrict__ x) {
    if (d->done) return;
    const double* v = V + (long long)d->j * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v[i];
}

// partial[blk][k] = sum over the block's rows of V[k][i] w[i], k <= j (all:
// the j + 1 basis vectors; else only w with itself)
__global__ void k_b_dots(long long n, const double* __restrict__ V, long long ld, const double* __restrict__ w,
                         double* __restrict__ partial, int kmax, const BatchDev* __restrict__ d, int all) {
    if (d->done) return;
    __shared__ double red[256];
    const int nk = all ? d->j + 1 : 1;
    const double* base = all ? V : w;
    long long chunk = (n + gridDim.x - 1) / gridDim.x;
    long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int k = 0; k < nk; ++k) {
        double s = 0.0;
        const double* v = base + (long long)k * ld;
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

__global__ void k_b_dots_reduce(int nblk, const double* __restrict__ partial, int kmax, double* __restrict__ h,
                                const BatchDev* __restrict__ d, int all) {
    if (d->done) return;
    const int nk = all ? d->j + 1 : 1;
    const int k = threadIdx.x + blockIdx.x * blockDim.x;
    if (k >= nk) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(long long)b * kmax + k];
    h[k] = s;
}

// w -= sum_k h[k] V[k], k <= j (h staged in shared memory, kmax + 1 doubles)
__global__ void k_b_update(long long n, const double* __restrict__ V, long long ld, const double* __restrict__ h,
                           double* __restrict__ w, const BatchDev* __restrict__ d) {
    if (d->done) return;
    extern __shared__ double sh[];
    const int nk = d->j + 1;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) sh[k] = h[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int k = 0; k < nk; ++k) s -= sh[k] * V[(long long)k * ld + i];
        w[i] = s;
    }
}

__global__ void k_b_vadd(const double* __restrict__ a, double* __restrict__ b, const BatchDev* __restrict__ d) {
    if (d->done) return;
    for (int k = threadIdx.x; k <= d->j; k += blockDim.x) b[k] += a[k];
}

// Hessenberg column j -> Givens update, the convergence test, and j + 1
__global__ void k_b_givens(int kmax, const double* __restrict__ h, const double* __restrict__ nrm2, double* H,
                           double* cs, double* sn, double* g, double beta, double tol, BatchDev* d) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || d->done) return;
    const int j = d->j;
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
    d->resid = fabs(g[j + 1]);
    d->j = j + 1;
    if (d->resid <= tol * beta || j + 1 >= kmax) {
        d->done = 1;
        d->m = j + 1;
    }
}

// r = b - w (the residual of a restart)
__global__ void k_b_residual(long long n, const double* __restrict__ b, const double* __restrict__ w,
                             double* __restrict__ r) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = b[i] - w[i];
}

// V[j] = w / ||w|| (j already advanced by k_b_givens); skipped once done
__global__ void k_b_scale(long long n, const double* __restrict__ w, const double* __restrict__ nrm2,
                          double* __restrict__ V, const BatchDev* __restrict__ d) {
    if (d->done) return;
    const double inv = 1.0 / sqrt(*nrm2);
    double* out = V + (long long)d->j * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
}
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
    DBuf<BatchDev> dev;               // iteration state on the device
    double beta = 0.0;                // ||P^-1 b||: the convergence test is relative to it in every cycle
    int j = 0;
    int tot = 0;                      // iterations of the completed (restarted) cycles
    bool active = true;
    int status = PB_ENOCONV;
    ~BatchSystem() {
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
        const bool p1 = M->basis == PB_P1;
        if (!p1) ensure_singular_public(M, R->kappa);
        const int nt = (int)M->nt, nq = M->nq;
        const long long np = (long long)nt * nq;
        S->n = 2LL * M->nunk;
        S->kmax = ctx->restart > 0 ? std::min(ctx->restart, max_iter) : max_iter;   // vectors of one cycle
        S->nb = (int)std::min<long long>(kDotBlocksB, (S->n + 255) / 256);
        S->ub = (int)std::min<long long>(4LL * ctx->sm_count, (S->n + 255) / 256);
        S->V.alloc((size_t)(S->kmax + 1) * S->n, main);
        S->partial.alloc((size_t)kDotBlocksB * (S->kmax + 1), main);
        S->h.alloc(S->kmax + 2, main); S->h2.alloc(S->kmax + 2, main);
        S->H.alloc((size_t)(S->kmax + 1) * S->kmax, main);
        S->cs.alloc(S->kmax + 1, main); S->sn.alloc(S->kmax + 1, main); S->g.alloc(S->kmax + 2, main);
        S->nrm2.alloc(1, main); S->resid.alloc(1, main); S->yv.alloc(S->kmax + 1, main);
        S->xin.alloc(S->n, main); S->xout.alloc(S->n, main); S->b.alloc(S->n, main);
        S->g.zero(main);
        S->xin.zero(main);
        R->x.alloc(S->n, main);
        R->x.zero(main);
        if (p1) {
            rhs_p1(M, R, S->b.p);              // the formulation's right-hand side (P1 test functions)
        } else {
            S->f.alloc(np, main);
            coulomb_at_points(M, R, S->f.p);
            k_rhs<<<div_up(nt, 128), 128, 0, main>>>(nt, nq, S->f.p, M->qw_d.p, M->adj_off.p, M->adj_ids.p,
                                                     M->S_d.p, M->area.p, R->eps_in / R->eps_out, 1, S->b.p);
            PB_CHECK_LAUNCH();
        }
        // warm mat-vec: singular entries, operators and workspaces exist before the capture
        mesh_matvec(M, R->eps_in, R->eps_out, R->kappa, R->precision, S->xin.p, S->xout.p, 1, R->formulation);
        PB_CUDA(cudaMallocHost((void**)&S->host, 2 * sizeof(double)));
        sys[s] = std::move(S);
    }
    PB_CUDA(cudaStreamSynchronize(main));
    // phase 1: one stream per system; r0 = P^{-1} b, beta = ||r0||
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
        S.dev.alloc(1, main);
        PB_CUDA(cudaMemsetAsync(S.dev.p, 0, sizeof(BatchDev), main));
        PB_CUDA(cudaStreamSynchronize(main));
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
    // One lockstep iteration of every active system as one graph, captured
    // on `origin` with a fork to each system's stream and a join back.
    cudaStream_t origin = nullptr;
    PB_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    std::vector<cudaEvent_t> evs;
    auto new_event = [&]() {
        cudaEvent_t e;
        PB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        evs.push_back(e);
        return e;
    };
    cudaEvent_t fork = new_event();
    std::vector<cudaEvent_t> joins;
    for (int s = 0; s < nsys; ++s) joins.push_back(new_event());
    DBuf<BatchDev> flags;              // device state of all systems, gathered for one copy
    flags.alloc(nsys, main);
    BatchDev* hflags = nullptr;
    PB_CUDA(cudaMallocHost((void**)&hflags, nsys * sizeof(BatchDev)));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    struct GraphGuard {
        cudaGraph_t* g;
        cudaGraphExec_t* e;
        cudaStream_t* o;
        std::vector<cudaEvent_t>* evs;
        BatchDev** hf;
        ~GraphGuard() {
            if (*e) cudaGraphExecDestroy(*e);
            if (*g) cudaGraphDestroy(*g);
            if (*o) { cudaStreamSynchronize(*o); cudaStreamDestroy(*o); }
            for (auto ev : *evs) cudaEventDestroy(ev);
            if (*hf) cudaFreeHost(*hf);
        }
    } guard{&graph, &exec, &origin, &evs, &hflags};
    auto capture = [&]() {
        if (exec) { PB_CUDA(cudaGraphExecDestroy(exec)); exec = nullptr; }
        if (graph) { PB_CUDA(cudaGraphDestroy(graph)); graph = nullptr; }
        PB_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        PB_CUDA(cudaEventRecord(fork, origin));
        for (int s = 0; s < nsys; ++s) {
            BatchSystem& S = *sys[s];
            cudaStream_t st = S.sub.stream;
            PB_CUDA(cudaStreamWaitEvent(st, fork, 0));
            if (S.active) {
                pb_result* R = S.R;
                k_b_copy_in<<<S.ub, 256, 0, st>>>(S.n, S.V.p, S.dev.p, S.xin.p);
                PB_CHECK_LAUNCH();
                mesh_matvec(S.M, R->eps_in, R->eps_out, R->kappa, R->precision, S.xin.p, S.xout.p, 1,
                            R->formulation);
                for (int pass = 0; pass < 2; ++pass) {       // CGS2
                    double* hp = pass == 0 ? S.h.p : S.h2.p;
                    k_b_dots<<<S.nb, 256, 0, st>>>(S.n, S.V.p, S.n, S.xout.p, S.partial.p, S.kmax + 1, S.dev.p, 1);
                    k_b_dots_reduce<<<div_up(S.kmax + 1, 128), 128, 0, st>>>(S.nb, S.partial.p, S.kmax + 1, hp,
                                                                            S.dev.p, 1);
                    k_b_update<<<S.ub, 256, (S.kmax + 1) * sizeof(double), st>>>(S.n, S.V.p, S.n, hp, S.xout.p,
                                                                                S.dev.p);
                    PB_CHECK_LAUNCH();
                }
                k_b_vadd<<<1, 256, 0, st>>>(S.h2.p, S.h.p, S.dev.p);
                k_b_dots<<<S.nb, 256, 0, st>>>(S.n, S.xout.p, S.n, S.xout.p, S.partial.p, S.kmax + 1, S.dev.p, 0);
                k_b_dots_reduce<<<1, 128, 0, st>>>(S.nb, S.partial.p, S.kmax + 1, S.nrm2.p, S.dev.p, 0);
                k_b_givens<<<1, 1, 0, st>>>(S.kmax, S.h.p, S.nrm2.p, S.H.p, S.cs.p, S.sn.p, S.g.p, S.beta, tol,
                                            S.dev.p);
                k_b_scale<<<S.ub, 256, 0, st>>>(S.n, S.xout.p, S.nrm2.p, S.V.p, S.dev.p);
                PB_CHECK_LAUNCH();
            }
            PB_CUDA(cudaMemcpyAsync(flags.p + s, S.dev.p, sizeof(BatchDev), cudaMemcpyDeviceToDevice, st));
            PB_CUDA(cudaEventRecord(joins[s], st));
            PB_CUDA(cudaStreamWaitEvent(origin, joins[s], 0));
        }
        PB_CUDA(cudaMemcpyAsync(hflags, flags.p, nsys * sizeof(BatchDev), cudaMemcpyDeviceToHost, origin));
        PB_CUDA(cudaStreamEndCapture(origin, &graph));
        PB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    };
    // k_b_update stages up to kmax + 1 coefficients in shared memory
    PB_CUDA(cudaFuncSetAttribute(k_b_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(48 * 1024, (sys[0]->kmax + 1) * sizeof(double))));
    // end of an unconverged cycle of GMRES(m): x += V y, r = P^-1 b - P^-1 A x,
    // V[0] = r / ||r||, g[0] = ||r||, j = 0 (the captured graph stays valid)
    auto restart = [&](BatchSystem& S, int m) {
        cudaStream_t st = S.sub.stream;
        pb_result* R = S.R;
        k_backsolve<<<1, 1, 0, st>>>(m, S.kmax, S.H.p, S.g.p, S.yv.p);
        k_axpy_basis<<<S.ub, 256, m * sizeof(double), st>>>(S.n, S.V.p, S.n, m, S.yv.p, R->x.p);
        PB_CHECK_LAUNCH();
        mesh_matvec(S.M, R->eps_in, R->eps_out, R->kappa, R->precision, R->x.p, S.xout.p, 1, R->formulation);
        k_b_residual<<<S.ub, 256, 0, st>>>(S.n, S.b.p, S.xout.p, S.xin.p);
        PB_CHECK_LAUNCH();
        batch_dots(S, S.xin.p, 1, S.xin.p, S.nrm2.p, 0);
        k_scale<<<S.ub, 256, 0, st>>>(S.n, S.xin.p, S.nrm2.p, S.V.p);
        k_set_g0<<<1, 1, 0, st>>>(S.nrm2.p, S.g.p);
        PB_CHECK_LAUNCH();
        PB_CUDA(cudaMemsetAsync(S.dev.p, 0, sizeof(BatchDev), st));
    };
    int nactive = 0;
    for (auto& Sp : sys) nactive += Sp->active ? 1 : 0;
    int captured = 0;           // active systems when the graph was captured
    bool restarted = false;
    for (int it = 0; it < max_iter && nactive > 0; ++it) {
        // a finished system's Arnoldi kernels return at once, but its
        // mat-vec still runs: re-capture once a quarter of the captured
        // systems have finished (not for every one, which at hundreds of
        // systems would cost more than it saves)
        if (captured == 0 || 4 * nactive <= 3 * captured) {
            capture();
            captured = nactive;
        }
        PB_CUDA(cudaGraphLaunch(exec, origin));
        PB_CUDA(cudaStreamSynchronize(origin));
        for (int s = 0; s < nsys; ++s) {
            BatchSystem& S = *sys[s];
            if (!S.active) continue;
            S.j = hflags[s].j;
            S.R->residual = hflags[s].resid / S.beta;
            if (hflags[s].done) {
                const int m = hflags[s].m;
                const bool conv = S.R->residual <= tol;
                if (conv || S.tot + m >= max_iter) {
                    S.active = false;
                    S.j = m;
                    S.status = conv ? PB_OK : PB_ENOCONV;
                    --nactive;
                } else {
                    restart(S, m);
                    S.tot += m;
                    S.j = 0;
                    restarted = true;
                }
            }
        }
        // the next graph launch (on `origin`) must see the restarts' work
        if (restarted) {
            for (auto& Sp : sys) PB_CUDA(cudaStreamSynchronize(Sp->sub.stream));
            restarted = false;
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
        S.R->iterations = S.tot + m;
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

// time the paired apply (the FMM work of one direct-formulation mat-vec) for
// every candidate ncrit and every leaf / M2L tile shape; leave the fastest
// tile shapes set on the context
void tune_fmm(pb_ctx* ctx, const float* xyz_dev, long long n, int p, const int* cand, int ncand, int* best,
              int* best_nt, int* best_tile, double* best_ms) {
    cudaStream_t st = ctx->stream;
    const int nt0 = ctx->leaf_nt, tile0 = ctx->m2l_tile;
    DBuf<float> q, nrm, outL, outY;
    q.alloc(n, st); nrm.alloc(3 * n, st); outL.alloc(n, st); outY.alloc(n, st);
    k_fill<<<div_up(n, 256), 256, 0, st>>>(n, 1.0f, q.p);
    k_fill<<<div_up(3 * n, 256), 256, 0, st>>>(3 * n, 0.57735026f, nrm.p);
    PB_CHECK_LAUNCH();
    cudaEvent_t a, b;
    PB_CUDA(cudaEventCreate(&a));
    PB_CUDA(cudaEventCreate(&b));
    double bestv = 1e300;
    int bc = cand[0], bnt = 4, btile = 0;
    try {
        for (int c = 0; c < ncand; ++c) {
            fmm_tree T;
            T.ctx = ctx;
            T.ns = n;
            T.nt = n;
            T.same = true;
            T.ncrit = cand[c];
            build_tree(&T, xyz_dev, nullptr);
            for (int nt : {2, 4})
                for (int tile : {0, 1}) {
                    ctx->leaf_nt = nt;
                    ctx->m2l_tile = tile;
                    auto run = [&]() {
                        fmm_apply_pair_impl(&T, 0.125, p, PB_MIXED, q.p, q.p, q.p, nrm.p, nullptr, outL.p, outY.p,
                                            nullptr, nullptr);
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
                    if (tot / 3 < bestv) { bestv = tot / 3; bc = cand[c]; bnt = nt; btile = tile; }
                }
            PB_CUDA(cudaStreamSynchronize(st));
        }
    } catch (...) {
        ctx->leaf_nt = nt0;
        ctx->m2l_tile = tile0;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        throw;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->leaf_nt = bnt;
    ctx->m2l_tile = btile;
    *best = bc;
    if (best_nt) *best_nt = bnt;
    if (best_tile) *best_tile = btile;
    if (best_ms) *best_ms = bestv;
}

}  // namespace pbfmm
