// C-ABI entry points (declared in include/pbfmm.h).  Every entry point turns
// internal exceptions into a status code and a message on the context.
#include "bem.cuh"
#include <new>
#include <memory>

namespace pbfmm {
void build_tree(fmm_tree* T, const float* src, const float* tgt);
void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn);
void fmm_apply_pair_impl(fmm_tree* Tr, double kappa, int p, int precision, const void* qL, const void* qY,
                         const void* dip, const void* src_n, const void* tgt_n, void* outL, void* outY, void* dnL,
                         void* dnY);
void mesh_setup(pb_mesh* M, const double* verts, const int* tris);

int solve(pb_mesh* M, pb_result* R, double tol, int max_iter);
void reaction_energy(pb_result* R, double* phir_host, double* dG);
void ensure_singular_public(pb_mesh* M, double kappa);
void ensure_singular_p1_public(pb_mesh* M, double kappa);
int energy_gradient(pb_result* R, double tol, int max_iter, double* dEdq_host, double* dEdx_host);
void solve_batch(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, pb_result** results, double tol, int max_iter,
                 int* status);
void tune_ncrit(pb_ctx* ctx, const float* xyz_dev, long long n, int p, const int* cand, int ncand, int* best,
                double* best_ms);
void tune_fmm(pb_ctx* ctx, const float* xyz_dev, long long n, int p, const int* cand, int ncand, int* best,
              int* best_nt, int* best_tile, double* best_ms);

// A result object for the charges of one system (atoms as (x, y, z, q) on the device).
pb_result* make_result(pb_ctx* ctx, pb_mesh* M, const double* atoms, const double* q, int64_t na, double eps_in,
                       double eps_out, double kappa, int precision, int formulation = PB_FORM_DIRECT) {
    std::unique_ptr<pb_result> owner(new pb_result());
    pb_result* R = owner.get();
    R->mesh = M;
    R->nt = M->nt;
    R->na = na;
    R->eps_in = eps_in;
    R->eps_out = eps_out;
    R->kappa = kappa;
    R->precision = precision;
    R->formulation = formulation;
    R->nunk = M->nunk;
    std::vector<double> a4(4 * na), ha(3 * na), hq(na);
    cudaError_t e1 = cudaMemcpy(ha.data(), atoms, 3 * na * sizeof(double), cudaMemcpyDefault);
    cudaError_t e2 = cudaMemcpy(hq.data(), q, na * sizeof(double), cudaMemcpyDefault);
    if (e1 != cudaSuccess || e2 != cudaSuccess) throw Error(PB_ECUDA, "copying atoms/charges failed");
    for (int64_t k = 0; k < na; ++k) {
        a4[4 * k] = ha[3 * k]; a4[4 * k + 1] = ha[3 * k + 1]; a4[4 * k + 2] = ha[3 * k + 2]; a4[4 * k + 3] = hq[k];
    }
    R->atoms.alloc(4 * na, ctx->stream);
    PB_CUDA(cudaMemcpyAsync(R->atoms.p, a4.data(), 4 * na * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
    return owner.release();
}

thread_local long long g_launch_count = 0;
std::atomic<long long> g_alloc_count{0};
std::atomic<long long> g_alloc_fail_at{0};
constexpr long long kDefaultWaitLimit = 2000000000LL;
std::atomic<long long> g_wait_limit{kDefaultWaitLimit};

void profile_collect(pb_ctx* ctx) {
    for (auto& e : ctx->pending) {
        cudaEventSynchronize(e.second.second);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.second.first, e.second.second);
        ctx->prof_ms[e.first] += ms;
        ctx->prof_calls[e.first] += 1;
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    ctx->pending.clear();
}

bool is_device_ptr(const void* p) {
    if (!p) return true;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device copy of a possibly-host buffer (nbytes); returns the device pointer to use.
struct Staged {
    DBuf<char> buf;
    const void* dev = nullptr;
    void in(const void* p, size_t nbytes, cudaStream_t st) {
        if (!p) { dev = nullptr; return; }
        if (is_device_ptr(p)) { dev = p; return; }
        buf.alloc(nbytes, st);
        PB_CUDA(cudaMemcpyAsync(buf.p, p, nbytes, cudaMemcpyHostToDevice, st));
        dev = buf.p;
    }
};
}  // namespace pbfmm

using namespace pbfmm;

#define PB_API_BEGIN try {
#define PB_API_END(ctx)                                                     \
    }                                                                       \
    catch (const pbfmm::Error& e) {                                         \
        if (ctx) (ctx)->last_error = e.what();                              \
        return e.code;                                                      \
    }                                                                       \
    catch (const std::bad_alloc&) {                                         \
        if (ctx) (ctx)->last_error = "host allocation failed";             \
        return PB_ENOMEM;                                                   \
    }                                                                       \
    catch (const std::exception& e) {                                       \
        if (ctx) (ctx)->last_error = e.what();                              \
        return PB_EINVAL;                                                   \
    }                                                                       \
    if (ctx) (ctx)->last_error.clear();                                     \
    return PB_OK;

extern "C" {

int pb_create(pb_ctx** out, int device, void* cuda_stream) {
    if (!out) return PB_EINVAL;
    *out = nullptr;
    pb_ctx* ctx = new (std::nothrow) pb_ctx();
    if (!ctx) return PB_ENOMEM;
    PB_API_BEGIN
    PB_CUDA(cudaSetDevice(device));
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    PB_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
    // keep freed stream-ordered allocations in the pool between calls
    cudaMemPool_t pool;
    PB_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    PB_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    PB_CUDA(cudaMalloc((void**)&ctx->dev_err, sizeof(int)));
    PB_CUDA(cudaMemset(ctx->dev_err, 0, sizeof(int)));
    PB_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    PB_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    PB_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    *out = ctx;
    PB_API_END(ctx)
}

int pb_destroy(pb_ctx* ctx) {
    if (!ctx) return PB_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->aux) {
        cudaStreamSynchronize(ctx->aux);
        cudaStreamDestroy(ctx->aux);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    delete ctx;
    return PB_OK;
}

const char* pb_last_error(pb_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

// Read and clear the device error flag (after a stream synchronisation).
void check_device_error(pb_ctx* ctx) {
    int h = 0;
    PB_CUDA(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h) {
        PB_CUDA(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream));
        throw Error(PB_ETIMEOUT, "a device-side wait timed out (tensor-core M2L); results of the affected call are invalid");
    }
}

int pb_sync(pb_ctx* ctx) {
    if (!ctx) return PB_EINVAL;
    PB_API_BEGIN
    PB_CUDA(cudaSetDevice(ctx->device));
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
    check_device_error(ctx);
    PB_API_END(ctx)
}

int pb_profile(pb_ctx* ctx, int enable) {
    if (!ctx) return PB_EINVAL;
    PB_API_BEGIN
    profile_collect(ctx);
    ctx->profile = enable != 0;
    for (int i = 0; i < PB_PH_COUNT; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_calls[i] = 0; }
    ctx->launch_base = g_launch_count;
    PB_API_END(ctx)
}

int pb_set_option(pb_ctx* ctx, int option, int value) {
    if (!ctx) return PB_EINVAL;
    if (option == PB_OPT_COUPLING && value >= 0 && value <= 2) { ctx->coupling = value; return PB_OK; }
    if (option == PB_OPT_DETERMINISTIC && (value == 0 || value == 1)) { ctx->deterministic = value; return PB_OK; }
    if (option == PB_OPT_SINGULAR && value >= 0 && value <= 2) { ctx->singular = value; return PB_OK; }
    if (option == PB_OPT_OVERLAP && (value == 0 || value == 1)) { ctx->overlap = value; return PB_OK; }
    if (option == PB_OPT_LEAF_NT && (value == 0 || value == 2 || value == 4)) { ctx->leaf_nt = value; return PB_OK; }
    if (option == PB_OPT_LEAF_PACKED && (value == 0 || value == 1)) { ctx->leaf_packed = value; return PB_OK; }
    if (option == PB_OPT_M2L_TILE && (value == 0 || value == 1)) { ctx->m2l_tile = value; return PB_OK; }
    if (option == PB_OPT_LIST_DIRECT && value >= 0 && value <= 3) { ctx->list_direct = value; return PB_OK; }
    if (option == PB_OPT_RESTART && value >= 0 && value <= 2000) { ctx->restart = value; return PB_OK; }
    ctx->last_error = "pb_set_option: unknown option or value";
    return PB_EINVAL;
}

int pb_profile_read(pb_ctx* ctx, int phase, double* ms, int64_t* calls) {
    if (!ctx) return PB_EINVAL;
    PB_API_BEGIN
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
    profile_collect(ctx);
    if (phase == PB_PH_LAUNCHES) {
        if (calls) *calls = g_launch_count - ctx->launch_base;
        if (ms) *ms = 0.0;
    } else {
        PB_REQUIRE(phase >= 0 && phase < PB_PH_COUNT, PB_EINVAL, "pb_profile_read: unknown phase");
        if (ms) *ms = ctx->prof_ms[phase];
        if (calls) *calls = ctx->prof_calls[phase];
    }
    PB_API_END(ctx)
}

int fmm_tree_build(pb_ctx* ctx, const float* src_xyz, int64_t n_src, const float* tgt_xyz, int64_t n_tgt,
                   int ncrit, fmm_tree** out) {
    if (!ctx || !out) return PB_EINVAL;
    *out = nullptr;
    fmm_tree* T = nullptr;
    PB_API_BEGIN
    PB_REQUIRE(src_xyz && n_src >= 1 && ncrit >= 1, PB_EINVAL, "fmm_tree_build: need sources and ncrit >= 1");
    PB_REQUIRE(n_src < (1LL << 31) - 1 && n_tgt < (1LL << 31) - 1, PB_EINVAL, "fmm_tree_build: too many points");
    PB_REQUIRE(!tgt_xyz || n_tgt >= 1, PB_EINVAL, "fmm_tree_build: empty target set");
    PB_CUDA(cudaSetDevice(ctx->device));
    T = new fmm_tree();
    T->ctx = ctx;
    T->ns = n_src;
    T->same = (tgt_xyz == nullptr);
    T->nt = T->same ? n_src : n_tgt;
    T->ncrit = ncrit;
    Staged s, t;
    s.in(src_xyz, (size_t)n_src * 3 * sizeof(float), ctx->stream);
    if (!T->same) t.in(tgt_xyz, (size_t)n_tgt * 3 * sizeof(float), ctx->stream);
    build_tree(T, (const float*)s.dev, (const float*)t.dev);
    *out = T;
    T = nullptr;
    }
    catch (const pbfmm::Error& e) {
        delete T;
        ctx->last_error = e.what();
        return e.code;
    }
    catch (const std::exception& e) {
        delete T;
        ctx->last_error = e.what();
        return PB_EINVAL;
    }
    ctx->last_error.clear();
    return PB_OK;
}

int fmm_tree_destroy(fmm_tree* T) {
    if (!T) return PB_EINVAL;
    cudaSetDevice(T->ctx->device);
    cudaStreamSynchronize(T->ctx->stream);
    delete T;
    return PB_OK;
}

int fmm_tree_info(const fmm_tree* T, fmm_tree_info_t* info) {
    if (!T || !info) return PB_EINVAL;
    info->n_src = T->ns;
    info->n_tgt = T->nt;
    info->n_box = T->nbox;
    info->n_leaf = T->nleaf;
    info->n_levels = T->nlev;
    info->same = T->same ? 1 : 0;
    info->n_u = T->n_u;
    info->n_v = T->n_v;
    info->n_w = T->n_w;
    info->n_x = T->n_x;
    for (int a = 0; a < 3; ++a) info->center[a] = T->c[a];
    info->half_width = T->R;
    info->p2p_pairs = T->work[0];
    info->m2p_targets = T->work[1];
    info->p2l_sources = T->work[2];
    info->l2p_targets = T->work[3];
    info->p2m_sources = T->work[4];
    info->n_dense_box = T->work[5];
    return PB_OK;
}

int fmm_tree_export_points(const fmm_tree* T, int32_t* perm_src, uint64_t* keys_src, int32_t* perm_tgt,
                           uint64_t* keys_tgt) {
    if (!T) return PB_EINVAL;
    pb_ctx* ctx = T->ctx;
    PB_API_BEGIN
    cudaStream_t st = ctx->stream;
    if (perm_src) PB_CUDA(cudaMemcpyAsync(perm_src, T->perm_s.p, T->ns * 4, cudaMemcpyDeviceToHost, st));
    if (keys_src) PB_CUDA(cudaMemcpyAsync(keys_src, T->keys_s.p, T->ns * 8, cudaMemcpyDeviceToHost, st));
    const int* pt = T->same ? T->perm_s.p : T->perm_t.p;
    const uint64_t* kt = T->same ? T->keys_s.p : T->keys_t.p;
    if (perm_tgt) PB_CUDA(cudaMemcpyAsync(perm_tgt, pt, T->nt * 4, cudaMemcpyDeviceToHost, st));
    if (keys_tgt) PB_CUDA(cudaMemcpyAsync(keys_tgt, kt, T->nt * 8, cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    PB_API_END(ctx)
}

int fmm_tree_export_boxes(const fmm_tree* T, int32_t* level, int32_t* parent, int32_t* first_child,
                          int32_t* nchild, int32_t* anchor, int32_t* src_begin, int32_t* src_end,
                          int32_t* tgt_begin, int32_t* tgt_end) {
    if (!T) return PB_EINVAL;
    pb_ctx* ctx = T->ctx;
    PB_API_BEGIN
    cudaStream_t st = ctx->stream;
    const size_t n = T->nbox;
    auto cp = [&](int32_t* dst, const int* src) {
        if (dst) PB_CUDA(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToHost, st));
    };
    cp(level, T->level.p); cp(parent, T->parent.p); cp(first_child, T->first_child.p); cp(nchild, T->nchild.p);
    cp(src_begin, T->sb.p); cp(src_end, T->se.p);
    cp(tgt_begin, T->same ? T->sb.p : T->tb.p); cp(tgt_end, T->same ? T->se.p : T->te.p);
    if (anchor) {
        std::vector<int4> a(n);
        PB_CUDA(cudaMemcpyAsync(a.data(), T->anchor.p, n * sizeof(int4), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < n; ++i) { anchor[3 * i] = a[i].x; anchor[3 * i + 1] = a[i].y; anchor[3 * i + 2] = a[i].z; }
    }
    PB_CUDA(cudaStreamSynchronize(st));
    PB_API_END(ctx)
}

int fmm_tree_export_list(const fmm_tree* T, int which, int64_t* off, int32_t* ids) {
    if (!T || !off || which < 0 || which > 3) return PB_EINVAL;
    pb_ctx* ctx = T->ctx;
    PB_API_BEGIN
    cudaStream_t st = ctx->stream;
    const int n = T->nbox;
    if (which == 0 || which == 2) {
        std::vector<int> o(n + 1);
        const DBuf<int>& O = which == 0 ? T->U_off : T->W_off;
        const DBuf<int>& I = which == 0 ? T->U_ids : T->W_ids;
        PB_CUDA(cudaMemcpyAsync(o.data(), O.p, (n + 1) * 4, cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i <= n; ++i) off[i] = o[i];
        if (ids && o[n] > 0) PB_CUDA(cudaMemcpyAsync(ids, I.p, (size_t)o[n] * 4, cudaMemcpyDeviceToHost, st));
    } else {
        const int cap = which == 1 ? kVCap : kXCap;
        std::vector<int> cnt(n), all((size_t)n * cap);
        PB_CUDA(cudaMemcpyAsync(cnt.data(), (which == 1 ? T->V_n : T->X_n).p, n * 4, cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaMemcpyAsync(all.data(), (which == 1 ? T->V : T->X).p, (size_t)n * cap * 4,
                                cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        off[0] = 0;
        for (int i = 0; i < n; ++i) {
            off[i + 1] = off[i] + cnt[i];
            if (ids)
                for (int k = 0; k < cnt[i]; ++k) ids[off[i] + k] = all[(size_t)i * cap + k];
        }
    }
    PB_CUDA(cudaStreamSynchronize(st));
    PB_API_END(ctx)
}

int fmm_apply_pair(pb_ctx* ctx, fmm_tree* T, double kappa, int p, int precision, const void* q_lap,
                   const void* q_yuk, const void* dip, const void* src_n, const void* tgt_n, void* out_lap,
                   void* out_yuk, void* dn_lap, void* dn_yuk) {
    if (!ctx || !T) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(kappa > 0.0, PB_EINVAL, "fmm_apply_pair: kappa must be > 0");
    PB_REQUIRE(p >= 2 && p <= 10, PB_EINVAL, "fmm_apply_pair: p must be in [2, 10]");
    PB_REQUIRE(precision == PB_MIXED || precision == PB_FP64, PB_EINVAL, "fmm_apply_pair: unknown precision");
    PB_REQUIRE(out_lap && out_yuk, PB_EINVAL, "fmm_apply_pair: out_lap and out_yuk are required");
    PB_REQUIRE(!dip || src_n, PB_EINVAL, "fmm_apply_pair: double layer needs source normals");
    PB_REQUIRE((dn_lap == nullptr) == (dn_yuk == nullptr), PB_EINVAL,
               "fmm_apply_pair: give both normal-derivative outputs or neither");
    PB_REQUIRE(!dn_lap || tgt_n, PB_EINVAL, "fmm_apply_pair: normal derivative needs target normals");
    PB_REQUIRE(!(dip && dn_lap), PB_EINVAL,
               "fmm_apply_pair: hypersingular kernel (dipole + target derivative) not provided");
    PB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t es = precision == PB_FP64 ? 8 : 4;
    Staged sqL, sqY, sd, sn, tn;
    sqL.in(q_lap, T->ns * es, st);
    if (q_yuk != q_lap) sqY.in(q_yuk, T->ns * es, st);     // the same host array is staged once
    else sqY.dev = sqL.dev;
    sd.in(dip, T->ns * es, st);
    sn.in(src_n, T->ns * 3 * es, st);
    tn.in(tgt_n, T->nt * 3 * es, st);
    void* outs[4] = {out_lap, out_yuk, dn_lap, dn_yuk};
    void* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    DBuf<char> bufs[4];
    bool any_host = sqL.buf.p || sqY.buf.p || sd.buf.p || sn.buf.p || tn.buf.p;
    for (int k = 0; k < 4; ++k) {
        if (!outs[k]) continue;
        if (is_device_ptr(outs[k])) { dev[k] = outs[k]; continue; }
        bufs[k].alloc(T->nt * es, st);
        dev[k] = bufs[k].p;
        any_host = true;
    }
    fmm_apply_pair_impl(T, kappa, p, precision, sqL.dev, sqY.dev, sd.dev, sn.dev, tn.dev, dev[0], dev[1], dev[2],
                        dev[3]);
    for (int k = 0; k < 4; ++k)
        if (bufs[k].p) PB_CUDA(cudaMemcpyAsync(outs[k], dev[k], T->nt * es, cudaMemcpyDeviceToHost, st));
    if (any_host) {
        PB_CUDA(cudaStreamSynchronize(st));
        check_device_error(ctx);
    }
    PB_API_END(ctx)
}

int fmm_apply(pb_ctx* ctx, fmm_tree* T, int kernel, double kappa, int p, int precision, const void* q,
              const void* dip, const void* src_n, const void* tgt_n, void* out, void* out_dn) {
    if (!ctx || !T) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(kernel == FMM_LAPLACE || kernel == FMM_YUKAWA, PB_EINVAL, "fmm_apply: unknown kernel");
    PB_REQUIRE(kernel == FMM_LAPLACE || kappa > 0.0, PB_EINVAL, "fmm_apply: Yukawa needs kappa > 0");
    PB_REQUIRE(p >= 2 && p <= 10, PB_EINVAL, "fmm_apply: p must be in [2, 10]");
    PB_REQUIRE(precision == PB_MIXED || precision == PB_FP64, PB_EINVAL, "fmm_apply: unknown precision");
    PB_REQUIRE(out != nullptr, PB_EINVAL, "fmm_apply: out is required");
    PB_REQUIRE(!dip || src_n, PB_EINVAL, "fmm_apply: double layer needs source normals");
    PB_REQUIRE(!out_dn || tgt_n, PB_EINVAL, "fmm_apply: normal derivative needs target normals");
    PB_REQUIRE(!(dip && out_dn), PB_EINVAL, "fmm_apply: hypersingular kernel (dipole + target derivative) not provided");
    PB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t es = precision == PB_FP64 ? 8 : 4;
    Staged sq, sd, sn, tn;
    sq.in(q, T->ns * es, st);
    sd.in(dip, T->ns * es, st);
    sn.in(src_n, T->ns * 3 * es, st);
    tn.in(tgt_n, T->nt * 3 * es, st);
    bool out_host = !is_device_ptr(out), dn_host = out_dn && !is_device_ptr(out_dn);
    DBuf<char> ob, db;
    void* o = out;
    void* od = out_dn;
    if (out_host) { ob.alloc(T->nt * es, st); o = ob.p; }
    if (dn_host) { db.alloc(T->nt * es, st); od = db.p; }
    fmm_apply_impl(T, kernel, kappa, p, precision, sq.dev, sd.dev, sn.dev, tn.dev, o, od);
    if (out_host) PB_CUDA(cudaMemcpyAsync(out, o, T->nt * es, cudaMemcpyDeviceToHost, st));
    if (dn_host) PB_CUDA(cudaMemcpyAsync(out_dn, od, T->nt * es, cudaMemcpyDeviceToHost, st));
    if (out_host || dn_host || sq.buf.p || sd.buf.p || sn.buf.p || tn.buf.p) {
        PB_CUDA(cudaStreamSynchronize(st));
        check_device_error(ctx);
    }
    PB_API_END(ctx)
}

int pb_mesh_setup(pb_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt, int basis,
                  int nquad, const pb_fmm_params* params, pb_mesh** out) {
    if (!ctx || !out) return PB_EINVAL;
    *out = nullptr;
    pb_mesh* M = nullptr;
    PB_API_BEGIN
    PB_REQUIRE(verts && tris && nv >= 3 && nt >= 1, PB_EINVAL, "pb_mesh_setup: empty mesh");
    PB_REQUIRE(basis == PB_P0 || basis == PB_P1, PB_EINVAL, "pb_mesh_setup: basis must be PB_P0 or PB_P1");
    PB_REQUIRE(nquad == 3 || nquad == 6, PB_EINVAL, "pb_mesh_setup: nquad must be 3 or 6");
    PB_REQUIRE(nt * nquad < (1LL << 31) - 1, PB_EINVAL, "pb_mesh_setup: too many quadrature points");
    PB_CUDA(cudaSetDevice(ctx->device));
    M = new pb_mesh();
    M->ctx = ctx;
    M->nv = nv;
    M->nt = nt;
    M->nq = nquad;
    M->basis = basis;
    if (params) {
        PB_REQUIRE(params->p >= 2 && params->p <= 10 && params->ncrit >= 1, PB_EINVAL, "pb_mesh_setup: bad FMM params");
        M->p = params->p;
        M->ncrit = params->ncrit;
    }
    mesh_setup(M, verts, tris);
    *out = M;
    M = nullptr;
    }
    catch (const pbfmm::Error& e) {
        if (M) { delete M->tree; delete M; }
        ctx->last_error = e.what();
        return e.code;
    }
    catch (const std::exception& e) {
        if (M) { delete M->tree; delete M; }
        ctx->last_error = e.what();
        return PB_EINVAL;
    }
    ctx->last_error.clear();
    return PB_OK;
}

int pb_mesh_destroy(pb_mesh* M) {
    if (!M) return PB_EINVAL;
    cudaSetDevice(M->ctx->device);
    cudaStreamSynchronize(M->ctx->stream);
    delete M->tree;
    delete M;
    return PB_OK;
}

int pb_mesh_unknowns(const pb_mesh* M, int64_t* n) {
    if (!M || !n) return PB_EINVAL;
    *n = M->nunk;
    return PB_OK;
}

int pb_mesh_info(const pb_mesh* M, int64_t* nt, int64_t* nqp, int64_t* nadj) {
    if (!M) return PB_EINVAL;
    if (nt) *nt = M->nt;
    if (nqp) *nqp = M->nt * M->nq;
    if (nadj) *nadj = M->nadj;
    return PB_OK;
}

int pb_mesh_export_singular(pb_ctx* ctx, pb_mesh* M, double kappa, int64_t* adj_off, int32_t* adj_ids, double* S) {
    if (!ctx || !M) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(kappa > 0, PB_EINVAL, "pb_mesh_export_singular: kappa must be > 0");
    cudaStream_t st = ctx->stream;
    if (M->basis == PB_P1) ensure_singular_p1_public(M, kappa);
    else ensure_singular_public(M, kappa);
    if (adj_off) {
        std::vector<int> o(M->nt + 1);
        PB_CUDA(cudaMemcpyAsync(o.data(), M->adj_off.p, (M->nt + 1) * 4, cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i <= M->nt; ++i) adj_off[i] = o[i];
    }
    if (adj_ids) PB_CUDA(cudaMemcpyAsync(adj_ids, M->adj_ids.p, M->nadj * 4, cudaMemcpyDeviceToHost, st));
    if (S && M->basis == PB_P1)
        PB_CUDA(cudaMemcpyAsync(S, M->D1.p, M->nadj * 36 * sizeof(double), cudaMemcpyDeviceToHost, st));
    else if (S)
        PB_CUDA(cudaMemcpyAsync(S, M->S_d.p, M->nadj * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    PB_API_END(ctx)
}

int pb_mesh_matvec(pb_ctx* ctx, pb_mesh* M, double eps_in, double eps_out, double kappa, int precision, int precond,
                   const double* x, double* y) {
    return pb_mesh_matvec_ex(ctx, M, eps_in, eps_out, kappa, precision, precond, PB_FORM_DIRECT, x, y);
}

int pb_mesh_matvec_ex(pb_ctx* ctx, pb_mesh* M, double eps_in, double eps_out, double kappa, int precision,
                      int precond, int formulation, const double* x, double* y) {
    if (!ctx || !M) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(x && y && eps_in > 0 && eps_out > 0 && kappa > 0, PB_EINVAL, "pb_mesh_matvec: bad arguments");
    PB_REQUIRE(precision == PB_MIXED || precision == PB_FP64, PB_EINVAL, "pb_mesh_matvec: unknown precision");
    PB_REQUIRE(formulation >= PB_FORM_DIRECT && formulation <= PB_FORM_INTERIOR, PB_EINVAL,
               "pb_mesh_matvec: unknown formulation");
    PB_REQUIRE(formulation == PB_FORM_DIRECT || M->basis == PB_P1, PB_EINVAL,
               "pb_mesh_matvec: the derivative formulations need a PB_P1 mesh");
    PB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t nb = 2 * M->nunk * sizeof(double);
    Staged sx;
    sx.in(x, nb, st);
    bool yh = !is_device_ptr(y);
    DBuf<char> yb;
    double* yd = y;
    if (yh) { yb.alloc(nb, st); yd = (double*)yb.p; }
    mesh_matvec(M, eps_in, eps_out, kappa, precision, (const double*)sx.dev, yd, precond, formulation);
    if (yh) PB_CUDA(cudaMemcpyAsync(y, yd, nb, cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    check_device_error(ctx);
    PB_API_END(ctx)
}

int pb_solve(pb_ctx* ctx, pb_mesh* M, const double* atoms, const double* q, int64_t na, double eps_in, double eps_out,
             double kappa, double tol, int max_iter, int precision, pb_result** out) {
    return pb_solve_ex(ctx, M, atoms, q, na, eps_in, eps_out, kappa, tol, max_iter, precision, PB_FORM_DIRECT, out);
}

int pb_solve_ex(pb_ctx* ctx, pb_mesh* M, const double* atoms, const double* q, int64_t na, double eps_in,
                double eps_out, double kappa, double tol, int max_iter, int precision, int formulation,
                pb_result** out) {
    if (!ctx || !M || !out) return PB_EINVAL;
    *out = nullptr;
    int status = PB_OK;
    PB_API_BEGIN
    PB_REQUIRE(atoms && q && na >= 1, PB_EINVAL, "pb_solve: need at least one charge");
    PB_REQUIRE(eps_in > 0 && eps_out > 0 && kappa > 0, PB_EINVAL, "pb_solve: eps and kappa must be > 0");
    PB_REQUIRE(tol >= 0 && max_iter >= 1 && max_iter <= 2000, PB_EINVAL, "pb_solve: tol >= 0 and 1 <= max_iter <= 2000");
    PB_REQUIRE(precision == PB_MIXED || precision == PB_FP64, PB_EINVAL, "pb_solve: unknown precision");
    PB_REQUIRE(formulation >= PB_FORM_DIRECT && formulation <= PB_FORM_INTERIOR, PB_EINVAL,
               "pb_solve: unknown formulation");
    PB_REQUIRE(formulation == PB_FORM_DIRECT || M->basis == PB_P1, PB_EINVAL,
               "pb_solve: the derivative formulations need a PB_P1 mesh");
    PB_CUDA(cudaSetDevice(ctx->device));
    pb_result* R = make_result(ctx, M, atoms, q, na, eps_in, eps_out, kappa, precision, formulation);
    *out = R;
    try {
        status = solve(M, R, tol, max_iter);
        check_device_error(ctx);
    } catch (...) {
        // no result object survives a failed call (PB_ENOCONV keeps its result)
        cudaStreamSynchronize(ctx->stream);
        delete R;
        *out = nullptr;
        throw;
    }
    if (status != PB_OK) {
        ctx->last_error = "pb_solve: GMRES did not reach tol within max_iter";
        return status;
    }
    PB_API_END(ctx)
}

int pb_result_destroy(pb_result* R) {
    if (!R) return PB_EINVAL;
    cudaStreamSynchronize(R->mesh->ctx->stream);
    delete R;
    return PB_OK;
}

int pb_result_get(const pb_result* R, int* iterations, double* residual, double* x) {
    if (!R) return PB_EINVAL;
    if (iterations) *iterations = R->iterations;
    if (residual) *residual = R->residual;
    if (x) {
        cudaError_t e = cudaMemcpy(x, R->x.p, 2 * R->nunk * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return PB_ECUDA;
    }
    return PB_OK;
}

int pb_solvation_energy(pb_ctx* ctx, pb_result* R, double* dG, double* phir) {
    if (!ctx || !R || !dG) return PB_EINVAL;
    PB_API_BEGIN
    PB_CUDA(cudaSetDevice(ctx->device));
    reaction_energy(R, phir, dG);
    R->energy = *dG;
    R->have_energy = true;
    PB_API_END(ctx)
}

int pb_solve_batch(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, const double* const* atoms,
                   const double* const* charges, const int64_t* na, double eps_in, double eps_out, double kappa,
                   double tol, int max_iter, int precision, pb_result** out, int* status) {
    return pb_solve_batch_ex(ctx, meshes, nsys, atoms, charges, na, eps_in, eps_out, kappa, tol, max_iter, precision,
                             PB_FORM_DIRECT, out, status);
}

int pb_solve_batch_ex(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, const double* const* atoms,
                      const double* const* charges, const int64_t* na, double eps_in, double eps_out, double kappa,
                      double tol, int max_iter, int precision, int formulation, pb_result** out, int* status) {
    if (!ctx || !meshes || nsys < 1 || !atoms || !charges || !na || !out || !status) return PB_EINVAL;
    for (int s = 0; s < nsys; ++s) out[s] = nullptr;
    int rc = PB_OK;
    PB_API_BEGIN
    PB_REQUIRE(eps_in > 0 && eps_out > 0 && kappa > 0, PB_EINVAL, "pb_solve_batch: eps and kappa must be > 0");
    PB_REQUIRE(tol >= 0 && max_iter >= 1 && max_iter <= 2000, PB_EINVAL, "pb_solve_batch: bad tol or max_iter");
    PB_REQUIRE(precision == PB_MIXED || precision == PB_FP64, PB_EINVAL, "pb_solve_batch: unknown precision");
    PB_REQUIRE(formulation >= PB_FORM_DIRECT && formulation <= PB_FORM_INTERIOR, PB_EINVAL,
               "pb_solve_batch: unknown formulation");
    for (int s = 0; s < nsys; ++s) {
        PB_REQUIRE(meshes[s] && atoms[s] && charges[s] && na[s] >= 1, PB_EINVAL, "pb_solve_batch: empty system");
        PB_REQUIRE(formulation == PB_FORM_DIRECT || meshes[s]->basis == PB_P1, PB_EINVAL,
                   "pb_solve_batch: the derivative formulations need PB_P1 meshes");
        for (int t = 0; t < s; ++t)
            PB_REQUIRE(meshes[t] != meshes[s], PB_EINVAL, "pb_solve_batch: meshes must be distinct");
    }
    PB_CUDA(cudaSetDevice(ctx->device));
    try {
        for (int s = 0; s < nsys; ++s)
            out[s] = make_result(ctx, meshes[s], atoms[s], charges[s], na[s], eps_in, eps_out, kappa, precision,
                                 formulation);
        solve_batch(ctx, meshes, nsys, out, tol, max_iter, status);
        check_device_error(ctx);
    } catch (...) {
        cudaStreamSynchronize(ctx->stream);
        for (int s = 0; s < nsys; ++s) {
            delete out[s];
            out[s] = nullptr;
        }
        throw;
    }
    for (int s = 0; s < nsys; ++s)
        if (status[s] != PB_OK) rc = PB_ENOCONV;
    if (rc != PB_OK) {
        ctx->last_error = "pb_solve_batch: some systems did not reach tol within max_iter";
        return rc;
    }
    PB_API_END(ctx)
}

int pb_tune_ncrit(pb_ctx* ctx, const float* xyz, int64_t n, int p, const int32_t* cand, int ncand, int* best,
                  double* best_ms) {
    if (!ctx || !xyz || n < 1 || !cand || ncand < 1 || !best) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(p >= 2 && p <= 10, PB_EINVAL, "pb_tune_ncrit: p must be in [2, 10]");
    for (int c = 0; c < ncand; ++c) PB_REQUIRE(cand[c] >= 1, PB_EINVAL, "pb_tune_ncrit: ncrit must be >= 1");
    PB_CUDA(cudaSetDevice(ctx->device));
    Staged s;
    s.in(xyz, (size_t)n * 3 * sizeof(float), ctx->stream);
    tune_ncrit(ctx, (const float*)s.dev, n, p, cand, ncand, best, best_ms);
    check_device_error(ctx);
    PB_API_END(ctx)
}

int pb_tune(pb_ctx* ctx, const float* xyz, int64_t n, int p, const int32_t* cand, int ncand, int* best,
            int* best_nt, int* best_tile, double* best_ms) {
    if (!ctx || !xyz || n < 1 || !cand || ncand < 1 || !best) return PB_EINVAL;
    PB_API_BEGIN
    PB_REQUIRE(p >= 2 && p <= 10, PB_EINVAL, "pb_tune: p must be in [2, 10]");
    for (int c = 0; c < ncand; ++c) PB_REQUIRE(cand[c] >= 1, PB_EINVAL, "pb_tune: ncrit must be >= 1");
    PB_CUDA(cudaSetDevice(ctx->device));
    Staged s;
    s.in(xyz, (size_t)n * 3 * sizeof(float), ctx->stream);
    tune_fmm(ctx, (const float*)s.dev, n, p, cand, ncand, best, best_nt, best_tile, best_ms);
    check_device_error(ctx);
    PB_API_END(ctx)
}

int pb_energy_grad(pb_ctx* ctx, pb_result* R, double tol, int max_iter, double* dEdq, double* dEdx) {
    if (!ctx || !R) return PB_EINVAL;
    int status = PB_OK;
    PB_API_BEGIN
    PB_REQUIRE(tol >= 0 && max_iter >= 1 && max_iter <= 2000, PB_EINVAL, "pb_energy_grad: bad tol or max_iter");
    PB_REQUIRE(R->mesh->basis == PB_P0 && R->formulation == PB_FORM_DIRECT, PB_EINVAL,
               "pb_energy_grad: direct-formulation results on P0 meshes only");
    PB_CUDA(cudaSetDevice(ctx->device));
    status = energy_gradient(R, tol, max_iter, dEdq, dEdx);
    check_device_error(ctx);
    if (status != PB_OK) {
        ctx->last_error = "pb_energy_grad: adjoint GMRES did not reach tol within max_iter";
        return status;
    }
    PB_API_END(ctx)
}

// ---------------------------------------------------------------------------
// test hooks (include/pbfmm_testing.h)
// ---------------------------------------------------------------------------
int64_t pbfmm_test_alloc_count(void) { return g_alloc_count.load(); }

void pbfmm_test_fail_alloc(int64_t nth) {
    g_alloc_fail_at.store(nth > 0 ? g_alloc_count.load() + nth : 0);
}

int64_t pbfmm_test_pool_used(int device) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return -1;
    uint64_t used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) return -1;
    return (int64_t)used;
}

void pbfmm_test_wait_limit(int64_t cycles) { g_wait_limit.store(cycles > 0 ? cycles : kDefaultWaitLimit); }

}  // extern "C"
