// C-ABI entry points (declared in include/pbfmm.h).  Every entry point turns
// internal exceptions into a status code and a message on the context.
#include "fmm.cuh"
#include <new>

namespace pbfmm {
void build_tree(fmm_tree* T, const float* src, const float* tgt);
void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn);

thread_local long long g_launch_count = 0;

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
    *out = ctx;
    PB_API_END(ctx)
}

int pb_destroy(pb_ctx* ctx) {
    if (!ctx) return PB_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return PB_OK;
}

const char* pb_last_error(pb_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

int pb_sync(pb_ctx* ctx) {
    if (!ctx) return PB_EINVAL;
    PB_API_BEGIN
    PB_CUDA(cudaSetDevice(ctx->device));
    PB_CUDA(cudaStreamSynchronize(ctx->stream));
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
    if (out_host || dn_host || sq.buf.p || sd.buf.p || sn.buf.p || tn.buf.p) PB_CUDA(cudaStreamSynchronize(st));
    PB_API_END(ctx)
}

}  // extern "C"
