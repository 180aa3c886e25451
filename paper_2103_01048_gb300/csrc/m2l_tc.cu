// M2L on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// The V-list pairs (Sec. "Fast multipole method": interaction list I(B)) are
// grouped by (level, relative offset): all pairs of a group share one M2L
// operator (with the DC2DE solve folded in, FP64-built, FP32-stored).  A CTA
// owns one group chunk and one part of the operator: a block of its output
// rows times a block of its inner columns (two row halves up to p = 6;
// 4 x 2 parts at p = 8, 4 x 4 at p = 10), so that the part fits in shared
// memory:
//   * the operator part, split into TF32 hi + lo parts and pre-swizzled in
//     global memory (128B swizzle, K-major), is copied into shared memory
//     once with cp.async.bulk and stays resident;
//   * 128-pair row tiles stream through: the producer threads gather the
//     source boxes' upward densities (the part's columns of the Qu rows),
//     split them into TF32 hi + lo and write them swizzled into a ring of
//     A stages;
//   * one thread issues tcgen05.mma kind::tf32 (M = 128 pairs, N = the
//     part's rows, K = 8 per instruction), three products per k-step
//     (hi*hi + hi*lo + lo*hi: FP32-level accuracy), accumulating in TMEM;
//   * the epilogue reads the accumulator with tcgen05.ld and adds each row
//     into the target box's downward density with red.global.add.v4.f32
//     (targets of one group are distinct; groups and inner parts overlap,
//     hence the reduction).  Summation order across groups is not fixed.
// Every wait is bounded (~1 s); on a timeout the kernel records an error
// code, drains its own MMAs, frees TMEM and returns.
#include "fmm.cuh"
#include "tc_ptx.cuh"
#include <cub/cub.cuh>
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <memory>

namespace pbfmm {

void radix_sort_pairs(const unsigned* keys_in, const int* vals_in, unsigned* keys_out, int* vals_out, long long n,
                      int bits, cudaStream_t st);

constexpr int kTcRows = 128;           // pairs per row tile (MMA M)
constexpr int kTcItemPairs = 2048;     // pairs per M2L work item (one operator load each)
constexpr int kTcSmallItemPairs = 512; // M2M / L2L / check->equivalent items: fewer pairs per operator, more CTAs
constexpr int kTcOffItemPairs = 8192;  // items of a level-invariant M2L set (one offset, all levels)

// Operator split per padded size: NS parts of the output rows (MMA N =
// npad / NS) times KS parts of the inner dimension (npad / KS columns,
// whole 32-column blocks), so that one part (TF32 hi + lo) stays resident
// in shared memory beside a ring of STAGES A stages.  Each CTA owns one
// part; the KS parts of a row add into the target with the reduction.
template <int NPAD> struct TcCfg { static constexpr int NS = 2, KS = 1, STAGES = 3; };
template <> struct TcCfg<320> { static constexpr int NS = 4, KS = 2, STAGES = 3; };   // p = 8
template <> struct TcCfg<512> { static constexpr int NS = 4, KS = 4, STAGES = 2; };   // p = 10
static bool tc_split(int npad, int& ns, int& ks) {
    switch (npad) {
        case 32: case 64: case 128: case 160: ns = 2; ks = 1; return true;
        case 320: ns = TcCfg<320>::NS; ks = TcCfg<320>::KS; return true;
        case 512: ns = TcCfg<512>::NS; ks = TcCfg<512>::KS; return true;
        default: return false;
    }
}

// TF32 part of x, rounded to nearest (ties away from zero); x - hi is exact in FP32
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// ---------------------------------------------------------------------------
// operator packing: [matrix][part = ns * KS + ks][hi|lo][kb][nh rows][32]
// swizzled (nh = npad / NS output rows, KB = npad / KS / 32 blocks of 32
// inner columns); the part a CTA owns is one contiguous block
// ---------------------------------------------------------------------------
__global__ void k_pack_m2l_tc(int npad, int NS, int KS, long long nmat, const float* __restrict__ m2l,
                              float* __restrict__ out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long m2 = (long long)npad * npad;
    if (idx >= nmat * m2) return;
    long long mat = idx / m2;
    int n = (int)((idx % m2) / npad), k = (int)(idx % npad);
    const int nh = npad / NS, kc = npad / KS, kb_n = kc / 32;
    int ns = n / nh, nr = n % nh, ks = k / kc, kk = k % kc, kb = kk / 32, kq = kk % 32;
    float x = m2l[idx];
    float hi = tf32_hi(x), lo = x - hi;
    const long long part_bytes = 2LL * kb_n * nh * 128;
    char* base = (char*)out + (mat * NS * KS + ns * KS + ks) * part_bytes;
    uint32_t off = (uint32_t)kb * nh * 128 + sw128_off(nr, kq);
    *(float*)(base + off) = hi;
    *(float*)(base + (long long)kb_n * nh * 128 + off) = lo;
}

static void pack_tc(int npad, long long nmat, const float* src, DBuf<float>& dst, cudaStream_t st) {
    int ns = 0, ks = 0;
    if (!tc_split(npad, ns, ks)) throw Error(PB_EINVAL, "no tensor-core split for this operator size");
    const long long m2 = (long long)npad * npad;
    dst.alloc(nmat * m2 * 2, st);
    k_pack_m2l_tc<<<div_up(nmat * m2, 256), 256, 0, st>>>(npad, ns, ks, nmat, src, dst.p);
    PB_CHECK_LAUNCH();
}

// Laplace M2L operators (the down-check -> down-equivalent solve folded in)
// do not depend on the level: the 1/r kernel scales as 2^l with the box
// size and the regularised pseudo-inverse as 2^-l.  Their tensor-core copy
// keeps one level (the first with interaction lists), indexed by offset.
void pack_m2l_tc(Operators& O, cudaStream_t st) {
    int ns = 0, ks = 0;
    if (!tc_split(O.npad, ns, ks)) { O.have_tc = false; return; }
    O.m2l_tc_single = O.kernel == FMM_LAPLACE && O.nlev > 2;
    if (O.m2l_tc_single) pack_tc(O.npad, kNumOffsets, O.m2l.p + 2LL * kNumOffsets * O.npad * O.npad, O.m2l_tc, st);
    else pack_tc(O.npad, (long long)O.nlev * kNumOffsets, O.m2l.p, O.m2l_tc, st);
    if (O.m2m.p) pack_tc(O.npad, (long long)O.nlev * 8, O.m2m.p, O.m2m_tc, st);
    if (O.l2l.p) pack_tc(O.npad, (long long)O.nlev * 8, O.l2l.p, O.l2l_tc, st);
    if (O.uc2ue_w1.p) {
        pack_tc(O.npad, O.nlev, O.uc2ue_w1.p, O.uc2ue_w1_tc, st);
        pack_tc(O.npad, O.nlev, O.uc2ue_w2.p, O.uc2ue_w2_tc, st);
        pack_tc(O.npad, O.nlev, O.dc2de_w1.p, O.dc2de_w1_tc, st);
        pack_tc(O.npad, O.nlev, O.dc2de_w2.p, O.dc2de_w2_tc, st);
    }
    O.have_tc = true;
}

// ---------------------------------------------------------------------------
// V-list pairs grouped by (level, offset)
// ---------------------------------------------------------------------------
__global__ void k_pairs_emit(int nbox, const int* V, const int* V_n, const int* V_off, const int4* anchor,
                             int* key, int* tgt, int* src) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int4 ab = anchor[b];
    for (int i = 0; i < V_n[b]; ++i) {
        int s = V[(long long)b * kVCap + i];
        int4 as = anchor[s];
        int o = (as.x - ab.x + 3) * 49 + (as.y - ab.y + 3) * 7 + (as.z - ab.z + 3);
        int e = V_off[b] + i;
        key[e] = o * 32 + ab.w;            // offset-major, then level (< 22)
        tgt[e] = b;
        src[e] = s;
    }
}

__global__ void k_gather_int(int n, const int* idx, const int* a, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[idx[i]];
}

void build_m2l_pairs(fmm_tree* T) {
    cudaStream_t st = T->ctx->stream;
    const int nb = T->nbox;
    const long long np = T->n_v;
    auto& P = T->m2l_pairs;
    P.npairs = np;
    P.nitems = 0;
    if (np == 0) return;
    DBuf<int> voff, key, tgt, src, idx, key_s, idx_s;
    voff.alloc(nb + 1, st);
    {
        size_t tmp = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tmp, T->V_n.p, voff.p, nb, st);
        DBuf<char> t;
        t.alloc(std::max<size_t>(tmp, 1), st);
        cub::DeviceScan::ExclusiveSum(t.p, tmp, T->V_n.p, voff.p, nb, st);
    }
    key.alloc(np, st); tgt.alloc(np, st); src.alloc(np, st);
    k_pairs_emit<<<div_up(nb, 128), 128, 0, st>>>(nb, T->V.p, T->V_n.p, voff.p, T->anchor.p, key.p, tgt.p, src.p);
    PB_CHECK_LAUNCH();
    idx.alloc(np, st); key_s.alloc(np, st); idx_s.alloc(np, st);
    std::vector<int> hidx(np);
    for (long long i = 0; i < np; ++i) hidx[i] = (int)i;
    PB_CUDA(cudaMemcpyAsync(idx.p, hidx.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    // group by (offset, level) keeping each group in box order (stable sort;
    // offset * 32 + level < 2^14)
    radix_sort_pairs((const unsigned*)key.p, idx.p, (unsigned*)key_s.p, idx_s.p, np, 14, st);
    P.tgt.alloc(np, st);
    P.src.alloc(np, st);
    k_gather_int<<<div_up(np, 256), 256, 0, st>>>((int)np, idx_s.p, tgt.p, P.tgt.p);
    k_gather_int<<<div_up(np, 256), 256, 0, st>>>((int)np, idx_s.p, src.p, P.src.p);
    PB_CHECK_LAUNCH();
    std::vector<int> hk(np);
    PB_CUDA(cudaMemcpyAsync(hk.data(), key_s.p, np * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    // work items: (first pair, pair count <= kTcItemPairs, operator index =
    // level * 343 + offset, 0) per (offset, level) group; and per offset
    // (all levels, <= kTcOffItemPairs pairs, operator index = offset) for a
    // level-invariant operator set
    std::vector<int4> items, items_off;
    long long i = 0;
    while (i < np) {
        long long j = i;
        while (j < np && hk[j] == hk[i]) ++j;
        const int off = hk[i] / 32, lvl = hk[i] % 32;
        for (long long a = i; a < j; a += kTcItemPairs)
            items.push_back(make_int4((int)a, (int)std::min<long long>(kTcItemPairs, j - a), lvl * kNumOffsets + off, 0));
        i = j;
    }
    i = 0;
    while (i < np) {
        long long j = i;
        while (j < np && hk[j] / 32 == hk[i] / 32) ++j;
        for (long long a = i; a < j; a += kTcOffItemPairs)
            items_off.push_back(make_int4((int)a, (int)std::min<long long>(kTcOffItemPairs, j - a), hk[i] / 32, 0));
        i = j;
    }
    P.nitems_off = (int)items_off.size();
    P.items_off.alloc(items_off.size(), st);
    PB_CUDA(cudaMemcpyAsync(P.items_off.p, items_off.data(), items_off.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            st));
    P.nitems = (int)items.size();
    P.items.alloc(items.size(), st);
    PB_CUDA(cudaMemcpyAsync(P.items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    std::vector<int4> items32;
    for (const int4& it : items)
        for (int a = 0; a < it.y; a += 32) items32.push_back(make_int4(it.x + a, std::min(32, it.y - a), it.z, 0));
    P.nitems32 = (int)items32.size();
    P.items32.alloc(items32.size(), st);
    PB_CUDA(cudaMemcpyAsync(P.items32.p, items32.data(), items32.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaStreamSynchronize(st));
}

// Items of the check -> equivalent solves on the tensor cores: the boxes of
// each level (one row each) in chunks of at most kTcItemPairs.
static void level_items(const std::vector<int>& lvl_off, int nlev, DBuf<int4>& items, int& n, cudaStream_t st) {
    std::vector<int4> h;
    for (int l = 0; l < nlev; ++l)
        for (int a = lvl_off[l]; a < lvl_off[l + 1]; a += kTcSmallItemPairs)
            h.push_back(make_int4(a, std::min(kTcSmallItemPairs, lvl_off[l + 1] - a), l, 0));
    n = (int)h.size();
    if (h.empty()) return;
    items.alloc(h.size(), st);
    PB_CUDA(cudaMemcpyAsync(items.p, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaStreamSynchronize(st));
}

void build_c2e_items(fmm_tree* T) {
    cudaStream_t st = T->ctx->stream;
    if ((int)T->sleaf_lvl_off.size() == T->nlev + 1)
        level_items(T->sleaf_lvl_off, T->nlev, T->c2e_items_up, T->n_c2e_up, st);
    if ((int)T->xbox_lvl_off.size() == T->nlev + 1)
        level_items(T->xbox_lvl_off, T->nlev, T->c2e_items_dn, T->n_c2e_dn, st);
}

// Parent-child pairs for M2M / L2L on the tensor cores: children of level
// >= 3 grouped by (level, octant), ascending box order inside a group.
void build_pc_pairs(fmm_tree* T) {
    cudaStream_t st = T->ctx->stream;
    auto& P = T->pc_pairs;
    const int nb = T->nbox;
    std::vector<int> par(nb);
    std::vector<int4> anc(nb);
    PB_CUDA(cudaMemcpyAsync(par.data(), T->parent.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(anc.data(), T->anchor.p, nb * sizeof(int4), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    std::vector<std::vector<int>> bucket((size_t)T->nlev * 8);
    for (int c = 0; c < nb; ++c) {
        if (anc[c].w < 3) continue;
        int oct = ((anc[c].x & 1) << 2) | ((anc[c].y & 1) << 1) | (anc[c].z & 1);
        bucket[(size_t)anc[c].w * 8 + oct].push_back(c);
    }
    std::vector<int> hp, hc;
    std::vector<int4> items;
    P.level_item_off.assign(T->nlev + 1, 0);
    for (int l = 0; l < T->nlev; ++l) {
        P.level_item_off[l] = (int)items.size();
        for (int o = 0; o < 8; ++o) {
            auto& v = bucket[(size_t)l * 8 + o];
            for (size_t a = 0; a < v.size(); a += kTcSmallItemPairs) {
                int cnt = (int)std::min<size_t>(kTcSmallItemPairs, v.size() - a);
                items.push_back(make_int4((int)hc.size(), cnt, l * 8 + o, 0));
                for (int k = 0; k < cnt; ++k) { hc.push_back(v[a + k]); hp.push_back(par[v[a + k]]); }
            }
        }
    }
    P.level_item_off[T->nlev] = (int)items.size();
    P.nitems = (int)items.size();
    if (items.empty()) return;
    P.parent.alloc(hp.size(), st);
    P.child.alloc(hc.size(), st);
    P.items.alloc(items.size(), st);
    PB_CUDA(cudaMemcpyAsync(P.parent.p, hp.data(), hp.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(P.child.p, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaMemcpyAsync(P.items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    PB_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// the kernel: warp-specialised pipeline
//   warps 0-7   producers: two threads per pair row gather the source box's
//               Qu row, split it into TF32 hi + lo and write it swizzled
//               into a ring of A stages (one K block each);
//   warps 8-11  epilogue: one TMEM lane quarter each; read the finished
//               accumulator and add every row into its target's Qd row;
//   warp 12     one thread issues the MMAs and the commits.
// Two TMEM accumulators alternate between tiles, so the epilogue of a tile
// overlaps the MMAs of the next and the gathers of the one after.
// ---------------------------------------------------------------------------
constexpr int kTcProdWarps = 8;
constexpr int kTcEpiWarps = 4;
constexpr int kTcThreads = 32 * (kTcProdWarps + kTcEpiWarps + 1);

constexpr int kTcEpiLd = 16;                    // accumulator columns per epilogue TMEM load
constexpr int kTcEpiStride = 20;                // padded row of the epilogue transpose buffer (floats)

template <int STAGES>
struct TcSmem {
    // per epilogue warp: 32 rows x kTcEpiLd columns, transposed through shared
    // memory so that each reduction instruction covers 8 rows x 64 B
    alignas(16) float epi[kTcEpiWarps][32][kTcEpiStride];
    uint64_t barB, full[STAGES], empty[STAGES], accf[2], acce[2];
    uint32_t tmem_slot;
    int failed;
};

// bounded wait that gives up as soon as another role of the CTA has failed;
// a timeout marks the CTA failed
__device__ __forceinline__ bool mbar_wait_cta(uint64_t* bar, uint32_t parity, volatile int* failed,
                                              long long limit) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*failed) return false;
        if (clock64() - t0 > limit) {
            *failed = 1;
            return false;
        }
    }
    return true;
}

// Operator set and box vectors of one launch; blockIdx.z selects the set, so
// one launch serves the Laplace and the Yukawa half of the paired apply
// (their pair lists and operator indices coincide).
struct TcSets {
    const float* ops[2];
    const float* X[2];
    float* Y[2];
    int single[2];           // 1: the set holds one level of M2L operators, indexed by offset alone
    long long wait_limit;    // cycles a role waits on a barrier before giving up (set at launch)
    int* trace;              // optional progress markers of the CTA-pair kernel (host-mapped), or null
    int ncols;               // output columns that can be nonzero (n_e; the rest is padding); 0: all
};

// progress marker of the CTA-pair kernel (self-test diagnostics): slot k of
// cluster rank r of the first cluster, written to host-mapped memory so it
// stays readable after a failed launch
__device__ __forceinline__ void tc_mark(int* trace, uint32_t rank, int k, int v) {
    if (trace && blockIdx.y == 0 && blockIdx.x < 2 && blockIdx.z == 0) {
        *(volatile int*)&trace[rank * 8 + k] = v;
        __threadfence_system();
    }
}

template <int NPAD>
__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(const int4* __restrict__ items, const int* __restrict__ ptgt,
                                                          const int* __restrict__ psrc, const TcSets sets,
                                                          int* __restrict__ err) {
    // Generic tensor-core box-operator product: for every pair p of the
    // item, Y[tgt[p]] += Op(item) X[src[p]] (Op resident for the CTA).
    // Used for M2L (operator per level and offset), for M2M / L2L
    // (operator per child level and octant) and for the factored
    // check -> equivalent solves (operator per level).
    const float* __restrict__ ops = sets.ops[blockIdx.z];
    const float* __restrict__ Qu = sets.X[blockIdx.z];
    float* __restrict__ Qd = sets.Y[blockIdx.z];
    const long long wl = sets.wait_limit;
    constexpr int NS = TcCfg<NPAD>::NS, KS = TcCfg<NPAD>::KS, kTcStages = TcCfg<NPAD>::STAGES;
    constexpr int NH = NPAD / NS;                    // output rows of this CTA (MMA N)
    constexpr int KC = NPAD / KS;                    // inner columns of this CTA
    constexpr int KB = KC / 32;                      // K blocks of 32 tf32 (128 B)
    static_assert(NH % 16 == 0 && NH <= 256 && KC % 32 == 0, "tensor-core split");
    constexpr uint32_t B_SPLIT = KB * NH * 128;      // bytes of one of hi / lo
    constexpr uint32_t A_SPLIT = kTcRows * 128;      // 16 KB
    constexpr uint32_t ACOLS = NH <= 32 ? 32 : (NH <= 64 ? 64 : (NH <= 128 ? 128 : 256));   // one accumulator
    constexpr uint32_t TCOLS = 2 * ACOLS;
    constexpr uint32_t IDESC = idesc_tf32(NH);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem;                               // [hi|lo][KB][NH][128]
    uint8_t* sA = smem + 2 * B_SPLIT;                 // [stage][hi|lo][128][128]
    TcSmem<kTcStages>* S = (TcSmem<kTcStages>*)(sA + kTcStages * 2 * A_SPLIT);
    volatile int* failed = &S->failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 it = items[blockIdx.x];
    const int part = blockIdx.y;                     // operator part: rows half, inner columns kpart
    const int half = part / KS, kpart = part % KS;
    const int first = it.x, npairs = it.y;
    const int opi = sets.single[blockIdx.z] ? it.z % kNumOffsets : it.z;
    const int ntile = (npairs + kTcRows - 1) / kTcRows;

    if (tid == 0) {
        mbar_init(&S->barB, 1);
        for (int q = 0; q < kTcStages; ++q) {
            mbar_init(&S->full[q], kTcProdWarps * 32);
            mbar_init(&S->empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&S->accf[q], 1);
            mbar_init(&S->acce[q], kTcEpiWarps * 32);
        }
        S->failed = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&S->tmem_slot, TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = S->tmem_slot;

    // resident operator part: hi and lo, one bulk copy each
    if (tid == 0) {
        const uint8_t* gB = (const uint8_t*)ops + ((long long)opi * (NS * KS) + part) * (2LL * B_SPLIT);
        mbar_arrive_expect_tx(&S->barB, 2 * B_SPLIT);
        bulk_g2s(sB, gB, B_SPLIT, &S->barB);
        bulk_g2s(sB + B_SPLIT, gB + B_SPLIT, B_SPLIT, &S->barB);
    }

    if (warp < kTcProdWarps) {
        // ---- producers: lane l8 = lane % 8 carries 16 B of a 128-B K-block row;
        // a warp instruction covers 4 whole rows (coalesced). Thread rows:
        // i * 32 + warp * 4 + lane / 8, i = 0..3.
        const int l8 = lane & 7, rbase = warp * 4 + (lane >> 3);
        auto src_of = [&](int tile, int i) -> int {
            const int r = tile * kTcRows + i * 32 + rbase;
            return (tile < ntile && r < npairs) ? psrc[first + r] : -1;
        };
        // Register rotation: once K block kb of a tile is in its stage, the
        // same registers load block kb of the next tile, so each gather has a
        // whole tile of MMA time to arrive.
        float4 v[KB][4];
        int sn[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s0 = src_of(0, i);
            const float4* q4 = s0 >= 0 ? (const float4*)(Qu + (size_t)s0 * NPAD + kpart * KC) : nullptr;
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) v[kb][i] = q4 ? q4[kb * 8 + l8] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) sn[i] = src_of(1, i);
        int g = 0;
        for (int tile = 0; tile < ntile; ++tile) {
#pragma unroll
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = g % kTcStages, n = g / kTcStages;
                if (n > 0 && !mbar_wait_cta(&S->empty[s], (n - 1) & 1, failed, wl)) goto prod_done;
                uint8_t* aHi = sA + (size_t)s * 2 * A_SPLIT;
                uint8_t* aLo = aHi + A_SPLIT;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 x = v[kb][i];
                    float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
                    uint32_t off = sw128_off(i * 32 + rbase, l8 * 4);
                    *(float4*)(aHi + off) = h;
                    *(float4*)(aLo + off) = l;
                }
                fence_proxy_async();
                mbar_arrive(&S->full[s]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4* qn = sn[i] >= 0 ? (const float4*)(Qu + (size_t)sn[i] * NPAD + kpart * KC) : nullptr;
                    v[kb][i] = qn ? qn[kb * 8 + l8] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sn[i] = src_of(tile + 2, i);
        }
    prod_done:
        __syncwarp();
    } else if (warp < kTcProdWarps + kTcEpiWarps) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) ... + 31
        const int q = warp & 3;
        const int erow = q * 32 + lane;
        for (int tile = 0; tile < ntile; ++tile) {
            const int a = tile & 1, u = tile >> 1;
            const int r = tile * kTcRows + erow;
            const int t = r < npairs ? ptgt[first + r] : -1;
            bool ok = mbar_wait_cta(&S->accf[a], u & 1, failed, wl);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            float (*buf)[kTcEpiStride] = S->epi[q];
#pragma unroll 1
            for (int c0 = 0; c0 < NH; c0 += kTcEpiLd) {
                float v[kTcEpiLd];
                tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + a * ACOLS + c0, v);
#pragma unroll
                for (int c = 0; c < kTcEpiLd; c += 4)
                    *(float4*)&buf[lane][c] = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
                __syncwarp();
                // lane: row j * 8 + lane / 4 of the warp's 32, columns 4 (lane % 4) .. + 3
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int rr = j * 8 + (lane >> 2), cc = (lane & 3) * 4;
                    const float4 x = *(const float4*)&buf[rr][cc];
                    const int tr = __shfl_sync(0xffffffffu, t, rr);
                    if (tr >= 0) red_add_v4(Qd + (size_t)tr * NPAD + half * NH + c0 + cc, x.x, x.y, x.z, x.w);
                }
                __syncwarp();
            }
            tc_fence_before();
            mbar_arrive(&S->acce[a]);
        }
        __syncwarp();
    } else {
        // ---- MMA issuer
        if (lane == 0) {
            uint64_t* last = nullptr;      // barrier of the last commit, and its phase parity
            uint32_t last_par = 0;
            int g = 0;
            bool ok = mbar_wait_cta(&S->barB, 0, failed, wl);
            for (int tile = 0; ok && tile < ntile; ++tile) {
                const int a = tile & 1, u = tile >> 1;
                if (u > 0 && !(ok = mbar_wait_cta(&S->acce[a], (u - 1) & 1, failed, wl))) break;
                const uint32_t dacc = taddr + a * ACOLS;
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int s = g % kTcStages, n = g / kTcStages;
                    if (!(ok = mbar_wait_cta(&S->full[s], n & 1, failed, wl))) break;
                    tc_fence_after();
                    const uint32_t aH = smem_u32(sA + (size_t)s * 2 * A_SPLIT), aL = aH + A_SPLIT;
                    const uint32_t bH = smem_u32(sB) + kb * NH * 128, bL = bH + B_SPLIT;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc0 = (kb > 0 || ks > 0) ? 1u : 0u;
                        mma_tf32(dacc, sw128_desc(aH + ks * 32), sw128_desc(bH + ks * 32), IDESC, acc0);
                        mma_tf32(dacc, sw128_desc(aH + ks * 32), sw128_desc(bL + ks * 32), IDESC, 1u);
                        mma_tf32(dacc, sw128_desc(aL + ks * 32), sw128_desc(bH + ks * 32), IDESC, 1u);
                    }
                    mma_commit(&S->empty[s]);
                    last = &S->empty[s];
                    last_par = n & 1;
                }
                if (!ok) break;
                mma_commit(&S->accf[a]);
                last = &S->accf[a];
                last_par = u & 1;
            }
            // after a failure: every MMA issued here has completed before TMEM is freed
            if (!ok && last) mbar_wait(last, last_par);
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && S->failed) {
        atomicExch(err, 1);
        mbar_wait(&S->barB, 0);         // the operator copy has landed before shared memory is released
    }
    if (warp == 0) tmem_dealloc(taddr, TCOLS);
}

// ---------------------------------------------------------------------------
// CTA-pair variant (cluster of two CTAs, tcgen05 cta_group::2).  The two CTAs
// of a cluster (consecutive along grid x: the pairs of tcgen05 cta_group::2
// are formed along the cluster's x dimension) hold the two row parts
// ns = 2 c and 2 c + 1 of the same inner
// part and split every 256-pair row tile: CTA r gathers the tile's rows
// r * 128 ... r * 128 + 127 into its own A stages.  The even CTA issues
// MMAs of M = 256, N = 2 NH: A rows come from both CTAs' stages, B columns
// from both CTAs' operator parts (the same shared-memory offsets in both),
// and each CTA's tensor memory receives its own 128 rows x 2 NH columns.
// Against the single-CTA kernel every source row is gathered once instead
// of once per row part, and each A tile feeds twice the columns.
//   producers and epilogues arrive (one per warp) on their own CTA's
//   barriers; the odd CTA's warp 12 relays each completed event (operator
//   part, full A stage, drained accumulator) to the even CTA's barrier with
//   one cluster-scope arrival;
//   MMA issuer (even CTA): commits to `empty` / `accf` of both CTAs.
// Cluster barriers after the set-up and before the teardown keep every
// remote arrival and MMA inside the lifetime of both CTAs.
// ---------------------------------------------------------------------------
template <int STAGES>
struct TcPairSmem {
    alignas(16) float epi[kTcEpiWarps][32][kTcEpiStride];
    uint64_t barB, barBp, full[STAGES], empty[STAGES], accf[2], acce[2];
    uint64_t pfull[STAGES], pacce[2];     // odd CTA: its warps' arrivals, relayed to the even CTA
    uint32_t tmem_slot;
    int failed;
};

// bounded wait on a barrier that threads of the other CTA arrive on
__device__ __forceinline__ bool mbar_wait_cta_cl(uint64_t* bar, uint32_t parity, volatile int* failed,
                                                 long long limit) {
    long long t0 = clock64();
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (*failed) return false;
        if (clock64() - t0 > limit) {
            *failed = 1;
            return false;
        }
    }
    return true;
}

template <int NPAD>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc2(const int4* __restrict__ items, const int* __restrict__ ptgt, const int* __restrict__ psrc,
              const TcSets sets, int* __restrict__ err) {
    const float* __restrict__ ops = sets.ops[blockIdx.z];
    const float* __restrict__ Qu = sets.X[blockIdx.z];
    float* __restrict__ Qd = sets.Y[blockIdx.z];
    const long long wl = sets.wait_limit;
    constexpr int NS = TcCfg<NPAD>::NS, KS = TcCfg<NPAD>::KS, kTcStages = TcCfg<NPAD>::STAGES;
    constexpr int NH = NPAD / NS;                    // operator rows held by this CTA
    constexpr int NP = 2 * NH;                       // MMA N: the rows of the pair
    constexpr int KC = NPAD / KS;                    // inner columns of this part
    constexpr int KB = KC / 32;                      // K blocks of 32 tf32 (128 B)
    constexpr int TILE = 2 * kTcRows;                // pairs per MMA row tile (M = 256)
    static_assert(NS % 2 == 0 && NP % 16 == 0 && NP >= 32 && NP <= 256 && KC % 32 == 0, "CTA-pair split");
    constexpr uint32_t B_SPLIT = KB * NH * 128;      // bytes of one of hi / lo
    constexpr uint32_t A_SPLIT = kTcRows * 128;      // 16 KB
    constexpr uint32_t ACOLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : 256));
    constexpr uint32_t TCOLS = 2 * ACOLS;
    constexpr uint32_t IDESC = idesc_tf32_mn(256, NP);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem;                               // [hi|lo][KB][NH][128]
    uint8_t* sA = smem + 2 * B_SPLIT;                 // [stage][hi|lo][128][128]
    TcPairSmem<kTcStages>* S = (TcPairSmem<kTcStages>*)(sA + kTcStages * 2 * A_SPLIT);
    volatile int* failed = &S->failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // grid (x: 2 x part pairs, y: items, z: operator sets), clusters of two along x
    const uint32_t rank = cluster_ctarank();         // 0: issues the pair's MMAs
    const int4 it = items[blockIdx.y];
    const int c = blockIdx.x >> 1;                   // part pair: row-part pair nsp, inner part kpart
    const int nsp = c / KS, kpart = c % KS;
    const int part = (2 * nsp + (int)rank) * KS + kpart;
    const int first = it.x, npairs = it.y;
    const int opi = sets.single[blockIdx.z] ? it.z % kNumOffsets : it.z;
    const int ntile = (npairs + TILE - 1) / TILE;
    const int rofs = (int)rank * kTcRows;            // this CTA's rows of a tile
    const int ncols = sets.ncols > 0 ? sets.ncols : NPAD;
    static_assert(NP % (2 * kTcEpiLd) == 0, "epilogue chunks");

    if (tid == 0) {
        mbar_init(&S->barB, 1);
        mbar_init(&S->barBp, 1);
        // even CTA: its own warps arrive locally, the odd CTA's relay once
        for (int q = 0; q < kTcStages; ++q) {
            mbar_init(&S->full[q], kTcProdWarps + 1);
            mbar_init(&S->empty[q], 1);
            mbar_init(&S->pfull[q], kTcProdWarps);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&S->accf[q], 1);
            mbar_init(&S->acce[q], kTcEpiWarps + 1);
            mbar_init(&S->pacce[q], kTcEpiWarps);
        }
        S->failed = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc_pair(&S->tmem_slot, TCOLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();                              // both CTAs' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t taddr = S->tmem_slot;
    if (tid == 0) {
        tc_mark(sets.trace, rank, 0, 1);
        tc_mark(sets.trace, rank, 1, (int)taddr);
    }

    // resident operator part: hi and lo, one bulk copy each
    if (tid == 0) {
        const uint8_t* gB = (const uint8_t*)ops + ((long long)opi * (NS * KS) + part) * (2LL * B_SPLIT);
        mbar_arrive_expect_tx(&S->barB, 2 * B_SPLIT);
        bulk_g2s(sB, gB, B_SPLIT, &S->barB);
        bulk_g2s(sB + B_SPLIT, gB + B_SPLIT, B_SPLIT, &S->barB);
    }

    if (warp < kTcProdWarps) {
        // ---- producers (as in the single-CTA kernel, on this CTA's rows)
        const int l8 = lane & 7, rbase = warp * 4 + (lane >> 3);
        auto src_of = [&](int tile, int i) -> int {
            const int r = tile * TILE + rofs + i * 32 + rbase;
            return (tile < ntile && r < npairs) ? psrc[first + r] : -1;
        };
        float4 v[KB][4];
        int sn[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s0 = src_of(0, i);
            const float4* q4 = s0 >= 0 ? (const float4*)(Qu + (size_t)s0 * NPAD + kpart * KC) : nullptr;
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) v[kb][i] = q4 ? q4[kb * 8 + l8] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) sn[i] = src_of(1, i);
        int g = 0;
        for (int tile = 0; tile < ntile; ++tile) {
#pragma unroll
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = g % kTcStages, n = g / kTcStages;
                if (n > 0 && !mbar_wait_cta(&S->empty[s], (n - 1) & 1, failed, wl)) goto prod_done;
                uint8_t* aHi = sA + (size_t)s * 2 * A_SPLIT;
                uint8_t* aLo = aHi + A_SPLIT;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 x = v[kb][i];
                    float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
                    uint32_t off = sw128_off(i * 32 + rbase, l8 * 4);
                    *(float4*)(aHi + off) = h;
                    *(float4*)(aLo + off) = l;
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(rank == 0 ? &S->full[s] : &S->pfull[s]);
                if (tid == 0) tc_mark(sets.trace, rank, 5, g + 1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4* qn = sn[i] >= 0 ? (const float4*)(Qu + (size_t)sn[i] * NPAD + kpart * KC) : nullptr;
                    v[kb][i] = qn ? qn[kb * 8 + l8] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sn[i] = src_of(tile + 2, i);
        }
    prod_done:
        __syncwarp();
    } else if (warp < kTcProdWarps + kTcEpiWarps) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) ... + 31 of this CTA
        const int q = warp & 3;
        const int erow = q * 32 + lane;
        for (int tile = 0; tile < ntile; ++tile) {
            const int a = tile & 1, u = tile >> 1;
            const int r = tile * TILE + rofs + erow;
            const int t = r < npairs ? ptgt[first + r] : -1;
            bool ok = mbar_wait_cta(&S->accf[a], u & 1, failed, wl);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            float (*buf)[kTcEpiStride] = S->epi[q];
            const uint32_t tbase = taddr + ((uint32_t)(q * 32) << 16) + a * ACOLS;
            // one 16-column chunk: transpose through shared memory so that a
            // reduction instruction covers 8 rows x 64 B, skip padding columns
            auto drain = [&](const uint32_t* r, int c0) {
#pragma unroll
                for (int cc = 0; cc < kTcEpiLd; cc += 4)
                    *(float4*)&buf[lane][cc] = make_float4(__uint_as_float(r[cc]), __uint_as_float(r[cc + 1]),
                                                           __uint_as_float(r[cc + 2]), __uint_as_float(r[cc + 3]));
                __syncwarp();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int rr = j * 8 + (lane >> 2), cc = (lane & 3) * 4;
                    const float4 x = *(const float4*)&buf[rr][cc];
                    const int tr = __shfl_sync(0xffffffffu, t, rr);
                    const int col = nsp * NP + c0 + cc;
                    if (tr >= 0 && col < ncols) red_add_v4(Qd + (size_t)tr * NPAD + col, x.x, x.y, x.z, x.w);
                }
                __syncwarp();
            };
            // the next chunk's TMEM load runs while the current one drains
            uint32_t ra[kTcEpiLd], rb[kTcEpiLd];
            tmem_ld16_issue(tbase, ra);
            tmem_wait16(ra);
#pragma unroll 1
            for (int c0 = 0; c0 < NP; c0 += 2 * kTcEpiLd) {        // NP is a multiple of 32
                tmem_ld16_issue(tbase + c0 + kTcEpiLd, rb);
                drain(ra, c0);
                tmem_wait16(rb);
                if (c0 + 2 * kTcEpiLd < NP) tmem_ld16_issue(tbase + c0 + 2 * kTcEpiLd, ra);
                drain(rb, c0 + kTcEpiLd);
                if (c0 + 2 * kTcEpiLd < NP) tmem_wait16(ra);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(rank == 0 ? &S->acce[a] : &S->pacce[a]);
            if (warp == kTcProdWarps && lane == 0) tc_mark(sets.trace, rank, 4, tile + 1);
        }
        __syncwarp();
    } else if (rank == 0) {
        // ---- MMA issuer of the pair
        if (lane == 0) {
            uint64_t* last = nullptr;
            uint32_t last_par = 0;
            int g = 0;
            bool ok = mbar_wait_cta(&S->barB, 0, failed, wl) && mbar_wait_cta_cl(&S->barBp, 0, failed, wl);
            tc_mark(sets.trace, rank, 2, ok ? 1 : -1);
            for (int tile = 0; ok && tile < ntile; ++tile) {
                const int a = tile & 1, u = tile >> 1;
                if (u > 0 && !(ok = mbar_wait_cta_cl(&S->acce[a], (u - 1) & 1, failed, wl))) break;
                const uint32_t dacc = taddr + a * ACOLS;
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int s = g % kTcStages, n = g / kTcStages;
                    if (!(ok = mbar_wait_cta_cl(&S->full[s], n & 1, failed, wl))) break;
                    tc_fence_after();
                    const uint32_t aH = smem_u32(sA + (size_t)s * 2 * A_SPLIT), aL = aH + A_SPLIT;
                    const uint32_t bH = smem_u32(sB) + kb * NH * 128, bL = bH + B_SPLIT;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc0 = (kb > 0 || ks > 0) ? 1u : 0u;
                        mma_tf32_pair(dacc, sw128_desc(aH + ks * 32), sw128_desc(bH + ks * 32), IDESC, acc0);
                        mma_tf32_pair(dacc, sw128_desc(aH + ks * 32), sw128_desc(bL + ks * 32), IDESC, 1u);
                        mma_tf32_pair(dacc, sw128_desc(aL + ks * 32), sw128_desc(bH + ks * 32), IDESC, 1u);
                    }
                    mma_commit_pair(&S->empty[s], 0x3);
                    tc_mark(sets.trace, rank, 3, g + 1);
                    last = &S->empty[s];
                    last_par = n & 1;
                }
                if (!ok) break;
                mma_commit_pair(&S->accf[a], 0x3);
                last = &S->accf[a];
                last_par = u & 1;
            }
            // after a failure: every MMA issued here has completed before TMEM is freed
            if (!ok && last) mbar_wait(last, last_par);
        }
        __syncwarp();
    } else {
        // ---- odd CTA relays (one cluster-scope arrival per event instead
        // of one per warp): lane 0 its operator part and its full A stages,
        // lane 1 its drained accumulators, in the order the issuer needs them
        if (lane == 0) {
            bool ok = mbar_wait_cta(&S->barB, 0, failed, wl);
            if (ok) mbar_arrive_cluster(mapa_shared(smem_u32(&S->barBp), 0));
            tc_mark(sets.trace, rank, 2, ok ? 1 : -1);
            for (int g = 0; ok && g < ntile * KB; ++g) {
                const int s = g % kTcStages, n = g / kTcStages;
                if ((ok = mbar_wait_cta(&S->pfull[s], n & 1, failed, wl)))
                    mbar_arrive_cluster(mapa_shared(smem_u32(&S->full[s]), 0));
            }
        } else if (lane == 1) {
            bool ok = true;
            for (int tile = 0; ok && tile < ntile; ++tile) {
                const int a = tile & 1, u = tile >> 1;
                if ((ok = mbar_wait_cta(&S->pacce[a], u & 1, failed, wl)))
                    mbar_arrive_cluster(mapa_shared(smem_u32(&S->acce[a]), 0));
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();                              // no remote arrival or MMA of the pair is pending
    tc_fence_after();
    if (tid == 0) {
        tc_mark(sets.trace, rank, 7, S->failed);
        tc_mark(sets.trace, rank, 6, 1);
    }
    if (tid == 0 && S->failed) {
        atomicExch(err, 1);
        mbar_wait(&S->barB, 0);         // the operator copy has landed before shared memory is released
    }
    if (warp == 0) tmem_dealloc_pair(taddr, TCOLS);
}

template <int NPAD>
static constexpr size_t tc_pair_smem_bytes() {
    using C = TcCfg<NPAD>;
    return 1024 + 2 * (size_t)(NPAD / C::KS / 32) * (NPAD / C::NS) * 128 + C::STAGES * 2 * (size_t)kTcRows * 128 +
           sizeof(TcPairSmem<C::STAGES>);
}

template <int NPAD>
static constexpr size_t tc_smem_bytes() {
    using C = TcCfg<NPAD>;
    return 1024 + 2 * (size_t)(NPAD / C::KS / 32) * (NPAD / C::NS) * 128 + C::STAGES * 2 * (size_t)kTcRows * 128 +
           sizeof(TcSmem<C::STAGES>);
}
static_assert(tc_smem_bytes<160>() <= 232448 && tc_smem_bytes<320>() <= 232448 && tc_smem_bytes<512>() <= 232448,
              "shared memory per CTA");
static_assert(tc_pair_smem_bytes<160>() <= 232448 && tc_pair_smem_bytes<320>() <= 232448 &&
                  tc_pair_smem_bytes<512>() <= 232448,
              "shared memory per CTA");

// Kernel choice: CTA pairs (k_m2l_tc2) where the operator size allows,
// else one CTA per operator part (k_m2l_tc).
static std::atomic<int> g_tc_pair{1};
static bool tc_pair_for(int npad) { return g_tc_pair.load() != 0 && npad >= 128; }

// opt in to the large shared-memory carve-out once per process, kernel and
// device (not a stream operation, so it stays out of captured graphs)
template <typename F>
static void smem_optin(F* kernel, size_t bytes, bool* done) {
    int dev = 0;
    PB_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !done[dev]) {
        PB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        done[dev] = true;
    }
}

template <int NPAD>
static void launch_tc_items(const int4* items, int nitems, const int* tgt, const int* src, const TcSets& sets,
                            int nsets, int* err, cudaStream_t st, bool allow_pair) {
    if (nitems <= 0) return;
    dim3 grid(nitems, TcCfg<NPAD>::NS * TcCfg<NPAD>::KS, nsets);
    TcSets s2 = sets;
    s2.wait_limit = g_wait_limit.load();
    if constexpr (NPAD >= 128) {
        if (allow_pair && tc_pair_for(NPAD)) {
            static bool done[64] = {false};
            const size_t sm = tc_pair_smem_bytes<NPAD>();
            smem_optin(k_m2l_tc2<NPAD>, sm, done);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;                // the two row parts of a part pair
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            for (int i0 = 0; i0 < nitems; i0 += 65535) {  // items along grid y
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(TcCfg<NPAD>::NS * TcCfg<NPAD>::KS, std::min(65535, nitems - i0), nsets);
                cfg.blockDim = dim3(kTcThreads);
                cfg.dynamicSmemBytes = sm;
                cfg.stream = st;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                PB_CUDA(cudaLaunchKernelEx(&cfg, k_m2l_tc2<NPAD>, items + i0, tgt, src, s2, err));
                PB_CHECK_LAUNCH();
            }
            return;
        }
    }
    static bool done[64] = {false};
    const size_t sm = tc_smem_bytes<NPAD>();
    smem_optin(k_m2l_tc<NPAD>, sm, done);
    k_m2l_tc<NPAD><<<grid, kTcThreads, sm, st>>>(items, tgt, src, s2, err);
    PB_CHECK_LAUNCH();
}

// allow_pair: the launch may use the CTA-pair kernel (the M2L, whose work
// items hold up to 2,048 pairs; the M2M / L2L / solve items are smaller and
// keep one CTA per operator part)
static bool tc_dispatch(int npad, const int4* items, int nitems, const int* tgt, const int* src, const TcSets& sets,
                        int nsets, int* err, cudaStream_t st, bool allow_pair = false) {
    switch (npad) {
        case 32: launch_tc_items<32>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        case 64: launch_tc_items<64>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        case 128: launch_tc_items<128>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        case 160: launch_tc_items<160>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        case 320: launch_tc_items<320>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        case 512: launch_tc_items<512>(items, nitems, tgt, src, sets, nsets, err, st, allow_pair); return true;
        default: return false;
    }
}

static bool tc_ok(const Operators& O) {
    int ns, ks;
    return O.have_tc && tc_split(O.npad, ns, ks);
}

// M2M (up = true: parents at level l - 1 += M2M children at level l) or L2L
// (children at level l += L2L parents at level l - 1) on the tensor cores,
// for one operator set (O2 == nullptr) or for two in one launch; false when
// the tensor-core path does not apply
bool pc_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, int child_level, bool up, float* Q,
                   float* Q2, int* err, cudaStream_t st) {
    if (!tc_ok(O) || !O.m2m_tc.p || !O.l2l_tc.p) return false;
    if (O2 && (!tc_ok(*O2) || !O2->m2m_tc.p || !O2->l2l_tc.p || O2->npad != O.npad)) return false;
    const auto& P = T->pc_pairs;
    if (child_level < 3 || child_level >= T->nlev || (int)P.level_item_off.size() != T->nlev + 1) return false;
    const int i0 = P.level_item_off[child_level], i1 = P.level_item_off[child_level + 1];
    if (i1 <= i0) return true;
    const int* tgt = up ? P.parent.p : P.child.p;
    const int* src = up ? P.child.p : P.parent.p;
    TcSets sets{{up ? O.m2m_tc.p : O.l2l_tc.p, O2 ? (up ? O2->m2m_tc.p : O2->l2l_tc.p) : nullptr},
                {Q, Q2}, {Q, Q2}};
    return tc_dispatch(O.npad, P.items.p + i0, i1 - i0, tgt, src, sets, O2 ? 2 : 1, err, st);
}

bool pc_tc_launch(const fmm_tree* T, const Operators& O, int child_level, bool up, float* Q, int* err,
                  cudaStream_t st) {
    return pc_tc_launch2(T, O, nullptr, child_level, up, Q, nullptr, err, st);
}

// Check -> equivalent solve Y = W2 (W1 X) at the upward (sleaf) or downward
// (X-list) boxes on the tensor cores: two passes through `tmp`, which is
// zeroed first (every row of a pass receives exactly one product, so the
// result does not depend on the order of the reductions). Y rows of those
// boxes must be zero on entry. One operator set, or two (O2, X2, Y2, tmp2)
// in the same launches. False when the tensor-core path does not apply.
bool c2e_tc_ok(const Operators& O) { return tc_ok(O) && O.uc2ue_w1_tc.p; }

// The X-list boxes that keep P2L at a direct-list threshold (see the
// field comment in fmm_tree), with their check -> equivalent items; once per
// tree and threshold, on the host (the first apply runs uncaptured).
void build_xbox_far(fmm_tree* T, int thrX) {
    if (T->xfar_thr == thrX) return;
    cudaStream_t st = T->ctx->stream;
    const int nb = T->nbox, nx = T->n_xbox;
    std::vector<int> ids(std::max(nx, 1)), nch(nb), b0(nb), b1(nb);
    if (nx) PB_CUDA(cudaMemcpyAsync(ids.data(), T->xbox_ids.p, nx * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(nch.data(), T->nchild.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(b0.data(), T->same ? T->sb.p : T->tb.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaMemcpyAsync(b1.data(), T->same ? T->se.p : T->te.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    std::vector<int> far;
    far.reserve(nx);
    for (int i = 0; i < nx; ++i) {
        const int b = ids[i];
        if (!(nch[b] == 0 && b1[b] - b0[b] <= thrX)) far.push_back(b);
    }
    std::vector<int> lvl(T->nlev + 1, 0);
    for (int l = 0; l <= T->nlev; ++l)
        lvl[l] = (int)(std::lower_bound(far.begin(), far.end(), T->lvl_off[l]) - far.begin());
    T->xfar_ids.alloc(std::max<size_t>(far.size(), 1), st);
    if (!far.empty())
        PB_CUDA(cudaMemcpyAsync(T->xfar_ids.p, far.data(), far.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    T->n_xfar = (int)far.size();
    T->n_c2e_xfar = 0;
    level_items(lvl, T->nlev, T->c2e_items_xfar, T->n_c2e_xfar, st);
    T->xfar_thr = thrX;
}

bool c2e_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, bool up, const float* X, float* Y,
                    float* tmp, const float* X2, float* Y2, float* tmp2, int* err, cudaStream_t st, bool xfar) {
    if (!tc_ok(O) || !O.uc2ue_w1_tc.p) return false;
    if (O2 && (!tc_ok(*O2) || !O2->uc2ue_w1_tc.p || O2->npad != O.npad)) return false;
    const bool far = !up && xfar;
    const int nitems = up ? T->n_c2e_up : (far ? T->n_c2e_xfar : T->n_c2e_dn);
    if (nitems == 0) return true;
    const int4* items = up ? T->c2e_items_up.p : (far ? T->c2e_items_xfar.p : T->c2e_items_dn.p);
    const int* ids = up ? T->sleaf_ids.p : (far ? T->xfar_ids.p : T->xbox_ids.p);
    auto w1 = [&](const Operators& o) { return up ? o.uc2ue_w1_tc.p : o.dc2de_w1_tc.p; };
    auto w2 = [&](const Operators& o) { return up ? o.uc2ue_w2_tc.p : o.dc2de_w2_tc.p; };
    const size_t bytes = (size_t)T->nbox * O.npad * sizeof(float);
    PB_CUDA(cudaMemsetAsync(tmp, 0, bytes, st));
    if (O2) PB_CUDA(cudaMemsetAsync(tmp2, 0, bytes, st));
    const int ns = O2 ? 2 : 1;
    TcSets p1{{w1(O), O2 ? w1(*O2) : nullptr}, {X, X2}, {tmp, tmp2}};
    TcSets p2{{w2(O), O2 ? w2(*O2) : nullptr}, {tmp, tmp2}, {Y, Y2}};
    if (!tc_dispatch(O.npad, items, nitems, ids, ids, p1, ns, err, st)) return false;
    return tc_dispatch(O.npad, items, nitems, ids, ids, p2, ns, err, st);
}

bool c2e_tc_launch(const fmm_tree* T, const Operators& O, bool up, const float* X, float* Y, float* tmp, int* err,
                   cudaStream_t st, bool xfar) {
    return c2e_tc_launch2(T, O, nullptr, up, X, Y, tmp, nullptr, nullptr, nullptr, err, st, xfar);
}

// M2L on the tensor cores for one or two operator sets; false when the
// tensor-core path does not apply (caller uses the CUDA-core kernel)
bool m2l_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, const float* Qu, float* Qd,
                    const float* Qu2, float* Qd2, int* err, cudaStream_t st) {
    if (!tc_ok(O) || (O2 && (!tc_ok(*O2) || O2->npad != O.npad))) return false;
    if (T->m2l_pairs.nitems == 0) return true;
    const auto& P = T->m2l_pairs;
    const bool pair = T->ctx->m2l_tile == 0;       // PB_OPT_M2L_TILE: 256-pair tiles on CTA pairs
    const bool single1 = O.m2l_tc_single, single2 = O2 && O2->m2l_tc_single;
    if (!single1 && !single2) {
        // both sets per (level, offset): one launch, grid z selects the set
        TcSets sets{{O.m2l_tc.p, O2 ? O2->m2l_tc.p : nullptr}, {Qu, Qu2}, {Qd, Qd2}, {0, 0}, 0, nullptr, O.ne};
        return tc_dispatch(O.npad, P.items.p, P.nitems, P.tgt.p, P.src.p, sets, O2 ? 2 : 1, err, st, pair);
    }
    // a level-invariant set takes the per-offset items (every level of an
    // offset under one operator load); the other set its per-level items
    auto one = [&](const Operators& o, const float* X, float* Y) {
        TcSets sets{{o.m2l_tc.p, nullptr}, {X, nullptr}, {Y, nullptr}, {o.m2l_tc_single ? 1 : 0, 0}, 0, nullptr, o.ne};
        if (o.m2l_tc_single && P.nitems_off > 0)
            return tc_dispatch(o.npad, P.items_off.p, P.nitems_off, P.tgt.p, P.src.p, sets, 1, err, st, pair);
        return tc_dispatch(o.npad, P.items.p, P.nitems, P.tgt.p, P.src.p, sets, 1, err, st, pair);
    };
    if (!one(O, Qu, Qd)) return false;
    return O2 ? one(*O2, Qu2, Qd2) : true;
}

bool m2l_tc_launch(const fmm_tree* T, const Operators& O, const float* Qu, float* Qd, int* err, cudaStream_t st) {
    return m2l_tc_launch2(T, O, nullptr, Qu, Qd, nullptr, nullptr, err, st);
}

}  // namespace pbfmm

// ---------------------------------------------------------------------------
// Self-test hook (not part of the documented ABI): D = Q Op^T for one
// operator through the tensor-core M2L kernel, host buffers.
// ---------------------------------------------------------------------------
using namespace pbfmm;
extern "C" int pbfmm_test_tc_pair(int mode) { return g_tc_pair.exchange(mode ? 1 : 0); }

// launch properties of the CTA-pair kernel at npad 128 (no launch):
// out = {registers, max threads per block, static shared bytes, dynamic
// shared bytes requested, max co-resident clusters of two for that launch}
extern "C" int pbfmm_test_tc_pair_info(int* out) {
    try {
        static bool done[64] = {false};
        const size_t sm = tc_pair_smem_bytes<128>();
        smem_optin(k_m2l_tc2<128>, sm, done);
        cudaFuncAttributes fa;
        PB_CUDA(cudaFuncGetAttributes(&fa, k_m2l_tc2<128>));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = sm;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = -1;
        PB_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, k_m2l_tc2<128>, &cfg));
        out[0] = fa.numRegs;
        out[1] = fa.maxThreadsPerBlock;
        out[2] = (int)fa.sharedSizeBytes;
        out[3] = (int)sm;
        out[4] = nclusters;
        return PB_OK;
    } catch (const Error& e) {
        std::fprintf(stderr, "pbfmm_test_tc_pair_info: %s\n", e.what());
        return e.code;
    }
}

extern "C" int pbfmm_selftest_m2l_tc(int nrows, int npad, const float* Q, const float* Op, float* D) {
    try {
        int ns_, ks_;
        if (nrows < 1 || !tc_split(npad, ns_, ks_)) return PB_EINVAL;
        cudaStream_t st = nullptr;
        fmm_tree T;
        Operators O;
        O.npad = npad;
        O.nlev = 1;
        DBuf<float> m2l, q, d;
        DBuf<int> e;
        m2l.alloc((size_t)kNumOffsets * npad * npad, st);
        m2l.zero(st);
        PB_CUDA(cudaMemcpyAsync(m2l.p, Op, (size_t)npad * npad * 4, cudaMemcpyHostToDevice, st));   // offset slot 0
        O.m2l.p = m2l.p;
        pack_m2l_tc(O, st);
        O.m2l.p = nullptr;
        q.alloc((size_t)nrows * npad, st);
        d.alloc((size_t)nrows * npad, st);
        d.zero(st);
        e.alloc(1, st);
        e.zero(st);
        PB_CUDA(cudaMemcpyAsync(q.p, Q, (size_t)nrows * npad * 4, cudaMemcpyHostToDevice, st));
        std::vector<int> id(nrows);
        for (int i = 0; i < nrows; ++i) id[i] = i;
        T.m2l_pairs.tgt.alloc(nrows, st);
        T.m2l_pairs.src.alloc(nrows, st);
        PB_CUDA(cudaMemcpyAsync(T.m2l_pairs.tgt.p, id.data(), nrows * 4, cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T.m2l_pairs.src.p, id.data(), nrows * 4, cudaMemcpyHostToDevice, st));
        std::vector<int4> items;
        for (int a = 0; a < nrows; a += kTcItemPairs) items.push_back(make_int4(a, std::min(kTcItemPairs, nrows - a), 0, 0));
        // (operator index 0: level 0, offset slot 0)
        T.m2l_pairs.nitems = (int)items.size();
        T.m2l_pairs.items.alloc(items.size(), st);
        PB_CUDA(cudaMemcpyAsync(T.m2l_pairs.items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        // progress markers of the CTA-pair kernel in host-mapped memory
        int* trace_h = nullptr;
        int* trace_d = nullptr;
        PB_CUDA(cudaHostAlloc((void**)&trace_h, 16 * sizeof(int), cudaHostAllocMapped));
        std::unique_ptr<int, void (*)(int*)> trace_guard(trace_h, [](int* p) { cudaFreeHost(p); });
        for (int i = 0; i < 16; ++i) trace_h[i] = 0;
        PB_CUDA(cudaHostGetDevicePointer((void**)&trace_d, trace_h, 0));
        try {
            TcSets sets{{O.m2l_tc.p, nullptr}, {q.p, nullptr}, {d.p, nullptr}, {O.m2l_tc_single ? 1 : 0, 0}, 0,
                        trace_d};
            if (!tc_dispatch(O.npad, T.m2l_pairs.items.p, T.m2l_pairs.nitems, T.m2l_pairs.tgt.p, T.m2l_pairs.src.p,
                             sets, 1, e.p, st, true))
                return PB_EINVAL;
            int herr = 0;
            PB_CUDA(cudaMemcpyAsync(&herr, e.p, 4, cudaMemcpyDeviceToHost, st));
            PB_CUDA(cudaMemcpyAsync(D, d.p, (size_t)nrows * npad * 4, cudaMemcpyDeviceToHost, st));
            PB_CUDA(cudaStreamSynchronize(st));
            return herr ? PB_ETIMEOUT : PB_OK;
        } catch (const Error& ex) {
            std::fprintf(stderr, "pbfmm_selftest_m2l_tc: %s; pair-kernel markers:", ex.what());
            for (int i = 0; i < 16; ++i) std::fprintf(stderr, " %d", ((volatile int*)trace_h)[i]);
            std::fprintf(stderr, "\n");
            throw;
        }
    } catch (const Error& e) {
        return e.code;
    }
}
