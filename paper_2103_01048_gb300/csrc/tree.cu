// Octree build and interaction lists on the GPU (Sec. "Fast multipole
// method": enclosing cube, recursive subdivision until a leaf holds at most
// ncrit points, near field and interaction lists; adaptive U/V/W/X lists of
// the kernel-independent FMM the paper cites).
//
// Steps (each a kernel): bounding box -> 63-bit Morton keys from an FP64
// quantisation with correctly rounded operations -> stable radix sort of
// (key, index) -> level-synchronous box splitting -> box centres ->
// colleague / V / X lists top-down -> U / W lists of leaves by a bounded
// depth-first search -> per-tile M2L schedule.
#include "tree.cuh"
#include <cub/cub.cuh>
#include <algorithm>

namespace pbfmm {

void radix_sort_pairs(const uint64_t* keys_in, const int* vals_in, uint64_t* keys_out, int* vals_out, long long n,
                      int bits, cudaStream_t st);

// ---------------------------------------------------------------------------
// bounding box
// ---------------------------------------------------------------------------
__device__ __forceinline__ int float_to_ordered(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

__global__ void k_bbox(const float* __restrict__ xyz, long long n, int* __restrict__ mm) {
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            int v = float_to_ordered(xyz[3 * i + a]);
            lo[a] = min(lo[a], v);
            hi[a] = max(hi[a], v);
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(mm + a, lo[a]);
            atomicMax(mm + 3 + a, hi[a]);
        }
    }
}

__global__ void k_bbox_decode(const int* mm, float* out) {
    if (threadIdx.x < 6) out[threadIdx.x] = ordered_to_float(mm[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Morton keys: per axis floor((x - lo) * scale), clamped, bits interleaved
// x, y, z from the most significant bit.  __dsub_rn / __dmul_rn keep every
// step a correctly rounded FP64 operation (no contraction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

__global__ void k_keys(const float* __restrict__ xyz, long long n, double lx, double ly, double lz,
                       double scale, uint64_t* __restrict__ keys, int* __restrict__ idx) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lo[3] = {lx, ly, lz};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        double t = __dmul_rn(__dsub_rn((double)xyz[3 * i + a], lo[a]), scale);
        double f = floor(t);
        if (f < 0.0) f = 0.0;
        if (f > (double)((1 << kMaxLevel) - 1)) f = (double)((1 << kMaxLevel) - 1);
        q[a] = (uint32_t)f;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    idx[i] = (int)i;
}

__global__ void k_gather_pos(const float* __restrict__ xyz, const int* __restrict__ perm, long long n,
                             float4* __restrict__ out) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long i = perm[k];
    out[k] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
}

// ---------------------------------------------------------------------------
// level-synchronous splitting
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lower_digit(const uint64_t* keys, int b, int e, int d, int shift) {
    // first k in [b, e) with digit(key[k]) >= d (digits are monotone in the range)
    while (b < e) {
        int m = (b + e) >> 1;
        int dm = (int)((keys[m] >> shift) & 7ULL);
        if (dm < d) b = m + 1;
        else e = m;
    }
    return b;
}

__global__ void k_count_children(int lo, int hi, int lev, int ncrit, int same,
                                 const int* sb, const int* se, const int* tb, const int* te,
                                 const uint64_t* keys_s, const uint64_t* keys_t, int* nchild) {
    int b = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int cnt = (se[b] - sb[b]) + (same ? 0 : (te[b] - tb[b]));
    if (cnt <= ncrit || lev >= kMaxLevel) { nchild[b] = 0; return; }
    int shift = 3 * (kMaxLevel - 1 - lev);
    int nc = 0;
    for (int d = 0; d < 8; ++d) {
        int s0 = lower_digit(keys_s, sb[b], se[b], d, shift);
        int s1 = lower_digit(keys_s, sb[b], se[b], d + 1, shift);
        int t0 = 0, t1 = 0;
        if (!same) {
            t0 = lower_digit(keys_t, tb[b], te[b], d, shift);
            t1 = lower_digit(keys_t, tb[b], te[b], d + 1, shift);
        }
        if (s1 > s0 || t1 > t0) ++nc;
    }
    nchild[b] = nc;
}

__global__ void k_write_children(int lo, int hi, int lev, int base, int same, const int* scan,
                                 const int* nchild, int* first_child,
                                 int* sb, int* se, int* tb, int* te, int* level, int* parent,
                                 int4* anchor, const uint64_t* keys_s, const uint64_t* keys_t) {
    int b = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    if (nchild[b] == 0) { first_child[b] = -1; return; }
    int shift = 3 * (kMaxLevel - 1 - lev);
    int c = base + scan[b - lo];
    first_child[b] = c;
    int4 a = anchor[b];
    for (int d = 0; d < 8; ++d) {
        int s0 = lower_digit(keys_s, sb[b], se[b], d, shift);
        int s1 = lower_digit(keys_s, sb[b], se[b], d + 1, shift);
        int t0, t1;
        if (same) { t0 = s0; t1 = s1; }
        else {
            t0 = lower_digit(keys_t, tb[b], te[b], d, shift);
            t1 = lower_digit(keys_t, tb[b], te[b], d + 1, shift);
        }
        if (s1 == s0 && t1 == t0) continue;
        sb[c] = s0; se[c] = s1; tb[c] = t0; te[c] = t1;
        level[c] = lev + 1;
        parent[c] = b;
        anchor[c] = make_int4(2 * a.x + ((d >> 2) & 1), 2 * a.y + ((d >> 1) & 1), 2 * a.z + (d & 1), lev + 1);
        ++c;
    }
}

__global__ void k_centers(int nbox, const int4* anchor, double lx, double ly, double lz, double R,
                          double4* center) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int4 a = anchor[b];
    double h = ldexp(R, -a.w);          // half-width R / 2^level (exact)
    double side = 2.0 * h;
    center[b] = make_double4(lx + (a.x + 0.5) * side, ly + (a.y + 0.5) * side, lz + (a.z + 0.5) * side, h);
}

// ---------------------------------------------------------------------------
// lists
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool adjacent(int4 A, int4 B) {
    int L = max(A.w, B.w);
    int sa = L - A.w, sb = L - B.w;
    int a0x = A.x << sa, a0y = A.y << sa, a0z = A.z << sa;
    int a1x = (A.x + 1) << sa, a1y = (A.y + 1) << sa, a1z = (A.z + 1) << sa;
    int b0x = B.x << sb, b0y = B.y << sb, b0z = B.z << sb;
    int b1x = (B.x + 1) << sb, b1y = (B.y + 1) << sb, b1z = (B.z + 1) << sb;
    return a0x <= b1x && b0x <= a1x && a0y <= b1y && b0y <= a1y && a0z <= b1z && b0z <= a1z;
}

__device__ __forceinline__ void sort_small(int* a, int n) {
    for (int i = 1; i < n; ++i) {
        int v = a[i], j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

__global__ void k_lists_root(int* coll, int* coll_n, int* cn_n, int* V_n, int* X_n) {
    coll[0] = 0; coll_n[0] = 1; cn_n[0] = 0; V_n[0] = 0; X_n[0] = 0;
}

// Coll(B), V(B), X(B) and the coarser adjacent leaves CN(B), from the parent's.
__global__ void k_lists_level(int lo, int hi, const int* parent, const int* first_child, const int* nchild,
                              const int4* anchor, int* coll, int* coll_n, int* cn, int* cn_n,
                              int* V, int* V_n, int* X, int* X_n) {
    int b = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int P = parent[b];
    int4 ab = anchor[b];
    int nco = 0, ncn = 0, nv = 0, nx = 0;
    int* mycoll = coll + (long long)b * kCollCap;
    int* mycn = cn + (long long)b * kCoarseCap;
    int* myV = V + (long long)b * kVCap;
    int* myX = X + (long long)b * kXCap;
    const int* pc = coll + (long long)P * kCollCap;
    for (int i = 0; i < coll_n[P]; ++i) {
        int C = pc[i];
        if (nchild[C] == 0) {
            if (adjacent(anchor[C], ab)) mycn[ncn++] = C;
            else myX[nx++] = C;
        } else {
            int f = first_child[C];
            for (int D = f; D < f + nchild[C]; ++D) {
                if (adjacent(anchor[D], ab)) mycoll[nco++] = D;
                else myV[nv++] = D;
            }
        }
    }
    const int* pcn = cn + (long long)P * kCoarseCap;
    for (int i = 0; i < cn_n[P]; ++i) {
        int A = pcn[i];
        if (adjacent(anchor[A], ab)) mycn[ncn++] = A;
        else myX[nx++] = A;
    }
    sort_small(mycn, ncn);
    sort_small(myX, nx);
    coll_n[b] = nco; cn_n[b] = ncn; V_n[b] = nv; X_n[b] = nx;
}

// U and W lists of leaf boxes.  pass 0 counts, pass 1 writes (sorted).
__global__ void k_leaf_lists(int nbox, int pass, const int* nchild, const int* first_child,
                             const int4* anchor, const int* coll, const int* coll_n,
                             const int* cn, const int* cn_n,
                             int* U_cnt, int* W_cnt, const int* U_off, const int* W_off,
                             int* U_ids, int* W_ids, int* overflow) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    if (nchild[b] != 0) {
        if (pass == 0) { U_cnt[b] = 0; W_cnt[b] = 0; }
        return;
    }
    int4 ab = anchor[b];
    int nu = 0, nw = 0;
    int* Uo = pass ? U_ids + U_off[b] : nullptr;
    int* Wo = pass ? W_ids + W_off[b] : nullptr;
    const int* mcn = cn + (long long)b * kCoarseCap;
    for (int i = 0; i < cn_n[b]; ++i) { if (pass) Uo[nu] = mcn[i]; ++nu; }
    const int* mc = coll + (long long)b * kCollCap;
    int stack[8 * (kMaxLevel + 1)];
    for (int i = 0; i < coll_n[b]; ++i) {
        int C = mc[i];
        if (nchild[C] == 0) { if (pass) Uo[nu] = C; ++nu; continue; }
        int sp = 0;
        for (int D = first_child[C]; D < first_child[C] + nchild[C]; ++D) stack[sp++] = D;
        while (sp > 0) {
            int D = stack[--sp];
            if (adjacent(anchor[D], ab)) {
                if (nchild[D] == 0) { if (pass) Uo[nu] = D; ++nu; }
                else {
                    if (sp + nchild[D] > 8 * (kMaxLevel + 1)) { atomicExch(overflow, 1); continue; }
                    for (int E = first_child[D]; E < first_child[D] + nchild[D]; ++E) stack[sp++] = E;
                }
            } else {
                if (pass) Wo[nw] = D;
                ++nw;
            }
        }
    }
    if (pass == 0) { U_cnt[b] = nu; W_cnt[b] = nw; }
    else { sort_small(Uo, nu); sort_small(Wo, nw); }
}

__global__ void k_flag(int n, const int* a, int* flag, int mode, const int* b2, const int* b3) {
    // mode 0: leaf with targets; 1: leaf with sources; 2: X list non-empty
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f;
    if (mode == 0) f = (a[i] == 0) && (b3[i] > b2[i]);
    else if (mode == 1) f = (a[i] == 0) && (b3[i] > b2[i]);
    else f = a[i] > 0;
    flag[i] = f;
}

// algorithmic work of one apply: p2p pairs, m2p targets, p2l sources,
// l2p targets, p2m sources, boxes at level >= 2
__global__ void k_work(int nbox, const int* nchild, const int* level, const int* sb, const int* se,
                       const int* tb, const int* te, const int* U_off, const int* U_ids, const int* W_off,
                       const int* X, const int* X_n, unsigned long long* w) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    long long ntb = te[b] - tb[b], nsb = se[b] - sb[b];
    if (nchild[b] == 0) {
        if (ntb > 0) {
            long long s = 0;
            for (int i = U_off[b]; i < U_off[b + 1]; ++i) s += se[U_ids[i]] - sb[U_ids[i]];
            atomicAdd(w + 0, (unsigned long long)(ntb * s));
            atomicAdd(w + 1, (unsigned long long)(ntb * (W_off[b + 1] - W_off[b])));
            if (level[b] >= 2) atomicAdd(w + 3, (unsigned long long)ntb);
        }
        atomicAdd(w + 4, (unsigned long long)nsb);
    }
    long long xs = 0;
    for (int i = 0; i < X_n[b]; ++i) {
        int a = X[(long long)b * kXCap + i];
        xs += se[a] - sb[a];
    }
    atomicAdd(w + 2, (unsigned long long)xs);
    if (level[b] >= 2) atomicAdd(w + 5, 1ULL);
}

// ---------------------------------------------------------------------------
// M2L tile schedule
// ---------------------------------------------------------------------------
__device__ __forceinline__ int offset_index(int4 t, int4 s) {
    return (s.x - t.x + 3) * 49 + (s.y - t.y + 3) * 7 + (s.z - t.z + 3);
}

// pass 0: number of distinct offsets used by the tile; pass 1: write entries
__global__ void k_m2l_schedule(int ntile, const int* tile_box, const int4* anchor, const int* V,
                               const int* V_n, const int* entry_off, int* entry_cnt,
                               int* entry_offset_idx, int* entry_src, int pass) {
    __shared__ int slot[kNumOffsets];
    int t = blockIdx.x;
    if (t >= ntile) return;
    for (int i = threadIdx.x; i < kNumOffsets; i += blockDim.x) slot[i] = 0;
    __syncthreads();
    const int* tb = tile_box + (long long)t * kM2LTile;
    for (int c = threadIdx.x; c < kM2LTile; c += blockDim.x) {
        int b = tb[c];
        if (b < 0) continue;
        int4 ab = anchor[b];
        for (int i = 0; i < V_n[b]; ++i) {
            int s = V[(long long)b * kVCap + i];
            slot[offset_index(ab, anchor[s])] = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int k = 0;
        for (int i = 0; i < kNumOffsets; ++i) {
            if (slot[i]) {
                if (pass) entry_offset_idx[entry_off[t] + k] = i;
                slot[i] = k + 1;     // 1-based position
                ++k;
            } else slot[i] = 0;
        }
        if (!pass) entry_cnt[t] = k;
    }
    __syncthreads();
    if (!pass) return;
    int nent = entry_off[t + 1] - entry_off[t];
    int* src = entry_src + (long long)entry_off[t] * kM2LTile;
    for (int i = threadIdx.x; i < nent * kM2LTile; i += blockDim.x) src[i] = -1;
    __syncthreads();
    for (int c = threadIdx.x; c < kM2LTile; c += blockDim.x) {
        int b = tb[c];
        if (b < 0) continue;
        int4 ab = anchor[b];
        for (int i = 0; i < V_n[b]; ++i) {
            int s = V[(long long)b * kVCap + i];
            int e = slot[offset_index(ab, anchor[s])] - 1;
            src[(long long)e * kM2LTile + c] = s;
        }
    }
}

__global__ void k_compact_scatter(int n, const int* flag, const int* pos, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = i;
}

static void exclusive_scan(const int* in, int* out, int n, cudaStream_t st);
template <typename T> static T read1(const T* d, cudaStream_t st);

// compaction helper: indices i with flag[i] != 0, in order
static int compact(const int* flag, int n, DBuf<int>& out, cudaStream_t st) {
    DBuf<int> pos;
    pos.alloc(n + 1, st);
    out.alloc(std::max(n, 1), st);
    exclusive_scan(flag, pos.p, n, st);
    k_compact_scatter<<<div_up(n, 256), 256, 0, st>>>(n, flag, pos.p, out.p);
    PB_CHECK_LAUNCH();
    return read1(pos.p + n - 1, st) + read1(flag + n - 1, st);
}

static void exclusive_scan(const int* in, int* out, int n, cudaStream_t st) {
    size_t tmp = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, st);
    DBuf<char> t;
    t.alloc(std::max<size_t>(tmp, 1), st);
    cub::DeviceScan::ExclusiveSum(t.p, tmp, in, out, n, st);
    PB_CHECK_LAUNCH();
}

template <typename T>
static T read1(const T* d, cudaStream_t st) {
    T h;
    PB_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    return h;
}

void build_m2l_pairs(fmm_tree* T);
void build_pc_pairs(fmm_tree* T);
void build_c2e_items(fmm_tree* T);

void build_tree(fmm_tree* T, const float* src, const float* tgt) {
    cudaStream_t st = T->ctx->stream;
    const long long ns = T->ns, nt = T->same ? T->ns : T->nt;
    // 1. bounding box (exact FP32 min/max)
    DBuf<int> mm;
    mm.alloc(6, st);
    int init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    PB_CUDA(cudaMemcpyAsync(mm.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
    int nsm = T->ctx->sm_count;
    k_bbox<<<std::min(div_up(ns, 256), 4 * nsm), 256, 0, st>>>(src, ns, mm.p);
    if (!T->same) k_bbox<<<std::min(div_up(nt, 256), 4 * nsm), 256, 0, st>>>(tgt, nt, mm.p);
    DBuf<float> mmf;
    mmf.alloc(6, st);
    k_bbox_decode<<<1, 32, 0, st>>>(mm.p, mmf.p);
    PB_CHECK_LAUNCH();
    float bb[6];
    PB_CUDA(cudaMemcpyAsync(bb, mmf.p, sizeof(bb), cudaMemcpyDeviceToHost, st));
    PB_CUDA(cudaStreamSynchronize(st));
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double lo = bb[a], hi = bb[3 + a];
        T->c[a] = (lo + hi) * 0.5;
        ext = std::max(ext, hi - lo);
    }
    // half-width: the smallest power of two >= half the extent (slightly
    // enlarged), so that trees of similar size share box sizes and hence
    // translation operators
    T->R = (0.5 * ext) * (1.0 + 1.0 / 1048576.0);
    if (T->R == 0.0) {
        T->R = 1.0;
    } else {
        int e = 0;
        const double m = std::frexp(T->R, &e);     // R = m 2^e, 0.5 <= m < 1 (exact)
        if (m != 0.5) T->R = std::ldexp(1.0, e);
    }
    const double lo3[3] = {T->c[0] - T->R, T->c[1] - T->R, T->c[2] - T->R};
    const double scale = (double)(1 << kMaxLevel) / (2.0 * T->R);

    // 2-3. keys and stable sort
    auto sort_set = [&](const float* xyz, long long n, DBuf<uint64_t>& keys, DBuf<int>& perm, DBuf<float4>& pos) {
        DBuf<uint64_t> k0;
        DBuf<int> i0;
        k0.alloc(n, st); i0.alloc(n, st);
        keys.alloc(n, st); perm.alloc(n, st);
        k_keys<<<div_up(n, 256), 256, 0, st>>>(xyz, n, lo3[0], lo3[1], lo3[2], scale, k0.p, i0.p);
        PB_CHECK_LAUNCH();
        radix_sort_pairs(k0.p, i0.p, keys.p, perm.p, n, 63, st);      // stable: ties keep the input order
        pos.alloc(n, st);
        k_gather_pos<<<div_up(n, 256), 256, 0, st>>>(xyz, perm.p, n, pos.p);
        PB_CHECK_LAUNCH();
    };
    sort_set(src, ns, T->keys_s, T->perm_s, T->pos_s);
    if (!T->same) sort_set(tgt, nt, T->keys_t, T->perm_t, T->pos_t);
    const uint64_t* keys_t = T->same ? T->keys_s.p : T->keys_t.p;

    // 4. boxes, level by level
    size_t cap = 1024;
    auto growall = [&](size_t n) {
        if (n <= T->level.n) return;
        size_t c = std::max(n, 2 * T->level.n);
        T->level.grow(c, st); T->parent.grow(c, st); T->first_child.grow(c, st);
        T->nchild.grow(c, st); T->sb.grow(c, st); T->se.grow(c, st); T->tb.grow(c, st);
        T->te.grow(c, st); T->anchor.grow(c, st);
    };
    growall(cap);
    {
        int z = 0, m1 = -1, nsi = (int)ns, nti = (int)nt;
        int4 a0 = make_int4(0, 0, 0, 0);
        PB_CUDA(cudaMemcpyAsync(T->level.p, &z, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->parent.p, &m1, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->sb.p, &z, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->se.p, &nsi, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->tb.p, &z, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->te.p, &nti, sizeof(int), cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(T->anchor.p, &a0, sizeof(int4), cudaMemcpyHostToDevice, st));
    }
    T->lvl_off.assign(1, 0);
    T->lvl_off.push_back(1);
    int lo = 0, hi = 1, lev = 0;
    DBuf<int> scan;
    while (hi > lo) {
        int nb = hi - lo;
        k_count_children<<<div_up(nb, 128), 128, 0, st>>>(lo, hi, lev, T->ncrit, T->same, T->sb.p, T->se.p,
                                                           T->tb.p, T->te.p, T->keys_s.p, keys_t, T->nchild.p);
        PB_CHECK_LAUNCH();
        scan.alloc(nb + 1, st);
        exclusive_scan(T->nchild.p + lo, scan.p, nb, st);
        int last_scan = read1(scan.p + nb - 1, st);
        int last_n = read1(T->nchild.p + hi - 1, st);
        int total = last_scan + last_n;
        growall((size_t)hi + total);
        k_write_children<<<div_up(nb, 128), 128, 0, st>>>(lo, hi, lev, hi, T->same, scan.p, T->nchild.p,
                                                           T->first_child.p, T->sb.p, T->se.p, T->tb.p, T->te.p,
                                                           T->level.p, T->parent.p, T->anchor.p, T->keys_s.p,
                                                           keys_t);
        PB_CHECK_LAUNCH();
        lo = hi;
        hi = hi + total;
        ++lev;
        if (total > 0) T->lvl_off.push_back(hi);
    }
    T->nbox = lo;
    T->nlev = (int)T->lvl_off.size() - 1;
    // leaves of the last level have nchild set by the final count pass; first_child too
    {
        int nb = T->nbox;
        T->center.alloc(nb, st);
        k_centers<<<div_up(nb, 128), 128, 0, st>>>(nb, T->anchor.p, lo3[0], lo3[1], lo3[2], T->R, T->center.p);
        PB_CHECK_LAUNCH();
    }

    // 5. colleague / V / X lists, top-down
    const int nb = T->nbox;
    T->coll.alloc((size_t)nb * kCollCap, st); T->coll_n.alloc(nb, st);
    T->cn.alloc((size_t)nb * kCoarseCap, st); T->cn_n.alloc(nb, st);
    T->V.alloc((size_t)nb * kVCap, st); T->V_n.alloc(nb, st);
    T->X.alloc((size_t)nb * kXCap, st); T->X_n.alloc(nb, st);
    k_lists_root<<<1, 1, 0, st>>>(T->coll.p, T->coll_n.p, T->cn_n.p, T->V_n.p, T->X_n.p);
    for (int l = 1; l < T->nlev; ++l) {
        int a = T->lvl_off[l], b = T->lvl_off[l + 1];
        k_lists_level<<<div_up(b - a, 128), 128, 0, st>>>(a, b, T->parent.p, T->first_child.p, T->nchild.p,
                                                          T->anchor.p, T->coll.p, T->coll_n.p, T->cn.p, T->cn_n.p,
                                                          T->V.p, T->V_n.p, T->X.p, T->X_n.p);
        PB_CHECK_LAUNCH();
    }
    // 6. U / W lists of leaves
    DBuf<int> ucnt, wcnt, ovf;
    ucnt.alloc(nb + 1, st); wcnt.alloc(nb + 1, st); ovf.alloc(1, st);
    ovf.zero(st);
    T->U_off.alloc(nb + 1, st); T->W_off.alloc(nb + 1, st);
    k_leaf_lists<<<div_up(nb, 128), 128, 0, st>>>(nb, 0, T->nchild.p, T->first_child.p, T->anchor.p, T->coll.p,
                                                  T->coll_n.p, T->cn.p, T->cn_n.p, ucnt.p, wcnt.p, nullptr,
                                                  nullptr, nullptr, nullptr, ovf.p);
    PB_CHECK_LAUNCH();
    PB_CUDA(cudaMemsetAsync(ucnt.p + nb, 0, sizeof(int), st));
    PB_CUDA(cudaMemsetAsync(wcnt.p + nb, 0, sizeof(int), st));
    exclusive_scan(ucnt.p, T->U_off.p, nb + 1, st);
    exclusive_scan(wcnt.p, T->W_off.p, nb + 1, st);
    T->n_u = read1(T->U_off.p + nb, st);
    T->n_w = read1(T->W_off.p + nb, st);
    T->U_ids.alloc(std::max<long long>(T->n_u, 1), st);
    T->W_ids.alloc(std::max<long long>(T->n_w, 1), st);
    k_leaf_lists<<<div_up(nb, 128), 128, 0, st>>>(nb, 1, T->nchild.p, T->first_child.p, T->anchor.p, T->coll.p,
                                                  T->coll_n.p, T->cn.p, T->cn_n.p, nullptr, nullptr, T->U_off.p,
                                                  T->W_off.p, T->U_ids.p, T->W_ids.p, ovf.p);
    PB_CHECK_LAUNCH();
    PB_REQUIRE(read1(ovf.p, st) == 0, PB_EINVAL, "octree too deep for the list search stack");

    // list totals
    {
        DBuf<int> tot;
        tot.alloc(1, st);
        size_t tmp = 0;
        cub::DeviceReduce::Sum(nullptr, tmp, T->V_n.p, tot.p, nb, st);
        DBuf<char> t;
        t.alloc(tmp, st);
        cub::DeviceReduce::Sum(t.p, tmp, T->V_n.p, tot.p, nb, st);
        T->n_v = read1(tot.p, st);
        cub::DeviceReduce::Sum(t.p, tmp, T->X_n.p, tot.p, nb, st);
        T->n_x = read1(tot.p, st);
    }

    // work counters
    {
        DBuf<unsigned long long> w;
        w.alloc(6, st);
        w.zero(st);
        const int* tbeg0 = T->same ? T->sb.p : T->tb.p;
        const int* tend0 = T->same ? T->se.p : T->te.p;
        k_work<<<div_up(nb, 128), 128, 0, st>>>(nb, T->nchild.p, T->level.p, T->sb.p, T->se.p, tbeg0, tend0,
                                                T->U_off.p, T->U_ids.p, T->W_off.p, T->X.p, T->X_n.p, w.p);
        PB_CHECK_LAUNCH();
        unsigned long long hw[6];
        PB_CUDA(cudaMemcpyAsync(hw, w.p, sizeof(hw), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < 6; ++i) T->work[i] = (long long)hw[i];
    }

    // 7. index sets used by the FMM passes
    DBuf<int> flag;
    flag.alloc(nb, st);
    const int* tbeg = T->same ? T->sb.p : T->tb.p;
    const int* tend = T->same ? T->se.p : T->te.p;
    k_flag<<<div_up(nb, 256), 256, 0, st>>>(nb, T->nchild.p, flag.p, 0, tbeg, tend);
    T->n_tleaf = compact(flag.p, nb, T->leaf_ids, st);
    k_flag<<<div_up(nb, 256), 256, 0, st>>>(nb, T->nchild.p, flag.p, 1, T->sb.p, T->se.p);
    int nsl = compact(flag.p, nb, T->sleaf_ids, st);
    // leaves with sources are in box order = level order: find level boundaries
    {
        std::vector<int> ids(std::max(nsl, 1));
        if (nsl) PB_CUDA(cudaMemcpyAsync(ids.data(), T->sleaf_ids.p, nsl * sizeof(int), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        T->sleaf_lvl_off.assign(T->nlev + 1, 0);
        for (int l = 0; l <= T->nlev; ++l)
            T->sleaf_lvl_off[l] = (int)(std::lower_bound(ids.begin(), ids.begin() + nsl, T->lvl_off[l]) - ids.begin());
    }
    k_flag<<<div_up(nb, 256), 256, 0, st>>>(nb, T->X_n.p, flag.p, 2, nullptr, nullptr);
    T->n_xbox = compact(flag.p, nb, T->xbox_ids, st);
    {
        std::vector<int> ids(std::max(T->n_xbox, 1));
        if (T->n_xbox)
            PB_CUDA(cudaMemcpyAsync(ids.data(), T->xbox_ids.p, T->n_xbox * sizeof(int), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        T->xbox_lvl_off.assign(T->nlev + 1, 0);
        for (int l = 0; l <= T->nlev; ++l)
            T->xbox_lvl_off[l] =
                (int)(std::lower_bound(ids.begin(), ids.begin() + T->n_xbox, T->lvl_off[l]) - ids.begin());
    }
    {
        // number of leaves
        std::vector<int> nch(nb);
        PB_CUDA(cudaMemcpyAsync(nch.data(), T->nchild.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        T->nleaf = (int)std::count(nch.begin(), nch.end(), 0);
    }

    // 8. M2L tile schedule: boxes with a non-empty V list, per level, tiles of kM2LTile
    {
        std::vector<int> vn(nb);
        PB_CUDA(cudaMemcpyAsync(vn.data(), T->V_n.p, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        std::vector<int> tiles, tlev;
        for (int l = 0; l < T->nlev; ++l) {
            std::vector<int> cur;
            for (int b = T->lvl_off[l]; b < T->lvl_off[l + 1]; ++b)
                if (vn[b] > 0) cur.push_back(b);
            for (size_t i = 0; i < cur.size(); i += kM2LTile) {
                for (int c = 0; c < kM2LTile; ++c)
                    tiles.push_back(i + c < cur.size() ? cur[i + c] : -1);
                tlev.push_back(l);
            }
        }
        M2LSchedule& S = T->m2l;
        S.ntile = (int)tlev.size();
        S.tile_level_h = tlev;
        S.npairs = T->n_v;
        if (S.ntile > 0) {
            S.tile_box.alloc(tiles.size(), st);
            S.tile_level.alloc(S.ntile, st);
            PB_CUDA(cudaMemcpyAsync(S.tile_box.p, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            PB_CUDA(cudaMemcpyAsync(S.tile_level.p, tlev.data(), tlev.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            DBuf<int> cnt;
            cnt.alloc(S.ntile + 1, st);
            cnt.zero(st);
            S.entry_off.alloc(S.ntile + 1, st);
            k_m2l_schedule<<<S.ntile, 128, 0, st>>>(S.ntile, S.tile_box.p, T->anchor.p, T->V.p, T->V_n.p, nullptr,
                                                    cnt.p, nullptr, nullptr, 0);
            PB_CHECK_LAUNCH();
            exclusive_scan(cnt.p, S.entry_off.p, S.ntile + 1, st);
            S.nentry = read1(S.entry_off.p + S.ntile, st);
            S.entry_offset_idx.alloc(std::max<long long>(S.nentry, 1), st);
            S.entry_src.alloc(std::max<long long>(S.nentry, 1) * kM2LTile, st);
            k_m2l_schedule<<<S.ntile, 128, 0, st>>>(S.ntile, S.tile_box.p, T->anchor.p, T->V.p, T->V_n.p,
                                                    S.entry_off.p, nullptr, S.entry_offset_idx.p, S.entry_src.p, 1);
            PB_CHECK_LAUNCH();
        }
    }
    // 9. V-list pairs grouped by (level, offset) for the tensor-core M2L
    build_m2l_pairs(T);
    build_pc_pairs(T);
    build_c2e_items(T);
    PB_CUDA(cudaStreamSynchronize(st));
}

}  // namespace pbfmm
