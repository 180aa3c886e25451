// Stable least-significant-digit radix sort of (key, value) pairs: the
// Morton-key sort of the octree build (keys of 63 bits, values the input
// indices: the sort by (key, index) of the tree's definition) and the
// grouping of the M2L pairs by (level, offset).
//
// One pass per 8-bit digit, each in three steps over tiles of 2048 pairs:
//   1. per tile, the digit histogram (shared-memory counters);
//   2. an exclusive scan of all histograms in digit-major order, so that
//      tile b's pairs of digit d start at offset[d][b] (tiles in order);
//   3. per tile, a stable partition by the digit in shared memory (eight
//      one-bit splits, each a block-wide scan), then every pair goes to
//      offset[d][b] + its rank among the tile's pairs of digit d.
// Each pass keeps the order of equal digits, so the result is stable.
#include "common.cuh"
#include <algorithm>

namespace pbfmm {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;     // 2048 pairs per tile
constexpr int kRsBins = 256;

template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K* __restrict__ keys, long long n, int shift,
                                                        int ntiles, int* __restrict__ counts) {
    __shared__ int h[kRsBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const long long g = base + i;
        if (g < n) atomicAdd(&h[(int)((keys[g] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    counts[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m ints in chunks of 2048 (one block each), chunk totals
__global__ void __launch_bounds__(kRsThreads) k_scan_chunks(const int* __restrict__ in, long long m,
                                                            int* __restrict__ out, int* __restrict__ totals) {
    __shared__ int warp_tot[kRsThreads / 32];
    const long long base = (long long)blockIdx.x * kRsTile + (long long)threadIdx.x * kRsItems;
    int v[kRsItems], s = 0;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        v[k] = base + k < m ? in[base + k] : 0;
        s += v[k];
    }
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += warp_tot[w];
    int run = wpre + incl - s;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        if (base + k < m) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kRsThreads - 1) totals[blockIdx.x] = wpre + incl;
}

// exclusive scan of the chunk totals in place (one block, sequential over
// blocks of 256)
__global__ void k_scan_totals(int* __restrict__ totals, int nchunk) {
    __shared__ int buf[kRsThreads];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nchunk; b0 += kRsThreads) {
        const int i = b0 + threadIdx.x;
        const int v = i < nchunk ? totals[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kRsThreads; o <<= 1) {
            const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nchunk) totals[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kRsThreads - 1) carry += buf[kRsThreads - 1];
        __syncthreads();
    }
}

__global__ void k_scan_add(int* __restrict__ out, long long m, const int* __restrict__ totals) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < m) out[i] += totals[i / kRsTile];
}

template <typename K, typename V>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K* __restrict__ kin, const V* __restrict__ vin,
                                                           long long n, int shift, int ntiles,
                                                           const int* __restrict__ offsets, K* __restrict__ kout,
                                                           V* __restrict__ vout) {
    __shared__ K sk[kRsTile];
    __shared__ V sv[kRsTile];
    __shared__ int start[kRsBins];
    __shared__ int warp_tot[kRsThreads / 32];
    const long long base = (long long)blockIdx.x * kRsTile;
    const int valid = (int)min((long long)kRsTile, n - base);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // blocked arrangement: thread t holds tile items t * kRsItems ... + 7
    K k[kRsItems];
    V v[kRsItems];
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int li = t * kRsItems + i;
        if (li < valid) {
            k[i] = kin[base + li];
            v[i] = vin[base + li];
        } else {
            k[i] = ~(K)0;            // past the end: the largest digit, kept behind the valid pairs
            v[i] = 0;
        }
    }
    // stable partition of the tile by the digit: one-bit splits, LSB first
    for (int bit = 0; bit < 8; ++bit) {
        int zeros = 0;
#pragma unroll
        for (int i = 0; i < kRsItems; ++i) zeros += ((k[i] >> (shift + bit)) & 1) ? 0 : 1;
        int incl = zeros;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();                       // the previous split's shared reads are done
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int wpre = 0, total = 0;
        for (int w = 0; w < kRsThreads / 32; ++w) {
            if (w < warp) wpre += warp_tot[w];
            total += warp_tot[w];
        }
        int zpos = wpre + incl - zeros;                          // zeros before this thread's items
        int opos = total + (t * kRsItems - (wpre + incl - zeros));  // ones before: items before minus zeros
#pragma unroll
        for (int i = 0; i < kRsItems; ++i) {
            const bool one = (k[i] >> (shift + bit)) & 1;
            const int dst = one ? opos++ : zpos++;
            sk[dst] = k[i];
            sv[dst] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kRsItems; ++i) {
            k[i] = sk[t * kRsItems + i];
            v[i] = sv[t * kRsItems + i];
        }
    }
    // first position of every digit in the sorted tile (valid pairs only)
    if (t < kRsBins) start[t] = kRsTile;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int pos = t * kRsItems + i;
        if (pos < valid) {
            const int d = (int)((k[i] >> shift) & 0xFF);
            const int prev = pos > 0 ? (int)((sk[pos - 1] >> shift) & 0xFF) : -1;
            if (d != prev) start[d] = pos;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int pos = t * kRsItems + i;
        if (pos < valid) {
            const int d = (int)((k[i] >> shift) & 0xFF);
            const long long o = (long long)offsets[(long long)d * ntiles + blockIdx.x] + (pos - start[d]);
            kout[o] = k[i];
            vout[o] = v[i];
        }
    }
}

// Sort n pairs by the low `bits` bits of the keys (stable); keys_in /
// vals_in are left unchanged, the result is in keys_out / vals_out.
template <typename K, typename V>
static void radix_sort_pairs_t(const K* keys_in, const V* vals_in, K* keys_out, V* vals_out, long long n, int bits,
                               cudaStream_t st) {
    if (n <= 0) return;
    const int ntiles = div_up(n, kRsTile);
    const long long m = (long long)kRsBins * ntiles;
    const int nchunk = div_up(m, kRsTile);
    DBuf<int> counts, offsets, totals;
    DBuf<K> ktmp;
    DBuf<V> vtmp;
    counts.alloc(m, st); offsets.alloc(m, st); totals.alloc(nchunk, st);
    ktmp.alloc(n, st); vtmp.alloc(n, st);
    const int npass = std::max(1, (bits + 7) / 8);
    // ping-pong so that the last pass writes keys_out / vals_out
    const K* ks = keys_in;
    const V* vs = vals_in;
    for (int p = 0; p < npass; ++p) {
        const bool to_out = ((npass - 1 - p) % 2) == 0;
        K* kd = to_out ? keys_out : ktmp.p;
        V* vd = to_out ? vals_out : vtmp.p;
        const int shift = 8 * p;
        k_rs_hist<K><<<ntiles, kRsThreads, 0, st>>>(ks, n, shift, ntiles, counts.p);
        PB_CHECK_LAUNCH();
        k_scan_chunks<<<nchunk, kRsThreads, 0, st>>>(counts.p, m, offsets.p, totals.p);
        PB_CHECK_LAUNCH();
        k_scan_totals<<<1, kRsThreads, 0, st>>>(totals.p, nchunk);
        PB_CHECK_LAUNCH();
        k_scan_add<<<div_up(m, 256), 256, 0, st>>>(offsets.p, m, totals.p);
        PB_CHECK_LAUNCH();
        k_rs_scatter<K, V><<<ntiles, kRsThreads, 0, st>>>(ks, vs, n, shift, ntiles, offsets.p, kd, vd);
        PB_CHECK_LAUNCH();
        ks = kd;
        vs = vd;
    }
}

void radix_sort_pairs(const uint64_t* keys_in, const int* vals_in, uint64_t* keys_out, int* vals_out, long long n,
                      int bits, cudaStream_t st) {
    radix_sort_pairs_t<uint64_t, int>(keys_in, vals_in, keys_out, vals_out, n, bits, st);
}

void radix_sort_pairs(const unsigned* keys_in, const int* vals_in, unsigned* keys_out, int* vals_out, long long n,
                      int bits, cudaStream_t st) {
    radix_sort_pairs_t<unsigned, int>(keys_in, vals_in, keys_out, vals_out, n, bits, st);
}

}  // namespace pbfmm

// test hook (include/pbfmm_testing.h): sort host pairs through the GPU
extern "C" int pbfmm_test_radix_sort(const uint64_t* keys, const int32_t* vals, int64_t n, int bits,
                                     uint64_t* keys_out, int32_t* vals_out) {
    using namespace pbfmm;
    try {
        if (n < 0 || bits < 1 || bits > 64) return PB_EINVAL;
        if (n == 0) return PB_OK;
        cudaStream_t st = nullptr;
        DBuf<uint64_t> ki, ko;
        DBuf<int> vi, vo;
        ki.alloc(n, st); ko.alloc(n, st); vi.alloc(n, st); vo.alloc(n, st);
        PB_CUDA(cudaMemcpyAsync(ki.p, keys, n * 8, cudaMemcpyHostToDevice, st));
        PB_CUDA(cudaMemcpyAsync(vi.p, vals, n * 4, cudaMemcpyHostToDevice, st));
        radix_sort_pairs(ki.p, vi.p, ko.p, vo.p, n, bits, st);
        PB_CUDA(cudaMemcpyAsync(keys_out, ko.p, n * 8, cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaMemcpyAsync(vals_out, vo.p, n * 4, cudaMemcpyDeviceToHost, st));
        PB_CUDA(cudaStreamSynchronize(st));
        return PB_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

