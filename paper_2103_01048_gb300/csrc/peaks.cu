// Microbenchmarks of the GPU's arithmetic pipes: the roofline denominators
// of the kernels that are bound by plain ALU work (the near field and the
// check potentials: FP32 fused multiply-add and the MUFU reciprocal square
// root and base-2 exponential), by FP64 arithmetic (the all-FP64 path), or
// by the tensor cores (box operators: tcgen05 kind::tf32).  The BF16
// tensor-core rate is measured with the same loop to compare this method
// with a library GEMM's measured rate, and the packed FP32 FMA
// (fma.rn.f32x2, two FMAs per instruction) to see whether packing raises
// the FP32 rate or only halves the instructions.
//
// Each ALU kernel runs independent dependency chains in every thread (enough
// of them to hide the pipe's latency), unrolled so that loop overhead takes
// about 1% of the issue slots, on a grid that fills every SM.  The tensor-core
// kernel keeps its operands resident in shared memory and one thread per SM
// issues M = 128, N = 256 MMAs into one TMEM accumulator, committing every
// 64 MMAs to an mbarrier (at most two batches in flight); every wait is
// bounded and a timeout is reported instead of hanging.
#include "common.cuh"
#include "tc_ptx.cuh"
#include <algorithm>

namespace pbfmm {

constexpr int kChains = 16;

__global__ void __launch_bounds__(512) k_peak_ffma(long long iters, float b, float c, float* out) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = __fmaf_rn(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) out[0] = s;      // never true: keeps the chains live
}

// packed FP32 (two lanes per register pair): fma.rn.f32x2
__device__ __forceinline__ unsigned long long ffma2_u(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float x, float y) {
    return (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
}

__global__ void __launch_bounds__(512) k_peak_ffma2(long long iters, float b, float c, float* out) {
    unsigned long long a[kChains / 2];
    const unsigned long long bb = pack2(b, b), cc = pack2(c, c);
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) a[j] = pack2(1.0f + 1e-3f * (threadIdx.x + j), 1.0f + 2e-3f * j);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains / 2; ++j) a[j] = ffma2_u(a[j], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) s += __uint_as_float((unsigned)a[j]) + __uint_as_float((unsigned)(a[j] >> 32));
    if (s == -1.0f) out[0] = s;
}

__global__ void __launch_bounds__(512) k_peak_dfma(long long iters, double b, double c, double* out) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = __fma_rn(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0) out[0] = s;
}

__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 1/sqrt(x) converges to 1; x <- 2^(-x) to 0.6412: no denormals, no inf
__global__ void __launch_bounds__(512) k_peak_rsqrt(long long iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 2.0f + 1e-3f * (threadIdx.x + j);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = mufu_rsqrt(a[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) out[0] = s;
}

__global__ void __launch_bounds__(512) k_peak_ex2(long long iters, float* out) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.5f + 1e-3f * (threadIdx.x + j);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = mufu_ex2(-a[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.0f) out[0] = s;
}

// ---------------------------------------------------------------------------
// tensor cores: D[128 x 256] += A[128 x K] B[256 x K]^T, K-major, 128B swizzle
// ---------------------------------------------------------------------------
constexpr int kPkN = 256;
constexpr int kPkBatch = 64;          // MMAs per commit

// kind::tf32 (K = 8 per MMA) or kind::f16 with BF16 A and B (K = 16)
__device__ __forceinline__ void mma_kind(bool bf16, uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
    if (bf16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        mma_tf32(dt, ad, bd, idesc, acc);
    }
}

// instruction descriptor: D f32, A and B both BF16, K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

struct PeakSmem {
    uint64_t bar[2];
    uint32_t tmem_slot;
};

__global__ void __launch_bounds__(128, 1) k_peak_mma(long long nbatch, int bf16, int* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                          // 128 rows x 128 B
    uint8_t* sB = smem + 128 * 128;              // 256 rows x 128 B
    PeakSmem* S = (PeakSmem*)(sB + kPkN * 128);
    const int tid = threadIdx.x;
    // operands: small finite values (as FP32 words for TF32; each word is two
    // BF16 values, 0.0078 and a tiny one, for BF16)
    for (int i = tid; i < (128 + kPkN) * 32; i += blockDim.x) ((float*)sA)[i] = 0.0078125f * (1 + (i % 7));
    if (tid == 0) {
        mbar_init(&S->bar[0], 1);
        mbar_init(&S->bar[1], 1);
        fence_mbar_init();
    }
    if (tid < 32) {
        tmem_alloc(&S->tmem_slot, kPkN);
        tmem_relinquish();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = S->tmem_slot;
    if (tid == 0) {
        const uint32_t idesc = bf16 ? idesc_bf16(kPkN) : idesc_tf32(kPkN);
        const uint32_t aB = smem_u32(sA), bB = smem_u32(sB);
        bool ok = true;
        long long b = 0;
        for (; b < nbatch; ++b) {
            // at most two batches in flight: wait for the batch before the last
            if (b >= 2 && !mbar_wait(&S->bar[b & 1], ((b - 2) >> 1) & 1)) { ok = false; break; }
            for (int m = 0; m < kPkBatch; m += 4)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_kind(bf16 != 0, taddr, sw128_desc(aB + ks * 32), sw128_desc(bB + ks * 32), idesc,
                             (b > 0 || m > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&S->bar[b & 1]);
        }
        // drain: the last two commits (bounded; on a timeout wait once more
        // before the accumulator is freed)
        for (long long k = std::max(0LL, b - 2); k < b; ++k) {
            if (!mbar_wait(&S->bar[k & 1], (k >> 1) & 1)) {
                ok = false;
                mbar_wait(&S->bar[k & 1], (k >> 1) & 1);
            }
        }
        if (!ok) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) tmem_dealloc(taddr, kPkN);
}

}  // namespace pbfmm

using namespace pbfmm;

extern "C" int pbfmm_measure_peaks(int device, double* out) {
    if (!out) return PB_EINVAL;
    try {
        PB_CUDA(cudaSetDevice(device));
        int sms = 0;
        PB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        cudaStream_t st;
        PB_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        cudaEvent_t e0, e1;
        PB_CUDA(cudaEventCreate(&e0));
        PB_CUDA(cudaEventCreate(&e1));
        float* fo = nullptr;
        double* dof = nullptr;
        int* err = nullptr;
        PB_CUDA(cudaMalloc((void**)&fo, 64));
        PB_CUDA(cudaMalloc((void**)&dof, 64));
        PB_CUDA(cudaMalloc((void**)&err, 64));
        PB_CUDA(cudaMemset(err, 0, 64));
        // as many 512-thread blocks as fit on every SM at once (one wave)
        int occ = 0;
        PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak_dfma, 512, 0));
        const int threads = 512, blocks = std::max(1, occ) * sms;
        const double nthreads = (double)threads * blocks;
        const double per_iter = 16.0 * kChains;               // operations per thread per loop trip
        auto timed = [&](auto launch) -> double {
            launch(true);                                     // warm-up (clocks up, code loaded)
            PB_CUDA(cudaEventRecord(e0, st));
            launch(false);
            PB_CUDA(cudaEventRecord(e1, st));
            PB_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            PB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            return ms * 1e-3;
        };
        const long long it_f = 10000, it_m = 1500, it_d = 200;
        double t;
        t = timed([&](bool w) { k_peak_ffma<<<blocks, threads, 0, st>>>(w ? it_f / 10 : it_f, 0.999f, 1e-3f, fo); });
        PB_CHECK_LAUNCH();
        out[0] = 2.0 * nthreads * per_iter * it_f / t * 1e-12;            // FP32 TFLOP/s
        t = timed([&](bool w) { k_peak_rsqrt<<<blocks, threads, 0, st>>>(w ? it_m / 10 : it_m, fo); });
        PB_CHECK_LAUNCH();
        out[1] = nthreads * per_iter * it_m / t * 1e-12;                  // T rsqrt/s
        t = timed([&](bool w) { k_peak_ex2<<<blocks, threads, 0, st>>>(w ? it_m / 10 : it_m, fo); });
        PB_CHECK_LAUNCH();
        out[2] = nthreads * per_iter * it_m / t * 1e-12;                  // T ex2/s
        t = timed([&](bool w) { k_peak_dfma<<<blocks, threads, 0, st>>>(w ? it_d / 10 : it_d, 0.999, 1e-3, dof); });
        PB_CHECK_LAUNCH();
        out[3] = 2.0 * nthreads * per_iter * it_d / t * 1e-12;            // FP64 TFLOP/s
        // shared memory sized so that one CTA fills an SM (one issuing thread per tensor core)
        const size_t sm = std::max<size_t>(1024 + (128 + kPkN) * 128 + sizeof(PeakSmem), 160 * 1024);
        PB_CUDA(cudaFuncSetAttribute(k_peak_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const long long nb = 6000;                                         // batches of 64 MMAs per SM
        for (int bf = 0; bf < 2; ++bf) {
            t = timed([&](bool w) { k_peak_mma<<<sms, 128, sm, st>>>(w ? nb / 10 : nb, bf, err); });
            PB_CHECK_LAUNCH();
            const double k = bf ? 16.0 : 8.0;
            out[4 + bf] = 2.0 * 128 * kPkN * k * kPkBatch * nb * sms / t * 1e-12;   // TFLOP/s
        }
        int herr = 0;
        // packed FP32: the same FLOPs per thread in half the instructions
        t = timed([&](bool w) { k_peak_ffma2<<<blocks, threads, 0, st>>>(w ? it_f / 10 : it_f, 0.999f, 1e-3f, fo); });
        PB_CHECK_LAUNCH();
        out[6] = 2.0 * nthreads * per_iter * it_f / t * 1e-12;            // FP32 TFLOP/s, f32x2 FMA
        PB_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        cudaFree(fo);
        cudaFree(dof);
        cudaFree(err);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
        return herr ? PB_ETIMEOUT : PB_OK;
    } catch (const Error& e) {
        return e.code;
    }
}
