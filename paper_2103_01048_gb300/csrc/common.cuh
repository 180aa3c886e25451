// Shared internals of the pbfmm library (device helpers, context, errors).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <tuple>
#include <memory>
#include <map>
#include <vector>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <atomic>

#include "../../include/pbfmm.h"
#include <nvtx3/nvToolsExt.h>

namespace pbfmm {

constexpr int kMaxLevel = 21;      // 21 bits per axis in a 63-bit Morton key
constexpr int kCollCap = 27;       // same-level adjacent boxes, self included
constexpr int kCoarseCap = 26;     // coarser adjacent leaves (disjoint cubes touching a cube)
constexpr int kVCap = 189;         // 6^3 - 3^3 children of the parent's colleagues
constexpr int kXCap = 26;
constexpr int kNumOffsets = 343;   // 7^3 relative offsets of a V-list pair (27 unused)

// Error carried through the C-ABI: every internal failure throws this and the
// entry point converts it to a status code + message.
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define PB_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            throw ::pbfmm::Error(PB_ECUDA, std::string(#call) + ": " +             \
                                               cudaGetErrorString(e_));            \
    } while (0)

// Counts the library's kernel launches (reported by pb_profile_read); called
// once after every launch.
extern thread_local long long g_launch_count;
#define PB_CHECK_LAUNCH()                         \
    do {                                          \
        ++::pbfmm::g_launch_count;                \
        PB_CUDA(cudaGetLastError());              \
    } while (0)

#define PB_REQUIRE(cond, code, msg)                                                \
    do {                                                                           \
        if (!(cond)) throw ::pbfmm::Error(code, msg);                              \
    } while (0)

// Device allocations made through DBuf (all of the library's device memory
// except the context's error flag), counted for tests; and an injected
// failure: when g_alloc_fail_at > 0, the allocation with that count number
// throws PB_ENOMEM as a failed cudaMallocAsync would (pbfmm_testing.h).
extern std::atomic<long long> g_alloc_count;
extern std::atomic<long long> g_alloc_fail_at;
inline void count_alloc() {
    const long long k = ++g_alloc_count;
    if (k == g_alloc_fail_at.load()) throw Error(PB_ENOMEM, "device allocation failed (injected by a test)");
}
// Cycle limit of the tensor-core kernels' bounded waits (about 1 s at the
// boost clock); tests shorten it to make a wait give up (pbfmm_testing.h).
extern std::atomic<long long> g_wait_limit;

// Owning device buffer (stream-ordered allocations on the context stream).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        if (count) {
            count_alloc();
            cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), stream);
            if (e != cudaSuccess) {
                p = nullptr;
                throw Error(PB_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
            }
            n = count;
        }
    }
    // grow keeping contents
    void grow(size_t count, cudaStream_t stream) {
        if (count <= n) return;
        count_alloc();
        T* q = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&q, count * sizeof(T), stream);
        if (e != cudaSuccess) throw Error(PB_ENOMEM, "device allocation failed");
        if (n) PB_CUDA(cudaMemcpyAsync(q, p, n * sizeof(T), cudaMemcpyDeviceToDevice, stream));
        if (p) cudaFreeAsync(p, s);
        p = q;
        n = count;
        s = stream;
    }
    void zero(cudaStream_t stream) {
        if (n) PB_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
    }
};

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace pbfmm

// The opaque context of the C-ABI.
struct pb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    int sm_count = 0;
    // per-phase device timers
    bool profile = false;
    double prof_ms[PB_PH_COUNT] = {};
    long long prof_calls[PB_PH_COUNT] = {};
    long long launch_base = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    // device-side error flag of kernels with bounded waits (0 = fine); read
    // and cleared by the next synchronising call, reported as PB_ETIMEOUT
    int* dev_err = nullptr;
    // options (pb_set_option)
    int coupling = 0;          // 0 auto, 1 direct sums, 2 FMM
    int deterministic = 0;     // 1: no run-dependent reductions (SIMT M2L/M2M/L2L)
    int singular = 0;          // singular entries: 0 auto, 1 FP64 (depth 5), 2 FP32 (depth 4)
    int overlap = 0;           // 1: near field of the paired apply on `aux`, beside the far field
    int leaf_nt = 0;           // targets per thread of the paired leaf kernel (0: by precision)
    int leaf_packed = 1;       // FP32 paired leaf kernel with packed (f32x2) arithmetic
    int m2l_tile = 0;          // 0: M = 256 (CTA pairs) where allowed; 1: M = 128 (one CTA per part)
    int list_direct = 1;       // small W boxes and small leaves' X lists evaluated directly (packed path)
    int restart = 0;           // GMRES restart length of the batched solves (0: none)
    // second stream (and fork / join events) for the near field of the paired
    // apply; null: everything on `stream`
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // translation-operator sets shared by the context's trees, keyed by
    // (kernel, kappa, p, root half-width, levels); weak references, so a set
    // lives as long as some tree uses it
    std::map<std::tuple<int, double, int, double, int>, std::weak_ptr<void>> op_cache;
};

namespace pbfmm {
// A phase of the library's work: an NVTX range named after the phase (for
// profilers and tracers; without a tool attached the calls do nothing) and,
// with pb_profile on, a pair of CUDA events on the context stream.
constexpr const char* kPhaseNames[PB_PH_COUNT] = {"gather", "p2m", "m2m", "p2l", "m2l",
                                                  "down", "leaf", "scatter", "bem", "gmres"};
struct PhaseTimer {
    pb_ctx* ctx;
    int phase;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseTimer(pb_ctx* c, int ph) : PhaseTimer(c, ph, c->stream) {}
    PhaseTimer(pb_ctx* c, int ph, cudaStream_t s) : ctx(c), phase(ph), st(s) {
        nvtxRangePushA(kPhaseNames[ph]);
        if (ctx->profile) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
        }
    }
    ~PhaseTimer() {
        if (a) {
            cudaEventRecord(b, st);
            ctx->pending.push_back({phase, {a, b}});
        }
        nvtxRangePop();
    }
};
void profile_collect(pb_ctx* ctx);
}  // namespace pbfmm
