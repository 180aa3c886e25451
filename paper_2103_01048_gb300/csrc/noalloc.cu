// Solvation energy of a solved system without any device allocation.
//
// pb_solvation_energy() allocates a small device buffer for the reaction
// potential at the atoms on every call.  Callers that cannot allocate device
// memory at that point (code running while a CUDA graph is being captured,
// allocators that are locked down after start-up, or real-time loops that
// must not touch the allocator) use pb_solvation_energy_noalloc() instead:
// it runs the same two steps (reaction potential at every atom, then the
// FP64 energy sum) with the reaction potential kept in a fixed scratch
// array that lives in this file for the life of the process.
#include "bem.cuh"

namespace pbfmm {

// Largest atom count the scratch array holds (2 MB of doubles).  Every GPU
// that loads the library keeps this array until the process exits.
constexpr int64_t kNoAllocMaxAtoms = 1 << 18;

static __device__ __align__(256) double g_phir_scratch[kNoAllocMaxAtoms];

constexpr double kInv4PiN = 0.07957747154594767;
constexpr double kKcalN = 332.0637;

// reaction potential at each atom, written to the scratch array
__global__ void k_phi_reac_scratch(int na, const double4* __restrict__ atoms, long long np, int nq, int nt,
                                   const double* __restrict__ qp, const double* __restrict__ qn,
                                   const double* __restrict__ qw, const double* __restrict__ x,
                                   double* __restrict__ scratch) {
    __shared__ double s_p[128][4];
    __shared__ double s_n[128][3];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double px = 0, py = 0, pz = 0;
    if (k < na) { px = atoms[k].x; py = atoms[k].y; pz = atoms[k].z; }
    double acc = 0.0;
    for (long long b0 = 0; b0 < np; b0 += 128) {
        __syncthreads();
        long long b = b0 + threadIdx.x;
        if (b < np) {
            int t = (int)(b / nq);
            double w = qw[b];
            s_p[threadIdx.x][0] = qp[3 * b];
            s_p[threadIdx.x][1] = qp[3 * b + 1];
            s_p[threadIdx.x][2] = qp[3 * b + 2];
            s_p[threadIdx.x][3] = w * x[nt + t];
            double d = -w * x[t];
            s_n[threadIdx.x][0] = d * qn[3 * b];
            s_n[threadIdx.x][1] = d * qn[3 * b + 1];
            s_n[threadIdx.x][2] = d * qn[3 * b + 2];
        }
        __syncthreads();
        int cnt = (int)min((long long)128, np - b0);
        for (int m = 0; m < cnt; ++m) {
            double dx = px - s_p[m][0], dy = py - s_p[m][1], dz = pz - s_p[m][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rinv = r2 > 0 ? rsqrt(r2) : 0.0;
            acc += rinv * s_p[m][3] + (dx * s_n[m][0] + dy * s_n[m][1] + dz * s_n[m][2]) * rinv * rinv * rinv;
        }
    }
    if (k < na) scratch[k] = acc * kInv4PiN;
}

// 1/2 sum q phi_reac * 4 pi C in FP64 (one block, fixed order)
__global__ void k_energy_scratch(int na, const double4* __restrict__ atoms, const double* __restrict__ scratch,
                                 double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        double v = atoms[k].w * scratch[k] - c;
        double t = s + v;
        c = (t - s) - v;
        s = t;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * red[0] * 4.0 * M_PI * kKcalN;
}

// Device address of the scratch array, looked up once per device (the
// array's name in host code is only a host-side handle).
constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {nullptr};

static double* scratch_for_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) throw Error(PB_EINVAL, "device ordinal out of range");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_phir_scratch);
        if (e != cudaSuccess)
            throw Error(PB_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = (double*)p;
    }
    return g_scratch_addr[dev];
}

}  // namespace pbfmm

using namespace pbfmm;

extern "C" int pb_solvation_energy_noalloc(pb_ctx* ctx, const pb_result* res, double* dG_device) {
    if (!ctx || !res || !dG_device) return PB_EINVAL;
    try {
        if (res->na > kNoAllocMaxAtoms) {
            ctx->last_error = "pb_solvation_energy_noalloc: more atoms than the scratch array holds (262144)";
            return PB_EINVAL;
        }
        PB_CUDA(cudaSetDevice(ctx->device));
        double* scratch = scratch_for_device(ctx->device);
        const pb_mesh* M = res->mesh;
        cudaStream_t st = ctx->stream;
        const int nt = (int)M->nt, nq = M->nq;
        const long long np = (long long)nt * nq;
        const int na = (int)res->na;
        k_phi_reac_scratch<<<div_up(na, 128), 128, 0, st>>>(na, (const double4*)res->atoms.p, np, nq, nt, M->qp_d.p,
                                                          M->qn_d.p, M->qw_d.p, res->x.p, scratch);
        PB_CHECK_LAUNCH();
        k_energy_scratch<<<1, 1024, 0, st>>>(na, (const double4*)res->atoms.p, scratch, dG_device);
        PB_CHECK_LAUNCH();
    } catch (const Error& e) {
        ctx->last_error = e.what();
        return e.code;
    }
    ctx->last_error.clear();
    return PB_OK;
}
