// Solvation energy of a solved system without any device allocation.
//
// pb_solvation_energy() allocates small device buffers (the reaction
// potential at the atoms and its partial sums) on every call.  Some callers
// cannot allocate device memory at the point where they need the energy: an
// application whose device allocator is locked after start-up (a fixed
// memory budget reserved up front), or a real-time loop that must not enter
// the driver's allocator and risk its latency or an out-of-memory failure
// half-way through a step.  pb_solvation_energy_noalloc() serves them: it
// runs the same two steps (reaction potential at every atom by the direct
// FP64 sum, then the FP64 energy sum) with all intermediate values kept in
// one fixed scratch array that lives in this file for the life of the
// process.  It has no counterpart in the paper.
#include "bem.cuh"

namespace pbfmm {

// Largest atom count accepted, and the scratch array: 2 x 262,144 doubles
// (4 MB), enough for at least two partial sums per atom.  Every GPU that
// loads the library keeps this array until the process exits.
constexpr int64_t kNoAllocMaxAtoms = 1 << 18;
constexpr int64_t kNoAllocScratch = 2 * kNoAllocMaxAtoms;

static __device__ __align__(256) double g_phir_scratch[kNoAllocScratch];

constexpr double kInv4PiN = 0.07957747154594767;
constexpr double kKcalN = 332.0637;

// Partial reaction potentials (Eq. phi_reac, -K_L[phi] + V_L[dphi] at the
// atoms, without the 1/(4 pi)): grid (atom tiles of 128, nsplit ranges of
// quadrature points); range `split` writes scratch[split * na + atom].
// Every scratch entry in [0, nsplit * na) is written, so nothing needs
// clearing between calls.
__global__ void k_phi_reac_scratch(int na, const double4* __restrict__ atoms, long long np, int nq, int nt,
                                   const double* __restrict__ qp, const double* __restrict__ qn,
                                   const double* __restrict__ qw, const double* __restrict__ x, int nsplit,
                                   double* __restrict__ scratch) {
    __shared__ double s_p[128][4];
    __shared__ double s_n[128][3];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int split = blockIdx.y;
    const long long b_lo = np * split / nsplit, b_hi = np * (split + 1) / nsplit;
    double px = 0, py = 0, pz = 0;
    if (k < na) { px = atoms[k].x; py = atoms[k].y; pz = atoms[k].z; }
    double acc = 0.0;
    for (long long b0 = b_lo; b0 < b_hi; b0 += 128) {
        __syncthreads();
        long long b = b0 + threadIdx.x;
        if (b < b_hi) {
            int t = (int)(b / nq);
            double w = qw[b];
            s_p[threadIdx.x][0] = qp[3 * b];
            s_p[threadIdx.x][1] = qp[3 * b + 1];
            s_p[threadIdx.x][2] = qp[3 * b + 2];
            s_p[threadIdx.x][3] = w * x[nt + t];          // monopole w dphi
            double d = -w * x[t];                         // dipole -w phi
            s_n[threadIdx.x][0] = d * qn[3 * b];
            s_n[threadIdx.x][1] = d * qn[3 * b + 1];
            s_n[threadIdx.x][2] = d * qn[3 * b + 2];
        }
        __syncthreads();
        int cnt = (int)min((long long)128, b_hi - b0);
        for (int m = 0; m < cnt; ++m) {
            double dx = px - s_p[m][0], dy = py - s_p[m][1], dz = pz - s_p[m][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rinv = r2 > 0 ? rsqrt(r2) : 0.0;
            acc += rinv * s_p[m][3] + (dx * s_n[m][0] + dy * s_n[m][1] + dz * s_n[m][2]) * rinv * rinv * rinv;
        }
    }
    if (k < na) scratch[(long long)split * na + k] = acc;
}

// Eq. energy: 1/2 sum_k q_k phi_reac(r_k) * 4 pi C in FP64, one block; the
// partial sums of each atom are added in split order, the atoms with a
// Kahan sum per thread and a fixed tree across threads.
__global__ void k_energy_scratch(int na, int nsplit, const double4* __restrict__ atoms,
                                 const double* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
        double phir = 0.0;
        for (int q = 0; q < nsplit; ++q) phir += scratch[(long long)q * na + k];
        double v = atoms[k].w * (phir * kInv4PiN) - c;
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

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side handle,
// not a device address).
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
    if (!ctx) return PB_EINVAL;
    if (!res || !dG_device) {
        ctx->last_error = "pb_solvation_energy_noalloc: null result or output";
        return PB_EINVAL;
    }
    try {
        if (res->na > kNoAllocMaxAtoms) {
            ctx->last_error = "pb_solvation_energy_noalloc: more atoms than the scratch array holds (262144)";
            return PB_EINVAL;
        }
        if (res->mesh->basis != PB_P0) {
            ctx->last_error = "pb_solvation_energy_noalloc: results on P0 meshes only";
            return PB_EINVAL;
        }
        PB_CUDA(cudaSetDevice(ctx->device));
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, dG_device) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != ctx->device) {
            cudaGetLastError();
            ctx->last_error = "pb_solvation_energy_noalloc: dG_device must be device memory of the context's GPU";
            return PB_EINVAL;
        }
        double* scratch = scratch_for_device(ctx->device);
        const pb_mesh* M = res->mesh;
        cudaStream_t st = ctx->stream;
        const int nt = (int)M->nt, nq = M->nq;
        const long long np = (long long)nt * nq;
        const int na = (int)res->na;
        // split the quadrature points so that the grid has at least two CTAs
        // per SM, as far as the scratch array holds the partial sums
        const int tiles = div_up(na, 128);
        long long nsplit = std::max<long long>(1, div_up(2 * ctx->sm_count, tiles));
        nsplit = std::min<long long>(nsplit, std::max<long long>(1, div_up(np, 128)));
        nsplit = std::min<long long>(nsplit, kNoAllocScratch / na);
        k_phi_reac_scratch<<<dim3(tiles, (unsigned)nsplit), 128, 0, st>>>(
            na, (const double4*)res->atoms.p, np, nq, nt, M->qp_d.p, M->qn_d.p, M->qw_d.p, res->x.p, (int)nsplit,
            scratch);
        PB_CHECK_LAUNCH();
        k_energy_scratch<<<1, 1024, 0, st>>>(na, (int)nsplit, (const double4*)res->atoms.p, scratch, dG_device);
        PB_CHECK_LAUNCH();
    } catch (const Error& e) {
        ctx->last_error = e.what();
        return e.code;
    }
    ctx->last_error.clear();
    return PB_OK;
}
