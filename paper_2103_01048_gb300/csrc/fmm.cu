// KIFMM apply (Sec. "Fast multipole method"): upward pass (P2M at leaves,
// M2M in post-order), M2L over the interaction lists, downward pass (L2L in
// pre-order), then L2P + P2P at the leaves.  Adaptive-tree extras: M2P for
// the W list and P2L for the X list.
//
// Layout in HBM: Morton-sorted sources as float4 (x, y, z, q) plus float4
// (d n_x, d n_y, d n_z, 0) for double-layer sources; equivalent densities
// and check potentials box-major [n_box][npad].  Everything here is templated
// on the arithmetic type: float (mixed path) and double (all-FP64 path).
#include "fmm.cuh"
#include <algorithm>
#include <climits>
#include <memory>
#include <type_traits>

namespace pbfmm {

bool m2l_tc_launch(const fmm_tree* T, const Operators& O, const float* Qu, float* Qd, int* err, cudaStream_t st);
bool pc_tc_launch(const fmm_tree* T, const Operators& O, int child_level, bool up, float* Q, int* err,
                  cudaStream_t st);
bool c2e_tc_launch(const fmm_tree* T, const Operators& O, bool up, const float* X, float* Y, float* tmp, int* err,
                   cudaStream_t st, bool xfar = false);
// two operator sets (Laplace, Yukawa) in the same launches
bool m2l_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, const float* Qu, float* Qd,
                    const float* Qu2, float* Qd2, int* err, cudaStream_t st);
bool pc_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, int child_level, bool up, float* Q,
                   float* Q2, int* err, cudaStream_t st);
bool c2e_tc_launch2(const fmm_tree* T, const Operators& O, const Operators* O2, bool up, const float* X, float* Y,
                    float* tmp, const float* X2, float* Y2, float* tmp2, int* err, cudaStream_t st, bool xfar = false);
// X-list boxes that keep P2L when small leaves sum their X lists directly
bool c2e_tc_ok(const Operators& O);
void build_xbox_far(fmm_tree* T, int thrX);

constexpr double kInv4PiD = 0.07957747154594767;
constexpr double kLog2E = 1.4426950408889634;     // log2(e)
constexpr int kTC = 32;    // boxes per tile of the dense box-vector products (= kM2LTile)
static_assert(kTC == kM2LTile, "M2L tile width");

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
// FP32: the MUFU approximations with denormals flushed (distances and
// exponentials of the far field never reach the denormal range; r = 0 is
// guarded before use)
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
// 2^x
template <typename T> __device__ __forceinline__ T exp2_t(T x);
template <> __device__ __forceinline__ float exp2_t<float>(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double exp2_t<double>(double x) { return exp2(x); }
template <typename T> __device__ __forceinline__ T exp_t(T x);
template <> __device__ __forceinline__ float exp_t<float>(float x) { return exp2_t<float>(x * float(kLog2E)); }
template <> __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// One source-target interaction, without the 1/(4 pi) factor:
//   pot += g q + (d.m) f,   dn += -(d.n_t) f q,   d = x_t - y_s,
//   g = e/r, f = e (1 + kappa r)/r^3, e = exp(-kappa r) (Yukawa) or 1.
// GUARD: the pair may coincide (r = 0 contributes nothing).  Coincident
// points share a Morton key, hence a leaf, so only a leaf's own box needs it.
template <typename T, bool YUK, bool DL, bool DN, bool GUARD = true>
__device__ __forceinline__ void interact(T dx, T dy, T dz, T q, T mx, T my, T mz, T nx, T ny, T nz, T kappa,
                                         T& pot, T& dn) {
    T r2 = dx * dx + dy * dy + dz * dz;
    T rinv = GUARD ? (r2 > T(0) ? rsqrt_t<T>(r2) : T(0)) : rsqrt_t<T>(r2);
    T g = rinv, f = rinv * rinv * rinv;
    if (YUK) {
        T r = r2 * rinv;
        T e = exp_t<T>(-kappa * r);
        g *= e;
        f *= e * (T(1) + kappa * r);
    }
    pot += g * q;
    if (DL) pot += (dx * mx + dy * my + dz * mz) * f;
    if (DN) dn -= (dx * nx + dy * ny + dz * nz) * f * q;
}

// The Laplace and the Yukawa interaction of one pair with the geometry
// shared (the direct formulation applies both kernels to the same points),
// without the 1/(4 pi) factor; both kernels take the same dipole m:
//   potL += g qL + (d.m) f,               dnL -= (d.n) f qL,
//   potY += e (g qY + (d.m) f (1 + kr)),  dnY -= e (1 + kr) (d.n) f qY,
//   g = 1/r, f = 1/r^3, e = exp(-kappa r) (Sec. "Fast multipole method").
// kl2 = -kappa log2(e), so that e = 2^(kl2 r).  Grouped as
//   potL += (qL + (d.m) / r^2) / r,   potY += (e / r) (qY + (d.m)(1 + kr) / r^2).
template <typename T, bool DL, bool DN, bool GUARD>
__device__ __forceinline__ void interact_pair(T dx, T dy, T dz, T qL, T qY, T mx, T my, T mz, T nx, T ny, T nz,
                                              T kappa, T kl2, T& potL, T& potY, T& dnL, T& dnY) {
    T r2 = dx * dx + dy * dy + dz * dz;
    T rinv = GUARD ? (r2 > T(0) ? rsqrt_t<T>(r2) : T(0)) : rsqrt_t<T>(r2);
    T r = r2 * rinv;
    T er = exp2_t<T>(kl2 * r) * rinv;              // e^{-kr} / r
    if (DL || DN) {
        T rinv2 = rinv * rinv;
        T u = kappa * r + T(1);
        if (DL) {
            T w = (dx * mx + dy * my + dz * mz) * rinv2;
            potL += rinv * (w + qL);
            potY += er * (w * u + qY);
        } else {
            potL += rinv * qL;
            potY += er * qY;
        }
        if (DN) {
            T dn = (dx * nx + dy * ny + dz * nz) * rinv2;
            dnL -= rinv * dn * qL;
            dnY -= er * u * dn * qY;
        }
    } else {
        potL += rinv * qL;
        potY += er * qY;
    }
}

// ---------------------------------------------------------------------------
// gather of the densities into Morton order
// ---------------------------------------------------------------------------
template <typename T, typename In>
__global__ void k_gather_src(long long n, const int* __restrict__ perm, const float4* __restrict__ pos,
                             const In* __restrict__ q, const In* __restrict__ dip, const In* __restrict__ nrm,
                             typename V4<T>::type* __restrict__ sq, typename V4<T>::type* __restrict__ sm) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long i = perm[k];
    float4 p = pos[k];
    T qq = q ? (T)q[i] : T(0);
    sq[k] = {(T)p.x, (T)p.y, (T)p.z, qq};
    if (sm) {
        T d = (T)dip[i];
        sm[k] = {d * (T)nrm[3 * i], d * (T)nrm[3 * i + 1], d * (T)nrm[3 * i + 2], T(0)};
    }
}

// paired apply: sq = (x, y, z, q_lap), sm = (d n_x, d n_y, d n_z, q_yuk)
template <typename T, typename In>
__global__ void k_gather_pair(long long n, const int* __restrict__ perm, const float4* __restrict__ pos,
                              const In* __restrict__ qL, const In* __restrict__ qY, const In* __restrict__ dip,
                              const In* __restrict__ nrm, typename V4<T>::type* __restrict__ sq,
                              typename V4<T>::type* __restrict__ sm) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long i = perm[k];
    float4 p = pos[k];
    sq[k] = {(T)p.x, (T)p.y, (T)p.z, qL ? (T)qL[i] : T(0)};
    T d = dip ? (T)dip[i] : T(0);
    sm[k] = {dip ? d * (T)nrm[3 * i] : T(0), dip ? d * (T)nrm[3 * i + 1] : T(0), dip ? d * (T)nrm[3 * i + 2] : T(0),
             qY ? (T)qY[i] : T(0)};
}

template <typename T, typename In>
__global__ void k_gather_tn(long long n, const int* __restrict__ perm, const In* __restrict__ nrm,
                            typename V4<T>::type* __restrict__ tn) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long i = perm[k];
    tn[k] = {(T)nrm[3 * i], (T)nrm[3 * i + 1], (T)nrm[3 * i + 2], T(0)};
}

template <typename T, typename Out>
__global__ void k_scatter(long long n, const int* __restrict__ perm, const T* __restrict__ v, Out* __restrict__ out) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[perm[k]] = (Out)v[k];
}

// ---------------------------------------------------------------------------
// P2M / P2L: source points -> check surface of a box.
// One CTA per box.  Sources are taken relative to the box centre (FP64
// subtraction) so the surface geometry keeps full relative precision.
// mode 0 (P2M): sources = the box's own points, check surface at 2.95 r.
// mode 1 (P2L): sources = points of the X-list leaves, check surface at 1.05 r.
// ---------------------------------------------------------------------------
template <typename T, bool YUK, bool DL, int MAXP>
__global__ void __launch_bounds__(256) k_p2check(int nbox, const int* __restrict__ boxes, int mode,
                                                 const double4* __restrict__ center, const int* __restrict__ sb,
                                                 const int* __restrict__ se, const int* __restrict__ X,
                                                 const int* __restrict__ X_n,
                                                 const typename V4<T>::type* __restrict__ sq,
                                                 const typename V4<T>::type* __restrict__ sm,
                                                 const float4* __restrict__ surf, int ne, int npad, T kappa,
                                                 T* __restrict__ chk, const int* __restrict__ nchild,
                                                 const int* __restrict__ tb, const int* __restrict__ te, int thrX) {
    // one (MAXP = 1) or two check points per thread; blockDim.x <= 256
    using V = typename V4<T>::type;
    __shared__ V s_q[256];
    __shared__ V s_m[DL ? 256 : 1];
    const int CH = blockDim.x;
    int bi = blockIdx.x;
    if (bi >= nbox) return;
    int b = boxes[bi];
    if (mode == 1 && thrX >= 0 && nchild[b] == 0 && te[b] - tb[b] <= thrX) {
        // a leaf of at most thrX targets takes its X list directly in the leaf kernel
        for (int i = threadIdx.x; i < npad; i += CH) chk[(long long)b * npad + i] = T(0);
        return;
    }
    double4 c = center[b];
    T alpha = T(mode == 0 ? kAlphaOuter : kAlphaInner) * (T)c.w;
    T px[MAXP], py[MAXP], pz[MAXP], acc[MAXP];
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
        int i = threadIdx.x + m * CH;
        float4 s = (i < ne) ? surf[i] : make_float4(0, 0, 0, 0);
        px[m] = alpha * (T)s.x; py[m] = alpha * (T)s.y; pz[m] = alpha * (T)s.z;
        acc[m] = T(0);
    }
    int nlist = (mode == 0) ? 1 : X_n[b];
    T dummy = T(0);
    for (int li = 0; li < nlist; ++li) {
        int a = (mode == 0) ? b : X[(long long)b * kXCap + li];
        int j0 = sb[a], j1 = se[a];
        for (int jc = j0; jc < j1; jc += CH) {
            int j = jc + threadIdx.x;
            __syncthreads();
            if (j < j1) {
                V v = sq[j];
                s_q[threadIdx.x] = {(T)((double)v.x - c.x), (T)((double)v.y - c.y), (T)((double)v.z - c.z), v.w};
                if (DL) s_m[threadIdx.x] = sm[j];
            }
            __syncthreads();
            int cnt = min(CH, j1 - jc);
            for (int t = 0; t < cnt; ++t) {
                V s = s_q[t];
                T mx = 0, my = 0, mz = 0;
                if (DL) { V mm = s_m[t]; mx = mm.x; my = mm.y; mz = mm.z; }
#pragma unroll
                for (int m = 0; m < MAXP; ++m)
                    interact<T, YUK, DL, false>(px[m] - s.x, py[m] - s.y, pz[m] - s.z, s.w, mx, my, mz, 0, 0, 0,
                                                kappa, acc[m], dummy);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
        int i = threadIdx.x + m * CH;
        if (i < npad) chk[(long long)b * npad + i] = (i < ne) ? acc[m] * T(kInv4PiD) : T(0);
    }
}

// ---- staging of a leaf's source stream in shared memory
// 16-byte asynchronous global -> shared copy (no register round trip; the
// CTA waits once per staged window instead of once per source box).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename V>
__device__ __forceinline__ void cp_async_v(V* smem, const V* gmem) {
    static_assert(sizeof(V) % 16 == 0, "16-byte pieces");
#pragma unroll
    for (int i = 0; i < (int)(sizeof(V) / 16); ++i)
        cp_async16(reinterpret_cast<char*>(smem) + 16 * i, reinterpret_cast<const char*>(gmem) + 16 * i);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// P2M / P2L of the paired apply: Laplace and Yukawa check potentials of the
// same sources in one pass (sm carries the dipole and the Yukawa monopole).
template <typename T, bool DL, int MAXP>
__global__ void __launch_bounds__(256) k_p2check_pair(int nbox, const int* __restrict__ boxes, int mode,
                                                      const double4* __restrict__ center, const int* __restrict__ sb,
                                                      const int* __restrict__ se, const int* __restrict__ X,
                                                      const int* __restrict__ X_n,
                                                      const typename V4<T>::type* __restrict__ sq,
                                                      const typename V4<T>::type* __restrict__ sm,
                                                      const float4* __restrict__ surf, int ne, int npad, T kappa,
                                                      T* __restrict__ chkL, T* __restrict__ chkY) {
    using V = typename V4<T>::type;
    __shared__ V s_q[256];
    __shared__ V s_m[256];
    const int CH = blockDim.x;
    int bi = blockIdx.x;
    if (bi >= nbox) return;
    int b = boxes[bi];
    double4 c = center[b];
    T alpha = T(mode == 0 ? kAlphaOuter : kAlphaInner) * (T)c.w;
    T px[MAXP], py[MAXP], pz[MAXP], aL[MAXP], aY[MAXP];
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
        int i = threadIdx.x + m * CH;
        float4 s = (i < ne) ? surf[i] : make_float4(0, 0, 0, 0);
        px[m] = alpha * (T)s.x; py[m] = alpha * (T)s.y; pz[m] = alpha * (T)s.z;
        aL[m] = aY[m] = T(0);
    }
    // sources: B's own (P2M) or those of the X-list boxes (P2L), the boxes
    // concatenated into full chunks by a uniform cursor over their ranges
    __shared__ int s_xb[kXCap], s_xn[kXCap];
    const int nlist = (mode == 0) ? 1 : X_n[b];
    if (threadIdx.x < nlist) {
        const int a = (mode == 0) ? b : X[(long long)b * kXCap + threadIdx.x];
        s_xb[threadIdx.x] = sb[a];
        s_xn[threadIdx.x] = se[a] - sb[a];
    }
    T d0 = T(0), d1 = T(0);
    const T kl2 = -kappa * T(kLog2E);
    int ui = 0, off = 0;
    while (ui < nlist) {
        __syncthreads();
        int filled = 0;
        while (filled < CH && ui < nlist) {
            const int n = s_xn[ui];
            const int m = min(CH - filled, n - off);
            const int t = threadIdx.x - filled;
            if (t >= 0 && t < m) {
                const int j = s_xb[ui] + off + t;
                V v = sq[j];
                s_q[threadIdx.x] = {(T)((double)v.x - c.x), (T)((double)v.y - c.y), (T)((double)v.z - c.z), v.w};
                s_m[threadIdx.x] = sm[j];
            }
            filled += m;
            off += m;
            if (off >= n) { ++ui; off = 0; }
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < filled; ++t) {
            V s = s_q[t], mm = s_m[t];
#pragma unroll
            for (int m = 0; m < MAXP; ++m)
                interact_pair<T, DL, false, false>(px[m] - s.x, py[m] - s.y, pz[m] - s.z, s.w, mm.w, mm.x, mm.y,
                                                   mm.z, 0, 0, 0, kappa, kl2, aL[m], aY[m], d0, d1);
        }
    }
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
        int i = threadIdx.x + m * CH;
        if (i < npad) {
            chkL[(long long)b * npad + i] = (i < ne) ? aL[m] * T(kInv4PiD) : T(0);
            chkY[(long long)b * npad + i] = (i < ne) ? aY[m] * T(kInv4PiD) : T(0);
        }
    }
}

// ---------------------------------------------------------------------------
// Dense operator x box-vector products (UC2UE, DC2DE, M2M, L2L, M2L), SIMT.
// A CTA computes C[npad x 32 boxes] = sum over terms of Op_term x X_gathered,
// 256 threads as 16 row groups x 16 column pairs, K chunks of 16 in smem.
// ---------------------------------------------------------------------------

enum GemmMode { G_DENSE = 0, G_M2M = 1, G_L2L = 2, G_M2L = 3, G_PAIRS = 4 };

struct GemmArgs {
    int mode;
    int ncols;                 // number of column boxes (modes 0-2)
    const int* cols;           // column box ids (modes 0-2); NULL: col_base + i
    int col_base;
    const int* first_child;
    const int* nchild;
    const int4* anchor;
    const int* parent;
    // M2L schedule
    const int* tile_box;
    const int* tile_level;
    const int* entry_off;
    const int* entry_oidx;
    const int* entry_src;
    int level;                 // operator level (modes 0-2)
    int accumulate;            // mode 0: Y += (else Y =)
    // G_PAIRS: items (first pair, count <= 32, operator index) over (tgt, src)
    // pairs that share one operator; results added into Y with reductions
    const int4* pitems;
    const int* ptgt;
    const int* psrc;
};

// T: type of the box vectors; TO: type of the operator and the accumulation
// (double for the ill-conditioned check-to-equivalent solves).
template <typename T, typename TO, int NPAD>
__device__ __forceinline__ void box_gemm_body(const GemmArgs& a, const TO* __restrict__ ops, const T* __restrict__ Xv,
                                              T* __restrict__ Yv) {
    constexpr int KC = (sizeof(TO) * NPAD * 16 > 40000) ? 8 : 16;
    constexpr int RPT = NPAD / 16;
    __shared__ TO s_op[KC][NPAD + 1];
    __shared__ TO s_x[KC][kTC + 1];
    __shared__ int s_src[kTC];
    __shared__ int s_dst[kTC];
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;   // row group, column pair
    const int tile = blockIdx.x;
    const size_t m2 = (size_t)NPAD * NPAD;
    int nterm, level;
    if (a.mode == G_M2L) {
        nterm = a.entry_off[tile + 1] - a.entry_off[tile];
        level = a.tile_level[tile];
    } else if (a.mode == G_PAIRS) {
        nterm = 1;
        level = a.pitems[tile].z;          // operator index
    } else {
        nterm = (a.mode == G_DENSE) ? 1 : 8;
        level = a.level;
    }
    TO acc[RPT][2];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r][0] = acc[r][1] = TO(0);
    for (int term = 0; term < nterm; ++term) {
        // columns: source box for this term, destination box
        __syncthreads();
        if (tid < kTC) {
            int src = -1, dst = -1;
            if (a.mode == G_M2L) {
                int e = a.entry_off[tile] + term;
                src = a.entry_src[(long long)e * kTC + tid];
                dst = a.tile_box[(long long)tile * kTC + tid];
            } else if (a.mode == G_PAIRS) {
                const int4 it = a.pitems[tile];
                if (tid < it.y) {
                    src = a.psrc[it.x + tid];
                    dst = a.ptgt[it.x + tid];
                }
            } else {
                int ci = tile * kTC + tid;
                int b = ci < a.ncols ? (a.cols ? a.cols[ci] : a.col_base + ci) : -1;
                if (b >= 0) {
                    if (a.mode == G_DENSE) { src = b; dst = b; }
                    else {
                        // child of b in octant `term` (M2M: source; L2L: destination)
                        int ch = -1;
                        int f = a.first_child[b], nc = a.nchild[b];
                        for (int k = 0; k < nc; ++k) {
                            int4 an = a.anchor[f + k];
                            int oct = ((an.x & 1) << 2) | ((an.y & 1) << 1) | (an.z & 1);
                            if (oct == term) ch = f + k;
                        }
                        if (a.mode == G_M2M) { src = ch; dst = nc > 0 ? b : -1; }
                        else { src = (ch >= 0) ? b : -1; dst = ch; }
                    }
                }
            }
            s_src[tid] = src;
            s_dst[tid] = dst;
        }
        __syncthreads();
        bool any = false;
        for (int c = 0; c < kTC; ++c) any |= (s_src[c] >= 0);
        if (!any) continue;
        const TO* op;
        if (a.mode == G_M2L) op = ops + ((size_t)level * kNumOffsets + a.entry_oidx[a.entry_off[tile] + term]) * m2;
        else if (a.mode == G_PAIRS) op = ops + (size_t)level * m2;
        else if (a.mode == G_DENSE) op = ops + (size_t)level * m2;
        else op = ops + ((size_t)level * 8 + term) * m2;
        for (int k0 = 0; k0 < NPAD; k0 += KC) {
            __syncthreads();
            for (int i = tid; i < NPAD * KC; i += 256) {
                int row = i / KC, kk = i % KC;
                s_op[kk][row] = op[(size_t)row * NPAD + k0 + kk];
            }
            for (int i = tid; i < kTC * KC; i += 256) {
                int c = i / KC, kk = i % KC;
                int s = s_src[c];
                s_x[kk][c] = (s >= 0) ? (TO)Xv[(size_t)s * NPAD + k0 + kk] : TO(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                TO x0 = s_x[kk][2 * tx], x1 = s_x[kk][2 * tx + 1];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    TO o = s_op[kk][ty + 16 * r];
                    acc[r][0] += o * x0;
                    acc[r][1] += o * x1;
                }
            }
        }
        if (a.mode == G_L2L) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                int d = s_dst[2 * tx + cc];
                if (d >= 0) {
#pragma unroll
                    for (int r = 0; r < RPT; ++r) Yv[(size_t)d * NPAD + ty + 16 * r] += (T)acc[r][cc];
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; ++r) acc[r][0] = acc[r][1] = TO(0);
        }
    }
    if (a.mode == G_L2L) return;
    if (a.mode == G_PAIRS) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            int d = s_dst[2 * tx + cc];
            if (d < 0) continue;
#pragma unroll
            for (int r = 0; r < RPT; ++r) atomicAdd(&Yv[(size_t)d * NPAD + ty + 16 * r], (T)acc[r][cc]);
        }
        return;
    }
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
        int d = s_dst[2 * tx + cc];
        if (d < 0) continue;
        bool add = (a.mode == G_M2L) || (a.mode == G_DENSE && a.accumulate);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            size_t o = (size_t)d * NPAD + ty + 16 * r;
            Yv[o] = add ? Yv[o] + (T)acc[r][cc] : (T)acc[r][cc];
        }
    }
}

// One kernel name per use so launch lists and profiles separate them.
template <typename T, typename TO, int NPAD>
__global__ void __launch_bounds__(256) k_m2l_simt(GemmArgs a, const TO* __restrict__ ops, const T* __restrict__ X,
                                                  T* __restrict__ Y) { box_gemm_body<T, TO, NPAD>(a, ops, X, Y); }
template <typename T, typename TO, int NPAD>
__global__ void __launch_bounds__(256) k_m2m(GemmArgs a, const TO* __restrict__ ops, const T* __restrict__ X,
                                             T* __restrict__ Y) { box_gemm_body<T, TO, NPAD>(a, ops, X, Y); }
template <typename T, typename TO, int NPAD>
__global__ void __launch_bounds__(256) k_l2l(GemmArgs a, const TO* __restrict__ ops, const T* __restrict__ X,
                                             T* __restrict__ Y) { box_gemm_body<T, TO, NPAD>(a, ops, X, Y); }
template <typename T, typename TO, int NPAD>
__global__ void __launch_bounds__(256) k_check2equiv(GemmArgs a, const TO* __restrict__ ops,
                                                     const T* __restrict__ X, T* __restrict__ Y) {
    box_gemm_body<T, TO, NPAD>(a, ops, X, Y);
}

// ---------------------------------------------------------------------------
// Leaf evaluation: P2P over U(B), M2P over W(B), L2P of B's own downward
// equivalent density, at every target of leaf B.  One CTA (128 threads) per
// target leaf; each thread carries NT targets (t, t + slots, ...) so every
// staged source is loaded once for NT pairs.  A leaf holds at most ncrit
// targets, usually fewer than 128 * NT: the CTA is split into
// G = floor(128 / slots) groups of slots = ceil(target count / NT) threads
// (at least 4); group g takes its share of each staged chunk and the G
// partial sums are added at the end.  The threads past G * slots idle (a
// warp of them issues nothing); the lanes that compute padding targets are
// at most NT - 1 per group, against up to half the CTA with power-of-two
// group sizes.
// ---------------------------------------------------------------------------
template <typename T, bool YUK, bool DL, bool DN, int NT>
__global__ void __launch_bounds__(128) k_leaf_eval(const int* __restrict__ leaves, int nleaf,
                                                   const int* __restrict__ tb, const int* __restrict__ te,
                                                   const int* __restrict__ sb, const int* __restrict__ se,
                                                   const int* __restrict__ U_off, const int* __restrict__ U_ids,
                                                   const int* __restrict__ W_off, const int* __restrict__ W_ids,
                                                   const int* __restrict__ level, const double4* __restrict__ center,
                                                   const float4* __restrict__ tpos,
                                                   const typename V4<T>::type* __restrict__ tn,
                                                   const typename V4<T>::type* __restrict__ sq,
                                                   const typename V4<T>::type* __restrict__ sm,
                                                   const T* __restrict__ Qu, const T* __restrict__ Qd,
                                                   const float4* __restrict__ surf, int ne, int npad, T kappa,
                                                   T* __restrict__ pot_out, T* __restrict__ dn_out) {
    using V = typename V4<T>::type;
    constexpr int CH = 128;
    __shared__ V s_q[CH];
    __shared__ V s_m[DL ? CH : 1];
    __shared__ T s_red[DN ? 2 : 1][NT * CH];
    int li = blockIdx.x;
    if (li >= nleaf) return;
    const int b = leaves[li];
    const int t0 = tb[b], t1 = te[b];
    const int slots = min(CH, max(4, (t1 - t0 + NT - 1) / NT));
    const int G = CH / slots;
    const int tloc = threadIdx.x % slots, g = threadIdx.x / slots;
    const int nw = W_off[b + 1] - W_off[b];
    const int nsrcbox = nw + (level[b] >= 2 ? 1 : 0);
    for (int tc = t0; tc < t1; tc += NT * slots) {
        int ti[NT];
        bool vt[NT];
        float4 xt[NT];
        T nx[NT], ny[NT], nz[NT], pot[NT], dn[NT];
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            ti[u] = tc + tloc + u * slots;
            vt[u] = ti[u] < t1;
            xt[u] = vt[u] ? tpos[ti[u]] : make_float4(0, 0, 0, 0);
            nx[u] = ny[u] = nz[u] = T(0);
            if (DN && vt[u]) { V nn = tn[ti[u]]; nx[u] = nn.x; ny[u] = nn.y; nz[u] = nn.z; }
            pot[u] = dn[u] = T(0);
        }
        // P2P
        for (int ui = U_off[b]; ui < U_off[b + 1]; ++ui) {
            const int a = U_ids[ui];
            const int j0 = sb[a], j1 = se[a];
            for (int jc = j0; jc < j1; jc += CH) {
                int j = jc + threadIdx.x;
                __syncthreads();
                if (j < j1) {
                    s_q[threadIdx.x] = sq[j];
                    if (DL) s_m[threadIdx.x] = sm[j];
                }
                __syncthreads();
                const int cnt = min(CH, j1 - jc);
                if (a == b) {
                    for (int k = g; g < G && k < cnt; k += G) {
                        V s = s_q[k];
                        T mx = 0, my = 0, mz = 0;
                        if (DL) { V mm = s_m[k]; mx = mm.x; my = mm.y; mz = mm.z; }
#pragma unroll
                        for (int u = 0; u < NT; ++u)
                            interact<T, YUK, DL, DN, true>((T)xt[u].x - s.x, (T)xt[u].y - s.y, (T)xt[u].z - s.z, s.w,
                                                           mx, my, mz, nx[u], ny[u], nz[u], kappa, pot[u], dn[u]);
                    }
                } else {
                    for (int k = g; g < G && k < cnt; k += G) {
                        V s = s_q[k];
                        T mx = 0, my = 0, mz = 0;
                        if (DL) { V mm = s_m[k]; mx = mm.x; my = mm.y; mz = mm.z; }
#pragma unroll
                        for (int u = 0; u < NT; ++u)
                            interact<T, YUK, DL, DN, false>((T)xt[u].x - s.x, (T)xt[u].y - s.y, (T)xt[u].z - s.z,
                                                            s.w, mx, my, mz, nx[u], ny[u], nz[u], kappa, pot[u], dn[u]);
                    }
                }
            }
        }
        // M2P (W list) and L2P (own downward equivalent): monopole equivalent densities
        for (int wi = 0; wi < nsrcbox; ++wi) {
            const int a = (wi < nw) ? W_ids[W_off[b] + wi] : b;
            const T* Q = (wi < nw) ? Qu : Qd;
            const double4 ca = center[a];
            const T alpha = T(wi < nw ? kAlphaInner : kAlphaOuter) * (T)ca.w;
            T rx[NT], ry[NT], rz[NT];
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                rx[u] = (T)((double)xt[u].x - ca.x);
                ry[u] = (T)((double)xt[u].y - ca.y);
                rz[u] = (T)((double)xt[u].z - ca.z);
            }
            for (int jc = 0; jc < ne; jc += CH) {
                int j = jc + threadIdx.x;
                __syncthreads();
                if (j < ne) {
                    float4 s = surf[j];
                    s_q[threadIdx.x] = {alpha * (T)s.x, alpha * (T)s.y, alpha * (T)s.z, Q[(size_t)a * npad + j]};
                }
                __syncthreads();
                const int cnt = min(CH, ne - jc);
                for (int k = g; g < G && k < cnt; k += G) {
                    V s = s_q[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact<T, YUK, false, DN, false>(rx[u] - s.x, ry[u] - s.y, rz[u] - s.z, s.w, 0, 0, 0,
                                                           nx[u], ny[u], nz[u], kappa, pot[u], dn[u]);
                }
            }
        }
        // combine the G partial sums of each target
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            s_red[0][u * CH + threadIdx.x] = pot[u];
            if (DN) s_red[DN ? 1 : 0][u * CH + threadIdx.x] = dn[u];
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                T sp = 0, sd = 0;
                for (int q = 0; q < G; ++q) {
                    sp += s_red[0][u * CH + tloc + q * slots];
                    if (DN) sd += s_red[DN ? 1 : 0][u * CH + tloc + q * slots];
                }
                if (vt[u]) {
                    pot_out[ti[u]] = sp * T(kInv4PiD);
                    if (DN) dn_out[ti[u]] = sd * T(kInv4PiD);
                }
            }
        }
    }
}

// Position in a U list taken in the order "the leaf itself first, then the
// others in list order" (selfpos = the leaf's index in the list, or -1).
__device__ __forceinline__ int u_at(int vi, int selfpos) {
    return selfpos < 0 ? vi : (vi == 0 ? selfpos : (vi <= selfpos ? vi - 1 : vi));
}

// Copies the next window (at most CAP points) of the concatenated sources of
// the U-list boxes into s_q (and s_m if WITH_M), advancing the cursor
// (vi = box in self-first order, off = points of that box already staged).
// Returns the number of points staged; the caller synchronises the CTA.
template <typename V, bool WITH_M, int CAP>
__device__ __forceinline__ int stage_near(V* s_q, V* s_m, const V* __restrict__ sq, const V* __restrict__ sm,
                                          const int* __restrict__ ul, int nu, int selfpos,
                                          const int* __restrict__ sb, const int* __restrict__ se, int& vi,
                                          int& off) {
    int filled = 0;
    while (filled < CAP && vi < nu) {
        const int a = ul[u_at(vi, selfpos)];
        const int j0 = sb[a] + off, len = se[a] - j0;
        const int take = min(len, CAP - filled);
        for (int e = threadIdx.x; e < take; e += blockDim.x) {
            cp_async_v(s_q + filled + e, sq + j0 + e);
            if (WITH_M) cp_async_v(s_m + filled + e, sm + j0 + e);
        }
        filled += take;
        if (take == len) { ++vi; off = 0; } else off += take;
    }
    cp_async_wait_all();
    return filled;
}

// Leaf evaluation of the paired apply (Laplace and Yukawa sums of every pair
// taken together), one 128-thread CTA per target leaf.  Targets: NT per
// thread in slots = ceil(n_t / NT) threads; the CTA holds G = 128 / slots
// groups of slots threads.  Sources: the leaf's whole near field (the
// U-list boxes, the leaf itself first, concatenated) is staged in windows
// of CAP points with asynchronous copies, then the far field (W-list upward
// and the leaf's own downward equivalent surfaces) in windows of generated
// points; group g takes the points g, g + G, g + 2G, ... of a window, so
// the lanes of a warp read neighbouring points (no bank conflicts) and
// every group has the same count to within one.  Only the leaf's own box
// can hold a coincident pair (equal points share a Morton key), so only its
// points take the r = 0 guard.  The G partial sums of each target are
// added in a fixed order at the end.
// PART 0: everything; 1: the near field (P2P) only, writing the outputs;
// 2: the far field (M2P, L2P) only, adding to the outputs of a PART 1 launch.
template <typename T, bool DL, bool DN, int NT, int PART>
__global__ void __launch_bounds__(128) k_leaf_pair(const int* __restrict__ leaves, int nleaf,
                                                   const int* __restrict__ tb, const int* __restrict__ te,
                                                   const int* __restrict__ sb, const int* __restrict__ se,
                                                   const int* __restrict__ U_off, const int* __restrict__ U_ids,
                                                   const int* __restrict__ W_off, const int* __restrict__ W_ids,
                                                   const int* __restrict__ level, const double4* __restrict__ center,
                                                   const float4* __restrict__ tpos,
                                                   const typename V4<T>::type* __restrict__ tn,
                                                   const typename V4<T>::type* __restrict__ sq,
                                                   const typename V4<T>::type* __restrict__ sm,
                                                   const T* __restrict__ QuL, const T* __restrict__ QdL,
                                                   const T* __restrict__ QuY, const T* __restrict__ QdY,
                                                   const float4* __restrict__ surf, int ne, int npad, T kappa,
                                                   T* __restrict__ potL_out, T* __restrict__ potY_out,
                                                   T* __restrict__ dnL_out, T* __restrict__ dnY_out) {
    using V = typename V4<T>::type;
    constexpr int CH = 128;
    constexpr int CAP = 16384 / (int)sizeof(V);     // points per window: 16 KB per array
    constexpr int NR = DN ? 4 : 2;
    static_assert(NR * NT * CH * (int)sizeof(T) <= CAP * (int)sizeof(V), "reduction fits the staging buffer");
    __shared__ __align__(16) V s_q[CAP];
    __shared__ __align__(16) V s_m[CAP];
    __shared__ int s_self;
    T* s_red = reinterpret_cast<T*>(s_q);            // [NR][NT * CH], after the last window
    T* s_qy = reinterpret_cast<T*>(s_m);             // far windows: the Yukawa densities
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    const int b = leaves[li];
    const int t0 = tb[b], t1 = te[b];
    const int slots = min(CH, max(4, (t1 - t0 + NT - 1) / NT));
    const int G = CH / slots;
    const int tloc = threadIdx.x % slots, g = threadIdx.x / slots;
    const bool active = g < G;
    const int* ul = U_ids + U_off[b];
    const int nu = U_off[b + 1] - U_off[b];
    const int nw = W_off[b + 1] - W_off[b];
    const int nsrcbox = nw + (level[b] >= 2 ? 1 : 0);
    const int nf = nsrcbox * ne;
    const double4 cb = center[b];
    const T kl2 = -kappa * T(kLog2E);
    if (threadIdx.x == 0) s_self = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < nu; i += CH)
        if (ul[i] == b) s_self = i;
    __syncthreads();
    const int selfpos = s_self;
    const int nself = selfpos >= 0 ? se[b] - sb[b] : 0;
    for (int tc = t0; tc < t1; tc += NT * slots) {
        int ti[NT];
        bool vt[NT];
        T xt[NT], yt[NT], zt[NT];
        T nx[NT], ny[NT], nz[NT], pL[NT], pY[NT], dL[NT], dY[NT];
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            ti[u] = tc + tloc + u * slots;
            vt[u] = ti[u] < t1;
            const float4 x = vt[u] ? tpos[ti[u]] : make_float4(0, 0, 0, 0);
            xt[u] = x.x; yt[u] = x.y; zt[u] = x.z;
            nx[u] = ny[u] = nz[u] = T(0);
            if (DN && vt[u]) { V nn = tn[ti[u]]; nx[u] = nn.x; ny[u] = nn.y; nz[u] = nn.z; }
            pL[u] = pY[u] = dL[u] = dY[u] = T(0);
        }
        // P2P over the staged windows of the near field
        if (PART != 2) {
            int vi = 0, off = 0;
            while (vi < nu) {
                const int self_left = (selfpos >= 0 && vi == 0) ? nself - off : 0;
                const int n = stage_near<V, true, CAP>(s_q, s_m, sq, sm, ul, nu, selfpos, sb, se, vi, off);   // sm.w: Yukawa monopole
                __syncthreads();
                const int selfhi = min(self_left, n);
                int k = g;
                for (; active && k < selfhi; k += G) {
                    const V s = s_q[k], mm = s_m[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_pair<T, DL, DN, true>(xt[u] - s.x, yt[u] - s.y, zt[u] - s.z, s.w, mm.w, mm.x, mm.y,
                                                       mm.z, nx[u], ny[u], nz[u], kappa, kl2, pL[u], pY[u], dL[u],
                                                       dY[u]);
                }
#pragma unroll 4
                for (; active && k < n; k += G) {
                    const V s = s_q[k], mm = s_m[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_pair<T, DL, DN, false>(xt[u] - s.x, yt[u] - s.y, zt[u] - s.z, s.w, mm.w, mm.x,
                                                        mm.y, mm.z, nx[u], ny[u], nz[u], kappa, kl2, pL[u], pY[u],
                                                        dL[u], dY[u]);
                }
                __syncthreads();
            }
        }
        // M2P (W list, upward equivalents) and L2P (own downward equivalent),
        // in coordinates relative to the leaf's centre
        if (PART != 1 && nf > 0) {
            T rx[NT], ry[NT], rz[NT];
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                rx[u] = (T)((double)xt[u] - cb.x);
                ry[u] = (T)((double)yt[u] - cb.y);
                rz[u] = (T)((double)zt[u] - cb.z);
            }
            for (int w0 = 0; w0 < nf; w0 += CAP) {
                const int n = min(CAP, nf - w0);
                for (int e = threadIdx.x; e < n; e += CH) {
                    const int v = w0 + e, i = v / ne, j = v - i * ne;
                    const bool isw = i < nw;
                    const int a = isw ? W_ids[W_off[b] + i] : b;
                    const double4 ca = center[a];
                    const T alpha = T(isw ? kAlphaInner : kAlphaOuter) * (T)ca.w;
                    const float4 s = surf[j];
                    const size_t o = (size_t)a * npad + j;
                    V w;
                    w.x = (T)(ca.x - cb.x) + alpha * (T)s.x;
                    w.y = (T)(ca.y - cb.y) + alpha * (T)s.y;
                    w.z = (T)(ca.z - cb.z) + alpha * (T)s.z;
                    w.w = isw ? QuL[o] : QdL[o];
                    s_q[e] = w;
                    s_qy[e] = isw ? QuY[o] : QdY[o];
                }
                __syncthreads();
#pragma unroll 4
                for (int k = g; active && k < n; k += G) {
                    const V s = s_q[k];
                    const T qy = s_qy[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_pair<T, false, DN, false>(rx[u] - s.x, ry[u] - s.y, rz[u] - s.z, s.w, qy, 0, 0, 0,
                                                           nx[u], ny[u], nz[u], kappa, kl2, pL[u], pY[u], dL[u],
                                                           dY[u]);
                }
                __syncthreads();
            }
        }
        // combine the G partial sums of each target (the staging buffer is free)
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            s_red[(0 * NT + u) * CH + threadIdx.x] = pL[u];
            s_red[(1 * NT + u) * CH + threadIdx.x] = pY[u];
            if (DN) {
                s_red[((NR - 2) * NT + u) * CH + threadIdx.x] = dL[u];
                s_red[((NR - 1) * NT + u) * CH + threadIdx.x] = dY[u];
            }
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                for (int q = 0; q < G; ++q) {
                    const int o = u * CH + tloc + q * slots;
                    a0 += s_red[0 * NT * CH + o];
                    a1 += s_red[1 * NT * CH + o];
                    if (DN) { a2 += s_red[(NR - 2) * NT * CH + o]; a3 += s_red[(NR - 1) * NT * CH + o]; }
                }
                if (vt[u]) {
                    if (PART == 2) {          // after the near-field launch (each target has one thread)
                        potL_out[ti[u]] += a0 * T(kInv4PiD);
                        potY_out[ti[u]] += a1 * T(kInv4PiD);
                        if (DN) {
                            dnL_out[ti[u]] += a2 * T(kInv4PiD);
                            dnY_out[ti[u]] += a3 * T(kInv4PiD);
                        }
                    } else {
                        potL_out[ti[u]] = a0 * T(kInv4PiD);
                        potY_out[ti[u]] = a1 * T(kInv4PiD);
                        if (DN) {
                            dnL_out[ti[u]] = a2 * T(kInv4PiD);
                            dnY_out[ti[u]] = a3 * T(kInv4PiD);
                        }
                    }
                }
            }
        }
        __syncthreads();              // s_red is the next chunk's staging buffer
    }
}

// ---- packed FP32: two sources per instruction
// add / sub / mul / fma .rn.f32x2 on 64-bit register pairs {lo, hi}: one
// issue slot for two lanes' worth of FP32 work (the FMA pipe time is the
// same as two scalar instructions; the freed issue slots take the MUFU,
// shared-memory and loop instructions of an issue-bound kernel).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
    f32x2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float x2_lo(f32x2 a) {
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a));
    return l;
}
__device__ __forceinline__ float x2_hi(f32x2 a) {
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a));
    return h;
}
template <bool GUARD>
__device__ __forceinline__ f32x2 x2_rsqrt(f32x2 a) {
    const float l = x2_lo(a), h = x2_hi(a);
    if (GUARD) return x2_pack(l > 0.f ? rsqrt_t<float>(l) : 0.f, h > 0.f ? rsqrt_t<float>(h) : 0.f);
    return x2_pack(rsqrt_t<float>(l), rsqrt_t<float>(h));
}
__device__ __forceinline__ f32x2 x2_exp2(f32x2 a) { return x2_pack(exp2_t<float>(x2_lo(a)), exp2_t<float>(x2_hi(a))); }

// interact_pair for one target (coordinates in both halves) and two sources
// (one per half), the same grouping of the arithmetic.  Source pair layout:
// A = {x, y}, B = {z, qL}, C = {mx, my}, D = {mz, qY}, each a pair.
// KM: 3 both kernels; 1 Laplace only (density qL, sum pL); 2 Yukawa only
// (density in the qL slot, sum pY).
template <bool DL, bool GUARD, int KM = 3>
__device__ __forceinline__ void interact_x2(f32x2 X, f32x2 Y, f32x2 Z, const ulonglong2& A, const ulonglong2& B,
                                            const ulonglong2& C, const ulonglong2& D, f32x2 kap, f32x2 kl2,
                                            f32x2 one, f32x2& pL, f32x2& pY) {
    const f32x2 dx = x2_sub(X, A.x), dy = x2_sub(Y, A.y), dz = x2_sub(Z, B.x);
    const f32x2 r2 = x2_fma(dx, dx, x2_fma(dy, dy, x2_mul(dz, dz)));
    const f32x2 rinv = x2_rsqrt<GUARD>(r2);
    if (KM == 1) {
        if (DL) {
            const f32x2 w = x2_mul(x2_fma(dx, C.x, x2_fma(dy, C.y, x2_mul(dz, D.x))), x2_mul(rinv, rinv));
            pL = x2_fma(rinv, x2_add(w, B.y), pL);
        } else {
            pL = x2_fma(rinv, B.y, pL);
        }
        return;
    }
    const f32x2 r = x2_mul(r2, rinv);
    const f32x2 er = x2_mul(x2_exp2(x2_mul(kl2, r)), rinv);        // e^{-kr} / r
    if (DL) {
        const f32x2 rinv2 = x2_mul(rinv, rinv);
        const f32x2 u = x2_fma(kap, r, one);
        const f32x2 w = x2_mul(x2_fma(dx, C.x, x2_fma(dy, C.y, x2_mul(dz, D.x))), rinv2);
        if (KM == 3) pL = x2_fma(rinv, x2_add(w, B.y), pL);
        pY = x2_fma(er, x2_fma(w, u, KM == 3 ? D.y : B.y), pY);
    } else {
        if (KM == 3) pL = x2_fma(rinv, B.y, pL);
        pY = x2_fma(er, KM == 3 ? D.y : B.y, pY);
    }
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Copies source j (sq = {x, y, z, qL}, sm = {mx, my, mz, qY}) into half
// e & 1 of pair slot e >> 1 of the packed window with 4-byte asynchronous
// copies (the dipole only if DL, the Yukawa monopole only if QY).
template <bool DL, bool QY = true>
__device__ __forceinline__ void copy_src_x2(ulonglong2* sA, ulonglong2* sB, ulonglong2* sC, ulonglong2* sD, int e,
                                            const float4* __restrict__ sq, const float4* __restrict__ sm,
                                            int j) {
    const int p = e >> 1, h = e & 1;
    float* a = reinterpret_cast<float*>(sA + p);
    float* b = reinterpret_cast<float*>(sB + p);
    float* c = reinterpret_cast<float*>(sC + p);
    float* d = reinterpret_cast<float*>(sD + p);
    const float* q = reinterpret_cast<const float*>(sq + j);
    const float* m = reinterpret_cast<const float*>(sm + j);
    cp_async4(a + h, q);
    cp_async4(a + 2 + h, q + 1);
    cp_async4(b + h, q + 2);
    cp_async4(b + 2 + h, q + 3);
    if (DL) {
        cp_async4(c + h, m);
        cp_async4(c + 2 + h, m + 1);
        cp_async4(d + h, m + 2);
    }
    if (QY) cp_async4(d + 2 + h, m + 3);
}

// Writes one source (or equivalent point) into half h of pair slot p of the
// packed window (A..D as above).
__device__ __forceinline__ void put_src_x2(ulonglong2* sA, ulonglong2* sB, ulonglong2* sC, ulonglong2* sD, int e,
                                           float x, float y, float z, float qL, float mx, float my, float mz,
                                           float qY) {
    const int p = e >> 1, h = e & 1;
    float* a = reinterpret_cast<float*>(sA + p);
    float* b = reinterpret_cast<float*>(sB + p);
    float* c = reinterpret_cast<float*>(sC + p);
    float* d = reinterpret_cast<float*>(sD + p);
    a[h] = x; a[2 + h] = y;
    b[h] = z; b[2 + h] = qL;
    c[h] = mx; c[2 + h] = my;
    d[h] = mz; d[2 + h] = qY;
}

// The paired leaf kernel in packed FP32 (no target-normal derivatives): the
// work split of k_leaf_pair (NT targets per thread, G groups, the near field
// in windows of the concatenated U-list sources, the leaf itself first, then
// the far field in windows of generated equivalent points), with each window
// stored as pairs of points, every value pair one 64-bit half of a 16-byte
// vector, so that group g takes the pairs g, g + G, ... and one packed
// instruction serves two sources.  An odd window is padded with a point of
// zero weight 1e10 away (its terms are exactly 0).
template <bool DL, int NT, int PART, int KM = 3>
__global__ void __launch_bounds__(128, 5) k_leaf_pair_x2(const int* __restrict__ leaves, int nleaf,
                                                      const int* __restrict__ tb, const int* __restrict__ te,
                                                      const int* __restrict__ sb, const int* __restrict__ se,
                                                      const int* __restrict__ U_off, const int* __restrict__ U_ids,
                                                      const int* __restrict__ W_off, const int* __restrict__ W_ids,
                                                      const int* __restrict__ level,
                                                      const double4* __restrict__ center,
                                                      const float4* __restrict__ tpos, const float4* __restrict__ sq,
                                                      const float4* __restrict__ sm, const float* __restrict__ QuL,
                                                      const float* __restrict__ QdL, const float* __restrict__ QuY,
                                                      const float* __restrict__ QdY, const float4* __restrict__ surf,
                                                      int ne, int npad, float kappa, float* __restrict__ potL_out,
                                                      float* __restrict__ potY_out, const int* __restrict__ Xl,
                                                      const int* __restrict__ Xn, int thrW, int thrX) {
    constexpr int CH = 128;
    constexpr int CAP = 1024;                    // points per window (512 pairs, 32 KB)
    constexpr int CP = CAP / 2;
    static_assert(2 * NT * CH * 4 <= CP * 16, "reduction fits one staging array");
    __shared__ ulonglong2 sA[CP], sB[CP], sC[CP], sD[CP];
    __shared__ int s_self;
    constexpr int VC = 256;                      // near-list entries resolved per chunk
    constexpr int FC = CH;                       // far candidates resolved per chunk
    constexpr int kSkip = INT_MIN;               // far candidate evaluated directly instead
    __shared__ int s_vb[VC], s_vn[VC];           // near entry: first source, sources taken (0: none)
    __shared__ float4 s_fb[FC];                  // far candidate: centre - the leaf's centre, radius
    __shared__ int s_fc[FC];                     // box id (W list), -1 - id (own downward) or kSkip
    __shared__ int s_sel[CH];                    // far window: the candidates it takes
    __shared__ int s_nb, s_fcur;
    float* s_red = reinterpret_cast<float*>(sA);
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    const int b = leaves[li];
    const int t0 = tb[b], t1 = te[b];
    const int slots = min(CH, max(4, (t1 - t0 + NT - 1) / NT));
    const int G = CH / slots;
    const int tloc = threadIdx.x % slots, g = threadIdx.x / slots;
    const bool active = g < G;
    const int* ul = U_ids + U_off[b];
    const int nu = U_off[b + 1] - U_off[b];
    const int nw = W_off[b + 1] - W_off[b];
    const int nsrcbox = nw + (level[b] >= 2 ? 1 : 0);
    // near stream: U list, then the W boxes of at most thrW sources, then the
    // X list when the leaf has at most thrX targets (thr < 0: none)
    const int nxd = (thrX >= 0 && t1 - t0 <= thrX) ? Xn[b] : 0;
    const int nvirt = nu + (thrW >= 0 ? nw : 0) + nxd;
    const int* xl = Xl + (long long)b * kXCap;
    const double4 cb = center[b];
    const float kl2s = -kappa * float(kLog2E);
    const f32x2 kap = x2_pack(kappa, kappa), kl2 = x2_pack(kl2s, kl2s), one = x2_pack(1.f, 1.f);
    if (threadIdx.x == 0) s_self = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < nu; i += CH)
        if (ul[i] == b) s_self = i;
    __syncthreads();
    const int selfpos = s_self;
    const int nself = selfpos >= 0 ? se[b] - sb[b] : 0;
    // list entries resolved in parallel into shared memory (one round of
    // dependent loads per chunk instead of one per box in the cursor loops)
    auto load_near = [&](int v0) {
        for (int v = v0 + threadIdx.x; v < min(nvirt, v0 + VC); v += CH) {
            int a;
            bool inc = true;
            if (v < nu) {
                a = ul[u_at(v, selfpos)];
            } else if (thrW >= 0 && v < nu + nw) {
                a = W_ids[W_off[b] + (v - nu)];
                inc = se[a] - sb[a] <= thrW;
            } else {
                a = xl[v - nu - (thrW >= 0 ? nw : 0)];
            }
            s_vb[v - v0] = sb[a];
            s_vn[v - v0] = inc ? se[a] - sb[a] : 0;
        }
    };
    auto load_far = [&](int f0) {
        for (int i = f0 + threadIdx.x; i < min(nsrcbox, f0 + FC); i += CH) {
            int code = -1 - b;
            if (i < nw) {
                const int a = W_ids[W_off[b] + i];
                code = (thrW < 0 || se[a] - sb[a] > thrW) ? a : kSkip;
            }
            if (code != kSkip) {
                const bool isw = code >= 0;
                const double4 ca = center[isw ? code : -1 - code];
                s_fb[i - f0] = make_float4((float)(ca.x - cb.x), (float)(ca.y - cb.y), (float)(ca.z - cb.z),
                                           float(isw ? kAlphaInner : kAlphaOuter) * (float)ca.w);
            }
            s_fc[i - f0] = code;
        }
    };
    int vbase = 0, fbase = 0;
    load_near(0);
    load_far(0);
    __syncthreads();
    for (int tc = t0; tc < t1; tc += NT * slots) {
        if (vbase != 0 || fbase != 0) {          // a later target chunk: the first list chunks again
            __syncthreads();
            vbase = fbase = 0;
            load_near(0);
            load_far(0);
            __syncthreads();
        }
        int ti[NT];
        bool vt[NT];
        f32x2 X[NT], Y[NT], Z[NT], pL[NT], pY[NT];
        float xs[NT], ys[NT], zs[NT];
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            ti[u] = tc + tloc + u * slots;
            vt[u] = ti[u] < t1;
            const float4 x = vt[u] ? tpos[ti[u]] : make_float4(0, 0, 0, 0);
            xs[u] = x.x; ys[u] = x.y; zs[u] = x.z;
            X[u] = x2_pack(x.x, x.x); Y[u] = x2_pack(x.y, x.y); Z[u] = x2_pack(x.z, x.z);
            pL[u] = pY[u] = 0ull;
        }
        if (PART != 2) {
            int vi = 0, off = 0;
            while (vi < nvirt) {
                const int self_left = (selfpos >= 0 && vi == 0) ? nself - off : 0;
                int filled = 0;
                while (filled < CAP && vi < nvirt) {
                    if (vi >= vbase + VC) {      // next chunk of resolved entries
                        __syncthreads();
                        vbase += VC;
                        load_near(vbase);
                        __syncthreads();
                    }
                    const int j0 = s_vb[vi - vbase] + off, len = s_vn[vi - vbase] - off;
                    const int take = min(len, CAP - filled);
                    for (int e = threadIdx.x; e < take; e += CH)
                        copy_src_x2<DL, KM == 3>(sA, sB, sC, sD, filled + e, sq, sm, j0 + e);
                    filled += take;
                    if (take == len) { ++vi; off = 0; } else off += take;
                }
                if ((filled & 1) && threadIdx.x == 0)
                    put_src_x2(sA, sB, sC, sD, filled, 1e10f, 1e10f, 1e10f, 0.f, 0.f, 0.f, 0.f, 0.f);
                cp_async_wait_all();
                __syncthreads();
                const int np = (filled + 1) >> 1;
                const int selfp = (min(self_left, filled) + 1) >> 1;      // pairs holding a point of the leaf
                int k = g;
                for (; active && k < selfp; k += G) {
                    const ulonglong2 A = sA[k], B = sB[k], C = DL ? sC[k] : make_ulonglong2(0, 0), D = sD[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_x2<DL, true, KM>(X[u], Y[u], Z[u], A, B, C, D, kap, kl2, one, pL[u], pY[u]);
                }
#pragma unroll 2
                for (; active && k < np; k += G) {
                    const ulonglong2 A = sA[k], B = sB[k], C = DL ? sC[k] : make_ulonglong2(0, 0), D = sD[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_x2<DL, false, KM>(X[u], Y[u], Z[u], A, B, C, D, kap, kl2, one, pL[u], pY[u]);
                }
                __syncthreads();
            }
        }
        if (PART != 1 && nsrcbox > 0) {
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                const float rx = (float)((double)xs[u] - cb.x), ry = (float)((double)ys[u] - cb.y),
                            rz = (float)((double)zs[u] - cb.z);
                X[u] = x2_pack(rx, rx); Y[u] = x2_pack(ry, ry); Z[u] = x2_pack(rz, rz);
            }
            const int nbw = CAP / ne;                    // whole boxes per window (ne <= CAP: host)
            int fcur = 0;                                // next far candidate: W list, then the leaf's own
            while (fcur < nsrcbox) {
                if (fcur >= fbase + FC) {                // next chunk of resolved candidates
                    __syncthreads();
                    fbase += FC;
                    load_far(fbase);
                    __syncthreads();
                }
                // warp 0 picks the window's boxes: up to nbw candidates of this
                // chunk that are not evaluated directly
                if (threadIdx.x < 32) {
                    const int lane = threadIdx.x;
                    const int cend = min(nsrcbox, fbase + FC);
                    int nb = 0, c = fcur;
                    while (nb < nbw && c < cend) {
                        const int i = c + lane;
                        const bool ok = i < cend && s_fc[i - fbase] != kSkip;
                        const unsigned m = __ballot_sync(0xffffffffu, ok);
                        const int rank = __popc(m & ((1u << lane) - 1u));
                        const int want = nbw - nb, have = __popc(m);
                        if (ok && rank < want) s_sel[nb + rank] = i - fbase;
                        if (have <= want) {
                            nb += have;
                            c = min(c + 32, cend);
                        } else {
                            const unsigned last = __ballot_sync(0xffffffffu, ok && rank == want - 1);
                            c += __ffs(last);            // one past the last box taken
                            nb += want;
                        }
                    }
                    if (lane == 0) { s_nb = nb; s_fcur = c; }
                }
                __syncthreads();
                const int nb = s_nb, n = nb * ne;
                fcur = s_fcur;
                for (int i = 0; i < nb; ++i) {
                    const int slot = s_sel[i];
                    const float4 bx = s_fb[slot];
                    const int code = s_fc[slot];
                    const bool isw = code >= 0;
                    const size_t base = (size_t)(isw ? code : -1 - code) * npad;
                    const float* QL = isw ? QuL : QdL;
                    const float* QY = isw ? QuY : QdY;
                    for (int j = threadIdx.x; j < ne; j += CH) {
                        const float4 sf = surf[j];
                        put_src_x2(sA, sB, sC, sD, i * ne + j, bx.x + bx.w * sf.x, bx.y + bx.w * sf.y,
                                   bx.z + bx.w * sf.z, QL[base + j], 0.f, 0.f, 0.f, KM == 3 ? QY[base + j] : 0.f);
                    }
                }
                if ((n & 1) && threadIdx.x == 0)
                    put_src_x2(sA, sB, sC, sD, n, 1e10f, 1e10f, 1e10f, 0.f, 0.f, 0.f, 0.f, 0.f);
                __syncthreads();
                const int np = (n + 1) >> 1;
                const ulonglong2 C0 = make_ulonglong2(0, 0);
#pragma unroll 2
                for (int k = g; active && k < np; k += G) {
                    const ulonglong2 A = sA[k], B = sB[k], D = sD[k];
#pragma unroll
                    for (int u = 0; u < NT; ++u)
                        interact_x2<false, false, KM>(X[u], Y[u], Z[u], A, B, C0, D, kap, kl2, one, pL[u], pY[u]);
                }
                __syncthreads();
            }
        }
        // combine: the two halves of each accumulator, then the G groups
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            s_red[u * CH + threadIdx.x] = x2_lo(pL[u]) + x2_hi(pL[u]);
            s_red[(NT + u) * CH + threadIdx.x] = x2_lo(pY[u]) + x2_hi(pY[u]);
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int u = 0; u < NT; ++u) {
                float a0 = 0.f, a1 = 0.f;
                for (int q = 0; q < G; ++q) {
                    a0 += s_red[u * CH + tloc + q * slots];
                    a1 += s_red[(NT + u) * CH + tloc + q * slots];
                }
                if (vt[u]) {
                    if (PART == 2) {
                        if (KM & 1) potL_out[ti[u]] += a0 * float(kInv4PiD);
                        if (KM & 2) potY_out[ti[u]] += a1 * float(kInv4PiD);
                    } else {
                        if (KM & 1) potL_out[ti[u]] = a0 * float(kInv4PiD);
                        if (KM & 2) potY_out[ti[u]] = a1 * float(kInv4PiD);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// P2M / P2L of the paired apply in packed FP32 (two sources per
// instruction), for the FP32 path.  One 128-thread CTA per box: NP check
// points per thread in slots = ceil(ne / NP) threads, G = 128 / slots groups
// taking the source pairs g, g + G, ...  Coordinates relative to the box:
// with cf = the centre rounded to FP32, a source at s enters as s - cf (an
// FP32 difference of two nearby numbers, exact up to the rounding of the
// difference itself) and a check point as alpha u + (c - cf), so that no
// digit of the absolute coordinates is lost.  Windows of CAP sources (B's
// own for P2M, its X-list boxes' for P2L), odd windows padded with a point
// of zero weight 1e10 away.
template <bool DL, int NP>
__global__ void __launch_bounds__(128) k_p2check_pair_x2(int nbox, const int* __restrict__ boxes, int mode,
                                                         const double4* __restrict__ center,
                                                         const int* __restrict__ sb, const int* __restrict__ se,
                                                         const int* __restrict__ X, const int* __restrict__ X_n,
                                                         const float4* __restrict__ sq, const float4* __restrict__ sm,
                                                         const float4* __restrict__ surf, int ne, int npad,
                                                         float kappa, float* __restrict__ chkL,
                                                         float* __restrict__ chkY, const int* __restrict__ nchild,
                                                         const int* __restrict__ tb, const int* __restrict__ te,
                                                         int thrX) {
    constexpr int CH = 128;
    constexpr int CAP = 512;
    constexpr int CP = CAP / 2;
    static_assert(2 * NP * CH * 4 <= 4 * CP * 16, "reduction fits the staging arrays");
    __shared__ ulonglong2 sA[CP], sB[CP], sC[CP], sD[CP];
    float* s_red = reinterpret_cast<float*>(sA);     // [2][NP][CH], spans sA..sD
    const int bi = blockIdx.x;
    if (bi >= nbox) return;
    const int b = boxes[bi];
    if (mode == 1 && thrX >= 0 && nchild[b] == 0 && te[b] - tb[b] <= thrX) {
        // a leaf of at most thrX targets takes its X list directly in the leaf kernel
        for (int i = threadIdx.x; i < npad; i += CH) {
            chkL[(long long)b * npad + i] = 0.f;
            chkY[(long long)b * npad + i] = 0.f;
        }
        return;
    }
    const double4 c = center[b];
    const float cfx = (float)c.x, cfy = (float)c.y, cfz = (float)c.z;
    const float ox = (float)(c.x - (double)cfx), oy = (float)(c.y - (double)cfy), oz = (float)(c.z - (double)cfz);
    const float alpha = float(mode == 0 ? kAlphaOuter : kAlphaInner) * (float)c.w;
    const int slots = (ne + NP - 1) / NP;            // <= 128 (host)
    const int G = CH / slots;
    const int tloc = threadIdx.x % slots, g = threadIdx.x / slots;
    const bool active = g < G;
    const float kl2s = -kappa * float(kLog2E);
    const f32x2 kap = x2_pack(kappa, kappa), kl2 = x2_pack(kl2s, kl2s), one = x2_pack(1.f, 1.f);
    f32x2 PX[NP], PY[NP], PZ[NP], aL[NP], aY[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int i = tloc + m * slots;
        const float4 u = (i < ne) ? surf[i] : make_float4(0, 0, 0, 0);
        const float px = alpha * u.x + ox, py = alpha * u.y + oy, pz = alpha * u.z + oz;
        PX[m] = x2_pack(px, px); PY[m] = x2_pack(py, py); PZ[m] = x2_pack(pz, pz);
        aL[m] = aY[m] = 0ull;
    }
    const int nlist = (mode == 0) ? 1 : X_n[b];
    const int* xl = X + (long long)b * kXCap;
    int ui = 0, off = 0;
    while (ui < nlist) {
        int filled = 0;
        while (filled < CAP && ui < nlist) {
            const int a = (mode == 0) ? b : xl[ui];
            const int j0 = sb[a] + off, len = se[a] - j0;
            const int take = min(len, CAP - filled);
            for (int e = threadIdx.x; e < take; e += CH) {
                const float4 q = sq[j0 + e], m = sm[j0 + e];
                put_src_x2(sA, sB, sC, sD, filled + e, q.x - cfx, q.y - cfy, q.z - cfz, q.w, m.x, m.y, m.z, m.w);
            }
            filled += take;
            if (take == len) { ++ui; off = 0; } else off += take;
        }
        if ((filled & 1) && threadIdx.x == 0)
            put_src_x2(sA, sB, sC, sD, filled, 1e10f, 1e10f, 1e10f, 0.f, 0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int np = (filled + 1) >> 1;
#pragma unroll 2
        for (int k = g; active && k < np; k += G) {
            const ulonglong2 A = sA[k], B = sB[k], C = DL ? sC[k] : make_ulonglong2(0, 0), D = sD[k];
#pragma unroll
            for (int m = 0; m < NP; ++m)
                interact_x2<DL, false>(PX[m], PY[m], PZ[m], A, B, C, D, kap, kl2, one, aL[m], aY[m]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        s_red[m * CH + threadIdx.x] = x2_lo(aL[m]) + x2_hi(aL[m]);
        s_red[(NP + m) * CH + threadIdx.x] = x2_lo(aY[m]) + x2_hi(aY[m]);
    }
    __syncthreads();
    if (g == 0) {
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int i = tloc + m * slots;
            float sL = 0.f, sY = 0.f;
            for (int q = 0; q < G; ++q) {
                sL += s_red[m * CH + tloc + q * slots];
                sY += s_red[(NP + m) * CH + tloc + q * slots];
            }
            if (i < ne) {
                chkL[(long long)b * npad + i] = sL * float(kInv4PiD);
                chkY[(long long)b * npad + i] = sY * float(kInv4PiD);
            }
        }
    }
    for (int i = ne + threadIdx.x; i < npad; i += CH) {
        chkL[(long long)b * npad + i] = 0.f;
        chkY[(long long)b * npad + i] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <typename T>
struct Work {
    DBuf<typename V4<T>::type> sq, sm, tn;
    DBuf<T> Qu, Qd, chk, pot, dn;
    DBuf<T> tmp;          // FP32 path: intermediate of the factored check -> equivalent solves
};

template <typename T, typename TO, int NPAD>
static void gemm_launch(cudaStream_t st, int nblocks, const GemmArgs& a, const TO* ops, const T* X, T* Y) {
    if (nblocks <= 0) return;
    switch (a.mode) {
        case G_M2L:
        case G_PAIRS: k_m2l_simt<T, TO, NPAD><<<nblocks, 256, 0, st>>>(a, ops, X, Y); break;
        case G_M2M: k_m2m<T, TO, NPAD><<<nblocks, 256, 0, st>>>(a, ops, X, Y); break;
        case G_L2L: k_l2l<T, TO, NPAD><<<nblocks, 256, 0, st>>>(a, ops, X, Y); break;
        default: k_check2equiv<T, TO, NPAD><<<nblocks, 256, 0, st>>>(a, ops, X, Y); break;
    }
    PB_CHECK_LAUNCH();
}

template <typename T, typename TO>
static void gemm_dispatch(int npad, cudaStream_t st, int nblocks, const GemmArgs& a, const TO* ops, const T* X, T* Y) {
    switch (npad) {
        case 32: gemm_launch<T, TO, 32>(st, nblocks, a, ops, X, Y); break;
        case 64: gemm_launch<T, TO, 64>(st, nblocks, a, ops, X, Y); break;
        case 128: gemm_launch<T, TO, 128>(st, nblocks, a, ops, X, Y); break;
        case 160: gemm_launch<T, TO, 160>(st, nblocks, a, ops, X, Y); break;
        case 224: gemm_launch<T, TO, 224>(st, nblocks, a, ops, X, Y); break;
        case 320: gemm_launch<T, TO, 320>(st, nblocks, a, ops, X, Y); break;
        case 416: gemm_launch<T, TO, 416>(st, nblocks, a, ops, X, Y); break;
        case 512: gemm_launch<T, TO, 512>(st, nblocks, a, ops, X, Y); break;
        default: throw Error(PB_EINVAL, "unsupported expansion order");
    }
}

template <typename T, bool YUK, bool DL>
static void launch_p2check(cudaStream_t st, int nbox, const int* boxes, int mode, fmm_tree* Tr, Work<T>& W,
                           const Operators& O, T kappa, int thrX = -1) {
    if (nbox <= 0) return;
    const int* tb = Tr->same ? Tr->sb.p : Tr->tb.p;
    const int* te = Tr->same ? Tr->se.p : Tr->te.p;
    if (O.npad <= 256)
        k_p2check<T, YUK, DL, 1><<<nbox, O.npad, 0, st>>>(nbox, boxes, mode, Tr->center.p, Tr->sb.p, Tr->se.p,
                                                          Tr->X.p, Tr->X_n.p, W.sq.p, W.sm.p,
                                                          (const float4*)O.surf_f.p, O.ne, O.npad, kappa, W.chk.p,
                                                          Tr->nchild.p, tb, te, thrX);
    else       // two check points per thread, threads rounded up from n_pad / 2
        k_p2check<T, YUK, DL, 2><<<nbox, std::min(256, (O.npad / 2 + 31) / 32 * 32), 0, st>>>(
                                                       nbox, boxes, mode, Tr->center.p, Tr->sb.p, Tr->se.p, Tr->X.p,
                                                       Tr->X_n.p, W.sq.p, W.sm.p, (const float4*)O.surf_f.p, O.ne,
                                                       O.npad, kappa, W.chk.p, Tr->nchild.p, tb, te, thrX);
    PB_CHECK_LAUNCH();
}

// the two check -> equivalent conversions: the FP64 solve for the FP64
// path; for the FP32 path the factored solve Y = W2 (W1 X), two FP32
// passes through `tmp` (box-major like X and Y)
template <typename T>
static void check2equiv(const Operators& O, int level, bool up, cudaStream_t st, GemmArgs ga, int ncols,
                        const int* cols, const T* X, T* Y, T* tmp);
template <>
void check2equiv<float>(const Operators& O, int level, bool up, cudaStream_t st, GemmArgs ga, int ncols,
                        const int* cols, const float* X, float* Y, float* tmp) {
    ga.mode = G_DENSE; ga.ncols = ncols; ga.cols = cols; ga.col_base = 0; ga.level = level; ga.accumulate = 0;
    gemm_dispatch<float, float>(O.npad, st, div_up(ncols, kTC), ga, up ? O.uc2ue_w1.p : O.dc2de_w1.p, X, tmp);
    gemm_dispatch<float, float>(O.npad, st, div_up(ncols, kTC), ga, up ? O.uc2ue_w2.p : O.dc2de_w2.p, tmp, Y);
}
template <>
void check2equiv<double>(const Operators& O, int level, bool up, cudaStream_t st, GemmArgs ga, int ncols,
                         const int* cols, const double* X, double* Y, double*) {
    ga.mode = G_DENSE; ga.ncols = ncols; ga.cols = cols; ga.col_base = 0; ga.level = level; ga.accumulate = 0;
    gemm_dispatch<double, double>(O.npad, st, div_up(ncols, kTC), ga, up ? O.uc2ue_d.p : O.dc2de_d.p, X, Y);
}

template <typename T, bool YUK, bool DL, bool DN>
static void launch_leaf(cudaStream_t st, fmm_tree* Tr, Work<T>& W, const Operators& O, T kappa, int thrW = -1,
                        int thrX = -1) {
    if (Tr->n_tleaf <= 0) return;
    const float4* tpos = Tr->same ? Tr->pos_s.p : Tr->pos_t.p;
    const int* tb = Tr->same ? Tr->sb.p : Tr->tb.p;
    const int* te = Tr->same ? Tr->se.p : Tr->te.p;
    if constexpr (std::is_same<T, float>::value && !DN) {
        if (Tr->ctx->leaf_packed && O.ne <= 1024) {
            // the packed leaf kernel for one kernel (KM 1: Laplace, 2: Yukawa)
            constexpr int KM = YUK ? 2 : 1;
            const int NT = Tr->ctx->leaf_nt ? Tr->ctx->leaf_nt : 4;
            auto k = NT == 4 ? k_leaf_pair_x2<DL, 4, 0, KM> : k_leaf_pair_x2<DL, 2, 0, KM>;
            k<<<Tr->n_tleaf, 128, 0, st>>>(Tr->leaf_ids.p, Tr->n_tleaf, tb, te, Tr->sb.p, Tr->se.p, Tr->U_off.p,
                                           Tr->U_ids.p, Tr->W_off.p, Tr->W_ids.p, Tr->level.p, Tr->center.p, tpos,
                                           W.sq.p, W.sm.p, W.Qu.p, W.Qd.p, nullptr, nullptr,
                                           (const float4*)O.surf_f.p, O.ne, O.npad, kappa,
                                           YUK ? nullptr : W.pot.p, YUK ? W.pot.p : nullptr, Tr->X.p, Tr->X_n.p,
                                           thrW, thrX);
            PB_CHECK_LAUNCH();
            return;
        }
    }
    PB_REQUIRE(thrW < 0 && thrX < 0, PB_EINVAL, "direct W/X-list evaluation needs the packed leaf kernel");
    constexpr int NT = 2;     // 4 measured slower (register pressure)
    k_leaf_eval<T, YUK, DL, DN, NT><<<Tr->n_tleaf, 128, 0, st>>>(
        Tr->leaf_ids.p, Tr->n_tleaf, tb, te, Tr->sb.p, Tr->se.p, Tr->U_off.p, Tr->U_ids.p, Tr->W_off.p, Tr->W_ids.p,
        Tr->level.p, Tr->center.p, tpos, W.tn.p, W.sq.p, W.sm.p, W.Qu.p, W.Qd.p, (const float4*)O.surf_f.p, O.ne, O.npad, kappa,
        W.pot.p, W.dn.p);
    PB_CHECK_LAUNCH();
}

template <typename T>
static const T* opsel(const Operators& O, const DBuf<float>& f, const DBuf<double>& d);
template <>
const float* opsel<float>(const Operators&, const DBuf<float>& f, const DBuf<double>&) { return f.p; }
template <>
const double* opsel<double>(const Operators&, const DBuf<float>&, const DBuf<double>& d) { return d.p; }

// ---- far-field steps of one kernel (operators O, work W), shared by the
// single and the paired apply
template <typename T>
static GemmArgs tree_gemm_args(const fmm_tree* Tr) {
    GemmArgs ga{};
    ga.first_child = Tr->first_child.p;
    ga.nchild = Tr->nchild.p;
    ga.anchor = Tr->anchor.p;
    ga.parent = Tr->parent.p;
    return ga;
}

// UC2UE at every leaf with sources (upward check potentials in W.chk)
template <typename T>
static void far_uc2ue(fmm_tree* Tr, const Operators& O, Work<T>& W) {
    if constexpr (std::is_same<T, float>::value) {
        if (c2e_tc_launch(Tr, O, true, W.chk.p, W.Qu.p, W.tmp.p, Tr->ctx->dev_err, Tr->ctx->stream)) return;
    }
    GemmArgs ga = tree_gemm_args<T>(Tr);
    for (int l = 0; l < Tr->nlev; ++l) {
        int a0 = Tr->sleaf_lvl_off[l], a1 = Tr->sleaf_lvl_off[l + 1];
        if (a1 <= a0) continue;
        check2equiv<T>(O, l, true, Tr->ctx->stream, ga, a1 - a0, Tr->sleaf_ids.p + a0, W.chk.p, W.Qu.p, W.tmp.p);
    }
}

// M2M, post-order: parents at level l from children at level l + 1 (leaves
// of level l keep their P2M result: the kernels skip them)
template <typename T>
static void m2m_level(fmm_tree* Tr, const Operators& O, Work<T>& W, int l) {
    pb_ctx* ctx = Tr->ctx;
    cudaStream_t st = ctx->stream;
    if constexpr (std::is_same<T, float>::value) {
        if (!ctx->deterministic && pc_tc_launch(Tr, O, l + 1, true, W.Qu.p, ctx->dev_err, st)) return;
    }
    GemmArgs ga = tree_gemm_args<T>(Tr);
    int a0 = Tr->lvl_off[l], a1 = Tr->lvl_off[l + 1];
    ga.mode = G_M2M; ga.ncols = a1 - a0; ga.cols = nullptr; ga.col_base = a0; ga.level = l + 1;
    gemm_dispatch<T, T>(O.npad, st, div_up(a1 - a0, kTC), ga, opsel<T>(O, O.m2m, O.m2m_d), W.Qu.p, W.Qu.p);
}

template <typename T>
static void far_m2m(fmm_tree* Tr, const Operators& O, Work<T>& W) {
    for (int l = Tr->nlev - 2; l >= 2; --l) m2m_level(Tr, O, W, l);
}

// DC2DE at every X-list box (downward check potentials of P2L in W.chk);
// writes Qd of those boxes before the M2L accumulates
template <typename T>
static void far_dc2de_x(fmm_tree* Tr, const Operators& O, Work<T>& W, bool xfar = false) {
    if constexpr (std::is_same<T, float>::value) {
        if (c2e_tc_launch(Tr, O, false, W.chk.p, W.Qd.p, W.tmp.p, Tr->ctx->dev_err, Tr->ctx->stream, xfar)) return;
    }
    PB_REQUIRE(!xfar, PB_EINVAL, "reduced X-box list without the tensor-core solve");
    GemmArgs ga = tree_gemm_args<T>(Tr);
    for (int l = 0; l < Tr->nlev; ++l) {
        int a0 = Tr->xbox_lvl_off[l], a1 = Tr->xbox_lvl_off[l + 1];
        if (a1 <= a0) continue;
        check2equiv<T>(O, l, false, Tr->ctx->stream, ga, a1 - a0, Tr->xbox_ids.p + a0, W.chk.p, W.Qd.p, W.tmp.p);
    }
}

// M2L over the V lists with DC2DE folded into the operators: accumulate into Qd
template <typename T>
static void far_m2l(fmm_tree* Tr, const Operators& O, Work<T>& W) {
    pb_ctx* ctx = Tr->ctx;
    bool tc_done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (Tr->m2l_pairs.nitems > 0 && !ctx->deterministic)
            tc_done = m2l_tc_launch(Tr, O, W.Qu.p, W.Qd.p, ctx->dev_err, ctx->stream);
    }
    if (!tc_done && !ctx->deterministic && Tr->m2l_pairs.nitems32 > 0) {
        // one CTA per at most 32 V-list pairs of one (level, offset) group:
        // parallel over pairs, so small trees fill the GPU too
        GemmArgs ga = tree_gemm_args<T>(Tr);
        ga.mode = G_PAIRS;
        ga.pitems = Tr->m2l_pairs.items32.p;
        ga.ptgt = Tr->m2l_pairs.tgt.p;
        ga.psrc = Tr->m2l_pairs.src.p;
        gemm_dispatch<T, T>(O.npad, ctx->stream, Tr->m2l_pairs.nitems32, ga, opsel<T>(O, O.m2l, O.m2l_d), W.Qu.p,
                            W.Qd.p);
        tc_done = true;
    }
    if (!tc_done && Tr->m2l.ntile > 0) {
        GemmArgs ga = tree_gemm_args<T>(Tr);
        ga.mode = G_M2L;
        ga.tile_box = Tr->m2l.tile_box.p;
        ga.tile_level = Tr->m2l.tile_level.p;
        ga.entry_off = Tr->m2l.entry_off.p;
        ga.entry_oidx = Tr->m2l.entry_offset_idx.p;
        ga.entry_src = Tr->m2l.entry_src.p;
        gemm_dispatch<T, T>(O.npad, ctx->stream, Tr->m2l.ntile, ga, opsel<T>(O, O.m2l, O.m2l_d), W.Qu.p, W.Qd.p);
    }
}

// L2L, pre-order (DC2DE folded), from parents at level l - 1
template <typename T>
static void l2l_level(fmm_tree* Tr, const Operators& O, Work<T>& W, int l) {
    pb_ctx* ctx = Tr->ctx;
    cudaStream_t st = ctx->stream;
    if constexpr (std::is_same<T, float>::value) {
        if (!ctx->deterministic && pc_tc_launch(Tr, O, l, false, W.Qd.p, ctx->dev_err, st)) return;
    }
    GemmArgs ga = tree_gemm_args<T>(Tr);
    int p0 = Tr->lvl_off[l - 1], p1 = Tr->lvl_off[l];
    ga.mode = G_L2L; ga.ncols = p1 - p0; ga.cols = nullptr; ga.col_base = p0; ga.level = l;
    gemm_dispatch<T, T>(O.npad, st, div_up(p1 - p0, kTC), ga, opsel<T>(O, O.l2l, O.l2l_d), W.Qd.p, W.Qd.p);
}

template <typename T>
static void far_l2l(fmm_tree* Tr, const Operators& O, Work<T>& W) {
    for (int l = 3; l < Tr->nlev; ++l) l2l_level(Tr, O, W, l);
}

// ---- the far-field steps of the paired apply: both kernels in one
// tensor-core launch where that path applies, else one kernel after the other
template <typename T>
static void far_pair_c2e(fmm_tree* Tr, const Operators& OL, const Operators& OY, Work<T>& WL, Work<T>& WY, bool up,
                         bool xfar = false) {
    if constexpr (std::is_same<T, float>::value) {
        if (c2e_tc_launch2(Tr, OL, &OY, up, WL.chk.p, up ? WL.Qu.p : WL.Qd.p, WL.tmp.p, WY.chk.p,
                           up ? WY.Qu.p : WY.Qd.p, WY.tmp.p, Tr->ctx->dev_err, Tr->ctx->stream, xfar))
            return;
    }
    PB_REQUIRE(!xfar, PB_EINVAL, "reduced X-box list without the tensor-core solve");
    if (up) { far_uc2ue(Tr, OL, WL); far_uc2ue(Tr, OY, WY); }
    else { far_dc2de_x(Tr, OL, WL); far_dc2de_x(Tr, OY, WY); }
}

template <typename T>
static void far_pair_m2m(fmm_tree* Tr, const Operators& OL, const Operators& OY, Work<T>& WL, Work<T>& WY) {
    pb_ctx* ctx = Tr->ctx;
    for (int l = Tr->nlev - 2; l >= 2; --l) {
        if constexpr (std::is_same<T, float>::value) {
            if (!ctx->deterministic &&
                pc_tc_launch2(Tr, OL, &OY, l + 1, true, WL.Qu.p, WY.Qu.p, ctx->dev_err, ctx->stream))
                continue;
        }
        m2m_level(Tr, OL, WL, l);
        m2m_level(Tr, OY, WY, l);
    }
}

template <typename T>
static void far_pair_l2l(fmm_tree* Tr, const Operators& OL, const Operators& OY, Work<T>& WL, Work<T>& WY) {
    pb_ctx* ctx = Tr->ctx;
    for (int l = 3; l < Tr->nlev; ++l) {
        if constexpr (std::is_same<T, float>::value) {
            if (!ctx->deterministic &&
                pc_tc_launch2(Tr, OL, &OY, l, false, WL.Qd.p, WY.Qd.p, ctx->dev_err, ctx->stream))
                continue;
        }
        l2l_level(Tr, OL, WL, l);
        l2l_level(Tr, OY, WY, l);
    }
}

template <typename T>
static void far_pair_m2l(fmm_tree* Tr, const Operators& OL, const Operators& OY, Work<T>& WL, Work<T>& WY) {
    pb_ctx* ctx = Tr->ctx;
    if constexpr (std::is_same<T, float>::value) {
        if (Tr->m2l_pairs.nitems > 0 && !ctx->deterministic &&
            m2l_tc_launch2(Tr, OL, &OY, WL.Qu.p, WL.Qd.p, WY.Qu.p, WY.Qd.p, ctx->dev_err, ctx->stream))
            return;
    }
    far_m2l(Tr, OL, WL);
    far_m2l(Tr, OY, WY);
}

// equivalent densities and check potentials of one kernel
template <typename T>
static void alloc_far(Work<T>& W, size_t nbox_npad, cudaStream_t st) {
    W.Qu.alloc(nbox_npad, st);
    W.Qd.alloc(nbox_npad, st);
    W.chk.alloc(nbox_npad, st);
    W.Qu.zero(st);
    W.Qd.zero(st);
    W.chk.zero(st);
    if (std::is_same<T, float>::value) W.tmp.alloc(nbox_npad, st);
}

template <typename T, typename In, bool YUK>
static void apply_t(fmm_tree* Tr, const Operators& O, double kappa_d, const In* q, const In* dip, const In* src_n,
                    const In* tgt_n, In* out, In* out_dn) {
    cudaStream_t st = Tr->ctx->stream;
    const long long ns = Tr->ns, nt = Tr->same ? Tr->ns : Tr->nt;
    const T kappa = (T)kappa_d;
    const bool DL = dip != nullptr, DN = out_dn != nullptr;
    if (DL && DN) throw Error(PB_EINVAL, "double layer with target-normal derivative is not provided");
    // small W boxes and small leaves' X lists summed directly (see list_direct)
    const int ldm = Tr->ctx->list_direct;
    const bool ld = std::is_same<T, float>::value && !DN && Tr->ctx->leaf_packed && ldm != 0 && O.ne <= 1024;
    const int thrW = ld && ldm != 2 ? O.ne / 2 : -1, thrX = ld && ldm != 3 ? O.ne : -1;
    Work<T> W;
    W.sq.alloc(ns, st);
    if (DL) W.sm.alloc(ns, st);
    alloc_far(W, (size_t)Tr->nbox * O.npad, st);
    W.pot.alloc(nt, st);
    if (DN) { W.dn.alloc(nt, st); W.tn.alloc(nt, st); }
    pb_ctx* ctx = Tr->ctx;
    auto ph = std::make_unique<PhaseTimer>(ctx, PB_PH_GATHER);
    k_gather_src<T, In><<<div_up(ns, 256), 256, 0, st>>>(ns, Tr->perm_s.p, Tr->pos_s.p, q, dip, src_n, W.sq.p,
                                                          DL ? W.sm.p : nullptr);
    PB_CHECK_LAUNCH();
    if (DN) {
        const int* pt = Tr->same ? Tr->perm_s.p : Tr->perm_t.p;
        k_gather_tn<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, tgt_n, W.tn.p);
        PB_CHECK_LAUNCH();
    }
    const int nsl = Tr->sleaf_lvl_off[Tr->nlev];
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_P2M);
    // ---- upward pass: P2M at leaves with sources, then UC2UE per level
    if (DL) launch_p2check<T, YUK, true>(st, nsl, Tr->sleaf_ids.p, 0, Tr, W, O, kappa);
    else launch_p2check<T, YUK, false>(st, nsl, Tr->sleaf_ids.p, 0, Tr, W, O, kappa);
    far_uc2ue(Tr, O, W);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_M2M);
    far_m2m(Tr, O, W);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_P2L);
    // ---- far field into downward equivalent densities.
    // P2L: X-list sources -> downward check -> DC2DE, per level
    if (Tr->n_xbox > 0) {
        bool xfar = false;
        if constexpr (std::is_same<T, float>::value) xfar = thrX >= 0 && c2e_tc_ok(O);
        if (xfar) build_xbox_far(Tr, thrX);
        const int nx = xfar ? Tr->n_xfar : Tr->n_xbox;
        const int* xids = xfar ? Tr->xfar_ids.p : Tr->xbox_ids.p;
        if (DL) launch_p2check<T, YUK, true>(st, nx, xids, 1, Tr, W, O, kappa, thrX);
        else launch_p2check<T, YUK, false>(st, nx, xids, 1, Tr, W, O, kappa, thrX);
        far_dc2de_x(Tr, O, W, xfar);
    }
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_M2L);
    far_m2l(Tr, O, W);
    // ---- downward pass
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_DOWN);
    far_l2l(Tr, O, W);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_LEAF);
    // ---- leaves: P2P + M2P + L2P
    if (DL) launch_leaf<T, YUK, true, false>(st, Tr, W, O, kappa, thrW, thrX);
    else if (DN) launch_leaf<T, YUK, false, true>(st, Tr, W, O, kappa, thrW, thrX);
    else launch_leaf<T, YUK, false, false>(st, Tr, W, O, kappa, thrW, thrX);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_SCATTER);
    const int* pt = Tr->same ? Tr->perm_s.p : Tr->perm_t.p;
    k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, W.pot.p, out);
    PB_CHECK_LAUNCH();
    if (DN) k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, W.dn.p, out_dn);
    if (DN) PB_CHECK_LAUNCH();
    ph.reset();
}

// ---- paired apply: Laplace (operators OL) and Yukawa (OY) in one traversal
template <typename T, bool DL>
static void launch_p2check_pair(cudaStream_t st, int nbox, const int* boxes, int mode, fmm_tree* Tr, Work<T>& WL,
                                Work<T>& WY, const Operators& O, T kappa, int thrX = -1) {
    if (nbox <= 0) return;
    // P2L (the X-list sources of a box, often several hundred) in packed
    // groups; P2M (at most n_crit sources) keeps one thread per check point,
    // which measured faster for so little work per box
    if constexpr (std::is_same<T, float>::value) {
        if (Tr->ctx->leaf_packed && mode == 1) {
            // check points per thread: the choice that leaves the fewest lanes idle
            // (p = 4: 4 -> 9 groups of 14 threads; p = 6: 4 -> 3 x 38; p = 8: 8 -> 3 x 37; p = 10: 4 -> 1 x 122)
            int best = 0;
            double best_eff = 0.0;
            for (int np : {2, 4, 8}) {
                const int slots = (O.ne + np - 1) / np;
                if (slots > 128) continue;
                const int warps = (128 / slots * slots + 31) / 32;
                const double eff = double(O.ne) / (double(slots) * np) * (128 / slots) * slots / (32.0 * warps);
                if (eff > best_eff + 1e-9) { best_eff = eff; best = np; }
            }
            if (best) {
                auto k = best == 2 ? k_p2check_pair_x2<DL, 2>
                                   : (best == 4 ? k_p2check_pair_x2<DL, 4> : k_p2check_pair_x2<DL, 8>);
                k<<<nbox, 128, 0, st>>>(nbox, boxes, mode, Tr->center.p, Tr->sb.p, Tr->se.p, Tr->X.p, Tr->X_n.p,
                                        WL.sq.p, WL.sm.p, (const float4*)O.surf_f.p, O.ne, O.npad, kappa,
                                        WL.chk.p, WY.chk.p, Tr->nchild.p, Tr->same ? Tr->sb.p : Tr->tb.p,
                                        Tr->same ? Tr->se.p : Tr->te.p, thrX);
                PB_CHECK_LAUNCH();
                return;
            }
        }
    }
    PB_REQUIRE(thrX < 0, PB_EINVAL, "direct X-list evaluation needs the packed check-potential kernel");
    if (O.npad <= 256)
        k_p2check_pair<T, DL, 1><<<nbox, O.npad, 0, st>>>(nbox, boxes, mode, Tr->center.p, Tr->sb.p, Tr->se.p,
                                                          Tr->X.p, Tr->X_n.p, WL.sq.p, WL.sm.p,
                                                          (const float4*)O.surf_f.p, O.ne, O.npad, kappa, WL.chk.p,
                                                          WY.chk.p);
    else
        // two check points per thread, the threads rounded up from n_pad / 2
        // (p = 8: 160 threads for 296 points; a fixed 256 left 42% of the
        // slots idle: P2M 2.12 -> 1.63 ms at 4M)
        k_p2check_pair<T, DL, 2><<<nbox, std::min(256, (O.npad / 2 + 31) / 32 * 32), 0, st>>>(
                                                       nbox, boxes, mode, Tr->center.p, Tr->sb.p, Tr->se.p,
                                                       Tr->X.p, Tr->X_n.p, WL.sq.p, WL.sm.p,
                                                       (const float4*)O.surf_f.p, O.ne, O.npad, kappa, WL.chk.p,
                                                       WY.chk.p);
    PB_CHECK_LAUNCH();
}

template <typename T, bool DL, bool DN, int PART>
static void launch_leaf_pair(cudaStream_t st, fmm_tree* Tr, Work<T>& WL, Work<T>& WY, const Operators& O, T kappa,
                             int thrW = -1, int thrX = -1) {
    if (Tr->n_tleaf <= 0) return;
    const float4* tpos = Tr->same ? Tr->pos_s.p : Tr->pos_t.p;
    const int* tb = Tr->same ? Tr->sb.p : Tr->tb.p;
    const int* te = Tr->same ? Tr->se.p : Tr->te.p;
    const int nt_opt = Tr->ctx->leaf_nt;
    if constexpr (std::is_same<T, float>::value && !DN) {
        if (Tr->ctx->leaf_packed && O.ne <= 1024) {
            const int NT = nt_opt ? nt_opt : 4;
            auto k = NT == 4 ? k_leaf_pair_x2<DL, 4, PART> : k_leaf_pair_x2<DL, 2, PART>;
            k<<<Tr->n_tleaf, 128, 0, st>>>(Tr->leaf_ids.p, Tr->n_tleaf, tb, te, Tr->sb.p, Tr->se.p, Tr->U_off.p,
                                           Tr->U_ids.p, Tr->W_off.p, Tr->W_ids.p, Tr->level.p, Tr->center.p, tpos,
                                           WL.sq.p, WL.sm.p, WL.Qu.p, WL.Qd.p, WY.Qu.p, WY.Qd.p,
                                           (const float4*)O.surf_f.p, O.ne, O.npad, kappa, WL.pot.p, WY.pot.p,
                                           Tr->X.p, Tr->X_n.p, thrW, thrX);
            PB_CHECK_LAUNCH();
            return;
        }
    }
    PB_REQUIRE(thrW < 0 && thrX < 0, PB_EINVAL, "direct W/X-list evaluation needs the packed leaf kernel");
    const int NT = nt_opt ? nt_opt : (sizeof(T) == 4 ? 4 : 2);
    auto k = NT == 4 ? k_leaf_pair<T, DL, DN, 4, PART> : k_leaf_pair<T, DL, DN, 2, PART>;
    k<<<Tr->n_tleaf, 128, 0, st>>>(
        Tr->leaf_ids.p, Tr->n_tleaf, tb, te, Tr->sb.p, Tr->se.p, Tr->U_off.p, Tr->U_ids.p, Tr->W_off.p, Tr->W_ids.p,
        Tr->level.p, Tr->center.p, tpos, WL.tn.p, WL.sq.p, WL.sm.p, WL.Qu.p, WL.Qd.p, WY.Qu.p, WY.Qd.p,
        (const float4*)O.surf_f.p, O.ne, O.npad, kappa, WL.pot.p, WY.pot.p, WL.dn.p, WY.dn.p);
    PB_CHECK_LAUNCH();
}

// Adaptive-list pairs taken directly (exact) where that is less work than the
// equivalent surfaces (PB_OPT_LIST_DIRECT, FP32 packed kernels): a W-list box
// of at most n_e / 2 sources (M2P costs n_e monopole terms per target, a
// direct pair with a dipole about twice one of them), and the X list of a
// leaf of at most n_e targets (P2L would put the same sources on n_e check
// points).  Returns the two thresholds, -1 when off.
static void list_direct(const fmm_tree* Tr, const Operators& O, bool fp32, bool DN, int& thrW, int& thrX) {
    const int mode = Tr->ctx->list_direct;         // 0 off, 1 W and X, 2 X only, 3 W only
    const bool on = fp32 && !DN && Tr->ctx->leaf_packed && mode != 0 && O.ne <= 1024;
    thrW = on && mode != 2 ? O.ne / 2 : -1;
    thrX = on && mode != 3 ? O.ne : -1;
}

template <typename T, typename In>
static void apply_pair_t(fmm_tree* Tr, const Operators& OL, const Operators& OY, double kappa_d, const In* qL,
                         const In* qY, const In* dip, const In* src_n, const In* tgt_n, In* outL, In* outY,
                         In* dnL, In* dnY) {
    cudaStream_t st = Tr->ctx->stream;
    const long long ns = Tr->ns, nt = Tr->same ? Tr->ns : Tr->nt;
    const T kappa = (T)kappa_d;
    const bool DL = dip != nullptr, DN = dnL != nullptr;
    if (DL && DN) throw Error(PB_EINVAL, "double layer with target-normal derivative is not provided");
    int thrW, thrX;
    list_direct(Tr, OL, std::is_same<T, float>::value, DN, thrW, thrX);
    Work<T> WL, WY;
    WL.sq.alloc(ns, st);
    WL.sm.alloc(ns, st);
    alloc_far(WL, (size_t)Tr->nbox * OL.npad, st);
    alloc_far(WY, (size_t)Tr->nbox * OY.npad, st);
    WL.pot.alloc(nt, st);
    WY.pot.alloc(nt, st);
    if (DN) { WL.dn.alloc(nt, st); WY.dn.alloc(nt, st); WL.tn.alloc(nt, st); }
    pb_ctx* ctx = Tr->ctx;
    auto ph = std::make_unique<PhaseTimer>(ctx, PB_PH_GATHER);
    k_gather_pair<T, In><<<div_up(ns, 256), 256, 0, st>>>(ns, Tr->perm_s.p, Tr->pos_s.p, qL, qY, dip, src_n, WL.sq.p,
                                                           WL.sm.p);
    PB_CHECK_LAUNCH();
    if (DN) {
        const int* pt = Tr->same ? Tr->perm_s.p : Tr->perm_t.p;
        k_gather_tn<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, tgt_n, WL.tn.p);
        PB_CHECK_LAUNCH();
    }
    // the near field needs only the gathered sources: on the second stream,
    // beside the far-field passes below (joined before the far leaf part)
    const bool fork = ctx->aux && ctx->overlap && Tr->n_tleaf > 0;
    if (fork) {
        PB_CUDA(cudaEventRecord(ctx->ev_fork, st));
        PB_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        {
            PhaseTimer phn(ctx, PB_PH_LEAF, ctx->aux);
            if (DL) launch_leaf_pair<T, true, false, 1>(ctx->aux, Tr, WL, WY, OL, kappa, thrW, thrX);
            else if (DN) launch_leaf_pair<T, false, true, 1>(ctx->aux, Tr, WL, WY, OL, kappa, thrW, thrX);
            else launch_leaf_pair<T, false, false, 1>(ctx->aux, Tr, WL, WY, OL, kappa, thrW, thrX);
        }
        PB_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
    }
    const int nsl = Tr->sleaf_lvl_off[Tr->nlev];
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_P2M);
    if (DL) launch_p2check_pair<T, true>(st, nsl, Tr->sleaf_ids.p, 0, Tr, WL, WY, OL, kappa);
    else launch_p2check_pair<T, false>(st, nsl, Tr->sleaf_ids.p, 0, Tr, WL, WY, OL, kappa);
    far_pair_c2e(Tr, OL, OY, WL, WY, true);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_M2M);
    far_pair_m2m(Tr, OL, OY, WL, WY);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_P2L);
    if (Tr->n_xbox > 0) {
        // with the small leaves' X lists summed in the leaf kernel, P2L and its
        // solve run on the other X-list boxes only (tensor-core solve path)
        bool xfar = false;
        if constexpr (std::is_same<T, float>::value) xfar = thrX >= 0 && c2e_tc_ok(OL) && c2e_tc_ok(OY);
        if (xfar) build_xbox_far(Tr, thrX);
        const int nx = xfar ? Tr->n_xfar : Tr->n_xbox;
        const int* xids = xfar ? Tr->xfar_ids.p : Tr->xbox_ids.p;
        if (DL) launch_p2check_pair<T, true>(st, nx, xids, 1, Tr, WL, WY, OL, kappa, thrX);
        else launch_p2check_pair<T, false>(st, nx, xids, 1, Tr, WL, WY, OL, kappa, thrX);
        far_pair_c2e(Tr, OL, OY, WL, WY, false, xfar);
    }
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_M2L);
    far_pair_m2l(Tr, OL, OY, WL, WY);
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_DOWN);
    far_pair_l2l(Tr, OL, OY, WL, WY);
    if (fork) PB_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_LEAF);
    if (fork) {
        if (DL) launch_leaf_pair<T, true, false, 2>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
        else if (DN) launch_leaf_pair<T, false, true, 2>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
        else launch_leaf_pair<T, false, false, 2>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
    } else {
        if (DL) launch_leaf_pair<T, true, false, 0>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
        else if (DN) launch_leaf_pair<T, false, true, 0>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
        else launch_leaf_pair<T, false, false, 0>(st, Tr, WL, WY, OL, kappa, thrW, thrX);
    }
    ph.reset(); ph = std::make_unique<PhaseTimer>(ctx, PB_PH_SCATTER);
    const int* pt = Tr->same ? Tr->perm_s.p : Tr->perm_t.p;
    k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, WL.pot.p, outL);
    PB_CHECK_LAUNCH();
    k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, WY.pot.p, outY);
    PB_CHECK_LAUNCH();
    if (DN) {
        k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, WL.dn.p, dnL);
        PB_CHECK_LAUNCH();
        k_scatter<T, In><<<div_up(nt, 256), 256, 0, st>>>(nt, pt, WY.dn.p, dnY);
        PB_CHECK_LAUNCH();
    }
    ph.reset();
}

void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn) {
    auto O = get_operators(Tr, kernel, kappa, p, precision == PB_FP64);
    bool yuk = kernel == FMM_YUKAWA;
    if (precision == PB_FP64) {
        auto f = yuk ? apply_t<double, double, true> : apply_t<double, double, false>;
        f(Tr, *O, kappa, (const double*)q, (const double*)dip, (const double*)src_n, (const double*)tgt_n,
          (double*)out, (double*)out_dn);
    } else {
        auto f = yuk ? apply_t<float, float, true> : apply_t<float, float, false>;
        f(Tr, *O, kappa, (const float*)q, (const float*)dip, (const float*)src_n, (const float*)tgt_n, (float*)out,
          (float*)out_dn);
    }
}


void fmm_apply_pair_impl(fmm_tree* Tr, double kappa, int p, int precision, const void* qL, const void* qY,
                         const void* dip, const void* src_n, const void* tgt_n, void* outL, void* outY, void* dnL,
                         void* dnY) {
    const bool fp64 = precision == PB_FP64;
    auto OL = get_operators(Tr, FMM_LAPLACE, 0.0, p, fp64);
    auto OY = get_operators(Tr, FMM_YUKAWA, kappa, p, fp64);
    if (fp64)
        apply_pair_t<double, double>(Tr, *OL, *OY, kappa, (const double*)qL, (const double*)qY, (const double*)dip,
                                     (const double*)src_n, (const double*)tgt_n, (double*)outL, (double*)outY,
                                     (double*)dnL, (double*)dnY);
    else
        apply_pair_t<float, float>(Tr, *OL, *OY, kappa, (const float*)qL, (const float*)qY, (const float*)dip,
                                   (const float*)src_n, (const float*)tgt_n, (float*)outL, (float*)outY,
                                   (float*)dnL, (float*)dnY);
}

}  // namespace pbfmm
