/*
 * Test hooks of the pbfmm library.  They are not part of the solver's
 * interface (include/pbfmm.h): the library's own tests use them to reach
 * failure paths that a healthy GPU never takes, without faulting or hanging
 * the GPU.  All of them act process-wide (every context, every thread).
 */
#ifndef PBFMM_TESTING_H
#define PBFMM_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of device allocations the library has made so far (every buffer
 * of trees, meshes, operators, results and per-call workspace; not the
 * context's 4-byte error flag nor the scratch array of
 * pb_solvation_energy_noalloc, which is static). */
int64_t pbfmm_test_alloc_count(void);

/* Make the nth device allocation from now (nth >= 1) fail as a failed
 * cudaMallocAsync would: the call that needs it returns PB_ENOMEM and
 * releases whatever it had allocated.  nth <= 0 switches the injection
 * off.  The injection fires once. */
void pbfmm_test_fail_alloc(int64_t nth);

/* Bytes currently allocated (not cached) from the default stream-ordered
 * memory pool of CUDA device `device`, from which the library takes all its
 * buffers; -1 if the query fails.  Work queued on the library's streams
 * should be synchronised first. */
int64_t pbfmm_test_pool_used(int device);

/* Cycle limit of the bounded mbarrier waits in the tensor-core box-operator
 * kernel (M2L, M2M, L2L and the check -> equivalent solves; default 2e9
 * cycles, about one second).  A small limit makes waits give up: the CTA
 * then stops its roles, lets its issued MMAs and copies finish, frees its
 * tensor memory and reports PB_ETIMEOUT through the next synchronising call
 * (pb_sync).  cycles <= 0 restores the default.  Read at kernel launch, so
 * a CUDA graph captured meanwhile keeps the value it was captured with. */
void pbfmm_test_wait_limit(int64_t cycles);

/* Stable sort of n (key, value) pairs by the low `bits` bits of the keys
 * (1 <= bits <= 64) with the library's radix sort (the Morton-key sort of
 * the octree build); host buffers in and out.  PB_OK or PB_EINVAL. */
int pbfmm_test_radix_sort(const uint64_t* keys, const int32_t* vals, int64_t n, int bits, uint64_t* keys_out,
                          int32_t* vals_out);

/* Kernel of the tensor-core M2L: mode 1 (the default) runs pairs of CTAs
 * (a cluster of two, whose MMAs of M = 256 take A rows and B columns from
 * both CTAs' shared memory) at n_pad >= 128, mode 0 one CTA per operator
 * part.  M2M, L2L and the check -> equivalent solves always use one CTA per
 * part.  Returns the previous mode.  Read at kernel launch. */
int pbfmm_test_tc_pair(int mode);

/* Launch properties of the CTA-pair kernel at npad 128, without launching
 * it: out[0] registers per thread, out[1] max threads per block, out[2]
 * static shared bytes, out[3] dynamic shared bytes of a launch, out[4] the
 * number of clusters of two such CTAs that can be resident at once (0: the
 * launch cannot run on this device).  PB_OK or PB_ECUDA. */
int pbfmm_test_tc_pair_info(int* out);

/* Eigendecomposition of a symmetric n x n matrix A (row-major, FP64) with
 * the host eigensolver of the operator precomputation: w[j] eigenvalue j,
 * V[k * n + j] component k of its unit eigenvector (A = V diag(w) V^T).
 * Runs on the host only.  PB_OK or PB_EINVAL. */
int pbfmm_test_sym_eig(int n, const double* A, double* w, double* V);

/* D = Q Op^T for one operator through the tensor-core box-operator kernel
 * (host buffers: Q [nrows][npad], Op [npad][npad], D [nrows][npad]; npad in
 * {32, 64, 128, 160, 320, 512}).  PB_OK, PB_EINVAL or PB_ETIMEOUT. */
int pbfmm_selftest_m2l_tc(int nrows, int npad, const float* Q, const float* Op, float* D);

#ifdef __cplusplus
}
#endif

#endif /* PBFMM_TESTING_H */
