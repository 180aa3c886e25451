/*
 * pbfmm — C-ABI of a GB300-native (sm_103a) fast-multipole boundary-element
 * solver for the linearised Poisson–Boltzmann equation, after the method of
 * Wang, Cooper, Betcke & Barba, "High-productivity, high-performance workflow
 * for virus-scale electrostatic simulations with Bempp-Exafmm" (arXiv
 * 2103.01048).
 *
 * Conventions for every entry point
 *   - Return value: PB_OK (0) on success, else one of the PB_E* codes below;
 *     no C++ exception crosses the ABI.  pb_last_error(ctx) gives a message.
 *   - Pointers are plain host or device pointers.  Where an argument says
 *     "host or device", the library inspects it with cudaPointerGetAttributes
 *     and stages host data through its own device buffers.
 *   - Work is ordered on the stream given to pb_create.  Calls documented as
 *     "asynchronous" return before the GPU finishes; read results after a
 *     stream synchronisation.
 *   - Objects returned through `out` parameters are owned by the library and
 *     released by the matching *_destroy call.  Caller buffers stay caller
 *     owned; the library never keeps a pointer to them after the call.
 *   - Coordinates are array-of-structures [n][3]; lengths in Angstrom,
 *     charges in e, energies in kcal/mol.
 */
#ifndef PBFMM_H
#define PBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
    PB_OK = 0,
    PB_EINVAL = 1,    /* invalid argument (null, size, unsupported option) */
    PB_ENOMEM = 2,    /* device allocation failed */
    PB_ECUDA = 3,     /* a CUDA runtime call failed */
    PB_EMESH = 4,     /* degenerate or non-manifold mesh */
    PB_ENOCONV = 5,   /* GMRES reached max_iter; last iterate kept */
    PB_ETIMEOUT = 6   /* a bounded device-side wait gave up */
};

/* Green's function families (Eq. single_double):
 * FMM_LAPLACE g = 1/(4 pi r), FMM_YUKAWA g = exp(-kappa r)/(4 pi r). */
enum { FMM_LAPLACE = 0, FMM_YUKAWA = 1 };

/* arithmetic of the FMM passes */
enum { PB_MIXED = 0 /* FP32 kernels */, PB_FP64 = 1 /* all-FP64 kernels */ };

typedef struct pb_ctx pb_ctx;
typedef struct fmm_tree fmm_tree;
typedef struct pb_mesh pb_mesh;
typedef struct pb_result pb_result;

/* trial/test spaces (Sec. "An introduction to Bempp") */
enum { PB_P0 = 0 /* piecewise constant, one unknown per triangle */,
       PB_P1 = 1 /* continuous piecewise linear, one unknown per vertex */ };

/* boundary integral formulations (Sec. "Boundary integral formulation of
 * electrostatics in molecular solvation"):
 *   PB_FORM_DIRECT    Eq. direct, unknowns [phi_1, dphi_1/dn] on the surface
 *   PB_FORM_EXTERIOR  Eq. lu (exterior derivative formulation), unknowns
 *                     [phi_2, dphi_2/dn] (exterior values)
 *   PB_FORM_INTERIOR  Eq. juffer (interior derivative formulation),
 *                     unknowns [phi_1, dphi_1/dn]
 * The derivative formulations need the P1 basis (their hypersingular
 * operators W are applied in the integrated-by-parts form, which needs
 * continuous trial and test functions). */
enum { PB_FORM_DIRECT = 0, PB_FORM_EXTERIOR = 1, PB_FORM_INTERIOR = 2 };

typedef struct {
    int p;        /* FMM expansion order, 2..10 */
    int ncrit;    /* maximum points per octree leaf */
} pb_fmm_params;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`; `cuda_stream` (a cudaStream_t,
 * may be NULL for the legacy default stream) orders every later call.  The
 * library owns *out; free it with pb_destroy. */
int pb_create(pb_ctx** out, int device, void* cuda_stream);

/* Synchronise the context stream and free every library-owned resource of
 * the context.  Trees created on it must be destroyed first. */
int pb_destroy(pb_ctx* ctx);

/* Message of the last failing call on this context (static storage owned by
 * the context; valid until the next call).  Never NULL. */
const char* pb_last_error(pb_ctx* ctx);

/* Wait for all work queued on the context stream; PB_ETIMEOUT if a kernel
 * with a bounded device-side wait gave up since the last check. */
int pb_sync(pb_ctx* ctx);

/* Per-phase device timers (CUDA events on the context stream).
 * pb_profile(ctx, 1) enables and resets them, pb_profile(ctx, 0) disables.
 * pb_profile_read returns, for phase `phase` (PB_PH_*), the accumulated
 * device milliseconds and the number of timed phase executions; phase
 * PB_PH_LAUNCHES returns in *calls the number of kernels the library
 * launched since the reset (ms unused).  Reading synchronises the stream. */
enum {
    PB_PH_GATHER = 0,  /* densities into Morton order                  */
    PB_PH_P2M = 1,     /* leaf sources -> upward check -> UC2UE        */
    PB_PH_M2M = 2,
    PB_PH_P2L = 3,
    PB_PH_M2L = 4,
    PB_PH_DOWN = 5,    /* L2L + DC2DE per level                        */
    PB_PH_LEAF = 6,    /* P2P + M2P + L2P                              */
    PB_PH_SCATTER = 7,
    PB_PH_BEM = 8,     /* sparse Galerkin glue around the FMM          */
    PB_PH_GMRES = 9,   /* FP64 Arnoldi / Givens                        */
    PB_PH_COUNT = 10,
    PB_PH_LAUNCHES = 100
};
int pb_profile(pb_ctx* ctx, int enable);

/* Context options.
 *   PB_OPT_COUPLING       0 (default): charge -> surface right-hand side,
 *                         surface -> charge reaction potential and the
 *                         adjoint right-hand side by direct FP64 sums when
 *                         atoms x quadrature points <= 4e9, else by the FMM
 *                         (trees over atoms and quadrature points, order p
 *                         of the mesh); 1: always direct; 2: always FMM.
 *   PB_OPT_DETERMINISTIC  0 (default): M2L/M2M/L2L with row reductions
 *                         (tensor cores, or CUDA cores parallel over pairs;
 *                         summation order run-dependent); 1: CUDA-core
 *                         kernels with a fixed order, bitwise reproducible
 *                         results.
 *   PB_OPT_SINGULAR       singular Galerkin entries of vertex-sharing pairs
 *                         (analytic inner integrals, graded outer rule):
 *                         0 (default): FP64 with a 5-level graded rule up to
 *                         262,144 triangles, else FP32 with a 4-level rule;
 *                         1: always FP64; 2: always FP32.
 *   PB_OPT_OVERLAP        0 (default): one stream; 1: the near field (P2P) of
 *                         fmm_apply_pair runs on a second stream of the
 *                         context, beside the far-field passes (fork and join
 *                         by events, also inside captured graphs).  On the
 *                         4M-point p = 6 workload it does not pay: the
 *                         tensor-core kernels cannot share an SM with the
 *                         near-field CTAs (shared memory).
 *   PB_OPT_RESTART        GMRES restart length m of pb_solve_batch(_ex):
 *                         0 (default): no restart (max_iter + 1 Krylov
 *                         vectors per system); m >= 1: GMRES(m), at most
 *                         m + 1 vectors per system, max_iter still bounding
 *                         the total iterations.  A system whose cycle ends
 *                         unconverged takes its update, recomputes its
 *                         residual with one mat-vec and starts a new cycle.
 *   PB_OPT_LEAF_NT        targets per thread of the leaf (P2P + M2P + L2P)
 *                         kernel of fmm_apply_pair: 0 (default): 4 in FP32,
 *                         2 in FP64; 2 or 4.  A tile-shape knob of the
 *                         autotuner (pb_tune); results differ only by
 *                         the summation order of each target's partial sums.
 *   PB_OPT_LEAF_PACKED    1 (default): the FP32 leaf kernel of fmm_apply_pair
 *                         without target-normal derivatives takes two sources
 *                         per packed instruction (add/mul/fma .f32x2); 0: one
 *                         source per scalar instruction.  Same arithmetic per
 *                         pair, summation order of the partial sums differs.
 *   PB_OPT_M2L_TILE       row tile of the tensor-core M2L: 0 (default): 256
 *                         pairs per MMA on CTA pairs (tcgen05 cta_group::2)
 *                         where the operator size allows (n_pad >= 128), else
 *                         128; 1: 128 pairs per MMA, one CTA per operator
 *                         part.  A tile-shape knob of the autotuner (pb_tune).
 *   PB_OPT_LIST_DIRECT    1 (default): in the FP32 applies without
 *                         target-normal derivatives (fmm_apply_pair and
 *                         fmm_apply on the packed kernels, PB_OPT_LEAF_PACKED
 *                         1), the pairs of the adaptive lists are summed directly
 *                         where that is less work than the equivalent
 *                         surfaces: a W-list box of at most n_e / 2 sources
 *                         instead of its M2P, and the X list of a leaf of at
 *                         most n_e targets instead of its P2L (the direct
 *                         sums are exact); 0: every W and X pair through the
 *                         equivalent surfaces, as in the KIFMM the paper
 *                         cites; 2: X lists only; 3: W boxes only.
 * Errors: PB_EINVAL for an unknown option or value. */
enum { PB_OPT_COUPLING = 1, PB_OPT_DETERMINISTIC = 2, PB_OPT_SINGULAR = 3, PB_OPT_OVERLAP = 4, PB_OPT_RESTART = 5,
       PB_OPT_LEAF_NT = 6, PB_OPT_LEAF_PACKED = 7, PB_OPT_M2L_TILE = 8, PB_OPT_LIST_DIRECT = 9 };
int pb_set_option(pb_ctx* ctx, int option, int value);
int pb_profile_read(pb_ctx* ctx, int phase, double* ms, int64_t* calls);

/* ------------------------------------------------------------------------ */
/* Octree and interaction lists (Sec. "Fast multipole method": enclosing     */
/* cube, recursive subdivision until each leaf holds at most ncrit points;   */
/* near field N(B) and interaction list I(B); adaptive U/V/W/X lists of the  */
/* kernel-independent FMM the paper cites).                                  */
/* ------------------------------------------------------------------------ */

/* Build the tree over sources `src_xyz` (device, float [n_src][3]) and, if
 * `tgt_xyz` is non-NULL, a distinct target set (device, float [n_tgt][3]);
 * with tgt_xyz NULL the targets are the sources (n_tgt ignored).
 * ncrit >= 1 is the maximum point count of a leaf (sources plus targets when
 * the sets differ).  Synchronous (returns when the tree is built).  The tree
 * is defined exactly (the oracle reproduces it bit for bit):
 *   - cube: centre = midpoint of the FP32 coordinate extremes, half-width
 *     R = (max extent / 2)(1 + 2^-20), in FP64;
 *   - Morton keys: per axis floor((x - lo) 2^21 / (2R)) clamped to
 *     [0, 2^21 - 1], computed with correctly rounded FP64 operations (no
 *     fused multiply-add), bits interleaved x, y, z from the most
 *     significant; 63-bit keys sorted stably (ties keep the input order);
 *   - a box splits while it holds more than ncrit points and its level is
 *     below 21; empty children are dropped; boxes are numbered level by
 *     level in Morton order;
 *   - lists (adjacency = the closed cubes intersect; colleagues = the
 *     adjacent boxes of the same level): U(B), for a leaf B, every adjacent
 *     leaf, B included (near field, P2P); V(B) the children of the parent's
 *     colleagues not adjacent to B (interaction list, M2L); W(B), for a leaf
 *     B, the descendants D of B's colleagues with D not adjacent to B but
 *     D's parent adjacent (M2P); X(B) the coarser leaves adjacent to B's
 *     parent but not to B (P2L).
 * Errors: PB_EINVAL for n_src < 1, ncrit < 1 or NULL src_xyz. */
int fmm_tree_build(pb_ctx* ctx, const float* src_xyz, int64_t n_src,
                   const float* tgt_xyz, int64_t n_tgt, int ncrit, fmm_tree** out);

int fmm_tree_destroy(fmm_tree* tree);

typedef struct {
    int64_t n_src, n_tgt, n_box, n_leaf;
    int32_t n_levels;      /* deepest level + 1 */
    int32_t same;          /* 1 if targets are the sources */
    int64_t n_u, n_v, n_w, n_x;   /* total entries of each list */
    double center[3], half_width; /* the enclosing cube */
    /* algorithmic work of one apply on this tree (exact, from the lists) */
    int64_t p2p_pairs;     /* point pairs of the U lists (near field)      */
    int64_t m2p_targets;   /* sum over leaves of targets x |W list|        */
    int64_t p2l_sources;   /* sum over boxes of X-list source points       */
    int64_t l2p_targets;   /* targets in leaves at level >= 2              */
    int64_t p2m_sources;   /* sources in leaves                            */
    int64_t n_dense_box;   /* boxes at level >= 2 (UC2UE/DC2DE/M2M/L2L)    */
} fmm_tree_info_t;

int fmm_tree_info(const fmm_tree* tree, fmm_tree_info_t* info);

/* Copy the sorted order out to HOST buffers (any may be NULL):
 * perm_*[k] = original index of the k-th point in Morton order; keys_* are
 * the sorted 63-bit keys.  Synchronous. */
int fmm_tree_export_points(const fmm_tree* tree, int32_t* perm_src, uint64_t* keys_src,
                           int32_t* perm_tgt, uint64_t* keys_tgt);

/* Copy the boxes out to HOST buffers [n_box] (anchor is [n_box][3]); boxes
 * are numbered level by level in Morton order, children of a box are
 * contiguous.  src_begin/src_end index the Morton-sorted sources. */
int fmm_tree_export_boxes(const fmm_tree* tree, int32_t* level, int32_t* parent,
                          int32_t* first_child, int32_t* nchild, int32_t* anchor,
                          int32_t* src_begin, int32_t* src_end,
                          int32_t* tgt_begin, int32_t* tgt_end);

/* Copy one interaction list out as CSR to HOST buffers: which = 0 (U), 1 (V),
 * 2 (W), 3 (X); off [n_box + 1], ids [off[n_box]] in ascending box order. */
int fmm_tree_export_list(const fmm_tree* tree, int which, int64_t* off, int32_t* ids);

/* ------------------------------------------------------------------------ */
/* FMM matrix-vector product (Eq. nbody_sum through the KIFMM of Sec. "Fast   */
/* multipole method": P2M, M2M, M2L, L2L, L2P, P2P; equivalent densities      */
/* matched on check surfaces, Eq. multipole_local).                          */
/* ------------------------------------------------------------------------ */

/* out[i] = sum_j g(x_i, y_j) q[j] + dg/dn_y(x_i, y_j) dip[j]        (r > 0)
 * out_dn[i] = sum_j dg/dn_x(x_i, y_j) q[j]     (adjoint double layer, K')
 * for every target x_i of the tree, approximated by the KIFMM with
 * expansion order p (points per edge of the equivalent/check surfaces,
 * n_e = 6(p-1)^2 + 2 surface points; 2 <= p <= 10).
 *   kernel    FMM_LAPLACE or FMM_YUKAWA (kappa > 0 for Yukawa).
 *   q         source monopole densities [n_src] or NULL (single layer).
 *   dip       source dipole densities [n_src] or NULL (double layer); needs
 *             src_n, the source unit normals [n_src][3].
 *   tgt_n     target unit normals [n_tgt][3]; needed iff out_dn != NULL.
 *   out       [n_tgt] potentials in ORIGINAL target order (required).
 *   out_dn    [n_tgt] target-normal derivatives or NULL.  With out_dn the
 *             dipole term must be absent (the hypersingular kernel is not
 *             provided).
 *   precision PB_MIXED (FP32 arithmetic, FP32 buffers: pass float*) or
 *             PB_FP64 (FP64 arithmetic, every density/normal/output buffer
 *             is double*).
 * Buffers may be host or device memory (see conventions).  With device
 * buffers the call is asynchronous; with any host buffer it synchronises.
 * Operators for (kernel, kappa, p, tree size) are precomputed on first use
 * and cached in the tree.  With PB_MIXED and p in 2..6, 8 or 10 the M2L,
 * M2M, L2L and the check -> equivalent solves run on the tensor cores (TF32
 * split into hi + lo parts, three products per step; at p = 8 and 10 each
 * operator is split into parts that fit in shared memory); with p = 7 or 9
 * or PB_FP64 on the CUDA cores, the
 * M2L parallel over interaction pairs.  The M2L / M2M / L2L reductions make
 * the summation order run-dependent (~1e-7 in FP32, ~1e-16 in FP64);
 * PB_OPT_DETERMINISTIC selects fixed-order CUDA-core kernels.  The tensor-core
 * waits are bounded: a timeout is reported as PB_ETIMEOUT by the next
 * synchronising call (pb_sync, or this call when it synchronises).
 * Errors: PB_EINVAL for missing normals, p out of range, kappa <= 0 with
 * FMM_YUKAWA, dip together with out_dn. */
int fmm_apply(pb_ctx* ctx, fmm_tree* tree, int kernel, double kappa, int p, int precision,
              const void* q, const void* dip, const void* src_n, const void* tgt_n,
              void* out, void* out_dn);

/* Laplace and Yukawa in one traversal (Eq. bempp_fmm_matvec: the direct
 * formulation applies both kernels to the same quadrature points in every
 * mat-vec).  With g_L = 1/(4 pi r), g_Y = e^{-kappa r}/(4 pi r):
 *   out_lap[i] = sum_j g_L(x_i, y_j) q_lap[j] + dg_L/dn_y(x_i, y_j) dip[j]
 *   out_yuk[i] = sum_j g_Y(x_i, y_j) q_yuk[j] + dg_Y/dn_y(x_i, y_j) dip[j]
 *   dn_lap[i]  = sum_j dg_L/dn_x(x_i, y_j) q_lap[j]
 *   dn_yuk[i]  = sum_j dg_Y/dn_x(x_i, y_j) q_yuk[j]
 * The two kernels share the dipole densities and the geometry of every
 * pair (one distance and one reciprocal square root per pair); the far
 * field keeps one set of operators per kernel.  Arguments as fmm_apply:
 * q_lap / q_yuk / dip may each be NULL (no such term), dip needs src_n,
 * dn_lap and dn_yuk are both NULL or both given (then tgt_n is required and
 * dip must be NULL).  Results equal two fmm_apply calls up to rounding.
 * q_lap and q_yuk may be the same array (copied once when on the host).
 * Errors: PB_EINVAL as fmm_apply, and kappa <= 0. */
int fmm_apply_pair(pb_ctx* ctx, fmm_tree* tree, double kappa, int p, int precision,
                   const void* q_lap, const void* q_yuk, const void* dip, const void* src_n,
                   const void* tgt_n, void* out_lap, void* out_yuk, void* dn_lap, void* dn_yuk);

/* ------------------------------------------------------------------------ */
/* Boundary-element mesh and the direct formulation (Eq. direct).            */
/* ------------------------------------------------------------------------ */

/* Set up a closed triangulated surface: verts (host or device, double
 * [nv][3]), tris (host or device, int32 [nt][3], counter-clockwise seen from
 * outside so that normals point out of the solute, Eq. pde).  basis is PB_P0
 * (one unknown per triangle and block) or PB_P1 (one per vertex: the mesh
 * must be a closed surface whose every vertex belongs to a triangle); nquad
 * (3 or 6) is the regular quadrature rule per triangle (3: the
 * interior degree-2 rule (2/3,1/6,1/6); 6: Dunavant degree 4).  Builds
 * normals, areas, quadrature points, the vertex-sharing adjacency (the
 * pairs that need singular quadrature) and the octree over the quadrature
 * points.  Copies the inputs; synchronous.
 * Errors: PB_EMESH for invalid indices or a triangle with area below
 * 1e-12 times the mean area; PB_EINVAL for other bad arguments. */
int pb_mesh_setup(pb_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                  int basis, int nquad, const pb_fmm_params* params, pb_mesh** out);
int pb_mesh_destroy(pb_mesh* mesh);

/* Sizes of a mesh: triangles, quadrature points, vertex-sharing pairs. */
int pb_mesh_info(const pb_mesh* mesh, int64_t* nt, int64_t* nquad_points, int64_t* nadj);

/* Unknowns per block of the 2 x 2 systems: nt for PB_P0, nv for PB_P1 (the
 * solution and mat-vec vectors hold 2 n doubles). */
int pb_mesh_unknowns(const pb_mesh* mesh, int64_t* n);

/* Singular Galerkin entries for Yukawa parameter kappa, to HOST buffers:
 * adj_off [nt + 1] and adj_ids [nadj] (CSR of the pairs, ascending), and
 *   P0 mesh: S [nadj][4] = (V_L, K_L, V_Y, K_Y) entries int_Ti int_Tj of the
 *            kernels of Eq. single_double (identical or vertex-sharing
 *            triangle pairs);
 *   P1 mesh: S [nadj][4][3][3] = for the same four kernels, the blocks
 *            int_Ti lambda_a int_Tj lambda_b k (a the test vertex of T_i, b the
 *            trial vertex of T_j, in the triangles' vertex order) minus the
 *            same blocks under the regular product rule: what the mat-vec
 *            adds to its point sums for these pairs.
 * Synchronous; assembles S on first use for this kappa. */
int pb_mesh_export_singular(pb_ctx* ctx, pb_mesh* mesh, double kappa, int64_t* adj_off, int32_t* adj_ids,
                            double* S);

/* y = A x for the Galerkin matrix of Eq. direct (precond = 0), or
 * y = P^{-1} A x with the block-diagonal preconditioner (precond = 1),
 * through the split A x = P2^T (G - C) P1 x + S x (Eq. bempp_fmm_matvec).
 * x, y: double [2 nt] (phi, then dphi/dn), host or device.  precision
 * PB_MIXED runs the FMM and the corrections in FP32, PB_FP64 in FP64.
 * Synchronous when a host buffer is given. */
int pb_mesh_matvec(pb_ctx* ctx, pb_mesh* mesh, double eps_in, double eps_out, double kappa, int precision,
                   int precond, const double* x, double* y);

/* y = A x (precond = 0) or y = P^{-1} A x (precond = 1) for the Galerkin
 * matrix of `formulation` (PB_FORM_*) on the mesh's basis; x, y: double
 * [2 n] (n from pb_mesh_unknowns), host or device.  P0: PB_FORM_DIRECT only,
 * block-diagonal preconditioner as pb_mesh_matvec.  P1: every formulation,
 * with the blocks (e12 = eps_in/eps_out, e21 = eps_out/eps_in, M the P1
 * mass matrix, K' the adjoint double layer, W the hypersingular operator of
 * Eq. adj_hyp):
 *   direct    [ M/2 + K_L, -V_L ; M/2 - K_Y, e12 V_Y ]
 *   exterior  [ (1+e12)/2 M - (K_Y - e12 K_L), V_Y - V_L ;
 *               e12 (W_Y - W_L), (1+e12)/2 M + e12 K'_Y - K'_L ]   (Eq. lu)
 *   interior  [ (1+e21)/2 M - (e21 K_Y - K_L), V_Y - V_L ;
 *               W_Y - W_L, (1+e12)/2 M + e12 K'_Y - K'_L ]         (Eq. juffer)
 * and the lumped-mass preconditioner P = diag(lumped M, lumped M) (row sums
 * of M; Sec. "Matrix conditioning of two derivative formulations").  W is
 * applied in its integrated-by-parts form <W u, v> = int int g curl u .
 * curl v (+ kappa^2 n_x.n_y g_Y u v for Yukawa): one FMM pass per curl
 * component, three Yukawa passes of the phi n components, and one pass of
 * target-normal derivatives for K', beside the V/K pass of every mat-vec.
 * Synchronous when a host buffer is given.
 * Errors: PB_EINVAL for an unknown formulation or a derivative formulation
 * on a P0 mesh. */
int pb_mesh_matvec_ex(pb_ctx* ctx, pb_mesh* mesh, double eps_in, double eps_out, double kappa, int precision,
                      int precond, int formulation, const double* x, double* y);

/* Solve Eq. direct for point charges q (double [na], e) at atoms (double
 * [na][3]) inside the surface, eps_in / eps_out relative permittivities,
 * kappa the inverse Debye length (1/A).  Full GMRES (no restart, x0 = 0,
 * left block-diagonal preconditioning) in FP64 until the preconditioned
 * relative residual is <= tol or max_iter (1..2000) iterations.  Returns PB_OK, or
 * PB_ENOCONV with *out still holding the last iterate.  Synchronous.
 * From the second solve on a mesh with unchanged eps, kappa, precision and
 * options, the mat-vec is replayed from a CUDA graph the mesh keeps (the
 * first solve launches it directly and fills the caches); pb_profile's
 * phase timers and launch count then cover only directly launched work. */
int pb_solve(pb_ctx* ctx, pb_mesh* mesh, const double* atoms, const double* q, int64_t na, double eps_in,
             double eps_out, double kappa, double tol, int max_iter, int precision, pb_result** out);

/* pb_solve for any formulation (PB_FORM_*): the system of pb_mesh_matvec_ex
 * with its preconditioner, right-hand side [int psi_i f ; int psi_i df/dn]
 * of the Coulomb field f = sum_k q_k / (4 pi eps |x - r_k|), eps = eps_in
 * (interior, direct; the direct formulation's second block is 0) or
 * eps_out (exterior).  pb_result_get returns the formulation's unknowns
 * (the exterior formulation's are the exterior values phi_2, dphi_2/dn);
 * pb_solvation_energy converts to the interior fields (phi_1 = phi_2,
 * dphi_1/dn = (eps_out/eps_in) dphi_2/dn) for Eq. phi_reac.  For P1 meshes
 * the charge <-> surface sums are always direct FP64 sums.
 * pb_energy_grad takes direct-formulation P0 systems only; pb_solve_batch_ex
 * takes any formulation with its basis.
 * Errors: as pb_solve, and PB_EINVAL for a derivative formulation on a P0
 * mesh. */
int pb_solve_ex(pb_ctx* ctx, pb_mesh* mesh, const double* atoms, const double* q, int64_t na, double eps_in,
                double eps_out, double kappa, double tol, int max_iter, int precision, int formulation,
                pb_result** out);
int pb_result_destroy(pb_result* res);

/* Iterations, final relative residual, and (if x != NULL) the solution to a
 * HOST buffer double [2 n] (n from pb_mesh_unknowns): phi on the triangles
 * (P0) or vertices (P1), then dphi/dn. */
int pb_result_get(const pb_result* res, int* iterations, double* residual, double* x);

/* Polar solvation energy (Eq. energy) of a solved system, kcal/mol:
 * dG = 1/2 sum_k q_k phi_reac(r_k) * 4 pi * 332.0637, with the reaction
 * potential of Eq. phi_reac evaluated at the atoms by the regular rule.
 * phi_reac (HOST, double [na]) may be NULL.  Synchronous. */
int pb_solvation_energy(pb_ctx* ctx, pb_result* res, double* dG_kcal_per_mol, double* phi_reac);

/* Solve several systems together (same eps_in, eps_out, kappa, tol,
 * max_iter, precision; each its own mesh, charges and positions), direct
 * formulation (Eq. direct) on P0 meshes: the GMRES iterations of all systems
 * run in lockstep, one lockstep iteration of every active system (its
 * preconditioned mat-vec on its own stream, the Gram-Schmidt passes, the
 * Givens update and the convergence test on the device) is one CUDA graph
 * replayed every iteration, with one host synchronisation per iteration for
 * all systems; the graph is re-captured without the converged systems once a
 * quarter of them have finished.  meshes[nsys] must be distinct.  atoms[s]
 * (double [na[s]][3]) and charges[s] (double [na[s]]) are host or device
 * arrays.  out[nsys] receives one result per system (free each with
 * pb_result_destroy), status[nsys] PB_OK or PB_ENOCONV per system.  Returns
 * PB_OK if every system converged, else PB_ENOCONV.  Synchronous.  The
 * results match pb_solve up to the FMM's run-dependent summation order. */
int pb_solve_batch(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, const double* const* atoms,
                   const double* const* charges, const int64_t* na, double eps_in, double eps_out, double kappa,
                   double tol, int max_iter, int precision, pb_result** out, int* status);

/* pb_solve_batch with a formulation (PB_FORM_DIRECT, PB_FORM_EXTERIOR or
 * PB_FORM_INTERIOR, as pb_solve_ex): the derivative formulations need PB_P1
 * meshes (all systems of the batch; PB_EINVAL otherwise), whose GMRES
 * iteration counts stay flat under refinement (Sec. "Matrix conditioning of
 * two derivative formulations"), so a batch of large meshes needs far fewer
 * Krylov vectors than with the direct formulation. */
int pb_solve_batch_ex(pb_ctx* ctx, pb_mesh* const* meshes, int nsys, const double* const* atoms,
                      const double* const* charges, const int64_t* na, double eps_in, double eps_out, double kappa,
                      double tol, int max_iter, int precision, int formulation, pb_result** out, int* status);

/* Autotuner for the leaf size: for each candidate ncrit, build the octree of
 * the points xyz (host or device, float [n][3]) and time one Laplace and one
 * Yukawa single+double-layer FMM apply at order p (mean of 3 after a warm
 * run, CUDA events); *best_ncrit receives the fastest candidate and *best_ms
 * (may be NULL) its time.  Synchronous. */
int pb_tune_ncrit(pb_ctx* ctx, const float* xyz, int64_t n, int p, const int32_t* candidates, int ncand,
                  int* best_ncrit, double* best_ms);

/* Autotuner for the leaf size and the tile shapes of the two hot kernels,
 * on the work of one direct-formulation mat-vec: for each candidate ncrit
 * it builds the octree of xyz (host or device, float [n][3]) and times the
 * paired Laplace + Yukawa (kappa 0.125) single+double-layer apply
 * (fmm_apply_pair, mixed precision, order p; mean of 3 after a warm run,
 * CUDA events) with every combination of PB_OPT_LEAF_NT (2, 4) and
 * PB_OPT_M2L_TILE (0, 1).  On return the context's PB_OPT_LEAF_NT and
 * PB_OPT_M2L_TILE hold the fastest combination (on an error they keep their
 * values from before the call); *best_ncrit, *best_leaf_nt, *best_m2l_tile
 * and *best_ms (any of the last three may be NULL) receive it.  The tile
 * options change the summation order of partial sums only.  Synchronous. */
int pb_tune(pb_ctx* ctx, const float* xyz, int64_t n, int p, const int32_t* candidates, int ncand, int* best_ncrit,
            int* best_leaf_nt, int* best_m2l_tile, double* best_ms);

/* Gradient of the polar solvation energy of a solved system (kcal/mol per e
 * and per A) with respect to the atomic charges and positions, by one
 * adjoint GMRES solve with A^T (the transposed double layer is the adjoint
 * double layer K', Eq. adj_hyp) in the precision of `res`, to relative
 * residual tol (max_iter 1..2000).  The surface mesh is held fixed.
 *   dEdq  HOST double [na]        dE/dq_k
 *   dEdx  HOST double [na][3]     dE/dr_k
 * Either may be NULL.  Returns PB_OK or PB_ENOCONV (gradients from the last
 * adjoint iterate).  Synchronous. */
int pb_energy_grad(pb_ctx* ctx, pb_result* res, double tol, int max_iter, double* dEdq, double* dEdx);

/* The polar solvation energy of a solved system, like pb_solvation_energy,
 * but without allocating any device memory.  The paper has no counterpart:
 * this entry exists for callers that cannot allocate device memory at the
 * point where they need the energy, for example an application whose
 * device allocator is locked after start-up (a fixed memory budget reserved
 * up front), or a real-time loop that must not enter the allocator and risk
 * its latency or an out-of-memory failure in the middle of a step.
 *   - All intermediate values (partial reaction potentials at the atoms)
 *     live in one fixed scratch array compiled into the library: 524,288
 *     doubles (4 MB), held on every GPU that loads the library until the
 *     process exits.  res may hold at most 262,144 atoms (else PB_EINVAL).
 *   - The reaction potential is always the direct FP64 sum over the
 *     quadrature points (Eq. phi_reac), whatever PB_OPT_COUPLING says.
 *     Where pb_solvation_energy uses the FMM coupling instead (option 2, or
 *     atoms x quadrature points above 4e9 under the automatic setting) the
 *     two energies differ by the FMM's error (about 1e-6 relative at p = 6),
 *     otherwise by rounding only.  The direct sum costs atoms x quadrature
 *     points pair evaluations, so it is slow for very large systems.
 *   - dG_device must be a caller-owned DEVICE double on the context's GPU
 *     (else PB_EINVAL); it receives the energy in kcal/mol.
 *   - Asynchronous on the context stream.  The first call on a device looks
 *     up the scratch array's device address (once per device, with that
 *     device current).
 *   - All calls share the one scratch array and its contents are whatever
 *     the last call left: calls whose work overlaps on the GPU (other
 *     streams or contexts on the same device) race, and the caller must
 *     serialise them. */
int pb_solvation_energy_noalloc(pb_ctx* ctx, const pb_result* res, double* dG_device);

#ifdef __cplusplus
}
#endif

#endif /* PBFMM_H */
