// Galerkin BEM data of the direct formulation (Sec. "An introduction to
// Bempp", Eq. bempp_fmm_matvec, Eq. direct).
#pragma once
#include "fmm.cuh"
#include <functional>

struct pb_mesh {
    pb_ctx* ctx = nullptr;
    int64_t nv = 0, nt = 0;
    int nq = 3;              // regular quadrature points per triangle
    int basis = PB_P0;       // PB_P0: unknowns per triangle; PB_P1: per vertex
    int64_t nunk = 0;        // unknowns per block: nt (P0) or nv (P1)
    int p = 6, ncrit = 128;  // FMM parameters
    pbfmm::DBuf<double> verts;        // [nv][3]
    pbfmm::DBuf<int> tris;            // [nt][3]
    pbfmm::DBuf<double> nrm, area;    // [nt][3], [nt]
    // quadrature points a = i*nq + k (FP64 and FP32 copies)
    pbfmm::DBuf<double> qp_d, qn_d, qw_d;   // [N_Q][3], [N_Q][3], [N_Q] (w_k |T_i|)
    pbfmm::DBuf<float> qp_f, qn_f, qw_f;
    // triangles sharing at least one vertex (self included), CSR, ascending
    pbfmm::DBuf<int> adj_off, adj_ids;
    int64_t nadj = 0;
    // singular Galerkin entries of the adjacent pairs, per CSR entry:
    // [V_L, K_L, V_Y, K_Y] for kappa_S
    pbfmm::DBuf<double> S_d;
    pbfmm::DBuf<float> S_f;
    double kappa_S = -1.0;
    int sing_mode = 0;                // 1: FP64 rule, 2: FP32 rule
    pbfmm::DBuf<int> adj_tr;          // for CSR entry (i, j): the index of entry (j, i)
    // P1 (continuous piecewise-linear) data
    pbfmm::DBuf<int> vt_off, vt_ent;  // vertex -> incident (triangle, local vertex) = 3 t + a, CSR by triangle
    pbfmm::DBuf<double> lmass;        // [nv] lumped mass (row sums of the P1 mass matrix)
    pbfmm::DBuf<double> curl;         // [nt][3][3] surface curls of the three hat functions
    pbfmm::DBuf<double> rule;         // [nq][4] regular rule: barycentrics (l0, l1, l2) and weight
    pbfmm::DBuf<double> D1;           // [nadj][4][3][3] P1 singular blocks minus their regular-rule part
    double kappa_D1 = -1.0;
    int sing_mode1 = 0;
    fmm_tree* tree = nullptr;
    // preconditioned mat-vec of pb_solve captured as a CUDA graph (fixed
    // input/output vectors), valid for the parameters in mv_key
    cudaGraph_t mv_graph = nullptr;
    cudaGraphExec_t mv_exec = nullptr;
    pbfmm::DBuf<double> mv_in, mv_out;
    double mv_key[9] = {};
    bool mv_warm = false;             // one uncaptured mat-vec ran with mv_key (caches filled)
    ~pb_mesh() {
        if (mv_exec) cudaGraphExecDestroy(mv_exec);
        if (mv_graph) cudaGraphDestroy(mv_graph);
    }
};

namespace pbfmm {
int gmres(pb_mesh* M, const std::function<void(const double*, double*)>& matvec, const double* b, DBuf<double>& x,
          double tol, int max_iter, int* iterations, double* residual);
void ensure_singular_public(pb_mesh* M, double kappa);
void mesh_matvec(pb_mesh* M, double eps_in, double eps_out, double kappa, int precision, const double* x, double* y,
                 int precond, int formulation = PB_FORM_DIRECT);
// P1 basis and the derivative formulations (p1.cu)
void p1_setup(pb_mesh* M);
void matvec_p1(pb_mesh* M, double eps_in, double eps_out, double kappa, int precision, int formulation,
               const double* x, double* y, int precond);
void rhs_p1(pb_mesh* M, pb_result* R, double* b);
void reaction_potential_p1(pb_mesh* M, pb_result* R, double* phir);
void fmm_apply_impl(fmm_tree* Tr, int kernel, double kappa, int p, int precision, const void* q, const void* dip,
                    const void* src_n, const void* tgt_n, void* out, void* out_dn);
void fmm_apply_pair_impl(fmm_tree* Tr, double kappa, int p, int precision, const void* qL, const void* qY,
                         const void* dip, const void* src_n, const void* tgt_n, void* outL, void* outY, void* dnL,
                         void* dnY);
}  // namespace pbfmm

struct pb_result {
    pb_mesh* mesh = nullptr;
    int64_t nt = 0, na = 0;
    double eps_in = 4, eps_out = 80, kappa = 0.125;
    int precision = PB_MIXED;
    int formulation = PB_FORM_DIRECT;
    int64_t nunk = 0;                 // unknowns per block (nt for P0, nv for P1)
    int iterations = 0;
    double residual = 0.0;
    int status = PB_OK;
    pbfmm::DBuf<double> x;            // [2 nunk]: phi, then dphi/dn (exterior values for PB_FORM_EXTERIOR)
    pbfmm::DBuf<double> atoms, charges;
    double energy = 0.0;
    bool have_energy = false;
    // charge <-> surface couplings through the FMM (large atom counts)
    fmm_tree* tree_qa = nullptr;      // sources = quadrature points, targets = atoms
    fmm_tree* tree_aq = nullptr;      // sources = atoms, targets = quadrature points
    pbfmm::DBuf<float> atoms_f, q_f;  // atom positions [na][3], charges / eps1
    pbfmm::DBuf<double> q_d;
    ~pb_result() {
        delete tree_qa;
        delete tree_aq;
    }
    // adjoint solve (gradients)
    pbfmm::DBuf<double> lambda;       // [2 nt]
    int adj_iterations = 0;
    double adj_residual = 0.0;
};
