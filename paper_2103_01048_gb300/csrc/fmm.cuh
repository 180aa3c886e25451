// KIFMM operators and apply (Sec. "Fast multipole method").
#pragma once
#include "tree.cuh"

namespace pbfmm {

// Surface radii relative to the box half-width (kernel-independent FMM of
// Ying, Biros & Zorin, cited by the paper): upward equivalent surface close
// to the box, upward check surface outside it; the downward pair swapped.
constexpr double kAlphaInner = 1.05;
constexpr double kAlphaOuter = 2.95;

inline int surface_count(int p) { return 6 * (p - 1) * (p - 1) + 2; }
inline int pad32(int n) { return (n + 31) / 32 * 32; }

// Translation operators for one (kernel, kappa, p) on one tree, per level.
// Matrices are row-major [npad][npad] (row = output point, column = input
// point), zero-padded beyond ne.
struct Operators {
    int kernel = 0;
    double kappa = 0.0;
    int p = 0, ne = 0, npad = 0, nlev = 0;
    DBuf<double> surf;            // [ne][3] unit surface points
    DBuf<float> surf_f;           // [ne][4] float copy (x, y, z, 0)
    // FP32 copies
    // factored solves of the FP32 path: pinv = W2 W1 (W1 = D V^T K^T, W2 = V)
    DBuf<float> uc2ue_w1, uc2ue_w2, dc2de_w1, dc2de_w2;   // [nlev][npad^2]
    DBuf<float> m2m, l2l;         // [nlev][8][npad^2]  (child level index)
    DBuf<float> m2l;              // [nlev][343][npad^2]
    // tensor-core M2L: per level and offset (Laplace: one level), the
    // operator split into TF32 hi + lo parts, pre-swizzled (128B swizzle,
    // K-major) per part of its rows and inner columns:
    // [level][343][part][hi|lo][K blocks][rows of the part][128 B]
    DBuf<float> m2l_tc;
    DBuf<float> m2m_tc, l2l_tc;   // same packing, [level][8 octants]
    DBuf<float> uc2ue_w1_tc, uc2ue_w2_tc, dc2de_w1_tc, dc2de_w2_tc;   // same packing, [level]
    bool have_tc = false;
    bool m2l_tc_single = false;   // Laplace: m2l_tc holds one level (the operators are level-invariant)
    // FP64 copies (all-FP64 path)
    DBuf<double> uc2ue_d, dc2de_d, m2m_d, l2l_d, m2l_d;
    bool have_d = false;
};

std::shared_ptr<Operators> get_operators(fmm_tree* T, int kernel, double kappa, int p, bool need_fp64);

}  // namespace pbfmm
