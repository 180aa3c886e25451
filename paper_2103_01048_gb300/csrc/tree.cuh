// Device octree of the KIFMM (Sec. "Fast multipole method").
#pragma once
#include "common.cuh"
#include <map>
#include <memory>
#include <tuple>

namespace pbfmm {

struct Operators;   // fmm.cu: precomputed translation operators per level

// Per-tile M2L schedule for the target-stationary M2L: each tile is up to
// kM2LTile boxes of one level; for every relative offset used by any box of
// the tile, one entry lists the source box of each tile column (-1 = none).
constexpr int kM2LTile = 32;

struct M2LSchedule {
    int ntile = 0;
    std::vector<int> tile_level_h;     // level of each tile
    DBuf<int> tile_box;                // [ntile][kM2LTile] target box ids (-1 pad)
    DBuf<int> tile_level;              // [ntile]
    DBuf<int> entry_off;               // [ntile + 1] CSR over entries
    DBuf<int> entry_offset_idx;        // [nentry] offset index 0..342
    DBuf<int> entry_src;               // [nentry][kM2LTile] source box ids (-1 = none)
    long long nentry = 0;
    long long npairs = 0;              // total V-list pairs (algorithmic work)
};

// V-list pairs sorted by (level, offset) for the tensor-core M2L, cut into
// work items (first pair, count <= 1024, level, offset).
struct M2LPairs {
    DBuf<int> tgt, src;
    DBuf<int4> items;
    int nitems = 0;
    long long npairs = 0;
    DBuf<int4> items32;        // the same groups in chunks of at most 32 pairs (CUDA-core M2L)
    int nitems32 = 0;
    // items of a level-invariant operator set (Laplace): all levels of one
    // offset together (the pairs are ordered by offset, then level)
    DBuf<int4> items_off;
    int nitems_off = 0;
};

// Parent-child pairs (children of level >= 3) grouped by (level, octant) for
// M2M / L2L on the tensor cores; items of child level l are
// [level_item_off[l], level_item_off[l + 1]).
struct PCPairs {
    DBuf<int> parent, child;
    DBuf<int4> items;
    std::vector<int> level_item_off;
    int nitems = 0;
};

}  // namespace pbfmm

struct fmm_tree {
    pb_ctx* ctx = nullptr;
    int64_t ns = 0, nt = 0;
    bool same = true;
    int ncrit = 0;
    double c[3] = {0, 0, 0}, R = 1.0;

    pbfmm::DBuf<uint64_t> keys_s, keys_t;
    pbfmm::DBuf<int> perm_s, perm_t;
    pbfmm::DBuf<float4> pos_s, pos_t;        // Morton-sorted (x, y, z, 0)

    int nbox = 0, nlev = 0, nleaf = 0;
    std::vector<int> lvl_off;                // boxes of level l: [lvl_off[l], lvl_off[l+1])
    pbfmm::DBuf<int> level, parent, first_child, nchild, sb, se, tb, te;
    pbfmm::DBuf<int4> anchor;                // (ax, ay, az, level)
    pbfmm::DBuf<double4> center;             // (cx, cy, cz, half-width)

    pbfmm::DBuf<int> coll, coll_n, cn, cn_n, V, V_n, X, X_n;
    pbfmm::DBuf<int> U_off, U_ids, W_off, W_ids;
    long long n_u = 0, n_v = 0, n_w = 0, n_x = 0;
    // algorithmic work counters of one apply (see fmm_tree_info_t)
    long long work[6] = {0, 0, 0, 0, 0, 0};
    pbfmm::DBuf<int> leaf_ids;               // leaves with at least one target
    int n_tleaf = 0;
    std::vector<int> leaf_level_h;           // per level: leaves with sources (host lists built on demand)

    // leaves with sources, grouped by level (for P2M + UC2UE)
    pbfmm::DBuf<int> sleaf_ids;              // sorted by level
    std::vector<int> sleaf_lvl_off;          // [nlev + 1]
    // boxes with a non-empty X list
    pbfmm::DBuf<int> xbox_ids;              // in box (= level) order
    int n_xbox = 0;
    std::vector<int> xbox_lvl_off;           // [nlev + 1]
    // non-leaf boxes per level (M2M parents) and all boxes per level for L2L
    pbfmm::M2LSchedule m2l;
    pbfmm::M2LPairs m2l_pairs;
    pbfmm::PCPairs pc_pairs;
    // tensor-core items of the check -> equivalent solves: (first, count,
    // level) over sleaf_ids (upward) and xbox_ids (downward), one box per row
    pbfmm::DBuf<int4> c2e_items_up, c2e_items_dn;
    int n_c2e_up = 0, n_c2e_dn = 0;
    // X-list boxes whose X lists the leaf kernel does not sum directly (it
    // does for leaves of at most xfar_thr targets): P2L and its solve run on
    // these only.  Built on first use for a threshold (-1: not built).
    int xfar_thr = -1;
    pbfmm::DBuf<int> xfar_ids;
    int n_xfar = 0;
    pbfmm::DBuf<int4> c2e_items_xfar;
    int n_c2e_xfar = 0;

    std::map<std::tuple<int, double, int, int>, std::shared_ptr<pbfmm::Operators>> ops;
};
