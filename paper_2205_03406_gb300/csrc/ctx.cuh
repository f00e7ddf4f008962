// Internal state of one compression job (the opaque hm_ctx of hm.h) and the
// interfaces between the modules: tree.cu, color.cu, sample.cu, sample_tc.cu,
// peel.cu, basis.cu, apply.cu and the C ABI in hm_api.cu.
#pragma once

#include "common.cuh"

namespace hm {

constexpr int QBITS = 21;       // integer grid: 2^21 cells per dimension
constexpr int MAX_LEVELS = 22;  // levels 0..21
constexpr int MAX_COLORS = 1024;
constexpr int BOX_FIELDS = 8;   // start, end, a0, a1, a2, parent, leaf, gid
constexpr int ENT_FIELDS = 8;   // level, index, gid, start, end, a0, a1, a2

// One level of the tree: its boxes, BOX_FIELDS int32 each.
struct Level {
    int nb = 0;
    DBuf box;
};

// A cut: level-l boxes plus carried leaves of coarser levels, in Morton order.
struct Cut {
    int nc = 0;
    DBuf ent;        // int32 [nc][ENT_FIELDS]
    DBuf parent;     // int32 [nc]: entry of cut l-1 holding this entry (l >= 1)
    DBuf kid_begin;  // int32 [nc]: first entry of cut l+1 inside this entry
    DBuf kid_end;    // int32 [nc]
    DBuf pt2ent;     // int32 [n]: entry holding each sorted point
    DBuf near_ptr, near_idx;  // CSR, sorted by entry
    DBuf int_ptr, int_idx;
    DBuf s_ptr, s_idx;        // near u int, sorted (the constraint zero sets)
    int64_t n_near = 0, n_int = 0;
    int max_rows = 0;         // largest entry
};

// Graph colouring of one cut (admissible pairs) or of the leaf neighbour pairs.
struct Coloring {
    bool done = false;
    bool leaf = false;
    int level = 0;            // cut level whose pairs are coloured
    int64_t n_pairs = 0, n_vertices = 0, n_edges = 0;
    int n_colors = 0;
    const int *pair_ptr = nullptr;   // CSR of pairs by row entry (borrowed: int or near list)
    const int *pair_col = nullptr;
    DBuf pair_alpha;      // int32 [n_pairs]
    DBuf pair_T;          // int32 [n_pairs]: index of the transposed pair (beta, alpha)
    DBuf pair_vertex;     // int32 [n_pairs]
    DBuf pair_color;      // int32 [n_pairs]
    DBuf vertex_pair;     // int32 [n_vertices]: first pair of each vertex
    DBuf vertex_beta;     // int32
    DBuf vertex_color;    // int32
    DBuf vertex_degree;   // int32
    DBuf act_ptr, act_box;     // colour -> active entries (CSR, sorted)
    DBuf ent_cptr, ent_col;    // entry -> colours it is active in (CSR, sorted)
    DBuf act_rows_ptr;         // colour -> offset into act_rows (int64, chi+1)
    DBuf act_rows;             // int32: rows (sorted points) active in each colour
    int64_t n_act_rows = 0;
    // output rows of each colour: the rows I_alpha of its pairs (alpha, beta),
    // i.e. of the sample tiles Y(I_alpha, c), grouped by colour in pair order
    DBuf out_rows_ptr;         // int64 [chi + 1]
    DBuf out_rows;             // int32
    std::vector<int64_t> h_out_rows_ptr;
    int m_cols = 0;            // columns per colour: r, or m_max at the leaf
};

// Low-rank factors of one level: U_p (|I_a| x kU, row-major), V_p (|I_b| x kV),
// B_p (kU x kV, row-major) for every admissible pair p.
struct Factors {
    bool done = false;
    int64_t n_pairs = 0;
    DBuf kU, kV;              // int32
    DBuf offU, offV, offB;    // int64 element offsets
    DBuf U, V, B;
    DBuf U32, V32, B32;       // FP32 copies for the HM_MIXED_BF16X6_F32 peel (made on first use)
    DBuf U2, V2, B2;          // double-float copies for the HM_MIXED_BF16X6 peel (made on first use)
    int64_t nU = 0, nV = 0, nB = 0;
    int max_k = 0;
    // H^2 (Section 4.3): the bases are per cut entry (a box of cut l), U and V
    // hold them at eoffU / eoffV (|I_e| x k_e row-major; the pairs' offU / offV
    // point at them); eS holds S^in and S^out ([nc][2][r], the first k valid);
    // Ut / Vt hold the short bases of this cut's entries in terms of their
    // children in cut l + 1: the block of child a (k_a x k_parent, row-major)
    // at offUt[a] / offVt[a], indexed by the child entry
    bool has_bases = false;
    int nc = 0;
    DBuf ekU, ekV;            // int32 [nc]
    DBuf eoffU, eoffV;        // int64 [nc + 1]
    DBuf eS;                  // double [nc][2][r]
    DBuf Ut, Vt;
    DBuf offUt, offVt;        // int64 [nc of cut l + 1, + 1]
    int64_t nUt = 0, nVt = 0;
    int64_t sumkU = 0, sumkV = 0;  // sum of ekU / ekV over the entries
    DBuf epU, epV;            // int64 [nc + 1]: prefix sums of ekU / ekV (apply expansions)
};

struct Leaf {
    bool done = false;
    int64_t n_pairs = 0;
    DBuf offD;                // int64
    DBuf D;
    int64_t nD = 0;
    int m_max = 0;
};

// Apply metadata, built once at the end of a compression so that an apply
// needs no scan and no read back: per admissible level the offsets of every
// pair's intermediate product t (prefix sums of k_U and of k_V, in units of
// one right-hand side), and per cut the stage-2 items (box, first row) of at
// most APPLY_ROWS rows each; the leaf cut's items also serve the near field.
constexpr int APPLY_ROWS = 64;
struct ApplyPlan {
    bool ready = false;
    std::vector<DBuf> toffU, toffV;   // int64 [np + 1], index l
    std::vector<DBuf> items;          // int32 [nitems][2], index l (cut l)
    std::vector<int64_t> nitems;
    std::vector<int> maxk;            // largest k of level l
    int64_t t_max = 0;                // largest sum of k over a level's pairs (both sides)
};

struct Samples {
    int level = -100;
    int chi = 0, cols = 0;    // colours, columns per colour
    DBuf Y, Z;                // double [chi][n][cols]
};

}  // namespace hm

struct hm_ctx {
    hm_config cfg;
    cudaStream_t st = nullptr;
    int dev = -1;             // the device current at hm_create (-1: none visible)
    std::string last_error;
    int stage = 0;            // 0 created, 1 tree built, 2 compressed

    // settings of the current tree and compression (hm_tree_build's leaf size,
    // hm_compress's truncation): fixed rank (0 in tolerance mode), tolerance
    // (0 with a fixed rank), cap on k (r, or r - p and the rank cap with a
    // tolerance), and the rank argument as given (0 = none)
    int leaf_size = 0;
    int rank_fixed = 0;
    double tol = 0.0;
    int kcap = 0;
    int rank_arg = 0;

    // points
    int64_t n = 0;
    int d = 0;
    double lo[3] = {0, 0, 0};
    double side = 1.0;
    hm::DBuf xs;              // double [n][3], sorted (Morton) order; unused dims are 0
    hm::DBuf perm;            // int32 [n]: original index of sorted point i
    hm::DBuf qs;              // int32 [n][3]: grid coordinates, sorted order
    hm::DBuf xdf;             // float4 [n][2]: double-float copy of xs (mixed precision)

    int L = 0;
    std::vector<hm::Level> levels;
    std::vector<hm::Cut> cuts;
    std::vector<int> level_off;     // gid offset of each level

    std::vector<hm::Coloring> colorings;   // index l (2..L); index L+1 = leaf
    std::vector<hm::Coloring> box_colorings;  // uniform H^1: box colouring of cut l (index l)
    std::vector<hm::Factors> factors;      // index l
    hm::Leaf leaf;
    std::vector<hm::Samples> kept;         // per level when cfg.keep_samples
    hm::Samples cur;                       // the current level's samples
    hm::DBuf GO, GP;                       // current level's Gaussians [n][r]
    int gauss_level = -100;
    // uniform H^1: the colouring whose tiles the sampler, the peel and the QR
    // of the current level work on when it is not the pair colouring (the box
    // colouring of stage 1), and the sides the peel updates (1 = Y, 2 = Z)
    const hm::Coloring *cur_tiles = nullptr;
    int peel_sides = 3;

    // scratch
    hm::DBuf scratch_a, scratch_b, scratch_c, scratch_d, scan_tmp;

    // streams on which two host threads colour the levels ahead of the level
    // loop (created on first use, destroyed with the context)
    cudaStream_t color_st[2] = {nullptr, nullptr};
    hm::DBuf color_scan_tmp[2];

    hm::ApplyPlan plan;
    hm::DBuf apply_t;                 // hm_apply's intermediate products (grow-only)

    hm_info info;
    double t_sample = 0.0;
    int bb_tc_levels = 0;     // levels of the last compression sampled on the tensor cores
    int bb_fp64_levels = 0;   // levels sampled in FP64 (SIMT kernel, dense or callback operator)
    double t_tc = 0.0;        // device time of the tensor-core contraction kernels
    // CUDA events around the peel update launches of the current compression,
    // and their multiply-add counter (double-float mode)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_update;
    hm::DBuf peel_macs;
    int64_t tc_evals = 0;     // kernel entries the tensor-core sampler evaluated (padding excluded)
};

namespace hm {

// tree.cu
Err build_tree(hm_ctx *c, const double *points_dev, int64_t n);
// color.cu
Err color_cut(hm_ctx *c, int level, bool leaf);  // on c->st
Err color_cut(hm_ctx *c, int level, bool leaf, cudaStream_t st, DBuf &scan_tmp);
Err color_boxes(hm_ctx *c, int level, cudaStream_t st, DBuf &scan_tmp);  // uniform H^1, stage 1
// sample.cu
Err make_gaussians(hm_ctx *c, int level);
// uniform H^1: the Gaussian k_a x r mixes M_a of the boxes vbox[0..nv) (Philox
// side 3, keyed like G), M_a at moff[v] row-major
Err make_mix(hm_ctx *c, int level, const int *vbox, int64_t nv, const int *kbox, const int64_t *moff, double *M);
Err sample_level(hm_ctx *c, const hm_op *op, int level, bool leaf);
Err op_apply_dense_vectors(hm_ctx *c, const hm_op *op, const double *x_sorted, double *y_sorted,
                           int nrhs, int trans);
// sample_tc.cu
Err sample_tc(hm_ctx *c, int level, int kernel);
Err sample_leaf_mixed(hm_ctx *c, int kernel);
bool tc_supported(const hm_ctx *c);
// peel.cu, peel_mixed.cu
Err peel_level(hm_ctx *c, int level, bool leaf);
Err peel_level_mixed(hm_ctx *c, int level, bool leaf);  // FP32 products (HM_MIXED_BF16X6_F32)
Err peel_level_fp64(hm_ctx *c, int level, bool leaf);   // the same structure in FP64
Err peel_level_df(hm_ctx *c, int level, bool leaf);     // double-float products (HM_MIXED_BF16X6)
// basis.cu
Err bases_and_cores(hm_ctx *c, int level);
// FP64 column-pivoted QR of tiles base[color[p]][I_box[p]][0:r] in place (the
// dispatch of bases_and_cores' FP64 modes); k <= tile_cap[p] (nullable) and
// <= cap; fixed rank when rank > 0, else tolerance tol; ranks into kout
Err qr_tiles_fp64(hm_ctx *c, int level, const int *tile_box, const int *tile_color, const int *tile_cap, int64_t nt,
                  int max_rows, double *base, int cap, int rank, double tol, int *kout);
Err extract_leaf(hm_ctx *c);
// uniform.cu
Err uniform_level(hm_ctx *c, const hm_op *op, int level, double *phase_secs);
// per-pair tables of a level whose bases are stored per box (uniform H^1, H^2):
// pair p = (a, b) takes k_U, offset of box vid[a] and k_V, offset of box
// vid[b]; then B_p = T^T V_b from the stage-2 tiles T = Z(I_b, 0:k_a)
Err box_pairs_and_cores(hm_ctx *c, int level, const int *vid, const int *kUb, const int *kVb,
                        const int64_t *offUb, const int64_t *offVb);
// W(I_b, :) = sum over the entries t of int(b) of Z[colour of pair t](I_b, 0:k_a) M_a
// (a = int_idx[t], looked up through vid) for the boxes vbox[0..nv); W is [n][r]
Err mix_sum(hm_ctx *c, int level, const int *vbox, int64_t nv, const int *vid, const int *kU, const int64_t *moff,
            const double *M, double *W);
// h2.cu
Err h2_level(hm_ctx *c, const hm_op *op, int level, double *phase_secs);
Err h2_finish(hm_ctx *c);  // after the leaf: keep the long bases of cut L and the short bases
Err apply_h2_into(hm_ctx *c, const double *x_sorted, double *y_sorted, int nrhs, int trans, double *t);
int64_t h2_scratch_elems(const hm_ctx *c);  // t of apply_h2_into, per right-hand side
// apply.cu: the leaf neighbour blocks, y += D x (or D^* x), on c->st
Err apply_near(hm_ctx *c, const double *x_sorted, double *y_sorted, int nrhs, int trans);
// apply.cu
Err build_apply_plan(hm_ctx *c);
// y = A~ x (trans 0) or A~^* x for row-major sorted [n][nrhs] vectors; t holds
// plan.t_max * nrhs doubles of scratch.  Asynchronous on c->st.
Err apply_sorted_into(hm_ctx *c, const double *x_sorted, double *y_sorted, int nrhs, int trans, double *t);
Err apply_sorted(hm_ctx *c, const double *x_sorted, double *y_sorted, int nrhs, int trans);
Err permute_rows(hm_ctx *c, const double *in, double *out, int nrhs, bool to_sorted);

}  // namespace hm
