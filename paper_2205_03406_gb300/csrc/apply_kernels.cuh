// Kernels and level table of the apply (apply.cu), shared with the
// allocation-free apply entry point (apply_noalloc.cu).
#pragma once

#include "ctx.cuh"

namespace hm {

struct ApplyLevel {
    const int *pt2ent, *ent, *int_ptr, *int_idx, *pairT;
    const int *kU, *kV;
    const int64_t *offU, *offV;
    const double *U, *V;
    const int64_t *toff;
    const double *tq;
};

__global__ void k_apply_stage1(const int *pair_alpha, const int *pair_col, const int *ent, int64_t np,
                               const int *kU, const int *kV, const int64_t *offU, const int64_t *offV,
                               const int64_t *offB, const double *U, const double *V, const double *B,
                               const double *x, int nrhs, int trans, const int64_t *toff, double *tq);
__global__ void k_apply_stage2(const int *ent_leaf, int nleaf, const ApplyLevel *lv, int nlev, const int *near_ptr,
                               const int *near_idx, const int *leaf_pairT, const int64_t *offD, const double *D,
                               const double *x, int nrhs, int trans, double *y);
__global__ void k_toff_sizes(const int *kU, const int *kV, int64_t np, int nrhs, int trans, int64_t *sz);

}  // namespace hm
