// Level table and entry point of the apply kernels (apply.cu), shared with the
// allocation-free apply entry point (apply_noalloc.cu).
#pragma once

#include "ctx.cuh"

namespace hm {

constexpr int APPLY_NB = 4;   // right-hand sides per CTA (grid dimension y)
constexpr int APPLY_UC = 64;  // neighbour points per shared-memory chunk of the near field

// one admissible level as the apply kernels read it
struct ApplyLevel {
    const int *ent, *int_ptr, *int_idx, *pair_alpha, *pairT;
    const int *kU, *kV;
    const int64_t *offU, *offV, *offB;
    const double *U, *V, *B;
    const int64_t *toffU, *toffV;  // t offsets (units of one right-hand side), forward / adjoint
};

}  // namespace hm
