// Mixed-precision black-box contraction on the tcgen05 tensor cores (placeholder
// until the kernel lands; the FP64 path is used meanwhile).
#include "ctx.cuh"

namespace hm {

bool tc_supported(const hm_ctx *) { return false; }

Err sample_tc(hm_ctx *, int, int) { return fail(HM_ENOTSUP, "tcgen05 sample not built"); }

}  // namespace hm
