// Coarse 9-point block stencil on tensor cores (row a8).  Placeholder until
// the tcgen05 kernel lands: reports that no tensor-core operand exists, so
// the coarse solves use the FP32 CUDA-core stencil.
#include "wd_internal.h"

namespace wd {
bool coarse_tc_ok(wd_ctx *) { return false; }
int coarse_tc_build(wd_ctx *) { return WD_OK; }
int coarse_tc_apply(wd_ctx *, const void *, float *, int) { set_error("tensor-core coarse stencil not built"); return WD_ENOTSUP; }
}  // namespace wd
