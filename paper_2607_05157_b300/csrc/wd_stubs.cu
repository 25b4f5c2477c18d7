// Entry points whose implementation lands in later files; they report
// WD_ENOTSUP until then.
#include "wd_internal.h"
using namespace wd;
void wd_mg_free(wd_ctx *) {}
namespace wd {
int mlmc2_estimate(wd_ctx *, int, int, uint64_t, int, int, int, double, double *, double *, int64_t *, double *) {
    set_error("MLMC2 needs the multigrid module");
    return WD_ENOTSUP;
}
}
extern "C" int wd_mlmc_level2_samples(wd_ctx *, double *, int) { return WD_ENOTSUP; }
extern "C" int wd_mg_setup(wd_ctx *, const double *, int, const int *, int, uint64_t) { return WD_ENOTSUP; }
extern "C" int wd_coarse_apply(wd_ctx *, const double *, double *, int, int) { return WD_ENOTSUP; }
extern "C" int wd_restrict(wd_ctx *, const double *, double *, int) { return WD_ENOTSUP; }
extern "C" int wd_prolong(wd_ctx *, const double *, double *, int) { return WD_ENOTSUP; }
extern "C" int wd_coarse_solve(wd_ctx *, const double *, double *, int, double, int, int, double *) { return WD_ENOTSUP; }
extern "C" int wd_link_force(wd_ctx *, const double *, const double *, int, double *, double *, int) { return WD_ENOTSUP; }
