// Entry points whose implementation lands in later files; they report
// WD_ENOTSUP until then.
#include "wd_internal.h"
using namespace wd;
extern "C" int wd_link_force(wd_ctx *, const double *, const double *, int, double *, double *, int) { return WD_ENOTSUP; }
