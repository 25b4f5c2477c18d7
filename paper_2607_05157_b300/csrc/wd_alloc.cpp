// Samples per level of a multilevel Monte Carlo estimator (Sec. 2, Eq. 6).
//
// Minimising the cost sum_l N_l C_l under the variance constraint
// sum_l V_l / N_l = eps^2 (Lagrange: N_l proportional to sqrt(V_l / C_l))
// gives N_l = eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i).  The counts are
// rounded up, so the variance stays within the target.
#include <math.h>
#include <stdint.h>

#include "../../include/wd.h"

namespace wd { void set_error(const char *fmt, ...); }

extern "C" int mlmc_allocate(int L, const double *V, const double *C, double eps, int64_t *N_out) {
    if (L < 1 || !V || !C || !N_out || !(eps > 0) || !isfinite(eps)) {
        wd::set_error("mlmc_allocate: bad argument");
        return WD_EINVAL;
    }
    double s = 0.0;
    for (int l = 0; l < L; ++l) {
        if (!(V[l] >= 0) || !(C[l] > 0) || !isfinite(V[l]) || !isfinite(C[l])) {
            wd::set_error("mlmc_allocate: level %d needs V >= 0 and C > 0", l);
            return WD_EINVAL;
        }
        s += sqrt(V[l] * C[l]);
    }
    for (int l = 0; l < L; ++l) {
        const double n = sqrt(V[l] / C[l]) * s / (eps * eps);
        const double r = ceil(n - 1e-9 * n);      // the formula's rounding noise must not add a sample
        if (!(r < 4.6e18)) {
            wd::set_error("mlmc_allocate: level %d needs more than 2^62 samples", l);
            return WD_EINVAL;
        }
        N_out[l] = r < 1.0 ? 1 : (int64_t)r;
    }
    return WD_OK;
}
