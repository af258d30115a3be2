// Device side of the Sec. III-C stopping test, shared by every engine.
#pragma once

#include <cmath>

#include "opf_internal.h"

namespace opf {

// Stopping test of Sec. III-C (plus the absolute gate on pres).
__device__ __forceinline__ void apply_test(DevStatus *st, const double s[6], double rho, long long add_iters) {
    const double pres = sqrt(s[0]);
    const double dres = rho * sqrt(s[1]);
    const double eprim = fmax(sqrt(s[2]), sqrt(s[3]));
    const double edual = sqrt(s[4]);
    st->iter += add_iters;
    st->pres = pres;
    st->dres = dres;
    st->eprim = eprim;
    st->edual = edual;
    st->obj = s[5];
    bool finite = true;
    for (int q = 0; q < 6; ++q) finite = finite && isfinite(s[q]);
    st->numeric = finite ? 0 : 1;
    st->converged = (finite && pres <= st->eps_rel * eprim && dres <= st->eps_rel * edual &&
                     pres <= st->eps_abs_pres) ? 1 : 0;
    if (st->converged || st->numeric || st->iter >= st->max_iter) st->done = 1;
}

}  // namespace opf
