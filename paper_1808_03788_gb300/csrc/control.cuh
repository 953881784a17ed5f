// Device-side CFL step of one solve (Sec. 3): dt = alpha / sum_d lambda_d^max / dx_d
// from the maxima the corrector (or k_cfl) accumulated for the current
// state, clipped so that t lands exactly on t_end; consumes the maxima.
#pragma once

#include "common.cuh"

namespace aderdg {

__device__ __forceinline__ void dt_update(Control *c)
{
    c->lim_count = 0u;   // the last step's troubled list is consumed (subcell limiter)
    c->dt_prev = c->dt;  // the step just taken (0 if none)
    const double t = c->t;
    if (!(t < c->t_end) || (c->flags & FLAG_NONFINITE)) {
        c->dt = 0.0;
        if (!(t < c->t_end)) c->flags |= FLAG_DONE;
        return;
    }
    c->flags &= ~FLAG_DONE;
    double S = 0.0;
    for (int d = 0; d < c->dim; ++d) {
        const double lam = __longlong_as_double((long long)c->lam_acc[d]);
        c->lam_used[d] = lam;
        S += lam * c->inv_dx[d];
    }
    const double dtc = c->alpha / S;
    double dt, tn;
    if (t + dtc >= c->t_end) { dt = c->t_end - t; tn = c->t_end; }
    else { dt = dtc; tn = t + dtc; }
    if (!(dt > 0.0) || !isfinite(dt)) {  // non-finite maxima: stop, flag it
        c->dt = 0.0;
        c->flags |= FLAG_NONFINITE;
        return;
    }
    c->dt = dt;
    c->t = tn;
    c->step += 1;
    for (int d = 0; d < 3; ++d) c->lam_acc[d] = 0ull;
}

}  // namespace aderdg
