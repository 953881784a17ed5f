// Tile-shape selection for the per-element kernels (see tune.cu).
#pragma once

#include <algorithm>
#include <cstdlib>
#include "common.cuh"

namespace aderdg {

// A tile-shape request is a shape index or ADERDG_SHAPE_AUTOTUNE (-1).
inline bool valid_shape_request(int r, int count) { return r == -1 || (r >= 0 && r < count); }
inline bool valid_shape_requests(int pred, int corr)
{
    return valid_shape_request(pred, NSHAPE_P) && valid_shape_request(corr, NSHAPE_C);
}

// Kernel set of one (PDE, d, N, precision), or NULL if none is compiled.
const KernelSet *lookup_kernels(int pde, int dim, int N, int prec);

// Copy of *ks launching the requested predictor / corrector shapes.  A
// request is a shape index (0 .. NSHAPE_P-1 / NSHAPE_C-1) or ADERDG_SHAPE_AUTOTUNE, which
// takes the fastest shape measured for this (PDE, d, N, precision) on the
// current device: from the process-wide table, else from the text file
// `cache` (may be NULL), else by timing every shape (and appending the
// result to `cache`).  Opts the chosen kernels in to their dynamic shared
// memory.  extrap selects the predictor variant of the extrapolation and
// CERK guesses (same shapes).  Returns an ADERDG_* status.
int resolve_shapes(const KernelSet *ks, int pde, int dim, int N, int prec, const PdeParams &pp, int pred_req,
                   int corr_req, const char *cache, bool extrap, KernelSet *out);

// The subcell limiter's kernels for a step of precision prec (Sec. 2.3):
// detection and the subcell scheme of the FP64 instance (they work on the
// FP64 state in both precisions) and the coupling of the step's own
// precision, with their dynamic shared memory opted in; keep selects the
// extremes kernel of solves that keep subcell data.  Returns ADERDG_OK,
// or an ADERDG_* status with *why set to the reason.
struct LimKernels {
    void (*minmax)(KParams), (*detect)(KParams), (*fv)(KParams), (*couple)(KParams);
    size_t smem, smem_w;  // per CTA: fv / couple / init, and minmax / detect
    int mm_epw;           // elements per warp and pass of minmax (grid: elements / (4 mm_epw))
    unsigned minmax_grid(long long elems) const
    {
        const long long per_cta = 4LL * mm_epw;
        return (unsigned)std::min<long long>((elems + per_cta - 1) / per_cta, 152LL * 16);
    }
    void (*init)(KParams);  // kept subcell data: the state of uploaded subcell averages
};
int limiter_kernels(int pde, int dim, int N, int prec, int guess, bool keep, LimKernels *out, const char **why);

// Doubles the limiter keeps per troubled element for its neighbours'
// coupling (SolveDesc::lim_fb: the subcell fluxes of its 2d faces), and the
// number of such slots of a solve of E elements: all elements where that
// takes at most 256 MB, else as many as fit; the environment variable
// ADERDG_LIMITER_FLUX_SLOTS lowers the count (0: none).  The coupling forms
// the fluxes of troubled elements beyond the slots itself.
inline long long limiter_flux_doubles(int dim, int N, int m, bool ncp)
{
    long long nline = 1;
    for (int k = 0; k < dim - 1; ++k) nline *= 2 * N + 1;
    return 2LL * dim * nline * (ncp ? 2 * m : m);
}
inline long long limiter_flux_slots(long long E, int dim, int N, int m, bool ncp)
{
    const long long per = limiter_flux_doubles(dim, N, m, ncp) * 8;
    long long slots = std::min<long long>(E, std::max<long long>(1, (256LL << 20) / per));
    if (const char *env = std::getenv("ADERDG_LIMITER_FLUX_SLOTS")) {
        const long long v = std::atoll(env);
        if (v >= 0) slots = std::min(slots, v);
    }
    return slots;
}

}  // namespace aderdg
