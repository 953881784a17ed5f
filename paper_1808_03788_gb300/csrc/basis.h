// Host-side basis construction (see basis.cpp).
#pragma once
#include "../../include/aderdg.h"
#include "common.cuh"

namespace aderdg {
int gauss_legendre01(int n, double *x, double *w);
int build_basis(int N, Basis &b);
double default_alpha(int N);
// Picard iterations after an initial guess (0 trivial, 1 second order, 2
// third order, 4 CERK): max(1, N + 1 - degree of the guess in time); 3
// (extrapolation, degree N): 2
int default_picard(int N, int guess);
// number of variables of PDE kind `kind` in dimension dim (-1: unknown)
int pde_nvar(int kind, int dim);
// Checks of a problem before any kernel sees it, shared by every entry
// point that takes a mesh.  check_mesh: dim 2 or 3, a PDE kind defined in
// that dimension, 1 <= cells[d] <= 2^30 and E = prod cells[d] <= 2^31
// (checked factor by factor, so the product cannot overflow), hi > lo;
// sets *E.  check_pde_params: Euler gamma > 1; elasticity rho > 0, mu > 0,
// lambda + 2 mu > 0; advection kappa >= 0 (all finite).  check_problem:
// both.  Each returns ADERDG_OK, or ADERDG_E_INVAL with *why set.
int check_mesh(const aderdg_mesh_t &mesh, int kind, long long *E, const char **why);
int check_pde_params(const aderdg_pde_t &pde, const char **why);
int check_problem(const aderdg_mesh_t &mesh, const aderdg_pde_t &pde, long long *E, const char **why);
// The FP32 lift coefficients of d (from its inv_dx and the degree-N basis),
// the same values as float(inv_dx[d] * inv_w[k] * F0|F1[k]) in double.
void fill_desc_lift(SolveDesc &d, int N);
// derived constants P.c / P.cf of PDE kind `kind` from P.p (see PdeParams)
void fill_pde_consts(int kind, PdeParams &P);
// fill kp.od / kp.of from kp.b
void fill_ops(KParams &kp);
}  // namespace aderdg
