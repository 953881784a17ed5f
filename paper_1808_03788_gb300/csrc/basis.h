// Host-side basis construction (see basis.cpp).
#pragma once
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
// derived constants P.c / P.cf of PDE kind `kind` from P.p (see PdeParams)
void fill_pde_consts(int kind, PdeParams &P);
// fill kp.od / kp.of from kp.b
void fill_ops(KParams &kp);
}  // namespace aderdg
