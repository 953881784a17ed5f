// Host-side basis construction (see basis.cpp).
#pragma once
#include "common.cuh"

namespace aderdg {
int gauss_legendre01(int n, double *x, double *w);
int build_basis(int N, Basis &b);
double default_alpha(int N);
// fill kp.od / kp.of from kp.b
void fill_ops(KParams &kp);
}  // namespace aderdg
