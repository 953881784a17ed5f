// The compiled (PDE, d, N) kernel instances: 2D advection and Euler for
// N = 1..7, 3D advection, Euler and elasticity for N = 1..4, the
// diffuse-interface system in 2D for N = 2..4 and in 3D for N = 2, 3.  Each entry
// X(tag, d, N) is built twice (double and float) from inst.cu; the build
// script reads this list.
#pragma once
#define ADERDG_INSTANCES(X) \
    X(advection, 2, 1) X(advection, 2, 2) X(advection, 2, 3) X(advection, 2, 4) \
    X(advection, 2, 5) X(advection, 2, 6) X(advection, 2, 7) \
    X(euler, 2, 1) X(euler, 2, 2) X(euler, 2, 3) X(euler, 2, 4) \
    X(euler, 2, 5) X(euler, 2, 6) X(euler, 2, 7) \
    X(advection, 3, 1) X(advection, 3, 2) X(advection, 3, 3) X(advection, 3, 4) \
    X(euler, 3, 1) X(euler, 3, 2) X(euler, 3, 3) X(euler, 3, 4) \
    X(elastic, 3, 1) X(elastic, 3, 2) X(elastic, 3, 3) X(elastic, 3, 4) \
    X(diffuse, 2, 2) X(diffuse, 2, 3) X(diffuse, 2, 4) X(diffuse, 3, 2) X(diffuse, 3, 3)
