// Kernel instantiations for 3D Euler equations, N = 1..4.
#include "kernels.cuh"

namespace aderdg {

const KernelSet *ks_euler3d(int N, int prec)
{
#define ADERDG_CASE(NN) \
    case NN: return prec ? &KS<Euler<3>, 3, NN, float>::value : &KS<Euler<3>, 3, NN, double>::value;
    switch (N) {
        ADERDG_CASE(1)
        ADERDG_CASE(2)
        ADERDG_CASE(3)
        ADERDG_CASE(4)
    default: return nullptr;
    }
#undef ADERDG_CASE
}

}  // namespace aderdg
