// Kernel instantiations for 2D Euler equations, N = 1..7.
#include "kernels.cuh"

namespace aderdg {

const KernelSet *ks_euler2d(int N, int prec)
{
#define ADERDG_CASE(NN) \
    case NN: return prec ? &KS<Euler<2>, 2, NN, float>::value : &KS<Euler<2>, 2, NN, double>::value;
    switch (N) {
        ADERDG_CASE(1)
        ADERDG_CASE(2)
        ADERDG_CASE(3)
        ADERDG_CASE(4)
        ADERDG_CASE(5)
        ADERDG_CASE(6)
        ADERDG_CASE(7)
    default: return nullptr;
    }
#undef ADERDG_CASE
}

}  // namespace aderdg
