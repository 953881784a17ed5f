// Kernel instantiations for 3D linear advection, N = 1..4.
#include "kernels.cuh"

namespace aderdg {

const KernelSet *ks_advection3d(int N, int prec)
{
#define ADERDG_CASE(NN) \
    case NN: return prec ? &KS<Advection<3>, 3, NN, float>::value : &KS<Advection<3>, 3, NN, double>::value;
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
