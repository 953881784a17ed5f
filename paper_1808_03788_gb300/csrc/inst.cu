// One kernel instance, compiled once per entry of instances.h and
// precision: the build defines ADERDG_INST_NAME (the accessor's name),
// ADERDG_INST_PDE (the PDE type), ADERDG_INST_DIM, ADERDG_INST_N and
// ADERDG_INST_T (double or float).
#include "kernels.cuh"

#if !defined(ADERDG_INST_NAME) || !defined(ADERDG_INST_PDE) || !defined(ADERDG_INST_DIM) || \
    !defined(ADERDG_INST_N) || !defined(ADERDG_INST_T)
#error "inst.cu is compiled by the build script with the instance's -D definitions"
#endif

namespace aderdg {

const KernelSet *ADERDG_INST_NAME()
{
    return &KS<ADERDG_INST_PDE, ADERDG_INST_DIM, ADERDG_INST_N, ADERDG_INST_T>::value;
}

}  // namespace aderdg
