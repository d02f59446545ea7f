// Kernel sets for subspace dimensions k = 1 .. 4 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_kernels.cuh"

namespace prost {

void register_ops_k01_04(const KernelOps **table)
{
    table[1] = Ops<1>::table();
    table[2] = Ops<2>::table();
    table[3] = Ops<3>::table();
    table[4] = Ops<4>::table();
}

} // namespace prost
