// Kernel sets for subspace dimensions k = 13 .. 16 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_kernels.cuh"

namespace prost {

void register_ops_k13_16(const KernelOps **table)
{
    table[13] = Ops<13>::table();
    table[14] = Ops<14>::table();
    table[15] = Ops<15>::table();
    table[16] = Ops<16>::table();
}

} // namespace prost
