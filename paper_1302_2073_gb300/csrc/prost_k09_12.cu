// Kernel sets for subspace dimensions k = 9 .. 12 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_kernels.cuh"

namespace prost {

void register_ops_k09_12(const KernelOps **table)
{
    table[9] = Ops<9>::table();
    table[10] = Ops<10>::table();
    table[11] = Ops<11>::table();
    table[12] = Ops<12>::table();
}

} // namespace prost
