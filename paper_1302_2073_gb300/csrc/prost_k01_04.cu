// Kernel sets for subspace dimensions k = 1 .. 4 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k01_04(const KernelOps **table)
{
    table[1] = kernel_table<1>();
    table[2] = kernel_table<2>();
    table[3] = kernel_table<3>();
    table[4] = kernel_table<4>();
}

} // namespace prost
