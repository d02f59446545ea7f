// Kernel sets for subspace dimensions k = 13 .. 16 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k13_16(const KernelOps **table)
{
    table[13] = kernel_table<13>();
    table[14] = kernel_table<14>();
    table[15] = kernel_table<15>();
    table[16] = kernel_table<16>();
}

} // namespace prost
