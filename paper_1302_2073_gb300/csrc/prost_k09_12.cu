// Kernel sets for subspace dimensions k = 9 .. 12 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k09_12(const KernelOps **table)
{
    table[9] = kernel_table<9>();
    table[10] = kernel_table<10>();
    table[11] = kernel_table<11>();
    table[12] = kernel_table<12>();
}

} // namespace prost
