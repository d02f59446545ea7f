// Kernel sets for subspace dimensions k = 5 .. 8 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k05_08(const KernelOps **table)
{
    table[5] = kernel_table<5>();
    table[6] = kernel_table<6>();
    table[7] = kernel_table<7>();
    table[8] = kernel_table<8>();
}

} // namespace prost
