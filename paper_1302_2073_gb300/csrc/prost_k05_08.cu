// Kernel sets for subspace dimensions k = 5 .. 8 (one translation unit per
// range so that the build compiles them in parallel).
#include "prost_kernels.cuh"

namespace prost {

void register_ops_k05_08(const KernelOps **table)
{
    table[5] = Ops<5>::table();
    table[6] = Ops<6>::table();
    table[7] = Ops<7>::table();
    table[8] = Ops<8>::table();
}

} // namespace prost
