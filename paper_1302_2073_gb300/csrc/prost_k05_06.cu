// Kernel sets for subspace dimensions k = 5 and 6, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k05_06(const KernelOps **f32, const KernelOps **bf16)
{
    f32[5] = kernel_table<5, float>();
    bf16[5] = kernel_table<5, __nv_bfloat16>();
    f32[6] = kernel_table<6, float>();
    bf16[6] = kernel_table<6, __nv_bfloat16>();
}

} // namespace prost
