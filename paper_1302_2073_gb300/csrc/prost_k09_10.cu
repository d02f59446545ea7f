// Kernel sets for subspace dimensions k = 9 and 10, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k09_10(const KernelOps **f32, const KernelOps **bf16)
{
    f32[9] = kernel_table<9, float>();
    bf16[9] = kernel_table<9, __nv_bfloat16>();
    f32[10] = kernel_table<10, float>();
    bf16[10] = kernel_table<10, __nv_bfloat16>();
}

} // namespace prost
