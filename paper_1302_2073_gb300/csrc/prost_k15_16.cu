// Kernel sets for subspace dimensions k = 15 and 16, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k15_16(const KernelOps **f32, const KernelOps **bf16)
{
    f32[15] = kernel_table<15, float>();
    bf16[15] = kernel_table<15, __nv_bfloat16>();
    f32[16] = kernel_table<16, float>();
    bf16[16] = kernel_table<16, __nv_bfloat16>();
}

} // namespace prost
