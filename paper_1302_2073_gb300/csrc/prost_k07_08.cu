// Kernel sets for subspace dimensions k = 7 and 8, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k07_08(const KernelOps **f32, const KernelOps **bf16)
{
    f32[7] = kernel_table<7, float>();
    bf16[7] = kernel_table<7, __nv_bfloat16>();
    f32[8] = kernel_table<8, float>();
    bf16[8] = kernel_table<8, __nv_bfloat16>();
}

} // namespace prost
