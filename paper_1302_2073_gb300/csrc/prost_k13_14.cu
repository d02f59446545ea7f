// Kernel sets for subspace dimensions k = 13 and 14, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k13_14(const KernelOps **f32, const KernelOps **bf16)
{
    f32[13] = kernel_table<13, float>();
    bf16[13] = kernel_table<13, __nv_bfloat16>();
    f32[14] = kernel_table<14, float>();
    bf16[14] = kernel_table<14, __nv_bfloat16>();
}

} // namespace prost
