// Kernel sets for subspace dimensions k = 3 and 4, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k03_04(const KernelOps **f32, const KernelOps **bf16)
{
    f32[3] = kernel_table<3, float>();
    bf16[3] = kernel_table<3, __nv_bfloat16>();
    f32[4] = kernel_table<4, float>();
    bf16[4] = kernel_table<4, __nv_bfloat16>();
}

} // namespace prost
