// Kernel sets for subspace dimensions k = 1 and 2, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k01_02(const KernelOps **f32, const KernelOps **bf16)
{
    f32[1] = kernel_table<1, float>();
    bf16[1] = kernel_table<1, __nv_bfloat16>();
    f32[2] = kernel_table<2, float>();
    bf16[2] = kernel_table<2, __nv_bfloat16>();
}

} // namespace prost
