// Kernel sets for subspace dimensions k = 11 and 12, float32 and bfloat16
// storage (one translation unit per pair so that the build compiles them in
// parallel).
#include "prost_frame.cuh"

namespace prost {

void register_ops_k11_12(const KernelOps **f32, const KernelOps **bf16)
{
    f32[11] = kernel_table<11, float>();
    bf16[11] = kernel_table<11, __nv_bfloat16>();
    f32[12] = kernel_table<12, float>();
    bf16[12] = kernel_table<12, __nv_bfloat16>();
}

} // namespace prost
