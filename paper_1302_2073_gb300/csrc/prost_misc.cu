// Kernels that do not depend on the subspace dimension: the seeded Gaussian
// initial subspace and the layout conversions of the ABI.
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "prost_device.h"

namespace prost {

// splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Standard normal draw number `ctr` of stream `seed` (Box-Muller on two
// 24-bit uniforms in (0, 1)).
__device__ __forceinline__ float gauss(uint64_t seed, uint64_t ctr)
{
    const uint64_t h1 = splitmix64(seed ^ splitmix64(2 * ctr));
    const uint64_t h2 = splitmix64(seed ^ splitmix64(2 * ctr + 1));
    const float u1 = ((float)(h1 >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = ((float)(h2 >> 40) + 0.5f) * (1.0f / 16777216.0f);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// (channel, pixel, column) of element i of the tile-blocked stored subspace
__device__ __forceinline__ void u_coords(const DevParams &prm, int64_t i, int64_t &c, int64_t &q, int &j)
{
    const int64_t blk = i / ((int64_t)prm.k * TILE_P);
    const int64_t rem = i - blk * prm.k * TILE_P;
    j = (int)(rem / TILE_P);
    c = blk / prm.npt;
    q = (blk - c * prm.npt) * TILE_P + (rem - (int64_t)j * TILE_P);
}

// U_st = N(0, 1)/sqrt(m) per entry (padding rows 0); its Cholesky-QR (run
// next) gives the orthonormal factor of a random m x k matrix (Section 3.4).
__device__ __forceinline__ void store(float *p, float v) { *p = v; }
__device__ __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

template <typename UT>
__global__ void k_init_gauss(UT *U, DevParams prm, uint64_t seed)
{
    const int64_t n = (int64_t)prm.C * prm.Pp * prm.k;
    const float s = rsqrtf((float)((double)prm.C * (double)prm.P));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c, q;
        int j;
        u_coords(prm, i, c, q, j);
        float v = 0.f;
        if (q < prm.P) v = s * gauss(seed, (uint64_t)((c * prm.P + q) * prm.k + j));
        store(U + i, v);
    }
}

// m x k row-major -> tile-blocked stored layout
template <typename UT>
__global__ void k_import_u(const float *Urow, UT *U, DevParams prm)
{
    const int64_t n = (int64_t)prm.C * prm.Pp * prm.k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c, q;
        int j;
        u_coords(prm, i, c, q, j);
        store(U + i, q < prm.P ? Urow[(c * prm.P + q) * prm.k + j] : 0.f);
    }
}

__global__ void k_import_labels(const uint8_t *src, uint8_t *labels, DevParams prm)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < prm.Pp;
         q += (int64_t)gridDim.x * blockDim.x)
        labels[q] = (src && q < prm.P && src[q]) ? 1 : 0;
}

__global__ void k_reset_fold(KState *ks, int k, int force)
{
    const bool due = force || ks->frames_since_rebase >= REBASE_EVERY;
    __syncthreads(); // every thread has read the counter before it restarts
    if (threadIdx.x == 0) ks->rebased = due ? 1 : 0;
    if (!due) return;
    if (threadIdx.x == 0) ks->frames_since_rebase = 0;
    for (int q = threadIdx.x; q < KMAX * KMAX; q += blockDim.x) {
        const int i = q / KMAX, j = q % KMAX;
        ks->R[q] = ks->T[q] = (i == j) ? 1.0 : 0.0;
        if (i < k && j < k) ks->Tf[i * k + j] = (i == j) ? 1.f : 0.f;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) ks->yf[i] = (float)ks->y[i];
}

static int grid_for(int64_t n)
{
    const int64_t b = (n + THREADS - 1) / THREADS;
    return (int)(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

cudaError_t launch_init_gauss(void *U, DevParams prm, uint64_t seed, cudaStream_t s)
{
    const int g = grid_for((int64_t)prm.C * prm.Pp * prm.k);
    if (prm.ubf16)
        k_init_gauss<<<g, THREADS, 0, s>>>(static_cast<__nv_bfloat16 *>(U), prm, seed);
    else
        k_init_gauss<<<g, THREADS, 0, s>>>(static_cast<float *>(U), prm, seed);
    return cudaGetLastError();
}

cudaError_t launch_import_u(const float *Urow, void *U, DevParams prm, cudaStream_t s)
{
    const int g = grid_for((int64_t)prm.C * prm.Pp * prm.k);
    if (prm.ubf16)
        k_import_u<<<g, THREADS, 0, s>>>(Urow, static_cast<__nv_bfloat16 *>(U), prm);
    else
        k_import_u<<<g, THREADS, 0, s>>>(Urow, static_cast<float *>(U), prm);
    return cudaGetLastError();
}

cudaError_t launch_reset_fold(KState *ks, DevParams prm, int force, cudaStream_t s)
{
    k_reset_fold<<<1, 256, 0, s>>>(ks, prm.k, force);
    return cudaGetLastError();
}

cudaError_t launch_import_labels(const uint8_t *src, uint8_t *labels, DevParams prm, cudaStream_t s)
{
    k_import_labels<<<grid_for(prm.Pp), THREADS, 0, s>>>(src, labels, prm);
    return cudaGetLastError();
}

} // namespace prost
