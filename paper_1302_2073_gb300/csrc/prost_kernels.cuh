// Building blocks of the CUDA path (arXiv:1302.2073, Section 3.3) for sm_103a:
// vector loads, deterministic reductions (per-thread FP32 sums, a split warp
// reduction, per-CTA partial rows in fixed slots, a fixed-order Kahan sum over
// CTAs), the FP64 Cholesky-QR of a Gram matrix, and the kernels that compute
// the Gram of a stored subspace (after initialisation or import) and export its
// orthonormal representative.  The per-frame kernel is in prost_frame.cuh.
#pragma once

#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "prost_device.h"

namespace prost {

// rows (pixels) per thread of the Gram kernel
template <int K> struct Cfg {
    static constexpr int VW = K <= 6 ? 4 : (K <= 12 ? 2 : 1);
};

// index of (j, l), j <= l, in a packed upper-triangular K x K matrix
template <int K> __host__ __device__ constexpr int tri(int j, int l)
{
    return j * K - (j * (j - 1)) / 2 + (l - j);
}

constexpr unsigned FULL = 0xffffffffu;

// ---- stored-subspace element types -----------------------------------------

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float ld_u(const float *p) { return *p; }
__device__ __forceinline__ float ld_u(const bf16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldg_u(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldg_u(const bf16 *p) { return __bfloat162float(__ldg(p)); }
// L2-only loads (streamed rows): one entry, or the entries of two consecutive
// rows (8 bytes of float32, 4 bytes of bfloat16 at an even row)
__device__ __forceinline__ float ldcg_u(const float *p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_u(const bf16 *p)
{
    return __uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short *>(p)) << 16);
}
__device__ __forceinline__ float2 ldcg_u2(const float *p) { return __ldcg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 ldcg_u2(const bf16 *p)
{
    const uint32_t w = __ldcg(reinterpret_cast<const unsigned int *>(p));
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
// round to nearest (imports, rebase)
__device__ __forceinline__ void st_u(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_u(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Counter-based 32-bit hash (the PCG output permutation applied to one LCG
// step; Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 2020).
__device__ __forceinline__ uint32_t pcg_hash(uint32_t x)
{
    const uint32_t state = x * 747796405u + 2891336453u;
    const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

// v rounded to bfloat16 stochastically with the 16 random bits r: the bits
// below the bfloat16 mantissa are a fraction of an ulp of |v|, and adding a
// uniform 16-bit number before truncating rounds |v| up with exactly that
// probability, so the rounding is unbiased (and zero stays zero).
__device__ __forceinline__ float round_bf16_sr(float v, uint32_t r)
{
    const uint32_t b = (__float_as_uint(v) + (r & 0xffffu)) & 0xffff0000u;
    return __uint_as_float(b);
}

// ---- vector loads and stores ------------------------------------------------

template <int VW> struct VL;

template <> struct VL<4> {
    static __device__ __forceinline__ void ldu(const float *p, float (&o)[4])
    {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void ldu_rw(const float *p, float (&o)[4])
    {
        float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void stu(float *p, const float (&o)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
    static __device__ __forceinline__ void ldlab(const uint8_t *p, uint8_t (&o)[4])
    {
        uchar4 v = *reinterpret_cast<const uchar4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void stlab(uint8_t *p, const uint8_t (&o)[4])
    {
        *reinterpret_cast<uchar4 *>(p) = make_uchar4(o[0], o[1], o[2], o[3]);
    }
    static __device__ __forceinline__ void ldx(const uint8_t *p, float (&o)[4])
    {
        uchar4 v = __ldg(reinterpret_cast<const uchar4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void ldx(const float *p, float (&o)[4])
    {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};

template <> struct VL<2> {
    static __device__ __forceinline__ void ldu(const float *p, float (&o)[2])
    {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void ldu_rw(const float *p, float (&o)[2])
    {
        float2 v = *reinterpret_cast<const float2 *>(p);
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void stu(float *p, const float (&o)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(o[0], o[1]);
    }
    static __device__ __forceinline__ void ldlab(const uint8_t *p, uint8_t (&o)[2])
    {
        uchar2 v = *reinterpret_cast<const uchar2 *>(p);
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void stlab(uint8_t *p, const uint8_t (&o)[2])
    {
        *reinterpret_cast<uchar2 *>(p) = make_uchar2(o[0], o[1]);
    }
    static __device__ __forceinline__ void ldx(const uint8_t *p, float (&o)[2])
    {
        uchar2 v = __ldg(reinterpret_cast<const uchar2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void ldx(const float *p, float (&o)[2])
    {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
};

template <> struct VL<1> {
    static __device__ __forceinline__ void ldu(const float *p, float (&o)[1]) { o[0] = __ldg(p); }
    static __device__ __forceinline__ void ldu_rw(const float *p, float (&o)[1]) { o[0] = *p; }
    static __device__ __forceinline__ void stu(float *p, const float (&o)[1]) { *p = o[0]; }
    static __device__ __forceinline__ void ldlab(const uint8_t *p, uint8_t (&o)[1]) { o[0] = *p; }
    static __device__ __forceinline__ void stlab(uint8_t *p, const uint8_t (&o)[1]) { *p = o[0]; }
    static __device__ __forceinline__ void ldx(const uint8_t *p, float (&o)[1]) { o[0] = __ldg(p); }
    static __device__ __forceinline__ void ldx(const float *p, float (&o)[1]) { o[0] = __ldg(p); }
};

// frame entries p0 .. p0+VW-1 of one plane; entries past the plane read as 0
template <int VW, typename FT>
__device__ __forceinline__ void load_x(const FT *f, int nvalid, int vec, float (&o)[VW])
{
    if (vec && nvalid == VW) {
        VL<VW>::ldx(f, o);
    } else {
#pragma unroll
        for (int r = 0; r < VW; ++r) o[r] = r < nvalid ? (float)__ldg(f + r) : 0.f;
    }
}

// ---- reductions -------------------------------------------------------------

// Split warp reduction of N values per lane (N a multiple of 32): after it,
// lane l holds the warp sums of values l*(N/32) .. l*(N/32) + N/32 - 1 in
// v[0 .. N/32).  Uses N - N/32 shuffles instead of 5 N.
template <int N> __device__ __forceinline__ void warp_split_reduce(float (&v)[N])
{
    static_assert(N % 32 == 0, "pad to a multiple of 32");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int off = 16 >> s;
        const int h = N >> (s + 1);
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = upper ? v[i] : v[i + h];
            const float keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
}

// CTA sums of the first nv of N per-thread values, written to out[0 .. nv).
template <int N>
__device__ __forceinline__ void block_partials(float (&v)[N], int nv, float *out, float *sred)
{
    warp_split_reduce<N>(v);
    constexpr int PER = N / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < PER; ++s) sred[w * N + lane * PER + s] = v[s];
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += THREADS) {
        float a = 0.f;
#pragma unroll
        for (int ww = 0; ww < THREADS / 32; ++ww) a += sred[ww * N + i];
        out[i] = a;
    }
}

// True in exactly one CTA: the last to arrive after all CTAs wrote partials.
__device__ __forceinline__ bool arrive_last(unsigned int *counter)
{
    __shared__ unsigned int s_ticket;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
    __syncthreads();
    const bool last = s_ticket == gridDim.x - 1;
    if (last) __threadfence();
    return last;
}

// Fixed-order sum over CTAs of NV partial rows (Kahan-compensated in FP32,
// NG interleaved groups combined in FP64).  Result in tot[0 .. NV).
template <int NV>
__device__ void reduce_partials(const float *partials, int nblocks, double *tot, float *scratch)
{
    static_assert(NV <= THREADS, "one thread per component");
    constexpr int NG = THREADS / NV;
    const int t = threadIdx.x;
    const int comp = t % NV, grp = t / NV;
    if (grp < NG) {
        float s = 0.f, c = 0.f;
        for (int b = grp; b < nblocks; b += NG) {
            const float v = __ldcg(partials + (size_t)b * NV + comp);
            const float yk = v - c;
            const float tk = s + yk;
            c = (tk - s) - yk;
            s = tk;
        }
        scratch[grp * NV + comp] = s;
    }
    __syncthreads();
    if (t < NV) {
        double a = 0.0;
        for (int gg = 0; gg < NG; ++gg) a += (double)scratch[gg * NV + t];
        tot[t] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// ---- k-space (one warp, FP64) -----------------------------------------------

// Cholesky-QR of the stored subspace from its Gram matrix G (packed upper):
// G = R^T R, T = R^{-1}; y (coefficients w.r.t. the stored rows) becomes
// R y in the orthonormal basis U_st T, so U y is unchanged.  One warp, FP64.
template <int K>
__device__ void finish_reorth(KState *ks, const double *G, double *sR, double *sT, bool frame_end,
                              double n_fg)
{
    const int l = threadIdx.x;
    const bool act = l < K;
    bool ok = true;
    double oerr = 0.0;
    if (act) {
        for (int j = 0; j < K; ++j) {
            const double gv = l <= j ? G[tri<K>(l, j)] : G[tri<K>(j, l)];
            oerr = fmax(oerr, fabs(gv - (j == l ? 1.0 : 0.0)));
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) oerr = fmax(oerr, __shfl_xor_sync(FULL, oerr, off));
    for (int a = 0; a < K; ++a) {
        double s = (act && l >= a) ? G[tri<K>(a, l)] : 0.0;
        for (int q = 0; q < a; ++q)
            if (act && l >= a) s -= sR[q * K + a] * sR[q * K + l];
        const double diag = __shfl_sync(FULL, s, a);
        if (!(diag > 0.0)) { ok = false; break; }
        const double rd = sqrt(diag);
        if (act) sR[a * K + l] = l == a ? rd : (l > a ? s / rd : 0.0);
        __syncwarp();
    }
    if (!ok) {
        if (act)
            for (int j = 0; j < K; ++j) sR[j * K + l] = sT[j * K + l] = (j == l) ? 1.0 : 0.0;
    } else if (act) {
        // column l of T = R^{-1} by back substitution (R upper triangular)
        for (int i = K - 1; i >= 0; --i) {
            double v;
            if (i > l) {
                v = 0.0;
            } else if (i == l) {
                v = 1.0 / sR[l * K + l];
            } else {
                double s = 0.0;
                for (int q = i + 1; q <= l; ++q) s += sR[i * K + q] * sT[q * K + l];
                v = -s / sR[i * K + i];
            }
            sT[i * K + l] = v;
        }
    }
    __syncwarp();
    // y in the stored basis -> R y in the orthonormal basis
    const double yst = act ? ks->y[l] : 0.0;
    double ynew = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const double yi = __shfl_sync(FULL, yst, i);
        if (act && i >= l) ynew += sR[l * K + i] * yi;
    }
    if (act) {
        for (int j = 0; j < K; ++j) {
            ks->R[l * KMAX + j] = sR[l * K + j];
            ks->T[l * KMAX + j] = sT[l * K + j];
            ks->Tf[l * K + j] = (float)sT[l * K + j];
        }
        ks->y[l] = ynew;
        ks->yf[l] = (float)yst;
    }
    if (l == 0) {
        ks->orth_err = oerr;
        if (!ok) ks->err_flags |= ERR_NOTSPD;
        if (frame_end) {
            ks->n_fg = (int64_t)n_fg;
            ks->frame_index += 1;
            ks->last_status = ok ? 0 : -6; // PROST_ENOTSPD
        } else if (!ok) {
            ks->last_status = -6;
        }
    }
}

// ---- per-pixel kernels -------------------------------------------------------

// Gram of the stored subspace and its Cholesky-QR (after init / import).
template <int K, typename UT>
__global__ void __launch_bounds__(THREADS) k_gram(const GramArgs a)
{
    constexpr int VW = Cfg<K>::VW;
    constexpr int NM = K * (K + 1) / 2;
    constexpr int NP = (NM + 31) / 32 * 32;
    __shared__ float sred[(THREADS / 32) * NP];
    __shared__ double tot[NM];
    __shared__ double sR[K * K], sT[K * K];
    const DevParams &prm = a.prm;
    if (a.after_rebase && !a.ks->rebased) return; // the periodic rebase was not due
    float acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.f;
    // VW consecutive rows of one tile block (TILE_P is a multiple of VW)
    constexpr int GPB = TILE_P / VW;
    const int nitems = prm.C * prm.npt * GPB;
    for (int it = blockIdx.x * THREADS + threadIdx.x; it < nitems; it += gridDim.x * THREADS) {
        const int blk = it / GPB;
        const int r0 = (it - blk * GPB) * VW;
        const UT *base = static_cast<const UT *>(a.U) + (int64_t)blk * K * TILE_P + r0;
        float u[K][VW];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if constexpr (sizeof(UT) == 4) {
                VL<VW>::ldu(reinterpret_cast<const float *>(base) + j * TILE_P, u[j]);
            } else {
#pragma unroll
                for (int r = 0; r < VW; ++r) u[j][r] = ldg_u(base + j * TILE_P + r);
            }
        }
#pragma unroll
        for (int r = 0; r < VW; ++r)
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(u[j][r], u[l2][r], acc[tri<K>(j, l2)]);
    }
    block_partials<NP>(acc, NM, a.partials + (size_t)blockIdx.x * NM, sred);
    if (!arrive_last(a.counter)) return;
    reduce_partials<NM>(a.partials, gridDim.x, tot, sred);
    if (threadIdx.x < 32) finish_reorth<K>(a.ks, tot, sR, sT, false, 0.0);
    if (threadIdx.x == 0) *a.counter = 0u;
}

// Orthonormal representative U = U_st T, written m x k row-major.
template <int K, typename UT>
__global__ void __launch_bounds__(THREADS) k_export(const UT *U, const KState *ks, float *out,
                                                     DevParams prm)
{
    __shared__ float sT[K * K];
    for (int i = threadIdx.x; i < K * K; i += THREADS) sT[i] = ks->Tf[i];
    __syncthreads();
    const int64_t m = (int64_t)prm.C * prm.P;
    for (int64_t e = (int64_t)blockIdx.x * THREADS + threadIdx.x; e < m; e += (int64_t)gridDim.x * THREADS) {
        const int c = (int)(e / prm.P);
        const int64_t q = e - (int64_t)c * prm.P;
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = ld_u(U + u_off(prm, c, q, j));
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(sT[i * K + j], u[i], s);
            out[e * K + j] = s;
        }
    }
}

// Rebase of the stored rows onto the orthonormal representative: U_st <- U_st T
// (each row u_st becomes T^T u_st), after which the fold is the identity.
template <int K, typename UT>
__global__ void __launch_bounds__(THREADS) k_rebase(UT *U, const KState *ks, DevParams prm, int force)
{
    // unforced, it runs only when the frames since the last rebase are due (a
    // frame refused by a stale barrier does not count)
    if (!force && ks->frames_since_rebase < REBASE_EVERY) return;
    __shared__ float sT[K * K];
    for (int i = threadIdx.x; i < K * K; i += THREADS) sT[i] = ks->Tf[i];
    __syncthreads();
    const int64_t rows = (int64_t)prm.C * prm.Pp;
    for (int64_t e = (int64_t)blockIdx.x * THREADS + threadIdx.x; e < rows; e += (int64_t)gridDim.x * THREADS) {
        const int c = (int)(e / prm.Pp);
        const int64_t q = e - (int64_t)c * prm.Pp;
        UT *base = U + u_off(prm, c, q, 0);
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = ld_u(base + (int64_t)j * TILE_P);
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(sT[i * K + j], u[i], s);
            u[j] = s;
        }
#pragma unroll
        for (int j = 0; j < K; ++j) st_u(base + (int64_t)j * TILE_P, u[j]);
    }
}

// ---- host launchers of one kernel set ----------------------------------------

template <int K, typename UT> struct Ops {
    static cudaError_t gram(const GramArgs &a, int grid, cudaStream_t s)
    {
        k_gram<K, UT><<<grid, THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t export_u(const void *U, const KState *ks, float *out, DevParams prm, cudaStream_t s)
    {
        const int64_t m = (int64_t)prm.C * prm.P;
        const int64_t nb = (m + THREADS - 1) / THREADS;
        const int grid = (int)(nb < 4096 ? nb : 4096);
        k_export<K, UT><<<grid, THREADS, 0, s>>>(static_cast<const UT *>(U), ks, out, prm);
        return cudaGetLastError();
    }
    static cudaError_t rebase(void *U, KState *ks, DevParams prm, int force, cudaStream_t s)
    {
        const int64_t nb = ((int64_t)prm.C * prm.Pp + THREADS - 1) / THREADS;
        k_rebase<K, UT><<<(int)(nb < 4096 ? nb : 4096), THREADS, 0, s>>>(static_cast<UT *>(U), ks, prm, force);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_reset_fold(ks, prm, force, s);
    }
    static int gram_occupancy()
    {
        int n = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gram<K, UT>, THREADS, 0);
        return e == cudaSuccess && n > 0 ? n : 1;
    }
};

} // namespace prost
