// The cost of pROST summed over a window of n frames and its gradients
// (arXiv:1302.2073, Eqs. weightedLPnorm and spcacost, the gradient of Section
// 3.3), and a Grassmannian step of U along the window gradient.
//
//   F(U, Y, mu) = sum_t sum_e w_te ((x_te - u_e^T y_t)^2 + mu)^(p/2)
//   eta_te = -p w_te r_te (r_te^2 + mu)^(p/2 - 1),  H = [eta_te]  (m x n)
//   dF/dU = H Y^T,  dF/dY = U^T H,  dF/dmu = sum w (p/2) (r^2 + mu)^(p/2 - 1)
//
// One pass over the window: a thread takes one row e (the k entries of u_e,
// the n entries x_1e .. x_ne, coalesced across the block), forms its n
// residuals with Y held in shared memory, accumulates the cost, dF/dmu and its
// row of dF/dU, and stages its eta_te in shared memory; the block then forms
// its share of dF/dY = U^T H from the staged tile (k x n outputs, each a sum
// over the tile's rows), each thread a 2 x 4 block of outputs over a subset of
// the rows (one 8-byte load of u and four of eta per 8 multiply-adds).
// Per-block partial sums are added in a fixed order
// (FP64 for the scalars), so results are deterministic.  At the window of the
// measured configuration (m = 76,800, n = 64, k = 10) the three products are
// about 3 x 98 MFLOP against 20 MB of frames: a few microseconds of CUDA-core
// time, as long as the frames take to stream.
//
// The U-step: G = (I - U U^T) dF/dU (the projection of Eq. gproject applied to
// the window gradient), V = U - t G, and the Cholesky-QR retraction
// U' = V R^{-1} with V^T V = R^T R factored in FP64, in one cooperative launch.
//
// The three products of the window pass were also built on tensor cores
// (mma.sync m16n8k8 tf32, operands split hi + mid + lo, a warp per 16 rows and
// all frames).  It matched the oracle once every product started from a zero
// accumulator (accumulating into a large one biased dY by 1.7e-5 relative),
// but at 16 rows per warp and up to 226 registers it ran at 8 warps per SM and
// took 31 us (forward) and 46 us (with gradients) against this pass's 21 and
// 34 us: at k = 10 the products are skinny and the pass is bound by its loads.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include "prost.h"
#include "prost_frame.cuh" // reduce_rows, cholesky_rl: the frame kernel's fixed-order sum and FP64 factors

namespace {

constexpr int WT = 256;      // threads per block, rows per tile
constexpr int NMAXW = 128;   // largest window
constexpr int KMAXW = 16;

struct WinArgs {
    const float *U, *Y, *X;
    const uint8_t *labels;   // n x P, or null (all weights 1)
    const float *mu;         // device scalar
    const float *gscale;     // device scalar multiplying the gradients, or null
    float *dU, *dY;
    double *partials;        // per block: [dY (k n) | cost | dmu]
    int64_t m, P;
    int k, n;
    float p, omega;
};

template <int K, bool GRAD>
__global__ void __launch_bounds__(WT, 2) k_window(WinArgs a)
{
    // Y transposed, frame t's k values contiguous and padded to a multiple of
    // 4: a thread takes y_t with K4 / 4 vector loads and keeps it for both
    // u^T y_t and its row of dF/dU
    constexpr int K4 = (K + 3) / 4 * 4;
    extern __shared__ float4 sm4[];
    float *sm = reinterpret_cast<float *>(sm4);
    float *Ys = sm;                          // n x K4
    float *Hs = Ys + K4 * a.n;               // WT x (n + 1)
    // the tile's rows, US floats apart (K rounded up to even: pairs of
    // columns as one 8-byte load)
    constexpr int US = (K + 1) / 2 * 2, JP = US / 2;
    float *Us = Hs + (GRAD ? WT * (a.n + 1) : 0); // WT x US
    const int n = a.n, tid = threadIdx.x;
    const float mu = *a.mu, pw = a.p, e2 = 0.5f * a.p - 1.f, om = a.omega;
    const float gs = (GRAD && a.gscale) ? *a.gscale : 1.f;
    for (int i = tid; i < K4 * n; i += WT) {
        const int t = i / K4, j = i - (i / K4) * K4;
        Ys[i] = j < K ? a.Y[j * n + t] : 0.f;
    }
    // the block's dY share, register-tiled: thread tid sums the 2 x 4 block
    // (columns 2 jp, 2 jp + 1; frames 4 tq .. 4 tq + 3) over the rows
    // r = g (mod G) of every tile, with G = WT / NB row groups (threads with
    // g >= G sit out); the groups are added in order at the end
    const int TQ = (n + 3) / 4, NB = JP * TQ, G = WT / NB;
    const int bb = tid % NB, g = tid / NB;
    const int jp = bb / TQ, tq = bb - (bb / TQ) * TQ;
    float dyacc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) dyacc[q] = 0.f;
    double cost = 0.0, dmu = 0.0;
    __syncthreads();
    const int64_t ntiles = (a.m + WT - 1) / WT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e = tile * WT + tid;
        const bool valid = e < a.m;
        float u[K], du[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            u[j] = valid ? a.U[e * K + j] : 0.f;
            du[j] = 0.f;
        }
        float cpart = 0.f, mpart = 0.f;
        const int64_t px = valid ? e % a.P : 0;
        // TB frames at a time: their entries and labels are loaded before any
        // arithmetic, so that TB loads per thread are in flight together (32:
        // 30.8 us with gradients against 33.5 us at 8)
        constexpr int TB = 32;
        for (int t0 = 0; t0 < n; t0 += TB) {
            float xv[TB];
            bool lv[TB];
#pragma unroll
            for (int q = 0; q < TB; ++q) {
                const int t = t0 + q;
                const bool in = valid && t < n;
                xv[q] = in ? __ldg(a.X + (int64_t)t * a.m + e) : 0.f;
                lv[q] = in && a.labels && __ldg(a.labels + (int64_t)t * a.P + px);
            }
#pragma unroll
            for (int q = 0; q < TB; ++q) {
                const int t = t0 + q;
                if (t >= n) break;
                float yt[K4];
#pragma unroll
                for (int j4 = 0; j4 < K4 / 4; ++j4) {
                    const float4 v = reinterpret_cast<const float4 *>(Ys + t * K4)[j4];
                    yt[4 * j4] = v.x;
                    yt[4 * j4 + 1] = v.y;
                    yt[4 * j4 + 2] = v.z;
                    yt[4 * j4 + 3] = v.w;
                }
                float uy = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) uy = fmaf(u[j], yt[j], uy);
                float eta = 0.f;
                if (valid) {
                    const float w = lv[q] ? om : 1.f;
                    const float r = xv[q] - uy;
                    const float z = fmaf(r, r, mu);
                    const float zp = __powf(z, e2);
                    cpart = fmaf(w * z, zp, cpart);
                    mpart = fmaf(w, zp, mpart);
                    eta = -pw * w * r * zp;
                }
                if (GRAD) {
#pragma unroll
                    for (int j = 0; j < K; ++j) du[j] = fmaf(eta, yt[j], du[j]);
                    Hs[tid * (n + 1) + t] = eta;
                }
            }
        }
        cost += (double)cpart;
        dmu += (double)mpart;
        if (GRAD) {
            if (valid)
#pragma unroll
                for (int j = 0; j < K; ++j) a.dU[e * K + j] = gs * du[j];
#pragma unroll
            for (int j = 0; j < US; ++j) Us[tid * US + j] = j < K ? u[j] : 0.f;
            __syncthreads();
            const int rows = (int)min((int64_t)WT, a.m - tile * WT);
            if (g < G) {
                const int t0 = 4 * tq;
                float s[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) s[q] = 0.f;
                for (int r = g; r < rows; r += G) {
                    const float2 uu = *reinterpret_cast<const float2 *>(Us + r * US + 2 * jp);
                    const float *hr = Hs + r * (n + 1) + t0;
                    float h[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) h[c] = t0 + c < n ? hr[c] : 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        s[c] = fmaf(uu.x, h[c], s[c]);
                        s[4 + c] = fmaf(uu.y, h[c], s[4 + c]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) dyacc[q] += s[q];
            }
            __syncthreads();
        }
    }
    // block partial: dY share, cost, dmu (the scalars reduced in FP64)
    double *part = a.partials + (size_t)blockIdx.x * (K * n + 2);
    if (GRAD) {
        // the row groups' sums added in group order (the eta and row tiles
        // are free now; the host sizes them to hold WT x 8 floats at least)
        float *red8 = Hs;
        if (g < G)
#pragma unroll
            for (int q = 0; q < 8; ++q) red8[(g * NB + bb) * 8 + q] = dyacc[q];
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v = 0.f;
                for (int gg = 0; gg < G; ++gg) v += red8[(gg * NB + bb) * 8 + q];
                const int j = 2 * jp + q / 4, t = 4 * tq + (q & 3);
                if (j < K && t < n) part[j * n + t] = (double)v;
            }
        }
    }
    __shared__ double red[2][WT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cost += __shfl_xor_sync(0xffffffffu, cost, o);
        dmu += __shfl_xor_sync(0xffffffffu, dmu, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = cost;
        red[1][tid >> 5] = dmu;
    }
    __syncthreads();
    if (tid == 0) {
        double c = 0.0, d = 0.0;
        for (int w = 0; w < WT / 32; ++w) {
            c += red[0][w];
            d += red[1][w];
        }
        part[K * n] = c;
        part[K * n + 1] = d;
    }
}

// fixed-order sum of a column of nb partial rows by one warp (each lane a
// strided subset, then a fixed shuffle tree: short FP64 chains)
__device__ __forceinline__ double warp_col_sum(const double *partials, int nb, int len, int i)
{
    double s = 0.0;
    for (int b = threadIdx.x & 31; b < nb; b += 32) s += partials[(size_t)b * len + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// fixed-order sum of the block partials, a warp per value: dY (scaled), the
// cost, dmu
__global__ void k_window_finish(const double *partials, int nblocks, int kn, const float *gscale, float p,
                                float *dY, float *cost, float *dmu)
{
    const float gs = gscale ? *gscale : 1.f;
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= kn + 2) return;
    {
        const double s = warp_col_sum(partials, nblocks, kn + 2, i);
        if ((threadIdx.x & 31) != 0) return;
        if (i < kn) {
            if (dY) dY[i] = gs * (float)s;
        } else if (i == kn) {
            if (cost) *cost = (float)s;
        } else if (dmu) {
            *dmu = gs * (float)(0.5 * (double)p * s);
        }
    }
}

// ---- U-step -----------------------------------------------------------------
//
// One cooperative launch, one CTA per SM, each CTA a contiguous range of rows:
//   A = U^T dU                        (partial per CTA, grid barrier, fixed-order sum)
//   V = U - t (dU - U A), Gram V^T V  (V written; partial per CTA, grid barrier, sum)
//   V^T V = R^T R, T = R^{-1}         (FP64, every CTA the same)
//   U_out = V T
// Rows go through shared memory in tiles of WT (U and dU, then V), and thread
// i forms entry i of U^T dU or of V^T V over the tile, so no thread holds a
// k x k accumulator.

constexpr long long UWAIT_LIMIT = 2000000000ll; // SM clock cycles (about 1 s)
constexpr int URS = KMAXW * KMAXW;              // floats per partial row

struct UstepArgs {
    const float *U, *D;
    float *V, *Uo;
    float *rows;       // 2 x G partial rows of URS floats
    unsigned int *bar; // arrival counter, abort flag (zeroed before the launch)
    int *status;
    int64_t m;
    float t;
    // failure-detection tests only (0 = off): barrier stall_at waits for one
    // arrival more than the launch makes and gives up after stall_limit cycles
    int stall_at;
    long long stall_limit;
};

// Grid barrier: arrive, then a bounded spin; false when it gave up (the abort
// flag then releases every other CTA too).
__device__ bool ustep_wait(unsigned int *bar, unsigned int target, long long limit = UWAIT_LIMIT)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        const long long t0 = clock64();
        unsigned int it = 0;
        for (;;) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if ((++it & 15u) == 0 && (*(volatile unsigned int *)(bar + 1) || clock64() - t0 > limit)) {
                atomicExch(bar + 1, 1u);
                ok = 0;
                break;
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int K>
__global__ void __launch_bounds__(WT, 1) k_ustep(UstepArgs a)
{
    constexpr int KK = K * K, NM = K * (K + 1) / 2;
    static_assert(KK <= WT, "one k x k entry per thread");
    __shared__ float Us[WT * K], Ds[WT * K];
    __shared__ float tot[KK], sA[KK], sTf[KK];
    __shared__ float scr[prost::RED_SCR];
    __shared__ double sR[KK], sT[KK], sW[KK], sinv[K];
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int64_t e0 = a.m * b / G, e1 = a.m * (b + 1) / G;
    const int ri = tid / K, rl = tid - (tid / K) * K; // this thread's entry (ri, rl)

    // A = U^T dU over this CTA's rows
    float acc = 0.f;
    for (int64_t t0 = e0; t0 < e1; t0 += WT) {
        const int nr = (int)min((int64_t)WT, e1 - t0);
        for (int q = tid; q < nr * K; q += WT) {
            Us[q] = a.U[t0 * K + q];
            Ds[q] = a.D[t0 * K + q];
        }
        __syncthreads();
        if (tid < KK)
            for (int r = 0; r < nr; ++r) acc = fmaf(Us[r * K + ri], Ds[r * K + rl], acc);
        __syncthreads();
    }
    if (tid < KK) a.rows[(size_t)b * URS + tid] = acc;
    if (!ustep_wait(a.bar, (unsigned)G + (a.stall_at == 1 ? 1u : 0u), a.stall_at == 1 ? a.stall_limit : UWAIT_LIMIT)) {
        if (b == 0 && tid == 0) *a.status = -2;
        return;
    }
    prost::reduce_rows<WT>(a.rows, G, URS, KK, tot, scr);
    for (int i = tid; i < KK; i += WT) sA[i] = tot[i];
    __syncthreads();

    // V = U - t (dU - U A) and its Gram
    const bool gram = tid < KK && ri <= rl;
    float gacc = 0.f;
    for (int64_t t0 = e0; t0 < e1; t0 += WT) {
        const int nr = (int)min((int64_t)WT, e1 - t0);
        if (tid < nr) {
            const int64_t e = t0 + tid;
            float u[K];
#pragma unroll
            for (int j = 0; j < K; ++j) u[j] = a.U[e * K + j];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                float ua = 0.f;
#pragma unroll
                for (int i = 0; i < K; ++i) ua = fmaf(u[i], sA[i * K + j], ua);
                const float v = u[j] - a.t * (a.D[e * K + j] - ua);
                a.V[e * K + j] = v;
                Us[tid * K + j] = v;
            }
        }
        __syncthreads();
        if (gram)
            for (int r = 0; r < nr; ++r) gacc = fmaf(Us[r * K + ri], Us[r * K + rl], gacc);
        __syncthreads();
    }
    if (gram) a.rows[(size_t)(G + b) * URS + prost::tri<K>(ri, rl)] = gacc;
    if (!ustep_wait(a.bar, 2u * (unsigned)G + (a.stall_at == 2 ? 1u : 0u),
                    a.stall_at == 2 ? a.stall_limit : UWAIT_LIMIT)) {
        if (b == 0 && tid == 0) *a.status = -2;
        return;
    }
    prost::reduce_rows<WT>(a.rows + (size_t)G * URS, G, URS, NM, tot, scr);
    if (tid < KK) sW[tid] = (double)(ri <= rl ? tot[prost::tri<K>(ri, rl)] : tot[prost::tri<K>(rl, ri)]);
    __syncthreads();
    const bool ok = prost::cholesky_rl<K, WT>(sR, sT, sW, sinv);
    if (b == 0 && tid == 0) *a.status = ok ? 0 : -1;
    if (!ok) return;
    if (tid < KK) sTf[tid] = (float)sT[tid];
    __syncthreads();

    // U_out = V T (each thread re-reads the rows it wrote)
    for (int64_t t0 = e0; t0 < e1; t0 += WT) {
        const int64_t e = t0 + tid;
        if (e >= e1) continue;
        float v[K];
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = a.V[e * K + j];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(v[i], sTf[i * K + j], s);
            a.Uo[e * K + j] = s;
        }
    }
}

std::string g_win_err;

} // namespace

struct prost_window {
    int64_t m, P;
    int k, n, C;
    float p, omega;
    cudaStream_t stream;
    int nblocks;      // window kernel
    int nb_u;         // U-step kernel (cooperative, one CTA per SM)
    size_t smem_grad, smem_cost;
    double *partials; // window kernel
    float *urows;     // U-step partial rows
    unsigned int *ubar; // U-step grid barrier
    float *V;
    int *status;
    int stall_at;       // armed for the next U-step by prost_window_inject_wait_timeout
    long long stall_limit;
    std::string err;
};

namespace {

template <int K> struct WinOps {
    static cudaError_t eval(prost_window *w, WinArgs &a, bool grad)
    {
        if (grad) {
            k_window<K, true><<<w->nblocks, WT, w->smem_grad, w->stream>>>(a);
        } else {
            k_window<K, false><<<w->nblocks, WT, w->smem_cost, w->stream>>>(a);
        }
        return cudaGetLastError();
    }
    static cudaError_t attrs(size_t smem_grad)
    {
        return cudaFuncSetAttribute(k_window<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_grad);
    }
    static cudaError_t ustep(prost_window *w, const float *U, const float *D, float t, float *Uo)
    {
        cudaError_t e = cudaMemsetAsync(w->ubar, 0, 2 * sizeof(unsigned int), w->stream);
        if (e != cudaSuccess) return e;
        UstepArgs a;
        a.U = U;
        a.D = D;
        a.V = w->V;
        a.Uo = Uo;
        a.rows = w->urows;
        a.bar = w->ubar;
        a.status = w->status;
        a.m = w->m;
        a.t = t;
        a.stall_at = w->stall_at;
        a.stall_limit = w->stall_limit;
        w->stall_at = 0; // one launch only
        void *args[] = {&a};
        return cudaLaunchCooperativeKernel((void *)k_ustep<K>, dim3(w->nb_u), dim3(WT), args, 0, w->stream);
    }
};

struct WinTable {
    cudaError_t (*eval)(prost_window *, WinArgs &, bool);
    cudaError_t (*attrs)(size_t);
    cudaError_t (*ustep)(prost_window *, const float *, const float *, float, float *);
};

template <int K> WinTable win_table() { return {&WinOps<K>::eval, &WinOps<K>::attrs, &WinOps<K>::ustep}; }

WinTable win_ops(int k)
{
    switch (k) {
    case 1: return win_table<1>();
    case 2: return win_table<2>();
    case 3: return win_table<3>();
    case 4: return win_table<4>();
    case 5: return win_table<5>();
    case 6: return win_table<6>();
    case 7: return win_table<7>();
    case 8: return win_table<8>();
    case 9: return win_table<9>();
    case 10: return win_table<10>();
    case 11: return win_table<11>();
    case 12: return win_table<12>();
    case 13: return win_table<13>();
    case 14: return win_table<14>();
    case 15: return win_table<15>();
    default: return win_table<16>();
    }
}

#define WIN_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            w->err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return e_ == cudaErrorMemoryAllocation ? PROST_ENOMEM : PROST_ECUDA;              \
        }                                                                                     \
    } while (0)

void win_free(prost_window *w)
{
    void *d[] = {w->partials, w->urows, w->ubar, w->V, w->status};
    for (void *p : d)
        if (p) cudaFree(p);
}

} // namespace

extern "C" int prost_window_init(int64_t m, int32_t channels, int32_t k, int32_t n, double p, double omega,
                                 void *stream, prost_window **out)
{
    if (!out) { g_win_err = "out is NULL"; return PROST_EINVAL; }
    *out = nullptr;
    if (m < 1 || channels < 1 || m % channels != 0 || k < 1 || k > KMAXW || n < 1 || n > NMAXW || !(p > 0.0) ||
        !(p <= 2.0) || !(omega >= 0.0) || !(omega <= 1.0) || m > (1ll << 30)) {
        g_win_err = "need m a multiple of channels, 1 <= k <= 16, 1 <= n <= 128, 0 < p <= 2, 0 <= omega <= 1";
        return PROST_EINVAL;
    }
    prost_window *w = new (std::nothrow) prost_window();
    if (!w) { g_win_err = "host allocation failed"; return PROST_ENOMEM; }
    w->m = m;
    w->C = channels;
    w->P = m / channels;
    w->k = k;
    w->n = n;
    w->p = (float)p;
    w->omega = (float)omega;
    w->stream = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (m + WT - 1) / WT;
    w->nblocks = (int)(tiles < 2 * sms ? tiles : 2 * sms);
    w->nb_u = sms; // cooperative: one CTA per SM
    w->smem_cost = (size_t)((k + 3) / 4 * 4) * n * sizeof(float);
    // the gradient pass's eta tile (WT x (n + 1)) and row tile (WT x even k),
    // at least WT x 8 floats: after the last tile that space holds the row
    // groups' 2 x 4 dY blocks (G x NB <= WT blocks of 8)
    const size_t grad_floats = std::max((size_t)WT * (n + 1) + (size_t)WT * ((k + 1) / 2 * 2), (size_t)WT * 8);
    w->smem_grad = w->smem_cost + grad_floats * sizeof(float);
    auto bail = [&](int code) {
        g_win_err = w->err;
        win_free(w);
        delete w;
        return code;
    };
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) w->err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaSuccess;
    };
    if (!ck(win_ops(k).attrs(w->smem_grad), "shared memory") ||
        !ck(cudaMalloc(&w->partials, (size_t)w->nblocks * (k * n + 2) * sizeof(double)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->urows, (size_t)2 * w->nb_u * URS * sizeof(float)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->ubar, 2 * sizeof(unsigned int)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->V, (size_t)m * k * sizeof(float)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->status, sizeof(int)), "cudaMalloc"))
        return bail(PROST_ENOMEM);
    *out = w;
    return PROST_OK;
}

extern "C" int prost_window_eval(prost_window *w, const float *U, const float *Y, const float *X,
                                 const uint8_t *labels, const float *mu, const float *gscale, float *cost,
                                 float *dU, float *dY, float *dmu)
{
    if (!w) return PROST_EINVAL;
    if (!U || !Y || !X || !mu) {
        w->err = "U, Y, X and mu must be device pointers";
        return PROST_EINVAL;
    }
    const bool grad = dU || dY || dmu;
    if (grad && !(dU && dY && dmu)) {
        w->err = "the gradients are written together: dU, dY and dmu";
        return PROST_EINVAL;
    }
    WinArgs a;
    memset(&a, 0, sizeof(a));
    a.U = U;
    a.Y = Y;
    a.X = X;
    a.labels = labels;
    a.mu = mu;
    a.gscale = gscale;
    a.dU = dU;
    a.dY = dY;
    a.partials = w->partials;
    a.m = w->m;
    a.P = w->P;
    a.k = w->k;
    a.n = w->n;
    a.p = w->p;
    a.omega = w->omega;
    WIN_CK(win_ops(w->k).eval(w, a, grad));
    const int nvals = w->k * w->n + 2;
    k_window_finish<<<(nvals * 32 + 255) / 256, 256, 0, w->stream>>>(w->partials, w->nblocks, w->k * w->n, gscale,
                                                                     w->p, grad ? dY : nullptr, cost,
                                                                     grad ? dmu : nullptr);
    WIN_CK(cudaGetLastError());
    return PROST_OK;
}

extern "C" int prost_window_ustep(prost_window *w, const float *U, const float *dU, float t, float *U_out,
                                  int32_t *status_out)
{
    if (!w) return PROST_EINVAL;
    if (!U || !dU || !U_out || U_out == U) {
        w->err = "U, dU and a distinct U_out must be device pointers";
        return PROST_EINVAL;
    }
    WIN_CK(win_ops(w->k).ustep(w, U, dU, t, U_out));
    if (status_out) WIN_CK(cudaMemcpyAsync(status_out, w->status, sizeof(int), cudaMemcpyDeviceToDevice, w->stream));
    return PROST_OK;
}

extern "C" int prost_window_inject_wait_timeout(prost_window *w, int32_t barrier, int64_t cycles)
{
    if (!w) return PROST_EINVAL;
    if (barrier < 1 || barrier > 2 || cycles < 1 || cycles > UWAIT_LIMIT) {
        w->err = "barrier must be 1 or 2 and cycles in 1..2e9";
        return PROST_EINVAL;
    }
    w->stall_at = barrier;
    w->stall_limit = cycles;
    return PROST_OK;
}

extern "C" const char *prost_window_last_error(const prost_window *w)
{
    return w ? w->err.c_str() : g_win_err.c_str();
}

extern "C" void prost_window_destroy(prost_window *w)
{
    if (!w) return;
    cudaStreamSynchronize(w->stream);
    win_free(w);
    delete w;
}
