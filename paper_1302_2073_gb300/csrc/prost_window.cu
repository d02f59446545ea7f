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
// over the tile's rows).  Per-block partial sums are added in a fixed order
// (FP64 for the scalars), so results are deterministic.  At the window of the
// measured configuration (m = 76,800, n = 64, k = 10) the three products are
// about 3 x 98 MFLOP against 20 MB of frames: a few microseconds of CUDA-core
// time, as long as the frames take to stream.
//
// The U-step: G = (I - U U^T) dF/dU (the projection of Eq. gproject applied to
// the window gradient), V = U - t G, and the Cholesky-QR retraction
// U' = V R^{-1} with V^T V = R^T R factored in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>

#include "prost.h"

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
__global__ void __launch_bounds__(WT) k_window(WinArgs a)
{
    extern __shared__ float sm[];
    float *Ys = sm;                          // K x n
    float *Hs = Ys + K * a.n;                // WT x (n + 1)
    float *Us = Hs + (GRAD ? WT * (a.n + 1) : 0); // WT x K
    const int n = a.n, tid = threadIdx.x;
    const float mu = *a.mu, pw = a.p, e2 = 0.5f * a.p - 1.f, om = a.omega;
    const float gs = (GRAD && a.gscale) ? *a.gscale : 1.f;
    for (int i = tid; i < K * n; i += WT) Ys[i] = a.Y[i];
    // this thread's entries of the block's dY share: i = tid + WT q
    constexpr int DQ = (K * NMAXW + WT - 1) / WT;
    float dyacc[DQ];
#pragma unroll
    for (int q = 0; q < DQ; ++q) dyacc[q] = 0.f;
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
        // arithmetic, so that TB loads per thread are in flight together
        constexpr int TB = 8;
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
                float uy = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) uy = fmaf(u[j], Ys[j * n + t], uy);
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
                    for (int j = 0; j < K; ++j) du[j] = fmaf(eta, Ys[j * n + t], du[j]);
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
            for (int j = 0; j < K; ++j) Us[tid * K + j] = u[j];
            __syncthreads();
            const int rows = (int)min((int64_t)WT, a.m - tile * WT);
#pragma unroll
            for (int q = 0; q < DQ; ++q) {
                const int i = tid + WT * q;
                if (i < K * n) {
                    const int j = i / n, t = i - (i / n) * n;
                    float s = 0.f;
                    for (int r = 0; r < rows; ++r) s = fmaf(Us[r * K + j], Hs[r * (n + 1) + t], s);
                    dyacc[q] += s;
                }
            }
            __syncthreads();
        }
    }
    // block partial: dY share, cost, dmu (the scalars reduced in FP64)
    double *part = a.partials + (size_t)blockIdx.x * (K * n + 2);
    if (GRAD) {
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
            const int i = tid + WT * q;
            if (i < K * n) part[i] = (double)dyacc[q];
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

// A = U^T D (k x k), per-block partials then a fixed-order sum
template <int K>
__global__ void __launch_bounds__(WT) k_utd(const float *U, const float *D, int64_t m, double *partials)
{
    float acc[K * K];
#pragma unroll
    for (int i = 0; i < K * K; ++i) acc[i] = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * WT + threadIdx.x; e < m; e += (int64_t)gridDim.x * WT) {
        float u[K], d[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            u[j] = U[e * K + j];
            d[j] = D[e * K + j];
        }
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int j = 0; j < K; ++j) acc[i * K + j] = fmaf(u[i], d[j], acc[i * K + j]);
    }
    __shared__ float red[WT / 32][K * K];
#pragma unroll
    for (int i = 0; i < K * K; ++i) {
        float v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K * K; i += WT) {
        double s = 0.0;
        for (int w = 0; w < WT / 32; ++w) s += red[w][i];
        partials[(size_t)blockIdx.x * K * K + i] = s;
    }
}

// V = U - t (D - U A): the step along the projected gradient, written to V;
// and the Gram V^T V (packed upper) per block
template <int K>
__global__ void __launch_bounds__(WT) k_vstep(const float *U, const float *D, const double *A, float t, int64_t m,
                                             float *V, double *partials)
{
    __shared__ float sA[K * K];
    for (int i = threadIdx.x; i < K * K; i += WT) sA[i] = (float)A[i];
    __syncthreads();
    constexpr int NM = K * (K + 1) / 2;
    float acc[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) acc[i] = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * WT + threadIdx.x; e < m; e += (int64_t)gridDim.x * WT) {
        float u[K], v[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = U[e * K + j];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float ua = 0.f;
#pragma unroll
            for (int i = 0; i < K; ++i) ua = fmaf(u[i], sA[i * K + j], ua);
            v[j] = u[j] - t * (D[e * K + j] - ua);
            V[e * K + j] = v[j];
        }
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int j = i; j < K; ++j) {
                const int q = i * K - (i * (i - 1)) / 2 + (j - i); // packed upper (i, j)
                acc[q] = fmaf(v[i], v[j], acc[q]);
            }
    }
    __shared__ float red[WT / 32][NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        float x = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = x;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NM; i += WT) {
        double s = 0.0;
        for (int w = 0; w < WT / 32; ++w) s += red[w][i];
        partials[(size_t)blockIdx.x * NM + i] = s;
    }
}

// fixed-order sum of nb partial rows of len values into out (a warp each)
__global__ void k_sum_rows(const double *partials, int nb, int len, double *out)
{
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= len) return;
    const double s = warp_col_sum(partials, nb, len, i);
    if ((threadIdx.x & 31) == 0) out[i] = s;
}

// T = R^{-1} from the packed Gram G = R^T R (FP64, one thread: k <= 16);
// status 0, or -1 when G is not positive definite
template <int K> __global__ void k_chol_inv(const double *G, double *T, int *status)
{
    if (threadIdx.x != 0) return;
    double R[K * K], W[K * K];
    int q = 0;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) W[i * K + j] = 0.0;
    for (int i = 0; i < K; ++i)
        for (int j = i; j < K; ++j) {
            W[i * K + j] = G[q];
            W[j * K + i] = G[q];
            ++q;
        }
    for (int i = 0; i < K * K; ++i) R[i] = 0.0;
    for (int j = 0; j < K; ++j) {
        double d = W[j * K + j];
        for (int l = 0; l < j; ++l) d -= R[l * K + j] * R[l * K + j];
        if (!(d > 0.0)) {
            *status = -1;
            return;
        }
        const double rjj = sqrt(d);
        const double inv = 1.0 / rjj; // one division per pivot (FP64 division is slow)
        R[j * K + j] = rjj;
        W[j * K + j] = inv;           // the reciprocal, kept for the back substitution
        for (int c = j + 1; c < K; ++c) {
            double s = W[j * K + c];
            for (int l = 0; l < j; ++l) s -= R[l * K + j] * R[l * K + c];
            R[j * K + c] = s * inv;
        }
    }
    // T = R^{-1}, upper triangular, by back substitution
    for (int i = 0; i < K * K; ++i) T[i] = 0.0;
    for (int c = 0; c < K; ++c) {
        for (int i = c; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int l = i + 1; l <= c; ++l) s -= R[i * K + l] * T[l * K + c];
            T[i * K + c] = s * W[i * K + i];
        }
    }
    *status = 0;
}

// U' = V T
template <int K>
__global__ void __launch_bounds__(WT) k_apply_t(const float *V, const double *T, int64_t m, float *Uo)
{
    __shared__ float sT[K * K];
    for (int i = threadIdx.x; i < K * K; i += WT) sT[i] = (float)T[i];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * WT + threadIdx.x; e < m; e += (int64_t)gridDim.x * WT) {
        float v[K];
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = V[e * K + j];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(v[i], sT[i * K + j], s);
            Uo[e * K + j] = s;
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
    int nb_u;         // U-step kernels
    size_t smem_grad, smem_cost;
    double *partials; // window kernel
    double *upart;    // U-step partials
    double *A, *G, *T;
    float *V;
    int *status;
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
        k_utd<K><<<w->nb_u, WT, 0, w->stream>>>(U, D, w->m, w->upart);
        k_sum_rows<<<(K * K * 32 + 255) / 256, 256, 0, w->stream>>>(w->upart, w->nb_u, K * K, w->A);
        k_vstep<K><<<w->nb_u, WT, 0, w->stream>>>(U, D, w->A, t, w->m, w->V, w->upart);
        k_sum_rows<<<(K * (K + 1) / 2 * 32 + 255) / 256, 256, 0, w->stream>>>(w->upart, w->nb_u, K * (K + 1) / 2,
                                                                                w->G);
        k_chol_inv<K><<<1, 32, 0, w->stream>>>(w->G, w->T, w->status);
        k_apply_t<K><<<w->nb_u, WT, 0, w->stream>>>(w->V, w->T, w->m, Uo);
        return cudaGetLastError();
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
    double *d[] = {w->partials, w->upart, w->A, w->G, w->T};
    for (double *p : d)
        if (p) cudaFree(p);
    if (w->V) cudaFree(w->V);
    if (w->status) cudaFree(w->status);
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
    w->nb_u = (int)(tiles < 4 * sms ? tiles : 4 * sms);
    w->smem_cost = (size_t)k * n * sizeof(float);
    w->smem_grad = w->smem_cost + (size_t)WT * (n + 1) * sizeof(float) + (size_t)WT * k * sizeof(float);
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
        !ck(cudaMalloc(&w->upart, (size_t)w->nb_u * k * k * sizeof(double)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->A, (size_t)k * k * sizeof(double)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->G, (size_t)k * k * sizeof(double)), "cudaMalloc") ||
        !ck(cudaMalloc(&w->T, (size_t)k * k * sizeof(double)), "cudaMalloc") ||
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
