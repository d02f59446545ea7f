// prost_cost_grad_static(): the cost and gradient of one frame for callers
// that cannot allocate device memory.  The only scratch this needs (the
// per-CTA partial sums and the arrival counter of the last-CTA reduction)
// lives in one file-scope static device array, so the call itself allocates
// nothing; the caller passes every input and output buffer.
#include <stdint.h>

#include <mutex>

#include "prost.h"
#include "prost_device.h"
#include "prost_kernels.cuh"

namespace prost {

constexpr int STATIC_MAX_CTAS = 1024;      // partial rows the array holds
constexpr int STATIC_KMAX = PROST_STATIC_MAX_K; // widest k (the kernel set below)
constexpr int STATIC_ROW = STATIC_KMAX + 2;      // gradient (k), cost, non-finite count

struct StaticScratch {
    float partials[STATIC_MAX_CTAS * STATIC_ROW];
    unsigned int counter;
};

// 1024 x 18 floats + the counter, about 74 KB; every GPU that loads the
// library holds it until the process exits.
static __device__ __align__(256) StaticScratch g_static_scratch;

struct StaticArgs {
    const float *U;          // m x k row-major (device)
    const void *frame;       // m entries (device)
    const uint8_t *labels;   // P bytes (device) or NULL
    double *out;             // k + 1 doubles (device): cost, then gradient
    int32_t *status;         // device or NULL
    int64_t m, P;
    float y[STATIC_KMAX];
    float p, mu, omega, in_scale, in_offset, e;
};

template <int K, typename FT>
__global__ void __launch_bounds__(THREADS) k_cost_grad_static(const StaticArgs a, StaticScratch *s)
{
    constexpr int NV = K + 2;
    constexpr int NP = (NV + 31) / 32 * 32;
    __shared__ float sred[(THREADS / 32) * NP];
    __shared__ double tot[NV];
    float acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.f;
    float y[K];
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = a.y[j];
    const FT *frame = static_cast<const FT *>(a.frame);
    for (int64_t e = (int64_t)blockIdx.x * THREADS + threadIdx.x; e < a.m;
         e += (int64_t)gridDim.x * THREADS) {
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = __ldg(a.U + e * K + j);
        const float v = (float)__ldg(frame + e);
        if constexpr (sizeof(FT) == 4) {
            if (!isfinite(v)) acc[K + 1] += 1.f;
        }
        float uy = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) uy = fmaf(u[j], y[j], uy);
        const float res = fmaf(v, a.in_scale, -a.in_offset) - uy;
        const float z = fmaf(res, res, a.mu);
        const float tz = __powf(z, a.e);
        const float wv = (a.labels && a.labels[e % a.P]) ? a.omega : 1.f;
        const float cw = wv * tz;
        acc[K] = fmaf(cw, z, acc[K]);
        const float eta = -a.p * cw * res;
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] = fmaf(eta, u[j], acc[j]);
    }
    block_partials<NP>(acc, NV, s->partials + (size_t)blockIdx.x * NV, sred);
    if (!arrive_last(&s->counter)) return;
    reduce_partials<NV>(s->partials, gridDim.x, tot, sred);
    if (threadIdx.x < K) a.out[1 + threadIdx.x] = tot[threadIdx.x];
    if (threadIdx.x == 0) {
        a.out[0] = tot[K];
        if (a.status) *a.status = tot[K + 1] > 0.0 ? PROST_EBADFRAME : PROST_OK;
        s->counter = 0u;
    }
}

template <int K>
static cudaError_t launch_static(const StaticArgs &a, StaticScratch *s, int fdt, int grid,
                                 cudaStream_t st)
{
    if (fdt == PROST_U8) k_cost_grad_static<K, uint8_t><<<grid, THREADS, 0, st>>>(a, s);
    else k_cost_grad_static<K, float><<<grid, THREADS, 0, st>>>(a, s);
    return cudaGetLastError();
}

typedef cudaError_t (*StaticLaunch)(const StaticArgs &, StaticScratch *, int, int, cudaStream_t);

static const StaticLaunch g_static_launch[STATIC_KMAX + 1] = {
    nullptr, launch_static<1>, launch_static<2>, launch_static<3>, launch_static<4>,
    launch_static<5>, launch_static<6>, launch_static<7>, launch_static<8>, launch_static<9>,
    launch_static<10>, launch_static<11>, launch_static<12>, launch_static<13>,
    launch_static<14>, launch_static<15>, launch_static<16>};

} // namespace prost

using namespace prost;

namespace {

constexpr int MAX_DEVICES = 128;
std::mutex g_static_mu;
StaticScratch *g_static_addr[MAX_DEVICES];
int g_static_sms[MAX_DEVICES];

// Device address of the static scratch on the current device, looked up once
// per device (the symbol's name is only a host-side stand-in in host code).
int static_scratch(StaticScratch **out, int *sms)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return PROST_ECUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PROST_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return PROST_ECUDA;
        g_static_sms[dev] = n;
        g_static_addr[dev] = static_cast<StaticScratch *>(p);
    }
    *out = g_static_addr[dev];
    *sms = g_static_sms[dev];
    return PROST_OK;
}

} // namespace

extern "C" int prost_cost_grad_static(const prost_params *prm, const float *U, const double *y,
                                      const void *frame, const uint8_t *labels, double *out,
                                      int32_t *status_out, void *stream)
{
    if (!prm || !U || !y || !frame || !out) return PROST_EINVAL;
    const prost_params &p = *prm;
    if (p.width <= 0 || p.height <= 0 || p.channels < 1 || p.channels > 4) return PROST_EINVAL;
    const int64_t P = (int64_t)p.width * p.height, m = P * p.channels;
    if (m > ((int64_t)1 << 30)) return PROST_EINVAL;
    // the static partial rows hold at most PROST_STATIC_MAX_K gradient entries
    if (p.k < 1 || p.k > STATIC_KMAX || (int64_t)p.k > m) return PROST_EINVAL;
    if (!(p.p > 0.0 && p.p <= 2.0) || !(p.delta > 0.0)) return PROST_EINVAL;
    const double mu = p.mu == 0.0 ? p.delta * p.delta * (1.0 - p.p) : p.mu;
    if (!(mu > 0.0) || !(p.omega >= 0.0 && p.omega <= 1.0)) return PROST_EINVAL;
    if (p.frame_dtype != PROST_U8 && p.frame_dtype != PROST_F32) return PROST_EINVAL;
    if (p.u_dtype != PROST_F32) return PROST_EINVAL;

    StaticScratch *s = nullptr;
    int sms = 0;
    int rc = static_scratch(&s, &sms);
    if (rc) return rc;
    StaticArgs a;
    a.U = U;
    a.frame = frame;
    a.labels = labels;
    a.out = out;
    a.status = status_out;
    a.m = m;
    a.P = P;
    for (int j = 0; j < STATIC_KMAX; ++j) a.y[j] = j < p.k ? (float)y[j] : 0.f;
    a.p = (float)p.p;
    a.mu = (float)mu;
    a.omega = (float)p.omega;
    a.in_scale = (float)p.in_scale;
    a.in_offset = (float)p.in_offset;
    a.e = (float)(0.5 * p.p - 1.0);
    int64_t grid = (m + THREADS - 1) / THREADS;
    if (grid > 2 * (int64_t)sms) grid = 2 * (int64_t)sms;
    if (grid > STATIC_MAX_CTAS) grid = STATIC_MAX_CTAS;
    cudaStream_t st = (cudaStream_t)stream;
    // the arrival counter must start at zero whatever an earlier call left
    if (cudaMemsetAsync(&s->counter, 0, sizeof(unsigned int), st) != cudaSuccess) return PROST_ECUDA;
    if (g_static_launch[p.k](a, s, p.frame_dtype, (int)grid, st) != cudaSuccess) return PROST_ECUDA;
    return PROST_OK;
}
