// Pre- and post-processing of pROST (arXiv:1302.2073, Section 3.4) on the GPU.
//
// Pre-processing: area resampling of the channel planes to the tracker's size,
// the running per-entry mean and the running standard deviation of all entries
// over the first i_init frames (fixed afterwards), and x = (v - mean) / std.
// The paper runs this part on the GPU as well.  Post-processing: the 3 x 3
// median of the foreground mask (on the CPU in the paper), border pixels
// replicated, i.e. a 5-of-9 majority on a binary mask.
//
// During the phase a frame takes three launches: resampling fused with the
// mean update and per-block FP64 partial sums of v and v^2; one block that adds
// the partials in a fixed order to the running sums and forms the deviation;
// the normalisation.  After the phase resampling and normalisation are one
// launch.  Every reduction has a fixed order, so results are deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>

#include "prost.h"

namespace {

constexpr int PT = 256;         // threads per block
constexpr int PB_MAX = 1024;    // blocks of the resampling launch

struct PreGeom {
    int w_in, h_in, C, w_out, h_out;
    int64_t n_out;              // C * h_out * w_out
    int64_t in_pitch;           // entries between input planes
};

// Area weights along one axis, in exact integers.  With s = n_in / n_out,
// output index i covers [i s, (i + 1) s) and input pixel q gets
// |[q, q + 1) ∩ that interval| / s.  In units of 1 / n_out the interval is
// [i n_in, (i + 1) n_in) and the pixel [q n_out, (q + 1) n_out), so the
// overlap is an integer ov and the weight is ov / n_in (a rounded float s
// would put the ends of the interval off by about n_in 2^-24).
__device__ __forceinline__ void footprint(int i, int n_in, int n_out, int &q0, int &q1, int64_t &lo, int64_t &hi)
{
    lo = (int64_t)i * n_in;
    hi = lo + n_in;
    q0 = (int)(lo / n_out);
    q1 = (int)min((int64_t)n_in, (hi + n_out - 1) / n_out);
}

__device__ __forceinline__ int64_t overlap(int q, int n_out, int64_t lo, int64_t hi)
{
    return min(hi, (int64_t)(q + 1) * n_out) - max(lo, (int64_t)q * n_out);
}

template <typename FT>
__device__ __forceinline__ float resample_at(const FT *in, const PreGeom &g, int64_t e)
{
    // n_out = C h_out w_out < 2^32 (planes of at most 2^30 pixels, C <= 4):
    // a 32-bit unsigned division is exact
    const uint32_t per = (uint32_t)g.h_out * (uint32_t)g.w_out;
    const uint32_t eu = (uint32_t)e;
    const int c = (int)(eu / per);
    const int r = (int)(eu - (uint32_t)c * per);
    const int i = r / g.w_out, j = r - (r / g.w_out) * g.w_out;
    int y0, y1, x0, x1;
    int64_t ylo, yhi, xlo, xhi;
    footprint(i, g.h_in, g.h_out, y0, y1, ylo, yhi);
    footprint(j, g.w_in, g.w_out, x0, x1, xlo, xhi);
    const FT *plane = in + (int64_t)c * g.in_pitch;
    float acc = 0.f;
    for (int y = y0; y < y1; ++y) {
        const int64_t oy = overlap(y, g.h_out, ylo, yhi);
        if (oy <= 0) continue;
        float row = 0.f;
        for (int x = x0; x < x1; ++x) {
            const int64_t ox = overlap(x, g.w_out, xlo, xhi);
            if (ox > 0) row = fmaf((float)ox, (float)plane[(int64_t)y * g.w_in + x], row);
        }
        acc = fmaf((float)oy, row, acc);
    }
    return acc / ((float)g.h_in * (float)g.w_in);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// phase frame: v = resampled entry, written raw to out; mean += (v - mean) / n;
// per-block FP64 partial sums of v and v^2 (fixed order within the block)
template <typename FT>
__global__ void __launch_bounds__(PT) k_pre_update(const FT *in, PreGeom g, float *out, float *mean, float inv_n,
                                                   double *partials)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * PT + threadIdx.x; e < g.n_out; e += (int64_t)gridDim.x * PT) {
        const float v = resample_at(in, g, e);
        const float m = mean[e];
        mean[e] = fmaf(v - m, inv_n, m);
        out[e] = v;
        s1 += (double)v;
        s2 += (double)v * (double)v;
    }
    __shared__ double sh[2][PT / 32];
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s1;
        sh[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < PT / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// one warp: running sums += the partials (each lane a strided subset, then a
// fixed shuffle tree: a fixed order, and short FP64 dependency chains); the
// sample deviation of all entries seen so far (1 while undefined or zero)
__global__ void k_pre_finish(const double *partials, int nblocks, double *sums, double cnt, float *sigma)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (threadIdx.x != 0) return;
    a += sums[0];
    b += sums[1];
    sums[0] = a;
    sums[1] = b;
    double sd = 1.0;
    if (cnt >= 2.0) {
        const double var = (b - a * a / cnt) / (cnt - 1.0);
        if (var > 0.0) sd = sqrt(var);
    }
    *sigma = (float)sd;
}

__global__ void __launch_bounds__(PT) k_pre_normalize(float *out, const float *mean, const float *sigma, int64_t n)
{
    const float inv = 1.f / *sigma;
    for (int64_t e = (int64_t)blockIdx.x * PT + threadIdx.x; e < n; e += (int64_t)gridDim.x * PT)
        out[e] = (out[e] - mean[e]) * inv;
}

// after the phase: resampling and normalisation with the fixed statistics
template <typename FT>
__global__ void __launch_bounds__(PT) k_pre_apply(const FT *in, PreGeom g, float *out, const float *mean,
                                                  const float *sigma)
{
    const float inv = 1.f / *sigma;
    for (int64_t e = (int64_t)blockIdx.x * PT + threadIdx.x; e < g.n_out; e += (int64_t)gridDim.x * PT)
        out[e] = (resample_at(in, g, e) - mean[e]) * inv;
}

// 3 x 3 median of a binary mask, border replicated: 1 iff at least 5 of 9
__global__ void __launch_bounds__(PT) k_median3x3(const uint8_t *in, uint8_t *out, int W, int H)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t p = (int64_t)blockIdx.x * PT + threadIdx.x; p < n; p += (int64_t)gridDim.x * PT) {
        const int y = (int)(p / W), x = (int)(p - (int64_t)y * W);
        int cnt = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = min(max(y + dy, 0), H - 1);
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = min(max(x + dx, 0), W - 1);
                cnt += in[(int64_t)yy * W + xx] != 0;
            }
        }
        out[p] = cnt >= 5 ? 1 : 0;
    }
}

int grid_for(int64_t n, int cap)
{
    const int64_t b = (n + PT - 1) / PT;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

std::string g_pre_err;

} // namespace

struct prost_pre {
    PreGeom g;
    int fdt, i_init, n;
    int device;
    cudaStream_t stream;
    float *mean, *sigma, *out_buf;
    double *sums, *partials;
    void *in_buf;
    int nblocks;
    std::string err;
};

#define PRE_CK(call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            p->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
            return e_ == cudaErrorMemoryAllocation ? PROST_ENOMEM : PROST_ECUDA;             \
        }                                                                                    \
    } while (0)

static void pre_free(prost_pre *p)
{
    if (p->mean) cudaFree(p->mean);
    if (p->sigma) cudaFree(p->sigma);
    if (p->sums) cudaFree(p->sums);
    if (p->partials) cudaFree(p->partials);
    if (p->in_buf) cudaFree(p->in_buf);
    if (p->out_buf) cudaFree(p->out_buf);
}

static int pre_alloc(prost_pre *p)
{
    const int64_t in_bytes = (int64_t)p->g.C * p->g.in_pitch * (p->fdt == PROST_U8 ? 1 : 4);
    PRE_CK(cudaMalloc(&p->mean, (size_t)p->g.n_out * sizeof(float)));
    PRE_CK(cudaMalloc(&p->sigma, sizeof(float)));
    PRE_CK(cudaMalloc(&p->sums, 2 * sizeof(double)));
    PRE_CK(cudaMalloc(&p->partials, (size_t)2 * p->nblocks * sizeof(double)));
    PRE_CK(cudaMalloc(&p->in_buf, (size_t)in_bytes));
    PRE_CK(cudaMalloc(&p->out_buf, (size_t)p->g.n_out * sizeof(float)));
    PRE_CK(cudaMemsetAsync(p->mean, 0, (size_t)p->g.n_out * sizeof(float), p->stream));
    PRE_CK(cudaMemsetAsync(p->sums, 0, 2 * sizeof(double), p->stream));
    const float one = 1.f;
    PRE_CK(cudaMemcpyAsync(p->sigma, &one, sizeof(float), cudaMemcpyHostToDevice, p->stream));
    PRE_CK(cudaStreamSynchronize(p->stream));
    return PROST_OK;
}

extern "C" int prost_pre_init(int32_t w_in, int32_t h_in, int32_t channels, int32_t w_out, int32_t h_out,
                              int32_t frame_dtype, int32_t i_init, void *stream, prost_pre **out)
{
    if (!out) { g_pre_err = "out is NULL"; return PROST_EINVAL; }
    *out = nullptr;
    if (w_in < 1 || h_in < 1 || w_out < 1 || h_out < 1 || channels < 1 || channels > 4) {
        g_pre_err = "sizes must be positive and channels in 1..4";
        return PROST_EINVAL;
    }
    if ((int64_t)w_in * h_in > (1ll << 30) || (int64_t)w_out * h_out > (1ll << 30)) {
        g_pre_err = "planes larger than 2^30 pixels";
        return PROST_EINVAL;
    }
    if (frame_dtype != PROST_U8 && frame_dtype != PROST_F32) { g_pre_err = "frame_dtype"; return PROST_EINVAL; }
    if (i_init < 1) { g_pre_err = "i_init must be >= 1"; return PROST_EINVAL; }
    prost_pre *p = new (std::nothrow) prost_pre();
    if (!p) { g_pre_err = "host allocation failed"; return PROST_ENOMEM; }
    p->g.w_in = w_in;
    p->g.h_in = h_in;
    p->g.C = channels;
    p->g.w_out = w_out;
    p->g.h_out = h_out;
    p->g.n_out = (int64_t)channels * h_out * w_out;
    p->g.in_pitch = (int64_t)w_in * h_in;
    p->fdt = frame_dtype;
    p->i_init = i_init;
    p->n = 0;
    p->stream = (cudaStream_t)stream;
    p->nblocks = grid_for(p->g.n_out, PB_MAX);
    if (cudaGetDevice(&p->device) != cudaSuccess) { g_pre_err = "no CUDA device"; delete p; return PROST_ECUDA; }
    const int rc = pre_alloc(p);
    if (rc) {
        g_pre_err = p->err;
        pre_free(p);
        delete p;
        return rc;
    }
    *out = p;
    return PROST_OK;
}

template <typename FT> static int pre_launch(prost_pre *p, const FT *in, float *dst)
{
    const int grid = p->nblocks;
    if (p->n < p->i_init) {
        p->n += 1;
        k_pre_update<FT><<<grid, PT, 0, p->stream>>>(in, p->g, dst, p->mean, 1.f / (float)p->n, p->partials);
        PRE_CK(cudaGetLastError());
        const double cnt = (double)p->n * (double)p->g.n_out;
        k_pre_finish<<<1, 32, 0, p->stream>>>(p->partials, grid, p->sums, cnt, p->sigma);
        PRE_CK(cudaGetLastError());
        k_pre_normalize<<<grid, PT, 0, p->stream>>>(dst, p->mean, p->sigma, p->g.n_out);
        PRE_CK(cudaGetLastError());
    } else {
        k_pre_apply<FT><<<grid, PT, 0, p->stream>>>(in, p->g, dst, p->mean, p->sigma);
        PRE_CK(cudaGetLastError());
    }
    return PROST_OK;
}

extern "C" int prost_pre_apply(prost_pre *p, const void *frame, int on_device, float *out)
{
    if (!p) return PROST_EINVAL;
    if (!frame || !out) { p->err = "frame and out must not be NULL"; return PROST_EINVAL; }
    const size_t eb = p->fdt == PROST_U8 ? 1 : 4;
    const size_t in_bytes = (size_t)p->g.C * p->g.in_pitch * eb;
    const void *src = frame;
    float *dst = out;
    if (!on_device) {
        PRE_CK(cudaMemcpyAsync(p->in_buf, frame, in_bytes, cudaMemcpyHostToDevice, p->stream));
        src = p->in_buf;
        dst = p->out_buf;
    }
    const int rc = p->fdt == PROST_U8 ? pre_launch(p, static_cast<const uint8_t *>(src), dst)
                                      : pre_launch(p, static_cast<const float *>(src), dst);
    if (rc) return rc;
    if (!on_device) {
        PRE_CK(cudaMemcpyAsync(out, dst, (size_t)p->g.n_out * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
        PRE_CK(cudaStreamSynchronize(p->stream));
    }
    return PROST_OK;
}

extern "C" int prost_pre_get_stats(prost_pre *p, float *mean_out, double *sigma_out, int32_t *frames_out)
{
    if (!p) return PROST_EINVAL;
    PRE_CK(cudaStreamSynchronize(p->stream));
    if (mean_out)
        PRE_CK(cudaMemcpy(mean_out, p->mean, (size_t)p->g.n_out * sizeof(float), cudaMemcpyDeviceToHost));
    if (sigma_out) {
        float s = 1.f;
        PRE_CK(cudaMemcpy(&s, p->sigma, sizeof(float), cudaMemcpyDeviceToHost));
        *sigma_out = s;
    }
    if (frames_out) *frames_out = p->n;
    return PROST_OK;
}

namespace {

// Checkpoint layout: this header, then the mean plane (n_out floats).
struct PreStateHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t w_in, h_in, C, w_out, h_out, fdt, i_init, n;
    double sums[2]; // FP64 running sums of v and v^2 over the frames counted
    float sigma;
    uint32_t pad;
    uint64_t mean_bytes;
};

} // namespace

extern "C" int prost_pre_get_state(prost_pre *p, void *buf, size_t *len)
{
    if (!p || !len) return PROST_EINVAL;
    const size_t mean_bytes = (size_t)p->g.n_out * sizeof(float);
    const size_t need = sizeof(PreStateHeader) + mean_bytes;
    if (!buf) {
        *len = need;
        return PROST_OK;
    }
    if (*len < need) { p->err = "buffer too small"; return PROST_EINVAL; }
    PreStateHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "PROSTPR1", 8);
    hd.version = 1;
    hd.header_bytes = sizeof(hd);
    hd.w_in = p->g.w_in;
    hd.h_in = p->g.h_in;
    hd.C = p->g.C;
    hd.w_out = p->g.w_out;
    hd.h_out = p->g.h_out;
    hd.fdt = p->fdt;
    hd.i_init = p->i_init;
    hd.n = p->n;
    hd.mean_bytes = mean_bytes;
    PRE_CK(cudaStreamSynchronize(p->stream));
    PRE_CK(cudaMemcpy(hd.sums, p->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    PRE_CK(cudaMemcpy(&hd.sigma, p->sigma, sizeof(float), cudaMemcpyDeviceToHost));
    char *b = static_cast<char *>(buf);
    memcpy(b, &hd, sizeof(hd));
    PRE_CK(cudaMemcpy(b + sizeof(hd), p->mean, mean_bytes, cudaMemcpyDeviceToHost));
    *len = need;
    return PROST_OK;
}

extern "C" int prost_pre_set_state(prost_pre *p, const void *buf, size_t len)
{
    if (!p || !buf) return PROST_EINVAL;
    PreStateHeader hd;
    if (len < sizeof(hd)) { p->err = "buffer too small"; return PROST_EINVAL; }
    memcpy(&hd, buf, sizeof(hd));
    const size_t mean_bytes = (size_t)p->g.n_out * sizeof(float);
    if (memcmp(hd.magic, "PROSTPR1", 8) != 0 || hd.version != 1 || hd.header_bytes != sizeof(hd) ||
        hd.mean_bytes != mean_bytes || len < sizeof(hd) + mean_bytes) {
        p->err = "not a pre-processor state buffer of this version";
        return PROST_EINVAL;
    }
    if (hd.w_in != p->g.w_in || hd.h_in != p->g.h_in || hd.C != p->g.C || hd.w_out != p->g.w_out ||
        hd.h_out != p->g.h_out || hd.fdt != p->fdt || hd.i_init != p->i_init || hd.n < 0 || hd.n > p->i_init ||
        !(hd.sigma > 0.f)) {
        p->err = "the state was made with other sizes, frame type or i_init";
        return PROST_EINVAL;
    }
    PRE_CK(cudaStreamSynchronize(p->stream));
    PRE_CK(cudaMemcpy(p->sums, hd.sums, 2 * sizeof(double), cudaMemcpyHostToDevice));
    PRE_CK(cudaMemcpy(p->sigma, &hd.sigma, sizeof(float), cudaMemcpyHostToDevice));
    PRE_CK(cudaMemcpy(p->mean, static_cast<const char *>(buf) + sizeof(hd), mean_bytes, cudaMemcpyHostToDevice));
    p->n = hd.n;
    return PROST_OK;
}

extern "C" const char *prost_pre_last_error(const prost_pre *p)
{
    return p ? p->err.c_str() : g_pre_err.c_str();
}

extern "C" void prost_pre_destroy(prost_pre *p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    pre_free(p);
    delete p;
}

extern "C" int prost_median3x3(const uint8_t *mask_in, uint8_t *mask_out, int32_t width, int32_t height,
                               int on_device, void *stream)
{
    if (!mask_in || !mask_out || width < 1 || height < 1 || (int64_t)width * height > (1ll << 30))
        return PROST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)width * height;
    const uint8_t *src = mask_in;
    uint8_t *dst = mask_out;
    uint8_t *buf = nullptr;
    if (!on_device) {
        if (cudaMalloc(&buf, (size_t)2 * n) != cudaSuccess) return PROST_ENOMEM;
        if (cudaMemcpyAsync(buf, mask_in, (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaFree(buf);
            return PROST_ECUDA;
        }
        src = buf;
        dst = buf + n;
    } else if (mask_in == mask_out) {
        return PROST_EINVAL; // the filter reads neighbours: it cannot run in place
    }
    k_median3x3<<<grid_for(n, 8192), PT, 0, s>>>(src, dst, width, height);
    int rc = cudaGetLastError() == cudaSuccess ? PROST_OK : PROST_ECUDA;
    if (!on_device) {
        if (rc == PROST_OK && (cudaMemcpyAsync(mask_out, dst, (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                               cudaStreamSynchronize(s) != cudaSuccess))
            rc = PROST_ECUDA;
        cudaFree(buf);
    }
    return rc;
}
