// One persistent, cooperative launch per frame of pROST's update
// (arXiv:1302.2073, Section 3.3) for sm_103a.
//
// Every CTA (one per SM) owns a fixed range of the stored subspace's tiles for
// the residual passes and a fixed range of pixel tiles for the update pass.
// In the register form (k <= 10) each warp streams its rows with coalesced
// loads straight into registers: the subspace (36.9 MB at 640x480x3, k = 10)
// stays resident in the 126 MB L2 across the n_cg + 2 passes of a frame, and
// from L2 many threads with loads in flight deliver about twice the rate of a
// single-thread bulk-copy ring.  The streaming form (k >= 11) stages rows
// through shared memory with asynchronous copies (prost_stage.cuh).
//
// Phases:
//   residual pass j = 0..n_cg: per row r = x - U y_j, the cost, U^T eta and
//     (j < n_cg) U^T diag(c) U; CTA partial row -> grid barrier -> every CTA
//     sums all partial rows in the same fixed order and runs the same k-space
//     step (PR+ CG step, or for j = n_cg the rank-one SVD and the geodesic
//     angle of Step 2), so all CTAs hold identical k-space state without a
//     second barrier.
//   update pass: geodesic update of every row (written back), labels and
//     weights of Step 3 (max over channels), optional background, Gram of the
//     new subspace; the last CTA to arrive factors that Gram (Cholesky-QR to
//     FP64 accuracy, folded into the next frame) and writes the k-space state
//     back.
//
// Every wait is bounded (about one second of SM clock): a grid barrier that
// does not complete sets a global abort flag and PROST_ETIMEOUT in the state
// and the CTAs return.  The grid barrier counter only grows; the host passes
// the value it must hold at launch, and a launch that finds another value (a
// previous launch aborted) does nothing but raise the error.
#pragma once

#include <string.h>

#include "prost_kernels.cuh"
#include "prost_stage.cuh"

namespace prost {

template <int K, typename UT = float> struct FCfg {
    // k <= 10: the register form, 16 warps (at most 4 per SM sub-partition,
    // so each thread may hold 128 registers), rows loaded straight into
    // registers and computed in FP32 whatever the storage type; the subspace
    // of the 640x480 workload stays in L2 across the passes of a frame.
    // k >= 11: the streaming form (prost_stage.cuh), rows staged through
    // shared memory: float32 8 warps of up to 255 registers; bfloat16 16 warps
    // of up to 128 registers (the products of the passes on tensor cores leave
    // a lane few sums).  One CTA per SM.
    static constexpr bool STREAM = K > KREG;
    static constexpr int THREADS = STREAM && sizeof(UT) == 4 ? 256 : 512;
    static constexpr int NW = THREADS / 32;
    static constexpr int TP = TILE_P;            // pixels per tile
    static constexpr int RW = 2;                 // rows per thread per item (8-byte loads)
    static constexpr int IPT = TP / RW;          // items per tile
    static constexpr int NM = K * (K + 1) / 2;
    static constexpr int NVR = K + NM + 3;       // CG pass partial row
    static constexpr int NVF = K + 3;            // final pass partial row
    static constexpr int NVU = NM + 1;           // update pass partial row
    static constexpr int NPR = (NVR + 31) / 32 * 32;
    static constexpr int NPF = (NVF + 31) / 32 * 32;
    static constexpr int NPU = (NVU + 31) / 32 * 32;
    static constexpr int NPMAX = NPR > NPU ? NPR : NPU;
};
static_assert(TILE_P % 2 == 0, "rows are read in pairs");

constexpr long long WAIT_LIMIT = 2000000000ll; // SM clock cycles (about 1 s)

template <int N> __device__ __forceinline__ void cons_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// two consecutive entries (RW = 2) of a frame plane or label row
__device__ __forceinline__ void ld2(const uint8_t *p, bool pair, int nvalid, float (&o)[2])
{
    if (pair) {
        const uchar2 v = __ldg(reinterpret_cast<const uchar2 *>(p));
        o[0] = v.x;
        o[1] = v.y;
    } else {
        o[0] = nvalid > 0 ? (float)__ldg(p) : 0.f;
        o[1] = nvalid > 1 ? (float)__ldg(p + 1) : 0.f;
    }
}
__device__ __forceinline__ void ld2(const float *p, bool pair, int nvalid, float (&o)[2])
{
    if (pair) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x;
        o[1] = v.y;
    } else {
        o[0] = nvalid > 0 ? __ldg(p) : 0.f;
        o[1] = nvalid > 1 ? __ldg(p + 1) : 0.f;
    }
}

// ---- shared k-space state (identical copy in every CTA) -----------------------

template <int K> struct SKState {
    double y[K];       // coefficients in the orthonormal basis U = U_st T (FP64 storage)
    float gprev[K], d[K];
    float yf[K];       // T y: coefficients of the stored rows
    float tv[K], tg[K];// T v and T g: dots of stored rows with v and g (Step 2)
    float w[K];        // R^T v: the update direction in the stored basis
    float Tf[K * K];   // T = R^{-1}, row-major upper triangular
    float Rf[K * K];   // R, row-major upper triangular
    float cm1, snp, yn;
    float apend;       // resident form: the last CG step's alpha, its FP64 y update pending
    int ypend;
    int proj;          // |pi(eta)| is formed by the explicit projection pass
    int skip;          // frame rejected (non-finite entry)
    int err;           // a grid barrier gave up
    int last;          // this CTA arrived last at the end of the frame
    int pad;
    int64_t frame_index;
};

// Sum of all CTAs' partial rows in a fixed order (Kahan-compensated FP32),
// by the NCONS threads of the CTA, identical in every CTA.  The nrows rows are
// dealt round-robin into ng groups of at most RED_ROWS rows (more groups when
// nv is small, so that every thread has work); a unit (group, value) is one
// thread's batch of loads and compensated sum, two units per thread are in
// flight at a time, and the ng group sums of each value are added in group
// order.  One out-of-line body serves every pass of the frame, so the code the
// last CTA runs at the end of the frame is already in the instruction caches.

__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float yk = v - c, tk = s + yk;
    c = (tk - s) - yk;
    s = tk;
}

template <int NCONS>
__device__ __noinline__ void reduce_rows(const float *rows, int nrows, int stride, int nv, float *tot, float *scr)
{
    static_assert(RED_SCR >= NCONS, "scratch of the group sums");
    const int t = threadIdx.x;
    int ng = max((nrows + RED_ROWS - 1) / RED_ROWS, NCONS / nv);
    ng = max(1, min(ng, min(nrows, RED_SCR / nv)));
    const int nu = ng * nv;
    const size_t step = (size_t)ng * stride; // between the rows of a unit
    // unit u: rows g, g + ng, ... of value c, with u = g nv + c
    auto unit1 = [&](int u) {
        const int g = u / nv, c = u - g * nv;
        const float *p = rows + (size_t)g * stride + c;
        float s = 0.f, k = 0.f;
        for (int b0 = g; b0 < nrows; b0 += RED_ROWS * ng, p += RED_ROWS * step) {
            float v[RED_ROWS];
#pragma unroll
            for (int q = 0; q < RED_ROWS; ++q) v[q] = b0 + q * ng < nrows ? __ldcg(p + q * step) : 0.f;
#pragma unroll
            for (int q = 0; q < RED_ROWS; ++q) kahan_add(s, k, v[q]);
        }
        scr[u] = s;
    };
    if (nu <= NCONS) {
        if (t < nu) unit1(t);
    } else {
        for (int u0 = t; u0 < nu; u0 += 2 * NCONS) {
            const int u1 = u0 + NCONS;
            if (u1 >= nu) {
                unit1(u0);
                continue;
            }
            // two units with their loads in flight together
            const int g0 = u0 / nv, c0 = u0 - g0 * nv;
            const int g1 = u1 / nv, c1 = u1 - g1 * nv;
            const float *p0 = rows + (size_t)g0 * stride + c0;
            const float *p1 = rows + (size_t)g1 * stride + c1;
            float s0 = 0.f, k0 = 0.f, s1 = 0.f, k1 = 0.f;
            for (int b0 = g0, b1 = g1; b0 < nrows;
                 b0 += RED_ROWS * ng, b1 += RED_ROWS * ng, p0 += RED_ROWS * step, p1 += RED_ROWS * step) {
                float v0[RED_ROWS], v1[RED_ROWS];
#pragma unroll
                for (int q = 0; q < RED_ROWS; ++q) {
                    v0[q] = b0 + q * ng < nrows ? __ldcg(p0 + q * step) : 0.f;
                    v1[q] = b1 + q * ng < nrows ? __ldcg(p1 + q * step) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < RED_ROWS; ++q) {
                    kahan_add(s0, k0, v0[q]);
                    kahan_add(s1, k1, v1[q]);
                }
            }
            scr[u0] = s0;
            scr[u1] = s1;
        }
    }
    cons_sync<NCONS>();
    for (int c = t; c < nv; c += NCONS) {
        float s = 0.f, k = 0.f;
        for (int g = 0; g < ng; ++g) kahan_add(s, k, scr[g * nv + c]);
        tot[c] = s;
    }
    cons_sync<NCONS>();
}

// Sum of all CTAs' partial values in a fixed order (Kahan-compensated FP32),
// by the NCONS threads of the CTA, identical in every CTA, for the frame
// kernel's value-major layout: value c of CTA b at cols[c * cstride + b]
// (cstride a multiple of 4, at least nrows).  A unit (value c, chunk q) sums
// rows [q RED_ROWS, (q + 1) RED_ROWS) of one value with 16-byte loads, a
// load only where it starts below nrows (so it ends inside the value's
// cstride entries); units of one value are then added in chunk order.
template <int NCONS>
__device__ __noinline__ void reduce_cols(const float *cols, int nrows, int cstride, int nv, float *tot, float *scr)
{
    static_assert(RED_ROWS % 4 == 0, "whole 16-byte loads per chunk");
    const int t = threadIdx.x;
    const int nq = (nrows + RED_ROWS - 1) / RED_ROWS;
    const int nu = nq * nv; // unit u = c nq + q
    for (int u = t; u < nu; u += NCONS) {
        const int c = u / nq, q = u - c * nq;
        const int r0 = q * RED_ROWS;
        const float4 *p = reinterpret_cast<const float4 *>(cols + (size_t)c * cstride + r0);
        float4 v[RED_ROWS / 4];
#pragma unroll
        for (int i = 0; i < RED_ROWS / 4; ++i)
            v[i] = r0 + 4 * i < nrows ? __ldcg(p + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        // four compensated sums, one per lane of the 16-byte loads (shorter
        // dependent chains), added in a fixed order
        float s0 = 0.f, k0 = 0.f, s1 = 0.f, k1 = 0.f, s2 = 0.f, k2 = 0.f, s3 = 0.f, k3 = 0.f;
#pragma unroll
        for (int i = 0; i < RED_ROWS / 4; ++i) {
            const int r = r0 + 4 * i;
            kahan_add(s0, k0, r < nrows ? v[i].x : 0.f);
            kahan_add(s1, k1, r + 1 < nrows ? v[i].y : 0.f);
            kahan_add(s2, k2, r + 2 < nrows ? v[i].z : 0.f);
            kahan_add(s3, k3, r + 3 < nrows ? v[i].w : 0.f);
        }
        float s = 0.f, k = 0.f;
        kahan_add(s, k, s0);
        kahan_add(s, k, s1);
        kahan_add(s, k, s2);
        kahan_add(s, k, s3);
        kahan_add(s, k, -((k0 + k1) + (k2 + k3)));
        scr[u] = s;
    }
    cons_sync<NCONS>();
    for (int c = t; c < nv; c += NCONS) {
        float s = 0.f, k = 0.f;
        for (int q = 0; q < nq; ++q) kahan_add(s, k, scr[c * nq + q]);
        tot[c] = s;
    }
    cons_sync<NCONS>();
}

// The same sum for the resident form, by warps: warp w takes values w, w + NW,
// ... (VPW at most), lane l the 16-byte chunks l, l + 32, ... (CPL at most) of
// each value's row, so that every load instruction of a warp reads 512
// contiguous bytes; all of a warp's loads are in flight before the first sum.
// Each lane adds its entries below nrows in order, then a fixed shuffle tree
// adds the 32 lane sums.  Plain FP32 (about log2(nrows) roundings per value)
// in a fixed order: identical in every CTA and from run to run.  Needs
// nv <= VPW * NT / 32 and nrows <= 128 * CPL.
template <int NT, int VPW, int CPL>
__device__ __noinline__ void reduce_cols_warp(const float *cols, int nrows, int cstride, int nv, float *tot)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nch = (nrows + 3) >> 2;
    float4 v[VPW][CPL];
#pragma unroll
    for (int i = 0; i < VPW; ++i) {
        const int c = w + i * NW;
        const float4 *row = reinterpret_cast<const float4 *>(cols + (size_t)(c < nv ? c : 0) * cstride);
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int ch = lane + 32 * j;
            v[i][j] = (c < nv && ch < nch) ? __ldcg(row + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
#pragma unroll
    for (int i = 0; i < VPW; ++i) {
        const int c = w + i * NW;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int r = 4 * (lane + 32 * j);
            s += r < nrows ? v[i][j].x : 0.f;
            s += r + 1 < nrows ? v[i][j].y : 0.f;
            s += r + 2 < nrows ? v[i][j].z : 0.f;
            s += r + 3 < nrows ? v[i][j].w : 0.f;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
        if (lane == 0 && c < nv) tot[c] = s;
    }
    cons_sync<NT>();
}

// The same out of line: the register form's grid launches keep more live
// values around their sums than the resident form, which inlines them.
template <int NT, int VPW, int CPL>
__device__ __noinline__ void reduce_cols_warp_call(const float *cols, int nrows, int cstride, int nv, float *tot)
{
    reduce_cols_warp<NT, VPW, CPL>(cols, nrows, cstride, nv, tot);
}

// CTA sum of N per-thread values (all threads), the first nv written to
// out[i * os] (and to nrep - 1 more copies, rstride floats apart).  The grid
// barrier that follows orders these stores before its arrival (CTA barrier,
// then one fence by the arriving thread).
template <int N, int NCW>
__device__ __forceinline__ void cons_partials(float (&v)[N], int nv, float *out, float *sred, int os, int nrep = 1,
                                              size_t rstride = 0)
{
    warp_split_reduce<N>(v);
    constexpr int PER = N / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < PER; ++s) sred[w * N + lane * PER + s] = v[s];
    cons_sync<NCW * 32>();
    for (int i = threadIdx.x; i < nv; i += NCW * 32) {
        float a = 0.f;
#pragma unroll
        for (int ww = 0; ww < NCW; ++ww) a += sred[ww * N + i];
        for (int r = 0; r < nrep; ++r) out[(size_t)i * os + r * rstride] = a;
    }
}

// As cons_partials, with a plain shuffle tree per value (static indices
// only): for the streaming form's long per-lane vectors, where the lane-
// dependent selects of the split reduction would put the vector in local memory.
template <int N, int NCW, int NA, int S0 = 0, int S1 = 0>
__device__ __forceinline__ void cons_partials_tree(float (&v)[NA], int nv, float *out, float *sred, int os,
                                                   int nrep = 1, size_t rstride = 0)
{
    static_assert(N <= NA, "values beyond the array");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i >= S0 && i < S1) continue; // values another reduction writes
        float x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
        if (lane == (i & 31)) sred[w * N + i] = x;
    }
    cons_sync<NCW * 32>();
    for (int i = threadIdx.x; i < nv; i += NCW * 32) {
        if (i >= S0 && i < S1) continue;
        float a = 0.f;
#pragma unroll
        for (int ww = 0; ww < NCW; ++ww) a += sred[ww * N + i];
        for (int r = 0; r < nrep; ++r) out[(size_t)i * os + r * rstride] = a;
    }
}

// The warps' 16 x 16 tensor-core results (at res_off in each warp's shared
// memory, warp_bytes apart) summed in a fixed order into the packed upper
// triangle out[0 .. K(K+1)/2).
template <int K, int NCW>
__device__ __forceinline__ void mma_row(const unsigned char *base, int warp_bytes, int res_off, float *out, int os)
{
    cons_sync<NCW * 32>(); // every warp has stored its result
    constexpr int NM = K * (K + 1) / 2;
    for (int i = threadIdx.x; i < NM; i += NCW * 32) {
        int j = 0, t = i;
        while (t >= K - j) {
            t -= K - j;
            ++j;
        }
        const int l = j + t;
        float a = 0.f;
        for (int w = 0; w < NCW; ++w) a += reinterpret_cast<const float *>(base + w * warp_bytes + res_off)[j * 16 + l];
        out[(size_t)i * os] = a;
    }
}

// Arrival at the grid barrier as one release reduction: the CTA barrier
// before it orders the other threads' stores, and the release makes them
// visible with the arrival (no separate fence, no returned value).
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier: arrive, wait (bounded) until all CTAs arrived.
// A wait that gives up (or sees another CTA's abort) marks the frame timed
// out: the abort flag, ERR_TIMEOUT and the frame's status PROST_ETIMEOUT.
// REL (the resident form): the arrival is a release reduction and the acquire
// load that ends the wait orders what follows; otherwise a fence, an atomic
// add, and a fence after the wait.
// ARRIVE = false: wait only (the resident form's end CTA, which arrived already).
template <int NCONS, bool REL = false, bool ARRIVE = true>
__device__ __forceinline__ bool grid_wait(GridBar *gb, unsigned long long target, int *s_err, KState *ks,
                                          int32_t *st_out, long long limit = WAIT_LIMIT)
{
    cons_sync<NCONS>();
    if (threadIdx.x == 0) {
        int ok = *s_err == 0;
        if (ok) {
            if constexpr (!ARRIVE) {
            } else if constexpr (REL) {
                red_release_add(&gb->count, 1ull);
            } else {
                __threadfence(); // the CTA's partial values (ordered by the CTA barrier) before the arrival
                atomicAdd(&gb->count, 1ull);
            }
            const long long t0 = clock64();
            unsigned it = 0;
            while (ld_acquire_u64(&gb->count) < target) {
                if ((++it & 15u) == 0) {
                    if (*(volatile int *)&gb->abort || clock64() - t0 > limit) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (!ok) {
            atomicExch(&gb->abort, 1);
            atomicOr(&ks->err_flags, ERR_TIMEOUT);
            ks->last_status = -5; // PROST_ETIMEOUT
            if (st_out) *st_out = -5;
            *s_err = 1;
        }
        if (!REL || !ok) __threadfence();
    }
    cons_sync<NCONS>();
    return *(volatile int *)s_err == 0;
}

// Barrier of the cluster form: every thread of every CTA of the cluster
// arrives (releasing its global-memory writes at cluster scope) and waits
// (acquiring the others').  It is the hardware cluster barrier, reached by
// all CTAs because the cluster form has no early return before the end of
// the frame (every decision between barriers is taken on identical data).
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The synchronisation between a pass's partial values and their reduction:
// the cluster barrier (cluster form) or the bounded grid barrier, whose
// failure marks the frame timed out.
template <bool CL, int NCONS, bool REL = false>
__device__ __forceinline__ bool pass_sync(GridBar *gb, unsigned long long target, int *s_err, KState *ks,
                                          int32_t *st_out, long long limit = WAIT_LIMIT)
{
    if constexpr (CL) {
        cluster_sync_all();
        return true;
    } else {
        return grid_wait<NCONS, REL>(gb, target, s_err, ks, st_out, limit);
    }
}

// ---- k-space steps on the shared copy (one warp) ---------------------------------

__device__ __forceinline__ float wsumf(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Step size of frame i (Section 3.3): t = max(exp(-tau i) t_init, t_min), to
// FP32 accuracy, which is all that theta = sigma t (FP32) uses.  The exponent
// is reduced as tau i = q ln 2 + r with the product and the reduction in FP64
// (two operations; a library FP64 exponential is a long chain on GB300's
// narrow FP64 pipe), then exp(-tau i) = 2^-q exp(-r) with |r| <= ln 2 in FP32.
__device__ __forceinline__ float step_size(const DevParams &prm, int64_t i)
{
    const double a = prm.tau * (double)i;
    float e = 0.f;
    if (a < 200.0) {
        const float q = rintf((float)a * 1.44269504f);
        const float r = (float)fma(-(double)q, 0.69314718055994530942, a);
        e = ldexpf(expf(-r) * (float)prm.t_init, -(int)q);
    }
    return fmaxf(e, (float)prm.t_min);
}

// Below this fraction of |eta|^2, |pi(eta)|^2 is formed by the explicit
// projection pass rather than as |eta|^2 - |U^T eta|^2: above it the FP32
// sums (relative error about 1e-6) leave |pi(eta)| accurate to about 2e-6.
constexpr float PROJ_RATIO = 0.25f;

// Step 2's angle from |pi(eta)| (one thread): sigma = |pi(eta)| |y| (Eq. svd),
// theta = sigma t (Eq. geodesic), skipped when |y| = 0 or |pi(eta)| = 0.
template <int K>
__device__ __forceinline__ void step_angle(SKState<K> &sk, const DevParams &prm, float pin, KState *gks, bool stats)
{
    const float yn = sk.yn;
    const bool upd = yn > 0.f && pin > 0.f;
    const float t = step_size(prm, sk.frame_index);
    const float sigma = pin * yn;
    const float theta = sigma * t;
    const float sh = sinf(0.5f * theta);
    sk.cm1 = upd ? -2.f * sh * sh : 0.f;
    sk.snp = upd ? sinf(theta) / pin : 0.f;
    if (stats) {
        gks->pi_norm = pin;
        gks->y_norm = yn;
        gks->sigma = sigma;
        gks->t = t;
        gks->theta = upd ? theta : 0.f;
        gks->updated = upd ? 1 : 0;
    }
}

// CG bookkeeping at iterate `pass` from the reduced sums tot:
//   WM:  tot = [g_st (K) | M_st packed (K(K+1)/2) | f | |eta|^2 | #non-finite]
//   !WM: tot = [g_st (K) | f | |eta|^2 | #non-finite]
// g_st = U_st^T eta and M_st = U_st^T diag(c) U_st refer to the stored rows;
// with U = U_st T the gradient is g = T^T g_st and d^T M d = (T d)^T M_st (T d).
// The k-vector algebra is FP32 (k <= 16 terms per dot product); y is kept in
// FP64 and the step size t (an exponential of the frame counter) is FP64.
// GB300's FP64 pipe is narrow and long-latency, so FP64 stays off the chains.
// CTA 0 also records the statistics in the global state.
// DEFER (the resident form): the FP64 update of y is left to another warp at
// the start of the next pass (sk.apend, sk.ypend), off this step's chain.
template <int K, bool WM, bool DEFER = false>
__device__ void kspace_cg(SKState<K> &sk, const DevParams &prm, const float *tot, int pass, KState *gks,
                          bool stats)
{
    constexpr int NM = WM ? K * (K + 1) / 2 : 0;
    const int l = threadIdx.x;
    const bool act = l < K;
    const float f = tot[K + NM], ee = tot[K + NM + 1], nbad = tot[K + NM + 2];
    if (pass == 0 && nbad > 0.f) {
        if (l == 0) sk.skip = 1;
        __syncwarp();
    }
    // g = T^T g_st (T upper triangular): every product issued at once
    float gl = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (act && i <= l) gl = fmaf(sk.Tf[i * K + l], tot[i], gl);
    const float gsq = wsumf(act ? gl * gl : 0.f);
    float beta = 0.f, dl;
    if (pass == 0) {
        dl = act ? -gl : 0.f;
    } else {
        const float gp = act ? sk.gprev[l] : 0.f;
        const float ggp = wsumf(gp * gp);
        const float num = wsumf(act ? gl * (gl - gp) : 0.f);
        beta = ggp > 0.f ? fmaxf(0.f, num / ggp) : 0.f;
        dl = act ? fmaf(beta, sk.d[l], -gl) : 0.f;
    }
    if (stats && l == 0) {
        gks->cost[pass] = f;
        gks->gnorm[pass] = sqrtf(gsq);
        gks->beta[pass] = beta;
    }
    if (sk.skip) return;
    if (pass < prm.n_cg) {
        const float dg = wsumf(act ? dl * gl : 0.f);
        float dst = 0.f; // (T d)_l, the direction in the stored basis
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float di = __shfl_sync(FULL, dl, i);
            if (act && i >= l) dst = fmaf(sk.Tf[l * K + i], di, dst);
        }
        float md = 0.f;
        if constexpr (WM) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const float si = __shfl_sync(FULL, dst, i);
                if (act) md = fmaf(tot[K + (l <= i ? tri<K>(l, i) : tri<K>(i, l))], si, md);
            }
        }
        const float den = prm.p * wsumf(act ? dst * md : 0.f);
        const float alpha = den > 0.f ? -dg / den : 0.f;
        if (act) {
            // y in FP64; the stored-basis coefficients T y move along T d
            if constexpr (!DEFER) sk.y[l] = fma((double)alpha, (double)dl, sk.y[l]);
            sk.yf[l] = fmaf(alpha, dst, sk.yf[l]);
            sk.d[l] = dl;
            sk.gprev[l] = gl;
        }
        if (DEFER && l == 0) {
            sk.apend = alpha;
            sk.ypend = 1;
        }
        if (stats && l == 0) gks->alpha[pass] = alpha;
    } else {
        const float yl = act ? (float)sk.y[l] : 0.f;
        const float yn = sqrtf(wsumf(yl * yl));
        // |pi(eta)|^2 = |eta|^2 - |U^T eta|^2 (Eq. gproject, U orthonormal)
        // cancels when most of eta lies in span(U): below a quarter of |eta|^2
        // the FP32 sums would leave too few digits, and the explicit pass
        // sum_e (eta_e - u_e^T g)^2 (proj_pass) forms the norm instead
        const float pin2 = ee - gsq;
        const bool proj = yn > 0.f && ee > 0.f && !(pin2 > PROJ_RATIO * ee);
        const float pin = (!proj && pin2 > 0.f) ? sqrtf(pin2) : 0.f;
        const bool upd = yn > 0.f && (proj || pin > 0.f);
        // the update pass works on the stored rows u_st (u = T^T u_st): it needs
        // T v and T g for the dots and w = R^T v, since u_st + gamma R^T v is
        // the stored row of u + gamma v
        const float vl = (act && upd) ? yl / yn : 0.f;
        float tv = 0.f, tg = 0.f, wl = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float vi = __shfl_sync(FULL, vl, i);
            const float gi = __shfl_sync(FULL, gl, i);
            if (act && i >= l) {
                tv = fmaf(sk.Tf[l * K + i], vi, tv);
                tg = fmaf(sk.Tf[l * K + i], gi, tg);
            }
            if (act && i <= l) wl = fmaf(sk.Rf[i * K + l], vi, wl);
        }
        if (act) {
            sk.tv[l] = tv;
            sk.tg[l] = tg;
            sk.w[l] = wl;
        }
        if (l == 0) {
            sk.yn = yn;
            sk.proj = proj ? 1 : 0;
            if (stats) {
                gks->eta_norm = sqrtf(fmaxf(ee, 0.f));
                gks->pi_explicit = proj ? 1 : 0;
                gks->n_cg_done = prm.n_cg;
            }
            if (!proj) step_angle(sk, prm, pin, gks, stats);
        }
    }
}

// FP64 with explicit rounding, so that every kernel running the deferred
// re-orthonormalisation below produces the same bits
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1/sqrt(d) in FP64: the FP32 reciprocal square root as the start, then two
// Newton-Raphson steps y <- y (3 - d y^2) / 2, each of which squares the
// relative error (about 1e-7, 1e-14, then FP64 rounding), so the chain is six
// dependent FP64 operations.  d outside the normal FP32 range takes the
// library square root and division.
__device__ __forceinline__ double rsqrt_fp64(double d)
{
    const float df = (float)d;
    if (!(df >= 1.17549435e-38f && df <= 3.0e38f)) return 1.0 / sqrt(d);
    const double hd = dmul(-0.5, d);
    double y = (double)rsqrtf(df);
    y = dmul(y, dfma(hd, dmul(y, y), 1.5));
    y = dmul(y, dfma(hd, dmul(y, y), 1.5));
    return y;
}

// Right-looking FP64 Cholesky G = R^T R (G in sW, overwritten) and T = R^{-1}
// (row-major k x k in sR, sT) for Gram matrices away from the identity, by
// the NT threads of the CTA, one entry of the k^2 per thread per step: GB300's
// FP64 pipe is narrow per SM sub-partition, so the updates are spread over all
// warps, and only warp 0 forms each pivot's reciprocal square root (inv).
// Returns false when G is not positive definite (then R = T = I).  The pivot
// loops stay rolled: this code runs once per frame, cold in the instruction
// caches, where its size costs more than its loop overhead.
template <int K, int NT>
__device__ bool cholesky_rl(double *sR, double *sT, double *sW, double *inv)
{
    static_assert(K * K <= NT && K <= 32, "one entry per thread, a row per warp");
    const int t = threadIdx.x;
    const bool el = t < K * K;
    const int i = t / K, l = t - (t / K) * K;
    if (el) sR[t] = 0.0;
    cons_sync<NT>();
    bool ok = true;
#pragma unroll 1
    for (int a = 0; a < K; ++a) {
        const double d = sW[a * K + a]; // the same value in every thread
        if (!(d > 0.0)) {
            ok = false;
            break;
        }
        if (t < 32) {
            const double ri = rsqrt_fp64(d);
            if (t == 0) inv[a] = ri;
            if (t >= a && t < K) sR[a * K + t] = t == a ? dmul(d, ri) : dmul(sW[a * K + t], ri);
        }
        cons_sync<NT>();
        if (el && i > a && l >= i) sW[t] = dfma(-sR[a * K + i], sR[a * K + l], sW[t]);
        cons_sync<NT>();
    }
    if (!ok) {
        if (el) sR[t] = sT[t] = i == l ? 1.0 : 0.0;
    } else {
        if (el) sW[t] = i == l ? 1.0 : 0.0;
        cons_sync<NT>();
#pragma unroll 1
        for (int r = K - 1; r >= 0; --r) {
            if (t < K) sT[r * K + t] = dmul(sW[r * K + t], inv[r]);
            cons_sync<NT>();
            if (el && i < r) sW[t] = dfma(-sR[i * K + r], sT[r * K + l], sW[t]);
            cons_sync<NT>();
        }
    }
    cons_sync<NT>();
    return ok;
}

// Scratch of the end-of-frame re-orthonormalisation (last CTA).
template <int K> struct ReorthScratch {
    double R[K * K], T[K * K], W[K * K], Told[K * K], ty[K];
    double D1[K * K], D2[K * K], inv[K];
    float Xh[K * K], Xl[K * K], X2[K * K], inv32[K];
    float emax;
    int ok;
};

// Cholesky-QR factors to FP64 accuracy for a Gram matrix away from the
// identity (G in rs.W, full symmetric FP64), by the NT threads of the CTA:
//   an FP32 right-looking Cholesky G ~ R0^T R0 and T0 = R0^{-1} (FP32);
//   E = T0^T G T0 - I in FP64 (about 1e-7 whatever G is: the FP32 backward error);
//   X upper with (I + X)^T (I + X) = I + E: X = Phi(E - X^T X), two sweeps
//     from X = 0 (error |E|^3), Phi taking the upper triangle, diagonal halved;
//   T = T0 (I + X)^{-1} = T0 (I - X + X^2) (error |E|^3), so T^T G T = I;
//   R = T^T G (= R^{-T} R^T R), the upper triangle.
// Six triangular FP64 products with chains of at most k, in place of the
// k-step pivot sequence of FP64 square roots.  The refinement needs |E| small
// (it is about 1e-7 for the Grams that arise here, within about 1e-3 of I);
// when max |E| exceeds 1e-4 (an ill-conditioned G) the right-looking FP64
// Cholesky takes over.  Returns false (R = T = I) when G is not positive
// definite.
template <int K, int NT>
__device__ bool cholesky_refined(ReorthScratch<K> &rs)
{
    static_assert(K * K <= NT && K <= 32, "one entry per thread, a row per warp");
    constexpr int KK = K * K;
    const int t = threadIdx.x;
    const bool el = t < KK;
    const int i = t / K, l = t - (t / K) * K;
    float *W32 = rs.Xh, *R0 = rs.Xl, *T0 = rs.X2, *inv = rs.inv32;
    if (el) {
        W32[t] = (float)rs.W[t];
        R0[t] = 0.f;
    }
    cons_sync<NT>();
    bool ok = true;
#pragma unroll 1
    for (int a = 0; a < K; ++a) {
        const float d = W32[a * K + a]; // the same value in every thread
        if (!(d > 0.f)) {
            ok = false;
            break;
        }
        if (t < 32) {
            float ri = rsqrtf(d);
            ri = ri * fmaf(-0.5f * d * ri, ri, 1.5f);
            if (t == 0) inv[a] = ri;
            if (t >= a && t < K) R0[a * K + t] = t == a ? d * ri : W32[a * K + t] * ri;
        }
        cons_sync<NT>();
        if (el && i > a && l >= i) W32[t] = fmaf(-R0[a * K + i], R0[a * K + l], W32[t]);
        cons_sync<NT>();
    }
    if (!ok) return cholesky_rl<K, NT>(rs.R, rs.T, rs.W, rs.inv);
    if (el) W32[t] = i == l ? 1.f : 0.f;
    cons_sync<NT>();
#pragma unroll 1
    for (int r = K - 1; r >= 0; --r) {
        if (t < K) T0[r * K + t] = W32[r * K + t] * inv[r];
        cons_sync<NT>();
        if (el && i < r) W32[t] = fmaf(-R0[i * K + r], T0[r * K + l], W32[t]);
        cons_sync<NT>();
    }
    const double *G = rs.W;
    double *A = rs.D1, *E = rs.D2, *X = rs.T;
    auto phi = [&](double v) { return l > i ? v : (l == i ? 0.5 * v : 0.0); };
    // A = G T0
    if (el) {
        double s = 0.0;
        for (int q = 0; q <= l; ++q) s = dfma(G[i * K + q], (double)T0[q * K + l], s);
        A[t] = s;
    }
    cons_sync<NT>();
    // E = T0^T A - I (upper)
    if (t == 0) rs.emax = 0.f;
    cons_sync<NT>();
    if (el) {
        double s = 0.0;
        if (i <= l)
            for (int q = 0; q <= i; ++q) s = dfma((double)T0[q * K + i], A[q * K + l], s);
        E[t] = i <= l ? s - (i == l ? 1.0 : 0.0) : 0.0;
        X[t] = phi(E[t]);
        // the bit patterns of non-negative floats order like the floats
        const float ae = fabsf((float)E[t]);
        if (ae > 0.f) atomicMax(reinterpret_cast<int *>(&rs.emax), __float_as_int(ae));
    }
    cons_sync<NT>();
    if (!(rs.emax <= 1e-4f)) return cholesky_rl<K, NT>(rs.R, rs.T, rs.W, rs.inv); // also NaN
    // X = Phi(E - X^T X) with the first sweep's X
    double xn = 0.0;
    if (el && i <= l) {
        double s = 0.0;
        for (int q = 0; q <= i; ++q) s = dfma(X[q * K + i], X[q * K + l], s);
        xn = phi(E[t] - s);
    }
    cons_sync<NT>();
    if (el) X[t] = xn;
    cons_sync<NT>();
    // Y = X - X^2 (upper), into A
    if (el) {
        double s = 0.0;
        if (i <= l)
            for (int q = i; q <= l; ++q) s = dfma(X[i * K + q], X[q * K + l], s);
        A[t] = X[t] - s;
    }
    cons_sync<NT>();
    // T = T0 - T0 Y (upper), into E
    if (el) {
        double s = 0.0;
        if (i <= l)
            for (int q = i; q <= l; ++q) s = dfma((double)T0[i * K + q], A[q * K + l], s);
        E[t] = i <= l ? (double)T0[t] - s : 0.0;
    }
    cons_sync<NT>();
    if (el) rs.T[t] = E[t];
    cons_sync<NT>();
    // R = T^T G (upper)
    if (el) {
        double s = 0.0;
        if (i <= l)
            for (int q = 0; q <= i; ++q) s = dfma(rs.T[q * K + i], G[q * K + l], s);
        rs.R[t] = i <= l ? s : 0.0;
    }
    cons_sync<NT>();
    return true;
}

// End of frame, all NT threads of the last CTA: the Cholesky-QR factors of the
// new stored rows from their Gram matrix G (packed upper, FP32 sums) to FP64
// accuracy, G = R^T R and T = R^{-1}; the new state R, T, y' = R T_old y (the
// background U y is kept) and the frame's results.
//
// For a near-identity Gram (|G - I| <= 1e-5, the usual case: the geodesic step
// keeps U orthonormal up to rounding) write R = I + X with X upper triangular.
// R^T R = G reads X + X^T = E - X^T X with E = G - I, so X is the fixed point of
// X <- Phi(E - X^T X), Phi taking the upper triangle with the diagonal halved.
// X is carried as an unevaluated float sum Xh + Xl: Xh = Phi(E) is exact in
// FP32 (G - I is exact by Sterbenz's lemma, halving is exact), and the
// correction Xl = -Phi(Xh^T Xh + Xh^T Xl + Xl^T Xh), of size |E|^2 <= 1e-10,
// takes two FP32 sweeps; its rounding and the neglected terms (|E|^3 and the
// Xl^T Xl product) stay below 1e-15 absolute.  T = R^{-1} is the Neumann
// series I - X + X^2 - X^3 (the next term is below 1e-20).  The pieces are
// summed into FP64, which gives R and T to FP64 accuracy without long FP64
// dependency chains (GB300's FP64 pipe has a long latency).  Gram matrices
// farther from I (bfloat16 stored rows, whose rounding moves the Gram away
// from I) take an FP32 factorisation refined in FP64 (cholesky_refined).
template <int K, int NT>
__device__ void end_frame(const SKState<K> &sk, KState *ks, const float *G, float n_fg, ReorthScratch<K> &rs,
                          int32_t *st_out)
{
    const int t = threadIdx.x;
    const int i = t / K, l = t - (t / K) * K;
    const bool el = t < K * K;
    if (sk.skip) {
        if (t == 0) {
            ks->err_flags |= ERR_BADFRAME;
            ks->last_status = -4; // PROST_EBADFRAME
            if (st_out) *st_out = -4;
            ks->bad_frames += 1;
            ks->frames_since_rebase += 1;
        }
        return;
    }
    float e = 0.f;
    if (el) {
        const float gv = i <= l ? G[tri<K>(i, l)] : G[tri<K>(l, i)];
        e = gv - (i == l ? 1.f : 0.f); // exact
        rs.W[t] = (double)gv;
        rs.Xh[t] = l > i ? e : (l == i ? 0.5f * e : 0.f);
        rs.Xl[t] = 0.f;
    }
    if (t == 0) rs.emax = 0.f;
    cons_sync<NT>();
    // the bit patterns of non-negative floats order like the floats
    if (el && fabsf(e) > 0.f) atomicMax(reinterpret_cast<int *>(&rs.emax), __float_as_int(fabsf(e)));
    cons_sync<NT>();
    const float emax = rs.emax;
    if (emax <= 1e-5f) {
        for (int sweep = 0; sweep < 2; ++sweep) {
            float pv = 0.f;
            if (el && l >= i)
                for (int r = 0; r <= i; ++r) {
                    pv = fmaf(rs.Xh[r * K + i], rs.Xh[r * K + l], pv);
                    pv = fmaf(rs.Xh[r * K + i], rs.Xl[r * K + l], pv);
                    pv = fmaf(rs.Xl[r * K + i], rs.Xh[r * K + l], pv);
                }
            cons_sync<NT>();
            if (el) rs.Xl[t] = l > i ? -pv : (l == i ? -0.5f * pv : 0.f);
            cons_sync<NT>();
        }
        // X^2 and X^3 (sizes |E|^2 and |E|^3) from the rounded sum Xh + Xl
        float x2 = 0.f;
        if (el && l >= i)
            for (int r = i; r <= l; ++r)
                x2 = fmaf(rs.Xh[i * K + r] + rs.Xl[i * K + r], rs.Xh[r * K + l] + rs.Xl[r * K + l], x2);
        if (el) rs.X2[t] = x2;
        cons_sync<NT>();
        float x3 = 0.f;
        if (el && l >= i)
            for (int r = i; r <= l; ++r) x3 = fmaf(rs.X2[i * K + r], rs.Xh[r * K + l], x3);
        if (el) {
            const double xh = (double)rs.Xh[t], xl = (double)rs.Xl[t];
            const double id = i == l ? 1.0 : 0.0;
            rs.R[t] = (id + xh) + xl;
            rs.T[t] = ((id - xh) - xl) + ((double)x2 - (double)x3);
        }
        if (t == 0) rs.ok = 1;
    } else {
        const bool ok = cholesky_refined<K, NT>(rs);
        if (t == 0) rs.ok = ok ? 1 : 0;
    }
    cons_sync<NT>();
    const bool ok = rs.ok != 0;
    // y' = R (T_old y), FP64
    if (t < K) {
        double ty = 0.0;
        for (int q = t; q < K; ++q) ty = dfma(rs.Told[t * K + q], sk.y[q], ty);
        rs.ty[t] = ty;
    }
    cons_sync<NT>();
    if (t < K) {
        double yn = 0.0;
        for (int q = t; q < K; ++q) yn = dfma(rs.R[t * K + q], rs.ty[q], yn);
        ks->y[t] = yn;
        ks->yf[t] = (float)rs.ty[t];
    }
    if (el) {
        ks->R[i * KMAX + l] = rs.R[t];
        ks->T[i * KMAX + l] = rs.T[t];
        ks->Tf[t] = (float)rs.T[t];
    }
    if (t == 0) {
        ks->orth_err = emax;
        if (!ok) ks->err_flags |= ERR_NOTSPD;
        ks->n_fg = (int64_t)n_fg;
        ks->frame_index = sk.frame_index + 1;
        ks->frames_since_rebase += 1;
        ks->last_status = ok ? 0 : -6; // PROST_ENOTSPD
        if (st_out) *st_out = ok ? 0 : -6;
        ks->skip = 0;
    }
}

// ---- the frame kernel --------------------------------------------------------

struct FrameTiles {
    int nres, r0, nupt, u0;
    __device__ FrameTiles(const DevParams &prm, int G, int b)
    {
        const long long NT = (long long)prm.C * prm.npt;
        r0 = (int)(NT * b / G);
        nres = (int)(NT * (b + 1) / G) - r0;
        u0 = (int)((long long)prm.npt * b / G);
        nupt = (int)((long long)prm.npt * (b + 1) / G) - u0;
    }
};

// One residual pass over this CTA's tiles: per-thread sums of the cost, U^T eta,
// |eta|^2, the non-finite count and (WM) U^T diag(c) U.
template <int K, typename FT, typename UT, bool WM>
__device__ __forceinline__ void residual_pass(const FrameArgs &a, const FrameTiles &tl, const SKState<K> &sk,
                                              float (&acc)[WM ? FCfg<K>::NPR : FCfg<K>::NPF], int t0)
{
    using F = FCfg<K>;
    constexpr int TP = F::TP, RW = F::RW, IPT = F::IPT;
    constexpr int NM = WM ? F::NM : 0;
    const DevParams &prm = a.prm;
    float y[K];
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = sk.yf[j];
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;
    const FT *frame = static_cast<const FT *>(a.frame);
    const int nitems = tl.nres * IPT;
    if ((int)threadIdx.x < t0) return; // threads [0, t0) do other work this pass
    for (int it = threadIdx.x - t0; it < nitems; it += F::THREADS - t0) {
        const int ti = tl.r0 + it / IPT;
        const int rp = it - (it / IPT) * IPT;
        const int c = ti / prm.npt;
        const int64_t p = (int64_t)(ti - c * prm.npt) * TP + rp * RW;
        const int nvalid = prm.P - p < RW ? (int)(prm.P - p) : RW;
        const UT *ub = static_cast<const UT *>(a.U) + (int64_t)ti * K * TP + rp * RW;
        float u[K][RW];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float2 v = ldcg_u2(ub + j * TP);
            u[j][0] = v.x;
            u[j][1] = v.y;
        }
        float xv[RW], lb[RW];
        ld2(frame + (int64_t)c * a.frame_pitch + p, nvalid == RW, nvalid, xv);
        ld2(a.labels + p, true, RW, lb);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const bool valid = r < nvalid;
            float uy = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) uy = fmaf(u[j][r], y[j], uy);
            if constexpr (sizeof(FT) == 4) {
                if (valid && !isfinite(xv[r])) acc[K + NM + 2] += 1.f;
            }
            const float res = valid ? fmaf(xv[r], sc, -of) - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float tz = __powf(z, e);
            const float wv = valid ? (lb[r] != 0.f ? om : 1.f) : 0.f;
            const float cw = wv * tz;
            acc[K + NM] = fmaf(cw, z, acc[K + NM]);
            const float eta = -pw * cw * res;
            acc[K + NM + 1] = fmaf(eta, eta, acc[K + NM + 1]);
#pragma unroll
            for (int j = 0; j < K; ++j) acc[j] = fmaf(eta, u[j][r], acc[j]);
            if constexpr (WM) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const float cu = cw * u[j][r];
#pragma unroll
                    for (int l2 = j; l2 < K; ++l2) acc[K + tri<K>(j, l2)] = fmaf(cu, u[l2][r], acc[K + tri<K>(j, l2)]);
                }
            }
        }
    }
}

// The explicit projection pass over this CTA's tiles (register form): the
// per-thread sum of pi(eta)_e^2 = (eta_e - u_e^T g)^2 at the final y
// (Eq. gproject), with u_e^T g = u_st,e^T (T g).
template <int K, typename FT, typename UT>
__device__ __forceinline__ void proj_pass(const FrameArgs &a, const FrameTiles &tl, const SKState<K> &sk,
                                          float &acc)
{
    using F = FCfg<K, UT>;
    constexpr int TP = F::TP, RW = F::RW, IPT = F::IPT;
    const DevParams &prm = a.prm;
    float y[K], tg[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        y[j] = sk.yf[j];
        tg[j] = sk.tg[j];
    }
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;
    const FT *frame = static_cast<const FT *>(a.frame);
    const int nitems = tl.nres * IPT;
    for (int it = threadIdx.x; it < nitems; it += F::THREADS) {
        const int ti = tl.r0 + it / IPT;
        const int rp = it - (it / IPT) * IPT;
        const int c = ti / prm.npt;
        const int64_t p = (int64_t)(ti - c * prm.npt) * TP + rp * RW;
        const int nvalid = prm.P - p < RW ? (int)(prm.P - p) : RW;
        const UT *ub = static_cast<const UT *>(a.U) + (int64_t)ti * K * TP + rp * RW;
        float u[K][RW];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float2 v = ldcg_u2(ub + j * TP);
            u[j][0] = v.x;
            u[j][1] = v.y;
        }
        float xv[RW], lb[RW];
        ld2(frame + (int64_t)c * a.frame_pitch + p, nvalid == RW, nvalid, xv);
        ld2(a.labels + p, true, RW, lb);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const bool valid = r < nvalid;
            float uy = 0.f, ug = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                uy = fmaf(u[j][r], y[j], uy);
                ug = fmaf(u[j][r], tg[j], ug);
            }
            const float res = valid ? fmaf(xv[r], sc, -of) - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float wv = valid ? (lb[r] != 0.f ? om : 1.f) : 0.f;
            const float eta = -pw * (wv * __powf(z, e)) * res;
            const float pe = valid ? eta - ug : 0.f;
            acc = fmaf(pe, pe, acc);
        }
    }
}

// ---- the resident form (k <= 10) ------------------------------------------------
// CTA b owns the pixels [pa, pa + 2 npair) of every channel plane, the planes
// cut into units of RES_UNIT pixels dealt evenly over the grid; an item is two
// consecutive pixels of one channel, items channel-major (item c npair + q).
// The first residual pass of a frame reads every item's rows, frame entries
// and labels from global memory and keeps them in shared memory: the frame
// entries and labels of every item, and the rows of items [ng, nitems) in ns
// slots (all of them when they fit).  The later passes of the frame read them
// from there and stream only the rows of items [0, ng) from L2 again; those are
// every thread's first items, so their load latency overlaps the other warps'
// shared-memory items.  The update pass reads the old rows the same way and
// writes the new ones to global memory.
struct ResPart {
    int64_t pa; // first pixel
    int npair;  // pixel pairs per channel (the last may hold one pixel)
    int nitems; // C npair
    int ng;     // items whose rows stream from global memory in every pass
    __device__ ResPart(const DevParams &prm, int G, int b, int ns)
    {
        const int64_t nu = res_units(prm.P);
        const int64_t lo = nu * b / G, hi = nu * (b + 1) / G;
        pa = lo * RES_UNIT;
        const int64_t pb = hi * RES_UNIT < prm.P ? hi * RES_UNIT : prm.P;
        const int npx = pb > pa ? (int)(pb - pa) : 0;
        npair = (npx + 1) / 2;
        nitems = prm.C * npair;
        ng = nitems > ns ? nitems - ns : 0;
    }
};

// a pair of consecutive stored entries: 8 bytes of float32, 4 of bfloat16
template <typename UT> struct RPair;
template <> struct RPair<float> {
    using T = float2;
    static __device__ __forceinline__ T ldg(const float *p) { return __ldcg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ float2 wide(T v) { return v; }
    static __device__ __forceinline__ T pack(float a, float b) { return make_float2(a, b); }
};
template <> struct RPair<bf16> {
    using T = uint32_t;
    static __device__ __forceinline__ T ldg(const bf16 *p) { return __ldcg(reinterpret_cast<const unsigned int *>(p)); }
    static __device__ __forceinline__ float2 wide(T w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    // a and b already hold bfloat16 values (stochastically rounded): exact
    static __device__ __forceinline__ T pack(float a, float b)
    {
        return (__float_as_uint(a) >> 16) | (__float_as_uint(b) & 0xffff0000u);
    }
};
// a pair of consecutive frame entries, as stored (the plane and its pitch are
// 16-byte aligned and p is even)
template <typename FT> struct XPair;
template <> struct XPair<uint8_t> {
    using T = uchar2;
    static __device__ __forceinline__ T ldg(const uint8_t *p, int nvalid)
    {
        if (nvalid == 2) return __ldg(reinterpret_cast<const uchar2 *>(p));
        return make_uchar2(nvalid > 0 ? __ldg(p) : (uint8_t)0, (uint8_t)0);
    }
    static __device__ __forceinline__ float2 wide(T v) { return make_float2((float)v.x, (float)v.y); }
};
template <> struct XPair<float> {
    using T = float2;
    static __device__ __forceinline__ T ldg(const float *p, int nvalid)
    {
        if (nvalid == 2) return __ldg(reinterpret_cast<const float2 *>(p));
        return make_float2(nvalid > 0 ? __ldg(p) : 0.f, 0.f);
    }
    static __device__ __forceinline__ float2 wide(T v) { return v; }
};

// bytes of dynamic shared memory: ns row slots, the frame entries and labels
// of npm pixel pairs per channel
template <int K, typename FT, typename UT>
__host__ __device__ inline size_t res_smem_bytes(int C, int npm, int ns)
{
    return res_al16((size_t)K * ns * sizeof(typename RPair<UT>::T)) +
           res_al16((size_t)C * npm * sizeof(typename XPair<FT>::T)) + res_al16((size_t)npm * sizeof(uchar2));
}

template <int K, typename FT, typename UT> struct ResSmem {
    typename RPair<UT>::T *us; // rows: column j of slot s at us[j ns + s]
    typename XPair<FT>::T *xs; // frame entries of item i at xs[i]
    uchar2 *ls;                // labels of pixel pair q at ls[q]
    int ns;
    __device__ ResSmem(unsigned char *base, const DevParams &prm, int G, int ns_) : ns(ns_)
    {
        const int npm = res_npair_max(prm.P, G);
        us = reinterpret_cast<typename RPair<UT>::T *>(base);
        unsigned char *x = base + res_al16((size_t)K * ns * sizeof(typename RPair<UT>::T));
        xs = reinterpret_cast<typename XPair<FT>::T *>(x);
        ls = reinterpret_cast<uchar2 *>(x + res_al16((size_t)prm.C * npm * sizeof(typename XPair<FT>::T)));
    }
};

// One pass of the resident form over this CTA's items.
//   MODE 0: a CG pass (cost, U^T eta, |eta|^2, non-finite count, U^T diag(c) U)
//   MODE 1: the final pass (the same without the matrix)
//   MODE 2: the explicit projection pass, sum of pi(eta)_e^2 = (eta_e - u_e^T g)^2
// FILL: 0 in the later passes of a frame; 1 in the first pass of a launch,
// which reads the rows, frame entries and labels from global memory and fills
// the shared-memory copies; 2 in the first pass of a later frame of the same
// launch, whose rows and labels the previous frame's update pass left in
// shared memory: only the frame entries are read and kept.
template <int K, typename FT, typename UT, int MODE, int FILL, int NA>
__device__ __forceinline__ void res_pass(const FrameArgs &a, const FT *frame, const ResPart &rp,
                                         const ResSmem<K, FT, UT> &sm, const SKState<K> &sk, float (&acc)[NA])
{
    using F = FCfg<K, UT>;
    using RP = RPair<UT>;
    using XP = XPair<FT>;
    constexpr int TP = F::TP, NT = F::THREADS;
    constexpr int NM = MODE == 0 ? F::NM : 0;
    static_assert(!(FILL && MODE == 2), "the projection pass is never a frame's first");
    static_assert(FILL >= 0 && FILL <= 2, "fill mode");
    const DevParams &prm = a.prm;
    float y[K], tg[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        y[j] = sk.yf[j];
        tg[j] = MODE == 2 ? sk.tg[j] : 0.f;
    }
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;
    const UT *U = static_cast<const UT *>(a.U);
    const int np = rp.npair;
    int c = 0, q = threadIdx.x;
    while (q >= np && c < prm.C) {
        q -= np;
        ++c;
    }
    for (int it = threadIdx.x; it < rp.nitems; it += NT) {
        const int64_t p = rp.pa + 2 * (int64_t)q;
        const int nvalid = prm.P - p < 2 ? (int)(prm.P - p) : 2;
        float u[K][2];
        if (FILL == 1 || it < rp.ng) {
            const int64_t pt = p / TP;
            const UT *ub = U + (((int64_t)c * prm.npt + pt) * K) * TP + (p - pt * TP);
            typename RP::T v[K];
#pragma unroll
            for (int j = 0; j < K; ++j) v[j] = RP::ldg(ub + j * TP);
            if (FILL == 1 && it >= rp.ng) {
#pragma unroll
                for (int j = 0; j < K; ++j) sm.us[j * sm.ns + (it - rp.ng)] = v[j];
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float2 w = RP::wide(v[j]);
                u[j][0] = w.x;
                u[j][1] = w.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float2 w = RP::wide(sm.us[j * sm.ns + (it - rp.ng)]);
                u[j][0] = w.x;
                u[j][1] = w.y;
            }
        }
        typename XP::T xr;
        uchar2 lr;
        if (FILL != 0) {
            xr = XP::ldg(frame + (int64_t)c * a.frame_pitch + p, nvalid);
            sm.xs[it] = xr;
        } else {
            xr = sm.xs[it];
        }
        if (FILL == 1) {
            lr = __ldg(reinterpret_cast<const uchar2 *>(a.labels + p));
            if (c == 0) sm.ls[q] = lr;
        } else {
            lr = sm.ls[q];
        }
        const float2 xw = XP::wide(xr);
        const float xv[2] = {xw.x, xw.y};
        const float lb[2] = {(float)lr.x, (float)lr.y};
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const bool valid = r < nvalid;
            float uy = 0.f, ug = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                uy = fmaf(u[j][r], y[j], uy);
                if (MODE == 2) ug = fmaf(u[j][r], tg[j], ug);
            }
            if constexpr (MODE != 2 && sizeof(FT) == 4) {
                if (valid && !isfinite(xv[r])) acc[K + NM + 2] += 1.f;
            }
            const float res = valid ? fmaf(xv[r], sc, -of) - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float tz = __powf(z, e);
            const float wv = valid ? (lb[r] != 0.f ? om : 1.f) : 0.f;
            const float cw = wv * tz;
            const float eta = -pw * cw * res;
            if constexpr (MODE == 2) {
                const float pe = valid ? eta - ug : 0.f;
                acc[0] = fmaf(pe, pe, acc[0]);
            } else {
                acc[K + NM] = fmaf(cw, z, acc[K + NM]);
                acc[K + NM + 1] = fmaf(eta, eta, acc[K + NM + 1]);
#pragma unroll
                for (int j = 0; j < K; ++j) acc[j] = fmaf(eta, u[j][r], acc[j]);
                if constexpr (MODE == 0) {
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const float cu = cw * u[j][r];
#pragma unroll
                        for (int l2 = j; l2 < K; ++l2)
                            acc[K + tri<K>(j, l2)] = fmaf(cu, u[l2][r], acc[K + tri<K>(j, l2)]);
                    }
                }
            }
        }
        q += NT;
        while (q >= np && c < prm.C) {
            q -= np;
            ++c;
        }
    }
}

// The next frame's entries of this CTA's pixels, fetched into L2 ahead of the
// next frame's first pass (a later frame of a resident-form launch reads them
// from global memory there): one 128-byte line per thread, only addresses
// inside the CTA's range of each plane.
template <typename FT>
__device__ __forceinline__ void res_prefetch_frame(const FT *next, int64_t pitch, const ResPart &rp, const DevParams &prm)
{
    const int64_t np = prm.P - rp.pa < 2 * (int64_t)rp.npair ? prm.P - rp.pa : 2 * (int64_t)rp.npair;
    if (np <= 0) return;
    const int64_t bytes = np * (int64_t)sizeof(FT);
    const int nl = (int)((bytes + 127) / 128);
    for (int i = threadIdx.x; i < prm.C * nl; i += blockDim.x) {
        const int c = i / nl, l = i - c * nl;
        const char *ad = reinterpret_cast<const char *>(next + (int64_t)c * pitch + rp.pa) + (int64_t)l * 128;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ad));
    }
}

// The update pass of the resident form: a thread takes a pixel pair and its
// channels in turn (the label of Step 3 is the maximum over the channels),
// the old rows from shared memory (or L2 for items [0, ng)), and writes the
// new rows, the labels and the optional outputs to global memory; per-thread
// sums of the Gram of the written rows and of the foreground count.  keep: a
// later frame of the launch follows, so the new rows and labels also replace
// the shared-memory copies it starts from.
template <int K, typename FT, typename UT>
__device__ __forceinline__ void res_update(const FrameArgs &a, uint8_t *mask_out, float *bg_out, bool keep,
                                           const ResPart &rp, const ResSmem<K, FT, UT> &sm, const SKState<K> &sk,
                                           float (&acc)[FCfg<K, UT>::NPU])
{
    using F = FCfg<K, UT>;
    using RP = RPair<UT>;
    using XP = XPair<FT>;
    constexpr int TP = F::TP, NT = F::THREADS, NM = F::NM;
    const DevParams &prm = a.prm;
    const float cm1 = sk.cm1, snp = sk.snp, yn = sk.yn;
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta;
    const float sc = prm.in_scale, of = prm.in_offset;
    const bool pre = prm.mask_pre != 0;
    const bool write = !sk.skip;
    // the k-space vectors, read from shared memory (broadcast loads); they do
    // not change during the pass, so the compiler may keep them in registers
    const float *vy = sk.yf;
    const float *vv = sk.tv;
    const float *vg = sk.tg;
    const float *vw = sk.w;
    UT *U = static_cast<UT *>(a.U);
    const int C = prm.C, np = rp.npair;
    const uint32_t sr_key = pcg_hash(prm.sr_seed ^ pcg_hash((uint32_t)sk.frame_index));
    for (int q = threadIdx.x; q < np; q += NT) {
        const int64_t p = rp.pa + 2 * (int64_t)q;
        const int nvalid = prm.P - p < 2 ? (int)(prm.P - p) : 2;
        const int64_t pt = p / TP;
        const int r0 = (int)(p - pt * TP);
        const uchar2 lr = sm.ls[q];
        const float wv[2] = {nvalid > 0 ? (lr.x ? om : 1.f) : 0.f, nvalid > 1 ? (lr.y ? om : 1.f) : 0.f};
        float mx[2] = {0.f, 0.f};
        for (int c = 0; c < C; ++c) {
            const int it = c * np + q;
            UT *ub = U + (((int64_t)c * prm.npt + pt) * K) * TP + r0;
            float u[K][2];
            if (it < rp.ng) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const float2 w = RP::wide(RP::ldg(ub + j * TP));
                    u[j][0] = w.x;
                    u[j][1] = w.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const float2 w = RP::wide(sm.us[j * sm.ns + (it - rp.ng)]);
                    u[j][0] = w.x;
                    u[j][1] = w.y;
                }
            }
            const float2 xw = XP::wide(sm.xs[it]);
            const float xv[2] = {xw.x, xw.y};
            // dots of the orthonormal rows u = T^T u_st through T y, T g, T v
            float uy[2] = {0.f, 0.f}, ug[2] = {0.f, 0.f}, uv[2] = {0.f, 0.f};
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float by = vy[j], bg = vg[j], bv = vv[j];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    uy[r] = fmaf(u[j][r], by, uy[r]);
                    ug[r] = fmaf(u[j][r], bg, ug[r]);
                    uv[r] = fmaf(u[j][r], bv, uv[r]);
                }
            }
            float gam[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const bool valid = r < nvalid;
                const float x = fmaf(xv[r], sc, -of);
                const float res = valid ? x - uy[r] : 0.f;
                const float z = fmaf(res, res, mu);
                const float tz = __powf(z, e);
                const float eta = -pw * wv[r] * tz * res;
                // u <- u + ((cos(theta) - 1) u^T v - sin(theta) pi(eta)_e / |pi(eta)|) v
                gam[r] = valid ? fmaf(cm1, uv[r], -snp * (eta - ug[r])) : 0.f;
                const float rn = pre ? res : fmaf(-gam[r], yn, res);
                if (valid) {
                    mx[r] = fmaxf(mx[r], fabsf(rn));
                    if (write && bg_out) bg_out[(int64_t)c * prm.P + p + r] = x - rn + of;
                }
            }
            // stored rows of u + gamma v: u_st + gamma R^T v; a bfloat16 row
            // is rounded stochastically (one hash per stored row, then the
            // linear congruential step per entry) and its Gram taken of the
            // stored values
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float bw = vw[j];
#pragma unroll
                for (int r = 0; r < 2; ++r) u[j][r] = fmaf(gam[r], bw, u[j][r]);
            }
            if constexpr (sizeof(UT) == 2) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    uint32_t rk = pcg_hash(sr_key ^ (uint32_t)(c * prm.Pp + p + r));
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        rk = rk * 1664525u + 1013904223u;
                        u[j][r] = round_bf16_sr(u[j][r], rk >> 16);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int j = 0; j < K; ++j)
#pragma unroll
                    for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(u[j][r], u[l2][r], acc[tri<K>(j, l2)]);
            if (write) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const typename RP::T v = RP::pack(u[j][0], u[j][1]);
                    *reinterpret_cast<typename RP::T *>(ub + j * TP) = v;
                    if (keep && it >= rp.ng) sm.us[j * sm.ns + (it - rp.ng)] = v;
                }
            }
        }
        const uint8_t nl0 = (nvalid > 0 && mx[0] >= dl) ? 1 : 0;
        const uint8_t nl1 = (nvalid > 1 && mx[1] >= dl) ? 1 : 0;
        acc[NM] += (float)(nl0 + nl1);
        if (write) {
            *reinterpret_cast<uchar2 *>(a.labels + p) = make_uchar2(nl0, nl1);
            if (keep) sm.ls[q] = make_uchar2(nl0, nl1);
            if (mask_out) {
                if (nvalid > 0) mask_out[p] = nl0;
                if (nvalid > 1) mask_out[p + 1] = nl1;
            }
        }
    }
}

// The k-space state a later frame of a resident-form launch takes from the
// global state after its first grid barrier: the factors, y and the frame
// counter the last CTA of the previous frame wrote (L2 loads: the values this
// CTA read before may still sit in its L1).  The CTA barriers of the
// reduction that follows order these stores before the k-space step.
template <int K>
__device__ __forceinline__ void reload_state(SKState<K> &sk, ReorthScratch<K> &rs, const KState *ks)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < K * K; i += blockDim.x) {
        sk.Tf[i] = __ldcg(&ks->Tf[i]);
        sk.Rf[i] = (float)__ldcg(&ks->R[(i / K) * KMAX + (i % K)]);
        rs.Told[i] = __ldcg(&ks->T[(i / K) * KMAX + (i % K)]);
    }
    if (tid < K) sk.y[tid] = __ldcg(&ks->y[tid]);
    if (tid == 0) sk.frame_index = __ldcg(&ks->frame_index);
}

// The frame of one stream, by CTA b of the G CTAs working on it.
// CL: the cluster form (the whole grid is one thread-block cluster, its
// barriers are the hardware cluster barrier, CTA 0 ends the frame); else the
// grid form (cooperative launch, bounded grid barriers, the last CTA to
// arrive ends the frame).  RES: the resident form of the grid form (k <= 10),
// rows, frame entries and labels kept in shared memory across the passes.
template <int K, typename FT, typename UT, bool CL = false, bool RES = false>
__device__ __forceinline__ void frame_body(const FrameArgs &a, const int G, const int b)
{
    using F = FCfg<K, UT>;
    constexpr int TP = F::TP, RW = F::RW, IPT = F::IPT, NT = F::THREADS, NW = F::NW;
    constexpr int NM = F::NM;
    constexpr int NREP = RES ? RES_NREP : 1; // copies of the partial values (see the pass loop)
    __shared__ float sred[NW * F::NPMAX];
    __shared__ float tot[F::NVR > F::NVU ? F::NVR : F::NVU];
    __shared__ float rscr[RED_SCR];
    __shared__ SKState<K> sk;
    extern __shared__ __align__(128) float stage_smem[]; // streaming and resident forms only
    static_assert(!(RES && (F::STREAM || CL)), "the resident form is a grid form of the register form");
    static_assert(!RES || (F::NVR <= RES_VPW * NW && F::NVU <= RES_VPW * NW), "values per warp of the sums");
    // the register form's grid launches (k <= KREG: one stream, or a batch's
    // streams) share the resident form's warp sums and release arrivals
    constexpr bool WSUM = RES || (!F::STREAM && !CL);
    auto reduce_warp_sums = [](const float *c, int nr, int st, int nv, float *t) {
        if constexpr (RES)
            reduce_cols_warp<NT, RES_VPW, RES_CPL>(c, nr, st, nv, t);
        else
            reduce_cols_warp_call<NT, RES_VPW, RES_CPL>(c, nr, st, nv, t);
    };
    static_assert(!WSUM || (F::NVR <= RES_VPW * NW && F::NVU <= RES_VPW * NW), "values per warp of the sums");
    __shared__ ReorthScratch<K> rs;

    const int tid = threadIdx.x, warp = tid >> 5;
    const DevParams &prm = a.prm;
    const FrameTiles tl(prm, G, b);

    if (tid == 0) {
        // grid form: the barrier count must be where this launch expects it
        // (a launch that gave up part-way leaves it elsewhere); the cluster
        // form has no software barrier to check
        if constexpr (CL) {
            sk.err = 0;
        } else {
            const unsigned long long c0 = ld_acquire_u64(&a.bar->count);
            sk.err = (c0 < a.bar_base || c0 >= a.bar_base + (unsigned long long)G) ? 1 : 0;
        }
        sk.skip = 0;
        sk.last = 0;
        sk.proj = 0;
        sk.ypend = 0;
        sk.frame_index = a.ks->frame_index;
    }
    for (int i = tid; i < K * K; i += NT) {
        sk.Tf[i] = a.ks->Tf[i];
        sk.Rf[i] = (float)a.ks->R[(i / K) * KMAX + (i % K)];
        rs.Told[i] = a.ks->T[(i / K) * KMAX + (i % K)];
    }
    if (tid < K) {
        sk.y[tid] = a.ks->y[tid];
        sk.yf[tid] = a.ks->yf[tid];
    }
    __syncthreads();
    if (sk.err) {
        if (tid == 0 && b == 0) {
            atomicOr(&a.ks->err_flags, ERR_TIMEOUT);
            a.ks->last_status = -5; // PROST_ETIMEOUT: the frame was refused
            if (a.status_out) *a.status_out = -5;
        }
        return;
    }

    // CTA 0 stamps the trace; the statistics of the k-space steps (FP64
    // conversions and stores) come from CTA 0, or in the resident form from
    // the end CTA, which streams no rows and so waits at every barrier anyway
    const bool stats = b == 0;
    const bool kstats = RES ? b == G - 1 : stats;
    using SC = StageCfg<K, FT, UT>;
    unsigned char *const sbase = reinterpret_cast<unsigned char *>(stage_smem);
    unsigned char *wstage = sbase + (size_t)warp * SC::WARP_B;
    constexpr int RES_OFF = SC::D * SC::STAGE_B + SC::RES_B; // a warp's tensor-core result
    // resident form: CTAs [0, G - 1) own the pixels, CTA G - 1 (the end CTA)
    // owns none and ends every frame (see the end of the frame)
    const ResPart rpart(prm, G - 1, b, a.res_ns);
    const ResSmem<K, FT, UT> rsm(sbase, prm, G - 1, a.res_ns);
    // the partial buffers alternate over every pass of the launch, so the
    // first pass of a frame never writes the buffer from which the last CTA
    // of the frame before is still reading the update pass's sums
    int buf = 0;
    // frames of this launch: one, or in the resident form nframes of the same
    // stream in turn, each frame a_frame_stride entries after the one before
    const int nfr = RES ? (a.nframes > 1 ? a.nframes : 1) : 1;
    for (int fr = 0; fr < nfr; ++fr) {
    const FT *fptr = static_cast<const FT *>(a.frame) + (int64_t)fr * a.frame_stride;
    uint8_t *mask_out = a.mask_out ? a.mask_out + (int64_t)fr * prm.P : nullptr;
    unsigned long long target =
        a.bar_base + (unsigned long long)fr * (unsigned long long)G * (unsigned long long)frame_arrivals(prm.n_cg);
    const int stall_at = fr == 0 ? a.stall_at : 0;
    if (stats && tid == 0) a.ks->phase_ts[0] = global_ns();

    for (int pass = 0; pass <= prm.n_cg; ++pass) {
        const int cs = a.col_stride;
        float *const bbase = a.partials + (size_t)buf * NREP * F::NVR * cs;
        // the resident form writes NREP copies of each CTA's partial values and
        // CTA b sums copy b % NREP, so that each L2 line of the partials serves
        // G / NREP readers rather than all G at once
        const float *cols = bbase + (size_t)(b % NREP) * F::NVR * cs;
        float *col = bbase + b;
        const size_t rstr = (size_t)F::NVR * cs;
        target += (unsigned long long)G;
        if constexpr (RES) {
            // the previous CG step's FP64 update of y, by the last warp
            if (warp == NW - 1 && sk.ypend) {
                const int l = tid & 31;
                if (l < K) sk.y[l] = fma((double)sk.apend, (double)sk.d[l], sk.y[l]);
                __syncwarp();
                if (l == 0) sk.ypend = 0;
            }
        }
        if (pass < prm.n_cg) {
            const bool trace = stats && tid == 0 && pass == 1;
            float acc[F::NPR];
#pragma unroll
            for (int i = 0; i < F::NPR; ++i) acc[i] = 0.f;
            if constexpr (RES) {
                if (pass == 0 && fr == 0)
                    res_pass<K, FT, UT, 0, 1>(a, fptr, rpart, rsm, sk, acc);
                else if (pass == 0)
                    res_pass<K, FT, UT, 0, 2>(a, fptr, rpart, rsm, sk, acc);
                else
                    res_pass<K, FT, UT, 0, 0>(a, fptr, rpart, rsm, sk, acc);
            } else if constexpr (F::STREAM)
                stream_residual<K, FT, UT, true, NW>(a, tl.r0, tl.nres, sk.yf, wstage, acc);
            else
                residual_pass<K, FT, UT, true>(a, tl, sk, acc, 0);
            if (trace) a.ks->sub_ts[0] = global_ns();
            if constexpr (F::STREAM && SC::TC) {
                cons_partials_tree<F::NVR, NW, F::NPR, K, K + NM>(acc, F::NVR, col, sred, cs);
                mma_row<K, NW>(sbase, SC::WARP_B, RES_OFF, col + (size_t)K * cs, cs);
            } else if constexpr (F::STREAM) {
                cons_partials_tree<F::NVR, NW>(acc, F::NVR, col, sred, cs);
            } else {
                cons_partials<F::NPR, NW>(acc, F::NVR, col, sred, cs, NREP, rstr);
            }
            if (trace) a.ks->sub_ts[1] = global_ns();
            if (!pass_sync<CL, NT, WSUM>(a.bar, target + (pass + 1 == stall_at ? 1ull : 0ull), &sk.err, a.ks,
                                   a.status_out, pass + 1 == stall_at ? a.stall_limit : WAIT_LIMIT))
                return;
            if (trace) a.ks->sub_ts[2] = global_ns();
            if (RES && fr > 0 && pass == 0) reload_state(sk, rs, a.ks);
            if constexpr (WSUM)
                reduce_warp_sums(cols, G, cs, F::NVR, tot);
            else
                reduce_cols<NT>(cols, G, cs, F::NVR, tot, rscr);
            if (trace) a.ks->sub_ts[3] = global_ns();
            if (warp == 0) kspace_cg<K, true, RES>(sk, prm, tot, pass, a.ks, kstats);
            if (trace) a.ks->sub_ts[4] = global_ns();
        } else {
            float acc[F::NPF];
#pragma unroll
            for (int i = 0; i < F::NPF; ++i) acc[i] = 0.f;
            if constexpr (RES) {
                if (pass == 0 && fr == 0)
                    res_pass<K, FT, UT, 1, 1>(a, fptr, rpart, rsm, sk, acc);
                else if (pass == 0)
                    res_pass<K, FT, UT, 1, 2>(a, fptr, rpart, rsm, sk, acc);
                else
                    res_pass<K, FT, UT, 1, 0>(a, fptr, rpart, rsm, sk, acc);
            } else if constexpr (F::STREAM)
                stream_residual<K, FT, UT, false, NW>(a, tl.r0, tl.nres, sk.yf, wstage, acc);
            else
                residual_pass<K, FT, UT, false>(a, tl, sk, acc, 0);
            if constexpr (F::STREAM)
                cons_partials_tree<F::NVF, NW>(acc, F::NVF, col, sred, cs);
            else
                cons_partials<F::NPF, NW>(acc, F::NVF, col, sred, cs, NREP, rstr);
            if (!pass_sync<CL, NT, WSUM>(a.bar, target + (pass + 1 == stall_at ? 1ull : 0ull), &sk.err, a.ks,
                                   a.status_out, pass + 1 == stall_at ? a.stall_limit : WAIT_LIMIT))
                return;
            if (RES && fr > 0 && pass == 0) reload_state(sk, rs, a.ks);
            if constexpr (WSUM)
                reduce_warp_sums(cols, G, cs, F::NVF, tot);
            else
                reduce_cols<NT>(cols, G, cs, F::NVF, tot, rscr);
            if (warp == 0) kspace_cg<K, false>(sk, prm, tot, pass, a.ks, kstats);
        }
        cons_sync<NT>();
        if (stats && tid == 0) a.ks->phase_ts[pass + 1] = global_ns();
        buf ^= 1;
    }

    // ---- |pi(eta)| by the explicit projection pass, where the norm identity
    // of the final pass cancels (the same decision in every CTA) ----
    if (sk.proj) {
        float *const pbase = a.partials + (size_t)buf * NREP * F::NVR * a.col_stride;
        const float *pcols = pbase + (size_t)(b % NREP) * F::NVR * a.col_stride;
        target += (unsigned long long)G;
        float acc1[1] = {0.f};
        if constexpr (RES)
            res_pass<K, FT, UT, 2, 0>(a, fptr, rpart, rsm, sk, acc1);
        else if constexpr (F::STREAM)
            stream_residual<K, FT, UT, false, NW, 1, true>(a, tl.r0, tl.nres, sk.yf, wstage, acc1, sk.tg);
        else
            proj_pass<K, FT, UT>(a, tl, sk, acc1[0]);
        cons_partials_tree<1, NW, 1>(acc1, 1, pbase + b, sred, a.col_stride, NREP, (size_t)F::NVR * a.col_stride);
        if (!pass_sync<CL, NT, WSUM>(a.bar, target, &sk.err, a.ks, a.status_out)) return;
        if constexpr (WSUM)
            reduce_warp_sums(pcols, G, a.col_stride, 1, tot);
        else
            reduce_cols<NT>(pcols, G, a.col_stride, 1, tot, rscr);
        if (tid == 0) step_angle(sk, prm, sqrtf(fmaxf(tot[0], 0.f)), a.ks, kstats);
        cons_sync<NT>();
        buf ^= 1;
    }

    // ---- update pass: Step 2 on every row, Step 3 labels, Gram of the new rows ----
    const float *ucols = a.partials + (size_t)buf * NREP * F::NVR * a.col_stride; // one copy: the last CTA reads it
    float *ucol = const_cast<float *>(ucols) + b;
    if constexpr (F::STREAM) {
        float acc[F::NPU];
#pragma unroll
        for (int i = 0; i < F::NPU; ++i) acc[i] = 0.f;
        UpdVecs<K> kv;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            kv.ty[j] = sk.yf[j];
            kv.tg[j] = sk.tg[j];
            kv.tv[j] = sk.tv[j];
            kv.w[j] = sk.w[j];
        }
        const uint32_t sr_key = pcg_hash(prm.sr_seed ^ pcg_hash((uint32_t)sk.frame_index));
        stream_update<K, FT, UT, NW>(a, tl.u0, tl.nupt, kv, sk.cm1, sk.snp, sk.yn, !sk.skip, sr_key, wstage, acc);
        if (tid == 0 && stats) a.ks->sub_ts[5] = global_ns();
        if constexpr (SC::TC) {
            cons_partials_tree<F::NVU, NW, F::NPU, 0, NM>(acc, F::NVU, ucol, sred, a.col_stride);
            mma_row<K, NW>(sbase, SC::WARP_B, RES_OFF, ucol, a.col_stride);
        } else {
            cons_partials_tree<F::NVU, NW>(acc, F::NVU, ucol, sred, a.col_stride);
        }
    } else if constexpr (RES) {
        float acc[F::NPU];
#pragma unroll
        for (int i = 0; i < F::NPU; ++i) acc[i] = 0.f;
        if (fr + 1 < nfr) res_prefetch_frame<FT>(fptr + a.frame_stride, a.frame_pitch, rpart, prm);
        res_update<K, FT, UT>(a, mask_out, nfr == 1 ? a.bg_out : nullptr, fr + 1 < nfr, rpart, rsm, sk, acc);
        if (tid == 0 && stats) a.ks->sub_ts[5] = global_ns();
        cons_partials<F::NPU, NW>(acc, F::NVU, ucol, sred, a.col_stride);
    } else {
    float acc[F::NPU];
#pragma unroll
    for (int i = 0; i < F::NPU; ++i) acc[i] = 0.f;
    {
        const float cm1 = sk.cm1, snp = sk.snp, yn = sk.yn;
        const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta;
        const float sc = prm.in_scale, of = prm.in_offset;
        const bool pre = prm.mask_pre != 0;
        const bool write = !sk.skip;
        // read the k-space vectors from shared memory at each use (broadcast
        // loads) rather than holding 4k of them in registers
        const volatile float *vy = sk.yf;
        const volatile float *vv = sk.tv;
        const volatile float *vg = sk.tg;
        const volatile float *vw = sk.w;
        const FT *frame = static_cast<const FT *>(a.frame);
        const UT *Ub = static_cast<const UT *>(a.U);
        const int C = prm.C, npt = prm.npt;
        const uint32_t sr_key = pcg_hash(prm.sr_seed ^ pcg_hash((uint32_t)sk.frame_index));
        // one step = one channel of one pixel, the channels of a pixel in
        // turn (the label of Step 3 is the maximum over them, written after
        // the last); the next step's row, frame entry and label are loaded
        // while this step computes
        const int nitems = tl.nupt * TP;
        int it = tid, c = 0;
        float un[K], xn = 0.f;
        uint8_t ln = 0;
        auto fetch = [&](int it2, int c2) {
            const int pt = tl.u0 + it2 / TP, r0 = it2 - (it2 / TP) * TP;
            const int64_t p = (int64_t)pt * TP + r0;
            const UT *ub = Ub + ((int64_t)c2 * npt + pt) * K * TP + r0;
#pragma unroll
            for (int j = 0; j < K; ++j) un[j] = ldcg_u(ub + j * TP);
            xn = p < prm.P ? (float)__ldg(frame + (int64_t)c2 * a.frame_pitch + p) : 0.f;
            if (c2 == 0) ln = a.labels[p];
        };
        if (it < nitems) fetch(it, 0);
        float wv = 0.f, mx = 0.f;
        while (it < nitems) {
            float u[K];
#pragma unroll
            for (int j = 0; j < K; ++j) u[j] = un[j];
            const float xv = xn;
            const int pt = tl.u0 + it / TP, r0 = it - (it / TP) * TP;
            const int64_t p = (int64_t)pt * TP + r0;
            const bool valid = p < prm.P;
            if (c == 0) {
                wv = valid ? (ln ? om : 1.f) : 0.f;
                mx = 0.f;
            }
            int itn = it, cn = c + 1;
            if (cn == C) {
                cn = 0;
                itn += NT;
            }
            if (itn < nitems) fetch(itn, cn);
            // dots of the orthonormal row u = T^T u_st through T y, T g, T v
            float uy = 0.f, ug = 0.f, uv = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                uy = fmaf(u[j], vy[j], uy);
                ug = fmaf(u[j], vg[j], ug);
                uv = fmaf(u[j], vv[j], uv);
            }
            const float x = fmaf(xv, sc, -of);
            const float res = valid ? x - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float tz = __powf(z, e);
            const float eta = -pw * wv * tz * res;
            // u <- u + ((cos(theta) - 1) u^T v - sin(theta) pi(eta)_e / |pi(eta)|) v
            const float gam = valid ? fmaf(cm1, uv, -snp * (eta - ug)) : 0.f;
            const float rn = pre ? res : fmaf(-gam, yn, res);
            if (valid) {
                mx = fmaxf(mx, fabsf(rn));
                if (write && a.bg_out) a.bg_out[(int64_t)c * prm.P + p] = x - rn + of;
            }
            // stored row of u + gamma v: u_st + gamma R^T v, its Gram, written
            // back; a bfloat16 row is rounded stochastically first, with the
            // streaming form's generator (one hash per stored row, then the
            // linear congruential step per entry), and its Gram taken of the
            // stored values
#pragma unroll
            for (int j = 0; j < K; ++j) u[j] = fmaf(gam, vw[j], u[j]);
            if constexpr (sizeof(UT) == 2) {
                uint32_t rk = pcg_hash(sr_key ^ (uint32_t)(c * prm.Pp + p));
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    rk = rk * 1664525u + 1013904223u;
                    u[j] = round_bf16_sr(u[j], rk >> 16);
                }
            }
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(u[j], u[l2], acc[tri<K>(j, l2)]);
            if (write) {
                UT *ub = static_cast<UT *>(a.U) + ((int64_t)c * npt + pt) * K * TP + r0;
#pragma unroll
                for (int j = 0; j < K; ++j) st_u(ub + j * TP, u[j]); // exact for a rounded bfloat16 value
            }
            if (c == C - 1) {
                const uint8_t nl = (valid && mx >= dl) ? 1 : 0;
                acc[NM] += (float)nl;
                if (write) {
                    a.labels[p] = nl;
                    if (a.mask_out && valid) a.mask_out[p] = nl;
                }
            }
            it = itn;
            c = cn;
        }
    }
    if (tid == 0 && stats) a.ks->sub_ts[5] = global_ns();
    cons_partials<F::NPU, NW>(acc, F::NVU, ucol, sred, a.col_stride);
    }
    cons_sync<NT>();
    if (tid == 0 && stats) a.ks->sub_ts[6] = global_ns();
    if constexpr (CL) {
        // cluster form: every CTA's partial values, then CTA 0 ends the frame
        cluster_sync_all();
        if (tid == 0) sk.last = b == 0;
    } else if constexpr (RES) {
        // resident form: every CTA arrives with its partial values (the
        // FRAME_ARRIVALS count as in the grid form) and goes on; the end CTA,
        // which streams no rows, waits for all arrivals and ends the frame
        // while the others run the next frame's first pass
        if (tid == 0) {
            red_release_add(&a.bar->count, sk.proj ? 1ull : 2ull);
            sk.last = b == G - 1;
        }
        if (b == G - 1) {
            const unsigned long long fend = a.bar_base + (unsigned long long)(fr + 1) * (unsigned long long)G *
                                                             (unsigned long long)frame_arrivals(prm.n_cg);
            if (!grid_wait<NT, true, false>(a.bar, fend, &sk.err, a.ks, a.status_out)) return;
        }
    } else if (tid == 0) {
        // every CTA arrives FRAME_ARRIVALS(n_cg) times per frame: once per
        // residual pass, once at the projection barrier (counted here when that
        // pass did not run) and once here; the last arrival of all is here
        __threadfence(); // the CTA's partial values before the arrival
        const unsigned long long inc = sk.proj ? 1ull : 2ull;
        const unsigned long long old = atomicAdd(&a.bar->count, inc);
        sk.last = old + inc == a.bar_base + (unsigned long long)(fr + 1) * (unsigned long long)G *
                                                (unsigned long long)frame_arrivals(prm.n_cg);
        __threadfence();
    }
    cons_sync<NT>();
    if (tid == 0 && stats) a.ks->sub_ts[7] = global_ns();
    if (sk.last) {
        if constexpr (WSUM)
            reduce_warp_sums(ucols, G, a.col_stride, F::NVU, tot);
        else
            reduce_cols<NT>(ucols, G, a.col_stride, F::NVU, tot, rscr);
        if (tid == 0) a.ks->sub_ts[8] = global_ns();
        end_frame<K, NT>(sk, a.ks, tot, tot[NM], rs, a.status_out);
        if (tid == 0) a.ks->sub_ts[9] = global_ns();
        if (tid == 0) a.ks->phase_ts[prm.n_cg + 2] = global_ns();
    }
    if (fr + 1 < nfr) {
        // the next frame of the launch starts at once in every CTA.  Its
        // residual passes need only the stored-row coefficients T y: each CTA
        // forms them from its own y and T_old with the operations of
        // end_frame (bit-identical to what the last CTA stores), or keeps them
        // after a rejected frame.  The new factors, y and frame counter, which
        // the last CTA writes before its first arrival of the next frame, are
        // read after the next frame's first grid barrier (reload_state).
        cons_sync<NT>();
        if (tid < K && !sk.skip) {
            double ty = 0.0;
            for (int q = tid; q < K; ++q) ty = dfma(rs.Told[tid * K + q], sk.y[q], ty);
            sk.yf[tid] = (float)ty;
        }
        cons_sync<NT>();
        if (tid == 0) {
            sk.skip = 0;
            sk.last = 0;
            sk.proj = 0;
        }
        buf ^= 1;
        cons_sync<NT>();
    }
    } // frames of the launch
}

// One stream: the whole grid.
template <int K, typename FT, typename UT>
__global__ void __launch_bounds__(FCfg<K, UT>::THREADS, 1) k_frame(const FrameArgs a)
{
    frame_body<K, FT, UT>(a, (int)gridDim.x, (int)blockIdx.x);
}

// One stream: the whole grid as one thread-block cluster (small frames).
template <int K, typename FT, typename UT>
__global__ void __launch_bounds__(FCfg<K, UT>::THREADS, 1) k_frame_cluster(const FrameArgs a)
{
    frame_body<K, FT, UT, true>(a, (int)gridDim.x, (int)blockIdx.x);
}

// One stream: the whole grid, in the resident form (k <= 10).
template <int K, typename FT, typename UT>
__global__ void __launch_bounds__(FCfg<K, UT>::THREADS, 1) k_frame_res(const FrameArgs a)
{
    if constexpr (!FCfg<K, UT>::STREAM) frame_body<K, FT, UT, false, true>(a, (int)gridDim.x, (int)blockIdx.x);
}

// Several streams of one kernel family in one cooperative launch: each CTA
// takes its stream's arguments from the device table (the grid barriers are
// per stream, and all CTAs of the launch are resident together, so a stream's
// CTAs wait only on each other).
template <int K, typename FT, typename UT>
__global__ void __launch_bounds__(FCfg<K, UT>::THREADS, 1) k_frame_multi(const FrameArgs *args, const int2 *map)
{
    __shared__ FrameArgs sa;
    const int2 mb = map[blockIdx.x];
    if (threadIdx.x == 0) sa = args[mb.x];
    __syncthreads();
    frame_body<K, FT, UT>(sa, sa.grid, mb.y);
}

template <int K, typename UT> struct FrameOps {
    using F = FCfg<K, UT>;
    // dynamic shared memory: the per-warp stages of the streaming form
    template <typename FT> static constexpr int dyn_smem()
    {
        return F::STREAM ? F::NW * StageCfg<K, FT, UT>::WARP_B : 0;
    }
    template <typename FT> static cudaError_t launch_t(const FrameArgs &a, int grid, cudaStream_t s)
    {
        void *args[] = {const_cast<FrameArgs *>(&a)};
        return cudaLaunchCooperativeKernel((void *)k_frame<K, FT, UT>, dim3(grid), dim3(F::THREADS), args,
                                           dyn_smem<FT>(), s);
    }
    static cudaError_t launch(const FrameArgs &a, int fdt, int grid, cudaStream_t s)
    {
        return fdt == 0 ? launch_t<uint8_t>(a, grid, s) : launch_t<float>(a, grid, s);
    }
    // the cluster form: one cluster of `grid` CTAs (up to 16, a non-portable size)
    template <typename FT> static cudaError_t cluster_attrs()
    {
        static cudaError_t done = cudaErrorNotReady; // once per instantiation
        if (done == cudaErrorNotReady) {
            done = cudaFuncSetAttribute(k_frame_cluster<K, FT, UT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (done == cudaSuccess && dyn_smem<FT>() > 0)
                done = cudaFuncSetAttribute(k_frame_cluster<K, FT, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            dyn_smem<FT>());
        }
        return done;
    }
    template <typename FT> static void cluster_cfg(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, int grid,
                                                   cudaStream_t s)
    {
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(F::THREADS);
        cfg.dynamicSmemBytes = dyn_smem<FT>();
        cfg.stream = s;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = grid;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    template <typename FT> static cudaError_t cluster_t(const FrameArgs &a, int grid, cudaStream_t s)
    {
        cudaError_t e = cluster_attrs<FT>();
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        cluster_cfg<FT>(cfg, at, grid, s);
        return cudaLaunchKernelEx(&cfg, k_frame_cluster<K, FT, UT>, a);
    }
    static cudaError_t cluster(const FrameArgs &a, int fdt, int grid, cudaStream_t s)
    {
        return fdt == 0 ? cluster_t<uint8_t>(a, grid, s) : cluster_t<float>(a, grid, s);
    }
    // clusters of `grid` CTAs that can be resident at once (0: the form cannot run)
    template <typename FT> static int cluster_fit_t(int grid)
    {
        if (cluster_attrs<FT>() != cudaSuccess) return 0;
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        cluster_cfg<FT>(cfg, at, grid, 0);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_frame_cluster<K, FT, UT>, &cfg) != cudaSuccess) return 0;
        return n;
    }
    static int cluster_fit(int fdt, int grid) { return fdt == 0 ? cluster_fit_t<uint8_t>(grid) : cluster_fit_t<float>(grid); }
    template <typename FT>
    static cudaError_t multi_t(const FrameArgs *args, const int2 *map, int ctas, cudaStream_t s)
    {
        void *kargs[] = {const_cast<FrameArgs **>(&args), const_cast<int2 **>(&map)};
        static bool attr = false; // the dynamic shared memory limit, once per instantiation
        if (!attr && dyn_smem<FT>() > 0) {
            const cudaError_t e = cudaFuncSetAttribute(k_frame_multi<K, FT, UT>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem<FT>());
            if (e != cudaSuccess) return e;
        }
        attr = true;
        return cudaLaunchCooperativeKernel((void *)k_frame_multi<K, FT, UT>, dim3(ctas), dim3(F::THREADS), kargs,
                                           dyn_smem<FT>(), s);
    }
    static cudaError_t multi(const FrameArgs *args, const int2 *map, int ctas, int fdt, cudaStream_t s)
    {
        return fdt == 0 ? multi_t<uint8_t>(args, map, ctas, s) : multi_t<float>(args, map, ctas, s);
    }
    template <typename FT> static int prepare_t()
    {
        int n = 0;
        if (dyn_smem<FT>() > 0 &&
            cudaFuncSetAttribute(k_frame<K, FT, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn_smem<FT>()) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_frame<K, FT, UT>, F::THREADS, dyn_smem<FT>()) !=
            cudaSuccess)
            return 0;
        return n;
    }
    // resident CTAs per SM (0: the kernel cannot run)
    static int prepare(int fdt) { return fdt == 0 ? prepare_t<uint8_t>() : prepare_t<float>(); }
    // the resident form's plan on the current device: the largest dynamic
    // shared memory its CTA can take (the opt-in limit less its static shared
    // memory), then as many row slots as fit beside the frame entries and
    // labels of the CTA with the most pixels
    template <typename FT> static int res_plan_t(int64_t P, int C, int grid, int *ns, int *smem)
    {
        if constexpr (F::STREAM) {
            return 0;
        } else {
            int dev = 0, optin = 0, n = 0;
            cudaFuncAttributes fa;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, k_frame_res<K, FT, UT>) != cudaSuccess)
                return 0;
            const int64_t cap = ((int64_t)optin - (int64_t)fa.sharedSizeBytes) & ~(int64_t)15;
            if (grid < 2) return 0;
            const int npm = res_npair_max(P, grid - 1); // grid - 1 CTAs own the pixels
            const int64_t nim = (int64_t)C * npm;
            const int64_t fixed = (int64_t)res_smem_bytes<K, FT, UT>(C, npm, 0);
            const int64_t slot = (int64_t)K * sizeof(typename RPair<UT>::T);
            if (cap <= fixed) return 0;
            int64_t nsl = (cap - fixed) / slot;
            if (nsl > nim) nsl = nim;
            const int64_t bytes = (int64_t)res_smem_bytes<K, FT, UT>(C, npm, (int)nsl);
            if (bytes > cap) return 0;
            // the attribute is the largest size any handle asks for: always the cap
            if (cudaFuncSetAttribute(k_frame_res<K, FT, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cap) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_frame_res<K, FT, UT>, F::THREADS, (int)bytes) !=
                    cudaSuccess ||
                n < 1)
                return 0;
            *ns = (int)nsl;
            *smem = (int)bytes;
            return 1;
        }
    }
    static int res_plan(int fdt, int64_t P, int C, int grid, int *ns, int *smem)
    {
        return fdt == 0 ? res_plan_t<uint8_t>(P, C, grid, ns, smem) : res_plan_t<float>(P, C, grid, ns, smem);
    }
    template <typename FT> static cudaError_t res_t(const FrameArgs &a, int grid, int smem, cudaStream_t s)
    {
        if constexpr (F::STREAM) {
            return cudaErrorInvalidValue;
        } else {
            void *args[] = {const_cast<FrameArgs *>(&a)};
            return cudaLaunchCooperativeKernel((void *)k_frame_res<K, FT, UT>, dim3(grid), dim3(F::THREADS), args,
                                               smem, s);
        }
    }
    static cudaError_t frame_res(const FrameArgs &a, int fdt, int grid, int smem, cudaStream_t s)
    {
        return fdt == 0 ? res_t<uint8_t>(a, grid, smem, s) : res_t<float>(a, grid, smem, s);
    }
};

template <int K, typename UT> const KernelOps *kernel_table()
{
    static const KernelOps ops = {&FrameOps<K, UT>::launch, &FrameOps<K, UT>::prepare, &FrameOps<K, UT>::multi,
                                  &FrameOps<K, UT>::cluster, &FrameOps<K, UT>::cluster_fit,
                                  &Ops<K, UT>::gram,
                                  &Ops<K, UT>::export_u, &Ops<K, UT>::gram_occupancy, &Ops<K, UT>::rebase,
                                  Cfg<K>::VW, FCfg<K, UT>::TP, FCfg<K, UT>::THREADS,
                                  FCfg<K, UT>::STREAM ? nullptr : &FrameOps<K, UT>::res_plan,
                                  FCfg<K, UT>::STREAM ? nullptr : &FrameOps<K, UT>::frame_res};
    return &ops;
}

} // namespace prost
