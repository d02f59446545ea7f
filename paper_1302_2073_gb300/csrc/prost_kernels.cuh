// Per-pixel kernels of pROST's per-frame update (arXiv:1302.2073, Section 3.3)
// for sm_103a, templated on the subspace dimension K.
//
// One frame runs n_cg + 2 launches, each a single streaming pass over the
// stored subspace (no residual vector is ever written):
//   k_pass<WM=true>   at CG iterate j < n_cg : r = x - U y_j, cost, gradient
//                     g = U^T eta, the weighted Gram M = U^T diag(c) U and the
//                     non-finite-entry count; the last CTA runs the CG step.
//   k_pass<WM=false>  at the final iterate  : cost, g, |eta|^2; the last CTA
//                     forms the rank-one SVD and the geodesic angle of Step 2.
//   k_ustep           geodesic update of every row, labels and weights of
//                     Step 3, optional background, Gram of the new subspace;
//                     the last CTA runs the FP64 Cholesky-QR that is folded
//                     into the next frame.
// Reductions are deterministic: per-thread FP32 sums, a split warp reduction,
// per-CTA partials in a fixed slot, and a fixed-order (Kahan) sum over CTAs in
// the last CTA to arrive.
#pragma once

#include <math.h>
#include <stdint.h>

#include "prost_device.h"

namespace prost {

// rows (pixels) per thread of the per-pixel kernels
template <int K> struct Cfg {
    static constexpr int VW = K <= 6 ? 4 : (K <= 12 ? 2 : 1);  // residual passes
    static constexpr int VWU = K <= 4 ? 4 : (K <= 8 ? 2 : 1);  // update pass (more live values per row)
};

// index of (j, l), j <= l, in a packed upper-triangular K x K matrix
template <int K> __host__ __device__ constexpr int tri(int j, int l)
{
    return j * K - (j * (j - 1)) / 2 + (l - j);
}

constexpr unsigned FULL = 0xffffffffu;

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

// ---- k-space steps (one warp of the last CTA, FP64) ------------------------

// CG bookkeeping at iterate `pass` from the reduced sums tot:
//   WM:  tot = [g_st (K) | M_st packed (K(K+1)/2) | f | |eta|^2 | #non-finite]
//   !WM: tot = [g_st (K) | f | |eta|^2 | #non-finite]
// g_st = U_st^T eta and M_st = U_st^T diag(c) U_st refer to the stored rows;
// with U = U_st T the gradient is g = T^T g_st and d^T M d = (T d)^T M_st (T d).
template <int K, bool WM>
__device__ void kspace_pass(KState *ks, const DevParams &prm, const double *tot, int pass)
{
    constexpr int NM = WM ? K * (K + 1) / 2 : 0;
    const int l = threadIdx.x;
    const bool act = l < K;
    const double f = tot[K + NM], ee = tot[K + NM + 1], nbad = tot[K + NM + 2];
    if (pass == 0) {
        if (nbad > 0.0) {
            if (l == 0) {
                ks->skip = 1;
                ks->err_flags |= ERR_BADFRAME;
                ks->last_status = -4; // PROST_EBADFRAME
                ks->bad_frames += 1;
            }
            return;
        }
        if (l == 0) ks->skip = 0;
    }
    double gl = 0.0;
    if (act)
        for (int i = 0; i <= l; ++i) gl += ks->T[i * KMAX + l] * tot[i];
    const double gsq = wsum(act ? gl * gl : 0.0);
    double beta = 0.0, dl;
    if (pass == 0) {
        dl = act ? -gl : 0.0;
    } else {
        const double gp = act ? ks->gprev[l] : 0.0;
        const double ggp = wsum(gp * gp);
        const double num = wsum(act ? gl * (gl - gp) : 0.0);
        beta = ggp > 0.0 ? fmax(0.0, num / ggp) : 0.0;
        dl = act ? -gl + beta * ks->d[l] : 0.0;
    }
    if (l == 0) {
        ks->cost[pass] = f;
        ks->gnorm[pass] = sqrt(gsq);
        ks->beta[pass] = beta;
    }
    if (pass < prm.n_cg) {
        // majorise-minimise line step: alpha = -d^T g / (p d^T M d)
        double dst = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const double di = __shfl_sync(FULL, dl, i);
            if (act && i >= l) dst += ks->T[l * KMAX + i] * di;
        }
        double md = 0.0;
        if constexpr (WM) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const double si = __shfl_sync(FULL, dst, i);
                if (act) md += tot[K + (l <= i ? tri<K>(l, i) : tri<K>(i, l))] * si;
            }
        }
        const double den = prm.pd * wsum(act ? dst * md : 0.0);
        const double dg = wsum(act ? dl * gl : 0.0);
        const double alpha = den > 0.0 ? -dg / den : 0.0;
        const double yl = act ? ks->y[l] + alpha * dl : 0.0;
        double ys = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const double yi = __shfl_sync(FULL, yl, i);
            if (act && i >= l) ys += ks->T[l * KMAX + i] * yi;
        }
        if (act) {
            ks->y[l] = yl;
            ks->d[l] = dl;
            ks->gprev[l] = gl;
            ks->yf[l] = (float)ys;
        }
        if (l == 0) ks->alpha[pass] = alpha;
    } else {
        // Step 2 quantities: |pi(eta)|^2 = |eta|^2 - |U^T eta|^2 (U orthonormal),
        // sigma_1 = |pi(eta)| |y|, v = y/|y| (Eq. svd), theta = sigma_1 t.
        const double yl = act ? ks->y[l] : 0.0;
        const double yn = sqrt(wsum(yl * yl));
        const double pin2 = ee - gsq;
        const double pin = pin2 > 0.0 ? sqrt(pin2) : 0.0;
        const double t = fmax(exp(-prm.tau * (double)ks->frame_index) * prm.t_init, prm.t_min);
        const double sigma = pin * yn;
        const double theta = sigma * t;
        const bool upd = yn > 0.0 && pin > 0.0;
        const double sh = sin(0.5 * theta);
        if (act) {
            ks->ye[l] = (float)yl;
            ks->gf[l] = (float)gl;
            ks->vf[l] = upd ? (float)(yl / yn) : 0.f;
            ks->g[l] = gl;
        }
        if (l == 0) {
            ks->cm1 = upd ? (float)(-2.0 * sh * sh) : 0.f;
            ks->sn_pin = upd ? (float)(sin(theta) / pin) : 0.f;
            ks->ynorm = (float)yn;
            ks->do_update = upd ? 1 : 0;
            ks->pi_norm = pin;
            ks->y_norm = yn;
            ks->sigma = sigma;
            ks->t = t;
            ks->theta = upd ? theta : 0.0;
            ks->updated = upd ? 1 : 0;
            ks->n_cg_done = prm.n_cg;
        }
    }
}

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

template <int K, typename FT, bool WM>
__global__ void __launch_bounds__(THREADS) k_pass(const PassArgs a)
{
    constexpr int VW = Cfg<K>::VW;
    constexpr int NM = WM ? K * (K + 1) / 2 : 0;
    constexpr int NV = K + NM + 3;
    constexpr int NP = (NV + 31) / 32 * 32;
    __shared__ float sred[(THREADS / 32) * NP];
    __shared__ double tot[NV];

    if (a.pass > 0 && a.ks->skip) return; // frame rejected by pass 0 (uniform)
    const DevParams &prm = a.prm;
    float y[K];
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = a.ks->yf[j];
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;

    float acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.f;

    const int ngroups = (int)(prm.Pp / VW);
    const int nitems = prm.C * ngroups;
    const FT *frame = static_cast<const FT *>(a.frame);
    for (int it = blockIdx.x * THREADS + threadIdx.x; it < nitems; it += gridDim.x * THREADS) {
        const int c = it / ngroups;
        const int64_t p0 = (int64_t)(it - c * ngroups) * VW;
        const int nvalid = prm.P - p0 < (int64_t)VW ? (int)(prm.P - p0) : VW;
        if (nvalid <= 0) continue;
        float u[K][VW];
#pragma unroll
        for (int j = 0; j < K; ++j) VL<VW>::ldu(a.U + ((int64_t)j * prm.C + c) * prm.Pp + p0, u[j]);
        float xv[VW];
        load_x<VW, FT>(frame + (int64_t)c * prm.P + p0, nvalid, prm.vec, xv);
        uint8_t lab[VW];
        VL<VW>::ldlab(a.labels + p0, lab);
#pragma unroll
        for (int r = 0; r < VW; ++r) {
            const bool valid = r < nvalid;
            float uy = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) uy = fmaf(u[j][r], y[j], uy);
            const float x = fmaf(xv[r], sc, -of);
            if constexpr (sizeof(FT) == 4) {
                if (valid && !isfinite(xv[r])) acc[K + NM + 2] += 1.f;
            }
            const float res = x - uy;
            const float z = fmaf(res, res, mu);
            const float tz = __powf(z, e);               // (r^2 + mu)^(p/2 - 1)
            const float wv = valid ? (lab[r] ? om : 1.f) : 0.f;
            const float cw = wv * tz;                     // c_e
            acc[K + NM] = fmaf(cw, z, acc[K + NM]);       // w (r^2 + mu)^(p/2)
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
    block_partials<NP>(acc, NV, a.partials + (size_t)blockIdx.x * NV, sred);
    if (!arrive_last(a.counter)) return;
    reduce_partials<NV>(a.partials, gridDim.x, tot, sred);
    if (threadIdx.x < 32) kspace_pass<K, WM>(a.ks, prm, tot, a.pass);
    if (threadIdx.x == 0) *a.counter = 0u;
}

template <int K, typename FT>
__global__ void __launch_bounds__(THREADS) k_ustep(const UstepArgs a)
{
    constexpr int VW = Cfg<K>::VWU;
    constexpr int NM = K * (K + 1) / 2;
    constexpr int NV = NM + 1;
    constexpr int NP = (NV + 31) / 32 * 32;
    __shared__ float sred[(THREADS / 32) * NP];
    __shared__ double tot[NV];
    __shared__ double sR[K * K], sT[K * K];
    __shared__ float s_T[K * K], s_y[K], s_g[K], s_v[K];

    if (a.ks->skip) return;
    const DevParams &prm = a.prm;
    for (int i = threadIdx.x; i < K * K; i += THREADS) s_T[i] = a.ks->Tf[i];
    if (threadIdx.x < K) {
        s_y[threadIdx.x] = a.ks->ye[threadIdx.x];
        s_g[threadIdx.x] = a.ks->gf[threadIdx.x];
        s_v[threadIdx.x] = a.ks->vf[threadIdx.x];
    }
    const float cm1 = a.ks->cm1, snp = a.ks->sn_pin, yn = a.ks->ynorm;
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta;
    const float sc = prm.in_scale, of = prm.in_offset;
    const bool pre = prm.mask_pre != 0;
    __syncthreads();

    float acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.f;

    const int ngroups = (int)(prm.Pp / VW);
    const FT *frame = static_cast<const FT *>(a.frame);
    for (int pg = blockIdx.x * THREADS + threadIdx.x; pg < ngroups; pg += gridDim.x * THREADS) {
        const int64_t p0 = (int64_t)pg * VW;
        const int nvalid = prm.P - p0 < (int64_t)VW ? (int)(prm.P - p0) : VW;
        if (nvalid <= 0) continue;
        uint8_t lab[VW];
        VL<VW>::ldlab(a.labels + p0, lab);
        float mx[VW];
#pragma unroll
        for (int r = 0; r < VW; ++r) mx[r] = 0.f;
        for (int c = 0; c < prm.C; ++c) {
            float u[K][VW];
#pragma unroll
            for (int j = 0; j < K; ++j) VL<VW>::ldu_rw(a.U + ((int64_t)j * prm.C + c) * prm.Pp + p0, u[j]);
            float xv[VW];
            load_x<VW, FT>(frame + (int64_t)c * prm.P + p0, nvalid, prm.vec, xv);
#pragma unroll
            for (int r = 0; r < VW; ++r) {
                const bool valid = r < nvalid;
                // row of the orthonormal representative: u = T^T u_st
                float ue[K];
#pragma unroll
                for (int j = K - 1; j >= 0; --j) {
                    float s = 0.f;
#pragma unroll
                    for (int i = 0; i <= j; ++i) s = fmaf(s_T[i * K + j], u[i][r], s);
                    ue[j] = s;
                }
                float uy = 0.f, ug = 0.f, uv = 0.f;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    uy = fmaf(ue[j], s_y[j], uy);
                    ug = fmaf(ue[j], s_g[j], ug);
                    uv = fmaf(ue[j], s_v[j], uv);
                }
                const float x = fmaf(xv[r], sc, -of);
                const float res = x - uy;
                const float z = fmaf(res, res, mu);
                const float tz = __powf(z, e);
                const float wv = valid ? (lab[r] ? om : 1.f) : 0.f;
                const float eta = -pw * wv * tz * res;
                // u <- u + ((cos(theta) - 1) u^T v - sin(theta) pi(eta)_e / |pi(eta)|) v
                const float gam = valid ? fmaf(cm1, uv, -snp * (eta - ug)) : 0.f;
                const float rn = pre ? res : fmaf(-gam, yn, res);
                if (valid) {
                    mx[r] = fmaxf(mx[r], fabsf(rn));
                    if (a.bg_out) a.bg_out[(int64_t)c * prm.P + p0 + r] = x - rn + of;
                }
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    ue[j] = fmaf(gam, s_v[j], ue[j]);
                    u[j][r] = ue[j];
                }
#pragma unroll
                for (int j = 0; j < K; ++j)
#pragma unroll
                    for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(ue[j], ue[l2], acc[tri<K>(j, l2)]);
            }
#pragma unroll
            for (int j = 0; j < K; ++j) VL<VW>::stu(a.U + ((int64_t)j * prm.C + c) * prm.Pp + p0, u[j]);
        }
        uint8_t nl[VW];
#pragma unroll
        for (int r = 0; r < VW; ++r) {
            nl[r] = (r < nvalid && mx[r] >= dl) ? 1 : 0;
            acc[NM] += (float)nl[r];
        }
        VL<VW>::stlab(a.labels + p0, nl);
        if (a.mask_out) {
#pragma unroll
            for (int r = 0; r < VW; ++r)
                if (r < nvalid) a.mask_out[p0 + r] = nl[r];
        }
    }
    block_partials<NP>(acc, NV, a.partials + (size_t)blockIdx.x * NV, sred);
    if (!arrive_last(a.counter)) return;
    reduce_partials<NV>(a.partials, gridDim.x, tot, sred);
    if (threadIdx.x < 32) finish_reorth<K>(a.ks, tot, sR, sT, true, tot[NM]);
    if (threadIdx.x == 0) *a.counter = 0u;
}

// Gram of the stored subspace and its Cholesky-QR (after init / import).
template <int K>
__global__ void __launch_bounds__(THREADS) k_gram(const GramArgs a)
{
    constexpr int VW = Cfg<K>::VW;
    constexpr int NM = K * (K + 1) / 2;
    constexpr int NP = (NM + 31) / 32 * 32;
    __shared__ float sred[(THREADS / 32) * NP];
    __shared__ double tot[NM];
    __shared__ double sR[K * K], sT[K * K];
    const DevParams &prm = a.prm;
    float acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.f;
    const int ngroups = (int)(prm.Pp / VW);
    const int nitems = prm.C * ngroups;
    for (int it = blockIdx.x * THREADS + threadIdx.x; it < nitems; it += gridDim.x * THREADS) {
        const int c = it / ngroups;
        const int64_t p0 = (int64_t)(it - c * ngroups) * VW;
        float u[K][VW];
#pragma unroll
        for (int j = 0; j < K; ++j) VL<VW>::ldu(a.U + ((int64_t)j * prm.C + c) * prm.Pp + p0, u[j]);
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
template <int K>
__global__ void __launch_bounds__(THREADS) k_export(const float *U, const KState *ks, float *out,
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
        for (int j = 0; j < K; ++j) u[j] = U[((int64_t)j * prm.C + c) * prm.Pp + q];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i <= j; ++i) s = fmaf(sT[i * K + j], u[i], s);
            out[e * K + j] = s;
        }
    }
}

// ---- host launchers of one kernel set ----------------------------------------

template <int K> struct Ops {
    template <typename FT> static cudaError_t pass_t(const PassArgs &a, bool wm, int grid, cudaStream_t s)
    {
        if (wm) k_pass<K, FT, true><<<grid, THREADS, 0, s>>>(a);
        else k_pass<K, FT, false><<<grid, THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t pass(const PassArgs &a, bool wm, int fdt, int grid, cudaStream_t s)
    {
        return fdt == 0 ? pass_t<uint8_t>(a, wm, grid, s) : pass_t<float>(a, wm, grid, s);
    }
    static cudaError_t ustep(const UstepArgs &a, int fdt, int grid, cudaStream_t s)
    {
        if (fdt == 0) k_ustep<K, uint8_t><<<grid, THREADS, 0, s>>>(a);
        else k_ustep<K, float><<<grid, THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t gram(const GramArgs &a, int grid, cudaStream_t s)
    {
        k_gram<K><<<grid, THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t export_u(const float *U, const KState *ks, float *out, DevParams prm, cudaStream_t s)
    {
        const int64_t m = (int64_t)prm.C * prm.P;
        const int64_t nb = (m + THREADS - 1) / THREADS;
        const int grid = (int)(nb < 4096 ? nb : 4096);
        k_export<K><<<grid, THREADS, 0, s>>>(U, ks, out, prm);
        return cudaGetLastError();
    }
    static int occupancy(int kind, int fdt)
    {
        int n = 0;
        cudaError_t e = cudaSuccess;
        if (kind == 0) e = fdt == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass<K, uint8_t, true>, THREADS, 0)
                                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass<K, float, true>, THREADS, 0);
        else if (kind == 1) e = fdt == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass<K, uint8_t, false>, THREADS, 0)
                                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass<K, float, false>, THREADS, 0);
        else if (kind == 2) e = fdt == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ustep<K, uint8_t>, THREADS, 0)
                                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ustep<K, float>, THREADS, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gram<K>, THREADS, 0);
        return e == cudaSuccess && n > 0 ? n : 1;
    }
    static const KernelOps *table()
    {
        static const KernelOps ops = {&pass, &ustep, &gram, &export_u, &occupancy, Cfg<K>::VW, Cfg<K>::VWU};
        return &ops;
    }
};

} // namespace prost
