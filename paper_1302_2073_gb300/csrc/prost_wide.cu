// The pass-sequence form of one frame (arXiv:1302.2073, Section 3.3): the
// frame as a sequence of ordinary launches, with k chosen at run time up to
// KMAX = 32 and float32 stored rows.  It serves every k above the widest
// compiled single-launch kernel set (k = 17..32), and any k on request.
//
// At these k a CG pass's per-thread sums U^T diag(c) U (k(k+1)/2 = 528 at
// k = 32) and the Gram of the new rows do not fit in registers, so each CG
// iteration takes two passes over the rows, as the majorise-minimise line step
// is written: a gradient pass (f, U^T eta, |eta|^2) at the current y, then a
// curvature pass, sum_e c_e (u_e^T d)^2, which with d^T g gives
// alpha = -d^T g / (p sum_e c_e (u_e^T d)^2).  The final gradient pass, the
// projection pass when |pi(eta)|^2 = |eta|^2 - |U^T eta|^2 would cancel, the
// update pass (geodesic step, labels, weights) and a tiled Gram pass of the
// new rows follow; one CTA then factors the Gram (Cholesky-QR, FP64).  Every
// cross-CTA sum is a fixed-order sum by the last CTA to finish, so results are
// reproducible run to run, and that CTA then takes the k-space step that
// follows the pass.  The k-space vectors live in KState between the
// launches.  Arrays are KMAX wide; entries at and beyond k are zero.
#include <stdint.h>
#include <string.h>

#include "prost.h"
#include "prost_frame.cuh"

namespace prost {

namespace {

constexpr int KW = KMAX;                  // widest subspace of this form
constexpr int WT = 256;                   // threads per CTA of the row passes
constexpr int NWG = KW * (KW + 1) / 2;    // packed upper triangle of a KW x KW matrix
constexpr int TOTF = 544;                 // floats of reduced sums ahead of the per-CTA rows
constexpr int NB4 = (KW / 4) * (KW / 4 + 1) / 2; // 4 x 4 blocks of the upper triangle (36)
constexpr int GT = NB4 * 8;               // threads of the Gram kernel: 8 row groups per block
constexpr int RS = KW + 4;                // shared row stride of a staged tile (16-byte rows)
constexpr int GPER = (KW * TILE_P + GT - 1) / GT; // a Gram thread's loads of one tile block
constexpr int MAX_CTAS = 320;             // CTAs of a pass at most (the sums' scratch)
constexpr int RCH = 16;                   // rows per unit of a pass's cross-CTA sum
constexpr int GCH = 40;                   // rows per unit of the Gram's cross-CTA sum
static_assert(NWG * ((MAX_CTAS + GCH - 1) / GCH) <= TILE_P * RS, "the Gram's chunk sums fit the tile");
static_assert(KW == 32, "the pass-sequence form is written for up to 32 columns");
static_assert(TOTF >= NWG + 1 && TOTF % 4 == 0, "reduced sums: the Gram, then the foreground count");
static_assert(TILE_P % 8 == 0 && RS % 4 == 0, "row groups and 16-byte rows");

struct WideArgs {
    float *U;                 // stored subspace, tile-blocked (float32)
    const void *frame;        // channel planes frame_pitch entries apart
    int64_t frame_pitch;
    uint8_t *labels, *mask_out;
    float *bg_out;
    KState *ks;
    float *part;              // per-CTA partial sums, one row per CTA
    float *tot;               // the reduced sums (TOTF floats)
    unsigned int *counter;    // arrival counter of the last-CTA reductions
    int32_t *status_out;
    DevParams prm;
};

// Fixed-order sum over nrows partial rows of nv values (part[b * nv + i]) by
// the nt threads of one CTA: the rows are cut into chunks of CH, a unit
// (value, chunk) has all its CH loads in flight at once and sums them with
// Kahan compensation, and the chunk sums of each value are then added in
// chunk order, so the result depends only on nrows and CH.  scr holds
// nv * ceil(nrows / CH) floats.
template <int CH>
__device__ __forceinline__ void chunked_sum(const float *part, int nrows, int nv, float *tot, float *scr, int nt)
{
    const int nch = (nrows + CH - 1) / CH;
    for (int u = threadIdx.x; u < nv * nch; u += nt) {
        const int c = u / nv, i = u - (u / nv) * nv;
        float v[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int b = c * CH + q;
            v[q] = b < nrows ? __ldcg(part + (size_t)b * nv + i) : 0.f;
        }
        float sum = 0.f, comp = 0.f;
#pragma unroll
        for (int q = 0; q < CH; ++q) kahan_add(sum, comp, v[q]);
        scr[c * nv + i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += nt) {
        float sum = 0.f, comp = 0.f;
        for (int c = 0; c < nch; ++c) kahan_add(sum, comp, scr[c * nv + i]);
        tot[i] = sum;
    }
}

// CTA sums of NV per-thread values (shuffle tree per value, then the warps in
// order) into the CTA's row of part, then the fixed-order sum over the CTAs
// (chunked_sum) by the last CTA to arrive into tot.
template <int NV>
__device__ __forceinline__ bool wide_reduce(const float (&acc)[NV], float *part, float *tot, unsigned int *counter)
{
    __shared__ float sw[WT / 32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float v = acc[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        if (lane == 0) sw[w][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += WT) {
        float a = 0.f;
#pragma unroll
        for (int ww = 0; ww < WT / 32; ++ww) a += sw[ww][i];
        part[(size_t)blockIdx.x * NV + i] = a;
    }
    if (!arrive_last(counter)) return false;
    __shared__ float scr[NV * ((MAX_CTAS + RCH - 1) / RCH)];
    chunked_sum<RCH>(part, (int)gridDim.x, NV, tot, scr, WT);
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads(); // tot is complete for the CTA
    return true;
}

// Step 2's angle from |pi(eta)| (one thread): sigma = |pi(eta)| |y| (Eq. svd),
// theta = sigma t (Eq. geodesic), skipped when |y| = 0 or |pi(eta)| = 0.
__device__ void wide_angle(KState *ks, const DevParams &prm, float pin)
{
    const float yn = ks->wyn;
    const bool upd = yn > 0.f && pin > 0.f;
    const float t = step_size(prm, ks->frame_index);
    const float sigma = pin * yn;
    const float theta = sigma * t;
    const float sh = sinf(0.5f * theta);
    ks->wcm1 = upd ? -2.f * sh * sh : 0.f;
    ks->wsnp = upd ? sinf(theta) / pin : 0.f;
    ks->pi_norm = pin;
    ks->y_norm = yn;
    ks->sigma = sigma;
    ks->t = t;
    ks->theta = upd ? theta : 0.f;
    ks->updated = upd ? 1 : 0;
}

// The k-space steps, run by the last CTA of the pass before, once it has
// reduced the pass's sums into tot: its threads stage T (and R) in shared
// memory, then one warp (lane l < k holds entry l) takes the step:
//   STAGE 0, after gradient pass `pass` < n_cg: g = T^T g_st, the PR+ beta,
//            d = -g + beta d, s = T d (the direction in the stored basis), d^T g;
//   STAGE 1, after its curvature pass: alpha, y += alpha d, T y += alpha s;
//   STAGE 2, after the final gradient pass: |pi(eta)| from the norm identity
//            or the request for the projection pass; v = y/|y|, T v, T g,
//            w = R^T v and (without the projection pass) the angle;
//   STAGE 3, after the projection pass: the angle from the explicit |pi(eta)|.
struct StepSmem {
    float T[KW * KW]; // T = R^{-1}, row-major, zero outside k x k
    float R[KW * KW]; // R, row-major, zero outside k x k (STAGE 2)
};

template <int STAGE>
__device__ void wide_step(const WideArgs &a, int pass, StepSmem &sm)
{
    KState *ks = a.ks;
    const DevParams &prm = a.prm;
    const int k = prm.k, l = threadIdx.x;
    if constexpr (STAGE == 0 || STAGE == 2) {
        for (int i = threadIdx.x; i < KW * KW; i += WT) {
            const int r = i / KW, c = i - (i / KW) * KW;
            const bool in = r < k && c < k;
            sm.T[i] = in ? ks->Tf[r * k + c] : 0.f;
            if (STAGE == 2) sm.R[i] = in ? (float)ks->R[r * KMAX + c] : 0.f;
        }
        __syncthreads();
    }
    if (threadIdx.x >= 32) return;
    const bool act = l < k;
    const float *tot = a.tot;
    if constexpr (STAGE == 1) {
        const float den = prm.p * tot[0];
        const float alpha = den > 0.f ? -ks->wdg / den : 0.f;
        if (act) {
            ks->y[l] = fma((double)alpha, (double)ks->wd[l], ks->y[l]);
            ks->yf[l] = fmaf(alpha, ks->ws[l], ks->yf[l]);
        }
        if (l == 0) ks->alpha[pass] = alpha;
    } else if constexpr (STAGE == 3) {
        if (l == 0) wide_angle(ks, prm, sqrtf(fmaxf(tot[0], 0.f)));
    } else {
        const float f = tot[KW], ee = tot[KW + 1], nbad = tot[KW + 2];
        // g = T^T g_st (T upper triangular; zero outside k x k)
        float gl = 0.f;
#pragma unroll
        for (int i = 0; i < KW; ++i) gl = fmaf(sm.T[i * KW + l], tot[i], gl);
        if (!act) gl = 0.f;
        const float gsq = wsumf(gl * gl);
        float beta = 0.f, dl;
        if (pass == 0) {
            dl = -gl;
        } else {
            const float gp = act ? ks->wgp[l] : 0.f;
            const float ggp = wsumf(gp * gp);
            const float num = wsumf(gl * (gl - gp));
            beta = ggp > 0.f ? fmaxf(0.f, num / ggp) : 0.f;
            dl = act ? fmaf(beta, ks->wd[l], -gl) : 0.f;
        }
        if (l == 0) {
            ks->cost[pass] = f;
            ks->gnorm[pass] = sqrtf(gsq);
            ks->beta[pass] = beta;
        }
        if (pass == 0 && nbad > 0.f) {
            if (l == 0) ks->wskip = 1; // the later launches of this frame return at once
            return;
        }
        if constexpr (STAGE == 0) {
            const float dg = wsumf(dl * gl);
            float sl = 0.f;
#pragma unroll
            for (int i = 0; i < KW; ++i) sl = fmaf(sm.T[l * KW + i], __shfl_sync(FULL, dl, i), sl);
            if (act) {
                ks->wd[l] = dl;
                ks->wgp[l] = gl;
                ks->ws[l] = sl;
            }
            if (l == 0) ks->wdg = dg;
        } else {
            const float yl = act ? (float)ks->y[l] : 0.f;
            const float yn = sqrtf(wsumf(yl * yl));
            // |pi(eta)|^2 = |eta|^2 - |U^T eta|^2 (Eq. gproject, U orthonormal)
            // cancels when most of eta lies in span(U); below PROJ_RATIO |eta|^2
            // the projection pass forms the norm explicitly instead
            const float pin2 = ee - gsq;
            const bool proj = yn > 0.f && ee > 0.f && !(pin2 > PROJ_RATIO * ee);
            const float pin = (!proj && pin2 > 0.f) ? sqrtf(pin2) : 0.f;
            const bool upd = yn > 0.f && (proj || pin > 0.f);
            const float vl = (act && upd) ? yl / yn : 0.f;
            float tv = 0.f, tg = 0.f, wl = 0.f;
#pragma unroll
            for (int i = 0; i < KW; ++i) {
                const float vi = __shfl_sync(FULL, vl, i);
                const float gi = __shfl_sync(FULL, gl, i);
                tv = fmaf(sm.T[l * KW + i], vi, tv);
                tg = fmaf(sm.T[l * KW + i], gi, tg);
                wl = fmaf(sm.R[i * KW + l], vi, wl);
            }
            if (act) {
                ks->wtv[l] = tv;
                ks->wtg[l] = tg;
                ks->ww[l] = wl;
            }
            if (l == 0) {
                ks->wyn = yn;
                ks->wproj = proj ? 1 : 0;
                ks->eta_norm = sqrtf(fmaxf(ee, 0.f));
                ks->pi_explicit = proj ? 1 : 0;
                ks->n_cg_done = prm.n_cg;
                if (!proj) wide_angle(ks, prm, pin);
            }
        }
    }
}

// One pass over the stored rows at the current y (float(T y) in yf):
// MODE 0, the gradient pass: [U_st^T eta (KW) | f | |eta|^2 | #non-finite];
// MODE 1, the curvature pass: sum_e c_e (u_st,e^T s)^2 with s = T d;
// MODE 2, the projection pass (only when the final step asked for it):
//         sum_e (eta_e - u_st,e^T tg)^2 with tg = T g (Eq. gproject).
template <typename FT, int MODE>
__global__ void __launch_bounds__(WT) k_wide_res(const WideArgs a, int pass)
{
    constexpr int NV = MODE == 0 ? KW + 3 : 1;
    const DevParams &prm = a.prm;
    const int k = prm.k;
    // every CTA reads the same flags, written by an earlier launch
    if (a.ks->wskip) return;
    if (MODE == 2 && !a.ks->wproj) return;
    __shared__ float sy[KW], sv[KW];
    if (threadIdx.x < KW) {
        const int j = threadIdx.x;
        sy[j] = j < k ? a.ks->yf[j] : 0.f;
        sv[j] = j < k ? (MODE == 1 ? a.ks->ws[j] : (MODE == 2 ? a.ks->wtg[j] : 0.f)) : 0.f;
    }
    __syncthreads();
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, sc = prm.in_scale, of = prm.in_offset;
    const FT *frame = static_cast<const FT *>(a.frame);
    const int64_t rows = (int64_t)prm.C * prm.Pp;
    for (int64_t r = (int64_t)blockIdx.x * WT + threadIdx.x; r < rows; r += (int64_t)gridDim.x * WT) {
        const int c = (int)(r / prm.Pp);
        const int64_t q = r - (int64_t)c * prm.Pp;
        const bool valid = q < prm.P;
        const float *ub = a.U + u_off(prm, c, q, 0);
        float u[KW];
#pragma unroll
        for (int j = 0; j < KW; ++j) u[j] = j < k ? __ldcg(ub + (int64_t)j * TILE_P) : 0.f;
        const float xv = valid ? (float)__ldg(frame + (int64_t)c * a.frame_pitch + q) : 0.f;
        const uint8_t lb = a.labels[q];
        float uy = 0.f, uv = 0.f;
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            uy = fmaf(u[j], sy[j], uy);
            if (MODE != 0) uv = fmaf(u[j], sv[j], uv);
        }
        const float res = valid ? fmaf(xv, sc, -of) - uy : 0.f;
        const float z = fmaf(res, res, mu);
        const float wv = valid ? (lb ? om : 1.f) : 0.f;
        const float cw = wv * __powf(z, e);
        if constexpr (MODE == 0) {
            if constexpr (sizeof(FT) == 4) {
                if (valid && !isfinite(xv)) acc[KW + 2] += 1.f;
            }
            acc[KW] = fmaf(cw, z, acc[KW]);
            const float eta = -pw * cw * res;
            acc[KW + 1] = fmaf(eta, eta, acc[KW + 1]);
#pragma unroll
            for (int j = 0; j < KW; ++j) acc[j] = fmaf(eta, u[j], acc[j]);
        } else if constexpr (MODE == 1) {
            acc[0] = fmaf(cw * uv, uv, acc[0]);
        } else {
            const float pe = valid ? -pw * cw * res - uv : 0.f;
            acc[0] = fmaf(pe, pe, acc[0]);
        }
    }
    if (!wide_reduce<NV>(acc, a.part, a.tot, a.counter)) return;
    __shared__ StepSmem sm;
    if constexpr (MODE == 0) {
        if (pass < prm.n_cg)
            wide_step<0>(a, pass, sm);
        else
            wide_step<2>(a, pass, sm);
    } else if constexpr (MODE == 1) {
        wide_step<1>(a, pass, sm);
    } else {
        wide_step<3>(a, pass, sm);
    }
}

// Update pass: one pixel per thread, its channels in turn: the geodesic step
// of each stored row (u_st + gamma R^T v is the stored row of u + gamma v),
// the residual against the new row, the label (maximum over the channels
// >= delta, Step 3), the optional background; the foreground count.
template <typename FT>
__global__ void __launch_bounds__(WT) k_wide_update(const WideArgs a)
{
    const DevParams &prm = a.prm;
    const int k = prm.k;
    if (a.ks->wskip) return;
    __shared__ float sy[KW], sg[KW], sv[KW], sw[KW];
    __shared__ float scal[3];
    if (threadIdx.x < KW) {
        const int j = threadIdx.x;
        sy[j] = j < k ? a.ks->yf[j] : 0.f;
        sg[j] = j < k ? a.ks->wtg[j] : 0.f;
        sv[j] = j < k ? a.ks->wtv[j] : 0.f;
        sw[j] = j < k ? a.ks->ww[j] : 0.f;
    }
    if (threadIdx.x == 0) {
        scal[0] = a.ks->wcm1;
        scal[1] = a.ks->wsnp;
        scal[2] = a.ks->wyn;
    }
    __syncthreads();
    const float cm1 = scal[0], snp = scal[1], yn = scal[2];
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta, sc = prm.in_scale,
                of = prm.in_offset;
    const bool pre = prm.mask_pre != 0;
    const FT *frame = static_cast<const FT *>(a.frame);
    float acc[1] = {0.f};
    for (int64_t q = (int64_t)blockIdx.x * WT + threadIdx.x; q < prm.Pp; q += (int64_t)gridDim.x * WT) {
        const bool valid = q < prm.P;
        const float wv = valid ? (a.labels[q] ? om : 1.f) : 0.f;
        float mx = 0.f;
        for (int c = 0; c < prm.C; ++c) {
            float *ub = a.U + u_off(prm, c, q, 0);
            float u[KW];
#pragma unroll
            for (int j = 0; j < KW; ++j) u[j] = j < k ? __ldcg(ub + (int64_t)j * TILE_P) : 0.f;
            const float xv = valid ? (float)__ldg(frame + (int64_t)c * a.frame_pitch + q) : 0.f;
            float uy = 0.f, ug = 0.f, uv = 0.f;
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                uy = fmaf(u[j], sy[j], uy);
                ug = fmaf(u[j], sg[j], ug);
                uv = fmaf(u[j], sv[j], uv);
            }
            const float x = fmaf(xv, sc, -of);
            const float res = valid ? x - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float eta = -pw * wv * __powf(z, e) * res;
            // u <- u + ((cos(theta) - 1) u^T v - sin(theta) pi(eta)_e / |pi(eta)|) v
            const float gam = valid ? fmaf(cm1, uv, -snp * (eta - ug)) : 0.f;
            const float rn = pre ? res : fmaf(-gam, yn, res);
            if (valid) {
                mx = fmaxf(mx, fabsf(rn));
                if (a.bg_out) a.bg_out[(int64_t)c * prm.P + q] = x - rn + of;
            }
#pragma unroll
            for (int j = 0; j < KW; ++j)
                if (j < k) ub[(int64_t)j * TILE_P] = fmaf(gam, sw[j], u[j]);
        }
        const uint8_t nl = (valid && mx >= dl) ? 1 : 0;
        acc[0] += (float)nl;
        a.labels[q] = nl;
        if (a.mask_out && valid) a.mask_out[q] = nl;
    }
    (void)wide_reduce<1>(acc, a.part, a.tot + NWG, a.counter);
}

// Gram of the stored rows, packed upper (k-wide rows), into tot.  Each CTA
// (two per SM, so that one loads while the other sums) stages one tile block
// (k columns of TILE_P rows) at a time in shared memory, transposed to rows of
// RS floats.  Thread t sums the 4 x 4 block t / 8 of the upper triangle (36
// blocks) over the rows r = t % 8 (mod 8), with one 16-byte load of each
// row's 4 + 4 entries per 16 multiply-adds, in FP32 within a tile and
// Kahan-compensated across tiles; the 8 row groups of a block (8 consecutive
// lanes) are added by a fixed shuffle tree.
__global__ void __launch_bounds__(GT, 2) k_wide_gram(const float *U, const KState *ks, DevParams prm, float *part,
                                                    float *tot, unsigned int *counter, int after_rebase)
{
    if (after_rebase && !ks->rebased) return; // the periodic rebase was not due
    __shared__ __align__(16) float tile[TILE_P * RS];
    const int k = prm.k;
    const int t = threadIdx.x;
    const int blk = t >> 3, g = t & 7;
    int bi = 0, rem = blk;
    while (rem >= KW / 4 - bi) {
        rem -= KW / 4 - bi;
        ++bi;
    }
    const int bj = bi + rem; // block (bi, bj), bi <= bj
    const int i0 = 4 * bi, j0 = 4 * bj;
    const bool work = j0 < k;
    for (int i = t; i < TILE_P * RS; i += GT) tile[i] = 0.f; // columns >= k stay zero
    float s[16], cs[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) s[q] = cs[q] = 0.f;
    const int n = k * TILE_P; // floats of one tile block
    const int ntiles = prm.C * prm.npt;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        __syncthreads(); // the previous block's sums (and the zero fill) are done
        const float *src = U + (int64_t)ti * n;
        float v[GPER]; // every load of the block in flight before the stores
#pragma unroll
        for (int q = 0; q < GPER; ++q) {
            const int i = t + GT * q;
            v[q] = i < n ? __ldcg(src + i) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < GPER; ++q) {
            const int i = t + GT * q;
            if (i < n) {
                const int j = i / TILE_P, r = i - j * TILE_P;
                tile[r * RS + j] = v[q];
            }
        }
        __syncthreads();
        if (work) {
            float a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) a[q] = 0.f;
            for (int r = g; r < TILE_P; r += 8) {
                const float4 x = *reinterpret_cast<const float4 *>(tile + r * RS + i0);
                const float4 z = *reinterpret_cast<const float4 *>(tile + r * RS + j0);
                const float xv[4] = {x.x, x.y, x.z, x.w}, zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) a[p * 4 + q] = fmaf(xv[p], zv[q], a[p * 4 + q]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) kahan_add(s[q], cs[q], a[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        float v = s[q];
        v += __shfl_xor_sync(FULL, v, 1);
        v += __shfl_xor_sync(FULL, v, 2);
        v += __shfl_xor_sync(FULL, v, 4);
        s[q] = v;
    }
    // each upper entry (i <= j < k) lies in exactly one block, written once
    if (work && g == 0) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + p, j = j0 + q;
                if (i <= j && j < k)
                    part[(size_t)blockIdx.x * (k * (k + 1) / 2) + (i * k - i * (i - 1) / 2 + (j - i))] = s[p * 4 + q];
            }
    }
    const int nm = k * (k + 1) / 2;
    if (!arrive_last(counter)) return;
    // the tile's shared memory is free now: the chunk sums of the reduction
    chunked_sum<GCH>(part, (int)gridDim.x, nm, tot, tile, GT); // rows nm apart (packed k-wide)
    if (t == 0) *counter = 0u;
}

// FP64 right-looking Cholesky G = R^T R (G in W, overwritten) and T = R^{-1}
// by back substitution, one matrix entry per thread (1024 threads); false
// when G is not positive definite (then R = T = I).
__device__ bool wide_cholesky(int k, double *R, double *T, double *W, double *inv)
{
    __shared__ int ok_s;
    const int t = threadIdx.x, i = t / KW, l = t - (t / KW) * KW;
    const bool el = i < k && l < k;
    if (el) R[i * KW + l] = 0.0;
    if (t == 0) ok_s = 1;
    __syncthreads();
    for (int a = 0; a < k; ++a) {
        const double d = W[a * KW + a];
        if (!(d > 0.0)) { // every thread reads the same pivot
            if (t == 0) ok_s = 0;
            break;
        }
        if (t >= a && t < k) {
            const double ri = rsqrt_fp64(d);
            if (t == a) inv[a] = ri;
            R[a * KW + t] = t == a ? dmul(d, ri) : dmul(W[a * KW + t], ri);
        }
        __syncthreads();
        if (el && i > a && l >= i) W[i * KW + l] = dfma(-R[a * KW + i], R[a * KW + l], W[i * KW + l]);
        __syncthreads();
    }
    __syncthreads();
    const bool ok = ok_s != 0;
    if (!ok) {
        if (el) R[i * KW + l] = T[i * KW + l] = i == l ? 1.0 : 0.0;
    } else {
        if (el) W[i * KW + l] = i == l ? 1.0 : 0.0;
        __syncthreads();
        for (int r = k - 1; r >= 0; --r) {
            if (t < k) T[r * KW + t] = dmul(W[r * KW + t], inv[r]);
            __syncthreads();
            if (el && i < r) W[i * KW + l] = dfma(-R[i * KW + r], T[r * KW + l], W[i * KW + l]);
            __syncthreads();
        }
    }
    __syncthreads();
    return ok;
}

// Cholesky-QR from the Gram in tot (packed upper, k-wide rows), one CTA of
// 1024 threads.  frame_end: the end of a frame (y' = R (T_old y) keeps U y,
// the frame's counters and status); else after the initial subspace, an
// import or a rebase (y in the stored basis becomes R y).
__global__ void __launch_bounds__(1024) k_wide_factor(const WideArgs a, int frame_end, int after_rebase)
{
    __shared__ double R[KW * KW], T[KW * KW], W[KW * KW], inv[KW], ty[KW];
    __shared__ float Xh[KW * KW], Xl[KW * KW], X2[KW * KW];
    __shared__ float emax;
    KState *ks = a.ks;
    const int k = a.prm.k;
    const int t = threadIdx.x, i = t / KW, l = t - (t / KW) * KW;
    const bool el = i < k && l < k;
    if (after_rebase && !ks->rebased) return;
    if (frame_end && ks->wskip) {
        if (t == 0) {
            ks->err_flags |= ERR_BADFRAME;
            ks->last_status = -4; // PROST_EBADFRAME
            if (a.status_out) *a.status_out = -4;
            ks->bad_frames += 1;
            ks->frames_since_rebase += 1;
        }
        return;
    }
    if (t == 0) emax = 0.f;
    __syncthreads();
    if (el) {
        const float gv = i <= l ? a.tot[i * k - i * (i - 1) / 2 + (l - i)] : a.tot[l * k - l * (l - 1) / 2 + (i - l)];
        W[i * KW + l] = (double)gv;
        // the bit patterns of non-negative floats order like the floats
        const float e = fabsf(gv - (i == l ? 1.f : 0.f));
        if (e > 0.f) atomicMax(reinterpret_cast<int *>(&emax), __float_as_int(e));
    }
    __syncthreads();
    bool ok = true;
    if (emax <= 1e-5f) {
        // G = I + E close to I (float32 rows re-orthonormalised every frame):
        // R = I + X with X upper triangular, X = upper_half(E - X^T X) by two
        // sweeps from X = upper_half(E) (upper_half halves the diagonal), split
        // as Xh + Xl in FP32; T = R^{-1} = I - X + X^2 - X^3 (the next terms are
        // below 1e-20); both summed in FP64
        const float e = el ? (float)W[t] - (i == l ? 1.f : 0.f) : 0.f; // exact
        Xh[t] = l > i ? e : (l == i ? 0.5f * e : 0.f);
        Xl[t] = 0.f;
        __syncthreads();
        for (int sweep = 0; sweep < 2; ++sweep) {
            float pv = 0.f;
            if (el && l >= i)
                for (int r = 0; r <= i; ++r) {
                    pv = fmaf(Xh[r * KW + i], Xh[r * KW + l], pv);
                    pv = fmaf(Xh[r * KW + i], Xl[r * KW + l], pv);
                    pv = fmaf(Xl[r * KW + i], Xh[r * KW + l], pv);
                }
            __syncthreads();
            if (el) Xl[t] = l > i ? -pv : (l == i ? -0.5f * pv : 0.f);
            __syncthreads();
        }
        float x2 = 0.f;
        if (el && l >= i)
            for (int r = i; r <= l; ++r) x2 = fmaf(Xh[i * KW + r] + Xl[i * KW + r], Xh[r * KW + l] + Xl[r * KW + l], x2);
        X2[t] = x2;
        __syncthreads();
        float x3 = 0.f;
        if (el && l >= i)
            for (int r = i; r <= l; ++r) x3 = fmaf(X2[i * KW + r], Xh[r * KW + l], x3);
        const double xh = (double)Xh[t], xl = (double)Xl[t], id = i == l ? 1.0 : 0.0;
        R[t] = el ? (id + xh) + xl : 0.0;
        T[t] = el ? ((id - xh) - xl) + ((double)x2 - (double)x3) : 0.0;
        __syncthreads();
    } else {
        ok = wide_cholesky(k, R, T, W, inv); // also NaN
    }
    if (t < k) {
        double v = 0.0;
        if (frame_end)
            for (int q = t; q < k; ++q) v = dfma(ks->T[t * KMAX + q], ks->y[q], v);
        else
            v = ks->y[t];
        ty[t] = v;
    }
    __syncthreads(); // every read of the old T and y is done
    if (t < k) {
        double yn = 0.0;
        for (int q = t; q < k; ++q) yn = dfma(R[t * KW + q], ty[q], yn);
        ks->y[t] = yn;
        ks->yf[t] = (float)ty[t];
    }
    if (el) {
        ks->R[i * KMAX + l] = R[i * KW + l];
        ks->T[i * KMAX + l] = T[i * KW + l];
        ks->Tf[i * k + l] = (float)T[i * KW + l];
    }
    if (t == 0) {
        ks->orth_err = emax;
        if (!ok) ks->err_flags |= ERR_NOTSPD;
        if (frame_end) {
            ks->n_fg = (int64_t)a.tot[NWG];
            ks->frame_index += 1;
            ks->frames_since_rebase += 1;
            ks->last_status = ok ? 0 : -6; // PROST_ENOTSPD
            if (a.status_out) *a.status_out = ok ? 0 : -6;
        } else if (!ok) {
            ks->last_status = -6;
        }
    }
}

// u_st T for one stored row (T upper triangular): column j sums i <= j
__device__ __forceinline__ float row_times_t(const float (&u)[KW], const float *sT, int j)
{
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < KW; ++i)
        if (i <= j) s = fmaf(sT[i * KW + j], u[i], s);
    return s;
}

__device__ __forceinline__ void load_t(const KState *ks, int k, float *sT)
{
    for (int i = threadIdx.x; i < KW * KW; i += WT) {
        const int r = i / KW, c = i - (i / KW) * KW;
        sT[i] = (r < k && c < k) ? ks->Tf[r * k + c] : 0.f;
    }
    __syncthreads();
}

// Orthonormal representative U = U_st T, m x k row-major.
__global__ void __launch_bounds__(WT) k_wide_export(const float *U, const KState *ks, float *out, DevParams prm)
{
    __shared__ float sT[KW * KW];
    const int k = prm.k;
    load_t(ks, k, sT);
    const int64_t m = (int64_t)prm.C * prm.P;
    for (int64_t e = (int64_t)blockIdx.x * WT + threadIdx.x; e < m; e += (int64_t)gridDim.x * WT) {
        const int c = (int)(e / prm.P);
        const int64_t q = e - (int64_t)c * prm.P;
        float u[KW];
#pragma unroll
        for (int j = 0; j < KW; ++j) u[j] = j < k ? U[u_off(prm, c, q, j)] : 0.f;
        for (int j = 0; j < k; ++j) out[e * k + j] = row_times_t(u, sT, j);
    }
}

// Rebase: U_st <- U_st T (each stored row u_st becomes T^T u_st), when due.
__global__ void __launch_bounds__(WT) k_wide_rebase(float *U, const KState *ks, DevParams prm, int force)
{
    if (!force && ks->frames_since_rebase < REBASE_EVERY) return;
    __shared__ float sT[KW * KW];
    const int k = prm.k;
    load_t(ks, k, sT);
    const int64_t rows = (int64_t)prm.C * prm.Pp;
    for (int64_t e = (int64_t)blockIdx.x * WT + threadIdx.x; e < rows; e += (int64_t)gridDim.x * WT) {
        const int c = (int)(e / prm.Pp);
        const int64_t q = e - (int64_t)c * prm.Pp;
        float *base = U + u_off(prm, c, q, 0);
        float u[KW];
#pragma unroll
        for (int j = 0; j < KW; ++j) u[j] = j < k ? base[(int64_t)j * TILE_P] : 0.f;
        for (int j = 0; j < k; ++j) base[(int64_t)j * TILE_P] = row_times_t(u, sT, j);
    }
}

// ---- host side -----------------------------------------------------------------

// SMs of the current device (the handle's: its calls run under a device
// guard), looked up once per device; the partial-sum buffers were sized
// from the same count
constexpr int MAX_DEV = 64;
int g_sms[MAX_DEV];

int sms_now()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < MAX_DEV && g_sms[dev] > 0) return g_sms[dev];
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev >= 0 && dev < MAX_DEV) g_sms[dev] = n;
    return n;
}

// CTAs of the row passes (two per SM, at most one per WT rows) and of the
// Gram pass (two per SM, at most one per tile block), at most MAX_CTAS
int row_grid(const DevParams &prm, int sms)
{
    const int64_t need = ((int64_t)prm.C * prm.Pp + WT - 1) / WT;
    const int64_t g = need < 2 * sms ? need : 2 * sms;
    return (int)(g < MAX_CTAS ? g : MAX_CTAS);
}

int gram_grid(const DevParams &prm, int sms)
{
    const int64_t nt = (int64_t)prm.C * prm.npt;
    const int64_t g = nt < 2 * sms ? nt : 2 * sms;
    return (int)(g < MAX_CTAS ? g : MAX_CTAS);
}

WideArgs wide_args(const FrameArgs &fa)
{
    WideArgs w;
    memset(&w, 0, sizeof(w));
    w.U = static_cast<float *>(fa.U);
    w.frame = fa.frame;
    w.frame_pitch = fa.frame_pitch;
    w.labels = fa.labels;
    w.mask_out = fa.mask_out;
    w.bg_out = fa.bg_out;
    w.ks = fa.ks;
    w.tot = fa.partials;
    w.part = fa.partials + TOTF;
    w.counter = fa.counter;
    w.status_out = fa.status_out;
    w.prm = fa.prm;
    return w;
}

#define WCK(launch)                                \
    do {                                           \
        launch;                                    \
        const cudaError_t e_ = cudaGetLastError(); \
        if (e_ != cudaSuccess) return e_;          \
    } while (0)

template <typename FT> cudaError_t frame_t(const WideArgs &w, cudaStream_t s)
{
    const int sms = sms_now();
    const int grid = row_grid(w.prm, sms);
    const int n_cg = w.prm.n_cg;
    static_assert(offsetof(KState, wproj) == offsetof(KState, wskip) + sizeof(int32_t), "flags side by side");
    const cudaError_t e0 = cudaMemsetAsync(&w.ks->wskip, 0, 2 * sizeof(int32_t), s); // wskip, wproj
    if (e0 != cudaSuccess) return e0;
    // each pass's last CTA takes the k-space step that follows it
    for (int pass = 0; pass < n_cg; ++pass) {
        WCK((k_wide_res<FT, 0><<<grid, WT, 0, s>>>(w, pass)));
        WCK((k_wide_res<FT, 1><<<grid, WT, 0, s>>>(w, pass)));
    }
    WCK((k_wide_res<FT, 0><<<grid, WT, 0, s>>>(w, n_cg)));
    // the projection pass returns at once unless the final step asked for it
    WCK((k_wide_res<FT, 2><<<grid, WT, 0, s>>>(w, n_cg)));
    WCK((k_wide_update<FT><<<grid, WT, 0, s>>>(w)));
    WCK((k_wide_gram<<<gram_grid(w.prm, sms), GT, 0, s>>>(w.U, w.ks, w.prm, w.part, w.tot, w.counter, 0)));
    WCK((k_wide_factor<<<1, 1024, 0, s>>>(w, 1, 0)));
    return cudaSuccess;
}

cudaError_t op_frame(const FrameArgs &fa, int frame_dtype, int, cudaStream_t s)
{
    if (fa.prm.ubf16 || fa.prm.k < 1 || fa.prm.k > KW || !fa.counter) return cudaErrorInvalidValue;
    const WideArgs w = wide_args(fa);
    return frame_dtype == PROST_U8 ? frame_t<uint8_t>(w, s) : frame_t<float>(w, s);
}

int op_prepare(int) { return 1; }

cudaError_t op_multi(const FrameArgs *, const int2 *, int, int, cudaStream_t) { return cudaErrorNotSupported; }

cudaError_t op_cluster(const FrameArgs &, int, int, cudaStream_t) { return cudaErrorNotSupported; }

int op_cluster_fit(int, int) { return 0; }

cudaError_t op_gram(const GramArgs &ga, int, cudaStream_t s)
{
    if (ga.prm.ubf16 || ga.prm.k < 1 || ga.prm.k > KW) return cudaErrorInvalidValue;
    WideArgs w;
    memset(&w, 0, sizeof(w));
    w.U = static_cast<float *>(const_cast<void *>(ga.U));
    w.ks = ga.ks;
    w.tot = ga.partials;
    w.part = ga.partials + TOTF;
    w.counter = ga.counter;
    w.prm = ga.prm;
    WCK((k_wide_gram<<<gram_grid(w.prm, sms_now()), GT, 0, s>>>(w.U, w.ks, w.prm, w.part, w.tot, w.counter,
                                                              ga.after_rebase)));
    WCK((k_wide_factor<<<1, 1024, 0, s>>>(w, 0, ga.after_rebase)));
    return cudaSuccess;
}

int blocks_for(int64_t n)
{
    const int64_t b = (n + WT - 1) / WT;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t op_export(const void *U, const KState *ks, float *out, DevParams prm, cudaStream_t s)
{
    WCK((k_wide_export<<<blocks_for((int64_t)prm.C * prm.P), WT, 0, s>>>(static_cast<const float *>(U), ks, out, prm)));
    return cudaSuccess;
}

cudaError_t op_rebase(void *U, KState *ks, DevParams prm, int force, cudaStream_t s)
{
    WCK((k_wide_rebase<<<blocks_for((int64_t)prm.C * prm.Pp), WT, 0, s>>>(static_cast<float *>(U), ks, prm, force)));
    return launch_reset_fold(ks, prm, force, s);
}

int op_gram_occupancy() { return 1; }

#undef WCK

KernelOps make_ops()
{
    KernelOps o;
    memset(&o, 0, sizeof(o));
    o.frame = op_frame;
    o.frame_prepare = op_prepare;
    o.frame_multi = op_multi;
    o.frame_cluster = op_cluster;
    o.cluster_fit = op_cluster_fit;
    o.gram = op_gram;
    o.export_u = op_export;
    o.gram_occupancy = op_gram_occupancy;
    o.rebase = op_rebase;
    o.vw = TILE_P;
    o.tile = TILE_P;
    o.frame_threads = WT;
    return o;
}

const KernelOps g_wide_ops = make_ops();

} // namespace

const KernelOps *wide_ops() { return &g_wide_ops; }

size_t wide_partial_floats(const DevParams &prm, int sms)
{
    const size_t rows = (size_t)row_grid(prm, sms) * (KW + 3);
    const size_t gram = (size_t)gram_grid(prm, sms) * NWG;
    return (size_t)TOTF + (rows > gram ? rows : gram);
}

} // namespace prost
