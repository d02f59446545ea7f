// Streaming form of the frame kernel's passes (k >= 11): 8 warps of up to
// 255 registers per SM, one lane per row, rows staged through shared memory
// by asynchronous copies.
//
// At these k the subspace (373 MB at 1920x1080x3, k = 15) is streamed from
// HBM in every pass, and a lane needs k(k+1)/2 + 2k + 3 sums of its own.
// Rather than many warps with few registers (whose loads in flight are then
// too few to cover HBM latency), each warp keeps STG_D steps of 32 rows in
// flight as 16-byte cp.async copies into its own ring of shared-memory stages
// (no registers held), and one lane processes one row per step with all its
// sums in registers.
//
// Stage layout (floats): column j of the step's 32 rows at 32*j, then the 32
// frame entries and the 32 labels (16-byte aligned).  Lane i reads row i, so
// every shared-memory read is conflict-free.
//
// Two designs were built and measured before this one, and are not kept:
// a bulk-copy (TMA) tile ring fed by one producer, whose per-copy cost in the
// copy engine held it to about half the HBM rate, and two lanes per row with
// 16 warps, which duplicated a third of the work per row.
#pragma once

#include "prost_kernels.cuh"

namespace prost {

constexpr int STG_D = 8;      // steps in flight per warp
constexpr int STG_ROWS = 32;  // rows per step (one per lane)
static_assert(TILE_P % STG_ROWS == 0, "whole steps per tile");

template <int K, typename FT> struct StageCfg {
    static constexpr int F_OFF = STG_ROWS * K;                          // floats
    static constexpr int F_F = STG_ROWS * (int)sizeof(FT) / 4;
    static constexpr int L_OFF = F_OFF + F_F;
    static constexpr int STAGE_F = (L_OFF + STG_ROWS / 4 + 7) / 8 * 8;  // 32-byte multiple
    static constexpr int NCU = K * STG_ROWS * 4 / 16;                   // 16-byte chunks: subspace
    static constexpr int NCF = STG_ROWS * (int)sizeof(FT) / 16;         // frame entries
    static constexpr int NCL = STG_ROWS / 16;                           // labels
    static constexpr int NCH = NCU + NCF + NCL;
    static constexpr int CPL = (NCH + 31) / 32;                         // chunks per lane
    static constexpr int STEPS_PER_TILE = TILE_P / STG_ROWS;
};

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t n = valid ? 16u : 0u; // 0: fill with zeros, read nothing
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This lane's chunks of a step: chunk q is number lane + 32 q of the step.
// kind 0: subspace column (element offset off from the tile's first row),
// 1: frame entries (offset in rows), 2: labels (offset in rows), 3: none.
template <int K, typename FT> struct Chunks {
    using S = StageCfg<K, FT>;
    int kind[S::CPL], off[S::CPL], soff[S::CPL];

    __device__ __forceinline__ explicit Chunks(int lane)
    {
#pragma unroll
        for (int q = 0; q < S::CPL; ++q) {
            const int ch = lane + 32 * q;
            if (ch < S::NCU) {
                const int col = ch / (STG_ROWS / 4), part = ch % (STG_ROWS / 4);
                kind[q] = 0;
                off[q] = col * TILE_P + 4 * part;
                soff[q] = STG_ROWS * col + 4 * part;
            } else if (ch < S::NCU + S::NCF) {
                const int part = ch - S::NCU;
                kind[q] = 1;
                off[q] = part * (16 / (int)sizeof(FT));
                soff[q] = S::F_OFF + 4 * part;
            } else if (ch < S::NCH) {
                const int part = ch - S::NCU - S::NCF;
                kind[q] = 2;
                off[q] = 16 * part;
                soff[q] = S::L_OFF + 4 * part;
            } else {
                kind[q] = 3;
                off[q] = 0;
                soff[q] = 0;
            }
        }
    }

    // rows rs .. rs + 31 of a tile: its subspace block ut, the frame entries
    // and labels of its first pixel (ft, lt), nval rows inside the plane;
    // with_labels false leaves the label slots unwritten
    __device__ __forceinline__ void issue(float *st, const float *ut, const FT *ft, const uint8_t *lt, int rs,
                                          int nval, bool with_labels) const
    {
#pragma unroll
        for (int q = 0; q < S::CPL; ++q) {
            if (kind[q] == 0) {
                cp_async16(st + soff[q], ut + off[q] + rs, true);
            } else if (kind[q] == 1) {
                const bool v = rs + off[q] < nval;
                cp_async16(st + soff[q], v ? (const void *)(ft + rs + off[q]) : (const void *)lt, v);
            } else if (kind[q] == 2 && with_labels) {
                cp_async16(st + soff[q], lt + rs + off[q], true);
            }
        }
    }
};

// One residual pass of this warp (all lanes) over its tiles r0 + warp,
// r0 + warp + NW, ... of the CTA's range: per-lane sums [g_st (K) | (WM)
// U_st^T diag(c) U_st packed | f | |eta|^2 | #non-finite], the standard
// partial-row layout.
template <int K, typename FT, bool WM, int NW, int NP>
__device__ __forceinline__ void stream_residual(const FrameArgs &a, int r0, int nres, const float *yf, float *wbuf,
                                                float (&acc)[NP])
{
    using S = StageCfg<K, FT>;
    constexpr int NM = WM ? K * (K + 1) / 2 : 0;
    constexpr int SPT = S::STEPS_PER_TILE;
    const DevParams &prm = a.prm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float y[K];
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = yf[j];
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;
    const int npt = prm.npt;
    const Chunks<K, FT> ch(lane);
    const int ntile = nres > warp ? (nres - warp + NW - 1) / NW : 0;
    const int nstep = ntile * SPT;

    // issue side: tile iti (plane ic, index in plane itp), step is
    int is = 0, iti = r0 + warp, ic = iti / npt, itp = iti - ic * npt;
    const float *iut = a.U + (int64_t)iti * K * TILE_P;
    const FT *ift = static_cast<const FT *>(a.frame) + (int64_t)ic * a.frame_pitch + (int64_t)itp * TILE_P;
    const uint8_t *ilt = a.labels + (int64_t)itp * TILE_P;
    int inval = (int)min((int64_t)TILE_P, prm.P - (int64_t)itp * TILE_P);
    auto issue_next = [&](int k) {
        if (k < nstep) {
            ch.issue(wbuf + (k % STG_D) * S::STAGE_F, iut, ift, ilt, STG_ROWS * is, inval, true);
            if (++is == SPT && k + 1 < nstep) {
                is = 0;
                iti += NW;
                itp += NW;
                while (itp >= npt) {
                    itp -= npt;
                    ++ic;
                }
                iut = a.U + (int64_t)iti * K * TILE_P;
                ift = static_cast<const FT *>(a.frame) + (int64_t)ic * a.frame_pitch + (int64_t)itp * TILE_P;
                ilt = a.labels + (int64_t)itp * TILE_P;
                inval = (int)min((int64_t)TILE_P, prm.P - (int64_t)itp * TILE_P);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < STG_D - 1; ++k) issue_next(k);

    // consume side: step cs of the tile whose index in its plane is ctp
    int cs = 0, ctp = (r0 + warp) % npt;
    int cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ctp * TILE_P);
    for (int k = 0; k < nstep; ++k) {
        issue_next(k + STG_D - 1);
        cp_async_wait<STG_D - 1>();
        __syncwarp();
        const float *st = wbuf + (k % STG_D) * S::STAGE_F;
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = st[STG_ROWS * j + lane];
        const FT xraw = reinterpret_cast<const FT *>(st + S::F_OFF)[lane];
        const uint8_t lb = reinterpret_cast<const uint8_t *>(st + S::L_OFF)[lane];
        __syncwarp(); // the stage is refilled by a later step's copies
        const bool valid = STG_ROWS * cs + lane < cnval;
        if (++cs == SPT) {
            cs = 0;
            ctp += NW;
            while (ctp >= npt) ctp -= npt;
            cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ctp * TILE_P);
        }
        const float xv = valid ? (float)xraw : 0.f;
        // u . y in four independent partial sums (shorter dependency chain)
        float uq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < K; ++j) uq[j & 3] = fmaf(u[j], y[j], uq[j & 3]);
        const float uy = (uq[0] + uq[1]) + (uq[2] + uq[3]);
        if constexpr (sizeof(FT) == 4) {
            if (valid && !isfinite(xv)) acc[K + NM + 2] += 1.f;
        }
        const float res = valid ? fmaf(xv, sc, -of) - uy : 0.f;
        const float z = fmaf(res, res, mu);
        const float tz = __powf(z, e);
        const float wv = valid ? (lb != 0 ? om : 1.f) : 0.f;
        const float cw = wv * tz;
        acc[K + NM] = fmaf(cw, z, acc[K + NM]);
        const float eta = -pw * cw * res;
        acc[K + NM + 1] = fmaf(eta, eta, acc[K + NM + 1]);
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] = fmaf(eta, u[j], acc[j]);
        if constexpr (WM) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float cu = cw * u[j];
#pragma unroll
                for (int l2 = j; l2 < K; ++l2) acc[K + tri<K>(j, l2)] = fmaf(cu, u[l2], acc[K + tri<K>(j, l2)]);
            }
        }
    }
    cp_async_wait<0>();
}

// k-space vectors of the update pass, held in registers
template <int K> struct UpdVecs {
    float ty[K], tg[K], tv[K], w[K];
};

// Update pass of this warp over its pixel tiles u0 + warp, u0 + warp + NW, ...:
// one step is 32 pixels of one channel; the channels of a pixel group follow
// each other, and the label (max over channels) is written after the last.
// Per-lane sums [Gram of the new stored rows packed | #foreground].
template <int K, typename FT, int NW, int NP>
__device__ __forceinline__ void stream_update(const FrameArgs &a, int u0, int nupt, const UpdVecs<K> &kv, float cm1,
                                             float snp, float yn, bool write, float *wbuf, float (&acc)[NP])
{
    using S = StageCfg<K, FT>;
    constexpr int NM = K * (K + 1) / 2;
    constexpr int SPT = S::STEPS_PER_TILE;
    const DevParams &prm = a.prm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta;
    const float sc = prm.in_scale, of = prm.in_offset;
    const bool pre = prm.mask_pre != 0;
    const int C = prm.C, npt = prm.npt;
    const int64_t cstride = (int64_t)npt * K * TILE_P; // one channel plane of the stored rows
    const Chunks<K, FT> ch(lane);
    const int ntile = nupt > warp ? (nupt - warp + NW - 1) / NW : 0;
    const int nstep = ntile * SPT * C;

    // issue side: pixel tile ipt, step is, channel icc
    int is = 0, icc = 0, ipt = u0 + warp;
    int inval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ipt * TILE_P);
    auto issue_next = [&](int k) {
        if (k < nstep) {
            const float *ut = a.U + icc * cstride + (int64_t)ipt * K * TILE_P;
            const FT *ft = static_cast<const FT *>(a.frame) + (int64_t)icc * a.frame_pitch + (int64_t)ipt * TILE_P;
            const uint8_t *lt = a.labels + (int64_t)ipt * TILE_P;
            ch.issue(wbuf + (k % STG_D) * S::STAGE_F, ut, ft, lt, STG_ROWS * is, inval, icc == 0);
            if (++icc == C) {
                icc = 0;
                if (++is == SPT) {
                    is = 0;
                    ipt += NW;
                    inval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ipt * TILE_P);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < STG_D - 1; ++k) issue_next(k);

    int cs = 0, cc = 0, cpt = u0 + warp;
    int cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)cpt * TILE_P);
    float wv = 0.f, mx = 0.f;
    for (int k = 0; k < nstep; ++k) {
        issue_next(k + STG_D - 1);
        cp_async_wait<STG_D - 1>();
        __syncwarp();
        const float *st = wbuf + (k % STG_D) * S::STAGE_F;
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = st[STG_ROWS * j + lane];
        const FT xraw = reinterpret_cast<const FT *>(st + S::F_OFF)[lane];
        const uint8_t lb = reinterpret_cast<const uint8_t *>(st + S::L_OFF)[lane];
        __syncwarp();
        const int row = STG_ROWS * cs + lane;
        const bool valid = row < cnval;
        const int64_t p = (int64_t)cpt * TILE_P + row;
        if (cc == 0) {
            wv = valid ? (lb ? om : 1.f) : 0.f;
            mx = 0.f;
        }
        const float x = valid ? fmaf((float)xraw, sc, -of) : 0.f;
        float dy[2] = {0.f, 0.f}, dg[2] = {0.f, 0.f}, dv[2] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < K; ++j) {
            dy[j & 1] = fmaf(u[j], kv.ty[j], dy[j & 1]);
            dg[j & 1] = fmaf(u[j], kv.tg[j], dg[j & 1]);
            dv[j & 1] = fmaf(u[j], kv.tv[j], dv[j & 1]);
        }
        const float uy = dy[0] + dy[1], ug = dg[0] + dg[1], uv = dv[0] + dv[1];
        const float res = valid ? x - uy : 0.f;
        const float z = fmaf(res, res, mu);
        const float tz = __powf(z, e);
        const float eta = -pw * wv * tz * res;
        // u <- u + ((cos(theta) - 1) u^T v - sin(theta) pi(eta)_e / |pi(eta)|) v
        const float gam = valid ? fmaf(cm1, uv, -snp * (eta - ug)) : 0.f;
        const float rn = pre ? res : fmaf(-gam, yn, res);
        if (valid) {
            mx = fmaxf(mx, fabsf(rn));
            if (write && a.bg_out) a.bg_out[(int64_t)cc * prm.P + p] = x - rn + of;
        }
        // stored row u_st + gamma R^T v, its Gram, written back
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = fmaf(gam, kv.w[j], u[j]);
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(u[j], u[l2], acc[tri<K>(j, l2)]);
        if (write) {
            float *ub = a.U + cc * cstride + (int64_t)cpt * K * TILE_P + row;
#pragma unroll
            for (int j = 0; j < K; ++j) ub[j * TILE_P] = u[j];
        }
        if (++cc == C) { // the pixel group's last channel: its label
            cc = 0;
            const uint8_t nl = (valid && mx >= dl) ? 1 : 0;
            acc[NM] += (float)nl;
            if (write) {
                a.labels[p] = nl;
                if (a.mask_out && valid) a.mask_out[p] = nl;
            }
            if (++cs == SPT) {
                cs = 0;
                cpt += NW;
                cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)cpt * TILE_P);
            }
        }
    }
    cp_async_wait<0>();
}

} // namespace prost
