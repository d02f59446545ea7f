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

template <int K, typename FT, typename UT> struct StageCfg {
    // bfloat16 storage: the products U^T diag(c) U and the Gram on tensor
    // cores (mma.sync m16n8k16, bf16 operands, FP32 accumulation); the stage
    // then holds 16 columns (zero beyond K) 80 bytes apart, which puts the 8
    // rows of every ldmatrix in distinct banks
    static constexpr bool TC = sizeof(UT) == 2;
    static constexpr int CS = TC ? 40 : STG_ROWS;                         // elements between columns
    static constexpr int UCOL = TC ? 16 : K;                             // columns held
    static constexpr int UB = UCOL * CS * (int)sizeof(UT);               // bytes of the subspace block
    static constexpr int F_OFF = UB;                                     // byte offsets
    static constexpr int L_OFF = F_OFF + STG_ROWS * (int)sizeof(FT);
    static constexpr int STAGE_B = (L_OFF + STG_ROWS + 127) / 128 * 128;
    static constexpr int CPC = STG_ROWS * (int)sizeof(UT) / 16;          // chunks per column
    static constexpr int NCU = K * CPC;                                  // 16-byte chunks: subspace
    static constexpr int NCF = STG_ROWS * (int)sizeof(FT) / 16;          // frame entries
    static constexpr int NCL = STG_ROWS / 16;                            // labels
    static constexpr int NCH = NCU + NCF + NCL;
    static constexpr int STEPS_PER_TILE = TILE_P / STG_ROWS;
    // per-warp tensor-core scratch after the stages: one row-major 32 x 16
    // bf16 tile (48-byte rows) and the warp's 16 x 16 FP32 result
    static constexpr int BT_ROW = 24;                                    // bf16 elements per tile row
    static constexpr int BT_B = STG_ROWS * BT_ROW * 2;
    static constexpr int RES_B = BT_B;                                   // offset of the result
    static constexpr int SCR_B = TC ? BT_B + 16 * 16 * 4 : 0;
    // steps in flight per warp: 8 (one tile ahead) with 8 warps per SM, 4
    // with bfloat16 storage, whose 16 warps per SM hide the latency instead
    // (6 measured no faster)
    static constexpr int D = TC ? 4 : STG_D;
    static constexpr int WARP_B = D * STAGE_B + SCR_B;
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

// ---- tensor-core helpers (bfloat16 storage) -----------------------------------

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p))
                 : "memory");
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p))
                 : "memory");
}
// d += a b for a 16 x 16 bf16 A (row-major) and a 16 x 8 bf16 B (column
// fragments), FP32 accumulation
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
// this lane's row (16 values, zero beyond K) as one row of a 48-byte-row tile
template <int K> __device__ __forceinline__ void store_tile_row(unsigned char *tile, const uint32_t (&w)[8])
{
    uint4 *row = reinterpret_cast<uint4 *>(tile + (threadIdx.x & 31) * 48);
    row[0] = make_uint4(w[0], w[1], w[2], w[3]);
    row[1] = make_uint4(w[4], w[5], w[6], w[7]);
}
// the rows of a warp's 16 x 16 mma result (two n-tiles) into a 16 x 16 array
__device__ __forceinline__ void store_result(float *res, const float (&d0)[4], const float (&d1)[4])
{
    const int l = threadIdx.x & 31, g = l >> 2, t = l & 3;
    res[g * 16 + 2 * t] = d0[0];
    res[g * 16 + 2 * t + 1] = d0[1];
    res[(g + 8) * 16 + 2 * t] = d0[2];
    res[(g + 8) * 16 + 2 * t + 1] = d0[3];
    res[g * 16 + 8 + 2 * t] = d1[0];
    res[g * 16 + 8 + 2 * t + 1] = d1[1];
    res[(g + 8) * 16 + 8 + 2 * t] = d1[2];
    res[(g + 8) * 16 + 8 + 2 * t + 1] = d1[3];
}

// This lane's chunks of a step.  Chunk number lane + 32 q of the step's
// subspace block is column (lane / CPC) + q (32 / CPC) at row part
// lane % CPC, so for the NQU whole rounds one base pointer per lane serves
// and round q is a fixed offset away (immediate operands, no branches); the
// last round mixes the remaining subspace chunks, the frame entries and the
// labels.
template <int K, typename FT, typename UT> struct Chunks {
    using S = StageCfg<K, FT, UT>;
    static constexpr int NQU = S::NCU / 32;                    // whole rounds of subspace chunks
    static constexpr int TR = (S::NCH - 32 * NQU + 31) / 32;   // rounds after them (1 or 2)
    static constexpr int QCOL = 32 / S::CPC;                   // columns per round
    static constexpr int RPC = 16 / (int)sizeof(UT);           // rows per subspace chunk
    static constexpr int QB = QCOL * S::CS * (int)sizeof(UT);  // stage bytes between rounds
    int uoff;      // element offset of this lane's subspace chunk in round 0
    int soff;      // byte offset in the stage
    int tkind[TR]; // later rounds: 0 subspace, 1 frame, 2 labels, 3 none
    int toff[TR];  // later rounds: row offset (frame, labels) of this lane's chunk
    int tsoff[TR]; // later rounds: byte offset in the stage

    __device__ __forceinline__ explicit Chunks(int lane)
    {
        uoff = (lane / S::CPC) * TILE_P + (lane % S::CPC) * RPC;
        soff = (lane / S::CPC) * S::CS * (int)sizeof(UT) + 16 * (lane % S::CPC);
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int ch = 32 * (NQU + r) + lane;
            tsoff[r] = 0;
            toff[r] = 0;
            if (ch < S::NCU) {
                tkind[r] = 0;
            } else if (ch < S::NCU + S::NCF) {
                tkind[r] = 1;
                toff[r] = (ch - S::NCU) * (16 / (int)sizeof(FT));
                tsoff[r] = S::F_OFF + 16 * (ch - S::NCU);
            } else if (ch < S::NCH) {
                tkind[r] = 2;
                toff[r] = 16 * (ch - S::NCU - S::NCF);
                tsoff[r] = S::L_OFF + 16 * (ch - S::NCU - S::NCF);
            } else {
                tkind[r] = 3;
            }
        }
    }

    // rows rs .. rs + 31 of a tile: its subspace block ut, the frame entries
    // and labels of its first pixel (ft, lt), nval rows inside the plane;
    // with_labels false leaves the label slots unwritten
    __device__ __forceinline__ void issue(unsigned char *st, const UT *ut, const FT *ft, const uint8_t *lt, int rs,
                                          int nval, bool with_labels) const
    {
        const UT *src = ut + uoff + rs;
        unsigned char *dst = st + soff;
#pragma unroll
        for (int q = 0; q < NQU; ++q) cp_async16(dst + q * QB, src + q * QCOL * TILE_P, true);
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (tkind[r] == 0) {
                cp_async16(dst + (NQU + r) * QB, src + (NQU + r) * QCOL * TILE_P, true);
            } else if (tkind[r] == 1) {
                const bool v = rs + toff[r] < nval;
                cp_async16(st + tsoff[r], v ? (const void *)(ft + rs + toff[r]) : (const void *)lt, v);
            } else if (tkind[r] == 2 && with_labels) {
                cp_async16(st + tsoff[r], lt + rs + toff[r], true);
            }
        }
    }
};

// One residual pass of this warp (all lanes) over its tiles r0 + warp,
// r0 + warp + NW, ... of the CTA's range: per-lane sums [g_st (K) | (WM)
// U_st^T diag(c) U_st packed | f | |eta|^2 | #non-finite], the standard
// partial-row layout; with bfloat16 storage the products U_st^T diag(c) U_st
// are formed on tensor cores instead (the warp's 16 x 16 result into its
// scratch).  With S::D = 8 = steps per tile + 1 the copies run exactly one
// tile ahead (step s of tile t + 1 is issued while step s of tile t is
// consumed: one pointer update per tile, the steps unrolled); otherwise a
// general pipeline keeps S::D - 1 steps in flight.
//
// PJ: the explicit projection pass instead, the one sum acc[0] of
// (eta_e - u_st,e^T tg)^2 = |pi(eta)|^2 with tg = T g (Eq. gproject).
template <int K, typename FT, typename UT, bool WM, int NW, int NP, bool PJ = false>
__device__ __forceinline__ void stream_residual(const FrameArgs &a, int r0, int nres, const float *yf,
                                                unsigned char *wbuf, float (&acc)[NP], const float *tgv = nullptr)
{
    static_assert(!(PJ && WM), "the projection pass forms no products");
    using S = StageCfg<K, FT, UT>;
    constexpr int NM = WM ? K * (K + 1) / 2 : 0;
    constexpr int SPT = S::STEPS_PER_TILE;
    constexpr int D = S::D;
    constexpr bool TCM = S::TC && WM;
    unsigned char *btile = wbuf + D * S::STAGE_B;
    float dm0[4] = {0.f, 0.f, 0.f, 0.f}, dm1[4] = {0.f, 0.f, 0.f, 0.f};
    const DevParams &prm = a.prm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (S::TC) { // zero the padded columns K .. 15 of every stage
        constexpr int per = (16 - K) * S::CS / 2;
        for (int i = lane; i < D * per; i += 32) {
            const int st = i / per, w = i - st * per;
            reinterpret_cast<uint32_t *>(wbuf + st * S::STAGE_B + K * S::CS * 2)[w] = 0u;
        }
        __syncwarp();
    }
    float y[K], tg[PJ ? K : 1];
#pragma unroll
    for (int j = 0; j < K; ++j) y[j] = yf[j];
    if constexpr (PJ) {
#pragma unroll
        for (int j = 0; j < K; ++j) tg[j] = tgv[j];
    }
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega;
    const float sc = prm.in_scale, of = prm.in_offset;
    const int npt = prm.npt;
    const Chunks<K, FT, UT> ch(lane);
    const UT *U = static_cast<const UT *>(a.U);
    const int ntile = nres > warp ? (nres - warp + NW - 1) / NW : 0;

    // one step: the row `lane` of the 32 rows staged at st
    auto step_body = [&](const unsigned char *st, bool valid) {
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = ld_u(reinterpret_cast<const UT *>(st) + S::CS * j + lane);
        const FT xraw = reinterpret_cast<const FT *>(st + S::F_OFF)[lane];
        const uint8_t lb = st[S::L_OFF + lane];
        if constexpr (!TCM) __syncwarp(); // the stage is refilled by a later step's copies
        const float xv = valid ? (float)xraw : 0.f;
        // u . y in four independent partial sums (shorter dependency chain)
        float uq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < K; ++j) uq[j & 3] = fmaf(u[j], y[j], uq[j & 3]);
        const float uy = (uq[0] + uq[1]) + (uq[2] + uq[3]);
        if constexpr (PJ) {
            const float res = valid ? fmaf(xv, sc, -of) - uy : 0.f;
            const float z = fmaf(res, res, mu);
            const float wv = valid ? (lb != 0 ? om : 1.f) : 0.f;
            const float eta = -pw * (wv * __powf(z, e)) * res;
            float gq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < K; ++j) gq[j & 3] = fmaf(u[j], tg[j], gq[j & 3]);
            const float pe = valid ? eta - ((gq[0] + gq[1]) + (gq[2] + gq[3])) : 0.f;
            acc[0] = fmaf(pe, pe, acc[0]);
        } else {
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
        if constexpr (TCM) {
            // B = diag(c) U of the step as a row-major bf16 tile (M feeds only
            // the CG line step; the rounding of c u averages out over the rows),
            // A = the stage itself (columns x rows)
            uint32_t wb[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                wb[q] = pack_bf16(2 * q < K ? cw * u[2 * q] : 0.f, 2 * q + 1 < K ? cw * u[2 * q + 1] : 0.f);
            store_tile_row<K>(btile, wb);
            __syncwarp();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t am[4], bm[4];
                ldsm_x4(am, st + ((lane & 7) + 8 * ((lane >> 3) & 1)) * (S::CS * 2) + (16 * ks + 8 * (lane >> 4)) * 2);
                ldsm_x4_t(bm, btile + (16 * ks + (lane & 7) + 8 * ((lane >> 3) & 1)) * 48 + 8 * (lane >> 4) * 2);
                mma_bf16(dm0, am, bm[0], bm[1]);
                mma_bf16(dm1, am, bm[2], bm[3]);
            }
            __syncwarp(); // the tile and the stage are rewritten later
        } else if constexpr (WM) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float cu = cw * u[j];
#pragma unroll
                for (int l2 = j; l2 < K; ++l2) acc[K + tri<K>(j, l2)] = fmaf(cu, u[l2], acc[K + tri<K>(j, l2)]);
            }
        }
        }
    };

    // a tile of this warp: subspace block, frame and label rows, rows in plane
    struct Tile {
        const UT *ut;
        const FT *ft;
        const uint8_t *lt;
        int nval;
    };
    int ti = r0 + warp, tc = ti / npt, tp = ti - tc * npt; // next tile to issue
    auto make_tile = [&]() {
        Tile t;
        t.ut = U + (int64_t)ti * K * TILE_P;
        t.ft = static_cast<const FT *>(a.frame) + (int64_t)tc * a.frame_pitch + (int64_t)tp * TILE_P;
        t.lt = a.labels + (int64_t)tp * TILE_P;
        t.nval = (int)min((int64_t)TILE_P, prm.P - (int64_t)tp * TILE_P);
        ti += NW;
        tp += NW;
        while (tp >= npt) {
            tp -= npt;
            ++tc;
        }
        return t;
    };

    if constexpr (D == SPT + 1) {
        Tile nxt = make_tile(), cur;
        if (ntile > 0) {
#pragma unroll
            for (int s = 0; s < SPT; ++s) {
                ch.issue(wbuf + s * S::STAGE_B, nxt.ut, nxt.ft, nxt.lt, STG_ROWS * s, nxt.nval, true);
                cp_async_commit();
            }
        }
        for (int t = 0; t < ntile; ++t) {
            cur = nxt;
            const bool more = t + 1 < ntile;
            if (more) nxt = make_tile();
            const int kbase = SPT * t;
#pragma unroll
            for (int s = 0; s < SPT; ++s) {
                const int k = kbase + s;
                if (more)
                    ch.issue(wbuf + ((k + SPT) & (D - 1)) * S::STAGE_B, nxt.ut, nxt.ft, nxt.lt, STG_ROWS * s,
                             nxt.nval, true);
                cp_async_commit();
                cp_async_wait<D - 1>();
                __syncwarp();
                step_body(wbuf + (k & (D - 1)) * S::STAGE_B, STG_ROWS * s + lane < cur.nval);
            }
        }
    } else {
        // general pipeline: issue position (tile it, step is), D - 1 steps ahead
        const int nstep = ntile * SPT;
        Tile it = make_tile();
        int is = 0;
        auto issue_next = [&](int k) {
            if (k < nstep) {
                ch.issue(wbuf + (k % D) * S::STAGE_B, it.ut, it.ft, it.lt, STG_ROWS * is, it.nval, true);
                if (++is == SPT && k + 1 < nstep) {
                    is = 0;
                    it = make_tile();
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int k = 0; k < D - 1; ++k) issue_next(k);
        int cs = 0, ctp = (r0 + warp) % npt;
        int cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ctp * TILE_P);
        for (int k = 0; k < nstep; ++k) {
            issue_next(k + D - 1);
            cp_async_wait<D - 1>();
            __syncwarp();
            step_body(wbuf + (k % D) * S::STAGE_B, STG_ROWS * cs + lane < cnval);
            if (++cs == SPT) {
                cs = 0;
                ctp += NW;
                while (ctp >= npt) ctp -= npt;
                cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ctp * TILE_P);
            }
        }
    }
    cp_async_wait<0>();
    if constexpr (TCM) store_result(reinterpret_cast<float *>(btile + S::RES_B), dm0, dm1);
}

// k-space vectors of the update pass, held in registers
template <int K> struct UpdVecs {
    float ty[K], tg[K], tv[K], w[K];
};

// Update pass of this warp over its pixel tiles u0 + warp, u0 + warp + NW, ...:
// one step is 32 pixels of one channel; the channels of a pixel group follow
// each other, and the label (max over channels) is written after the last.
// Per-lane sums [Gram of the new stored rows packed | #foreground].
template <int K, typename FT, typename UT, int NW, int NP>
__device__ __forceinline__ void stream_update(const FrameArgs &a, int u0, int nupt, const UpdVecs<K> &kv, float cm1,
                                             float snp, float yn, bool write, uint32_t sr_key, unsigned char *wbuf,
                                             float (&acc)[NP])
{
    using S = StageCfg<K, FT, UT>;
    constexpr int NM = K * (K + 1) / 2;
    constexpr int SPT = S::STEPS_PER_TILE;
    // bfloat16 storage: the Gram of the new rows on tensor cores (exact bf16
    // products, FP32 accumulation), the warp's 16 x 16 result into its scratch
    constexpr bool TC = S::TC;
    unsigned char *gtile = wbuf + S::D * S::STAGE_B; // the new rows, one per lane
    float dg0[4] = {0.f, 0.f, 0.f, 0.f}, dg1[4] = {0.f, 0.f, 0.f, 0.f};
    const DevParams &prm = a.prm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float mu = prm.mu, e = prm.e, pw = prm.p, om = prm.omega, dl = prm.delta;
    const float sc = prm.in_scale, of = prm.in_offset;
    const bool pre = prm.mask_pre != 0;
    const int C = prm.C, npt = prm.npt;
    const int64_t cstride = (int64_t)npt * K * TILE_P; // one channel plane of the stored rows
    const Chunks<K, FT, UT> ch(lane);
    UT *U = static_cast<UT *>(a.U);
    const int ntile = nupt > warp ? (nupt - warp + NW - 1) / NW : 0;
    const int nstep = ntile * SPT * C;

    // issue side: pixel tile ipt, step is, channel icc
    int is = 0, icc = 0, ipt = u0 + warp;
    int inval = (int)min((int64_t)TILE_P, prm.P - (int64_t)ipt * TILE_P);
    auto issue_next = [&](int k) {
        if (k < nstep) {
            const UT *ut = U + icc * cstride + (int64_t)ipt * K * TILE_P;
            const FT *ft = static_cast<const FT *>(a.frame) + (int64_t)icc * a.frame_pitch + (int64_t)ipt * TILE_P;
            const uint8_t *lt = a.labels + (int64_t)ipt * TILE_P;
            ch.issue(wbuf + (k % S::D) * S::STAGE_B, ut, ft, lt, STG_ROWS * is, inval, icc == 0);
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
    for (int k = 0; k < S::D - 1; ++k) issue_next(k);

    int cs = 0, cc = 0, cpt = u0 + warp;
    int cnval = (int)min((int64_t)TILE_P, prm.P - (int64_t)cpt * TILE_P);
    float wv = 0.f, mx = 0.f;
    for (int k = 0; k < nstep; ++k) {
        issue_next(k + S::D - 1);
        cp_async_wait<S::D - 1>();
        __syncwarp();
        const unsigned char *st = wbuf + (k % S::D) * S::STAGE_B;
        float u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = ld_u(reinterpret_cast<const UT *>(st) + S::CS * j + lane);
        const FT xraw = reinterpret_cast<const FT *>(st + S::F_OFF)[lane];
        const uint8_t lb = st[S::L_OFF + lane];
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
        // stored row u_st + gamma R^T v, its Gram, written back; a bfloat16
        // row is rounded stochastically first (round to nearest would drop
        // the per-frame updates that are smaller than half an ulp) and its
        // Gram taken of the stored values
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = fmaf(gam, kv.w[j], u[j]);
        if constexpr (sizeof(UT) == 2) {
            // one hash per stored row, then the 32-bit linear congruential
            // generator of Press et al. (Numerical Recipes, 1664525 x +
            // 1013904223 mod 2^32) per entry, its high 16 bits as the noise
            uint32_t rk = pcg_hash(sr_key ^ (uint32_t)(cc * prm.Pp + p));
#pragma unroll
            for (int j = 0; j < K; ++j) {
                rk = rk * 1664525u + 1013904223u;
                u[j] = round_bf16_sr(u[j], rk >> 16);
            }
        }
        if constexpr (TC) {
            // the rounded rows are bf16 values: their products are exact
            uint32_t wr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                wr[q] = pack_bf16(2 * q < K ? u[2 * q] : 0.f, 2 * q + 1 < K ? u[2 * q + 1] : 0.f);
            store_tile_row<K>(gtile, wr);
            __syncwarp();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t am[4], bm[4];
                ldsm_x4_t(am, gtile + (16 * ks + (lane & 7) + 8 * (lane >> 4)) * 48 + 8 * ((lane >> 3) & 1) * 2);
                ldsm_x4_t(bm, gtile + (16 * ks + (lane & 7) + 8 * ((lane >> 3) & 1)) * 48 + 8 * (lane >> 4) * 2);
                mma_bf16(dg0, am, bm[0], bm[1]);
                mma_bf16(dg1, am, bm[2], bm[3]);
            }
            __syncwarp(); // the tile is rewritten by the next step
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int l2 = j; l2 < K; ++l2) acc[tri<K>(j, l2)] = fmaf(u[j], u[l2], acc[tri<K>(j, l2)]);
        }
        if (write) {
            UT *ub = U + cc * cstride + (int64_t)cpt * K * TILE_P + row;
#pragma unroll
            for (int j = 0; j < K; ++j) st_u(ub + j * TILE_P, u[j]); // exact for a rounded bfloat16 value
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
    if constexpr (TC) store_result(reinterpret_cast<float *>(gtile + S::RES_B), dg0, dg1);
}

} // namespace prost
