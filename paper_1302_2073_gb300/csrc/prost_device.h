// Internal definitions shared by the kernels and the host side of libprost.
// Not part of the public ABI (see include/prost.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace prost {

constexpr int KMAX = 16;     // largest subspace dimension with a compiled kernel set
constexpr int CGMAX = 32;    // largest number of CG iterations per frame
constexpr int THREADS = 256; // threads per CTA of every per-pixel kernel

// Device-resident k-space state of one stream.  The stored subspace U_st is
// kept in float32; its orthonormal representative is U = U_st T with
// T = R^{-1}, U_st^T U_st = R^T R (Cholesky-QR folded into the next frame).
// All k-space arithmetic is FP64 and is done by one warp of the last CTA of
// each per-pixel pass; the float copies are what the per-pixel passes read.
struct KState {
    double y[KMAX];            // coefficients in the orthonormal basis U
    double g[KMAX];            // gradient of the cost w.r.t. y at the current iterate
    double gprev[KMAX];        // gradient at the previous iterate
    double d[KMAX];            // CG direction
    double R[KMAX * KMAX];     // Cholesky factor of Gram(U_st), row-major upper triangular
    double T[KMAX * KMAX];     // R^{-1}, row-major upper triangular
    float yf[KMAX];            // float(T y): y for the stored rows (residual passes)
    float ye[KMAX];            // float(y)   (Grassmann/label pass)
    float gf[KMAX];            // float(g) at the final y
    float vf[KMAX];            // v = y/|y|  (Eq. svd)
    float Tf[KMAX * KMAX];     // float(T)
    float cm1;                 // cos(theta) - 1
    float sn_pin;              // sin(theta) / |pi(eta)|
    float ynorm;               // |y|
    int32_t do_update;         // Step 2 not degenerate
    int64_t frame_index;       // i of the next frame (step-size rule)
    int32_t skip;              // current frame rejected (non-finite entry)
    uint32_t err_flags;        // sticky until prost_sync: 1 bad frame, 2 not SPD, 4 timeout
    int32_t last_status;       // status of the last frame
    int32_t n_cg_done;
    int64_t bad_frames;
    // statistics of the last frame
    double cost[CGMAX + 1], gnorm[CGMAX + 1], alpha[CGMAX], beta[CGMAX + 1];
    double pi_norm, y_norm, sigma, t, theta, orth_err;
    int32_t updated, pad0;
    int64_t n_fg;
};

constexpr uint32_t ERR_BADFRAME = 1u, ERR_NOTSPD = 2u, ERR_TIMEOUT = 4u;

// Parameters as the kernels use them.
struct DevParams {
    int64_t P;        // pixels per channel plane
    int64_t Pp;       // padded plane stride of the stored subspace (multiple of 64)
    int C;            // channels
    int k;            // subspace dimension
    int n_cg;         // CG iterations per frame
    int mask_pre;     // labels from the subspace before Step 2
    int vec;          // frame planes allow vector loads
    int pad;
    float p, mu, delta, omega, in_scale, in_offset, e; // e = p/2 - 1
    float pad2;
    double pd, t_init, t_min, tau;
};

struct PassArgs {
    const float *U;          // stored subspace, column j of channel c at U + (j*C + c)*Pp
    const void *frame;       // C x P entries (uint8 or float)
    const uint8_t *labels;   // previous labels, Pp bytes
    KState *ks;
    float *partials;         // gridDim.x rows of per-CTA sums
    unsigned int *counter;   // arrival counter of the last-CTA reduction (0 between launches)
    int pass;                // CG iterate index 0..n_cg
    int pad;
    DevParams prm;
};

struct UstepArgs {
    float *U;
    const void *frame;
    uint8_t *labels;         // in: previous labels (weights); out: this frame's labels
    uint8_t *mask_out;       // optional copy of the labels (device, P bytes)
    float *bg_out;           // optional background U y + in_offset (device, m floats)
    KState *ks;
    float *partials;
    unsigned int *counter;
    DevParams prm;
};

struct GramArgs {
    const float *U;
    KState *ks;
    float *partials;
    unsigned int *counter;
    DevParams prm;
};

// Host-side entry points of one compiled kernel set (one per k).
struct KernelOps {
    cudaError_t (*pass)(const PassArgs &, bool with_m, int frame_dtype, int grid, cudaStream_t);
    cudaError_t (*ustep)(const UstepArgs &, int frame_dtype, int grid, cudaStream_t);
    cudaError_t (*gram)(const GramArgs &, int grid, cudaStream_t);
    cudaError_t (*export_u)(const float *U, const KState *ks, float *out, DevParams prm,
                            cudaStream_t);
    // resident CTAs per SM of kernel kind (0 pass+M, 1 pass, 2 ustep, 3 gram)
    int (*occupancy)(int kind, int frame_dtype);
    int vw;  // pixels per thread of the residual passes and the Gram kernel
    int vwu; // pixels per thread of the update pass
};

// kernels without a k template
cudaError_t launch_init_gauss(float *U, DevParams prm, uint64_t seed, cudaStream_t s);
cudaError_t launch_import_u(const float *Urow, float *U, DevParams prm, cudaStream_t s);
cudaError_t launch_import_labels(const uint8_t *src, uint8_t *labels, DevParams prm,
                                 cudaStream_t s);

// per-k kernel sets, filled by the instantiation units
void register_ops_k01_04(const KernelOps **table);
void register_ops_k05_08(const KernelOps **table);
void register_ops_k09_12(const KernelOps **table);
void register_ops_k13_16(const KernelOps **table);

} // namespace prost
