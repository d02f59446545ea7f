// Internal definitions shared by the kernels and the host side of libprost.
// Not part of the public ABI (see include/prost.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace prost {

constexpr int KMAX = 32;     // largest subspace dimension (k-space state arrays are this wide)
constexpr int KFRAME = 16;   // largest k with a compiled single-launch frame kernel set
constexpr int CGMAX = 32;    // largest number of CG iterations per frame
constexpr int THREADS = 256; // threads per CTA of the Gram and layout kernels
constexpr int TILE_P = 224;  // pixels per tile of the stored subspace (16-byte multiple for uint8)

// Cross-CTA reductions (reduce_rows, reduce_cols): rows per unit, one batch
// of loads; floats of the per-unit sums in shared memory.  reduce_cols needs
// ceil(grid / RED_ROWS) * values <= RED_SCR, which the host keeps by capping
// the frame kernel's grid (max_frame_grid).
constexpr int RED_ROWS = 24;
constexpr int RED_SCR = 1280;
__host__ __device__ constexpr int max_frame_grid(int nv) { return RED_SCR / nv * RED_ROWS; }

// The register form of the single-launch frame kernel (rows loaded straight
// into registers) serves k <= KREG; the resident form is its variant.
constexpr int KREG = 10;

// The resident form deals the pixels of a plane to its CTAs in units of
// RES_UNIT pixels (every CTA takes all channels of its pixels).
constexpr int RES_UNIT = 64;
// copies of each CTA's partial values per residual pass in the resident form
constexpr int RES_NREP = 2;
// its cross-CTA sums (reduce_cols_warp): values per warp of a 512-thread CTA
// (the largest partial row, k = 10: 10 + 55 + 3 = 68 <= 5 * 16) and 16-byte
// chunks per lane (grids of at most RES_MAX_GRID = 4 * 32 * RES_CPL CTAs)
constexpr int RES_VPW = 5;
constexpr int RES_CPL = 2;
constexpr int RES_MAX_GRID = 128 * RES_CPL;
__host__ __device__ constexpr size_t res_al16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline int64_t res_units(int64_t P) { return (P + RES_UNIT - 1) / RES_UNIT; }
// pixel pairs per channel of the CTA with the most units
__host__ __device__ inline int res_npair_max(int64_t P, int G)
{
    return (int)((res_units(P) + G - 1) / G) * (RES_UNIT / 2);
}

// Grid-barrier arrivals of every frame-kernel CTA per frame: one per residual
// pass (n_cg + 1), one for the projection pass (made at the end of the frame
// when that pass does not run) and one at the end of the frame.
__host__ __device__ constexpr int frame_arrivals(int n_cg) { return n_cg + 3; }

// The stored rows are moved onto the orthonormal representative (U_st <- U_st
// T, T <- I) after every REBASE_EVERY completed frames.
constexpr uint32_t REBASE_EVERY = 1024;

// Device-resident k-space state of one stream.  The stored subspace U_st is
// kept in float32 or bfloat16; its orthonormal representative is U = U_st T
// with T = R^{-1}, U_st^T U_st = R^T R (Cholesky-QR folded into the next
// frame).  Every CTA of the frame kernel copies y, T y and the factors at the
// start of a frame and runs the k-space steps on its own shared-memory copy;
// the last CTA to finish the frame writes the new state back.
struct KState {
    double y[KMAX];            // coefficients in the orthonormal basis U
    double R[KMAX * KMAX];     // Cholesky factor of Gram(U_st), row-major upper triangular
    double T[KMAX * KMAX];     // R^{-1}, row-major upper triangular
    float yf[KMAX];            // float(T y): y for the stored rows (residual passes)
    float Tf[KMAX * KMAX];     // float(T)
    int64_t frame_index;       // i of the next frame (step-size rule)
    int32_t skip;              // current frame rejected (non-finite entry)
    uint32_t err_flags;        // sticky until prost_sync: 1 bad frame, 2 not SPD, 4 timeout
    int32_t last_status;       // status of the last frame
    int32_t n_cg_done;
    int64_t bad_frames;
    uint32_t frames_since_rebase; // frames that reached the end of the frame kernel since the last rebase
    int32_t rebased;              // the last rebase request ran (else it was not due)
    // statistics of the last frame
    double cost[CGMAX + 1], gnorm[CGMAX + 1], alpha[CGMAX], beta[CGMAX + 1];
    double pi_norm, y_norm, sigma, t, theta, orth_err;
    double eta_norm;           // |eta| at the final y
    int32_t updated;
    int32_t pi_explicit;       // |pi(eta)| came from the explicit projection pass
    int64_t n_fg;
    // %globaltimer (ns): start of the frame, end of each residual pass, end of the frame
    uint64_t phase_ts[CGMAX + 3];
    // %globaltimer (ns), CTA 0: CG pass 1 tiles done, partial row written, grid
    // barrier passed, all rows reduced, CG step done; update-pass rows done,
    // partial row written, arrived; last CTA: rows reduced, factors done
    uint64_t sub_ts[10];
    // k-space vectors of the pass-sequence form (one launch per pass), kept
    // here between its launches: d, the previous g, s = T d, T v, T g,
    // w = R^T v; d^T g, |y|, cos(theta) - 1, sin(theta) / |pi(eta)|
    float wd[KMAX], wgp[KMAX], ws[KMAX], wtv[KMAX], wtg[KMAX], ww[KMAX];
    float wdg, wyn, wcm1, wsnp;
    int32_t wskip;             // the frame was rejected (non-finite entry)
    int32_t wproj;             // the final step asked for the explicit projection pass
};

constexpr uint32_t ERR_BADFRAME = 1u, ERR_NOTSPD = 2u, ERR_TIMEOUT = 4u;

// Parameters as the kernels use them.
// Stored subspace layout (tile-blocked): each channel plane is cut into npt
// tiles of TILE_P pixels; tile (c, pt) is one contiguous block of k columns of
// TILE_P floats, so entry (e = c*P + q, j) sits at
//   ((c*npt + q/TILE_P)*k + j)*TILE_P + q%TILE_P.
// Pixels q in [P, Pp) with Pp = npt*TILE_P are padding rows holding zeros.
struct DevParams {
    int64_t P;        // pixels per channel plane
    int64_t Pp;       // padded plane length npt*TILE_P (also the pitch of staged frames)
    int C;            // channels
    int k;            // subspace dimension
    int n_cg;         // CG iterations per frame
    int mask_pre;     // labels from the subspace before Step 2
    int npt;          // tiles per channel plane
    int ubf16;        // stored subspace in bfloat16 (else float32)
    float p, mu, delta, omega, in_scale, in_offset, e; // e = p/2 - 1
    uint32_t sr_seed; // stochastic rounding of bfloat16 stores (from the handle's seed)
    double pd, t_init, t_min, tau;
};

// offset of entry (channel c, pixel q, column j) of the stored subspace
__host__ __device__ __forceinline__ int64_t u_off(const DevParams &prm, int c, int64_t q, int j)
{
    const int64_t pt = q / TILE_P;
    return (((int64_t)c * prm.npt + pt) * prm.k + j) * TILE_P + (q - pt * TILE_P);
}

struct GramArgs {
    const void *U;    // stored subspace (float32 or bfloat16)
    KState *ks;
    float *partials;
    unsigned int *counter;
    int after_rebase; // 1: only if the rebase just requested ran (ks->rebased)
    DevParams prm;
};

// Grid barrier of the frame kernel: the arrival count only grows.
struct GridBar {
    unsigned long long count; // arrivals since the handle was created
    int abort;                // set by a CTA whose wait gave up
    int pad;
};

struct FrameArgs {
    void *U;                  // stored subspace (tile-blocked, see DevParams; float32 or bfloat16)
    const void *frame;        // channel planes frame_pitch entries apart (uint8 or float)
    uint8_t *labels;          // in: previous labels (weights); out: this frame's labels
    uint8_t *mask_out;        // optional copy of the labels (device, P bytes)
    float *bg_out;            // optional background U y + in_offset (device, m floats)
    KState *ks;
    float *partials;          // 2 buffers, each value-major: value c of CTA b at [c * col_stride + b]
    GridBar *bar;
    unsigned long long bar_base; // bar->count at launch
    int64_t frame_pitch;
    int col_stride;           // entries per value: the grid size rounded up to a multiple of 4
    int grid;                 // CTAs working on this stream (its grid barrier's size)
    // failure-detection tests only (0 = off): at the grid barrier of residual
    // pass stall_at - 1 wait for one arrival more than any launch makes,
    // giving up after stall_limit SM clock cycles
    int stall_at;
    long long stall_limit;
    int32_t *status_out;      // optional (device): the frame's status, as last_status
    unsigned int *counter;    // arrival counter of the pass-sequence form's reductions (zero between launches)
    int res_ns;               // resident form: row slots (items) per CTA in shared memory
    int nframes;              // resident form: frames of the stream in this launch (0 or 1: one)
    int64_t frame_stride;     // entries from one frame of the launch to the next
    DevParams prm;
};

// Host-side entry points of one compiled kernel set (one per k).
struct KernelOps {
    cudaError_t (*frame)(const FrameArgs &, int frame_dtype, int grid, cudaStream_t);
    int (*frame_prepare)(int frame_dtype); // resident frame-kernel CTAs per SM (0: cannot run)
    // several streams in one launch: CTA b works on stream map[b].x as its
    // CTA map[b].y of args[map[b].x].grid (device tables)
    cudaError_t (*frame_multi)(const FrameArgs *args, const int2 *map, int ctas, int frame_dtype, cudaStream_t);
    // the cluster form: one cluster of `grid` CTAs; how many such clusters fit at once
    cudaError_t (*frame_cluster)(const FrameArgs &, int frame_dtype, int grid, cudaStream_t);
    int (*cluster_fit)(int frame_dtype, int grid);
    cudaError_t (*gram)(const GramArgs &, int grid, cudaStream_t);
    cudaError_t (*export_u)(const void *U, const KState *ks, float *out, DevParams prm,
                            cudaStream_t);
    int (*gram_occupancy)();
    // force = 0: only when frames_since_rebase >= REBASE_EVERY (else a no-op)
    cudaError_t (*rebase)(void *U, KState *ks, DevParams prm, int force, cudaStream_t);
    int vw;        // pixels per thread of the Gram kernel
    int tile;      // pixels per tile of the frame kernel
    int frame_threads;
    // the resident form (k <= 10; null otherwise): its plan for P pixels of
    // C channels on `grid` CTAs (the row slots per CTA and the dynamic shared
    // memory; 0 when it cannot run), and its launch
    int (*res_plan)(int frame_dtype, int64_t P, int C, int grid, int *ns, int *smem);
    cudaError_t (*frame_res)(const FrameArgs &, int frame_dtype, int grid, int smem, cudaStream_t);
};

// kernels without a k template
cudaError_t launch_init_gauss(void *U, DevParams prm, uint64_t seed, cudaStream_t s);
cudaError_t launch_import_u(const float *Urow, void *U, DevParams prm, cudaStream_t s);
cudaError_t launch_import_labels(const uint8_t *src, uint8_t *labels, DevParams prm,
                                 cudaStream_t s);
// after a rebase: R = T = I, the stored-row coefficients equal y and the
// rebase counter restarts (force = 0: only when the counter is due)
cudaError_t launch_reset_fold(KState *ks, DevParams prm, int force, cudaStream_t s);

// per-k kernel sets, filled by the instantiation units
void register_ops_k01_02(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k03_04(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k05_06(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k07_08(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k09_10(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k11_12(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k13_14(const KernelOps **f32, const KernelOps **bf16);
void register_ops_k15_16(const KernelOps **f32, const KernelOps **bf16);
// the pass-sequence form (k at run time, 1..KMAX, float32 stored rows) and the
// floats of partial sums it needs (prost_wide.cu)
const KernelOps *wide_ops();
size_t wide_partial_floats(const DevParams &prm, int sms);

} // namespace prost
