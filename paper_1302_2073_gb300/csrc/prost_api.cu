// Host side of the C ABI declared in include/prost.h: argument checking,
// device state, the launch sequence of one frame, copies and checkpoints.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>
#include <string>

#include "prost.h"
#include "prost_device.h"

using namespace prost;

struct prost_handle {
    prost_params prm;
    DevParams dp;
    const KernelOps *ops;
    cudaStream_t stream;
    int device;
    int num_sms;
    int grid_frame, grid_gram;
    int cluster_grid;      // > 0: the frame kernel runs as one cluster of this many CTAs
    int grid_res;          // > 0: the frame kernel runs in the resident form on this many CTAs
    int res_ns, res_smem;  // its row slots per CTA and dynamic shared memory (bytes)
    int wide;              // the passes form (a sequence of ordinary launches per frame)
    void *U;               // stored subspace (C x npt tile blocks of k x TILE_P float32 or bfloat16)
    uint8_t *labels;       // previous labels (Pp bytes)
    KState *ks;
    float *partials;
    unsigned int *counter;
    GridBar *bar;          // grid barrier of the frame kernel
    uint32_t steps_since_rebase; // frame launches since the stored rows were last rebased
    unsigned long long bar_base; // bar->count before the next launch
    void *frame_buf;       // staging of host or unaligned frames (planes Pp entries apart)
    void *many_buf;        // prost_step_many: staging of its frames (grown on demand)
    size_t many_bytes;
    uint8_t *many_mask;    // prost_step_many: device masks of host calls (grown on demand)
    size_t many_mask_bytes;
    float *bg_buf;         // staging of the background for host outputs
    float *u_buf;          // staging of subspaces crossing the ABI from/to host memory
    int32_t *h_word;       // pinned scratch for small device -> host reads
    size_t partial_floats;
    int stall_at;          // armed for the next frame by prost_inject_wait_timeout (0 = off)
    long long stall_limit;
    // pipelined host frames (prost_step_async / prost_wait): two slots, each
    // with device staging of its frame, labels and background, and status words
    cudaStream_t s_in, s_out;     // host-to-device and device-to-host copy streams
    void *af_buf[2];
    uint8_t *am_buf[2];
    void *mf_buf[2];              // prost_step_many_async: each slot's frames and masks,
    uint8_t *mm_buf[2];           // room for mcap[slot] frames (grown on demand)
    int32_t mcap[2];
    float *ab_buf[2];
    int32_t *ast_dev;             // 2 device status words
    int32_t *ast_host;            // 2 pinned status words
    cudaEvent_t ev_in[2], ev_done[2], ev_out[2];
    int a_head, a_count;          // oldest slot in flight, frames in flight
    int a_used[2];                // the slot has carried a frame (its events are recorded)
    int timing;            // record events around every kernel of prost_step()
    int timed_frames;      // traced frames since timing was enabled
    cudaEvent_t ev[CGMAX + 3];
    std::string err;
};

namespace {

std::string g_init_err;
const KernelOps *g_ops[2][KMAX + 1]; // [float32, bfloat16 subspace][k]
std::once_flag g_ops_once;

void load_ops()
{
    std::call_once(g_ops_once, [] {
        for (int i = 0; i <= KMAX; ++i) g_ops[0][i] = g_ops[1][i] = nullptr;
        register_ops_k01_02(g_ops[0], g_ops[1]);
        register_ops_k03_04(g_ops[0], g_ops[1]);
        register_ops_k05_06(g_ops[0], g_ops[1]);
        register_ops_k07_08(g_ops[0], g_ops[1]);
        register_ops_k09_10(g_ops[0], g_ops[1]);
        register_ops_k11_12(g_ops[0], g_ops[1]);
        register_ops_k13_14(g_ops[0], g_ops[1]);
        register_ops_k15_16(g_ops[0], g_ops[1]);
    });
}

// bytes of one stored subspace entry
size_t u_elem_bytes(const DevParams &dp) { return dp.ubf16 ? 2 : 4; }

// restores the caller's current device on scope exit
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define CK(h, call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            return e_ == cudaErrorMemoryAllocation ? PROST_ENOMEM : PROST_ECUDA;      \
        }                                                                             \
    } while (0)

int fail(prost_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

int64_t m_of(const prost_params &p) { return (int64_t)p.channels * p.width * p.height; }

// parameter check; on success fills dp (except vec)
int check_params(const prost_params *prm, DevParams *dp, std::string *why)
{
    if (!prm) { *why = "params is NULL"; return PROST_EINVAL; }
    const prost_params &p = *prm;
    if (p.width <= 0 || p.height <= 0) { *why = "width and height must be positive"; return PROST_EINVAL; }
    if (p.channels < 1 || p.channels > 4) { *why = "channels must be 1..4"; return PROST_EINVAL; }
    const int64_t P = (int64_t)p.width * p.height, m = m_of(p);
    if (m > (int64_t)1 << 30) { *why = "frame too large (m > 2^30)"; return PROST_EINVAL; }
    if (p.k < 1 || p.k > KMAX || (int64_t)p.k > m) { *why = "k must be in 1..min(m, 32)"; return PROST_EINVAL; }
    if (!(p.p > 0.0 && p.p <= 2.0)) { *why = "p must be in (0, 2]"; return PROST_EINVAL; }
    if (!(p.delta > 0.0) || !isfinite(p.delta)) { *why = "delta must be positive"; return PROST_EINVAL; }
    double mu = p.mu;
    if (mu == 0.0) mu = p.delta * p.delta * (1.0 - p.p);  // Eq. (opt_mu2)
    if (!(mu > 0.0) || !isfinite(mu)) { *why = "mu must be positive (mu = 0 selects delta^2 (1-p), which needs p < 1)"; return PROST_EINVAL; }
    if (!(p.omega >= 0.0 && p.omega <= 1.0)) { *why = "omega must be in [0, 1]"; return PROST_EINVAL; }
    if (!(p.t_init > 0.0) || !(p.t_min > 0.0) || !isfinite(p.t_init) || !isfinite(p.t_min)) { *why = "t_init and t_min must be positive"; return PROST_EINVAL; }
    if (p.i_init < 1) { *why = "i_init must be >= 1"; return PROST_EINVAL; }
    if (p.n_cg < 0 || p.n_cg > CGMAX) { *why = "n_cg must be in 0..32"; return PROST_EINVAL; }
    if (!isfinite(p.in_scale) || !isfinite(p.in_offset)) { *why = "in_scale and in_offset must be finite"; return PROST_EINVAL; }
    if (p.frame_dtype != PROST_U8 && p.frame_dtype != PROST_F32) { *why = "frame_dtype must be PROST_U8 or PROST_F32"; return PROST_EINVAL; }
    if (p.u_dtype != PROST_F32 && p.u_dtype != PROST_BF16) { *why = "u_dtype must be PROST_F32 or PROST_BF16"; return PROST_EINVAL; }
    if (p.mask_from != PROST_MASK_POST_UPDATE && p.mask_from != PROST_MASK_PRE_UPDATE) { *why = "mask_from must be 0 or 1"; return PROST_EINVAL; }
    if (p.form != PROST_FORM_AUTO && p.form != PROST_FORM_GRID && p.form != PROST_FORM_CLUSTER && p.form != PROST_FORM_PASSES && p.form != PROST_FORM_RESIDENT) { *why = "form must be PROST_FORM_AUTO, PROST_FORM_GRID, PROST_FORM_CLUSTER, PROST_FORM_PASSES or PROST_FORM_RESIDENT"; return PROST_EINVAL; }
    if (p.form == PROST_FORM_RESIDENT && p.k > KREG) { *why = "the resident form needs k <= 10"; return PROST_EINVAL; }
    const bool passes = p.form == PROST_FORM_PASSES || p.k > KFRAME;
    if (p.k > KFRAME && p.form != PROST_FORM_AUTO && p.form != PROST_FORM_PASSES) { *why = "k > 16 runs in the passes form only (form AUTO or PROST_FORM_PASSES)"; return PROST_EINVAL; }
    if (passes && p.u_dtype != PROST_F32) { *why = "the passes form (every k > 16) stores the subspace in float32 only"; return PROST_EINVAL; }
    if (dp) {
        memset(dp, 0, sizeof(*dp));
        dp->P = P;
        dp->npt = (int)((P + TILE_P - 1) / TILE_P);
        dp->Pp = (int64_t)dp->npt * TILE_P;
        dp->C = p.channels;
        dp->k = p.k;
        dp->n_cg = p.n_cg;
        dp->mask_pre = p.mask_from == PROST_MASK_PRE_UPDATE;
        dp->ubf16 = p.u_dtype == PROST_BF16;
        dp->sr_seed = (uint32_t)(p.seed ^ (p.seed >> 32)) ^ 0x5bd1e995u;
        dp->p = (float)p.p;
        dp->mu = (float)mu;
        dp->delta = (float)p.delta;
        dp->omega = (float)p.omega;
        dp->in_scale = (float)p.in_scale;
        dp->in_offset = (float)p.in_offset;
        dp->e = (float)(0.5 * p.p - 1.0);
        dp->pd = p.p;
        dp->t_init = p.t_init;
        dp->t_min = p.t_min;
        dp->tau = -log(p.t_min / p.t_init) / (double)p.i_init; // Section 3.4
    }
    return PROST_OK;
}

size_t frame_elem_bytes(const prost_params &p) { return p.frame_dtype == PROST_U8 ? 1 : 4; }

// partial rows of the widest reduction: a CG pass has k + k(k+1)/2 + 3 floats
size_t partial_row(int k) { return (size_t)k + (size_t)k * (k + 1) / 2 + 3; }

// entries per value of the frame kernel's value-major partials (16-byte loads)
int col_stride(int grid) { return (grid + 3) / 4 * 4; }

int grid_of(int occ, int sms, int64_t items)
{
    int64_t need = (items + THREADS - 1) / THREADS;
    int64_t g = (int64_t)occ * sms;
    if (need < g) g = need;
    return (int)(g > 0 ? g : 1);
}

void free_state(prost_handle *h)
{
    if (h->U) cudaFree(h->U);
    if (h->labels) cudaFree(h->labels);
    if (h->ks) cudaFree(h->ks);
    if (h->partials) cudaFree(h->partials);
    if (h->counter) cudaFree(h->counter);
    if (h->bar) cudaFree(h->bar);
    if (h->frame_buf) cudaFree(h->frame_buf);
    if (h->bg_buf) cudaFree(h->bg_buf);
    if (h->u_buf) cudaFree(h->u_buf);
    if (h->many_buf) cudaFree(h->many_buf);
    if (h->many_mask) cudaFree(h->many_mask);
    if (h->h_word) cudaFreeHost(h->h_word);
    for (int i = 0; i < 2; ++i) {
        if (h->af_buf[i]) cudaFree(h->af_buf[i]);
        if (h->am_buf[i]) cudaFree(h->am_buf[i]);
        if (h->mf_buf[i]) cudaFree(h->mf_buf[i]);
        if (h->mm_buf[i]) cudaFree(h->mm_buf[i]);
        h->mf_buf[i] = nullptr; h->mm_buf[i] = nullptr; h->mcap[i] = 0;
        if (h->ab_buf[i]) cudaFree(h->ab_buf[i]);
        if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
        if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
        h->af_buf[i] = nullptr; h->am_buf[i] = nullptr; h->ab_buf[i] = nullptr;
        h->ev_in[i] = h->ev_done[i] = h->ev_out[i] = nullptr;
    }
    if (h->ast_dev) cudaFree(h->ast_dev);
    if (h->ast_host) cudaFreeHost(h->ast_host);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    h->ast_dev = nullptr; h->ast_host = nullptr; h->s_in = h->s_out = nullptr;
    for (int i = 0; i < CGMAX + 3; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < CGMAX + 3; ++i) h->ev[i] = nullptr;
    h->U = nullptr; h->labels = nullptr; h->ks = nullptr; h->partials = nullptr;
    h->counter = nullptr; h->frame_buf = nullptr; h->bg_buf = nullptr; h->u_buf = nullptr;
    h->many_buf = nullptr; h->many_bytes = 0; h->many_mask = nullptr; h->many_mask_bytes = 0;
    h->h_word = nullptr; h->bar = nullptr;
}

int run_gram(prost_handle *h, int after_rebase = 0)
{
    GramArgs ga;
    ga.after_rebase = after_rebase;
    ga.U = h->U;
    ga.ks = h->ks;
    ga.partials = h->partials;
    ga.counter = h->counter;
    ga.prm = h->dp;
    CK(h, h->ops->gram(ga, h->grid_gram, h->stream));
    return PROST_OK;
}

// Move the stored rows onto the orthonormal representative (U_st <- U_st T,
// T <- I).  A bfloat16 subspace is rounded in the move, so its Gram and
// Cholesky-QR are taken again of the stored values.
int rebase(prost_handle *h, int force)
{
    CK(h, h->ops->rebase(h->U, h->ks, h->dp, force, h->stream));
    if (h->dp.ubf16) return run_gram(h, force ? 0 : 1);
    return PROST_OK;
}

int read_status(prost_handle *h, int *status)
{
    CK(h, cudaMemcpyAsync(h->h_word, &h->ks->last_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *status = h->h_word[0];
    return PROST_OK;
}

struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    prost_params prm;
    uint64_t u_bytes, ks_bytes, label_bytes;
    uint32_t steps_since_rebase;
    uint32_t pad;
};

} // namespace

extern "C" {

int prost_version(void) { return 102; }

const char *prost_strerror(int code)
{
    switch (code) {
    case PROST_OK: return "ok";
    case PROST_EINVAL: return "invalid argument";
    case PROST_ENOMEM: return "out of memory";
    case PROST_ECUDA: return "CUDA error";
    case PROST_EBADFRAME: return "frame has a non-finite entry";
    case PROST_ETIMEOUT: return "device wait timed out";
    case PROST_ENOTSPD: return "Gram matrix not positive definite";
    default: return "unknown error";
    }
}

const char *prost_last_error(const prost_handle *h) { return h ? h->err.c_str() : g_init_err.c_str(); }

int prost_state_bytes(const prost_params *prm, size_t *bytes)
{
    DevParams dp;
    std::string why;
    int rc = check_params(prm, &dp, &why);
    if (rc) return rc;
    if (!bytes) return PROST_EINVAL;
    size_t b = (size_t)prm->k * dp.C * dp.Pp * u_elem_bytes(dp) + (size_t)dp.Pp + sizeof(KState) +
               sizeof(unsigned int) + sizeof(GridBar) + (size_t)4096 * partial_row(prm->k) * sizeof(float) +
               (size_t)dp.C * dp.Pp * frame_elem_bytes(*prm);
    *bytes = b;
    return PROST_OK;
}

int prost_init(const prost_params *prm, void *stream, prost_handle **out)
{
    if (!out) { g_init_err = "out is NULL"; return PROST_EINVAL; }
    *out = nullptr;
    DevParams dp;
    std::string why;
    int rc = check_params(prm, &dp, &why);
    if (rc) { g_init_err = why; return rc; }
    load_ops();
    const bool wide = prm->form == PROST_FORM_PASSES || prm->k > KFRAME;
    const KernelOps *ops = wide ? wide_ops() : g_ops[prm->u_dtype == PROST_BF16 ? 1 : 0][prm->k];
    if (!ops) { g_init_err = "no kernel set for this k"; return PROST_EINVAL; }

    prost_handle *h = new (std::nothrow) prost_handle();
    if (!h) { g_init_err = "host allocation failed"; return PROST_ENOMEM; }
    h->prm = *prm;
    h->dp = dp;
    h->ops = ops;
    h->wide = wide ? 1 : 0;
    h->stream = (cudaStream_t)stream;
    h->U = nullptr; h->labels = nullptr; h->ks = nullptr; h->partials = nullptr;
    h->counter = nullptr; h->frame_buf = nullptr; h->bg_buf = nullptr; h->u_buf = nullptr;
    h->many_buf = nullptr; h->many_bytes = 0; h->many_mask = nullptr; h->many_mask_bytes = 0;
    h->h_word = nullptr; h->bar = nullptr; h->bar_base = 0;
    h->steps_since_rebase = 0;
    h->stall_at = 0;
    h->stall_limit = 0;
    h->timing = 0;
    h->timed_frames = 0;
    for (int i = 0; i < CGMAX + 3; ++i) h->ev[i] = nullptr;

    auto bail = [&](int code) {
        g_init_err = h->err;
        free_state(h);
        delete h;
        return code;
    };
#define CKI(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return bail(e_ == cudaErrorMemoryAllocation ? PROST_ENOMEM : PROST_ECUDA);     \
        }                                                                                  \
    } while (0)

    CKI(cudaGetDevice(&h->device));
    CKI(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    const int fdt = prm->frame_dtype;
    const int occ = ops->frame_prepare(fdt);
    if (occ < 1) { h->err = "the frame kernel does not fit on this device"; return bail(PROST_ECUDA); }
    if (ops->tile != TILE_P) { h->err = "tile size mismatch"; return bail(PROST_ECUDA); }
    int64_t gf = (int64_t)occ * h->num_sms;
    if (wide) gf = 1;              // the passes form sizes its own launches
    if (gf > dp.npt) gf = dp.npt;  // every CTA gets at least one pixel tile
    // the cross-CTA reduction's unit sums fit its shared scratch
    if (gf > max_frame_grid((int)partial_row(prm->k))) gf = max_frame_grid((int)partial_row(prm->k));
    // the register form's cross-CTA sums take one or two 16-byte chunks per lane
    if (prm->k <= KREG && gf > RES_MAX_GRID) gf = RES_MAX_GRID;
    h->grid_frame = (int)(gf > 0 ? gf : 1);
    h->grid_gram = grid_of(ops->gram_occupancy(), h->num_sms, (int64_t)dp.C * dp.npt * (TILE_P / ops->vw));
    // the cluster form for small subspaces: one cluster of up to 16 CTAs (a
    // power of two, at most one per pixel tile) that fits the device
    h->cluster_grid = 0;
    {
        const size_t ub = (size_t)prm->k * dp.C * dp.Pp * u_elem_bytes(dp);
        if (!wide && (prm->form == PROST_FORM_CLUSTER || (prm->form == PROST_FORM_AUTO && ub <= PROST_CLUSTER_MAX_U_BYTES))) {
            int g = 16;
            while (g > 1 && (g > dp.npt || g > h->grid_frame)) g /= 2;
            while (g >= 1 && ops->cluster_fit(fdt, g) < 1) g /= 2;
            if (g >= 1) h->cluster_grid = g;
            (void)cudaGetLastError(); // a refused cluster query leaves no error behind
            if (!h->cluster_grid && prm->form == PROST_FORM_CLUSTER) {
                h->err = "the cluster form does not fit this device";
                return bail(PROST_EINVAL);
            }
        }
    }
    // the resident form: every CTA keeps its rows in shared memory across the
    // passes of a frame; AUTO takes it when at least half of them fit
    h->grid_res = 0;
    h->res_ns = 0;
    h->res_smem = 0;
    if (!wide && !h->cluster_grid && ops->res_plan &&
        (prm->form == PROST_FORM_AUTO || prm->form == PROST_FORM_RESIDENT)) {
        int64_t g = (int64_t)occ * h->num_sms;
        // every CTA but the end CTA gets at least one unit
        if (g > res_units(dp.P) + 1) g = res_units(dp.P) + 1;
        if (g > max_frame_grid((int)partial_row(prm->k))) g = max_frame_grid((int)partial_row(prm->k));
        if (g > RES_MAX_GRID) g = RES_MAX_GRID; // the chunks of its cross-CTA sums
        int ns = 0, smem = 0;
        if (g >= 2 && ops->res_plan(fdt, dp.P, dp.C, (int)g, &ns, &smem)) {
            const int64_t nim = (int64_t)dp.C * res_npair_max(dp.P, (int)g - 1);
            if (prm->form == PROST_FORM_RESIDENT || 2 * (int64_t)ns >= nim) {
                h->grid_res = (int)g;
                h->res_ns = ns;
                h->res_smem = smem;
            }
        }
        (void)cudaGetLastError(); // a refused plan leaves no error behind
        if (!h->grid_res && prm->form == PROST_FORM_RESIDENT) {
            h->err = "the resident form does not fit this device";
            return bail(PROST_EINVAL);
        }
    }
    // the Gram kernel's rows, or the frame kernel's two value-major buffers
    h->partial_floats = std::max((size_t)h->grid_gram * partial_row(prm->k),
                                 (size_t)2 * col_stride(h->grid_frame) * partial_row(prm->k));
    // the resident form keeps RES_NREP copies of every pass's partial values
    h->partial_floats = std::max(h->partial_floats,
                                 (size_t)2 * RES_NREP * col_stride(h->grid_res) * partial_row(prm->k));
    if (wide) h->partial_floats = wide_partial_floats(dp, h->num_sms);

    CKI(cudaMalloc(&h->U, (size_t)prm->k * dp.C * dp.Pp * u_elem_bytes(dp)));
    CKI(cudaMalloc(&h->labels, (size_t)dp.Pp));
    CKI(cudaMalloc(&h->ks, sizeof(KState)));
    CKI(cudaMalloc(&h->partials, h->partial_floats * sizeof(float)));
    CKI(cudaMalloc(&h->counter, sizeof(unsigned int)));
    CKI(cudaMalloc(&h->bar, sizeof(GridBar)));
    CKI(cudaMalloc(&h->frame_buf, (size_t)dp.C * dp.Pp * frame_elem_bytes(*prm)));
    CKI(cudaMallocHost(&h->h_word, 64));

    CKI(cudaMemsetAsync(h->labels, 0, (size_t)dp.Pp, h->stream));
    CKI(cudaMemsetAsync(h->ks, 0, sizeof(KState), h->stream));
    CKI(cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), h->stream));
    CKI(cudaMemsetAsync(h->bar, 0, sizeof(GridBar), h->stream));
    CKI(cudaMemsetAsync(h->frame_buf, 0, (size_t)dp.C * dp.Pp * frame_elem_bytes(*prm), h->stream));
    CKI(launch_init_gauss(h->U, h->dp, prm->seed, h->stream));
    rc = run_gram(h);
    if (rc) return bail(rc);
    // store the orthonormal factor itself, so that the stored rows start orthonormal
    rc = rebase(h, 1);
    if (rc) return bail(rc);
    int st = 0;
    rc = read_status(h, &st);
    if (rc) return bail(rc);
    if (st != 0) { h->err = "initial subspace not full rank"; return bail(PROST_ENOTSPD); }
#undef CKI
    *out = h;
    return PROST_OK;
}

namespace {

// Enqueue one frame launch on the handle's stream (and the periodic rebase):
// frame planes at fptr, `pitch` entries apart; outputs and status optional.
// nframes > 1 (resident form only): that many frames of the stream in one
// launch, `stride` entries apart, their masks P bytes apart; the caller keeps
// the run inside one rebase period.
int launch_frame(prost_handle *h, const void *fptr, int64_t pitch, uint8_t *mask_dev, float *bg_dev,
                 int32_t *status_dev, int nframes = 1, int64_t stride = 0)
{
    FrameArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.U = h->U;
    fa.frame = fptr;
    fa.labels = h->labels;
    fa.mask_out = mask_dev;
    fa.bg_out = bg_dev;
    fa.ks = h->ks;
    fa.partials = h->partials;
    fa.bar = h->bar;
    fa.bar_base = h->bar_base;
    fa.frame_pitch = pitch;
    const bool cl = h->cluster_grid > 0;
    const bool res = h->grid_res > 0;
    const int grid = cl ? h->cluster_grid : (res ? h->grid_res : h->grid_frame);
    fa.col_stride = col_stride(grid);
    fa.grid = grid;
    fa.stall_at = h->stall_at;
    fa.stall_limit = h->stall_limit;
    fa.status_out = status_dev;
    fa.counter = h->counter;
    fa.res_ns = h->res_ns;
    fa.nframes = nframes;
    fa.frame_stride = stride;
    h->stall_at = 0; // one launch only
    fa.prm = h->dp;
    if (h->timing) CK(h, cudaEventRecord(h->ev[0], h->stream));
    if (cl)
        CK(h, h->ops->frame_cluster(fa, h->prm.frame_dtype, grid, h->stream));
    else if (res)
        CK(h, h->ops->frame_res(fa, h->prm.frame_dtype, grid, h->res_smem, h->stream));
    else
        CK(h, h->ops->frame(fa, h->prm.frame_dtype, grid, h->stream));
    if (h->timing) {
        CK(h, cudaEventRecord(h->ev[1], h->stream));
        h->timed_frames += 1;
    }
    // the grid barrier's arrivals (the cluster form does not use it)
    if (!cl && !h->wide)
        h->bar_base += (unsigned long long)nframes * (unsigned long long)grid *
                       (unsigned long long)frame_arrivals(h->prm.n_cg);
    // The frame kernel updates the stored rows in the stored basis (U = U_st T);
    // every REBASE_EVERY frames the stored rows are moved onto the orthonormal
    // representative so that the conditioning of U_st cannot drift.  The
    // device counts the frames that completed, and the rebase runs only when
    // that count is due, so a refused frame does not shift the rebase.
    h->steps_since_rebase += (uint32_t)nframes;
    if (h->steps_since_rebase >= REBASE_EVERY) {
        const int rc = rebase(h, 0);
        if (rc) return rc;
        h->steps_since_rebase = 0;
    }
    return PROST_OK;
}

} // namespace

int prost_step(prost_handle *h, const void *frame, int on_device, uint8_t *mask_out,
               float *background_out)
{
    if (!h) return PROST_EINVAL;
    if (!frame) return fail(h, PROST_EINVAL, "frame is NULL");
    if (h->a_count > 0) return fail(h, PROST_EINVAL, "prost_step with frames of prost_step_async in flight");
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const int64_t m = m_of(h->prm);
    const size_t eb = frame_elem_bytes(h->prm);
    // The frame kernel copies frame planes with 16-byte bulk copies: a device
    // frame whose planes start on 16-byte boundaries is read in place, any
    // other frame is first staged into a buffer with a padded plane pitch.
    const void *fptr = frame;
    int64_t pitch = dp.P;
    const bool direct = on_device && ((uintptr_t)frame % 16) == 0 && ((size_t)dp.P * eb) % 16 == 0;
    if (!direct) {
        CK(h, cudaMemcpy2DAsync(h->frame_buf, (size_t)dp.Pp * eb, frame, (size_t)dp.P * eb,
                                (size_t)dp.P * eb, (size_t)dp.C,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        fptr = h->frame_buf;
        pitch = dp.Pp;
    }
    float *bg_dev = nullptr;
    if (background_out) {
        if (on_device) {
            bg_dev = background_out;
        } else {
            if (!h->bg_buf) CK(h, cudaMalloc(&h->bg_buf, (size_t)m * sizeof(float)));
            bg_dev = h->bg_buf;
        }
    }
    int rc = launch_frame(h, fptr, pitch, on_device ? mask_out : nullptr, bg_dev, nullptr);
    if (rc) return rc;
    if (on_device) return PROST_OK;
    // host outputs: only a frame that completed writes them
    int st = 0;
    rc = read_status(h, &st);
    if (rc) return rc;
    if (st != PROST_OK && st != PROST_ENOTSPD) return st;
    if (mask_out)
        CK(h, cudaMemcpyAsync(mask_out, h->labels, (size_t)dp.P, cudaMemcpyDeviceToHost, h->stream));
    if (background_out)
        CK(h, cudaMemcpyAsync(background_out, h->bg_buf, (size_t)m * sizeof(float),
                              cudaMemcpyDeviceToHost, h->stream));
    if (mask_out || background_out) CK(h, cudaStreamSynchronize(h->stream));
    return st;
}

int prost_step_many(prost_handle *h, const void *frames, int32_t n, int on_device, uint8_t *masks_out)
{
    if (!h) return PROST_EINVAL;
    if (!frames) return fail(h, PROST_EINVAL, "frames is NULL");
    if (n < 1) return fail(h, PROST_EINVAL, "n must be at least 1");
    if (h->a_count > 0) return fail(h, PROST_EINVAL, "prost_step_many with frames of prost_step_async in flight");
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const size_t eb = frame_elem_bytes(h->prm);
    const size_t fbytes = (size_t)dp.C * dp.P * eb; // one frame as the caller lays it out
    if (h->grid_res == 0) {
        // the other forms: one launch per frame
        for (int32_t i = 0; i < n; ++i) {
            const int rc = prost_step(h, static_cast<const char *>(frames) + (size_t)i * fbytes, on_device,
                                      masks_out ? masks_out + (size_t)i * dp.P : nullptr, nullptr);
            if (rc) return rc;
        }
        return PROST_OK;
    }
    // the resident form: the frames of each rebase period in one launch
    const void *fptr = frames;
    int64_t pitch = dp.P, stride = (int64_t)dp.C * dp.P;
    const bool direct = on_device && ((uintptr_t)frames % 16) == 0 && ((size_t)dp.P * eb) % 16 == 0;
    if (!direct) {
        const size_t need = (size_t)n * dp.C * dp.Pp * eb;
        if (need > h->many_bytes) {
            if (h->many_buf) CK(h, cudaFree(h->many_buf));
            h->many_buf = nullptr;
            h->many_bytes = 0;
            CK(h, cudaMalloc(&h->many_buf, need));
            h->many_bytes = need;
        }
        CK(h, cudaMemcpy2DAsync(h->many_buf, (size_t)dp.Pp * eb, frames, (size_t)dp.P * eb, (size_t)dp.P * eb,
                                (size_t)n * dp.C, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                h->stream));
        fptr = h->many_buf;
        pitch = dp.Pp;
        stride = (int64_t)dp.C * dp.Pp;
    }
    uint8_t *mdev = on_device ? masks_out : nullptr;
    if (!on_device && masks_out) {
        const size_t need = (size_t)n * dp.P;
        if (need > h->many_mask_bytes) {
            if (h->many_mask) CK(h, cudaFree(h->many_mask));
            h->many_mask = nullptr;
            h->many_mask_bytes = 0;
            CK(h, cudaMalloc(&h->many_mask, need));
            h->many_mask_bytes = need;
        }
        mdev = h->many_mask;
    }
    for (int32_t i0 = 0; i0 < n;) {
        int32_t run = n - i0;
        const int64_t left = (int64_t)REBASE_EVERY - (int64_t)h->steps_since_rebase;
        if (left >= 1 && run > left) run = (int32_t)left;
        const int rc = launch_frame(h, static_cast<const char *>(fptr) + (size_t)i0 * stride * eb, pitch,
                                    mdev ? mdev + (size_t)i0 * dp.P : nullptr, nullptr, nullptr, run, stride);
        if (rc) return rc;
        i0 += run;
    }
    if (on_device) return PROST_OK;
    int st = 0;
    int rc = read_status(h, &st);
    if (rc) return rc;
    if (st != PROST_OK && st != PROST_ENOTSPD) return st;
    if (masks_out) {
        CK(h, cudaMemcpyAsync(masks_out, h->many_mask, (size_t)n * dp.P, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return st;
}

namespace {

// The copy streams, events, status words and one-frame buffers of the
// pipelined host calls (created by the first such call on a handle).
int async_setup(prost_handle *h)
{
    if (h->s_in) return PROST_OK;
    const DevParams &dp = h->dp;
    const size_t eb = frame_elem_bytes(h->prm);
    CK(h, cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
    CK(h, cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
    CK(h, cudaMalloc(&h->ast_dev, 2 * sizeof(int32_t)));
    CK(h, cudaMallocHost(&h->ast_host, 2 * sizeof(int32_t)));
    for (int i = 0; i < 2; ++i) {
        CK(h, cudaMalloc(&h->af_buf[i], (size_t)dp.C * dp.Pp * eb));
        CK(h, cudaMalloc(&h->am_buf[i], (size_t)dp.Pp));
        CK(h, cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming));
    }
    return PROST_OK;
}

} // namespace

int prost_step_many_async(prost_handle *h, const void *frames, int32_t n, uint8_t *masks_out)
{
    if (!h) return PROST_EINVAL;
    if (!frames) return fail(h, PROST_EINVAL, "frames is NULL");
    if (n < 1) return fail(h, PROST_EINVAL, "n must be at least 1");
    if (h->a_count >= 2) return fail(h, PROST_EINVAL, "two calls in flight: call prost_wait first");
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const size_t eb = frame_elem_bytes(h->prm);
    int rc = async_setup(h);
    if (rc) return rc;
    const int slot = (h->a_head + h->a_count) & 1;
    if (n > h->mcap[slot]) {
        // the slot's earlier call (two calls ago) must be done with its buffers
        if (h->a_used[slot]) CK(h, cudaEventSynchronize(h->ev_out[slot]));
        if (h->mf_buf[slot]) CK(h, cudaFree(h->mf_buf[slot]));
        if (h->mm_buf[slot]) CK(h, cudaFree(h->mm_buf[slot]));
        h->mf_buf[slot] = nullptr;
        h->mm_buf[slot] = nullptr;
        h->mcap[slot] = 0;
        CK(h, cudaMalloc(&h->mf_buf[slot], (size_t)n * dp.C * dp.Pp * eb));
        CK(h, cudaMalloc(&h->mm_buf[slot], (size_t)n * dp.P));
        h->mcap[slot] = n;
    }
    // as prost_step_async: the copy in waits for the slot's previous kernel,
    // the kernel for the copy in and for the slot's previous copies out
    if (h->a_used[slot]) CK(h, cudaStreamWaitEvent(h->s_in, h->ev_done[slot], 0));
    CK(h, cudaMemcpy2DAsync(h->mf_buf[slot], (size_t)dp.Pp * eb, frames, (size_t)dp.P * eb, (size_t)dp.P * eb,
                            (size_t)n * dp.C, cudaMemcpyHostToDevice, h->s_in));
    CK(h, cudaEventRecord(h->ev_in[slot], h->s_in));
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_in[slot], 0));
    if (h->a_used[slot]) CK(h, cudaStreamWaitEvent(h->stream, h->ev_out[slot], 0));
    const int64_t stride = (int64_t)dp.C * dp.Pp;
    for (int32_t i0 = 0; i0 < n;) {
        int32_t run = 1;
        if (h->grid_res > 0) { // the resident form: the frames of each rebase period in one launch
            run = n - i0;
            const int64_t left = (int64_t)REBASE_EVERY - (int64_t)h->steps_since_rebase;
            if (left >= 1 && run > left) run = (int32_t)left;
        }
        rc = launch_frame(h, static_cast<char *>(h->mf_buf[slot]) + (size_t)i0 * stride * eb, dp.Pp,
                          h->mm_buf[slot] + (size_t)i0 * dp.P, nullptr, h->ast_dev + slot, run, stride);
        if (rc) return rc;
        i0 += run;
    }
    CK(h, cudaEventRecord(h->ev_done[slot], h->stream));
    CK(h, cudaStreamWaitEvent(h->s_out, h->ev_done[slot], 0));
    if (masks_out)
        CK(h, cudaMemcpyAsync(masks_out, h->mm_buf[slot], (size_t)n * dp.P, cudaMemcpyDeviceToHost, h->s_out));
    CK(h, cudaMemcpyAsync(h->ast_host + slot, h->ast_dev + slot, sizeof(int32_t), cudaMemcpyDeviceToHost, h->s_out));
    CK(h, cudaEventRecord(h->ev_out[slot], h->s_out));
    h->a_used[slot] = 1;
    h->a_count += 1;
    return PROST_OK;
}

int prost_step_async(prost_handle *h, const void *frame, uint8_t *mask_out, float *background_out)
{
    if (!h) return PROST_EINVAL;
    if (!frame) return fail(h, PROST_EINVAL, "frame is NULL");
    if (h->a_count >= 2) return fail(h, PROST_EINVAL, "two frames in flight: call prost_wait first");
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const int64_t m = m_of(h->prm);
    const size_t eb = frame_elem_bytes(h->prm);
    {
        const int rs = async_setup(h);
        if (rs) return rs;
    }
    const int slot = (h->a_head + h->a_count) & 1;
    if (background_out && !h->ab_buf[slot]) CK(h, cudaMalloc(&h->ab_buf[slot], (size_t)m * sizeof(float)));
    // the copy in waits until the kernel that last read this slot's frame has
    // finished (it ran two frames ago); the compute stream waits for the copy
    // and for the copies out of this slot's previous outputs
    if (h->a_used[slot]) CK(h, cudaStreamWaitEvent(h->s_in, h->ev_done[slot], 0));
    CK(h, cudaMemcpy2DAsync(h->af_buf[slot], (size_t)dp.Pp * eb, frame, (size_t)dp.P * eb, (size_t)dp.P * eb,
                            (size_t)dp.C, cudaMemcpyHostToDevice, h->s_in));
    CK(h, cudaEventRecord(h->ev_in[slot], h->s_in));
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_in[slot], 0));
    if (h->a_used[slot]) CK(h, cudaStreamWaitEvent(h->stream, h->ev_out[slot], 0));
    int rc = launch_frame(h, h->af_buf[slot], dp.Pp, h->am_buf[slot], background_out ? h->ab_buf[slot] : nullptr,
                          h->ast_dev + slot);
    if (rc) return rc;
    CK(h, cudaEventRecord(h->ev_done[slot], h->stream));
    CK(h, cudaStreamWaitEvent(h->s_out, h->ev_done[slot], 0));
    if (mask_out) CK(h, cudaMemcpyAsync(mask_out, h->am_buf[slot], (size_t)dp.P, cudaMemcpyDeviceToHost, h->s_out));
    if (background_out)
        CK(h, cudaMemcpyAsync(background_out, h->ab_buf[slot], (size_t)m * sizeof(float), cudaMemcpyDeviceToHost,
                              h->s_out));
    CK(h, cudaMemcpyAsync(h->ast_host + slot, h->ast_dev + slot, sizeof(int32_t), cudaMemcpyDeviceToHost, h->s_out));
    CK(h, cudaEventRecord(h->ev_out[slot], h->s_out));
    h->a_used[slot] = 1;
    h->a_count += 1;
    return PROST_OK;
}

int prost_wait(prost_handle *h)
{
    if (!h) return PROST_EINVAL;
    if (h->a_count == 0) return fail(h, PROST_EINVAL, "no call of prost_step_async or prost_step_many_async in flight");
    DeviceGuard dg(h->device);
    const int slot = h->a_head;
    CK(h, cudaEventSynchronize(h->ev_out[slot]));
    h->a_head ^= 1;
    h->a_count -= 1;
    return h->ast_host[slot];
}

int prost_sync(prost_handle *h)
{
    if (!h) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    if (h->s_out) CK(h, cudaStreamSynchronize(h->s_out)); // the copies out of pipelined frames
    CK(h, cudaMemcpyAsync(h->h_word, &h->ks->err_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemsetAsync(&h->ks->err_flags, 0, sizeof(uint32_t), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const uint32_t f = (uint32_t)h->h_word[0];
    if (f & ERR_TIMEOUT) {
        // an aborted frame leaves the grid barrier count unknown: start it
        // afresh; the refused frames did not count towards the next rebase
        CK(h, cudaMemsetAsync(h->bar, 0, sizeof(GridBar), h->stream));
        CK(h, cudaMemcpyAsync(h->h_word, &h->ks->frames_since_rebase, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->bar_base = 0;
        h->steps_since_rebase = (uint32_t)h->h_word[0];
        return PROST_ETIMEOUT;
    }
    if (f & ERR_NOTSPD) return PROST_ENOTSPD;
    if (f & ERR_BADFRAME) return PROST_EBADFRAME;
    return PROST_OK;
}

int prost_inject_barrier_skew(prost_handle *h, int64_t delta)
{
    if (!h) return PROST_EINVAL;
    // a forward skew below the grid size looks like CTAs that already arrived:
    // the launch cannot tell it from a healthy barrier
    if (h->cluster_grid > 0) return fail(h, PROST_EINVAL, "the cluster form has no grid barrier");
    if (h->wide) return fail(h, PROST_EINVAL, "the passes form has no grid barrier");
    if (delta > 0 && delta < (int64_t)(h->grid_res > 0 ? h->grid_res : h->grid_frame))
        return fail(h, PROST_EINVAL, "a forward skew below the grid size is not detectable");
    DeviceGuard dg(h->device);
    GridBar g;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(&g, h->bar, sizeof(GridBar), cudaMemcpyDeviceToHost));
    g.count += (unsigned long long)delta;
    CK(h, cudaMemcpy(h->bar, &g, sizeof(GridBar), cudaMemcpyHostToDevice));
    return PROST_OK;
}

int prost_inject_wait_timeout(prost_handle *h, int32_t pass, int64_t cycles)
{
    if (!h) return PROST_EINVAL;
    if (pass < 0 || pass > h->prm.n_cg) return fail(h, PROST_EINVAL, "pass must be in 0..n_cg");
    if (h->cluster_grid > 0) return fail(h, PROST_EINVAL, "the cluster form has no software barrier to stall");
    if (h->wide) return fail(h, PROST_EINVAL, "the passes form has no grid barrier to stall");
    if (cycles < 1 || cycles > 2000000000ll) return fail(h, PROST_EINVAL, "cycles must be in 1..2e9");
    h->stall_at = pass + 1;
    h->stall_limit = cycles;
    return PROST_OK;
}

int prost_get_subspace(prost_handle *h, float *U_out, double *y_out, int on_device)
{
    if (!h) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    const int64_t m = m_of(h->prm);
    const int k = h->prm.k;
    if (U_out) {
        float *dst = U_out;
        if (!on_device) {
            if (!h->u_buf) CK(h, cudaMalloc(&h->u_buf, (size_t)m * k * sizeof(float)));
            dst = h->u_buf;
        }
        CK(h, h->ops->export_u(h->U, h->ks, dst, h->dp, h->stream));
        if (!on_device)
            CK(h, cudaMemcpyAsync(U_out, h->u_buf, (size_t)m * k * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    if (y_out)
        CK(h, cudaMemcpyAsync(y_out, h->ks->y, (size_t)k * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return PROST_OK;
}

int prost_set_subspace(prost_handle *h, const float *U, const double *y, int on_device)
{
    if (!h) return PROST_EINVAL;
    if (!U) return fail(h, PROST_EINVAL, "U is NULL");
    DeviceGuard dg(h->device);
    const int64_t m = m_of(h->prm);
    const int k = h->prm.k;
    const float *src = U;
    if (!on_device) {
        if (!h->u_buf) CK(h, cudaMalloc(&h->u_buf, (size_t)m * k * sizeof(float)));
        CK(h, cudaMemcpyAsync(h->u_buf, U, (size_t)m * k * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        src = h->u_buf;
    }
    CK(h, launch_import_u(src, h->U, h->dp, h->stream));
    h->steps_since_rebase = 0;
    if (y)
        CK(h, cudaMemcpyAsync(h->ks->y, y, (size_t)k * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    else
        CK(h, cudaMemsetAsync(h->ks->y, 0, (size_t)k * sizeof(double), h->stream));
    int rc = run_gram(h);
    if (rc) return rc;
    int st = 0;
    rc = read_status(h, &st);
    if (rc) return rc;
    if (st == PROST_ENOTSPD) return fail(h, PROST_ENOTSPD, "subspace columns are not linearly independent");
    // store the orthonormal factor itself, so that the stored rows start orthonormal
    rc = rebase(h, 1);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return PROST_OK;
}

int prost_set_labels(prost_handle *h, const uint8_t *labels, int on_device)
{
    if (!h) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    const uint8_t *src = labels;
    if (labels && !on_device) {
        // stage through the frame buffer (at least P bytes)
        CK(h, cudaMemcpyAsync(h->frame_buf, labels, (size_t)h->dp.P, cudaMemcpyHostToDevice, h->stream));
        src = (const uint8_t *)h->frame_buf;
    }
    CK(h, launch_import_labels(src, h->labels, h->dp, h->stream));
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream));
    return PROST_OK;
}

int prost_set_frame_index(prost_handle *h, int64_t i)
{
    if (!h) return PROST_EINVAL;
    if (i < 0) return fail(h, PROST_EINVAL, "frame index must be >= 0");
    DeviceGuard dg(h->device);
    int64_t *w = (int64_t *)h->h_word;
    CK(h, cudaStreamSynchronize(h->stream));
    w[0] = i;
    CK(h, cudaMemcpyAsync(&h->ks->frame_index, w, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PROST_OK;
}

int prost_get_stats(prost_handle *h, prost_stats *out)
{
    if (!h || !out) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    KState ks;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(&ks, h->ks, sizeof(KState), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->frames = ks.frame_index;
    out->bad_frames = ks.bad_frames;
    out->n_cg = ks.n_cg_done;
    out->status = ks.last_status;
    for (int j = 0; j <= CGMAX; ++j) {
        out->cost[j] = ks.cost[j];
        out->gnorm[j] = ks.gnorm[j];
        out->beta[j] = ks.beta[j];
        if (j < CGMAX) out->alpha[j] = ks.alpha[j];
    }
    out->pi_norm = ks.pi_norm;
    out->y_norm = ks.y_norm;
    out->sigma = ks.sigma;
    out->t = ks.t;
    out->theta = ks.theta;
    out->updated = ks.updated;
    out->n_foreground = ks.n_fg;
    out->orth_err = ks.orth_err;
    out->eta_norm = ks.eta_norm;
    out->pi_explicit = ks.pi_explicit;
    out->form = h->wide ? PROST_FORM_PASSES
                        : (h->cluster_grid > 0 ? PROST_FORM_CLUSTER
                                               : (h->grid_res > 0 ? PROST_FORM_RESIDENT : PROST_FORM_GRID));
    return PROST_OK;
}

int prost_get_state(prost_handle *h, void *buf, size_t *len)
{
    if (!h || !len) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const size_t u_bytes = (size_t)dp.k * dp.C * dp.Pp * u_elem_bytes(dp); // the stored layout as is
    const size_t need = sizeof(StateHeader) + u_bytes + sizeof(KState) + (size_t)dp.P;
    if (!buf) { *len = need; return PROST_OK; }
    if (*len < need) return fail(h, PROST_EINVAL, "buffer too small");
    StateHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "PROSTST1", 8);
    hd.version = 4; // 4: the k-space state 32 wide, with the passes form's vectors
    hd.header_bytes = sizeof(StateHeader);
    hd.prm = h->prm;
    hd.u_bytes = u_bytes;
    hd.ks_bytes = sizeof(KState);
    hd.label_bytes = (uint64_t)dp.P;
    hd.steps_since_rebase = h->steps_since_rebase;
    char *b = (char *)buf;
    memcpy(b, &hd, sizeof(hd));
    char *pu = b + sizeof(hd);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(pu, h->U, u_bytes, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(pu + u_bytes, h->ks, sizeof(KState), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(pu + u_bytes + sizeof(KState), h->labels, (size_t)dp.P, cudaMemcpyDeviceToHost));
    *len = need;
    return PROST_OK;
}

int prost_set_state(prost_handle *h, const void *buf, size_t len)
{
    if (!h || !buf) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    const DevParams &dp = h->dp;
    const size_t u_bytes = (size_t)dp.k * dp.C * dp.Pp * u_elem_bytes(dp);
    const size_t need = sizeof(StateHeader) + u_bytes + sizeof(KState) + (size_t)dp.P;
    if (len < sizeof(StateHeader)) return fail(h, PROST_EINVAL, "state buffer too short");
    StateHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "PROSTST1", 8) != 0 || hd.version != 4 || hd.header_bytes != sizeof(StateHeader))
        return fail(h, PROST_EINVAL, "not a prost state buffer of this version");
    prost_params a = hd.prm, b = h->prm;
    a.seed = b.seed = 0;
    if (memcmp(&a, &b, sizeof(prost_params)) != 0)
        return fail(h, PROST_EINVAL, "state was made with other parameters");
    if (len < need || hd.u_bytes != u_bytes || hd.ks_bytes != sizeof(KState) || hd.label_bytes != (uint64_t)dp.P)
        return fail(h, PROST_EINVAL, "state buffer sizes do not match");
    const char *pu = (const char *)buf + sizeof(hd);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->U, pu, u_bytes, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->ks, pu + u_bytes, sizeof(KState), cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->labels, 0, (size_t)dp.Pp));
    CK(h, cudaMemcpy(h->labels, pu + u_bytes + sizeof(KState), (size_t)dp.P, cudaMemcpyHostToDevice));
    h->steps_since_rebase = hd.steps_since_rebase;
    return PROST_OK;
}

int prost_set_timing(prost_handle *h, int enable)
{
    if (!h) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    if (enable && !h->ev[0])
        for (int i = 0; i < CGMAX + 3; ++i) CK(h, cudaEventCreate(&h->ev[i]));
    h->timing = enable ? 1 : 0;
    h->timed_frames = 0;
    return PROST_OK;
}

int prost_get_timing(prost_handle *h, float *ms, int *n)
{
    if (!h || !ms || !n) return PROST_EINVAL;
    if (!h->timing || h->timed_frames == 0) return fail(h, PROST_EINVAL, "no traced frame");
    DeviceGuard dg(h->device);
    const int nl = h->prm.n_cg + 2;
    CK(h, cudaEventSynchronize(h->ev[1]));
    uint64_t ts[CGMAX + 3];
    CK(h, cudaMemcpy(ts, h->ks->phase_ts, sizeof(uint64_t) * (size_t)(nl + 1), cudaMemcpyDeviceToHost));
    for (int j = 0; j < nl; ++j) ms[j] = (float)((double)(ts[j + 1] - ts[j]) * 1e-6);
    *n = nl;
    return PROST_OK;
}

int prost_get_trace(prost_handle *h, uint64_t *ts)
{
    if (!h || !ts) return PROST_EINVAL;
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(ts, h->ks->phase_ts, sizeof(uint64_t) * (CGMAX + 3), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(ts + CGMAX + 3, h->ks->sub_ts, sizeof(uint64_t) * 10, cudaMemcpyDeviceToHost));
    return PROST_OK;
}

void prost_destroy(prost_handle *h)
{
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        if (h->s_in) cudaStreamSynchronize(h->s_in);
        if (h->s_out) cudaStreamSynchronize(h->s_out);
        free_state(h);
    }
    delete h;
}

} // extern "C"

// ---- many streams per tick ------------------------------------------------------
//
// A batch owns one prost_handle per stream.  A tick advances every stream by
// one frame: the streams are grouped by kernel family (k, storage type, frame
// type) and each group is one cooperative launch of the multi-stream frame
// kernel, its CTAs split between the group's streams (each stream keeps its
// own grid barrier).  The launches read the per-stream arguments (frame and
// mask pointers, barrier bases) from a device table that the tick's first
// operation copies from one of two pinned host tables; with the CUDA graph on,
// that copy and the launches are captured once per table and a tick is one
// graph launch.  The rows of every stream are rebased together every
// REBASE_EVERY ticks, outside the graph.

namespace {

struct BatchGroup {
    const KernelOps *ops;
    int fdt;
    int first, count; // its streams are order[first .. first + count)
    int ctas;         // CTAs of its launch
    int2 *d_map;      // CTA -> (stream slot in the table, CTA within the stream)
};

int occupancy_ctas(prost_handle *h, const KernelOps *ops, int fdt)
{
    const int occ = ops->frame_prepare(fdt);
    return occ < 1 ? 0 : occ * h->num_sms;
}

} // namespace

extern "C" int prost_batch_split(int32_t budget, int32_t n, const double *weight, const int32_t *cap,
                                 int32_t *ctas)
{
    if (n < 1 || budget < n || !weight || !cap || !ctas) return PROST_EINVAL;
    double wsum = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(weight[i] > 0.0) || !std::isfinite(weight[i]) || cap[i] < 1) return PROST_EINVAL;
        wsum += weight[i];
    }
    if (!std::isfinite(wsum)) return PROST_EINVAL;
    std::vector<double> frac(n);
    int64_t used = 0;
    for (int i = 0; i < n; ++i) {
        const double share = budget * weight[i] / wsum;
        int c = (int)floor(share);
        c = c < 1 ? 1 : c;
        if (c > cap[i]) c = cap[i];
        ctas[i] = c;
        frac[i] = share - floor(share);
        used += c;
    }
    // hand out what is left, largest fractional part first (lowest index on a
    // tie), within the caps
    while (used < budget) {
        int best = -1;
        for (int i = 0; i < n; ++i)
            if (ctas[i] < cap[i] && (best < 0 || frac[i] > frac[best])) best = i;
        if (best < 0) break;
        ctas[best] += 1;
        frac[best] -= 1.0;
        used += 1;
    }
    // over budget (the minimum of one CTA each): take from the largest
    while (used > budget) {
        int big = 0;
        for (int i = 1; i < n; ++i)
            if (ctas[i] > ctas[big]) big = i;
        ctas[big] -= 1;
        used -= 1;
    }
    return PROST_OK;
}

struct prost_batch {
    std::vector<prost_handle *> h;
    std::vector<int> order;     // table slot -> stream index (grouped)
    std::vector<int> grid;      // CTAs per stream
    std::vector<BatchGroup> groups;
    cudaStream_t stream;
    int device;
    FrameArgs *d_args;          // device argument table (one slot per stream)
    FrameArgs *h_args[2];       // pinned host tables, alternating ticks
    cudaEvent_t used[2];        // recorded after the tick that read h_args[i]
    int buf;
    int use_graph;
    int graph_ok;               // the capture worked (cooperative kernel nodes)
    cudaGraphExec_t gexec[2];
    float alpha;                // CTAs of a stream proportional to (its rows)^alpha
    // concurrent groups: each group's launch on its own stream, forked from
    // and joined back into the batch stream, on its own share of the SMs
    int concurrent;
    std::vector<cudaStream_t> gstream;
    std::vector<cudaEvent_t> gjoin;
    cudaEvent_t fork;
    uint32_t ticks_since_rebase;
    void *save;                 // device scratch of the tuner (states saved around trial ticks)
    size_t save_bytes;
    std::string err;
};

namespace {

int bfail(prost_batch *b, int code, const std::string &why)
{
    b->err = why;
    return code;
}

#define BCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? PROST_ENOMEM : PROST_ECUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

// SMs of each group when the groups run concurrently: shares of the device in
// proportion to the bytes the group's streams move per tick (at least one SM
// per stream), summing to at most the SM count, so that every CTA of every
// group is resident at once and no group's grid barrier waits on SMs another
// group holds.  Empty when the groups cannot all be resident together.
std::vector<int> concurrent_sms(prost_batch *b)
{
    const int sms = b->h[0]->num_sms;
    const int ng = (int)b->groups.size();
    std::vector<double> w(ng, 0.0);
    std::vector<int> lo(ng), s(ng);
    double wsum = 0.0;
    int need = 0;
    for (int gi = 0; gi < ng; ++gi) {
        const BatchGroup &g = b->groups[gi];
        const int occ = g.ops->frame_prepare(g.fdt);
        if (occ < 1) return {};
        for (int i = 0; i < g.count; ++i) {
            const prost_handle *h = b->h[b->order[g.first + i]];
            w[gi] += (double)h->dp.C * (double)h->dp.Pp * (double)h->dp.k * (double)u_elem_bytes(h->dp) *
                     (double)(h->prm.n_cg + 3);
        }
        lo[gi] = (g.count + occ - 1) / occ;
        need += lo[gi];
        wsum += w[gi];
    }
    if (need > sms || !(wsum > 0.0)) return {};
    int used = 0;
    for (int gi = 0; gi < ng; ++gi) {
        s[gi] = std::max(lo[gi], (int)floor(sms * w[gi] / wsum));
        used += s[gi];
    }
    while (used > sms) { // take from the group with the most SMs per byte
        int big = -1;
        for (int gi = 0; gi < ng; ++gi)
            if (s[gi] > lo[gi] && (big < 0 || s[gi] / w[gi] > s[big] / w[big])) big = gi;
        s[big] -= 1;
        used -= 1;
    }
    while (used < sms) { // give to the group with the most bytes per SM
        int best = 0;
        for (int gi = 1; gi < ng; ++gi)
            if (w[gi] / s[gi] > w[best] / s[best]) best = gi;
        s[best] += 1;
        used += 1;
    }
    return s;
}

// Split each group's CTA budget between its streams (prost_batch_split), in
// proportion to rows^alpha, and upload the CTA -> stream map of its launch.
// Serial groups each take the whole device; concurrent groups their share.
int plan_ctas(prost_batch *b)
{
    std::vector<int> share;
    if (b->concurrent) {
        share = concurrent_sms(b);
        if (share.empty()) return bfail(b, PROST_EINVAL, "the groups cannot all be resident at once");
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        BatchGroup &g = b->groups[gi];
        prost_handle *h0 = b->h[b->order[g.first]];
        const int budget = b->concurrent ? share[gi] * g.ops->frame_prepare(g.fdt) : occupancy_ctas(h0, g.ops, g.fdt);
        if (budget < g.count) return bfail(b, PROST_EINVAL, "more streams in a group than resident CTAs");
        std::vector<double> w(g.count);
        std::vector<int32_t> cap(g.count), n(g.count);
        for (int i = 0; i < g.count; ++i) {
            prost_handle *h = b->h[b->order[g.first + i]];
            w[i] = pow((double)h->dp.C * (double)h->dp.P, (double)b->alpha);
            cap[i] = h->dp.npt;
            // the register form's cross-CTA sums cover at most RES_MAX_GRID CTAs
            if (h->prm.k <= KREG && cap[i] > RES_MAX_GRID) cap[i] = RES_MAX_GRID;
        }
        if (prost_batch_split(budget, g.count, w.data(), cap.data(), n.data()) != PROST_OK)
            return bfail(b, PROST_EINVAL, "CTA split");
        int used = 0;
        for (int i = 0; i < g.count; ++i) used += n[i];
        std::vector<int2> map;
        map.reserve(used);
        for (int i = 0; i < g.count; ++i) {
            const int slot = g.first + i;
            b->grid[b->order[slot]] = n[i];
            for (int c = 0; c < n[i]; ++c) map.push_back(make_int2(slot, c));
        }
        g.ctas = used;
        if (g.d_map) cudaFree(g.d_map);
        g.d_map = nullptr;
        BCK(cudaMalloc(&g.d_map, map.size() * sizeof(int2)));
        BCK(cudaMemcpy(g.d_map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    // partial-row space: every stream's handle holds rows for its own grid
    for (size_t s = 0; s < b->h.size(); ++s)
        if ((size_t)2 * col_stride(b->grid[s]) * partial_row(b->h[s]->prm.k) > b->h[s]->partial_floats)
            return bfail(b, PROST_EINVAL, "partial rows");
    return PROST_OK;
}

void drop_graphs(prost_batch *b)
{
    for (int i = 0; i < 2; ++i)
        if (b->gexec[i]) {
            cudaGraphExecDestroy(b->gexec[i]);
            b->gexec[i] = nullptr;
        }
}

// the tick's operations on the batch stream: table copy, one launch per
// group, in turn or (concurrent) each on its group stream between a fork and
// a join
int enqueue_tick(prost_batch *b, int t)
{
    BCK(cudaMemcpyAsync(b->d_args, b->h_args[t], b->h.size() * sizeof(FrameArgs), cudaMemcpyHostToDevice,
                        b->stream));
    // the CTA maps hold table slots of the whole batch
    if (!b->concurrent) {
        for (const BatchGroup &g : b->groups)
            BCK(g.ops->frame_multi(b->d_args, g.d_map, g.ctas, g.fdt, b->stream));
        return PROST_OK;
    }
    BCK(cudaEventRecord(b->fork, b->stream));
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const BatchGroup &g = b->groups[gi];
        BCK(cudaStreamWaitEvent(b->gstream[gi], b->fork, 0));
        BCK(g.ops->frame_multi(b->d_args, g.d_map, g.ctas, g.fdt, b->gstream[gi]));
        BCK(cudaEventRecord(b->gjoin[gi], b->gstream[gi]));
        BCK(cudaStreamWaitEvent(b->stream, b->gjoin[gi], 0));
    }
    return PROST_OK;
}

int capture(prost_batch *b, int t)
{
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_tick(b, t);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return bfail(b, PROST_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&b->gexec[t], graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return bfail(b, PROST_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    return PROST_OK;
}

} // namespace

extern "C" int prost_batch_init(const prost_params *prms, int32_t n, void *stream, prost_batch **out)
{
    if (!out) { g_init_err = "out is NULL"; return PROST_EINVAL; }
    *out = nullptr;
    if (!prms || n < 1) { g_init_err = "no streams"; return PROST_EINVAL; }
    prost_batch *b = new (std::nothrow) prost_batch();
    if (!b) { g_init_err = "host allocation failed"; return PROST_ENOMEM; }
    b->stream = (cudaStream_t)stream;
    b->alpha = 1.f;
    b->use_graph = 1;
    b->graph_ok = 1;
    auto bail = [&](int code) {
        if (g_init_err.empty()) g_init_err = b->err;
        prost_batch_destroy(b);
        return code;
    };
    g_init_err.clear();
    for (int i = 0; i < n; ++i)
        if (prms[i].k > KFRAME || prms[i].form == PROST_FORM_PASSES) {
            g_init_err = "stream " + std::to_string(i) + ": a batch runs the single-launch forms only (k <= 16, form not PASSES)";
            return bail(PROST_EINVAL);
        }
    for (int i = 0; i < n; ++i) {
        prost_handle *h = nullptr;
        const int rc = prost_init(&prms[i], stream, &h);
        if (rc) {
            g_init_err = "stream " + std::to_string(i) + ": " + g_init_err;
            return bail(rc);
        }
        b->h.push_back(h);
    }
    b->device = b->h[0]->device;
    b->grid.assign(n, 1);
    // group by kernel family, streams of a group in consecutive table slots
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        const prost_params &a = b->h[x]->prm, &c = b->h[y]->prm;
        if (a.k != c.k) return a.k < c.k;
        if (a.u_dtype != c.u_dtype) return a.u_dtype < c.u_dtype;
        return a.frame_dtype < c.frame_dtype;
    });
    b->order = idx;
    for (int i = 0; i < n;) {
        int j = i;
        const prost_params &a = b->h[idx[i]]->prm;
        while (j < n && b->h[idx[j]]->prm.k == a.k && b->h[idx[j]]->prm.u_dtype == a.u_dtype &&
               b->h[idx[j]]->prm.frame_dtype == a.frame_dtype)
            ++j;
        BatchGroup g;
        g.ops = b->h[idx[i]]->ops;
        g.fdt = a.frame_dtype;
        g.first = i;
        g.count = j - i;
        g.ctas = 0;
        g.d_map = nullptr;
        b->groups.push_back(g);
        i = j;
    }
    int rc = plan_ctas(b);
    if (rc) return bail(rc);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return bail(PROST_ECUDA);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(PROST_ECUDA);
        b->gstream.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(PROST_ECUDA);
        b->gjoin.push_back(e);
    }
    if (cudaMalloc(&b->d_args, (size_t)n * sizeof(FrameArgs)) != cudaSuccess) return bail(PROST_ENOMEM);
    for (int t = 0; t < 2; ++t) {
        if (cudaMallocHost(&b->h_args[t], (size_t)n * sizeof(FrameArgs)) != cudaSuccess) return bail(PROST_ENOMEM);
        if (cudaEventCreateWithFlags(&b->used[t], cudaEventDisableTiming) != cudaSuccess) return bail(PROST_ECUDA);
        cudaEventRecord(b->used[t], b->stream);
    }
    *out = b;
    return PROST_OK;
}

extern "C" int prost_batch_step(prost_batch *b, const void *const *frames, uint8_t *const *masks)
{
    if (!b) return PROST_EINVAL;
    if (!frames) return bfail(b, PROST_EINVAL, "frames is NULL");
    DeviceGuard dg(b->device);
    const int t = b->buf;
    BCK(cudaEventSynchronize(b->used[t])); // the tick before last has read this table
    FrameArgs *tab = b->h_args[t];
    const int n = (int)b->h.size();
    for (int slot = 0; slot < n; ++slot) {
        const int s = b->order[slot];
        prost_handle *h = b->h[s];
        const DevParams &dp = h->dp;
        const size_t eb = frame_elem_bytes(h->prm);
        if (!frames[s] || ((uintptr_t)frames[s] % 16) != 0 || ((size_t)dp.P * eb) % 16 != 0)
            return bfail(b, PROST_EINVAL, "frame " + std::to_string(s) +
                                              ": device frames of a batch must be 16-byte aligned planes");
        FrameArgs &fa = tab[slot];
        memset(&fa, 0, sizeof(fa));
        fa.U = h->U;
        fa.frame = frames[s];
        fa.labels = h->labels;
        fa.mask_out = masks ? masks[s] : nullptr;
        fa.bg_out = nullptr;
        fa.ks = h->ks;
        fa.partials = h->partials;
        fa.bar = h->bar;
        fa.bar_base = h->bar_base;
        fa.frame_pitch = dp.P;
        fa.col_stride = col_stride(b->grid[s]);
        fa.grid = b->grid[s];
        fa.prm = dp;
        h->bar_base += (unsigned long long)b->grid[s] * (unsigned long long)frame_arrivals(h->prm.n_cg);
    }
    if (b->use_graph && b->graph_ok) {
        if (!b->gexec[t]) {
            const int rc = capture(b, t);
            if (rc) { // the tick runs without a graph from now on; the reason is kept
                b->graph_ok = 0;
                drop_graphs(b);
                (void)cudaGetLastError(); // clear the capture's error
            }
        }
        if (b->gexec[t]) BCK(cudaGraphLaunch(b->gexec[t], b->stream));
    }
    if (!(b->use_graph && b->graph_ok)) {
        const int rc = enqueue_tick(b, t);
        if (rc) return rc;
    }
    BCK(cudaEventRecord(b->used[t], b->stream));
    b->buf ^= 1;
    if (++b->ticks_since_rebase >= REBASE_EVERY) {
        for (prost_handle *h : b->h) {
            const int rc = rebase(h, 0);
            if (rc) return bfail(b, rc, h->err);
            h->steps_since_rebase = 0;
        }
        b->ticks_since_rebase = 0;
    }
    return PROST_OK;
}

extern "C" int prost_batch_sync(prost_batch *b)
{
    if (!b) return PROST_EINVAL;
    DeviceGuard dg(b->device);
    BCK(cudaStreamSynchronize(b->stream));
    for (prost_handle *h : b->h) {
        const int rc = prost_sync(h);
        if (rc) return bfail(b, rc, h->err);
    }
    return PROST_OK;
}

extern "C" int prost_batch_stream(prost_batch *b, int32_t i, prost_handle **h)
{
    if (!b || !h || i < 0 || i >= (int32_t)b->h.size()) return PROST_EINVAL;
    *h = b->h[i];
    return PROST_OK;
}

extern "C" int prost_batch_set_graph(prost_batch *b, int enable)
{
    if (!b) return PROST_EINVAL;
    b->use_graph = enable ? 1 : 0;
    return PROST_OK;
}

extern "C" int prost_batch_set_concurrent(prost_batch *b, int enable)
{
    if (!b) return PROST_EINVAL;
    DeviceGuard dg(b->device);
    BCK(cudaStreamSynchronize(b->stream));
    const int old = b->concurrent;
    b->concurrent = enable ? 1 : 0;
    drop_graphs(b);
    const int rc = plan_ctas(b);
    if (rc) {
        const std::string why = b->err;
        b->concurrent = old;
        plan_ctas(b);
        b->err = why;
        return rc;
    }
    return PROST_OK;
}

extern "C" int prost_batch_get_concurrent(prost_batch *b, int32_t *enabled)
{
    if (!b || !enabled) return PROST_EINVAL;
    *enabled = b->concurrent;
    return PROST_OK;
}

extern "C" int prost_batch_plan(prost_batch *b, int32_t *ctas_per_stream, int32_t *n_groups, float *alpha,
                                int32_t *graph)
{
    if (!b) return PROST_EINVAL;
    if (ctas_per_stream)
        for (size_t s = 0; s < b->h.size(); ++s) ctas_per_stream[s] = b->grid[s];
    if (n_groups) *n_groups = (int32_t)b->groups.size();
    if (alpha) *alpha = b->alpha;
    if (graph) *graph = b->use_graph && b->graph_ok ? 1 : 0;
    return PROST_OK;
}

namespace {

// device copies of every stream's subspace, k-space state and labels (the
// tuner's trial ticks must not move the trackers)
int save_states(prost_batch *b, bool restore)
{
    size_t need = 0;
    for (prost_handle *h : b->h)
        need += (size_t)h->dp.k * h->dp.C * h->dp.Pp * u_elem_bytes(h->dp) + sizeof(KState) + (size_t)h->dp.Pp + 256;
    if (!restore && need > b->save_bytes) {
        if (b->save) cudaFree(b->save);
        b->save = nullptr;
        b->save_bytes = 0;
        BCK(cudaMalloc(&b->save, need));
        b->save_bytes = need;
    }
    char *p = static_cast<char *>(b->save);
    for (prost_handle *h : b->h) {
        const size_t ub = (size_t)h->dp.k * h->dp.C * h->dp.Pp * u_elem_bytes(h->dp);
        void *dst[3] = {p, p + ub, p + ub + sizeof(KState)};
        void *src[3] = {h->U, h->ks, h->labels};
        const size_t len[3] = {ub, sizeof(KState), (size_t)h->dp.Pp};
        for (int i = 0; i < 3; ++i)
            BCK(cudaMemcpyAsync(restore ? src[i] : dst[i], restore ? dst[i] : src[i], len[i],
                                cudaMemcpyDeviceToDevice, b->stream));
        p += (ub + sizeof(KState) + (size_t)h->dp.Pp + 255) / 256 * 256;
    }
    return PROST_OK;
}

} // namespace

// Pick the batch plan by measurement: the CTA split exponent alpha in
// {0.5, 0.75, 1}, the groups in turn or concurrent (when they can all be
// resident at once) and the graph on or off, each timed over `ticks` ticks on the
// given frames; the states are saved before and restored after every trial,
// so tuning leaves the trackers where they were (the frame counters included).
extern "C" int prost_batch_tune(prost_batch *b, const void *const *frames, int32_t ticks, float *best_ms)
{
    if (!b || !frames || ticks < 1) return PROST_EINVAL;
    DeviceGuard dg(b->device);
    int rc = save_states(b, false);
    if (rc) return rc;
    const float alphas[3] = {0.5f, 0.75f, 1.0f};
    float best = 1e30f, best_alpha = b->alpha;
    int best_graph = b->use_graph, best_conc = b->concurrent;
    const uint32_t ticks0 = b->ticks_since_rebase;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (int trial = 0; trial < 6 && !rc; ++trial) {
        const float al = alphas[trial % 3];
        b->concurrent = trial / 3;
        if (b->concurrent && concurrent_sms(b).empty()) break; // the groups cannot all be resident at once
        b->alpha = al;
        drop_graphs(b);
        rc = plan_ctas(b);
        if (rc) break;
        for (int gr = 0; gr < 2; ++gr) {
            b->use_graph = gr;
            rc = prost_batch_step(b, frames, nullptr); // warm (and capture)
            if (!rc) rc = prost_batch_step(b, frames, nullptr);
            if (rc) break;
            BCK(cudaEventRecord(e0, b->stream));
            for (int i = 0; i < ticks && !rc; ++i) rc = prost_batch_step(b, frames, nullptr);
            BCK(cudaEventRecord(e1, b->stream));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            ms /= (float)ticks;
            if (!rc && ms < best) {
                best = ms;
                best_alpha = al;
                best_graph = gr;
                best_conc = b->concurrent;
            }
            const int rs = save_states(b, true);
            if (!rc) rc = rs;
            if (rc) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ticks_since_rebase = ticks0;
    b->alpha = best_alpha;
    b->use_graph = best_graph;
    b->concurrent = best_conc;
    drop_graphs(b);
    const int rp = plan_ctas(b);
    if (!rc) rc = rp;
    BCK(cudaStreamSynchronize(b->stream));
    if (best_ms) *best_ms = best;
    return rc;
}

extern "C" const char *prost_batch_last_error(const prost_batch *b)
{
    return b ? b->err.c_str() : g_init_err.c_str();
}

extern "C" void prost_batch_destroy(prost_batch *b)
{
    if (!b) return;
    if (b->stream || !b->h.empty()) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (BatchGroup &g : b->groups)
        if (g.d_map) cudaFree(g.d_map);
    if (b->d_args) cudaFree(b->d_args);
    for (int t = 0; t < 2; ++t) {
        if (b->h_args[t]) cudaFreeHost(b->h_args[t]);
        if (b->used[t]) cudaEventDestroy(b->used[t]);
    }
    if (b->save) cudaFree(b->save);
    for (cudaStream_t s : b->gstream)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->gjoin)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (prost_handle *h : b->h) prost_destroy(h);
    delete b;
}
