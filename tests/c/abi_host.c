/* A plain C99 caller of the prost C ABI: it compiles include/prost.h as C,
 * links libprost, prints the layout of the public structs (for the ctypes
 * binding to be checked against) and exercises the entry points that need no
 * GPU: version, error names, parameter validation and sizes, the batch CTA
 * split.  Exit status 0 when every check holds. */

#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "prost.h"

#define FIELD(T, f) printf("%s %s %zu %zu\n", #T, #f, offsetof(T, f), sizeof(((T *)0)->f))

static int failures = 0;

static void check(int ok, const char *what)
{
    if (!ok) {
        fprintf(stderr, "FAILED: %s\n", what);
        failures += 1;
    }
}

static prost_params valid_params(void)
{
    prost_params p;
    memset(&p, 0, sizeof p);
    p.width = 64;
    p.height = 48;
    p.channels = 3;
    p.k = 10;
    p.p = 0.25;
    p.mu = 0.0; /* selects delta^2 (1 - p) */
    p.delta = 0.35;
    p.omega = 5e-5;
    p.t_init = 5e-3;
    p.t_min = 1e-4;
    p.i_init = 100;
    p.n_cg = 5;
    p.in_scale = 1.0 / 255.0;
    p.in_offset = 0.5;
    p.frame_dtype = PROST_U8;
    p.u_dtype = PROST_F32;
    p.mask_from = PROST_MASK_POST_UPDATE;
    p.seed = 1;
    return p;
}

int main(void)
{
    prost_params prm = valid_params();
    size_t bytes = 0;
    double w[3] = {1.0, 1.0, 1.0};
    int32_t cap[3] = {9, 9, 9};
    int32_t ctas[3] = {0, 0, 0};

    printf("sizeof prost_params %zu\n", sizeof(prost_params));
    FIELD(prost_params, width);
    FIELD(prost_params, height);
    FIELD(prost_params, channels);
    FIELD(prost_params, k);
    FIELD(prost_params, p);
    FIELD(prost_params, mu);
    FIELD(prost_params, delta);
    FIELD(prost_params, omega);
    FIELD(prost_params, t_init);
    FIELD(prost_params, t_min);
    FIELD(prost_params, i_init);
    FIELD(prost_params, n_cg);
    FIELD(prost_params, in_scale);
    FIELD(prost_params, in_offset);
    FIELD(prost_params, frame_dtype);
    FIELD(prost_params, u_dtype);
    FIELD(prost_params, mask_from);
    FIELD(prost_params, form);
    FIELD(prost_params, seed);
    printf("sizeof prost_stats %zu\n", sizeof(prost_stats));
    FIELD(prost_stats, frames);
    FIELD(prost_stats, bad_frames);
    FIELD(prost_stats, n_cg);
    FIELD(prost_stats, status);
    FIELD(prost_stats, cost);
    FIELD(prost_stats, gnorm);
    FIELD(prost_stats, alpha);
    FIELD(prost_stats, beta);
    FIELD(prost_stats, pi_norm);
    FIELD(prost_stats, y_norm);
    FIELD(prost_stats, sigma);
    FIELD(prost_stats, t);
    FIELD(prost_stats, theta);
    FIELD(prost_stats, updated);
    FIELD(prost_stats, pad0);
    FIELD(prost_stats, n_foreground);
    FIELD(prost_stats, orth_err);
    FIELD(prost_stats, eta_norm);
    FIELD(prost_stats, pi_explicit);
    FIELD(prost_stats, form);

    check(prost_version() == 102, "prost_version");
    check(prost_strerror(PROST_EINVAL) != NULL && strlen(prost_strerror(PROST_EINVAL)) > 0, "strerror");
    check(prost_state_bytes(&prm, &bytes) == PROST_OK, "state bytes of valid parameters");
    check(bytes > (size_t)64 * 48 * 3 * 10 * 4, "state holds at least the subspace");
    check(prost_state_bytes(&prm, NULL) == PROST_EINVAL, "NULL size pointer");
    check(prost_state_bytes(NULL, &bytes) == PROST_EINVAL, "NULL parameters");
    prm.k = 0;
    check(prost_state_bytes(&prm, &bytes) == PROST_EINVAL, "k = 0 rejected");
    prm = valid_params();
    prm.form = PROST_FORM_RESIDENT + 1;
    check(prost_state_bytes(&prm, &bytes) == PROST_EINVAL, "form beyond the five forms");
    prm = valid_params();
    prm.k = PROST_MAX_K;
    check(prost_state_bytes(&prm, &bytes) == PROST_OK, "k = 32 in the passes form");
    prm.k = PROST_MAX_K + 1;
    check(prost_state_bytes(&prm, &bytes) == PROST_EINVAL, "k = 33 rejected");
    prm.k = PROST_MAX_K_SINGLE + 1;
    prm.form = PROST_FORM_GRID;
    check(prost_state_bytes(&prm, &bytes) == PROST_EINVAL, "k = 17 has no grid form");
    prm = valid_params();
    prm.p = 3.0;
    check(prost_state_bytes(&prm, &bytes) == PROST_EINVAL, "p > 2 rejected");
    check(prost_init(NULL, NULL, NULL) == PROST_EINVAL, "prost_init without out");
    check(prost_inject_barrier_skew(NULL, 1) == PROST_EINVAL, "injection without a handle");
    check(prost_inject_wait_timeout(NULL, 0, 1000) == PROST_EINVAL, "wait injection without a handle");
    check(prost_step_async(NULL, NULL, NULL, NULL) == PROST_EINVAL, "pipelined step without a handle");
    check(prost_step_many(NULL, NULL, 1, 1, NULL) == PROST_EINVAL, "frames of a stream without a handle");
    check(prost_step_many_async(NULL, NULL, 1, NULL) == PROST_EINVAL, "pipelined frames without a handle");
    check(prost_wait(NULL) == PROST_EINVAL, "wait without a handle");
    check(prost_pre_get_state(NULL, NULL, NULL) == PROST_EINVAL, "pre-processor checkpoint without a handle");
    check(prost_pre_set_state(NULL, NULL, 0) == PROST_EINVAL, "pre-processor restore without a handle");
    check(prost_window_inject_wait_timeout(NULL, 1, 1000) == PROST_EINVAL, "window wait injection without a window");
    check(prost_batch_split(10, 3, w, cap, ctas) == PROST_OK, "batch split");
    check(ctas[0] == 4 && ctas[1] == 3 && ctas[2] == 3, "batch split of 10 over thirds");
    check(prost_batch_split(2, 3, w, cap, ctas) == PROST_EINVAL, "budget below the streams");
    check(prost_median3x3(NULL, NULL, 4, 4, 0, NULL) == PROST_EINVAL, "median of NULL");

    printf("failures %d\n", failures);
    return failures == 0 ? 0 : 1;
}
