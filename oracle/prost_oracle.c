/*
 * FP64 CPU oracle of pROST's per-frame update (Seidel, Hage, Kleinsteuber,
 * "pROST: A Smoothed l_p-norm Robust Online Subspace Tracking Method for
 * Realtime Background Subtraction in Video", arXiv:1302.2073).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load it; the library never does.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Everything is double precision, single threaded, in the order the paper
 * states it.  Layouts: U is m x k row-major (U[e*k + j], row e is u_e^T),
 * frames and vectors over the m entries are channel-planar (entry e = c*P + q
 * for pixel q of channel c, the colour stacking of Section 3.4), weights and
 * labels are per pixel (P entries).
 *
 * Readings where the paper leaves a choice open (each is listed with its
 * reason in the design notes of the repository):
 *   - Step 1 is a nonlinear conjugate-gradient method, Polak-Ribiere+ beta,
 *     warm-started at the previous frame's y, restarted (d = -g) every frame,
 *     exactly n_cg iterations, each with one majorise-minimise line step
 *     (closed form below; exact line search when p = 2).
 *   - Step 2 descends along B = -G_U with the rank-one SVD of Eq. (svd);
 *     the geodesic of Eq. (geodesic) is evaluated with the full thin SVD of B
 *     (the k-1 zero singular values keep U's other directions fixed), angle
 *     theta = sigma_1 * t.  Skipped when |y| = 0 or |pi(eta)| = 0.
 *   - Step 3 labels a pixel foreground when max_c |x_c - u_c^T y| >= delta
 *     (Section 3.4), using the updated subspace by default; its weight for the
 *     next frame is omega, else 1 (Eq. pixelweighting).  First frame: w = 1.
 *   - After Step 3 the representative is re-orthonormalised by Cholesky-QR,
 *     U <- U R^{-1}, y <- R y with U^T U = R^T R (not in the paper; the
 *     identity map in exact arithmetic since the geodesic stays on St_{k,m}).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTSPD (-3)

#define ORC_FRAME_U8 0
#define ORC_FRAME_F32 1
#define ORC_FRAME_F64 2

#define ORC_MAX_CG 64

typedef struct orc_params {
    int32_t width, height, channels, k;
    double p, mu, delta, omega;
    double t_init, t_min;
    int32_t i_init, n_cg;
    double in_scale, in_offset;
    int32_t mask_from; /* 0: Step 3 uses the updated subspace, 1: the one before Step 2 */
    int32_t reorth;    /* 1: Cholesky-QR re-orthonormalisation after each frame */
} orc_params;

typedef struct orc_trace {
    double cost[ORC_MAX_CG + 1];  /* h_{mu,w}(x - U y_j), j = 0..n_cg */
    double alpha[ORC_MAX_CG];     /* line step of CG iteration j */
    double beta[ORC_MAX_CG];      /* PR+ coefficient forming d_j (beta[0] = 0) */
    double gnorm[ORC_MAX_CG + 1]; /* |grad_y| at y_j */
    double pi_norm, y_norm, sigma, t, theta;
    int32_t updated;              /* 0 when the Grassmann step was skipped */
    int32_t pad;
    int64_t n_foreground;
} orc_trace;

static int64_t orc_m(const orc_params *prm)
{
    return (int64_t)prm->channels * prm->width * prm->height;
}

int orc_check_params(const orc_params *prm)
{
    if (!prm || prm->width <= 0 || prm->height <= 0 || prm->channels <= 0 || prm->k <= 0)
        return ORC_EINVAL;
    if ((int64_t)prm->k > orc_m(prm)) return ORC_EINVAL;
    if (!(prm->p > 0.0 && prm->p <= 2.0) || !(prm->mu > 0.0) || !(prm->delta > 0.0))
        return ORC_EINVAL;
    if (!(prm->omega >= 0.0 && prm->omega <= 1.0)) return ORC_EINVAL;
    if (!(prm->t_init > 0.0) || !(prm->t_min > 0.0) || prm->i_init < 1) return ORC_EINVAL;
    if (prm->n_cg < 0 || prm->n_cg > ORC_MAX_CG) return ORC_EINVAL;
    return ORC_OK;
}

/* ---- scalar pieces -------------------------------------------------------- */

/* One term of the smoothed l_p-norm, Eq. (smoothlpnorm): (r^2 + mu)^(p/2). */
double orc_h(double r, double mu, double p)
{
    return pow(r * r + mu, 0.5 * p);
}

/* mu coupled to the threshold by requiring d^2 h / dr^2 = 0 at r = delta,
 * Eq. (opt_mu) -> Eq. (opt_mu2). */
double orc_mu_heuristic(double delta, double p)
{
    return delta * delta * (1.0 - p);
}

/* Step-size rule of Section 3.4: t = max(exp(-tau i) t_init, t_min) with
 * tau = -log(t_min / t_init) / i_init; i counts frames from 0. */
double orc_step_size(const orc_params *prm, int64_t i)
{
    double tau = -log(prm->t_min / prm->t_init) / (double)prm->i_init;
    double t = exp(-tau * (double)i) * prm->t_init;
    return t > prm->t_min ? t : prm->t_min;
}

/* ---- vectors over the m entries ------------------------------------------ */

/* Input map of the hot path: x = in_scale * frame - in_offset (a fixed affine
 * stand-in for the mean subtraction and std normalisation of Section 3.4). */
void orc_preprocess(const orc_params *prm, const void *frame, int frame_dtype, double *x)
{
    int64_t m = orc_m(prm);
    for (int64_t e = 0; e < m; ++e) {
        double v;
        if (frame_dtype == ORC_FRAME_U8) v = (double)((const uint8_t *)frame)[e];
        else if (frame_dtype == ORC_FRAME_F32) v = (double)((const float *)frame)[e];
        else v = ((const double *)frame)[e];
        x[e] = prm->in_scale * v - prm->in_offset;
    }
}

/* Per-pixel weights of Eq. (pixelweighting): omega where the previous frame
 * labelled the pixel foreground, 1 elsewhere. */
void orc_weights(const orc_params *prm, const uint8_t *labels, double *w)
{
    int64_t P = (int64_t)prm->width * prm->height;
    for (int64_t q = 0; q < P; ++q) w[q] = (labels && labels[q]) ? prm->omega : 1.0;
}

/* r = x - U y. */
void orc_residual(int64_t m, int k, const double *U, const double *y, const double *x, double *r)
{
    for (int64_t e = 0; e < m; ++e) {
        double uy = 0.0;
        for (int j = 0; j < k; ++j) uy += U[e * k + j] * y[j];
        r[e] = x[e] - uy;
    }
}

/* Cost of Eq. (spcacost): h_{mu,w}(x - U y) = sum_e w_e ((x_e - u_e^T y)^2 + mu)^(p/2),
 * with the weighted norm of Eq. (weightedLPnorm); w_e is the weight of e's pixel. */
double orc_cost(const orc_params *prm, const double *U, const double *y, const double *x,
                const double *w)
{
    int64_t P = (int64_t)prm->width * prm->height, m = orc_m(prm);
    int k = prm->k;
    double f = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        double uy = 0.0;
        for (int j = 0; j < k; ++j) uy += U[e * k + j] * y[j];
        f += w[e % P] * orc_h(x[e] - uy, prm->mu, prm->p);
    }
    return f;
}

/* eta_e = -p w_e r_e (r_e^2 + mu)^(p/2 - 1), Section 3.3 (the derivative of the
 * cost with respect to U_{e,j} is eta_e y_j). */
void orc_eta(const orc_params *prm, const double *r, const double *w, double *eta)
{
    int64_t P = (int64_t)prm->width * prm->height, m = orc_m(prm);
    for (int64_t e = 0; e < m; ++e)
        eta[e] = -prm->p * w[e % P] * r[e] * pow(r[e] * r[e] + prm->mu, 0.5 * prm->p - 1.0);
}

/* out = U^T v (k entries).  With v = eta this is the gradient of the cost with
 * respect to y: d/dy sum w h(x - U y) = U^T eta. */
void orc_ut(int64_t m, int k, const double *U, const double *v, double *out)
{
    for (int j = 0; j < k; ++j) out[j] = 0.0;
    for (int64_t e = 0; e < m; ++e)
        for (int j = 0; j < k; ++j) out[j] += U[e * k + j] * v[e];
}

/* Euclidean gradient of the cost with respect to U: (eta y^T)_{e,j} = eta_e y_j. */
void orc_grad_U(int64_t m, int k, const double *eta, const double *y, double *G)
{
    for (int64_t e = 0; e < m; ++e)
        for (int j = 0; j < k; ++j) G[e * k + j] = eta[e] * y[j];
}

/* Projection onto the tangent space of the Grassmannian, Eq. (gproject):
 * pi(h) = (I - U U^T) h for one column h. */
void orc_project(int64_t m, int k, const double *U, const double *h, double *out)
{
    double *uth = (double *)malloc(sizeof(double) * (size_t)k);
    if (!uth) return;
    orc_ut(m, k, U, h, uth);
    for (int64_t e = 0; e < m; ++e) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += U[e * k + j] * uth[j];
        out[e] = h[e] - s;
    }
    free(uth);
}

static double dot(int k, const double *a, const double *b)
{
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += a[j] * b[j];
    return s;
}

/* ---- Step 1: y = argmin_y h_{mu,w}(x - U y), Eq. (onlinestep1) ------------ */
/*
 * Nonlinear CG with the Polak-Ribiere+ coefficient.  Line step: since
 * z -> (z + mu)^(p/2) is concave for p <= 2, each term is majorised by its
 * tangent line in z = r^2 at the current y, so with q = U d and
 * c_e = w_e (r_e^2 + mu)^(p/2 - 1)
 *   h(y + alpha d) <= h(y) + (p/2) sum_e c_e ((r_e - alpha q_e)^2 - r_e^2).
 * The right side is minimised by alpha = sum c r q / sum c q^2, which therefore
 * never increases the cost (and is the exact line minimiser when p = 2).
 */
int orc_cg(const orc_params *prm, const double *U, const double *x, const double *w,
           double *y, orc_trace *tr)
{
    int64_t P = (int64_t)prm->width * prm->height, m = orc_m(prm);
    int k = prm->k;
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *eta = (double *)malloc(sizeof(double) * (size_t)m);
    double *q = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)k);
    double *gn = (double *)malloc(sizeof(double) * (size_t)k);
    double *d = (double *)malloc(sizeof(double) * (size_t)k);
    if (!r || !eta || !q || !g || !gn || !d) {
        free(r); free(eta); free(q); free(g); free(gn); free(d);
        return ORC_ENOMEM;
    }
    /* gradient at the warm start y_0 */
    orc_residual(m, k, U, y, x, r);
    orc_eta(prm, r, w, eta);
    orc_ut(m, k, U, eta, g);
    if (tr) {
        tr->cost[0] = orc_cost(prm, U, y, x, w);
        tr->gnorm[0] = sqrt(dot(k, g, g));
        tr->beta[0] = 0.0;
    }
    for (int j = 0; j < k; ++j) d[j] = -g[j];

    for (int it = 0; it < prm->n_cg; ++it) {
        /* line step along d */
        double num = 0.0, den = 0.0;
        for (int64_t e = 0; e < m; ++e) {
            double qe = 0.0;
            for (int j = 0; j < k; ++j) qe += U[e * k + j] * d[j];
            q[e] = qe;
            double c = w[e % P] * pow(r[e] * r[e] + prm->mu, 0.5 * prm->p - 1.0);
            num += c * r[e] * qe;
            den += c * qe * qe;
        }
        double alpha = den > 0.0 ? num / den : 0.0;
        for (int j = 0; j < k; ++j) y[j] += alpha * d[j];

        /* gradient at the new point */
        orc_residual(m, k, U, y, x, r);
        orc_eta(prm, r, w, eta);
        orc_ut(m, k, U, eta, gn);
        double gg = dot(k, g, g);
        double beta = 0.0;
        if (gg > 0.0) {
            double num_b = 0.0;
            for (int j = 0; j < k; ++j) num_b += gn[j] * (gn[j] - g[j]);
            beta = num_b / gg;
            if (beta < 0.0) beta = 0.0;
        }
        for (int j = 0; j < k; ++j) {
            d[j] = -gn[j] + beta * d[j];
            g[j] = gn[j];
        }
        if (tr) {
            tr->alpha[it] = alpha;
            tr->cost[it + 1] = orc_cost(prm, U, y, x, w);
            tr->gnorm[it + 1] = sqrt(dot(k, g, g));
            if (it + 1 < ORC_MAX_CG) tr->beta[it + 1] = beta;
        }
    }
    free(r); free(eta); free(q); free(g); free(gn); free(d);
    return ORC_OK;
}

/* ---- Step 2: one geodesic step on the Grassmannian ----------------------- */
/*
 * Projected gradient G_U = pi(eta) y^T has rank one with SVD sigma_1 s v^T,
 * s = pi(eta)/|pi(eta)|, sigma_1 = |pi(eta)| |y|, v = y/|y|  (Eq. svd).
 * Moving along -G_U on the geodesic of Eq. (geodesic), with the thin SVD of
 * B = -G_U = (-s) sigma_1 v^T completed by zero singular values, gives
 *   U(t) = U + ((cos(sigma_1 t) - 1) U v - sin(sigma_1 t) s) v^T.
 */
int orc_grassmann_step(const orc_params *prm, double *U, const double *y, const double *eta,
                       double t, orc_trace *tr)
{
    int64_t m = orc_m(prm);
    int k = prm->k;
    double *pi = (double *)malloc(sizeof(double) * (size_t)m);
    double *v = (double *)malloc(sizeof(double) * (size_t)k);
    if (!pi || !v) { free(pi); free(v); return ORC_ENOMEM; }
    orc_project(m, k, U, eta, pi);
    double pin = 0.0;
    for (int64_t e = 0; e < m; ++e) pin += pi[e] * pi[e];
    pin = sqrt(pin);
    double yn = sqrt(dot(k, y, y));
    double sigma = pin * yn;
    double theta = sigma * t;
    int updated = (yn > 0.0 && pin > 0.0);
    if (updated) {
        for (int j = 0; j < k; ++j) v[j] = y[j] / yn;
        double cm1 = cos(theta) - 1.0, sn = sin(theta);
        for (int64_t e = 0; e < m; ++e) {
            double uv = 0.0;
            for (int j = 0; j < k; ++j) uv += U[e * k + j] * v[j];
            double s_e = pi[e] / pin;
            double coef = cm1 * uv - sn * s_e;
            for (int j = 0; j < k; ++j) U[e * k + j] += coef * v[j];
        }
    }
    if (tr) {
        tr->pi_norm = pin;
        tr->y_norm = yn;
        tr->sigma = sigma;
        tr->t = t;
        tr->theta = updated ? theta : 0.0;
        tr->updated = updated;
    }
    free(pi); free(v);
    return ORC_OK;
}

/* ---- Step 3: labels (and so the next frame's weights) -------------------- */
/* Pixel q is foreground when max_c |x_{c,q} - u_{c,q}^T y| >= delta (Section 3.4;
 * for one channel this is |x_q - u_q^T y| >= delta, the complement of the
 * weight-1 case of Eq. pixelweighting).  maxres (nullable) gets the per-pixel
 * maximum absolute residual.  Returns the number of foreground pixels. */
int64_t orc_labels(const orc_params *prm, const double *U, const double *y, const double *x,
                   uint8_t *labels, double *maxres)
{
    int64_t P = (int64_t)prm->width * prm->height;
    int k = prm->k, C = prm->channels;
    int64_t n_fg = 0;
    for (int64_t q = 0; q < P; ++q) {
        double mx = 0.0;
        for (int c = 0; c < C; ++c) {
            int64_t e = (int64_t)c * P + q;
            double uy = 0.0;
            for (int j = 0; j < k; ++j) uy += U[e * k + j] * y[j];
            double a = fabs(x[e] - uy);
            if (a > mx) mx = a;
        }
        uint8_t f = (uint8_t)(mx >= prm->delta);
        labels[q] = f;
        n_fg += f;
        if (maxres) maxres[q] = mx;
    }
    return n_fg;
}

/* ---- re-orthonormalisation (not in the paper) ----------------------------- */
/* Cholesky-QR: G = U^T U = R^T R (R upper triangular), U <- U R^{-1}, y <- R y,
 * so that U^T U = I and the background U y is unchanged. */
int orc_reorthonormalize(int64_t m, int k, double *U, double *y)
{
    double *G = (double *)calloc((size_t)k * k, sizeof(double));
    double *R = (double *)calloc((size_t)k * k, sizeof(double));
    double *ry = (double *)calloc((size_t)k, sizeof(double));
    double *row = (double *)calloc((size_t)k, sizeof(double));
    if (!G || !R || !ry || !row) { free(G); free(R); free(ry); free(row); return ORC_ENOMEM; }
    for (int64_t e = 0; e < m; ++e)
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) G[a * k + b] += U[e * k + a] * U[e * k + b];
    /* Cholesky, row by row of R: R[a][a] = sqrt(G[a][a] - sum_{l<a} R[l][a]^2) */
    for (int a = 0; a < k; ++a) {
        for (int b = a; b < k; ++b) {
            double s = G[a * k + b];
            for (int l = 0; l < a; ++l) s -= R[l * k + a] * R[l * k + b];
            if (b == a) {
                if (!(s > 0.0)) { free(G); free(R); free(ry); free(row); return ORC_ENOTSPD; }
                R[a * k + a] = sqrt(s);
            } else {
                R[a * k + b] = s / R[a * k + a];
            }
        }
    }
    /* each row of U solves z R = u (forward substitution, R upper triangular) */
    for (int64_t e = 0; e < m; ++e) {
        for (int b = 0; b < k; ++b) {
            double s = U[e * k + b];
            for (int l = 0; l < b; ++l) s -= row[l] * R[l * k + b];
            row[b] = s / R[b * k + b];
        }
        for (int b = 0; b < k; ++b) U[e * k + b] = row[b];
    }
    if (y) {
        for (int a = 0; a < k; ++a) {
            double s = 0.0;
            for (int b = a; b < k; ++b) s += R[a * k + b] * y[b];
            ry[a] = s;
        }
        for (int a = 0; a < k; ++a) y[a] = ry[a];
    }
    free(G); free(R); free(ry); free(row);
    return ORC_OK;
}

/* ---- one frame: Steps 1-3 of Section 3.3 ---------------------------------- */
/*
 * State in/out: U (m x k), y (k), labels (P; previous frame's labels on entry,
 * this frame's on exit).  i is the frame counter (0 for the first frame).
 * residual_out (nullable, m entries) gets x - U y with the subspace Step 3
 * used, before re-orthonormalisation.
 */
int orc_frame_step(const orc_params *prm, double *U, double *y, uint8_t *labels, int64_t i,
                   const void *frame, int frame_dtype, orc_trace *tr, double *residual_out)
{
    int rc = orc_check_params(prm);
    if (rc) return rc;
    int64_t P = (int64_t)prm->width * prm->height, m = orc_m(prm);
    int k = prm->k;
    double *x = (double *)malloc(sizeof(double) * (size_t)m);
    double *w = (double *)malloc(sizeof(double) * (size_t)P);
    double *r = (double *)malloc(sizeof(double) * (size_t)m);
    double *eta = (double *)malloc(sizeof(double) * (size_t)m);
    double *Uold = NULL;
    if (prm->mask_from) Uold = (double *)malloc(sizeof(double) * (size_t)(m * k));
    if (!x || !w || !r || !eta || (prm->mask_from && !Uold)) {
        free(x); free(w); free(r); free(eta); free(Uold);
        return ORC_ENOMEM;
    }
    orc_preprocess(prm, frame, frame_dtype, x);
    orc_weights(prm, labels, w);

    /* Step 1 */
    rc = orc_cg(prm, U, x, w, y, tr);
    if (rc) goto done;

    /* Step 2 */
    orc_residual(m, k, U, y, x, r);
    orc_eta(prm, r, w, eta);
    if (Uold) memcpy(Uold, U, sizeof(double) * (size_t)(m * k));
    rc = orc_grassmann_step(prm, U, y, eta, orc_step_size(prm, i), tr);
    if (rc) goto done;

    /* Step 3 */
    {
        const double *Ul = Uold ? Uold : U;
        int64_t nfg = orc_labels(prm, Ul, y, x, labels, NULL);
        if (tr) tr->n_foreground = nfg;
        if (residual_out) orc_residual(m, k, Ul, y, x, residual_out);
    }
    if (prm->reorth) rc = orc_reorthonormalize(m, k, U, y);
done:
    free(x); free(w); free(r); free(eta); free(Uold);
    return rc;
}
