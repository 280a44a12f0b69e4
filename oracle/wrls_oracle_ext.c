/*
 * wRLS denoiser ORACLE, extended predictor and weights -- test infrastructure only.
 *
 * Same rules as wrls_oracle.c (only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it; it shares no code with the CUDA path). This file restates
 * the per-frame denoiser of Iglesias-Guitian, Mane, Moon (IEEE TVCG 2020, Sec. 5.1-5.3)
 * for a predictor of any dimension d <= 8 and adds the alternatives that the paper
 * discusses and sets aside:
 *
 *   - G-buffer predictor (Sec. 2.1, 5.2: RLS denoisers such as [45] regress on auxiliary
 *     G-buffer features; Sec. 5.3 argues that path-traced volumes give noisy ones):
 *     p_j(t) = [1, z_j(t), g_j,1(t), ..., g_j,n(t)], d = 4 + n, or [1, g...] (d = 1 + n)
 *     without the temporal feature. g are the first n of the caller's feature planes of
 *     frame t.
 *   - sample-variance weight (Sec. 5.3: "the straightforward way" that the paper rejects
 *     for few samples): Eq. 13 with the squared colour distance ||I~ - z||^2 replaced by
 *     its expectation under the per-pixel sample variance, 3 sigma_j^2 (three channels):
 *     w = exp(-d_v^2 / h^2), d_v^2 = 3 sigma_j^2 / (min(||I~_j||, ||z_j||) + eps)^2.
 *   - nearest-pixel reprojection: the model at the pixel nearest to q (binary32
 *     floor(q + 0.5) per axis) instead of the bilinear fetch.
 *
 * Everything else is as in wrls_oracle.c (readings listed in its header): Eq. 12 feature
 * with the 3x3 clamp, Eq. 13 weight, Eq. 8 residual, Eq. 14 gain (Eq. 10 when w = 1),
 * Eq. 9 and Eq. 11 updates with one full d x d P per pixel shared by the three channels,
 * restarts, missing samples, the optional wind-up guard, and the 5x5 bilateral
 * cross-prediction blend. Additional readings of this file:
 *   - a G-buffer value that is not finite enters p as 0 and the sample gets weight 0 (it
 *     still enters z);
 *   - a variance that is not finite or is negative gives weight 0 (variance weight only);
 *   - a restarted pixel: beta = 0 (or the feature pass-through start, coefficients of the
 *     G-buffer entries 0) and P = p0_delta on the diagonal entries of the used predictor.
 *
 * State layout (per pixel n = y*W + x, d = predictor dimension):
 *   beta[n*3*d + c*d + a], P[n*d*d + a*d + b] (full), z[n*3 + c].
 * Pins: tests/test_oracle_ext_pins.py. Nothing here is blocked, fused or reordered.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double lambda;      /* forgetting factor (Sec. 5.2, Eq. 10-11) */
    double h;           /* wRLS bandwidth (Sec. 5.3, Eq. 13) */
    double alpha;       /* history weight of the temporal feature (Eq. 12, Sec. 6) */
    double eps;         /* Eq. 13 epsilon */
    double p0_delta;    /* initial inverse covariance P = p0_delta * I */
    double sigma_s;     /* blend: spatial Gaussian std in pixels */
    double h_s;         /* blend: feature-distance bandwidth */
    double p_trace_max; /* wind-up guard threshold, 0 = off */
    int radius;         /* blend window radius: 2 -> 5x5; 0 -> temporal only */
    int weight_mode;    /* 0 = Eq. 13; 1 = RLS (w = 1); 2 = sample-variance weight */
    int clamp_mode;     /* 0 = 3x3 clamp; 1 = no clamp */
    int blend_mode;     /* 0 = p_i beta_k; 1 = p_k beta_k */
    int feature_mode;   /* 0 = temporal feature in p; 1 = no temporal feature */
    int init_mode;      /* 0 = beta = 0; 1 = feature pass-through */
    int n_gbuf;         /* G-buffer planes appended to the predictor, 0..4 */
    int reproj_filter;  /* 0 = bilinear; 1 = nearest pixel */
} wrls_oracle_ext_params;

#define XNCH 3
#define XDMAX 8

int wrls_oracle_ext_dim(const wrls_oracle_ext_params* prm) {
    return (prm->feature_mode == 0 ? 4 : 1) + prm->n_gbuf;
}

static int xfinite3(const double v[3]) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

static double xnorm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* Denominator of the Eq. 13 distance: min of the two colour norms plus eps. */
static double xeq13_scale(const double a[3], const double b[3], double eps) {
    double na = xnorm3(a), nb = xnorm3(b);
    return (na < nb ? na : nb) + eps;
}

/* p = [1, z, g_1..g_n] (or [1, g_1..g_n] without the temporal feature). Returns 0 if a
 * G-buffer value is not finite (it enters p as 0). */
static int xpredictor(const wrls_oracle_ext_params* prm, const double z[3], const double* g,
                      double p[XDMAX]) {
    int ok = 1, a = 0;
    for (int i = 0; i < XDMAX; ++i) p[i] = 0.0;
    p[a++] = 1.0;
    if (prm->feature_mode == 0) {
        p[a++] = z[0];
        p[a++] = z[1];
        p[a++] = z[2];
    }
    for (int i = 0; i < prm->n_gbuf; ++i) {
        if (isfinite(g[i])) p[a + i] = g[i];
        else ok = 0;
    }
    return ok;
}

static void xinitial_model(const wrls_oracle_ext_params* prm, const double z[3],
                           double beta[XNCH][XDMAX], double P[XDMAX][XDMAX]) {
    int d = wrls_oracle_ext_dim(prm);
    for (int c = 0; c < XNCH; ++c)
        for (int a = 0; a < XDMAX; ++a) beta[c][a] = 0.0;
    if (prm->init_mode == 1) {
        if (prm->feature_mode == 0)
            for (int c = 0; c < XNCH; ++c) beta[c][c + 1] = 1.0;
        else
            for (int c = 0; c < XNCH; ++c) beta[c][0] = z[c];
    }
    for (int a = 0; a < XDMAX; ++a)
        for (int b = 0; b < XDMAX; ++b) P[a][b] = (a == b && a < d) ? prm->p0_delta : 0.0;
}

int wrls_oracle_ext_blend(const wrls_oracle_ext_params* prm, int W, int H, const double* beta,
                          const double* z, const float* gbuf, double* out);

/*
 * One frame. rad: 3 planes (binary32), mot: 2 planes (vx, vy), var: H*W sample variance
 * (required for weight_mode 2, else may be NULL), gbuf: n_gbuf planes of H*W (required
 * when n_gbuf > 0). State in the layout above, d = wrls_oracle_ext_dim(prm).
 * out: 3 planes of doubles. w_out (H*W) and valid_out (H*W) are optional.
 * Returns 0, or -1 on an invalid argument.
 */
int wrls_oracle_ext_frame(const wrls_oracle_ext_params* prm, int W, int H, int reset_all,
                          const double* beta_prev, const double* P_prev, const double* z_prev,
                          const float* rad, const float* mot, const float* var, const float* gbuf,
                          double* beta_next, double* P_next, double* z_next,
                          double* out, double* w_out, unsigned char* valid_out) {
    if (!prm || W <= 0 || H <= 0 || !rad || !mot || !beta_next || !P_next || !z_next || !out)
        return -1;
    if (prm->n_gbuf < 0 || prm->n_gbuf > 4 || prm->weight_mode < 0 || prm->weight_mode > 2)
        return -1;
    if ((prm->n_gbuf > 0 && !gbuf) || (prm->weight_mode == 2 && !var)) return -1;
    if (!reset_all && (!beta_prev || !P_prev || !z_prev)) return -1;
    const long n_pix = (long)W * (long)H;
    const int d = wrls_oracle_ext_dim(prm);

#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const long j = (long)y * W + x;
            double I[3] = {rad[j], rad[n_pix + j], rad[2 * n_pix + j]};
            const int missing = !xfinite3(I);

            /* reprojection q = j + v_j, in binary32 (Table 2, Sec. 5.3) */
            float qx = (float)x + mot[j];
            float qy = (float)y + mot[n_pix + j];
            int valid = !reset_all && qx >= 0.0f && qx <= (float)(W - 1) &&
                        qy >= 0.0f && qy <= (float)(H - 1);

            double beta[XNCH][XDMAX], P[XDMAX][XDMAX], zq[3];
            if (valid) {
                long tap[4];
                double wt[4];
                int ntap;
                if (prm->reproj_filter == 1) {
                    int xn = (int)floorf(qx + 0.5f), yn = (int)floorf(qy + 0.5f);
                    tap[0] = (long)yn * W + xn;
                    wt[0] = 1.0;
                    ntap = 1;
                } else {
                    int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
                    double fx = (double)qx - (double)x0, fy = (double)qy - (double)y0;
                    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
                    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
                    tap[0] = (long)y0 * W + x0;
                    tap[1] = (long)y0 * W + x1;
                    tap[2] = (long)y1 * W + x0;
                    tap[3] = (long)y1 * W + x1;
                    wt[0] = (1.0 - fx) * (1.0 - fy);
                    wt[1] = fx * (1.0 - fy);
                    wt[2] = (1.0 - fx) * fy;
                    wt[3] = fx * fy;
                    ntap = 4;
                }
                for (int c = 0; c < XNCH; ++c)
                    for (int a = 0; a < XDMAX; ++a) {
                        double acc = 0.0;
                        if (a < d)
                            for (int k = 0; k < ntap; ++k) acc += wt[k] * beta_prev[tap[k] * 3 * d + c * d + a];
                        beta[c][a] = acc;
                    }
                for (int a = 0; a < XDMAX; ++a)
                    for (int b = 0; b < XDMAX; ++b) {
                        double acc = 0.0;
                        if (a < d && b < d)
                            for (int k = 0; k < ntap; ++k) acc += wt[k] * P_prev[tap[k] * d * d + a * d + b];
                        P[a][b] = acc;
                    }
                for (int c = 0; c < 3; ++c) {
                    double acc = 0.0;
                    for (int k = 0; k < ntap; ++k) acc += wt[k] * z_prev[tap[k] * 3 + c];
                    zq[c] = acc;
                }
            }

            /* temporal feature, Eq. 12 */
            double z[3];
            if (valid) {
                double zc[3] = {zq[0], zq[1], zq[2]};
                if (prm->clamp_mode == 0) {
                    double lo[3] = {INFINITY, INFINITY, INFINITY};
                    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                    int any = 0;
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int xx = x + dx, yy = y + dy;
                            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                            long jj = (long)yy * W + xx;
                            double In[3] = {rad[jj], rad[n_pix + jj], rad[2 * n_pix + jj]};
                            if (!xfinite3(In)) continue;
                            any = 1;
                            for (int c = 0; c < 3; ++c) {
                                if (In[c] < lo[c]) lo[c] = In[c];
                                if (In[c] > hi[c]) hi[c] = In[c];
                            }
                        }
                    if (any)
                        for (int c = 0; c < 3; ++c) {
                            if (zc[c] < lo[c]) zc[c] = lo[c];
                            if (zc[c] > hi[c]) zc[c] = hi[c];
                        }
                }
                for (int c = 0; c < 3; ++c)
                    z[c] = missing ? zc[c] : prm->alpha * zc[c] + (1.0 - prm->alpha) * I[c];
            } else {
                for (int c = 0; c < 3; ++c) z[c] = missing ? 0.0 : I[c];
                xinitial_model(prm, z, beta, P);
            }

            /* predictor p = [1, z, g] of frame t */
            double g[4] = {0, 0, 0, 0};
            for (int i = 0; i < prm->n_gbuf; ++i) g[i] = gbuf[(long)i * n_pix + j];
            double p[XDMAX];
            const int g_ok = xpredictor(prm, z, g, p);

            /* weight: Eq. 13, w = 1 (RLS, Eq. 10) or the sample-variance weight */
            double w;
            if (missing || !g_ok) {
                w = 0.0;
            } else if (prm->weight_mode == 1) {
                w = 1.0;
            } else if (prm->weight_mode == 2) {
                double v = var[j];
                if (!isfinite(v) || v < 0.0) {
                    w = 0.0;
                } else {
                    double m = xeq13_scale(I, z, prm->eps);
                    double dv2 = 3.0 * v / (m * m);
                    w = exp(-dv2 / (prm->h * prm->h));
                }
            } else {
                double diff[3] = {I[0] - z[0], I[1] - z[1], I[2] - z[2]};
                double dist = xnorm3(diff) / xeq13_scale(I, z, prm->eps);
                w = exp(-(dist * dist) / (prm->h * prm->h));
            }

            /* Eq. 14 gain, Eq. 8 residual, Eq. 9 and Eq. 11 updates */
            double Pp[XDMAX], pP[XDMAX], pPp = 0.0;
            for (int a = 0; a < d; ++a) {
                Pp[a] = 0.0;
                for (int b = 0; b < d; ++b) Pp[a] += P[a][b] * p[b];
            }
            for (int b = 0; b < d; ++b) {
                pP[b] = 0.0;
                for (int a = 0; a < d; ++a) pP[b] += p[a] * P[a][b];
            }
            for (int a = 0; a < d; ++a) pPp += p[a] * Pp[a];
            double q[XDMAX];
            for (int a = 0; a < XDMAX; ++a) q[a] = 0.0;
            if (w > 0.0) {
                double denom = prm->lambda / w + pPp;
                for (int a = 0; a < d; ++a) q[a] = Pp[a] / denom;
            }
            for (int c = 0; c < XNCH; ++c) {
                double pred = 0.0;
                for (int a = 0; a < d; ++a) pred += p[a] * beta[c][a];
                double e = (missing || !g_ok) ? 0.0 : I[c] - pred;
                for (int a = 0; a < d; ++a) beta[c][a] += q[a] * e;
            }
            double Pn[XDMAX][XDMAX];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) Pn[a][b] = (P[a][b] - q[a] * pP[b]) / prm->lambda;
            if (prm->p_trace_max > 0.0) {
                double tr = 0.0;
                int bad = 0;
                for (int a = 0; a < d; ++a) {
                    tr += Pn[a][a];
                    if (!(Pn[a][a] > 0.0)) bad = 1;
                }
                if (bad || tr > prm->p_trace_max)
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) Pn[a][b] = a == b ? prm->p0_delta : 0.0;
            }

            for (int c = 0; c < XNCH; ++c)
                for (int a = 0; a < d; ++a) beta_next[j * 3 * d + c * d + a] = beta[c][a];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) P_next[j * d * d + a * d + b] = Pn[a][b];
            for (int c = 0; c < 3; ++c) z_next[j * 3 + c] = z[c];
            if (w_out) w_out[j] = w;
            if (valid_out) valid_out[j] = (unsigned char)valid;
        }
    }
    return wrls_oracle_ext_blend(prm, W, H, beta_next, z_next, gbuf, out);
}

/* Blend over the (2r+1)^2 window: out_i = sum_k b_ik (p_i beta_k) / sum_k b_ik (or p_k
 * beta_k with blend_mode 1), b_ik = exp(-|dx|^2 / (2 sigma_s^2)) exp(-d_z^2 / h_s^2). */
int wrls_oracle_ext_blend(const wrls_oracle_ext_params* prm, int W, int H, const double* beta,
                          const double* z, const float* gbuf, double* out) {
    if (!prm || W <= 0 || H <= 0 || !beta || !z || !out) return -1;
    if (prm->n_gbuf > 0 && !gbuf) return -1;
    const long n_pix = (long)W * (long)H;
    const int d = wrls_oracle_ext_dim(prm);
    const int r = prm->radius;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long i = (long)y * W + x;
            const double* zi = &z[i * 3];
            double gi[4] = {0, 0, 0, 0};
            for (int n = 0; n < prm->n_gbuf; ++n) gi[n] = gbuf[(long)n * n_pix + i];
            double pi_[XDMAX];
            xpredictor(prm, zi, gi, pi_);
            double num[3] = {0, 0, 0}, den = 0.0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int xx = x + dx, yy = y + dy;
                    if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                    const long k = (long)yy * W + xx;
                    const double* zk = &z[k * 3];
                    double diff[3] = {zi[0] - zk[0], zi[1] - zk[1], zi[2] - zk[2]};
                    double dz = xnorm3(diff) / xeq13_scale(zi, zk, prm->eps);
                    double b = exp(-(double)(dx * dx + dy * dy) / (2.0 * prm->sigma_s * prm->sigma_s)) *
                               exp(-(dz * dz) / (prm->h_s * prm->h_s));
                    double gk[4] = {0, 0, 0, 0};
                    for (int n = 0; n < prm->n_gbuf; ++n) gk[n] = gbuf[(long)n * n_pix + k];
                    double pk[XDMAX];
                    xpredictor(prm, zk, gk, pk);
                    const double* pu = prm->blend_mode == 0 ? pi_ : pk;
                    for (int c = 0; c < 3; ++c) {
                        double pred = 0.0;
                        for (int a = 0; a < d; ++a) pred += pu[a] * beta[k * 3 * d + c * d + a];
                        num[c] += b * pred;
                    }
                    den += b;
                }
            for (int c = 0; c < 3; ++c) out[c * n_pix + i] = num[c] / den;
        }
    return 0;
}
