/*
 * wRLS denoiser ORACLE -- test infrastructure only.
 *
 * A plain, slow, double-precision CPU restatement of the per-frame denoiser of
 * Iglesias-Guitian, Mane, Moon, "Real-Time Denoising of Volumetric Path Tracing for
 * Direct Volume Rendering" (IEEE TVCG 2020), Sec. 5.1-5.3. It exists only to check
 * the CUDA library against; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it. It shares no code, header or constant table with the
 * CUDA path (paper_2106_08034_gb300/csrc) and includes none of its files.
 *
 * Per frame t and pixel j, in the paper's order:
 *   1. reprojection q = pi(v_j) = j + v_j (Table 2, Sec. 5.3) and fetch of the
 *      previous linear model (beta, P) and temporal feature z at q;
 *   2. temporal feature, Eq. 12: z_j(t) = alpha * Psi[z_q(t-1), I~_j(t)] + (1-alpha) I~_j(t),
 *      Psi = neighbourhood clamp to the current frame;
 *   3. weight, Eq. 13;
 *   4. residual Eq. 8, gain Eq. 14 (Eq. 10 when w == 1), coefficients Eq. 9,
 *      inverse covariance Eq. 11, with predictor p = [1, z] (Sec. 5.1, Eq. 5);
 * then per pixel i:
 *   5. spatio-temporal blend (Sec. 5.3, last paragraph): bilateral-weighted average
 *      over a 5x5 window of the colours that the neighbours' linear models predict
 *      for pixel i.
 *
 * Readings where the paper is silent:
 *   - one scalar weight per pixel, L2 norms over RGB in Eq. 13;
 *   - one P per pixel shared by the three colour channels (p and w do not depend on
 *     the channel, so Eq. 11 evolves identically for R, G and B);
 *   - initial model beta = 0 and P = p0_delta * I (the usual start of an RLS
 *     recursion); a switch selects the feature pass-through start beta_c = e_{c+1}
 *     (prediction = z_c; beta_c = z_c when p = [1]);
 *   - reprojection: q computed in binary32 as (float)x + v_x, valid iff
 *     0 <= q <= dim-1 per axis, bilinear fetch of all state values with the upper
 *     taps clamped; an invalid q (or frame 0 / reset) restarts the pixel with the
 *     initial model and z = I~;
 *   - Psi: per-channel min/max of I~ over the 3x3 neighbours inside the image;
 *   - blend weight: exp(-|dx|^2 / (2 sigma_s^2)) * exp(-d_z^2 / h_s^2) with d_z the
 *     Eq. 13 distance between the two pixels' features; out-of-image neighbours are
 *     skipped; the blend uses the models after the frame-t update;
 *   - a sample with a non-finite channel is missing: it is skipped by Psi, it does
 *     not enter z (z = clamped history), and its weight is 0 (beta unchanged,
 *     P <- P / lambda);
 *   - optional wind-up guard (off by default): P <- P0 when trace(P) > p_trace_max or
 *     a diagonal entry is <= 0.
 *
 * Parity pins for this file live in tests/test_oracle_*.py (closed forms, brute-force
 * least squares, invariants). Nothing here is blocked, fused or reordered.
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
    int radius;         /* blend window radius: 2 -> 5x5 (Sec. 5.3); 0 -> temporal only */
    int weight_mode;    /* 0 = wRLS (Eq. 13, 14); 1 = RLS (w = 1, Eq. 10) */
    int clamp_mode;     /* 0 = 3x3 clamp; 1 = no clamp */
    int blend_mode;     /* 0 = neighbours' models predict pixel i (p_i beta_k);
                           1 = neighbours' own predictions (p_k beta_k) */
    int feature_mode;   /* 0 = p = [1, z] (d = 4); 1 = p = [1] (d = 1, no feature) */
    int init_mode;      /* 0 = beta = 0 (the usual RLS start); 1 = feature pass-through:
                           beta_c = e_{c+1}, or beta_c = z_c when p = [1] */
} wrls_oracle_params;

#define NCH 3
#define DMAX 4

static int oracle_dim(const wrls_oracle_params* prm) { return prm->feature_mode == 1 ? 1 : 4; }

static int is_finite3(const double v[3]) {
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* Eq. 13 distance between two colour vectors. */
static double eq13_distance(const double a[3], const double b[3], double eps) {
    double diff[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
    double na = norm3(a), nb = norm3(b);
    double m = na < nb ? na : nb;
    return norm3(diff) / (m + eps);
}

/* Predictor vector p = [1, z] (Sec. 5.1) or [1] without feature. */
static void predictor(const wrls_oracle_params* prm, const double z[3], double p[DMAX]) {
    p[0] = 1.0;
    if (prm->feature_mode == 0) { p[1] = z[0]; p[2] = z[1]; p[3] = z[2]; }
}

/* Initial model of a (re)started pixel. */
static void initial_model(const wrls_oracle_params* prm, const double z[3],
                          double beta[NCH][DMAX], double P[DMAX][DMAX]) {
    int d = oracle_dim(prm);
    for (int c = 0; c < NCH; ++c)
        for (int a = 0; a < DMAX; ++a) beta[c][a] = 0.0;
    if (prm->init_mode == 0) {
        /* zero model: every coefficient starts at 0 */
    } else if (d == 4) {
        for (int c = 0; c < NCH; ++c) beta[c][c + 1] = 1.0;
    } else {
        for (int c = 0; c < NCH; ++c) beta[c][0] = z[c];
    }
    for (int a = 0; a < DMAX; ++a)
        for (int b = 0; b < DMAX; ++b) P[a][b] = (a == b && a < d) ? prm->p0_delta : 0.0;
}

int wrls_oracle_blend(const wrls_oracle_params* prm, int W, int H,
                      const double* beta, const double* z, double* out);

/*
 * One frame.
 *   state layout (per pixel n = y*W + x):
 *     beta[n*12 + c*4 + a]   (channel c, coefficient a)
 *     P   [n*16 + a*4 + b]   (full 4x4; only the leading d x d block is used)
 *     z   [n*3 + c]
 *   rad: 3 planes of H*W binary32 (planar RGB); mot: 2 planes (vx, vy).
 *   reset_all != 0: every pixel restarts (first frame of a stream or an explicit reset).
 *   out: 3 planes of H*W doubles. w_out (H*W) and valid_out (H*W) are optional.
 * Returns 0, or -1 on an invalid argument.
 */
int wrls_oracle_frame(const wrls_oracle_params* prm, int W, int H, int reset_all,
                      const double* beta_prev, const double* P_prev, const double* z_prev,
                      const float* rad, const float* mot,
                      double* beta_next, double* P_next, double* z_next,
                      double* out, double* w_out, unsigned char* valid_out) {
    if (!prm || W <= 0 || H <= 0 || !rad || !mot || !beta_next || !P_next || !z_next || !out)
        return -1;
    if (!reset_all && (!beta_prev || !P_prev || !z_prev)) return -1;
    const long n_pix = (long)W * (long)H;
    const int d = oracle_dim(prm);

    /* ---- steps 1-4: per-pixel temporal update ---- */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const long j = (long)y * W + x;
            double I[3] = {rad[0 * n_pix + j], rad[1 * n_pix + j], rad[2 * n_pix + j]};
            const int missing = !is_finite3(I);

            /* 1. reprojection q = j + v_j, in binary32 */
            float qx = (float)x + mot[0 * n_pix + j];
            float qy = (float)y + mot[1 * n_pix + j];
            int valid = !reset_all && qx >= 0.0f && qx <= (float)(W - 1) &&
                        qy >= 0.0f && qy <= (float)(H - 1);

            double beta[NCH][DMAX], P[DMAX][DMAX], zq[3];
            if (valid) {
                int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
                double fx = (double)qx - (double)x0, fy = (double)qy - (double)y0;
                int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
                int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
                const long tap[4] = {(long)y0 * W + x0, (long)y0 * W + x1,
                                     (long)y1 * W + x0, (long)y1 * W + x1};
                const double wt[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy),
                                      (1.0 - fx) * fy, fx * fy};
                for (int c = 0; c < NCH; ++c)
                    for (int a = 0; a < DMAX; ++a) {
                        double acc = 0.0;
                        for (int k = 0; k < 4; ++k) acc += wt[k] * beta_prev[tap[k] * 12 + c * 4 + a];
                        beta[c][a] = acc;
                    }
                for (int a = 0; a < DMAX; ++a)
                    for (int b = 0; b < DMAX; ++b) {
                        double acc = 0.0;
                        for (int k = 0; k < 4; ++k) acc += wt[k] * P_prev[tap[k] * 16 + a * 4 + b];
                        P[a][b] = acc;
                    }
                for (int c = 0; c < NCH; ++c) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; ++k) acc += wt[k] * z_prev[tap[k] * 3 + c];
                    zq[c] = acc;
                }
            }

            /* 2. temporal feature, Eq. 12 */
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
                            if (!is_finite3(In)) continue;
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
                initial_model(prm, z, beta, P);
            }

            /* 3. weight, Eq. 13 (w = 1: plain RLS, Eq. 10) */
            double w;
            if (missing) w = 0.0;
            else if (prm->weight_mode == 1) w = 1.0;
            else {
                double dist = eq13_distance(I, z, prm->eps);
                w = exp(-(dist * dist) / (prm->h * prm->h));
            }

            /* 4. wRLS update with p = [1, z] */
            double p[DMAX] = {0, 0, 0, 0};
            predictor(prm, z, p);
            double Pp[DMAX], pP[DMAX], pPp = 0.0;
            for (int a = 0; a < d; ++a) {
                Pp[a] = 0.0;
                for (int b = 0; b < d; ++b) Pp[a] += P[a][b] * p[b];
            }
            for (int b = 0; b < d; ++b) {
                pP[b] = 0.0;
                for (int a = 0; a < d; ++a) pP[b] += p[a] * P[a][b];
            }
            for (int a = 0; a < d; ++a) pPp += p[a] * Pp[a];
            /* Eq. 14: q^w = P p / (lambda / w + p P p); w = 0 gives q = 0 */
            double q[DMAX] = {0, 0, 0, 0};
            if (w > 0.0) {
                double denom = prm->lambda / w + pPp;
                for (int a = 0; a < d; ++a) q[a] = Pp[a] / denom;
            }
            for (int c = 0; c < NCH; ++c) {
                /* Eq. 8: e = I~ - p beta(t-1) */
                double pred = 0.0;
                for (int a = 0; a < d; ++a) pred += p[a] * beta[c][a];
                double e = missing ? 0.0 : I[c] - pred;
                /* Eq. 9: beta(t) = beta(t-1) + q e */
                for (int a = 0; a < d; ++a) beta[c][a] += q[a] * e;
            }
            /* Eq. 11: P(t) = (P(t-1) - q p P(t-1)) / lambda */
            double Pn[DMAX][DMAX];
            for (int a = 0; a < DMAX; ++a)
                for (int b = 0; b < DMAX; ++b)
                    Pn[a][b] = (a < d && b < d) ? (P[a][b] - q[a] * pP[b]) / prm->lambda : 0.0;
            if (prm->p_trace_max > 0.0) {
                double tr = 0.0;
                int bad = 0;
                for (int a = 0; a < d; ++a) {
                    tr += Pn[a][a];
                    if (!(Pn[a][a] > 0.0)) bad = 1;
                }
                if (bad || tr > prm->p_trace_max)
                    for (int a = 0; a < DMAX; ++a)
                        for (int b = 0; b < DMAX; ++b)
                            Pn[a][b] = (a == b && a < d) ? prm->p0_delta : 0.0;
            }

            for (int c = 0; c < NCH; ++c)
                for (int a = 0; a < DMAX; ++a) beta_next[j * 12 + c * 4 + a] = beta[c][a];
            for (int a = 0; a < DMAX; ++a)
                for (int b = 0; b < DMAX; ++b) P_next[j * 16 + a * 4 + b] = Pn[a][b];
            for (int c = 0; c < 3; ++c) z_next[j * 3 + c] = z[c];
            if (w_out) w_out[j] = w;
            if (valid_out) valid_out[j] = (unsigned char)valid;
        }
    }

    /* ---- step 5: spatio-temporal blend over the (2r+1)^2 window ---- */
    return wrls_oracle_blend(prm, W, H, beta_next, z_next, out);
}

/* Step 5 on a given state: out_i = sum_k b_ik pred_k(i) / sum_k b_ik over the window. */
int wrls_oracle_blend(const wrls_oracle_params* prm, int W, int H,
                      const double* beta, const double* z, double* out) {
    if (!prm || W <= 0 || H <= 0 || !beta || !z || !out) return -1;
    const long n_pix = (long)W * (long)H;
    const int d = oracle_dim(prm);
    const int r = prm->radius;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long i = (long)y * W + x;
            const double* zi = &z[i * 3];
            double pi_[DMAX] = {0, 0, 0, 0};
            predictor(prm, zi, pi_);
            double num[3] = {0, 0, 0}, den = 0.0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int xx = x + dx, yy = y + dy;
                    if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                    const long k = (long)yy * W + xx;
                    double dz = eq13_distance(zi, &z[k * 3], prm->eps);
                    double b = exp(-(double)(dx * dx + dy * dy) / (2.0 * prm->sigma_s * prm->sigma_s)) *
                               exp(-(dz * dz) / (prm->h_s * prm->h_s));
                    double pk[DMAX] = {0, 0, 0, 0};
                    predictor(prm, &z[k * 3], pk);
                    const double* pu = prm->blend_mode == 0 ? pi_ : pk;
                    for (int c = 0; c < 3; ++c) {
                        double pred = 0.0;
                        for (int a = 0; a < d; ++a) pred += pu[a] * beta[k * 12 + c * 4 + a];
                        num[c] += b * pred;
                    }
                    den += b;
                }
            for (int c = 0; c < 3; ++c) out[c * n_pix + i] = num[c] / den;
        }
    return 0;
}

void wrls_oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int wrls_oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
