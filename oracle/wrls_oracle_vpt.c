/*
 * Volumetric path tracer ORACLE -- test infrastructure only.
 *
 * Same rules as wrls_oracle.c (only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it; it shares no code with the CUDA path). A plain FP64 C
 * restatement of the renderer that produces the denoiser's inputs (Iglesias-Guitian, Mane,
 * Moon, IEEE TVCG 2020, Sec. 3 and Sec. 6): progressive volumetric path tracing of a
 * heterogeneous medium with delta tracking.
 *
 *   - Eq. 1 / Eq. 3: one path per sample, built incrementally from the camera (Fig. 2-3);
 *     at every real collision y the path's throughput is multiplied by the single-scattering
 *     albedo mu_s / mu_t (the collision estimator of Eq. 3 with rho(y) proportional to
 *     mu_t T), the in-scattered light L_s(y) is estimated by connecting y to the light
 *     (next-event estimation, isotropic phase function 1 / (4 pi), Sec. 3), and a new
 *     direction is drawn from the phase function; a path that leaves the volume picks up
 *     the background radiance (the last term of Eq. 1).
 *   - Eq. 4: free paths by delta tracking with the majorant mu_t^max; a tentative collision
 *     at y is real with probability mu_t(y) / mu_t^max, null otherwise. The visibility of
 *     the light from y is estimated the same way (1 if the shadow ray leaves the volume
 *     before a real collision, else 0).
 *   - Sec. 6: the first real collision's world position (the one closest to the viewer
 *     among the pixel's samples) is kept for the velocity estimate.
 *
 * Readings where the paper is silent (it renders CT datasets with Exposure Render):
 *   - volume: the box [-1, 1]^3; density rho(x) = min(1, sum_i a_i exp(-|x - c_i|^2 /
 *     (2 r_i^2))) inside it, 0 outside; transfer function: opacity = clamp((rho - lo) /
 *     (hi - lo), 0, 1), mu_t = mu_max * opacity (so mu_max is the majorant), albedo colour
 *     = albedo * (color_lo + rho (color_hi - color_lo)) per channel;
 *   - lights: one directional light (direction towards the light, radiance per channel)
 *     and a uniform environment radiance; next-event estimation at every real collision;
 *     a path ends after max_bounces real collisions (contributing nothing further);
 *   - camera: ray from `eye` through the point inv_view_proj [ndc_x, ndc_y, 1, 1] (row-major,
 *     dehomogenised) with ndc = ((x + 0.5 + ox) / W * 2 - 1, 1 - (y + 0.5 + oy) / H * 2),
 *     sub-pixel offsets ox, oy = u - 0.5 from the first two random numbers;
 *   - random numbers: Philox4x32-10 (Salmon et al., SC 2011) with counter (pixel index,
 *     sample index, frame, block) and key seed; the path consumes the four 32-bit outputs
 *     of each block in order, then the next block; u = (bits >> 8) * 2^-24 in [0, 1).
 *     Consumption order: ox, oy; per tentative collision: the free path, then the
 *     acceptance; per real collision: the shadow ray's tentative collisions (free path,
 *     acceptance each), then the two direction numbers (z = 1 - 2u, phi = 2 pi u');
 *   - a path makes at most 2^20 tentative collisions (primary and shadow rays together);
 *     reaching the cap ends it with what it has gathered (a shadow ray then counts as
 *     blocked);
 *   - G-buffers of the closest first collision: depth (distance from the eye), normal
 *     (-grad rho / |grad rho|, analytic, 0 where the gradient vanishes), albedo colour; all
 *     0 for a pixel whose samples found no collision, whose world position is NaN.
 * Pins: tests/test_oracle_vpt_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define VPT_PI 3.14159265358979323846
#define VPT_MAX_STEPS (1 << 20)

typedef struct {
    uint32_t seed[2];
    float eye[3];
    float inv_view_proj[16];
    int n_blobs;
    float blobs[16][5]; /* cx, cy, cz, radius, amplitude */
    float mu_max;
    float tf_lo, tf_hi;
    float albedo;
    float color_lo[3], color_hi[3];
    float light_dir[3]; /* unit vector towards the light */
    float light_rgb[3];
    float env_rgb[3];
    int max_bounces;
} wrls_oracle_vpt_scene;

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) ---- */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void wrls_oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox4x32_10(ctr, key, out); }

typedef struct {
    uint32_t ctr[4], key[2], buf[4];
    int used;
    int steps; /* tentative collisions of the path so far */
} rng_t;

static double rng_u(rng_t* g) {
    if (g->used == 4) {
        philox4x32_10(g->ctr, g->key, g->buf);
        g->ctr[3] += 1u;
        g->used = 0;
    }
    uint32_t b = g->buf[g->used++];
    return (double)(b >> 8) * (1.0 / 16777216.0);
}

static double density(const wrls_oracle_vpt_scene* sc, const double p[3]) {
    if (fabs(p[0]) > 1.0 || fabs(p[1]) > 1.0 || fabs(p[2]) > 1.0) return 0.0;
    double s = 0.0;
    for (int i = 0; i < sc->n_blobs; ++i) {
        double dx = p[0] - sc->blobs[i][0], dy = p[1] - sc->blobs[i][1], dz = p[2] - sc->blobs[i][2];
        double r = sc->blobs[i][3];
        s += sc->blobs[i][4] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * r * r));
    }
    return s < 1.0 ? s : 1.0;
}

static double opacity(const wrls_oracle_vpt_scene* sc, double rho) {
    double o = (rho - sc->tf_lo) / ((double)sc->tf_hi - sc->tf_lo);
    return o < 0.0 ? 0.0 : (o > 1.0 ? 1.0 : o);
}

/* Distance interval [t0, t1] of the ray o + t d inside [-1, 1]^3 with t >= 0; 0 if none. */
static int box_interval(const double o[3], const double d[3], double* t0, double* t1) {
    double lo = 0.0, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double inv = 1.0 / d[a];
        double ta = (-1.0 - o[a]) * inv, tb = (1.0 - o[a]) * inv;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > lo) lo = ta;
        if (tb < hi) hi = tb;
    }
    *t0 = lo;
    *t1 = hi;
    return lo < hi;
}

/* Delta-tracking visibility from p along the unit direction w: 1 if the ray leaves the box
 * before a real collision. */
static int visible(const wrls_oracle_vpt_scene* sc, rng_t* g, const double p[3], const double w[3]) {
    double t0, t1;
    if (!box_interval(p, w, &t0, &t1)) return 1;
    double t = t0;
    for (;;) {
        if (++g->steps > VPT_MAX_STEPS) return 0;
        t += -log(1.0 - rng_u(g)) / sc->mu_max;
        if (t >= t1) return 1;
        double y[3] = {p[0] + t * w[0], p[1] + t * w[1], p[2] + t * w[2]};
        double mu = sc->mu_max * opacity(sc, density(sc, y));
        if (rng_u(g) < mu / sc->mu_max) return 0;
    }
}

/* One path. Returns its radiance in L; *hit and y_first receive the first real collision. */
static void trace(const wrls_oracle_vpt_scene* sc, rng_t* g, const double eye[3], const double dir[3], double L[3],
                  int* hit, double y_first[3], double* t_first) {
    double beta[3] = {1.0, 1.0, 1.0};
    double x[3] = {eye[0], eye[1], eye[2]}, w[3] = {dir[0], dir[1], dir[2]};
    L[0] = L[1] = L[2] = 0.0;
    *hit = 0;
    double t0, t1;
    if (!box_interval(x, w, &t0, &t1)) {
        for (int c = 0; c < 3; ++c) L[c] = sc->env_rgb[c];
        return;
    }
    double t = t0;
    int bounces = 0;
    for (;;) {
        if (++g->steps > VPT_MAX_STEPS) return;
        t += -log(1.0 - rng_u(g)) / sc->mu_max;
        if (t >= t1) {  /* leaves the volume: background */
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * sc->env_rgb[c];
            return;
        }
        double y[3] = {x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]};
        double rho = density(sc, y);
        double mu = sc->mu_max * opacity(sc, rho);
        if (!(rng_u(g) < mu / sc->mu_max)) continue; /* null collision */
        if (!*hit) {
            *hit = 1;
            for (int c = 0; c < 3; ++c) y_first[c] = y[c];
            *t_first = t; /* the first real collision is on the camera ray: t is its distance */
        }
        for (int c = 0; c < 3; ++c)
            beta[c] *= sc->albedo * (sc->color_lo[c] + rho * ((double)sc->color_hi[c] - sc->color_lo[c]));
        double ld[3] = {sc->light_dir[0], sc->light_dir[1], sc->light_dir[2]};
        if (visible(sc, g, y, ld))
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * sc->light_rgb[c] / (4.0 * VPT_PI);
        if (++bounces >= sc->max_bounces) return;
        double z = 1.0 - 2.0 * rng_u(g), phi = 2.0 * VPT_PI * rng_u(g);
        double r = sqrt(z * z < 1.0 ? 1.0 - z * z : 0.0);
        w[0] = r * cos(phi); w[1] = r * sin(phi); w[2] = z;
        for (int c = 0; c < 3; ++c) x[c] = y[c];
        if (!box_interval(x, w, &t0, &t1)) { t0 = 0.0; t1 = 0.0; }
        t = 0.0;
    }
}

static void grad_density(const wrls_oracle_vpt_scene* sc, const double p[3], double gr[3]) {
    gr[0] = gr[1] = gr[2] = 0.0;
    for (int i = 0; i < sc->n_blobs; ++i) {
        double d[3] = {p[0] - sc->blobs[i][0], p[1] - sc->blobs[i][1], p[2] - sc->blobs[i][2]};
        double r2 = (double)sc->blobs[i][3] * sc->blobs[i][3];
        double e = sc->blobs[i][4] * exp(-(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / (2.0 * r2));
        for (int a = 0; a < 3; ++a) gr[a] += -e * d[a] / r2;
    }
}

/*
 * Render one frame: samples (spp, 5, H, W) f32 (r, g, b, ox, oy), world (3, H, W) f32 of the
 * closest first collision (NaN: none), features (7, H, W) f32 or NULL: depth, normal (3),
 * albedo colour (3) there. Returns 0, or -1 on a bad argument.
 */
int wrls_oracle_render_vpt(const wrls_oracle_vpt_scene* sc, int W, int H, int spp, uint32_t frame, float* samples,
                           float* world, float* features) {
    if (!sc || W <= 0 || H <= 0 || spp <= 0 || !samples || !world || sc->n_blobs < 0 || sc->n_blobs > 16 ||
        !(sc->mu_max > 0.0f) || !(sc->tf_hi > sc->tf_lo) || sc->max_bounces < 1)
        return -1;
    const long np = (long)W * H;
    const double eye[3] = {sc->eye[0], sc->eye[1], sc->eye[2]};
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long j = (long)y * W + x;
            double best_t = INFINITY, best_y[3] = {NAN, NAN, NAN};
            for (int s = 0; s < spp; ++s) {
                rng_t g;
                g.ctr[0] = (uint32_t)j; g.ctr[1] = (uint32_t)s; g.ctr[2] = frame; g.ctr[3] = 0u;
                g.key[0] = sc->seed[0]; g.key[1] = sc->seed[1];
                g.used = 4;
                g.steps = 0;
                double ox = rng_u(&g) - 0.5, oy = rng_u(&g) - 0.5;
                double nd[4] = {((double)x + 0.5 + ox) / W * 2.0 - 1.0, 1.0 - ((double)y + 0.5 + oy) / H * 2.0, 1.0, 1.0};
                double P[4];
                for (int r = 0; r < 4; ++r) {
                    P[r] = 0.0;
                    for (int c = 0; c < 4; ++c) P[r] += (double)sc->inv_view_proj[r * 4 + c] * nd[c];
                }
                double dir[3] = {P[0] / P[3] - eye[0], P[1] / P[3] - eye[1], P[2] / P[3] - eye[2]};
                double n = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
                for (int a = 0; a < 3; ++a) dir[a] /= n;
                double L[3], yf[3], tf = 0.0;
                int hit;
                trace(sc, &g, eye, dir, L, &hit, yf, &tf);
                float* out = samples + (long)s * 5 * np;
                out[j] = (float)L[0];
                out[np + j] = (float)L[1];
                out[2 * np + j] = (float)L[2];
                out[3 * np + j] = (float)ox;
                out[4 * np + j] = (float)oy;
                if (hit && tf < best_t) {
                    best_t = tf;
                    for (int a = 0; a < 3; ++a) best_y[a] = yf[a];
                }
            }
            for (int a = 0; a < 3; ++a) world[a * np + j] = (float)best_y[a];
            if (features) {
                float f[7] = {0, 0, 0, 0, 0, 0, 0};
                if (isfinite(best_t)) {
                    double gr[3];
                    grad_density(sc, best_y, gr);
                    double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                    double rho = density(sc, best_y);
                    f[0] = (float)best_t;
                    for (int a = 0; a < 3; ++a) f[1 + a] = gn > 0.0 ? (float)(-gr[a] / gn) : 0.0f;
                    for (int c = 0; c < 3; ++c)
                        f[4 + c] = (float)(sc->color_lo[c] + rho * ((double)sc->color_hi[c] - sc->color_lo[c]));
                }
                for (int k = 0; k < 7; ++k) features[k * np + j] = f[k];
            }
        }
    return 0;
}
