/*
 * wRLS denoiser ORACLE, inputs of the denoiser -- test infrastructure only.
 *
 * Same rules as wrls_oracle.c (only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it; it shares no code with the CUDA path). Plain FP64 C
 * restatements of the two steps that produce the denoiser's per-frame inputs in the
 * paper's renderer (Iglesias-Guitian, Mane, Moon, IEEE TVCG 2020):
 *
 *   1. pixel reconstruction filter (Sec. 4, Table 2: the light-path contributions f_j of
 *      pixel j are filtered into the estimate I~_j; Sec. 6: a separable Gaussian kernel):
 *        I~_j = sum_k g(x_k - x_j) g(y_k - y_j) f_k / sum_k g(x_k - x_j) g(y_k - y_j)
 *      over the samples k of the 3x3 pixels around j, at their positions x_k (pixel centre
 *      + offset), g(d) = exp(-d^2 / (2 sigma^2)) for |d| <= radius, else 0;
 *   2. per-pixel velocity (Sec. 5.3, Sec. 6 "Optical flow estimation"): the world position
 *      X_j of the first real collision along pixel j's ray is projected with the previous
 *      frame's view-projection matrix; v_j = pi_{t-1}(X_j) - j.
 *
 * Readings where the paper is silent:
 *   - samples: spp per pixel, each an RGB value and an offset (ox, oy) in [-0.5, 0.5] from
 *     the pixel centre; planar layout ((s * 5 + k) * H + y) * W + x, k = r, g, b, ox, oy;
 *   - sigma = 0.5 px and radius = 1.5 px by default (with offsets in [-0.5, 0.5] the 3x3
 *     window holds every sample within 1.5 px); the support test |d| <= radius is taken in
 *     binary32 on d = (float)(x_p - x_j) + ox, as the GPU takes it;
 *   - a sample with a non-finite colour or offset is skipped; a pixel whose window holds no
 *     weight gets a non-finite estimate (the denoiser then treats it as a missing sample);
 *   - variance (optional output): the unbiased sample variance of pixel j's own valid
 *     samples, averaged over the three channels and divided by their count (the variance
 *     of the pixel mean); NaN with fewer than two valid samples;
 *   - projection: clip = M [X, Y, Z, 1]^T with M the 4x4 row-major view-projection matrix of
 *     frame t-1; pixel coordinates ((clip_x / clip_w + 1) W / 2 - 0.5,
 *     (1 - clip_y / clip_w) H / 2 - 0.5) (pixel centres at integers, row 0 at the top);
 *     clip_w <= 0 (behind the previous camera) gives NaN motion (the denoiser restarts);
 *     a pixel without a collision (non-finite X) gets v = 0 (miss_policy 0) or NaN
 *     (miss_policy 1).
 *
 * Pins: tests/test_oracle_upstream_pins.py.
 */
#include <math.h>
#include <stddef.h>

/* Step 1. out: 3 planes of doubles; var (optional): 1 plane. Returns 0 or -1. */
int wrls_oracle_reconstruct(int W, int H, int spp, const float* samples, double sigma, double radius,
                            double* out, double* var) {
    if (W <= 0 || H <= 0 || spp <= 0 || !samples || !out || !(sigma > 0.0) || !(radius > 0.0)) return -1;
    const long np = (long)W * H;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
            for (int py = y - 1; py <= y + 1; ++py)
                for (int px = x - 1; px <= x + 1; ++px) {
                    if (px < 0 || px >= W || py < 0 || py >= H) continue;
                    const long p = (long)py * W + px;
                    for (int s = 0; s < spp; ++s) {
                        const float* base = samples + (long)s * 5 * np;
                        double f[3] = {base[p], base[np + p], base[2 * np + p]};
                        if (!isfinite(f[0]) || !isfinite(f[1]) || !isfinite(f[2])) continue;
                        if (!isfinite(base[3 * np + p]) || !isfinite(base[4 * np + p])) continue;
                        float dx = (float)(px - x) + base[3 * np + p];
                        float dy = (float)(py - y) + base[4 * np + p];
                        if (fabsf(dx) > (float)radius || fabsf(dy) > (float)radius) continue;
                        double g = exp(-((double)dx * dx) / (2.0 * sigma * sigma)) *
                                   exp(-((double)dy * dy) / (2.0 * sigma * sigma));
                        for (int c = 0; c < 3; ++c) num[c] += g * f[c];
                        den += g;
                    }
                }
            const long j = (long)y * W + x;
            for (int c = 0; c < 3; ++c) out[c * np + j] = den > 0.0 ? num[c] / den : NAN;
            if (var) {
                double mean[3] = {0, 0, 0};
                int n = 0;
                for (int s = 0; s < spp; ++s) {
                    const float* base = samples + (long)s * 5 * np;
                    double f[3] = {base[j], base[np + j], base[2 * np + j]};
                    if (!isfinite(f[0]) || !isfinite(f[1]) || !isfinite(f[2])) continue;
                    if (!isfinite(base[3 * np + j]) || !isfinite(base[4 * np + j])) continue;
                    for (int c = 0; c < 3; ++c) mean[c] += f[c];
                    ++n;
                }
                if (n < 2) {
                    var[j] = NAN;
                    continue;
                }
                for (int c = 0; c < 3; ++c) mean[c] /= n;
                double ss = 0.0;
                for (int s = 0; s < spp; ++s) {
                    const float* base = samples + (long)s * 5 * np;
                    double f[3] = {base[j], base[np + j], base[2 * np + j]};
                    if (!isfinite(f[0]) || !isfinite(f[1]) || !isfinite(f[2])) continue;
                    if (!isfinite(base[3 * np + j]) || !isfinite(base[4 * np + j])) continue;
                    for (int c = 0; c < 3; ++c) ss += (f[c] - mean[c]) * (f[c] - mean[c]);
                }
                var[j] = ss / (3.0 * (n - 1)) / n;
            }
        }
    return 0;
}

/* Step 2. world: 3 planes (X, Y, Z) of frame t; M: 16 values, row-major; mot: 2 planes. */
int wrls_oracle_velocity(int W, int H, const float* world, const double* M, int miss_policy, double* mot) {
    if (W <= 0 || H <= 0 || !world || !M || !mot || miss_policy < 0 || miss_policy > 1) return -1;
    const long np = (long)W * H;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long j = (long)y * W + x;
            const double X[4] = {world[j], world[np + j], world[2 * np + j], 1.0};
            double vx, vy;
            if (!isfinite(X[0]) || !isfinite(X[1]) || !isfinite(X[2])) {
                vx = vy = miss_policy == 0 ? 0.0 : NAN;
            } else {
                double clip[4];
                for (int r = 0; r < 4; ++r) {
                    clip[r] = 0.0;
                    for (int c = 0; c < 4; ++c) clip[r] += M[r * 4 + c] * X[c];
                }
                if (!(clip[3] > 0.0)) {
                    vx = vy = NAN;
                } else {
                    double px = (clip[0] / clip[3] + 1.0) * 0.5 * W - 0.5;
                    double py = (1.0 - clip[1] / clip[3]) * 0.5 * H - 0.5;
                    vx = px - x;
                    vy = py - y;
                }
            }
            mot[j] = vx;
            mot[np + j] = vy;
        }
    return 0;
}
