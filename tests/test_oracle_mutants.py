"""The oracle pins must catch plausible mistakes: each mutant below is a copy of the
oracle source with one planted error (a flipped sign, a dropped term, a swapped index or
operand). Every mutant is compiled on the CPU and must fail at least one pin of
test_oracle_pins.py. Nothing here touches the CUDA library."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "wrls_oracle.c")
SRC_EXT = os.path.join(ROOT, "oracle", "wrls_oracle_ext.c")

MUTANTS = {
    "eq8_residual_sign": ("double e = missing ? 0.0 : I[c] - pred;",
                          "double e = missing ? 0.0 : pred - I[c];"),
    "eq14_lambda_times_w": ("prm->lambda / w + pPp", "prm->lambda * w + pPp"),
    "eq11_no_forgetting": ("(P[a][b] - q[a] * pP[b]) / prm->lambda", "(P[a][b] - q[a] * pP[b])"),
    "eq9_gain_without_denominator": ("beta[c][a] += q[a] * e;", "beta[c][a] += Pp[a] * e;"),
    "eq12_alpha_swapped": ("prm->alpha * zc[c] + (1.0 - prm->alpha) * I[c]",
                           "(1.0 - prm->alpha) * zc[c] + prm->alpha * I[c]"),
    "eq13_max_instead_of_min": ("double m = na < nb ? na : nb;", "double m = na < nb ? nb : na;"),
    "reprojection_sign": ("float qx = (float)x + mot[0 * n_pix + j];",
                          "float qx = (float)x - mot[0 * n_pix + j];"),
    "reprojection_axes_swapped": ("float qy = (float)y + mot[1 * n_pix + j];",
                                  "float qy = (float)y + mot[0 * n_pix + j];"),
    "bilinear_taps_transposed": ("(long)y0 * W + x1,\n                                     (long)y1 * W + x0",
                                 "(long)y1 * W + x0,\n                                     (long)y0 * W + x1"),
    "clamp_window_one_sided": ("for (int dy = -1; dy <= 1; ++dy)", "for (int dy = 0; dy <= 1; ++dy)"),
    "blend_own_prediction": ("const double* pu = prm->blend_mode == 0 ? pi_ : pk;",
                             "const double* pu = pk;"),
    "blend_range_term_dropped": (" *\n                               exp(-(dz * dz) / (prm->h_s * prm->h_s));", ";"),
    "blend_sigma_factor": ("(2.0 * prm->sigma_s * prm->sigma_s)", "(prm->sigma_s * prm->sigma_s)"),
}


# Mistakes planted in the extended oracle (d-generic predictor, variance weight, nearest
# reprojection); caught by test_oracle_ext_pins.py.
MUTANTS_EXT = {
    "variance_weight_channel_factor": ("double dv2 = 3.0 * v / (m * m);", "double dv2 = v / (m * m);"),
    "gbuffer_entries_reversed": ("if (isfinite(g[i])) p[a + i] = g[i];",
                                 "if (isfinite(g[i])) p[a + prm->n_gbuf - 1 - i] = g[i];"),
    "nearest_truncates": ("int xn = (int)floorf(qx + 0.5f)", "int xn = (int)floorf(qx)"),
    "beta_stride_transposed": ("acc += wt[k] * beta_prev[tap[k] * 3 * d + c * d + a];",
                               "acc += wt[k] * beta_prev[tap[k] * 3 * d + a * 3 + c];"),
    "blend_neighbours_gbuffer": ("const double* pu = prm->blend_mode == 0 ? pi_ : pk;",
                                 "const double* pu = pk;"),
    "nonfinite_gbuffer_kept": ("if (missing || !g_ok) {\n                w = 0.0;",
                               "if (missing) {\n                w = 0.0;"),
    "ext_eq11_no_forgetting": ("Pn[a][b] = (P[a][b] - q[a] * pP[b]) / prm->lambda;",
                               "Pn[a][b] = (P[a][b] - q[a] * pP[b]);"),
    "ext_eq14_lambda_times_w": ("double denom = prm->lambda / w + pPp;", "double denom = prm->lambda * w + pPp;"),
}

# Mistakes planted in the oracle of the input steps; caught by test_oracle_upstream_pins.py.
MUTANTS_UP = {
    "recon_sigma_factor": ("exp(-((double)dx * dx) / (2.0 * sigma * sigma))", "exp(-((double)dx * dx) / (sigma * sigma))"),
    "recon_offset_sign": ("float dx = (float)(px - x) + base[3 * np + p];", "float dx = (float)(px - x) - base[3 * np + p];"),
    "recon_variance_of_samples_not_mean": ("var[j] = ss / (3.0 * (n - 1)) / n;", "var[j] = ss / (3.0 * (n - 1));"),
    "velocity_y_not_flipped": ("double py = (1.0 - clip[1] / clip[3]) * 0.5 * H - 0.5;",
                               "double py = (1.0 + clip[1] / clip[3]) * 0.5 * H - 0.5;"),
    "velocity_no_half_pixel": ("double px = (clip[0] / clip[3] + 1.0) * 0.5 * W - 0.5;",
                               "double px = (clip[0] / clip[3] + 1.0) * 0.5 * W;"),
    "velocity_forward_not_backward": ("vx = px - x;", "vx = x - px;"),
    "velocity_matrix_transposed": ("clip[r] += M[r * 4 + c] * X[c];", "clip[r] += M[c * 4 + r] * X[c];"),
}
SRC_UP = os.path.join(ROOT, "oracle", "wrls_oracle_upstream.c")

# Mistakes planted in the path tracer oracle; caught by test_oracle_vpt_pins.py.
MUTANTS_VPT = {
    "vpt_majorant_halved": ("        if (++g->steps > VPT_MAX_STEPS) return;\n        t += -log(1.0 - rng_u(g)) / sc->mu_max;",
                            "        if (++g->steps > VPT_MAX_STEPS) return;\n        t += -log(1.0 - rng_u(g)) / (0.5 * sc->mu_max);"),
    "vpt_phase_function_dropped": ("beta[c] * sc->light_rgb[c] / (4.0 * VPT_PI);", "beta[c] * sc->light_rgb[c];"),
    "vpt_albedo_not_applied": ("beta[c] *= sc->albedo * (", "beta[c] *= (0.0 * sc->albedo + 1.0) * ("),
    "vpt_shadow_ray_not_tracked": ("if (visible(sc, g, y, ld))", "if (1)"),
    "vpt_acceptance_inverted": ("if (!(rng_u(g) < mu / sc->mu_max)) continue;", "if (rng_u(g) < mu / sc->mu_max) continue;"),
    "vpt_background_dropped": ("for (int c = 0; c < 3; ++c) L[c] += beta[c] * sc->env_rgb[c];",
                               "for (int c = 0; c < 3; ++c) L[c] += 0.0 * beta[c] * sc->env_rgb[c];"),
}
SRC_VPT = os.path.join(ROOT, "oracle", "wrls_oracle_vpt.c")
_SOURCES = {SRC: MUTANTS, SRC_EXT: MUTANTS_EXT, SRC_UP: MUTANTS_UP, SRC_VPT: MUTANTS_VPT}

_CASES = [(n, SRC, "test_oracle_pins.py") for n in sorted(MUTANTS)] + \
         [(n, SRC_EXT, "test_oracle_ext_pins.py") for n in sorted(MUTANTS_EXT)] + \
         [(n, SRC_UP, "test_oracle_upstream_pins.py") for n in sorted(MUTANTS_UP)] + \
         [(n, SRC_VPT, "test_oracle_vpt_pins.py") for n in sorted(MUTANTS_VPT)]


@pytest.mark.parametrize("name,src_path,pins", _CASES, ids=[c[0] for c in _CASES])
def test_pins_catch_planted_mistake(name, src_path, pins, tmp_path):
    old, new = _SOURCES[src_path][name]
    src = open(src_path).read()
    assert src.count(old) >= 1, "mutant anchor not found: " + name
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / os.path.basename(src_path)
    so_path = tmp_path / "libmutant.so"
    c_path.write_text(mutated)
    others = [p for p in _SOURCES if p != src_path]
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so_path), str(c_path), *others, "-lm"])
    env = dict(os.environ, WRLS_ORACLE_LIB=str(so_path), OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(HERE, pins)],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, "no pin caught mutant %s:\n%s" % (name, res.stdout[-2000:])
