"""The pins must catch plausible mistakes in the oracle.

Each mutant below plants one mistake in a temporary copy of the oracle's C
source (a dropped term, a flipped sign, a transposed operand, an off-by-one,
a wrong constant) on the CPU; the copy is built and the oracle's pin files
run against it, and at least one pin must fail.  An unmutated copy run the
same way must pass, so a mutant's failure is the pins' doing, not the copy's.

Left out as equivalent or as readings the paper does not fix (and therefore
checked only through the GPU parity tests, which share these readings): the
tie rule of the queue (smaller D_lo first), the binary32 form of an
interval's centre, the choice of the walked axis of a bound segment (either
axis gives the same supercover up to the 2^-8 px margin), and the exact
threshold of the fast mode's sampling (one value in 2^24).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_pins.py", "test_oracle_polarity.py", "test_oracle_ref.py", "test_oracle_warm.py",
             "test_oracle_fast.py"]

# (name, what the mistake is, text in oracle.c, its replacement)
MUTANTS = [
    # Eq. (11): the warp
    ("warp_t_sign", "the event's time enters the scale with the wrong sign",
     "float a = 1.0f - D * ti;", "float a = 1.0f + D * ti;"),
    ("warp_g_sign", "the reference time enters the scale with the wrong sign",
     "float q = 1.0f - D * tau;", "float q = 1.0f + D * tau;"),
    ("warp_no_g", "the scale's denominator 1 - D tau dropped",
     "    return a * g;", "    return a;"),
    ("cell_no_half", "pixel centres at integers dropped (floor instead of nearest)",
     "return (int32_t)floorf(p + 0.5f);", "return (int32_t)floorf(p);"),
    ("cell_no_foe", "the warped offset not moved back to the FOE",
     "float p = foe + d * s;", "float p = d * s;"),
    ("point_no_t0", "event times not taken relative to the window's start",
     "        float s = warp_s(D, w->t[i] - w->t0, g);\n        int32_t ux = cell(w->foe_x, dx, s), uy",
     "        float s = warp_s(D, w->t[i], g);\n        int32_t ux = cell(w->foe_x, dx, s), uy"),
    ("point_foe_transposed", "the row computed about the FOE's x",
     "int32_t ux = cell(w->foe_x, dx, s), uy = cell(w->foe_y, dy, s);",
     "int32_t ux = cell(w->foe_x, dx, s), uy = cell(w->foe_x, dy, s);"),
    ("point_frame_edge", "column 0 treated as outside the frame",
     "if (ux >= 0 && ux < w->W && uy >= 0 && uy < w->H) img[",
     "if (ux >= 1 && ux < w->W && uy >= 0 && uy < w->H) img["),
    ("point_image_transposed", "the image stored column-major",
     "img[plane_of(w, i) * M + (int64_t)uy * w->W + ux] += 1;",
     "img[plane_of(w, i) * M + (int64_t)ux * w->H + uy] += 1;"),
    ("point_ignores_t_ref", "the point warp ignores the reference time",
     "memset(img, 0, (size_t)(planes(w) * M) * sizeof(uint32_t));\n    float g = warp_g(D, w->t_ref);",
     "memset(img, 0, (size_t)(planes(w) * M) * sizeof(uint32_t));\n    float g = warp_g(D, w->tau);"),
    # Eqs. (12)-(13): the contrast key
    ("key_no_mean", "the squared mean term N_in^2 dropped",
     "return (i128)M * (i128)S - (i128)N * (i128)N;", "return (i128)M * (i128)S;"),
    ("key_mean_sign", "the squared mean term added",
     "return (i128)M * (i128)S - (i128)N * (i128)N;", "return (i128)M * (i128)S + (i128)N * (i128)N;"),
    ("sum_not_squared", "S sums the counts instead of their squares",
     "s += (uint64_t)img[u] * (uint64_t)img[u];", "s += (uint64_t)img[u];"),
    ("planes_last_only", "only the last polarity plane's key kept",
     "        k += key(M, s, n);", "        k = key(M, s, n);"),
    ("polarity_one_plane", "every event put in the first polarity plane",
     "return (w->p && w->p[i] <= 0) ? 1 : 0;", "return 0;"),
    ("polarity_planes_swapped", "the polarity planes swapped",
     "return (w->p && w->p[i] <= 0) ? 1 : 0;", "return w->p ? (w->p[i] <= 0 ? 0 : 1) : 0;"),
    # Eqs. (14)-(19): the bound
    ("no_widen_up", "the scale interval not widened upwards",
     "static const float WIDEN_UP = 1.0f + 0x1p-19f;", "static const float WIDEN_UP = 1.0f;"),
    ("widen_lower_end_up", "the lower end of the scale interval widened upwards",
     "*sa = (sl < sh ? sl : sh) * WIDEN_DN;", "*sa = (sl < sh ? sl : sh) * WIDEN_UP;"),
    ("interval_g_of_lo", "the upper end's scale taken with the lower end's g",
     "sh = warp_s(D_hi, ti, warp_g(D_hi, tau));", "sh = warp_s(D_hi, ti, warp_g(D_lo, tau));"),
    ("half_short", "the pixel half-width below 1/2",
     "static const float HALF_PLUS = 0.50390625f;", "static const float HALF_PLUS = 0.45f;"),
    ("half_wide", "the pixel margin a quarter pixel instead of 2^-8",
     "static const float HALF_PLUS = 0.50390625f;", "static const float HALF_PLUS = 0.75f;"),
    ("minor_one_cell", "one minor cell per major cell",
     "int32_t j1 = cell(fn, dn, lo), j2 = cell(fn, dn, hi);", "int32_t j1 = cell(fn, dn, lo), j2 = j1;"),
    ("major_last_cell_clipped", "the last major cell of the frame dropped",
     "if (k1 > Wm - 1) k1 = Wm - 1;", "if (k1 > Wm - 2) k1 = Wm - 2;"),
    ("minor_last_cell_clipped", "the last minor cell of the frame dropped",
     "if (jn > Wn - 1) jn = Wn - 1;", "if (jn > Wn - 2) jn = Wn - 2;"),
    ("full_always", "N_full counts every event",
     "int full = xa >= 0 && xa < W && ya >= 0 && ya < H && xb >= 0 && xb < W && yb >= 0 && yb < H;",
     "int full = 1;"),
    ("full_one_end", "N_full tests one end of the segment only",
     "int full = xa >= 0 && xa < W && ya >= 0 && ya < H && xb >= 0 && xb < W && yb >= 0 && yb < H;",
     "int full = xa >= 0 && xa < W && ya >= 0 && ya < H;"),
    ("bound_key_uses_cells", "the bound's mean term from the bound image's count",
     "k += key(M, s, nf[p]);", "k += key(M, s, c);"),
    ("bound_foe_event_dropped", "an event on the FOE adds nothing to the bound image",
     "if (xa >= 0 && xa < W && ya >= 0 && ya < H) img[(int64_t)ya * W + xa] += 1;",
     "if (0) img[(int64_t)ya * W + xa] += 1;"),
    ("bound_ignores_t_ref", "the bound ignores the reference time",
     "scale_interval(D_lo, D_hi, w->t[i] - w->t0, w->t_ref, &sa, &sb);",
     "scale_interval(D_lo, D_hi, w->t[i] - w->t0, w->tau, &sa, &sb);"),
    # Algorithm 1
    ("incumbent_strict", "a centre that ties the incumbent does not replace it",
     "if (kc[j] >= K_hat) { K_hat = kc[j]; D_hat = dc[j]; }",
     "if (kc[j] > K_hat) { K_hat = kc[j]; D_hat = dc[j]; }"),
    ("incumbent_D_kept", "the incumbent's key updated but not its D",
     "if (kc[j] >= K_hat) { K_hat = kc[j]; D_hat = dc[j]; }", "if (kc[j] >= K_hat) { K_hat = kc[j]; }"),
    ("gap_test_strict", "the search continues while the bound only ties the incumbent",
     "if (q.a[b].kb - K0 <= gamma_K) {", "if (q.a[b].kb - K0 < gamma_K) {"),
    ("push_strict", "children that only tie the incumbent are dropped",
     "if (kids[j].kb >= K_hat)", "if (kids[j].kb > K_hat)"),
    ("pop_smallest_bound", "the queue returns the smallest bound first",
     "if (q->a[i].kb > q->a[b].kb ||", "if (q->a[i].kb < q->a[b].kb ||"),
    ("gap_ignores_leaves", "the certificate ignores unsplit leaves",
     "if (have_leaf && leaf_max > top) top = leaf_max;", "if (0) top = leaf_max;"),
    ("D_end_sign", "the end-of-window divergence with the wrong sign of D tau",
     "r.D_end = (float)((double)D_hat / (1.0 - (double)D_hat * (double)w->tau));",
     "r.D_end = (float)((double)D_hat / (1.0 + (double)D_hat * (double)w->tau));"),
    ("contrast_over_M", "the reported contrast K / M instead of K / M^2",
     "r.contrast = (double)K_hat / ((double)M * (double)M);", "r.contrast = (double)K_hat / (double)M;"),
    ("cells_skip_root_centre", "the root centre's image left out of the cell count",
     "        cells += N;\n        node root = {D_lo, D_hi, 0};", "        node root = {D_lo, D_hi, 0};"),
    ("bound_cells_one_child", "one child's covered cells left out of the bound count",
     "            b.kb = eval_bound(w, b.lo, b.hi, img, &S, &nf, &nc);\n            cells += nc;\n            bcells += nc;",
     "            b.kb = eval_bound(w, b.lo, b.hi, img, &S, &nf, &nc);\n            cells += nc;"),
    ("bound_evals_one_per_split", "one bound evaluation counted per split",
     "            r.bound_evals += 2;", "            r.bound_evals += 1;"),
    ("event_warps_points_only", "event-warps counted for centres only",
     "        r.event_warps = w->n * (r.point_evals + r.bound_evals);", "        r.event_warps = w->n * r.point_evals;"),
    # brute force
    ("sweep_no_neighbours", "the sweep skips the binary32 neighbours of each breakpoint",
     "for (int u = 0; u < 4; u++) {", "for (int u = 0; u < 0; u++) {"),
    ("sweep_breakpoint_sign", "the breakpoints' denominator with the wrong sign",
     "double den = d * ti - c * tau;", "double den = d * ti + c * tau;"),
    ("grid_double_step", "the grid steps twice as far as asked",
     "float D = j <= steps ? (float)((double)D_lo + (double)j * (double)h) : D_hi;",
     "float D = j <= steps ? (float)((double)D_lo + 2.0 * (double)j * (double)h) : D_hi;"),
    ("grid_skips_upper_end", "the grid stops short of its last point",
     "for (int64_t j = 0; j <= steps + 1; j++) {", "for (int64_t j = 0; j < steps; j++) {"),
    # the learned warm start
    ("feature_radius_squared", "radial bins of the squared radius",
     "int rb = (int)floorf(sqrtf(u) * (float)OR_FEAT_R);", "int rb = (int)floorf(u * (float)OR_FEAT_R);"),
    ("feature_no_t0", "temporal bins of absolute times",
     "const float v = (w->t[i] - w->t0) * tsc;", "const float v = w->t[i] * tsc;"),
    ("feature_unscaled", "features as plain shares instead of 128 times the share",
     "(float)(c[k] * OR_FEATURES) / (float)w->n", "(float)c[k] / (float)w->n"),
    ("mlp_f32_no_relu", "the binary32 network without its ReLU",
     "y[j] = relu && !(acc > 0.0f) ? 0.0f : acc;", "y[j] = acc;"),
    ("mlp_f64_wrong_bias", "the binary64 network's second layer with the first layer's biases",
     "dense_f64(p + P_W2, p + P_B2, h1, OR_MLP_H, OR_MLP_H, 1, h2);",
     "dense_f64(p + P_W2, p + P_B1, h1, OR_MLP_H, OR_MLP_H, 1, h2);"),
    ("loss_grad_sign", "the gradient of the guess with the wrong sign",
     "go[0] = -q * e / (double)B;", "go[0] = q * e / (double)B;"),
    ("backprop_no_relu", "backprop through the first ReLU as if it were linear",
     "g1[k] = h1[k] > 0.0 ? a : 0.0;", "g1[k] = a;"),
    ("warm_map_floor", "the half-width's exponent truncated instead of rounded",
     "float v = l * OR_LOG2E + 0.5f;", "float v = l * OR_LOG2E;"),
    ("warm_piece_unclamped", "the upper cut not clamped to the domain",
     "if (!(b <= D_hi)) b = D_hi;", "if (0) b = D_hi;"),
    # the fast mode
    ("resample_floor", "coarse coordinates truncated instead of rounded",
     "int32_t cx = (int32_t)floorf((float)w->x[i] * kx + 0.5f);", "int32_t cx = (int32_t)floorf((float)w->x[i] * kx);"),
    ("splitmix_constant", "a SplitMix64 multiplier off by one",
     "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B8ull;"),
    ("resample_clamp", "the far-edge clamp one pixel short",
     "if (cx > W2 - 1) cx = W2 - 1;", "if (cx > W2 - 2) cx = W2 - 2;"),
    ("warm_piece_lower_unclamped", "the lower cut not clamped to the domain",
     "if (!(a >= D_lo)) a = D_lo;", "if (0) a = D_lo;"),
    ("loss_no_width_term", "the loss without its log half-width term",
     "loss += 0.5 * q * e * e + o[1];", "loss += 0.5 * q * e * e;"),
    ("feature_radius_x_only", "the largest radius from the x extent alone",
     "const float R2 = cx * cx + cy * cy;", "const float R2 = cx * cx;"),
    ("resample_foe_wrong_axis", "the coarse FOE's row scaled by the column ratio",
     "*fy2 = w->foe_y * ((float)H2 / (float)w->H);", "*fy2 = w->foe_y * ((float)W2 / (float)w->W);"),
    # the binary64 diagnostic
    ("fp64_counts_nothing", "the binary64 diagnostic never counts",
     "if (ux != cell(w->foe_x, dx, s) || uy != cell(w->foe_y, dy, s)) bad++;",
     "if (0) bad++;"),
    ("fp64_reference_tau", "the binary64 warp ignores the reference time",
     "double Dd = D, tau = w->t_ref;", "double Dd = D, tau = w->tau;"),
    ("fp64_no_half", "the binary64 pixel without the half pixel",
     "int64_t ux = (int64_t)floor((double)w->foe_x + X * sd + 0.5);",
     "int64_t ux = (int64_t)floor((double)w->foe_x + X * sd);"),
    # argument checks
    ("rejects_far_foe", "an FOE on the frame's far edge rejected",
     "w->foe_x > (float)w->W", "w->foe_x >= (float)w->W"),
    ("rejects_domain_edge", "D tau = 3/4 rejected",
     "return dt <= 0.75 && dt >= -64.0;", "return dt < 0.75 && dt >= -64.0;"),
    ("accepts_late_t_ref", "a reference time after the window's end accepted",
     "if (!(w->t_ref >= 0.0f) || !(w->t_ref <= w->tau)) return OR_ERR_ARG;",
     "if (!(w->t_ref >= 0.0f)) return OR_ERR_ARG;"),
    ("rejects_last_row", "the frame's last row rejected",
     "w->y[i] < 0 || w->y[i] >= w->H)", "w->y[i] < 0 || w->y[i] >= w->H - 1)"),
    ("rejects_window_end", "an event at the window's end rejected",
     "!(ti >= 0.0f) || !(ti <= w->tau)) return OR_ERR_ARG;", "!(ti >= 0.0f) || !(ti < w->tau)) return OR_ERR_ARG;"),
    ("accepts_late_events", "events after the window's end accepted",
     "if (!isfinite(w->t[i]) || !(ti >= 0.0f) || !(ti <= w->tau)) return OR_ERR_ARG;",
     "if (!isfinite(w->t[i]) || !(ti >= 0.0f)) return OR_ERR_ARG;"),
]


def _stage(dst, src_c):
    """A copy of the oracle, its pins and the input generators under dst,
    with oracle.c replaced by src_c."""
    ign = shutil.ignore_patterns("__pycache__", "*.so", "*.tmp")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "synth"), os.path.join(dst, "synth"), ignore=ign)
    os.makedirs(os.path.join(dst, "tests"))
    for f in ["conftest.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    with open(os.path.join(dst, "oracle", "oracle.c"), "w") as fh:
        fh.write(src_c)


def _run(dst):
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", dst] +
                       [os.path.join("tests", f) for f in PIN_FILES], cwd=dst, capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, PYTHONDONTWRITEBYTECODE="1"))
    tail = [line for line in r.stdout.splitlines() if line.strip()][-3:]
    return r.returncode, "\n".join(tail)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    jobs = {"control": src}
    for name, _, old, new in MUTANTS:
        assert src.count(old) == 1, (name, "the mutated text must occur exactly once in oracle.c")
        jobs[name] = src.replace(old, new)
    base = tmp_path_factory.mktemp("mutants")
    for name, text in jobs.items():
        _stage(str(base / name), text)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {name: ex.submit(_run, str(base / name)) for name in jobs}
        return {name: f.result() for name, f in futs.items()}


def test_unmutated_copy_passes_its_pins(outcomes):
    rc, tail = outcomes["control"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(outcomes, name):
    rc, tail = outcomes[name]
    what = next(m[1] for m in MUTANTS if m[0] == name)
    assert rc == 1, f"{name} ({what}) survived the pins (pytest exit {rc}):\n{tail}"
