/*
 * CPU oracle for exact contrast-maximisation divergence estimation
 * (arXiv 2209.13168).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * Every float operation below is one IEEE-754 binary32 operation rounded to
 * nearest (no contraction into FMA, no excess precision), in the order
 * written.  The pixel a warped event falls in is an integer decided by
 * floating point, so it is decided in binary32 here exactly as the kernels
 * decide it.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

static or_i128 pack(i128 v) {
    or_i128 r;
    r.lo = (uint64_t)(u128)v;
    r.hi = (int64_t)(uint64_t)((u128)v >> 64);
    return r;
}

/* ---------------------------------------------------------------- domain */

/* Reading of Sec. 4.1: nu in [-1/tau, 0] with Z0 = 1 becomes D = -nu; the
 * singular end D = 1/tau (1 + nu tau = 0) is excluded.  The bound's widening
 * (or_bound) is proven sufficient for D tau <= 3/4, so the domain is
 * D tau in [-64, 3/4]. */
static int d_ok(float D, float tau) {
    if (!isfinite(D)) return 0;
    double dt = (double)D * (double)tau;
    return dt <= 0.75 && dt >= -64.0;
}

int or_validate(const or_window* w, float D_lo, float D_hi) {
    if (!w || w->n < 0 || w->W < 1 || w->H < 1 || w->W > 4096 || w->H > 4096) return OR_ERR_ARG;
    if (w->n > 0 && (!w->x || !w->y || !w->t)) return OR_ERR_ARG;
    if (!isfinite(w->foe_x) || !isfinite(w->foe_y) || w->foe_x < 0.0f || w->foe_y < 0.0f ||
        w->foe_x > (float)w->W || w->foe_y > (float)w->H) return OR_ERR_ARG;
    if (!isfinite(w->tau) || !(w->tau > 0.0f) || !isfinite(w->t0)) return OR_ERR_ARG;
    if (!(w->t_ref >= 0.0f) || !(w->t_ref <= w->tau)) return OR_ERR_ARG;
    if (!d_ok(D_lo, w->tau) || !d_ok(D_hi, w->tau) || !(D_lo <= D_hi)) return OR_ERR_ARG;
    /* Events come from a W x H sensor: pixel coordinates inside the frame. */
    for (int64_t i = 0; i < w->n; i++) {
        float ti = w->t[i] - w->t0;
        if (!isfinite(w->t[i]) || !(ti >= 0.0f) || !(ti <= w->tau)) return OR_ERR_ARG;
        if (w->x[i] < 0 || w->x[i] >= w->W || w->y[i] < 0 || w->y[i] >= w->H) return OR_ERR_ARG;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ warp */

/* Eq. (11) with Z0 = 1 and nu = -D: the event keeps its direction from the
 * FOE and its offset is scaled by s_i(D) = (1 - D t_i) / (1 - D tau).
 * Evaluated as g = 1/(1 - D*tau) once per hypothesis, then
 * s_i = (1 - D*t_i) * g.  Warping to another reference time t_ref replaces
 * tau by t_ref in g (t_ref = 0: g = 1, the scale 1 - D t_i is linear in D). */
static float warp_g(float D, float tau) {
    float q = 1.0f - D * tau;
    return 1.0f / q;
}
static float warp_s(float D, float ti, float g) {
    float a = 1.0f - D * ti;
    return a * g;
}
/* Eq. (12): the pixel a warped event falls in.  Pixel u covers [u - 1/2, u + 1/2), so
 * integer event coordinates are pixel centres (reading; the paper is silent). */
static int32_t cell(float foe, float d, float s) {
    float p = foe + d * s;
    return (int32_t)floorf(p + 0.5f);
}

void or_warp_cells(const or_window* w, float D, int32_t* ux, int32_t* uy) {
    float g = warp_g(D, w->t_ref);
    for (int64_t i = 0; i < w->n; i++) {
        float dx = (float)w->x[i] - w->foe_x, dy = (float)w->y[i] - w->foe_y;
        float s = warp_s(D, w->t[i] - w->t0, g);
        ux[i] = cell(w->foe_x, dx, s);
        uy[i] = cell(w->foe_y, dy, s);
    }
}

/* The same warp in binary64 throughout; reports how many events land in a
 * different pixel than the binary32 warp.  Diagnostic only. */
int64_t or_fp64_disagreements(const or_window* w, float D) {
    int64_t bad = 0;
    float g = warp_g(D, w->t_ref);
    double Dd = D, tau = w->t_ref;
    for (int64_t i = 0; i < w->n; i++) {
        float dx = (float)w->x[i] - w->foe_x, dy = (float)w->y[i] - w->foe_y;
        float s = warp_s(D, w->t[i] - w->t0, g);
        double ti = (double)(w->t[i] - w->t0);
        double sd = (1.0 - Dd * ti) / (1.0 - Dd * tau);
        double X = (double)w->x[i] - (double)w->foe_x, Y = (double)w->y[i] - (double)w->foe_y;
        int64_t ux = (int64_t)floor((double)w->foe_x + X * sd + 0.5);
        int64_t uy = (int64_t)floor((double)w->foe_y + Y * sd + 0.5);
        if (ux != cell(w->foe_x, dx, s) || uy != cell(w->foe_y, dy, s)) bad++;
    }
    return bad;
}

/* ------------------------------------------------------------- contrast */

/* Eqs. (12)-(13).  C = (1/M) sum_u (H - mu)^2 = sum_u H^2 / M - mu^2 with
 * mu = N_in / M (the rewrite used in the supplementary proof), so
 *     M^2 C = M * S - N_in^2 =: K,  S = sum_u H(u)^2,  N_in = sum_u H(u),
 * an exact integer.  Comparisons of contrast are comparisons of K. */
static i128 key(int64_t M, uint64_t S, int64_t N) {
    return (i128)M * (i128)S - (i128)N * (i128)N;
}

/* Polarity (the paper leaves it out of Eq. (12) and notes it could be used):
 * with or_window.p given, each polarity gets its own image H_p of M pixels
 * and the objective is C_on + C_off, so
 *     M^2 (C_on + C_off) = M (S_on + S_off) - N_on^2 - N_off^2.
 * Each plane is an image of non-negative counts, so Eqs. (14)-(19) bound it
 * plane by plane and the bounds add. */
static int32_t planes(const or_window* w) { return w->p ? 2 : 1; }
static int64_t plane_of(const or_window* w, int64_t i) { return (w->p && w->p[i] <= 0) ? 1 : 0; }

static void sums(const uint32_t* img, int64_t M, uint64_t* S, int64_t* N) {
    uint64_t s = 0;
    int64_t n = 0;
    for (int64_t u = 0; u < M; u++) {
        s += (uint64_t)img[u] * (uint64_t)img[u];
        n += img[u];
    }
    *S = s;
    *N = n;
}

/* Eq. (13) over the planes of img: K = sum_p (M S_p - N_p^2); S, N totals. */
static i128 plane_key(const or_window* w, const uint32_t* img, uint64_t* S, int64_t* N) {
    int64_t M = (int64_t)w->W * w->H;
    i128 k = 0;
    *S = 0;
    *N = 0;
    for (int32_t p = 0; p < planes(w); p++) {
        uint64_t s;
        int64_t n;
        sums(img + p * M, M, &s, &n);
        k += key(M, s, n);
        *S += s;
        *N += n;
    }
    return k;
}

static void iwe_point(const or_window* w, float D, uint32_t* img) {
    int64_t M = (int64_t)w->W * w->H;
    memset(img, 0, (size_t)(planes(w) * M) * sizeof(uint32_t));
    float g = warp_g(D, w->t_ref);
    for (int64_t i = 0; i < w->n; i++) {
        float dx = (float)w->x[i] - w->foe_x, dy = (float)w->y[i] - w->foe_y;
        float s = warp_s(D, w->t[i] - w->t0, g);
        int32_t ux = cell(w->foe_x, dx, s), uy = cell(w->foe_y, dy, s);
        if (ux >= 0 && ux < w->W && uy >= 0 && uy < w->H) img[plane_of(w, i) * M + (int64_t)uy * w->W + ux] += 1;
    }
}

static i128 eval_point(const or_window* w, float D, uint32_t* img, uint64_t* S, int64_t* N) {
    iwe_point(w, D, img);
    return plane_key(w, img, S, N);
}

int or_contrast(const or_window* w, float D, or_i128* K, uint64_t* S, int64_t* N_in, uint32_t* iwe) {
    int rc = or_validate(w, D, D);
    if (rc) return rc;
    int64_t M = (int64_t)w->W * w->H;
    uint32_t* img = iwe ? iwe : (uint32_t*)malloc((size_t)(planes(w) * M) * sizeof(uint32_t));
    if (!img) return OR_ERR_OOM;
    uint64_t s;
    int64_t n;
    i128 k = eval_point(w, D, img, &s, &n);
    if (!iwe) free(img);
    if (K) *K = pack(k);
    if (S) *S = s;
    if (N_in) *N_in = n;
    return OR_OK;
}

/* ---------------------------------------------------------------- bound */

/* Relative widening of the scale interval.  For D tau <= 3/4 the binary32
 * evaluation of s_i(D) has relative error below 10 * 2^-24 against the real
 * s_i(D), and the real s_i is monotone in D (ds/dD = (tau - t)/(1 - D tau)^2
 * >= 0), so every binary32 s_i(D) with D in [D_lo, D_hi] lies inside
 * [min(s_lo, s_hi)(1 - 2^-19), max(s_lo, s_hi)(1 + 2^-19)].  The paper argues
 * in real arithmetic (supplementary proof of Eq. (17)); this widening is the
 * reading that keeps the bound valid for the binary32 warp. */
static const float WIDEN_DN = 1.0f - 0x1p-19f;
static const float WIDEN_UP = 1.0f + 0x1p-19f;
/* Half a pixel plus a margin of 2^-8 pixel, which exceeds the rounding error
 * of the binary32 cell computation for coordinates below 4096. */
static const float HALF_PLUS = 0.50390625f;

/* Eq. (16) for one event: every pixel the segment f_i(D_lo) <-> f_i(D_hi)
 * passes through gets +1 (each pixel at most once per event).  The segment
 * is radial, s in [s_a, s_b].  Walk the cells of the axis with the larger
 * |offset| (ties: x); for major cell k, the widened s-range in which the
 * major coordinate rounds to k gives the run of minor cells.  Returns
 * whether both end cells lie in the frame (Eq. (19)); the frame is convex and
 * each cell coordinate is monotone in s, so then the whole segment does. */
/* The widened scale interval [s_a, s_b] of one event over [D_lo, D_hi]. */
static void scale_interval(float D_lo, float D_hi, float ti, float tau, float* sa, float* sb) {
    float sl = warp_s(D_lo, ti, warp_g(D_lo, tau)), sh = warp_s(D_hi, ti, warp_g(D_hi, tau));
    *sa = (sl < sh ? sl : sh) * WIDEN_DN;
    *sb = (sl < sh ? sh : sl) * WIDEN_UP;
}

float or_scale(float D, float ti, float tau) { return warp_s(D, ti, warp_g(D, tau)); }

void or_scale_interval(float D_lo, float D_hi, float ti, float tau, float* sa, float* sb) {
    scale_interval(D_lo, D_hi, ti, tau, sa, sb);
}

static int segment(const or_window* w, float dx, float dy, float sa, float sb, uint32_t* img) {
    const int32_t W = w->W, H = w->H;
    int32_t xa = cell(w->foe_x, dx, sa), ya = cell(w->foe_y, dy, sa);
    int32_t xb = cell(w->foe_x, dx, sb), yb = cell(w->foe_y, dy, sb);
    int full = xa >= 0 && xa < W && ya >= 0 && ya < H && xb >= 0 && xb < W && yb >= 0 && yb < H;
    if (dx == 0.0f && dy == 0.0f) {          /* event on the FOE: one pixel for every D */
        if (xa >= 0 && xa < W && ya >= 0 && ya < H) img[(int64_t)ya * W + xa] += 1;
        return full;
    }
    int major_x = fabsf(dx) >= fabsf(dy);
    float fm = major_x ? w->foe_x : w->foe_y, fn = major_x ? w->foe_y : w->foe_x;
    float dm = major_x ? dx : dy, dn = major_x ? dy : dx;
    int32_t ka = major_x ? xa : ya, kb = major_x ? xb : yb;
    int32_t Wm = major_x ? W : H, Wn = major_x ? H : W;
    int32_t k0 = ka < kb ? ka : kb, k1 = ka < kb ? kb : ka;
    if (k0 < 0) k0 = 0;
    if (k1 > Wm - 1) k1 = Wm - 1;
    float rm = 1.0f / dm;
    for (int32_t k = k0; k <= k1; k++) {
        float e = (float)k - fm;
        float b1 = (e - HALF_PLUS) * rm, b2 = (e + HALF_PLUS) * rm;
        float lo = b1 < b2 ? b1 : b2, hi = b1 < b2 ? b2 : b1;
        if (lo < sa) lo = sa;
        if (hi > sb) hi = sb;
        if (lo > hi) continue;
        int32_t j1 = cell(fn, dn, lo), j2 = cell(fn, dn, hi);
        int32_t j0 = j1 < j2 ? j1 : j2, jn = j1 < j2 ? j2 : j1;
        if (j0 < 0) j0 = 0;
        if (jn > Wn - 1) jn = Wn - 1;
        for (int32_t j = j0; j <= jn; j++) {
            int64_t u = major_x ? (int64_t)j * W + k : (int64_t)k * W + j;
            img[u] += 1;
        }
    }
    return full;
}

/* Eqs. (14)-(19): Kbar = M * Sbar - N_full^2 with Sbar = sum_u Hbar(u)^2
 * (Eq. (18)) and N_full = M * mu_lower (Eq. (19)).  Since Sbar >= S(D) and
 * 0 <= N_full <= N_in(D) for every D in the interval, Kbar >= K(D).  With
 * polarity planes, per plane: Kbar = sum_p (M Sbar_p - N_full,p^2). */
static i128 eval_bound(const or_window* w, float D_lo, float D_hi, uint32_t* img, uint64_t* Sb,
                       int64_t* Nfull, int64_t* n_cells) {
    int64_t M = (int64_t)w->W * w->H;
    memset(img, 0, (size_t)(planes(w) * M) * sizeof(uint32_t));
    int64_t nf[2] = {0, 0};
    for (int64_t i = 0; i < w->n; i++) {
        float dx = (float)w->x[i] - w->foe_x, dy = (float)w->y[i] - w->foe_y;
        float sa, sb;
        scale_interval(D_lo, D_hi, w->t[i] - w->t0, w->t_ref, &sa, &sb);
        int64_t p = plane_of(w, i);
        nf[p] += segment(w, dx, dy, sa, sb, img + p * M);
    }
    i128 k = 0;
    *Sb = 0;
    *n_cells = 0;
    for (int32_t p = 0; p < planes(w); p++) {
        uint64_t s;
        int64_t c;
        sums(img + p * M, M, &s, &c);
        k += key(M, s, nf[p]);
        *Sb += s;
        *n_cells += c;
    }
    *Nfull = nf[0] + nf[1];
    return k;
}

int or_bound(const or_window* w, float D_lo, float D_hi, or_i128* Kbar, uint64_t* Sbar,
             int64_t* N_full, uint32_t* iwe) {
    int rc = or_validate(w, D_lo, D_hi);
    if (rc) return rc;
    int64_t M = (int64_t)w->W * w->H;
    uint32_t* img = iwe ? iwe : (uint32_t*)malloc((size_t)(planes(w) * M) * sizeof(uint32_t));
    if (!img) return OR_ERR_OOM;
    uint64_t s;
    int64_t nf, nc;
    i128 k = eval_bound(w, D_lo, D_hi, img, &s, &nf, &nc);
    if (!iwe) free(img);
    if (Kbar) *Kbar = pack(k);
    if (Sbar) *Sbar = s;
    if (N_full) *N_full = nf;
    return OR_OK;
}

/* ------------------------------------------------------------------ BnB */

typedef struct { float lo, hi; i128 kb; } node;

typedef struct { node* a; int64_t n, cap; } queue;

static int q_push(queue* q, node v) {
    if (q->n == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 64;
        node* na = (node*)realloc(q->a, (size_t)nc * sizeof(node));
        if (!na) return OR_ERR_OOM;
        q->a = na;
        q->cap = nc;
    }
    q->a[q->n++] = v;
    return OR_OK;
}

/* Index of the first item of the priority queue: largest Kbar; among equal
 * Kbar, the smaller D_lo (tie rule: a reading, the paper is silent). */
static int64_t q_top(const queue* q) {
    int64_t b = 0;
    for (int64_t i = 1; i < q->n; i++)
        if (q->a[i].kb > q->a[b].kb || (q->a[i].kb == q->a[b].kb && q->a[i].lo < q->a[b].lo)) b = i;
    return b;
}

static node q_take(queue* q, int64_t i) {
    node v = q->a[i];
    q->a[i] = q->a[q->n - 1];
    q->n--;
    return v;
}

static float centre(float lo, float hi) { return lo + 0.5f * (hi - lo); }

/* Algorithm 1 over D = -nu, in rounds that dequeue up to K_pop intervals
 * (K_pop = 1 is Algorithm 1 step for step):
 *   init       incumbent = centre of the domain, K_hat = K(centre); the
 *              domain enters the queue with priority Kbar
 *   dequeue    take the first item; stop if Kbar - K_hat <= gamma_K (gamma
 *              in contrast units, gamma_K = floor(gamma * M^2)); in a round,
 *              dequeuing stops at the first item that passes this test
 *              against the incumbent at the start of the round, and that
 *              item stays queued
 *   incumbent  evaluate every dequeued centre; in dequeue order, a centre
 *              with K >= K_hat becomes the incumbent
 *   bisect     split at the centre, unless the interval is no wider than
 *              tol_D (a leaf: its Kbar is kept in leaf_max and it is not
 *              split; the paper has no width rule, binary32 bounds need one)
 *   insert     evaluate both child bounds; insert children with
 *              Kbar >= K_hat, K_hat being the incumbent at the end of the
 *              round.
 * The certificate is gap_K = max(0, max(leaf_max, Kbar of the item that
 * stopped the search) - K_hat). */
int or_solve(const or_window* w, float D_lo, float D_hi, float tol_D, double gamma, int32_t K_pop,
             or_result* out, or_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    return or_solve_warm(w, D_lo, D_hi, tol_D, gamma, K_pop, 0, 0.0f, 0.0f, out, trace, trace_cap, trace_len);
}

/* The root pieces of a warm start at D_warm +- w_warm: the guess is clamped
 * into the domain, the cuts a = D0 - w, b = D0 + w (binary32) are clamped to
 * the domain, and the domain is cut at them into up to three intervals of
 * positive width, in increasing D.  Returns the number of pieces. */
static int warm_pieces(float D_lo, float D_hi, float D_warm, float w_warm, float* D0, node* piece) {
    float d = D_warm;
    if (!(d >= D_lo)) d = D_lo;                  /* also catches NaN */
    if (d > D_hi) d = D_hi;
    float a = d - w_warm, b = d + w_warm;
    if (!(a >= D_lo)) a = D_lo;
    if (!(b <= D_hi)) b = D_hi;
    float cut[4] = {D_lo, a, b, D_hi};
    int n = 0;
    for (int i = 0; i < 3; i++)
        if (cut[i] < cut[i + 1]) {
            piece[n].lo = cut[i];
            piece[n].hi = cut[i + 1];
            piece[n].kb = 0;
            n++;
        }
    *D0 = d;
    return n;
}

int or_solve_warm(const or_window* w, float D_lo, float D_hi, float tol_D, double gamma, int32_t K_pop,
                  int32_t warm, float D_warm, float w_warm, or_result* out, or_node_rec* trace,
                  int64_t trace_cap, int64_t* trace_len) {
    int rc = or_validate(w, D_lo, D_hi);
    if (rc) return rc;
    if (!out || K_pop < 1 || !(D_lo < D_hi) || !(tol_D >= 0.0f) || !isfinite(tol_D) || !(gamma >= 0.0) ||
        !isfinite(gamma))
        return OR_ERR_ARG;
    if (warm != 0 && (warm != 1 || !isfinite(D_warm) || !isfinite(w_warm) || !(w_warm > 0.0f)))
        return OR_ERR_ARG;
    const int64_t M = (int64_t)w->W * w->H;
    const i128 gamma_K = (i128)floor(gamma * (double)M * (double)M);
    uint32_t* img = (uint32_t*)malloc((size_t)(planes(w) * M) * sizeof(uint32_t));
    node* pop = (node*)malloc((size_t)K_pop * sizeof(node));
    i128* kc = (i128*)malloc((size_t)K_pop * sizeof(i128));
    float* dc = (float*)malloc((size_t)K_pop * sizeof(float));
    node* kids = (node*)malloc((size_t)2 * K_pop * sizeof(node));
    if (!img || !pop || !kc || !dc || !kids) {
        free(img); free(pop); free(kc); free(dc); free(kids);
        return OR_ERR_OOM;
    }
    queue q = {0, 0, 0};
    or_result r;
    memset(&r, 0, sizeof(r));
    int64_t tl = 0, cells = 0, bcells = 0;
    uint64_t S;
    int64_t N;

    int64_t nf, nc;
    float D_hat;
    i128 K_hat;
    if (!warm) {
        D_hat = centre(D_lo, D_hi);                           /* init: incumbent */
        K_hat = eval_point(w, D_hat, img, &S, &N);
        r.point_evals = 1;
        cells += N;
        node root = {D_lo, D_hi, 0};                          /* init: queue */
        root.kb = eval_bound(w, D_lo, D_hi, img, &S, &nf, &nc);
        r.bound_evals = 1;
        cells += nc;
        bcells += nc;
        if ((rc = q_push(&q, root))) goto done;
    } else {
        /* Warm start: the guess replaces the centre as the first incumbent,
         * and the domain enters the queue as the pieces around the guess;
         * a piece is queued when its bound reaches the incumbent, as
         * children are (the piece holding the guess always is). */
        node piece[3];
        const int np0 = warm_pieces(D_lo, D_hi, D_warm, w_warm, &D_hat, piece);
        K_hat = eval_point(w, D_hat, img, &S, &N);
        r.point_evals = 1;
        cells += N;
        for (int i = 0; i < np0; i++) {
            piece[i].kb = eval_bound(w, piece[i].lo, piece[i].hi, img, &S, &nf, &nc);
            r.bound_evals++;
            cells += nc;
            bcells += nc;
        }
        for (int i = 0; i < np0; i++)
            if (piece[i].kb >= K_hat)
                if ((rc = q_push(&q, piece[i]))) goto done;
    }
    r.max_queue = q.n;

    int have_leaf = 0, have_stop = 0;
    i128 leaf_max = 0, stop_kb = 0;
    while (q.n > 0) {                                          /* while queue */
        const i128 K0 = K_hat;
        int np = 0;
        while (np < K_pop && q.n > 0) {                        /* dequeue */
            int64_t b = q_top(&q);
            if (q.a[b].kb - K0 <= gamma_K) {                   /* gap test */
                if (np == 0) { have_stop = 1; stop_kb = q.a[b].kb; }
                break;
            }
            pop[np++] = q_take(&q, b);
        }
        if (np == 0) break;
        r.rounds++;
        for (int j = 0; j < np; j++) {                         /* centres */
            dc[j] = centre(pop[j].lo, pop[j].hi);
            kc[j] = eval_point(w, dc[j], img, &S, &N);
            cells += N;
            r.point_evals++;
            r.nodes_expanded++;
        }
        for (int j = 0; j < np; j++)                           /* incumbent */
            if (kc[j] >= K_hat) { K_hat = kc[j]; D_hat = dc[j]; }
        int nk = 0;
        for (int j = 0; j < np; j++) {                         /* bisect */  
            int leaf = !((pop[j].hi - pop[j].lo) > tol_D) || !(dc[j] > pop[j].lo) || !(dc[j] < pop[j].hi);
            if (trace && tl < trace_cap) {
                or_node_rec* t = &trace[tl];
                t->D_lo = pop[j].lo; t->D_hi = pop[j].hi; t->D_c = dc[j]; t->leaf = leaf;
                t->Kbar = pack(pop[j].kb); t->K_c = pack(kc[j]);
            }
            tl++;
            if (leaf) {
                if (!have_leaf || pop[j].kb > leaf_max) leaf_max = pop[j].kb;
                have_leaf = 1;
                continue;
            }
            node a = {pop[j].lo, dc[j], 0}, b = {dc[j], pop[j].hi, 0};
            a.kb = eval_bound(w, a.lo, a.hi, img, &S, &nf, &nc);
            cells += nc;
            bcells += nc;
            b.kb = eval_bound(w, b.lo, b.hi, img, &S, &nf, &nc);
            cells += nc;
            bcells += nc;
            r.bound_evals += 2;
            kids[nk++] = a;
            kids[nk++] = b;
        }
        for (int j = 0; j < nk; j++)                           /* insert */ 
            if (kids[j].kb >= K_hat)
                if ((rc = q_push(&q, kids[j]))) goto done;
        if (q.n > r.max_queue) r.max_queue = q.n;
    }
    {
        i128 top = K_hat;
        if (have_leaf && leaf_max > top) top = leaf_max;
        if (have_stop && stop_kb > top) top = stop_kb;
        i128 gap = top - K_hat;
        r.D_star = D_hat;
        r.D_end = (float)((double)D_hat / (1.0 - (double)D_hat * (double)w->tau));
        r.K_hat = pack(K_hat);
        r.gap_K = pack(gap);
        r.contrast = (double)K_hat / ((double)M * (double)M);
        r.bound_gap = (double)gap / ((double)M * (double)M);
        r.event_warps = w->n * (r.point_evals + r.bound_evals);
        r.cell_increments = cells;
        r.bound_increments = bcells;
        r.status = OR_OK;
        *out = r;
        if (trace_len) *trace_len = tl;
    }
done:
    free(q.a); free(img); free(pop); free(kc); free(dc); free(kids);
    return rc;
}

/* ------------------------------------------------------- brute force */

/* Dense grid: K at D_lo + j h (rounded to binary32), j = 0, 1, ... while the
 * point stays <= D_hi, plus D_hi itself.  Returns the largest K and the
 * smallest grid D attaining it. */
int or_grid_max(const or_window* w, float D_lo, float D_hi, float h, or_i128* K_max, float* D_at,
                int64_t* n_evals) {
    int rc = or_validate(w, D_lo, D_hi);
    if (rc) return rc;
    if (!(h > 0.0f)) return OR_ERR_ARG;
    int64_t M = (int64_t)w->W * w->H;
    uint32_t* img = (uint32_t*)malloc((size_t)(planes(w) * M) * sizeof(uint32_t));
    if (!img) return OR_ERR_OOM;
    int64_t steps = (int64_t)floor(((double)D_hi - (double)D_lo) / (double)h);
    i128 best = 0;
    float bd = D_lo;
    int64_t ne = 0;
    for (int64_t j = 0; j <= steps + 1; j++) {
        float D = j <= steps ? (float)((double)D_lo + (double)j * (double)h) : D_hi;
        if (D > D_hi) D = D_hi;
        uint64_t S;
        int64_t N;
        i128 k = eval_point(w, D, img, &S, &N);
        ne++;
        if (ne == 1 || k > best || (k == best && D < bd)) { best = k; bd = D; }
    }
    free(img);
    *K_max = pack(best);
    *D_at = bd;
    if (n_evals) *n_evals = ne;
    return OR_OK;
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : x > y;
}

static void add_bp(double** bp, int64_t* n, int64_t* cap, double v) {
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *bp = (double*)realloc(*bp, (size_t)*cap * sizeof(double));
    }
    (*bp)[(*n)++] = v;
}

/* Breakpoint sweep.  K(D) is piecewise constant: an event changes pixel only
 * where a coordinate of its warp crosses a pixel border k + 1/2, i.e. where
 * FOE + d (1 - D t)/(1 - D tau) = k + 1/2, so D = (d - c)/(d t - c tau) with
 * c = k + 1/2 - FOE (binary64).  K is evaluated at the binary32 values
 * within 4 ulps of each breakpoint and at the binary32 midpoint of each gap
 * between neighbouring breakpoints, plus D_lo and D_hi; the binary32 warp
 * can only change pixel within a few ulps of a real breakpoint.  Exhaustive
 * for tiny windows only (cost ~ breakpoints x N). */
int or_sweep_max(const or_window* w, float D_lo, float D_hi, or_i128* K_max, float* D_at,
                 int64_t* n_evals) {
    int rc = or_validate(w, D_lo, D_hi);
    if (rc) return rc;
    double* bp = NULL;
    int64_t nb = 0, cap = 0;
    double tau = w->t_ref;                        /* the warp's reference time */
    for (int64_t i = 0; i < w->n; i++) {
        double ti = (double)(w->t[i] - w->t0);
        for (int ax = 0; ax < 2; ax++) {
            double foe = ax ? w->foe_y : w->foe_x;
            double d = (double)(ax ? w->y[i] : w->x[i]) - foe;
            if (d == 0.0) continue;
            double sl = (1.0 - D_lo * ti) / (1.0 - D_lo * tau), sh = (1.0 - D_hi * ti) / (1.0 - D_hi * tau);
            double p1 = foe + d * sl, p2 = foe + d * sh;
            double pmin = p1 < p2 ? p1 : p2, pmax = p1 < p2 ? p2 : p1;
            for (int64_t k = (int64_t)floor(pmin - 0.5) - 1; k <= (int64_t)floor(pmax - 0.5) + 1; k++) {
                double c = (double)k + 0.5 - foe;
                double den = d * ti - c * tau;
                if (den == 0.0) continue;
                double D = (d - c) / den;
                if (D >= D_lo && D <= D_hi) add_bp(&bp, &nb, &cap, D);
            }
        }
    }
    add_bp(&bp, &nb, &cap, D_lo);
    add_bp(&bp, &nb, &cap, D_hi);
    qsort(bp, (size_t)nb, sizeof(double), cmp_double);
    int64_t M = (int64_t)w->W * w->H;
    uint32_t* img = (uint32_t*)malloc((size_t)(planes(w) * M) * sizeof(uint32_t));
    if (!img) { free(bp); return OR_ERR_OOM; }
    i128 best = 0;
    float bd = D_lo;
    int64_t ne = 0;
    for (int64_t b = 0; b < nb; b++) {
        float cand[10];
        int nc = 0;
        float f = (float)bp[b];
        float lo = f, hi = f;
        cand[nc++] = f;
        for (int u = 0; u < 4; u++) {
            lo = nextafterf(lo, -INFINITY);
            hi = nextafterf(hi, INFINITY);
            cand[nc++] = lo;
            cand[nc++] = hi;
        }
        if (b + 1 < nb) cand[nc++] = (float)(0.5 * (bp[b] + bp[b + 1]));
        for (int c = 0; c < nc; c++) {
            float D = cand[c];
            if (!(D >= D_lo && D <= D_hi)) continue;
            uint64_t S;
            int64_t N;
            i128 k = eval_point(w, D, img, &S, &N);
            ne++;
            if (ne == 1 || k > best || (k == best && D < bd)) { best = k; bd = D; }
        }
    }
    free(img);
    free(bp);
    *K_max = pack(best);
    *D_at = bd;
    if (n_evals) *n_evals = ne;
    return OR_OK;
}

/* ------------------------------------------------- learned warm start */

/* Input features of the learned warm start: event counts in 16 radial x 8
 * temporal bins as the bin's share of the window's events relative to an
 * even spread, 128 * count / n (one binary32 division; 1 on average).  The radius is the
 * event's distance from the FOE relative to R, the largest distance from the
 * FOE to a corner pixel centre; radial bin floor(16 r / R) (at most 15).
 * The temporal bin is floor(8 (t - t0) / tau) (at most 7).  Every step is
 * one binary32 operation in the order written (sqrtf and the divisions are
 * correctly rounded), so the bins are decided in binary32. */
int or_features(const or_window* w, float* f, int64_t* counts) {
    int rc = or_validate(w, 0.0f, 0.0f);
    if (rc) return rc;
    int64_t c[OR_FEATURES];
    memset(c, 0, sizeof(c));
    const float ax = w->foe_x, bx = (float)(w->W - 1) - w->foe_x;
    const float ay = w->foe_y, by = (float)(w->H - 1) - w->foe_y;
    const float cx = ax > bx ? ax : bx, cy = ay > by ? ay : by;
    const float R2 = cx * cx + cy * cy;
    const float tsc = (float)OR_FEAT_T / w->tau;
    for (int64_t i = 0; i < w->n; i++) {
        const float dx = (float)w->x[i] - w->foe_x, dy = (float)w->y[i] - w->foe_y;
        const float r2 = dx * dx + dy * dy;
        const float u = R2 > 0.0f ? r2 / R2 : 0.0f;
        int rb = (int)floorf(sqrtf(u) * (float)OR_FEAT_R);
        if (rb > OR_FEAT_R - 1) rb = OR_FEAT_R - 1;
        const float v = (w->t[i] - w->t0) * tsc;
        int tb = (int)floorf(v);
        if (tb < 0) tb = 0;
        if (tb > OR_FEAT_T - 1) tb = OR_FEAT_T - 1;
        c[rb * OR_FEAT_T + tb]++;
    }
    for (int k = 0; k < OR_FEATURES; k++) {
        if (f) f[k] = w->n > 0 ? (float)(c[k] * OR_FEATURES) / (float)w->n : 0.0f;
        if (counts) counts[k] = c[k];
    }
    return OR_OK;
}

/* Parameter vector of the network 128 -> 128 -> 128 -> 2 (ReLU after the two
 * hidden layers), weight matrices row-major [out][in]:
 *   W1[128][128] b1[128] W2[128][128] b2[128] W3[2][128] b3[2]. */
enum {
    P_W1 = 0,
    P_B1 = P_W1 + OR_MLP_H * OR_FEATURES,
    P_W2 = P_B1 + OR_MLP_H,
    P_B2 = P_W2 + OR_MLP_H * OR_MLP_H,
    P_W3 = P_B2 + OR_MLP_H,
    P_B3 = P_W3 + OR_MLP_OUT * OR_MLP_H,
    P_END = P_B3 + OR_MLP_OUT
};

/* The network in binary32 as the device evaluates it: each unit starts from
 * its bias and adds weight * input for inputs 0, 1, ..., 127 in turn (one
 * rounded product, one rounded sum), then the ReLU. */
static void dense_f32(const float* Wt, const float* b, const float* x, int n_in, int n_out, int relu, float* y) {
    for (int j = 0; j < n_out; j++) {
        float acc = b[j];
        for (int k = 0; k < n_in; k++) acc = acc + Wt[j * n_in + k] * x[k];
        y[j] = relu && !(acc > 0.0f) ? 0.0f : acc;
    }
}

void or_mlp_forward_f32(const float* p, const float* x, float* out) {
    float h1[OR_MLP_H], h2[OR_MLP_H];
    dense_f32(p + P_W1, p + P_B1, x, OR_FEATURES, OR_MLP_H, 1, h1);
    dense_f32(p + P_W2, p + P_B2, h1, OR_MLP_H, OR_MLP_H, 1, h2);
    dense_f32(p + P_W3, p + P_B3, h2, OR_MLP_H, OR_MLP_OUT, 0, out);
}

/* The same network in binary64 (the definition the binary32 one is checked
 * against). */
static void dense_f64(const double* Wt, const double* b, const double* x, int n_in, int n_out, int relu,
                      double* y) {
    for (int j = 0; j < n_out; j++) {
        double acc = b[j];
        for (int k = 0; k < n_in; k++) acc += Wt[j * n_in + k] * x[k];
        y[j] = relu && !(acc > 0.0) ? 0.0 : acc;
    }
}

void or_mlp_forward_f64(const double* p, const double* x, double* h1, double* h2, double* out) {
    double a[OR_MLP_H], b[OR_MLP_H];
    if (!h1) h1 = a;
    if (!h2) h2 = b;
    dense_f64(p + P_W1, p + P_B1, x, OR_FEATURES, OR_MLP_H, 1, h1);
    dense_f64(p + P_W2, p + P_B2, h1, OR_MLP_H, OR_MLP_H, 1, h2);
    dense_f64(p + P_W3, p + P_B3, h2, OR_MLP_H, OR_MLP_OUT, 0, out);
}

/* Training loss of the warm start, mean over B samples.  Output 0 is the
 * guess u of the dimensionless product D tau, output 1 the log half-width l
 * of the interval around it, read as 3 standard deviations of a Gaussian:
 *     loss = 9/2 (u* - u)^2 exp(-2 l) + l
 * (its negative log-likelihood up to a constant).  With grad != NULL, writes
 * d loss / d p (backprop, ReLU derivative 1 where the pre-activation is > 0). */
double or_mlp_loss_f64(const double* p, const double* X, const double* u_star, int64_t B, double* grad) {
    if (grad) memset(grad, 0, sizeof(double) * P_END);
    double loss = 0.0;
    for (int64_t s = 0; s < B; s++) {
        const double* x = X + s * OR_FEATURES;
        double h1[OR_MLP_H], h2[OR_MLP_H], o[OR_MLP_OUT];
        or_mlp_forward_f64(p, x, h1, h2, o);
        const double e = u_star[s] - o[0];
        const double q = 9.0 * exp(-2.0 * o[1]);
        loss += 0.5 * q * e * e + o[1];
        if (!grad) continue;
        double go[OR_MLP_OUT];
        go[0] = -q * e / (double)B;
        go[1] = (1.0 - q * e * e) / (double)B;
        double g2[OR_MLP_H], g1[OR_MLP_H];
        for (int k = 0; k < OR_MLP_H; k++) {
            double a = 0.0;
            for (int j = 0; j < OR_MLP_OUT; j++) {
                grad[P_W3 + j * OR_MLP_H + k] += go[j] * h2[k];
                a += p[P_W3 + j * OR_MLP_H + k] * go[j];
            }
            g2[k] = h2[k] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < OR_MLP_OUT; j++) grad[P_B3 + j] += go[j];
        for (int k = 0; k < OR_MLP_H; k++) {
            double a = 0.0;
            for (int j = 0; j < OR_MLP_H; j++) {
                grad[P_W2 + j * OR_MLP_H + k] += g2[j] * h1[k];
                a += p[P_W2 + j * OR_MLP_H + k] * g2[j];
            }
            g1[k] = h1[k] > 0.0 ? a : 0.0;
        }
        for (int j = 0; j < OR_MLP_H; j++) grad[P_B2 + j] += g2[j];
        for (int j = 0; j < OR_MLP_H; j++) {
            for (int k = 0; k < OR_FEATURES; k++) grad[P_W1 + j * OR_FEATURES + k] += g1[j] * x[k];
            grad[P_B1 + j] += g1[j];
        }
    }
    return loss / (double)B;
}

/* From the network's outputs to a warm start for a window of length tau:
 * D_warm = u / tau; the half-width exp(l) is rounded to the nearest power
 * of two 2^e (e = floor(l log2(e) + 1/2), clamped to [-20, 1]; NaN gives
 * -20) and w_warm = 2^e / tau. */
void or_warm_map(float u, float l, float tau, float* D_warm, float* w_warm) {
    *D_warm = u / tau;
    float v = l * OR_LOG2E + 0.5f;
    if (!(v >= -20.0f)) v = -20.0f;
    if (v > 1.0f) v = 1.0f;
    *w_warm = ldexpf(1.0f, (int)floorf(v)) / tau;
}

/* ------------------------------------------------ resized and resampled */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output i of the sequence
 * seeded with `state0` is the finaliser applied to state0 + (i + 1) * G. */
static uint64_t sm64(uint64_t state0, uint64_t i) {
    uint64_t z = state0 + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The paper's fast mode (Sec. 6, the resized and resampled sequences): event
 * coordinates scaled to a W2 x H2 frame and a random share `keep` of the
 * events kept.  Reading: a scaled coordinate goes to the nearest coarse pixel
 * centre, x2 = floor(x k + 1/2) with k = W2/W (binary32), clamped to the
 * frame; event i is kept when the top 24 bits of SplitMix64 output i of key
 * SplitMix64(seed, 0) fall below floor(keep 2^24).  Kept events keep their
 * order and times.  Returns the kept count (x2, y2, t2 have room for n). */
int64_t or_resample(const or_window* w, int32_t W2, int32_t H2, float keep, uint64_t seed, int16_t* x2, int16_t* y2,
                    float* t2) {
    const float kx = (float)W2 / (float)w->W, ky = (float)H2 / (float)w->H;
    const uint64_t key = sm64(seed, 0);
    const uint64_t thr = (uint64_t)floor((double)keep * 16777216.0);
    int64_t m = 0;
    for (int64_t i = 0; i < w->n; i++) {
        if ((sm64(key, (uint64_t)i) >> 40) >= thr) continue;
        int32_t cx = (int32_t)floorf((float)w->x[i] * kx + 0.5f);
        int32_t cy = (int32_t)floorf((float)w->y[i] * ky + 0.5f);
        if (cx > W2 - 1) cx = W2 - 1;
        if (cy > H2 - 1) cy = H2 - 1;
        x2[m] = (int16_t)cx;
        y2[m] = (int16_t)cy;
        t2[m] = w->t[i];
        m++;
    }
    return m;
}

/* The FOE in the coarse frame: foe k (binary32). */
void or_resample_foe(const or_window* w, int32_t W2, int32_t H2, float* fx2, float* fy2) {
    *fx2 = w->foe_x * ((float)W2 / (float)w->W);
    *fy2 = w->foe_y * ((float)H2 / (float)w->H);
}
