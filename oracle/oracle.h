/*
 * CPU oracle for exact contrast-maximisation divergence estimation
 * (McLeod et al., "Globally Optimal Event-Based Divergence Estimation for
 * Ventral Landing", arXiv 2209.13168).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * never links, loads or calls it, and shares no code with it.
 *
 * Plain, slow, obviously correct: every function follows one equation or
 * algorithm of the paper, cited at its definition in oracle.c.
 *
 * Parametrisation (reading of Sec. 4.1): the search variable is D = -nu, the
 * divergence at the window start with Z0 = 1, positive while approaching.
 * The warp of Eq. (11) to t = tau becomes
 *     x' = FOE + (x - FOE) * (1 - D t) / (1 - D tau);
 * or_window.t_ref generalises the reference time (tau in the paper):
 *     x' = FOE + (x - FOE) * (1 - D t) / (1 - D t_ref).
 * or_window.p, when given, splits the image of warped events into one plane
 * per polarity; the objective is the sum of the planes' contrasts, and images
 * (iwe arguments) hold both planes, plane 0 first (2 W H cells).
 *
 * Parity pins: see the module docstring of oracle/__init__.py and the tests
 * under tests/test_oracle_*.py.  Every function here is pinned.
 */
#ifndef DD_ORACLE_H
#define DD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t W, H;            /* frame size in pixels                              */
    float foe_x, foe_y;      /* focus of expansion, pixel units                    */
    const int16_t *x, *y;    /* event pixel coordinates [n]                        */
    const float *t;          /* event times [n], in [t0, t0 + tau]                 */
    int64_t n;
    float t0, tau;
    float t_ref;             /* time (since t0) the warp maps events to, in [0, tau]: */
                             /* the paper's tau, or 0 (the start of the window)       */
    const int8_t *p;         /* event polarities [n], or NULL: polarity unused (the   */
                             /* paper's objective); else one image per polarity      */
                             /* (plane 0: p > 0, plane 1: p <= 0), contrasts added   */
} or_window;

typedef struct { uint64_t lo; int64_t hi; } or_i128;   /* two's complement, little end first */

typedef struct {
    float D_star, D_end;
    double contrast, bound_gap;
    or_i128 K_hat, gap_K;
    int64_t nodes_expanded, point_evals, bound_evals, event_warps, cell_increments;
    int64_t bound_increments, rounds, max_queue;
    int32_t status;
} or_result;

typedef struct {            /* one expanded node, in expansion order */
    float D_lo, D_hi, D_c;
    int32_t leaf;
    or_i128 Kbar, K_c;
} or_node_rec;

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_OOM = -2 };

int or_validate(const or_window* w, float D_lo, float D_hi);
void or_warp_cells(const or_window* w, float D, int32_t* ux, int32_t* uy);
int64_t or_fp64_disagreements(const or_window* w, float D);
float or_scale(float D, float t_rel, float tau);
void or_scale_interval(float D_lo, float D_hi, float t_rel, float tau, float* s_a, float* s_b);
int or_contrast(const or_window* w, float D, or_i128* K, uint64_t* S, int64_t* N_in, uint32_t* iwe);
int or_bound(const or_window* w, float D_lo, float D_hi, or_i128* Kbar, uint64_t* Sbar,
             int64_t* N_full, uint32_t* iwe);
int or_solve(const or_window* w, float D_lo, float D_hi, float tol_D, double gamma, int32_t K_pop,
             or_result* out, or_node_rec* trace, int64_t trace_cap, int64_t* trace_len);
/* Algorithm 1 with an optional warm start (warm = 1): the first incumbent is
 * D_warm (clamped into the domain) instead of the centre, and the domain is
 * queued as the pieces cut at D_warm -/+ w_warm (w_warm > 0).  warm = 0 is
 * or_solve. */
int or_solve_warm(const or_window* w, float D_lo, float D_hi, float tol_D, double gamma, int32_t K_pop,
                  int32_t warm, float D_warm, float w_warm, or_result* out, or_node_rec* trace,
                  int64_t trace_cap, int64_t* trace_len);
int or_grid_max(const or_window* w, float D_lo, float D_hi, float h, or_i128* K_max, float* D_at,
                int64_t* n_evals);
int or_sweep_max(const or_window* w, float D_lo, float D_hi, or_i128* K_max, float* D_at,
                 int64_t* n_evals);

/* Learned warm start (features, network, loss, mapping to a warm start). */
#define OR_FEAT_R 16
#define OR_FEAT_T 8
#define OR_FEATURES (OR_FEAT_R * OR_FEAT_T)
#define OR_MLP_H 128
#define OR_MLP_OUT 2
#define OR_MLP_PARAMS (OR_MLP_H * OR_FEATURES + OR_MLP_H + OR_MLP_H * OR_MLP_H + OR_MLP_H + \
                       OR_MLP_OUT * OR_MLP_H + OR_MLP_OUT)
#define OR_LOG2E 1.44269504f
int or_features(const or_window* w, float* f, int64_t* counts);
void or_mlp_forward_f32(const float* params, const float* x, float* out);
void or_mlp_forward_f64(const double* params, const double* x, double* h1, double* h2, double* out);
double or_mlp_loss_f64(const double* params, const double* X, const double* u_star, int64_t B, double* grad);
void or_warm_map(float u, float l, float tau, float* D_warm, float* w_warm);

/* Fast mode: coordinates scaled to W2 x H2, a random share `keep` kept. */
int64_t or_resample(const or_window* w, int32_t W2, int32_t H2, float keep, uint64_t seed, int16_t* x2, int16_t* y2,
                    float* t2);
void or_resample_foe(const or_window* w, int32_t W2, int32_t H2, float* fx2, float* fy2);

#ifdef __cplusplus
}
#endif
#endif
