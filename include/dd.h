/*
 * dd.h -- C ABI of the GB300 (sm_103a) exact divergence estimator.
 *
 * The estimator is the contrast-maximisation method of McLeod et al.,
 * "Globally Optimal Event-Based Divergence Estimation for Ventral Landing"
 * (arXiv 2209.13168): every event of a window is warped radially about the
 * focus of expansion (FOE) to the end of the window (Eq. 11), counted into an
 * image of warped events (IWE, Eq. 12), and the contrast of that image
 * (Eq. 13) is maximised over the divergence by branch and bound
 * (Algorithm 1) with the interval upper bound of Eqs. 14-19.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Search variable.  D is the divergence at the window start with Z0 = 1,
 *   positive while approaching: D = -nu, where nu is the vertical velocity of
 *   Sec. 4.1.  The warp of event i (pixel x_i, time t_i, relative to t0) is
 *       x' = FOE + (x_i - FOE) * (1 - D t_i) / (1 - D tau),
 *   evaluated in IEEE binary32 with one rounding per operation in the order
 *       g = 1/(1 - D*tau);  s = (1 - D*t_i)*g;  x' = FOE + (x_i - FOE)*s,
 *   and the pixel is floor(x' + 1/2) (pixel u covers [u - 1/2, u + 1/2)).
 * - Domain.  Every D satisfies -64 <= D*tau <= 3/4 (the widening that keeps
 *   the bound valid in binary32 is proven on that range; the paper's singular
 *   end nu = -1/tau is excluded).
 * - Contrast key.  Contrast is reported and compared as the exact integer
 *       K = M * S - N_in^2 = M^2 * C,   S = sum_u H(u)^2,  N_in = sum_u H(u),
 *   M = W*H, as a signed 128-bit value (dd_i128).
 * - Status.  Every int-returning function returns DD_OK (0) or a negative
 *   DD_ERR_* code; outputs are written only on DD_OK.  dd_strerror() names it.
 * - Memory.  Host pointers are read (or written) during the call only and stay
 *   owned by the caller.  With dd_events.device_ptrs = 1, x/y/t are device
 *   pointers of the context's GPU, read in place and never retained.  The
 *   context owns its device buffers (allocated by dd_create and grown on
 *   demand), its CUDA stream and its BnB queue.
 * - Threads.  A context is not thread-safe: use one context per host thread.
 * - Events.  0 <= x < W, 0 <= y < H, t finite with 0 <= (t - t0) <= tau (the
 *   difference taken in binary32).  Polarity is not read (Sec. 4.2: the
 *   paper's objective leaves it out), unless the context was created with
 *   dd_config.polarity = 1.
 * - Polarity planes (dd_config.polarity = 1; the paper notes that polarity
 *   could be used and does not say how).  Each polarity gets its own image:
 *   plane 0 holds the events with p > 0, plane 1 those with p <= 0, each of
 *   M = W*H pixels, and the objective is the sum of the two planes' contrasts:
 *       K = M (S_0 + S_1) - N_0^2 - N_1^2,
 *   bounded plane by plane by Eqs. 14-19 (Kbar = M (Sbar_0 + Sbar_1) -
 *   N_full,0^2 - N_full,1^2).  S, N_in, N_full outputs are the planes' totals;
 *   images hold both planes, plane 0 first (2 M cells per hypothesis).
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    DD_OK = 0,
    DD_ERR_ARG = -1,            /* invalid argument or malformed events          */
    DD_ERR_OOM = -2,            /* device or host allocation failed              */
    DD_ERR_QUEUE_OVERFLOW = -3, /* the BnB queue exceeded its capacity           */
    DD_ERR_TIMEOUT = -4,        /* the round limit was reached before the proof  */
    DD_ERR_CUDA = -5,           /* a CUDA runtime call failed                    */
    DD_ERR_NO_DEVICE = -6,      /* no usable sm_103 device                       */
    DD_ERR_CAPACITY = -7,       /* input exceeds a fixed capacity (no-alloc scratch, */
                                /* serving slot)                                     */
    DD_ERR_CANCELLED = -8,      /* dd_serve_cancel stopped the request              */
    DD_PENDING = 1              /* dd_serve_poll: the request has not finished yet   */
};

typedef struct dd_ctx dd_ctx;

/* Signed 128-bit integer, two's complement, low word first. */
typedef struct { uint64_t lo; int64_t hi; } dd_i128;

/* Tuning knobs; pass NULL to dd_create for the defaults (0 = default). */
typedef struct {
    int32_t pop_k;          /* intervals dequeued per BnB round (default 1 = Algorithm 1) */
    int32_t queue_capacity; /* BnB queue entries per window (default 8192)               */
    int32_t band_rows;      /* rows of the shared-memory IWE tile (default: from W)      */
    int32_t threads;        /* threads per block of the IWE kernels, a multiple of 32    */
                            /* up to 512 (default 512)                                    */
    int32_t max_rounds;     /* BnB round limit, DD_ERR_TIMEOUT beyond (default 1<<20)    */
    int32_t host_loop;      /* 0: each solve's rounds run as one CUDA graph with a       */
                            /*    conditional loop (no host round trips); 1: the host    */
                            /*    launches the rounds in batches and polls for the end   */
    int32_t max_splits;     /* most blocks that share one row band of a bound (default 16) */
    int32_t warp_to_start;  /* 0: events warped to the window's end (Eq. 11, the paper's  */
                            /*    reference time tau); 1: to its start (reference time 0: */
                            /*    x' = FOE + (x - FOE)(1 - D t), linear in D)             */
    int32_t polarity;       /* 0: polarity unused (the paper's objective); 1: one image   */
                            /*    per polarity, contrasts added (H <= 2048; every        */
                            /*    dd_events must then carry p)                            */
    int32_t fuse_span;      /* an expanded interval whose events move by at most          */
                            /*    fuse_span/100 pixel across it (estimated from the scale  */
                            /*    change, as the split rule does) has its centre and both  */
                            /*    halves evaluated in one pass; 0: default (25), < 0:      */
                            /*    never.  A schedule choice: results do not depend on it   */
} dd_config;

/* One window of events in structure-of-arrays form. */
typedef struct {
    const int16_t* x;       /* [n] pixel column                                    */
    const int16_t* y;       /* [n] pixel row                                       */
    const float* t;         /* [n] timestamp, in [t0, t0 + tau]                    */
    int64_t n;              /* number of events, >= 0                              */
    float t0;               /* window start                                        */
    float tau;              /* window length, > 0                                  */
    int32_t device_ptrs;    /* 0: host arrays (copied in); 1: device arrays        */
    const int8_t* p;        /* [n] polarity (same memory as x/y/t): read only by a */
                            /* context with polarity = 1, which requires it;       */
                            /* NULL otherwise                                      */
} dd_events;

/* Result of one exact solve (Algorithm 1). */
typedef struct {
    float D_star;           /* incumbent divergence (window start), Sec. 4.1       */
    float D_end;            /* D_star/(1 - D_star tau): the paper's point estimate  */
                            /* nu_s/(1 + nu_s tau) with nu_s = -D_star, sign       */
                            /* flipped (positive while approaching), Sec. 4.1      */
    double contrast;        /* K_hat / M^2 = C(D_star), Eq. 13                      */
    double bound_gap;       /* gap_K / M^2: certified distance to the optimum       */
    dd_i128 K_hat;          /* contrast key of D_star                               */
    dd_i128 gap_K;          /* max(0, best open or leaf bound - K_hat)              */
    int64_t nodes_expanded; /* intervals dequeued and evaluated                     */
    int64_t point_evals;    /* contrast evaluations (root incumbent included)       */
    int64_t bound_evals;    /* upper-bound evaluations                              */
    int64_t event_warps;    /* n * (point_evals + bound_evals)                      */
    int64_t cell_increments;/* IWE increments over all evaluations                  */
    int64_t bound_increments;/* of which in bound images (Eq. 16)                   */
    int64_t rounds;         /* BnB rounds (dequeue batches)                         */
    int64_t max_queue;      /* largest queue length seen                            */
    int32_t status;         /* DD_OK                                                */
    float D_warm, w_warm;   /* the warm start the search began from (guess, clamped */
                            /* into the domain, and half-width); 0, 0 without one   */
} dd_result;

/* Warm start of one search (dd_window_params.warm). */
enum {
    DD_WARM_NONE = 0,       /* Algorithm 1 as printed: the first incumbent is the   */
                            /* centre of the domain, which is queued whole          */
    DD_WARM_GIVEN = 1,      /* start from the caller's guess D_warm +- w_warm       */
    DD_WARM_MODEL = 2       /* start from the context's learned model's guess       */
                            /* (dd_set_warm_model), computed on the device          */
};

/* Search parameters of one window of dd_solve_batch / dd_serve_submit. */
typedef struct {
    float D_lo, D_hi;       /* search range, D_lo < D_hi, both in the domain        */
    float tol_D;            /* leaf width (>= 0)                                     */
    int32_t warm;           /* DD_WARM_*                                             */
    double gamma;           /* stopping gap of Algorithm 1, contrast units (>= 0)    */
    float D_warm, w_warm;   /* DD_WARM_GIVEN: guess (finite) and half-width (> 0)   */
} dd_window_params;
/* A warm start changes where the search begins, never what it certifies:
 * the guess, clamped into [D_lo, D_hi], is the first incumbent in place of
 * the centre, and the domain enters the queue as the pieces
 * [D_lo, a], [a, b], [b, D_hi] of positive width, a = max(D_lo, guess - w),
 * b = min(D_hi, guess + w) (binary32), each queued if its bound reaches the
 * incumbent.  The certificate (gap_K) keeps its meaning. */

/* One expanded interval, in expansion order (dd_solve_trace). */
typedef struct {
    float D_lo, D_hi, D_c;
    int32_t leaf;           /* 1: not split (width <= tol_D or unsplittable)        */
    dd_i128 Kbar;           /* its bound key when dequeued                          */
    dd_i128 K_c;            /* contrast key at its centre                           */
} dd_node_rec;

/* Create a context for W x H frames (1..4096 each) with the FOE at
 * (foe_x, foe_y) in [0, W] x [0, H], on the current CUDA device (which must
 * be sm_103).  Allocates the context's device buffers and stream.
 * Errors: DD_ERR_ARG, DD_ERR_NO_DEVICE, DD_ERR_OOM, DD_ERR_CUDA. */
int dd_create(int32_t W, int32_t H, float foe_x, float foe_y, const dd_config* cfg, dd_ctx** out);

/* Release everything the context owns.  NULL is ignored. */
void dd_destroy(dd_ctx* ctx);

/* Run the context's work on `stream` (a cudaStream_t of the context's
 * device; NULL restores the context's own stream).  Every call still
 * synchronises that stream before returning its host results. */
int dd_set_stream(dd_ctx* ctx, void* stream);

/* Eqs. 11-13: the contrast key at each of nD hypotheses D[j] (host array).
 * Writes K[j] (required) and, where non-NULL, S[j], N_in[j], and the IWE of
 * every hypothesis to iwe[j*M + y*W + x] (host, nD*M uint32; with polarity
 * planes iwe[(2 j + plane) M + y W + x], 2 nD M uint32).
 * Errors: DD_ERR_ARG (bad events, D outside the domain, nD < 0), DD_ERR_OOM,
 * DD_ERR_CUDA. */
int dd_contrast(dd_ctx* ctx, const dd_events* ev, const float* D, int32_t nD, dd_i128* K,
                uint64_t* S, int64_t* N_in, uint32_t* iwe);

/* Eqs. 14-19: the bound key Kbar = M * Sbar - N_full^2 >= K(D) for every
 * binary32 D in [D_lo[j], D_hi[j]], j < n (host arrays, D_lo[j] <= D_hi[j]).
 * Hbar (Eq. 16) counts, per event, each pixel its segment
 * f(D_lo) <-> f(D_hi) passes through; N_full (Eq. 19, times M) counts the
 * events whose segment lies in the frame.  Optional outputs as dd_contrast.
 * Errors: as dd_contrast. */
int dd_bound(dd_ctx* ctx, const dd_events* ev, const float* D_lo, const float* D_hi, int32_t n,
             dd_i128* Kbar, uint64_t* Sbar, int64_t* N_full, uint32_t* iwe);

/* Algorithm 1: maximise the contrast over D in [D_lo, D_hi] (D_lo < D_hi).
 * Intervals no wider than tol_D (>= 0) are not split; gamma >= 0 is the
 * stopping gap of Algorithm 1 in contrast units.  The search runs on the
 * GPU: bounds, contrasts, the priority queue (largest Kbar first, ties to the
 * smaller D_lo), the incumbent update (a centre with K >= K_hat wins) and
 * pruning.  With pop_k > 1 each round dequeues up to pop_k intervals.
 * Errors: DD_ERR_ARG, DD_ERR_OOM, DD_ERR_QUEUE_OVERFLOW, DD_ERR_TIMEOUT,
 * DD_ERR_CUDA. */
int dd_solve(dd_ctx* ctx, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma,
             dd_result* out);

/* Algorithm 1 for n_windows independent windows at once (all of the
 * context's frame geometry): every round evaluates the pending intervals of
 * all windows in one launch and runs one control block per window; each
 * window keeps its own device-resident queue and incumbent, and a window that
 * has finished simply stops contributing work.  The rounds run as one CUDA
 * graph (or host-driven batches with dd_config.host_loop).  windows[w] and
 * params[w] (host arrays) describe window w; out[w] receives its result,
 * identical to dd_solve on that window alone with the same pop_k.
 * Returns DD_OK when every window succeeded; otherwise the first failing
 * window's status, with each out[w].status set (results of failed windows
 * are unspecified).  Errors: as dd_solve; DD_ERR_ARG if n_windows < 1. */
int dd_solve_batch(dd_ctx* ctx, const dd_events* windows, int32_t n_windows, const dd_window_params* params,
                   dd_result* out);

/* dd_solve that also records up to trace_cap expanded intervals (host
 * array) and their total count in *trace_len. */
int dd_solve_trace(dd_ctx* ctx, const dd_events* ev, float D_lo, float D_hi, float tol_D,
                   double gamma, dd_result* out, dd_node_rec* trace, int64_t trace_cap,
                   int64_t* trace_len);

/* One window with full search parameters (warm start included) and an
 * optional trace as dd_solve_trace (trace_cap 0: none). */
int dd_solve_window(dd_ctx* ctx, const dd_events* ev, const dd_window_params* p, dd_result* out,
                    dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len);

/* The paper's fast mode (Sec. 6, the resized and resampled sequences): the
 * events of a W x H window with their coordinates scaled to a W2 x H2 frame
 * and a random share `keep` (in [0, 1]) of them kept -- an ordinary window
 * for a context of the coarse frame, whose FOE dd_resample_foe gives.
 * Event i goes to the nearest coarse pixel centre, floor(x (W2/W) + 1/2) in
 * binary32 (likewise y), clamped to the frame, and is kept when the top 24
 * bits of output i of SplitMix64 with key SplitMix64(seed, 0) fall below
 * floor(keep 2^24).  Kept events keep their order and times.
 *   in           events of the fine frame (host or device, as dd_events)
 *   x_out, y_out, t_out  DEVICE arrays with room for in->n events
 *   n_out        receives the kept count (host)
 * Runs on the context's stream and synchronises it.  Errors: DD_ERR_ARG
 * (sizes outside 1..4096, keep outside [0, 1], events outside the fine
 * frame), DD_ERR_OOM, DD_ERR_CUDA. */
int dd_resample(dd_ctx* ctx, const dd_events* in, int32_t W, int32_t H, int32_t W2, int32_t H2, float keep,
                uint64_t seed, int16_t* x_out, int16_t* y_out, float* t_out, int64_t* n_out);

/* The stream-wise estimation of Sec. 4.4: the divergence of a time-sorted
 * event stream, window by window.  Window k covers [t0_k, t0_k + tau] with
 * t0_k = (float)(t_start + k hop): the events whose (t - t0_k) lies in
 * [0, tau] in binary32 (the test dd_solve applies), found by binary search
 * and read in place (a device stream is not copied), solved together as one
 * dd_solve_batch with the same params for every window.
 *   stream   events sorted by t (host or device), its t0/tau ignored
 *   out[k]   window k's result (status per window, as dd_solve_batch)
 *   ttc[k]   (nullable) its time to contact at the window's end, 1/D_end in
 *            seconds; infinity when D_end <= 0 or the window failed
 *   first[k] (nullable) index of window k's first event in the stream
 * Returns as dd_solve_batch.  Errors: DD_ERR_ARG (tau <= 0, hop <= 0,
 * n_windows < 1, non-finite t_start), and dd_solve_batch's. */
int dd_stream_solve(dd_ctx* ctx, const dd_events* stream, double t_start, float tau, double hop, int32_t n_windows,
                    const dd_window_params* params, dd_result* out, float* ttc, int64_t* first);

/* Checked builds (compiled with -DDD_CHECKED): the evaluation kernels test
 * every index into a shared tile, a window's events, a split accumulator and
 * the sorted-event output before using it; an index out of range sets a bit
 * of an error word and the access is skipped (bits: 1 point and one-pixel
 * tile cells, 2 segment tile cells, 4 event indices, 8 ingest positions, 16
 * accumulator and image cells).  *flags = that word of the current device
 * (0 in other builds), *checked = 1 in a checked build; reset != 0 clears
 * it.  Errors: DD_ERR_ARG (null outputs), DD_ERR_CUDA. */
int dd_check_flags(uint32_t* flags, int32_t* checked, int32_t reset);

/* The time span of a batch (Sec. 3.3 measures a batch's times from its
 * earliest event, so the batch covers [0, tau]): t0 = the least finite
 * timestamp, tau = (greatest - least) in binary32, so every event passes
 * the solver's window test 0 <= t - t0 <= tau.  ev's t0/tau are ignored;
 * device arrays are reduced on the context's stream.  Errors: DD_ERR_ARG
 * (n < 1, no finite timestamp, or all timestamps equal: no span). */
int dd_time_span(dd_ctx* ctx, const dd_events* ev, float* t0, float* tau);

/* The FOE of the coarse frame: foe (W2/W), foe (H2/H) in binary32. */
int dd_resample_foe(int32_t W, int32_t H, float foe_x, float foe_y, int32_t W2, int32_t H2, float* foe_x2,
                    float* foe_y2);

/* Counters of one context since dd_create or the last dd_reset_stats. */
typedef struct {
    int64_t kernel_launches;  /* kernels this library launched                      */
    int64_t eval_launches;    /* of which IWE evaluation kernels                    */
    int64_t h2d_bytes;        /* bytes copied host -> device                        */
    int64_t d2h_bytes;        /* bytes copied device -> host                        */
    int64_t host_syncs;       /* stream synchronisations                            */
    int64_t timed_launches;   /* IWE kernel launches timed (dd_set_timing)          */
    double eval_ms;           /* their summed device time, CUDA events on the        */
                              /* context's stream                                   */
} dd_stats;

/* Read (and, with dd_reset_stats, clear) the counters.  No GPU work. */
int dd_get_stats(dd_ctx* ctx, dd_stats* out);
int dd_reset_stats(dd_ctx* ctx);

/* enable != 0: bracket every IWE evaluation launch with CUDA events on the
 * context's stream and add its duration to dd_stats.eval_ms (costs a few
 * microseconds per launch; off by default).  While timing is on, a solve
 * launches its rounds from the host one round per poll (dd_config.host_loop
 * behaviour without the batching), so every timed launch evaluates work:
 * launch k of a solve is its round k. */
int dd_set_timing(dd_ctx* ctx, int32_t enable);

/* Telemetry: the device durations (ms) of the timed IWE launches since the
 * last dd_reset_stats, in launch order, the first DD_MAX_LAUNCH_TIMES of
 * them.  Copies min(cap, count) entries into ms (host array) and the count
 * into *n.  No GPU work.  Errors: DD_ERR_ARG (null ctx or n, cap < 0, ms
 * NULL with cap > 0). */
#define DD_MAX_LAUNCH_TIMES 65536
int dd_get_launch_times(dd_ctx* ctx, float* ms, int32_t cap, int32_t* n);

/* ------------------------------------------------------------------------
 * Learned warm start.  An extension of the paper's method: its Algorithm 1
 * starts every search from the centre of the domain; here a small network
 * trained on exactly solved windows proposes where to start instead.
 *
 * Features: the window's events counted in 16 radial x 8 temporal bins,
 * each count as 128 * count / n (the bin's share relative to an even
 * spread); feature 8*r + k counts radial bin r = floor(16 d/R) and
 * temporal bin k = floor(8 (t - t0)/tau) (each clamped to the last bin), d the
 * event's distance from the FOE and R the largest distance from the FOE to a
 * corner pixel centre, every step one binary32 operation.
 * Network: 128 -> 128 -> 128 -> 2, ReLU after both hidden layers, weights
 * bfloat16, biases, activations and accumulation binary32; each unit adds
 * weight * input for inputs 0..127 in turn onto its bias.  Output 0 is a
 * guess u of D*tau, output 1 the log of the half-width l (in D*tau units).
 * The guess is D_warm = u / tau and the half-width w_warm = 2^e / tau, e =
 * floor(l log2(e) + 1/2) clamped to [-20, 1].
 * Parameters (dd_mlp_get_params / set_params, host float arrays of
 * DD_MLP_PARAMS): W1[128][128] b1[128] W2[128][128] b2[128] W3[2][128] b3[2],
 * matrices [out][in] row-major.
 * Training loss: mean over samples of 9/2 (u* - u)^2 exp(-2 l) + l,
 * u* = D* tau of the exact solve (the negative log-likelihood of a Gaussian
 * whose 3 standard deviations are the half-width).
 */
#define DD_MLP_FEATURES 128
#define DD_MLP_PARAMS 33282
typedef struct dd_mlp dd_mlp;

/* A model on the current device, weights drawn uniformly in
 * +-sqrt(6/fan_in) from `seed` (biases 0, except b3[1] = log(0.05)).
 * Errors: DD_ERR_NO_DEVICE, DD_ERR_OOM, DD_ERR_CUDA. */
int dd_mlp_create(uint64_t seed, dd_mlp** out);
void dd_mlp_destroy(dd_mlp* m);

/* Run the model's work on `stream` (NULL: the legacy default stream). */
int dd_mlp_set_stream(dd_mlp* m, void* stream);

/* The parameters the network evaluates with (weights rounded to bfloat16),
 * n = DD_MLP_PARAMS floats (host).  set_params also resets the optimiser. */
int dd_mlp_get_params(dd_mlp* m, float* params, int64_t n);
int dd_mlp_set_params(dd_mlp* m, const float* params, int64_t n);

/* Save / load the binary32 master parameters: a 32-byte header ("DDMLP001",
 * parameter count, optimiser step, reserved) and DD_MLP_PARAMS
 * little-endian floats.  Errors: DD_ERR_ARG (I/O, bad header). */
int dd_mlp_save(dd_mlp* m, const char* path);
int dd_mlp_load(dd_mlp* m, const char* path);

/* Network outputs for B samples: X [B][128] and out [B][2] in DEVICE memory.
 * Synchronises the model's stream.  Errors: DD_ERR_ARG (B < 0, NULL),
 * DD_ERR_CUDA. */
int dd_mlp_forward(dd_mlp* m, const float* X, int32_t B, float* out);

/* Gradient of the training loss over B samples (1 <= B <= 4096): X [B][128],
 * u_star [B], grad [DD_MLP_PARAMS] and loss [1] in DEVICE memory (grad in
 * the parameter layout above; weight gradients are with respect to the
 * bfloat16 weights the network evaluates with).  Asynchronous on the model's
 * stream. */
int dd_mlp_grad(dd_mlp* m, const float* X, const float* u_star, int32_t B, float* grad, float* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) of learning rate lr on
 * the master parameters from the gradient over the B samples; the bfloat16
 * weights are re-rounded.  loss (DEVICE, nullable) receives the loss before
 * the step.  Asynchronous on the model's stream. */
int dd_mlp_train_step(dd_mlp* m, const float* X, const float* u_star, int32_t B, float lr, float* loss);

/* The features of n_windows windows (all of the context's geometry) into
 * feat [n_windows][128] in DEVICE memory, computed on the context's stream
 * (synchronised before return).  Errors: as dd_solve_batch's checks. */
int dd_features(dd_ctx* ctx, const dd_events* windows, int32_t n_windows, float* feat);

/* The model that DD_WARM_MODEL windows of this context (and of servers
 * started from it afterwards) take their warm start from; NULL clears it.
 * The model must live on the context's device and outlive its use. */
int dd_set_warm_model(dd_ctx* ctx, dd_mlp* m);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of windows from concurrent event streams
 * (the stream-wise estimation of Sec. 4.4, one estimate per window).
 *
 * A server owns max_slots device slots, each holding one window of up to
 * max_events events with its whole search state, and one host thread that
 * loops: admit every request whose arrival time has passed into a free slot
 * (copy in, ingest, start its search), run one BnB round for every busy slot
 * in shared launches, retire finished windows.  Requests join and leave
 * between rounds while others are running; each window's result is the same
 * as dd_solve on it alone with the context's pop_k.  The server uses the
 * context's geometry and knobs but its own buffers and stream.
 */
typedef struct dd_server dd_server;

/* Start a server.  max_slots = 0 picks the slot count from free device
 * memory (at most half of it, at most 64 slots).  Errors: DD_ERR_ARG,
 * DD_ERR_OOM, DD_ERR_CUDA. */
int dd_serve_start(dd_ctx* ctx, int32_t max_slots, int64_t max_events, dd_server** out);

/* The server's slot count and per-slot event capacity. */
int dd_serve_slots(dd_server* s, int32_t* slots, int64_t* max_events);

/* Queue one window (events and search parameters) that arrives at
 * arrival_s on the dd_serve_clock() scale (negative: now); it is admitted no
 * earlier than that.  The event arrays (host or device, ev->device_ptrs) must
 * stay valid and unchanged until the request finishes.  Writes a ticket.
 * Errors: DD_ERR_ARG, DD_ERR_CAPACITY (ev->n > max_events), a previous
 * DD_ERR_CUDA of the server. */
int dd_serve_submit(dd_server* s, const dd_events* ev, const dd_window_params* p, double arrival_s,
                    uint64_t* ticket);

/* Cancel a request.  Not yet admitted: it is dropped.  Running: its search
 * stops at the end of the current round (its slot's evaluations of that
 * round complete; nothing of it reaches other windows).  Finished: nothing
 * changes.  dd_serve_poll / dd_serve_wait then return the request's status,
 * DD_ERR_CANCELLED for a cancelled one.  Errors: DD_ERR_ARG (unknown or
 * already collected ticket). */
int dd_serve_cancel(dd_server* s, uint64_t ticket);

/* DD_PENDING while the request runs or waits; otherwise its status (results
 * and latency = finish time - arrival time, in seconds, written when not
 * NULL), and the ticket is released. */
int dd_serve_poll(dd_server* s, uint64_t ticket, dd_result* out, double* latency_s);

/* As dd_serve_poll, but blocks until the request has finished. */
int dd_serve_wait(dd_server* s, uint64_t ticket, dd_result* out, double* latency_s);

/* Rounds run, requests admitted and the largest number of windows that
 * shared a round, since dd_serve_start. */
int dd_serve_stats(dd_server* s, int64_t* rounds, int64_t* admitted, int64_t* peak_busy);

/* Finish every queued request, stop the loop thread and free the server. */
int dd_serve_stop(dd_server* s);

/* The serving clock: seconds on a monotonic clock. */
double dd_serve_clock(void);

/* ------------------------------------------------------------------------
 * Allocation-free contrast evaluation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * time they evaluate contrasts -- flight or embedded software whose rules
 * forbid any allocation after start-up (so no allocation can fail in the
 * guidance loop), or a plugin inside a host process that owns all device
 * memory through its own capped pool, where a cudaMalloc would bypass its
 * accounting or fail.
 *
 * dd_contrast_noalloc computes exactly what dd_contrast computes (the keys
 * K[j], Eqs. 11-13) without a context and without allocating: it calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its working memory
 * (sorted events, row tables, per-tile partial sums, keys) is one static
 * device array of DD_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads
 * this library holds until the process exits.
 *
 *   W, H, foe_x, foe_y  frame and FOE, as dd_create.
 *   ev                  events in DEVICE memory (ev->device_ptrs must be 1),
 *                       at most DD_NOALLOC_MAX_EVENTS of them.
 *   D, nD               hypotheses (host array), as dd_contrast.
 *   K                   host array of nD keys (unspecified after an error).
 *   stream              cudaStream_t to run on (NULL: the legacy default
 *                       stream); the call synchronises it before returning.
 *
 * Set-up: the first call on each device (made with that device current)
 * looks up the device address of the static array and caches it; make that
 * first call before any stream capture on the device.  The cached address
 * belongs to the device's primary context: after cudaDeviceReset on that
 * device it is stale, so this entry point must not be called on that device
 * again in the same process.  The first call may also load this library's
 * device code (and with it the static array) if nothing else has yet; later
 * calls leave the device's free memory unchanged.
 * Sharing: every call on a device uses the same array and leaves the last
 * call's contents in it (everything that must start at zero is cleared by the
 * call itself).  Calls whose GPU work overlaps -- from several host threads
 * or on several streams at once -- race on the array; serialise them.
 * Errors: DD_ERR_CAPACITY if ev->n > DD_NOALLOC_MAX_EVENTS; DD_ERR_ARG in
 * every case dd_contrast rejects (the same descriptor and domain checks), or
 * if the events are not device pointers; DD_ERR_NO_DEVICE; DD_ERR_CUDA. */
#define DD_NOALLOC_MAX_EVENTS (1 << 20)
#define DD_NOALLOC_SCRATCH_BYTES 25224704
int dd_contrast_noalloc(int32_t W, int32_t H, float foe_x, float foe_y, const dd_events* ev, const float* D,
                        int32_t nD, dd_i128* K, void* stream);

/* Roofline denominators measured on the current device (no counterpart in
 * the paper): shared-memory atomic increments per second (with the returned
 * previous value, at random cells of a 41 KB array per block, every SM
 * busy) and bytes per second streamed from a 32 MiB buffer resident in L2.
 * Best of six launches each, timed with CUDA events on `stream` (NULL: the
 * legacy default stream).  Allocates 32 MiB for the duration of the call.
 * Errors: DD_ERR_ARG, DD_ERR_NO_DEVICE, DD_ERR_OOM, DD_ERR_CUDA. */
int dd_probe_peaks(double* shared_atomics_per_s, double* l2_read_bytes_per_s, void* stream);

/* A static description of a status code. */
const char* dd_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* DD_H */
