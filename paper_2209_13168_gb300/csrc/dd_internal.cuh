// Internal types and launch interface shared by the kernels (dd_kernels.cu)
// and the host code (dd_api.cu, dd_noalloc.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/dd.h"

struct dd_ctx;
struct dd_mlp;

namespace dd {

typedef __int128 i128;

// A named range over a host-side phase (ingest, rounds, read-back) for
// profilers that record NVTX; free when none is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// One event after ingest: its offsets from the FOE as the warp uses them
// (binary32 x - FOE_x and y - FOE_y) and its time since t0 (binary32
// t - t0); one 16-byte load.
struct __align__(16) Ev {
    float dx, dy, t;
    int32_t pad;
};

enum TaskKind : int32_t { TASK_POINT = 0, TASK_BOUND = 1 };

// One evaluation: the contrast at D_lo (TASK_POINT) or the bound over
// [D_lo, D_hi] (TASK_BOUND).  `splits` (>= 1) is how many blocks share each
// of its row bands, each taking its own rows of the band; it changes the
// schedule only, never the result.
struct Task {
    float D_lo, D_hi;
    int32_t kind, splits;
};

// One schedulable job: split `split` of `splits` of task `task` of window
// `win`; a job covers every row band of the frame.  A fused job (splits < 0)
// evaluates the three tasks of one expanded interval together: the contrast
// at its centre (task `task`) and the bounds of its two halves (tasks
// `split` and `split` + 1).
struct Job {
    int32_t win, task, split, splits;
};

// Sums of one task's IWE: per task, over all its row bands; counts per
// polarity plane (plane 1 stays zero without polarity).
struct Partial {
    unsigned long long S;         // sum of squared counts, both planes
    unsigned long long cells[2];  // sum of counts (N_in for a point, increments for a bound)
    unsigned long long full[2];   // events whose bound segment lies in the frame
};

// Eq. (13) / Eq. (14) in integer form, summed over the polarity planes:
// K = M S - sum_p N_p^2 with N = N_in for a point and N = N_full for a bound.
__host__ __device__ inline i128 partial_key(int64_t M, const Partial& q, bool point) {
    const unsigned long long a = point ? q.cells[0] : q.full[0], b = point ? q.cells[1] : q.full[1];
    return (i128)M * (i128)q.S - (i128)a * (i128)a - (i128)b * (i128)b;
}

struct __align__(16) Node {
    float lo, hi;
    int32_t pad0, pad1;
    i128 kb;
};

struct __align__(16) Popped {
    float lo, hi, c;
    int32_t leaf;
    i128 kb;
    int32_t t_point, t_left, t_right, pad;
};

struct __align__(16) TraceRec {
    float D_lo, D_hi, D_c;
    int32_t leaf;
    i128 Kbar, K_c;
};

enum Phase : int32_t { PH_INIT = 0, PH_RUN = 1, PH_DONE = 2 };

constexpr int MAX_POP = 64;
constexpr int MAX_TASKS = 3 * MAX_POP;   // tasks of one window in one round
constexpr int CHUNK = 8192;              // events per ingest block

// Device-resident state of one BnB search (Algorithm 1).
struct __align__(16) SolveState {
    // parameters
    i128 gamma_K;
    int64_t M, max_rounds;
    float D_lo, D_hi, tol, tau;
    int32_t K_pop, qcap, trace_cap, warm;
    // search state
    i128 K_hat, leaf_max, stop_kb;
    float D_hat;
    int32_t phase, status, n_tasks, n_pop, q_n, q_start, q_cur, have_leaf, have_stop;
    float D_warm, w_warm;                 // the warm start the search began from
    int32_t cancel, pad_c0, pad_c1, pad_c2;   // set between rounds: stop at the next control step
    int64_t nodes_expanded, point_evals, bound_evals, cells, bcells, rounds, max_queue, trace_len;
    Popped pop[MAX_POP];
};

// Search parameters of one window.  warm: 0 none, 1 from (D_warm, w_warm);
// the model warm start writes its guess here on the device and sets warm = 1.
struct __align__(16) WinParams {
    i128 gamma_K;
    float D_lo, D_hi, tol;
    int32_t warm;
    float D_warm, w_warm;
    int32_t pad0, pad1;
};

// Device view of a warm-start model: bfloat16 weights transposed to
// [in][out] (unit j of a layer reads column j), binary32 biases.
struct MlpDev {
    const uint16_t* w1t;    // [128][128]
    const uint16_t* w2t;    // [128][128]
    const uint16_t* w3t;    // [128][2]
    const float* b1;
    const float* b2;
    const float* b3;
};
constexpr int FEAT_R = 16, FEAT_T = 8, FEATURES = FEAT_R * FEAT_T, MLP_H = 128, MLP_OUT = 2;

// One window's input and where its sorted events go.
struct WinIn {
    const int16_t* x;
    const int16_t* y;
    const float* t;
    const int8_t* p;       // polarities (read only with two polarity planes)
    int64_t n, ev_off;     // event count; offset in the sorted event buffers
    float t0, tau;
    int32_t chunk0, pad;   // first ingest chunk of the window
};

// Round bookkeeping of one context, in device memory.  Job lists and unit
// counters are double-buffered by round parity: the evaluation of round r
// reads list r % 2 and clears the other list's counters; the control blocks
// of round r fill list (r + 1) % 2; the last control block to finish counts
// the windows still searching and advances the round.
struct Sched {
    int32_t round;
    int32_t n_jobs[2];
    int32_t work[2];
    int32_t ticket, active, running;
};

// Geometry of a context.  Events are sorted by (polarity plane, time
// bucket, row): n_tb buckets of equal length over [0, tau], planes * n_tb *
// H <= 4096 bins, n_tb <= 8.  A job's units are its row bands, plane 0's
// first: n_tiles = planes * plane_tiles.
struct Geom {
    int32_t W, H;
    float fx, fy;
    int32_t band_rows, n_tiles, n_tb, max_splits;
    int32_t split_target;   // resident evaluation blocks: a round's bounds split to fill one wave (0: never)
    int32_t ref0;           // 1: the warp maps events to the window's start (t_ref = 0), not its end
    int32_t planes;         // 1: polarity unused; 2: one image per polarity (p > 0, p <= 0)
    int32_t plane_tiles;    // row bands of one plane
    float fuse_cells;       // an expanded interval whose bound_cells - 1 is at most this runs as one
                            // fused job (0: never); a schedule choice only
};

// Bins of one window's event sort.
__host__ __device__ inline int32_t bins_of(const Geom& g) { return g.planes * g.n_tb * g.H; }

// The warp's reference time for a window of length tau.
__host__ __device__ inline float warp_tref(const Geom& g, float tau) { return g.ref0 ? 0.0f : tau; }

// Covered cells per event of a bound over [D_lo, D_hi], estimated from the
// scale change at t = 0, |g(D_hi) - g(D_lo)| with g = 1/(1 - D tau), times a
// typical offset from the FOE, (W + H)/4.  Bounds of at least DENSE_CELLS are
// dense (their tiles are summed in one pass) and are the ones worth
// splitting over several blocks.  A schedule estimate only (the threshold
// and the per-lane walk limit in bound_pass were set by measurement).
constexpr float DENSE_CELLS = 2.0f;
// Split bands of bounds below SPLIT_ROWS_CELLS are divided by rows, longer
// ones by events (see eval_unit).
constexpr float SPLIT_ROWS_CELLS = 64.0f;
__host__ __device__ inline float bound_cells(const Geom& g, float D_lo, float D_hi, float tau) {
#ifdef __CUDA_ARCH__
    // an estimate: fast reciprocals (deterministic, so every unit of a task agrees)
    const float gl = __fdividef(1.0f, 1.0f - D_lo * tau), gh = __fdividef(1.0f, 1.0f - D_hi * tau);
#else
    const float gl = 1.0f / (1.0f - D_lo * tau), gh = 1.0f / (1.0f - D_hi * tau);
#endif
    return 1.0f + (gh > gl ? gh - gl : gl - gh) * 0.25f * (float)(g.W + g.H);
}

// Splits of dense bound task `rank` (0-based among the window's nb dense
// bound tasks) in a round of `units` unsplit (task, row band) units of the
// window: when they do not fill the window's share of one wave of the
// resident evaluation grid (`target` blocks: split_target for a search alone,
// split_target / n for n searches sharing the rounds), the spare blocks go to
// the dense bound tasks as extra splits, spread evenly (an extra split of a
// task adds n_tiles units), so the round runs as one wave of shorter units;
// none once the round fills the share (other tasks never split: their units
// are short already).  A split holds at least one row of a band.  A window's
// jobs stay below its tasks + target / n_tiles.  A schedule choice only.
__host__ __device__ inline int32_t fill_splits(const Geom& g, int32_t target, int32_t units, int32_t nb,
                                               int32_t rank) {
    if (target <= 0 || nb <= 0 || units >= target) return 1;
    const int32_t extra = (target - units) / g.n_tiles;
    const int32_t s = 1 + extra / nb + (rank < extra % nb ? 1 : 0);
    const int32_t cap = g.max_splits < g.band_rows ? g.max_splits : g.band_rows;   // a split holds a row at least
    return s > cap ? cap : s;
}

// Room for one window's jobs in a round's list: its tasks plus the extra
// splits fill_splits can give it (at most split_target / n_tiles).
inline int32_t jobs_per_window(const Geom& g, int32_t max_tasks) {
    return max_tasks + (g.split_target > 0 ? g.split_target / g.n_tiles : 0) + 1;
}

// Row pitch of a shared-memory IWE tile: odd, so that the cells of one
// column in consecutive rows fall in different shared-memory banks.
__host__ __device__ inline int32_t tile_pitch(const Geom& g) { return g.W | 1; }

// Time buckets for a sort over H rows (rows of every plane): as many as fit
// 4096 bins, at most 8.
inline int32_t time_buckets(int32_t H) {
    int32_t b = 4096 / H;
    return b < 1 ? 1 : (b > 8 ? 8 : b);
}

// Merge buffers of event-split jobs (single-window searches only; without
// them every split of a band is a split by rows).
struct Merge {
    uint32_t* acc;                 // [task][planes * M] counts, zero between uses
    int32_t* done;                 // [task][tile] finished splits, zero between uses
    Partial* sums;                 // [task][tile] sums of the splits, zero between uses
};

// Everything a control step (Algorithm 1's bookkeeping for a round) reads or
// writes; one control block per window.
struct CtlArgs {
    int32_t n_windows;
    struct SolveState* st_all;
    struct Node* queues;
    Task* tasks_all;
    int32_t task_stride;
    Partial* part_all;
    const int32_t* err_all;
    struct TraceRec* trace;
    Job* jobs_all;
    int32_t job_stride;
    struct Sched* sch;
    cudaGraphConditionalHandle loop;
    int32_t use_loop, split_ok;
    int32_t* phase_out;
};

// Everything an evaluation launch reads or writes.
struct EvalArgs {
    const Ev* ev;
    const float2* rcp;
    const int32_t* row_off;        // per window: bins_of(g) + 1 entries
    const WinIn* wins;
    const Task* tasks;             // per window: task_stride entries
    int32_t task_stride;
    const Job* jobs;               // two lists of job_stride entries
    int32_t job_stride;
    Sched* sch;
    Partial* part;                 // [win * task_stride + task]: the task's sums over its row
                                   // bands, accumulated by atomics; zero before the evaluation,
                                   // cleared by their reader
    uint32_t* iwe_out;             // nullable: [task][planes * M] (single window)
    Merge mg;
};

// Kernel launches (dd_kernels.cu).  All asynchronous on `s`.
cudaError_t launch_ingest(const Geom& g, const WinIn* wins_dev, int32_t n_windows, const int32_t* chunk_win_dev,
                          int32_t n_chunks, Ev* out, float2* rcp, int32_t* row_count, int32_t* row_off,
                          int32_t* cursor, int32_t* err, cudaStream_t s);
cudaError_t launch_eval(const Geom& g, const EvalArgs& a, int threads, int grid_blocks, cudaStream_t s);
int eval_resident_blocks(const Geom& g, int threads);
cudaError_t launch_keys(const Geom& g, const Task* tasks, int32_t n_tasks, Partial* part, i128* key,
                        unsigned long long* S, unsigned long long* cells, unsigned long long* full,
                        cudaStream_t s);
// Windows w0 .. w0 + n_windows - 1 start a search; split_ok < 0: split bound
// tasks only when n_windows == 1.
cudaError_t launch_init(const Geom& g, int32_t n_windows, SolveState* st, Task* tasks, int32_t task_stride,
                        Partial* part, const WinIn* wins, const WinParams* params, Job* jobs, int32_t job_stride,
                        Sched* sch, int32_t K_pop, int32_t qcap, int64_t max_rounds, int32_t trace_cap,
                        cudaStream_t s, int32_t w0 = 0, int32_t split_ok = -1);
// One control block per window 0 .. n_windows - 1; phase_out (nullable)
// receives each window's phase after the round.
CtlArgs control_args(int32_t n_windows, SolveState* st, Node* queues, Task* tasks, int32_t task_stride, Partial* part,
                     const int32_t* err, TraceRec* trace, Job* jobs, int32_t job_stride, Sched* sch,
                     cudaGraphConditionalHandle loop, int32_t use_loop, int32_t split_ok, int32_t* phase_out);
cudaError_t launch_control(const Geom& g, int32_t n_windows, SolveState* st, Node* queues, Task* tasks,
                           int32_t task_stride, Partial* part, const int32_t* err, TraceRec* trace,
                           Job* jobs, int32_t job_stride, Sched* sch, cudaGraphConditionalHandle loop,
                           int32_t use_loop, cudaStream_t s, int32_t split_ok = -1, int32_t* phase_out = nullptr);

// Learned warm start (dd_mlp.cu).  Feature counts of windows 0..n_windows-1
// (counts [w][128], zeroed by the caller) from their sorted events; then,
// for every window whose params have warm == 2, the network's guess written
// into its params (warm = 1).
cudaError_t launch_features(const Geom& g, const WinIn* wins, const int32_t* chunk_win, int32_t n_chunks,
                            const Ev* ev, int32_t* counts, cudaStream_t s);
cudaError_t launch_warm(const Geom& g, int32_t n_windows, const int32_t* counts, const WinIn* wins,
                        WinParams* params, const MlpDev& m, cudaStream_t s);
bool mlp_device_view(const struct ::dd_mlp* m, MlpDev* out, int* device);
// feat[w][k] = 128 counts[w][k] / n_w (binary32), windows 0..n_windows-1.
cudaError_t launch_feature_norm(int32_t n_windows, const int32_t* counts, const WinIn* wins, float* feat,
                                cudaStream_t s);

// Fast mode (dd_fast.cu): n events scaled from W x H to W2 x H2, the kept
// share compacted in order into x2/y2/t2; counts [resample_blocks(n)],
// offsets [resample_blocks(n) + 1] (offsets[last] = kept count), err set on
// events outside the fine frame.
int32_t resample_blocks(int64_t n);
cudaError_t launch_resample(const int16_t* x, const int16_t* y, const float* t, int64_t n, int32_t W, int32_t H,
                            int32_t W2, int32_t H2, float keep, uint64_t seed, int16_t* x2, int16_t* y2, float* t2,
                            int32_t* counts, int64_t* offsets, int32_t* err, cudaStream_t s);

// Time span of n timestamps (dd_fast.cu): out = (least, greatest) finite t;
// part holds span_blocks(n) entries.
int32_t span_blocks(int64_t n);
cudaError_t launch_time_span(const float* t, int64_t n, float2* part, float2* out, cudaStream_t s);

// Windows of a time-sorted stream (dd_fast.cu): for k < n_windows, the
// events with (t - t0_k) in [0, tau], t0_k = (float)(t_start + k hop): the
// first index and the count of them, and t0_k.
cudaError_t launch_stream_bounds(const float* t, int64_t n, double t_start, double hop, float tau, int32_t n_windows,
                                 int64_t* first, int64_t* count, float* t0, cudaStream_t s);

// The checked-build error word of the evaluation kernels (dd_kernels.cu).
cudaError_t check_flags(uint32_t* flags, int32_t* checked, bool reset);

// Context accessors for the serving engine (dd_serve.cu).
void ctx_info(const struct ::dd_ctx* c, Geom* g, int32_t* threads, int32_t* eval_blocks, int32_t* max_tasks,
              int32_t* pop_k, int32_t* queue_capacity, int64_t* max_rounds);
const struct ::dd_mlp* ctx_warm_model(const struct ::dd_ctx* c);
cudaStream_t ctx_stream(const struct ::dd_ctx* c);
cudaError_t eval_smem_setup(const Geom& g);

// Host checks shared by the entry points (dd_api.cu): a window descriptor
// (DD_OK or DD_ERR_ARG; with two polarity planes the events must carry p),
// and a hypothesis in the domain -64 <= D tau <= 3/4.
int check_events(const ::dd_events* ev, int32_t planes);
bool d_ok(float D, float tau);

}  // namespace dd
