// C ABI of the exact divergence estimator (include/dd.h): context, argument
// checks, buffer management and the host side of the device BnB loop.
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using dd::i128;
using dd::check_events;
using dd::d_ok;

struct dd_ctx {
    int device = 0;
    dd::Geom g{};
    dd_config cfg{};
    int threads = 512;
    int max_tasks = 0;            // task slots per window
    int eval_blocks = 0;          // resident blocks of the evaluation grid
    cudaStream_t own = nullptr, stream = nullptr;

    // events: sorted and reciprocals for all windows of a call
    dd::Ev* ev = nullptr;
    float2* rcp = nullptr;
    int64_t ev_cap = 0;
    int16_t *in_x = nullptr, *in_y = nullptr;   // staging of host-array inputs
    float* in_t = nullptr;
    int8_t* in_p = nullptr;
    int64_t in_cap = 0;

    // per-window buffers, sized for win_cap windows
    int win_cap = 0;
    int32_t *row_count = nullptr, *row_off = nullptr, *cursor = nullptr, *err = nullptr;
    dd::WinIn* wins = nullptr;
    dd::WinParams* params = nullptr;
    dd::SolveState* st = nullptr;
    dd::Node* queues = nullptr;   // per window: two buffers of queue_capacity nodes
    dd::Task* tasks = nullptr;
    dd::Partial* part = nullptr;
    dd::Job* jobs = nullptr;      // two lists of job_stride jobs
    int job_stride = 0;
    int32_t* chunk_win = nullptr;
    int64_t chunk_cap = 0;
    int32_t n_chunks = 0;         // ingest chunks of the last call

    // fast mode scratch
    int32_t* rs_counts = nullptr;
    int64_t* rs_offsets = nullptr;
    int32_t* rs_err = nullptr;
    int64_t rs_cap = 0;

    // learned warm start
    dd_mlp* warm_model = nullptr;
    int32_t* feat_counts = nullptr;   // [window][128]
    int feat_cap = 0;
    dd::Sched* sch = nullptr;

    // single-window extras
    uint32_t* macc = nullptr;     // merge buffers of split jobs (zero between uses)
    int32_t* mdone = nullptr;
    dd::Partial* msums = nullptr;
    i128* keys = nullptr;
    unsigned long long *S = nullptr, *C = nullptr, *F = nullptr;
    uint32_t* iwe = nullptr;
    size_t iwe_cap = 0;
    dd::TraceRec* trace = nullptr;
    int64_t trace_cap = 0;

    // the rounds of a solve as one CUDA graph (a conditional while loop)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int g_nw = 0;
    const void* g_key[3] = {nullptr, nullptr, nullptr};

    // telemetry (dd_stats) and optional per-launch timing of the IWE kernel
    dd_stats stats{};
    int timing = 0;
    std::vector<cudaEvent_t> t_ev;
    size_t t_used = 0;
    std::vector<float> t_ms;      // durations of the timed launches since the last reset

    // pinned host staging
    dd::SolveState* h_st = nullptr;
    dd::Task* h_tasks = nullptr;
    dd::Job* h_jobs = nullptr;
    dd::Sched* h_sch = nullptr;
    dd::WinIn* h_wins = nullptr;
    dd::WinParams* h_params = nullptr;
    int32_t* h_chunks = nullptr;
    int32_t* h_err = nullptr;
};

namespace {

#define DD_TRY(expr)                                   \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

int cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return DD_ERR_OOM;
    return DD_ERR_CUDA;
}

template <class T>
void release(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}
template <class T>
void release_host(T*& p) {
    if (p) cudaFreeHost(p);
    p = nullptr;
}

cudaError_t copy(dd_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    if (kind == cudaMemcpyHostToDevice) c->stats.h2d_bytes += (int64_t)bytes;
    if (kind == cudaMemcpyDeviceToHost) c->stats.d2h_bytes += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
}

cudaError_t sync(dd_ctx* c) {
    c->stats.host_syncs++;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && c->t_used) {        // fold the timed launches into eval_ms
        for (size_t i = 0; i + 1 < c->t_used; i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, c->t_ev[i], c->t_ev[i + 1]) == cudaSuccess) c->stats.eval_ms += ms;
            c->stats.timed_launches++;
            if (c->t_ms.size() < DD_MAX_LAUNCH_TIMES) c->t_ms.push_back(ms);
        }
        c->t_used = 0;
    }
    return e;
}

cudaError_t record(dd_ctx* c) {
    if (c->t_used == c->t_ev.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->t_ev.push_back(e);
    }
    return cudaEventRecord(c->t_ev[c->t_used++], c->stream);
}

void drop_graph(dd_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->g_nw = 0;
}

dd::EvalArgs eval_args(dd_ctx* c, uint32_t* iwe_out, bool single) {
    dd::EvalArgs a{};
    a.ev = c->ev;
    a.rcp = c->rcp;
    a.row_off = c->row_off;
    a.wins = c->wins;
    a.tasks = c->tasks;
    a.task_stride = c->max_tasks;
    a.jobs = c->jobs;
    a.job_stride = c->job_stride;
    a.sch = c->sch;
    a.part = c->part;
    a.iwe_out = iwe_out;
    a.mg.acc = single ? c->macc : nullptr;
    a.mg.done = single ? c->mdone : nullptr;
    a.mg.sums = single ? c->msums : nullptr;
    return a;
}

cudaError_t eval(dd_ctx* c, uint32_t* iwe, bool single) {
    if (c->timing) {
        cudaError_t e = record(c);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = dd::launch_eval(c->g, eval_args(c, iwe, single), c->threads, c->eval_blocks, c->stream);
    if (e != cudaSuccess) return e;
    c->stats.kernel_launches++;
    c->stats.eval_launches++;
    if (c->timing) return record(c);
    return cudaSuccess;
}

// Per-window buffers for at least nw windows.
int ensure_windows(dd_ctx* c, int nw) {
    if (nw <= c->win_cap) return DD_OK;
    drop_graph(c);
    const int cap = nw < 8 ? 8 : nw + nw / 2;
    const int bins = dd::bins_of(c->g);
    release(c->row_count);
    release(c->row_off);
    release(c->cursor);
    release(c->err);
    release(c->wins);
    release(c->params);
    release(c->st);
    release(c->queues);
    release(c->tasks);
    release(c->part);
    release(c->jobs);
    release_host(c->h_st);
    release_host(c->h_wins);
    release_host(c->h_params);
    release_host(c->h_err);
    c->win_cap = 0;
    const int jw = cap * dd::jobs_per_window(c->g, c->max_tasks);
    const int js = jw > c->max_tasks * c->g.max_splits ? jw : c->max_tasks * c->g.max_splits;
    int rc = DD_OK;
    auto A = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    auto AH = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMallocHost(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    A((void**)&c->row_count, sizeof(int32_t) * (size_t)bins * cap);
    A((void**)&c->row_off, sizeof(int32_t) * (size_t)(bins + 1) * cap);
    A((void**)&c->cursor, sizeof(int32_t) * (size_t)bins * cap);
    A((void**)&c->err, sizeof(int32_t) * (size_t)cap);
    A((void**)&c->wins, sizeof(dd::WinIn) * (size_t)cap);
    A((void**)&c->params, sizeof(dd::WinParams) * (size_t)cap);
    A((void**)&c->st, sizeof(dd::SolveState) * (size_t)cap);
    A((void**)&c->queues, sizeof(dd::Node) * 2 * (size_t)c->cfg.queue_capacity * cap);
    A((void**)&c->tasks, sizeof(dd::Task) * (size_t)c->max_tasks * cap);
    A((void**)&c->part, sizeof(dd::Partial) * (size_t)c->max_tasks * cap);
    A((void**)&c->jobs, sizeof(dd::Job) * 2 * (size_t)js);
    AH((void**)&c->h_st, sizeof(dd::SolveState) * (size_t)cap);
    AH((void**)&c->h_wins, sizeof(dd::WinIn) * (size_t)cap);
    AH((void**)&c->h_params, sizeof(dd::WinParams) * (size_t)cap);
    AH((void**)&c->h_err, sizeof(int32_t) * (size_t)cap);
    if (rc) return rc;
    c->job_stride = js;
    c->win_cap = cap;
    return DD_OK;
}

// Staging buffers for n host-array events (with polarities when the context
// has two planes).
int ensure_staging(dd_ctx* c, int64_t n) {
    if (n <= c->in_cap) return DD_OK;
    release(c->in_x);
    release(c->in_y);
    release(c->in_t);
    release(c->in_p);
    c->in_cap = 0;
    const int64_t nc = n + n / 4;
    DD_TRY(cudaMalloc((void**)&c->in_x, sizeof(int16_t) * nc));
    DD_TRY(cudaMalloc((void**)&c->in_y, sizeof(int16_t) * nc));
    DD_TRY(cudaMalloc((void**)&c->in_t, sizeof(float) * nc));
    if (c->g.planes > 1) DD_TRY(cudaMalloc((void**)&c->in_p, sizeof(int8_t) * nc));
    c->in_cap = nc;
    return DD_OK;
}

// Upload (host arrays) or alias (device arrays) the events of nw windows,
// then sort each window's events by (time bucket, row).  Sets err[w] on
// malformed events of window w.
int ingest(dd_ctx* c, const dd_events* evs, int nw) {
    dd::NvtxRange range("dd ingest");
    int rc = ensure_windows(c, nw);
    if (rc) return rc;
    int64_t total = 0, host_total = 0, chunks = 0;
    for (int w = 0; w < nw; w++) {
        total += evs[w].n;
        if (!evs[w].device_ptrs) host_total += evs[w].n;
        chunks += (evs[w].n + dd::CHUNK - 1) / dd::CHUNK;
    }
    if (total > c->ev_cap) {
        drop_graph(c);
        release(c->ev);
        release(c->rcp);
        c->ev_cap = 0;
        const int64_t nc = total < 1024 ? 1024 : total + total / 4;
        DD_TRY(cudaMalloc((void**)&c->ev, sizeof(dd::Ev) * nc));
        DD_TRY(cudaMalloc((void**)&c->rcp, sizeof(float2) * nc));
        c->ev_cap = nc;
    }
    rc = ensure_staging(c, host_total);
    if (rc) return rc;
    if (chunks > c->chunk_cap) {
        release(c->chunk_win);
        release_host(c->h_chunks);
        c->chunk_cap = 0;
        const int64_t nc = chunks < 256 ? 256 : chunks + chunks / 2;
        DD_TRY(cudaMalloc((void**)&c->chunk_win, sizeof(int32_t) * nc));
        DD_TRY(cudaMallocHost((void**)&c->h_chunks, sizeof(int32_t) * nc));
        c->chunk_cap = nc;
    }
    int64_t off = 0, hoff = 0;
    int32_t ch = 0;
    for (int w = 0; w < nw; w++) {
        const dd_events& e = evs[w];
        dd::WinIn& wi = c->h_wins[w];
        wi.x = e.x;
        wi.y = e.y;
        wi.t = e.t;
        wi.p = c->g.planes > 1 ? e.p : nullptr;
        if (!e.device_ptrs && e.n > 0) {
            DD_TRY(copy(c, c->in_x + hoff, e.x, sizeof(int16_t) * e.n, cudaMemcpyHostToDevice));
            DD_TRY(copy(c, c->in_y + hoff, e.y, sizeof(int16_t) * e.n, cudaMemcpyHostToDevice));
            DD_TRY(copy(c, c->in_t + hoff, e.t, sizeof(float) * e.n, cudaMemcpyHostToDevice));
            wi.x = c->in_x + hoff;
            wi.y = c->in_y + hoff;
            wi.t = c->in_t + hoff;
            if (c->g.planes > 1) {
                DD_TRY(copy(c, c->in_p + hoff, e.p, sizeof(int8_t) * e.n, cudaMemcpyHostToDevice));
                wi.p = c->in_p + hoff;
            }
            hoff += e.n;
        }
        wi.n = e.n;
        wi.ev_off = off;
        wi.t0 = e.t0;
        wi.tau = e.tau;
        wi.chunk0 = ch;
        wi.pad = 0;
        const int32_t nch = (int32_t)((e.n + dd::CHUNK - 1) / dd::CHUNK);
        for (int32_t k = 0; k < nch; k++) c->h_chunks[ch + k] = w;
        ch += nch;
        off += e.n;
    }
    DD_TRY(copy(c, c->wins, c->h_wins, sizeof(dd::WinIn) * nw, cudaMemcpyHostToDevice));
    if (ch) DD_TRY(copy(c, c->chunk_win, c->h_chunks, sizeof(int32_t) * ch, cudaMemcpyHostToDevice));
    c->n_chunks = ch;
    DD_TRY(dd::launch_ingest(c->g, c->wins, nw, c->chunk_win, ch, c->ev, c->rcp, c->row_count, c->row_off,
                             c->cursor, c->err, c->stream));
    c->stats.kernel_launches += ch ? 3 : 1;
    return DD_OK;
}

dd_i128 from_i128(i128 v) {
    dd_i128 r;
    r.lo = (uint64_t)(unsigned __int128)v;
    r.hi = (int64_t)(uint64_t)((unsigned __int128)v >> 64);
    return r;
}

// Evaluate n tasks (point or bound) of one window and copy keys, sums and
// images to the host.
int eval_tasks(dd_ctx* c, const dd_events* ev, int32_t n, int kind, const float* A, const float* B, dd_i128* K,
               uint64_t* S, int64_t* N, uint32_t* iwe) {
    const int64_t M = (int64_t)c->g.planes * c->g.W * c->g.H;     // image cells of one task
    dd::NvtxRange range(kind == dd::TASK_POINT ? "dd contrast" : "dd bound");
    for (int32_t j0 = 0; j0 < n; j0 += c->max_tasks) {
        const int32_t m = n - j0 < c->max_tasks ? n - j0 : c->max_tasks;
        int32_t nj = 0;
        int32_t n_dense = 0, rank = 0;
        for (int32_t j = 0; j < m; j++)
            n_dense += kind == dd::TASK_BOUND && dd::bound_cells(c->g, A[j0 + j], B[j0 + j], ev->tau) >= dd::DENSE_CELLS;
        for (int32_t j = 0; j < m; j++) {
            dd::Task& t = c->h_tasks[j];
            t.D_lo = A[j0 + j];
            t.D_hi = B[j0 + j];
            t.kind = kind;
            const bool dense = kind == dd::TASK_BOUND && dd::bound_cells(c->g, t.D_lo, t.D_hi, ev->tau) >= dd::DENSE_CELLS;
            t.splits = dense ? dd::fill_splits(c->g, c->g.split_target, m * c->g.n_tiles, n_dense, rank++) : 1;
        }
        for (int32_t j = m - 1; j >= 0; j--)              // heavier tasks first
            for (int32_t s = 0; s < c->h_tasks[j].splits; s++) {
                dd::Job& jb = c->h_jobs[nj++];
                jb.win = 0;
                jb.task = j;
                jb.split = s;
                jb.splits = c->h_tasks[j].splits;
            }
        std::memset(c->h_sch, 0, sizeof(dd::Sched));
        c->h_sch->n_jobs[0] = nj;
        DD_TRY(copy(c, c->tasks, c->h_tasks, sizeof(dd::Task) * m, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->jobs, c->h_jobs, sizeof(dd::Job) * nj, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->sch, c->h_sch, sizeof(dd::Sched), cudaMemcpyHostToDevice));
        DD_TRY(cudaMemsetAsync(c->part, 0, sizeof(dd::Partial) * m, c->stream));   // the tasks' sums start at zero
        uint32_t* iw = nullptr;
        if (iwe) {
            size_t need = (size_t)m * M;
            if (need > c->iwe_cap) {
                release(c->iwe);
                c->iwe_cap = 0;
                DD_TRY(cudaMalloc((void**)&c->iwe, need * sizeof(uint32_t)));
                c->iwe_cap = need;
            }
            iw = c->iwe;
        }
        DD_TRY(eval(c, iw, true));
        DD_TRY(dd::launch_keys(c->g, c->tasks, m, c->part, c->keys, c->S, c->C, c->F, c->stream));
        c->stats.kernel_launches++;
        std::vector<i128> hk(m);
        std::vector<unsigned long long> hs(m), hc(m), hf(m);
        DD_TRY(copy(c, hk.data(), c->keys, sizeof(i128) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hs.data(), c->S, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hc.data(), c->C, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hf.data(), c->F, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (iwe)
            DD_TRY(copy(c, iwe + (size_t)j0 * M, c->iwe, sizeof(uint32_t) * (size_t)m * M, cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        if (c->h_err[0]) return DD_ERR_ARG;
        for (int32_t j = 0; j < m; j++) {
            K[j0 + j] = from_i128(hk[j]);
            if (S) S[j0 + j] = hs[j];
            if (N) N[j0 + j] = (int64_t)(kind == dd::TASK_POINT ? hc[j] : hf[j]);
        }
    }
    return DD_OK;
}

// Build the solve graph for nw windows: a while node whose body is one round
// (IWE evaluation, then one control block per window; the last control block
// clears the loop condition when no window is still searching).  Kernel
// arguments are baked in, so the graph is rebuilt when a buffer it points to
// is reallocated or the window count changes.
int build_graph(dd_ctx* c, int nw, dd::TraceRec* trace) {
    drop_graph(c);
    DD_TRY(cudaGraphCreate(&c->graph, 0));
    cudaGraphConditionalHandle h;
    DD_TRY(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    DD_TRY(cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    DD_TRY(cudaStreamBeginCaptureToGraph(c->own, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = dd::launch_eval(c->g, eval_args(c, nullptr, nw == 1), c->threads, c->eval_blocks, c->own);
    cudaError_t e2 = dd::launch_control(c->g, nw, c->st, c->queues, c->tasks, c->max_tasks, c->part, c->err, trace,
                                        c->jobs, c->job_stride, c->sch, h, 1, c->own);
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(c->own, &captured);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        drop_graph(c);
        return DD_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&c->gexec, c->graph, 0) != cudaSuccess) {
        drop_graph(c);
        return DD_ERR_CUDA;
    }
    c->g_nw = nw;
    c->g_key[0] = c->ev;
    c->g_key[1] = trace;
    c->g_key[2] = c->st;
    return DD_OK;
}

void fill_result(const dd::SolveState& s, const dd_events& ev, int64_t M, dd_result* out) {
    // Sec. 4.1 retrieval and reporting (double precision, from the exact keys).
    dd_result r;
    std::memset(&r, 0, sizeof(r));
    r.D_star = s.D_hat;
    r.D_end = (float)((double)s.D_hat / (1.0 - (double)s.D_hat * (double)ev.tau));
    r.K_hat = from_i128(s.K_hat);
    r.gap_K = from_i128(s.stop_kb);
    r.contrast = (double)s.K_hat / ((double)M * (double)M);
    r.bound_gap = (double)s.stop_kb / ((double)M * (double)M);
    r.nodes_expanded = s.nodes_expanded;
    r.point_evals = s.point_evals;
    r.bound_evals = s.bound_evals;
    r.event_warps = ev.n * (s.point_evals + s.bound_evals);
    r.cell_increments = s.cells;
    r.bound_increments = s.bcells;
    r.rounds = s.rounds;
    r.max_queue = s.max_queue;
    r.status = s.status;
    r.D_warm = s.D_warm;
    r.w_warm = s.w_warm;
    *out = r;
}

// Feature counts of the nw windows just ingested, into c->feat_counts.
int feature_counts(dd_ctx* c, int nw) {
    if (nw > c->feat_cap) {
        release(c->feat_counts);
    release(c->rs_counts);
    release(c->rs_offsets);
    release(c->rs_err);
        c->feat_cap = 0;
        DD_TRY(cudaMalloc((void**)&c->feat_counts, sizeof(int32_t) * dd::FEATURES * (size_t)nw));
        c->feat_cap = nw;
    }
    DD_TRY(cudaMemsetAsync(c->feat_counts, 0, sizeof(int32_t) * dd::FEATURES * (size_t)nw, c->stream));
    DD_TRY(dd::launch_features(c->g, c->wins, c->chunk_win, c->n_chunks, c->ev, c->feat_counts, c->stream));
    c->stats.kernel_launches += c->n_chunks ? 1 : 0;
    return DD_OK;
}

// Checks of one window's search parameters (warm start included).
int check_params(const dd_ctx* c, const dd_window_params& p, float tau) {
    if (!d_ok(p.D_lo, tau) || !d_ok(p.D_hi, tau) || !(p.D_lo < p.D_hi)) return DD_ERR_ARG;
    if (!std::isfinite(p.tol_D) || !(p.tol_D >= 0.0f) || !std::isfinite(p.gamma) || !(p.gamma >= 0.0))
        return DD_ERR_ARG;
    if (p.warm == DD_WARM_GIVEN)
        return std::isfinite(p.D_warm) && std::isfinite(p.w_warm) && p.w_warm > 0.0f ? DD_OK : DD_ERR_ARG;
    if (p.warm == DD_WARM_MODEL) return c->warm_model ? DD_OK : DD_ERR_ARG;
    return p.warm == DD_WARM_NONE ? DD_OK : DD_ERR_ARG;
}

int solve_impl(dd_ctx* c, const dd_events* evs, int nw, const dd_window_params* prm, dd_result* out,
               dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    if (!c || !out || !evs || !prm || nw < 1) return DD_ERR_ARG;
    for (int w = 0; w < nw; w++) {
        int rc = check_events(&evs[w], c->g.planes);
        if (rc) return rc;
        rc = check_params(c, prm[w], evs[w].tau);
        if (rc) return rc;
    }
    if (trace_cap < 0 || (trace_cap > 0 && (!trace || nw != 1))) return DD_ERR_ARG;
    dd::NvtxRange range(nw == 1 ? "dd solve" : "dd solve batch");
    if (trace_cap > c->trace_cap) {
        release(c->trace);
        c->trace_cap = 0;
        DD_TRY(cudaMalloc((void**)&c->trace, sizeof(dd::TraceRec) * trace_cap));
        c->trace_cap = trace_cap;
    }
    int rc = ingest(c, evs, nw);
    if (rc) return rc;
    const int64_t M = (int64_t)c->g.W * c->g.H;
    bool model = false;
    for (int w = 0; w < nw; w++) {
        dd::WinParams& q = c->h_params[w];
        q.gamma_K = (i128)std::floor(prm[w].gamma * (double)M * (double)M);
        q.D_lo = prm[w].D_lo;
        q.D_hi = prm[w].D_hi;
        q.tol = prm[w].tol_D;
        q.warm = prm[w].warm;
        q.D_warm = prm[w].warm == DD_WARM_GIVEN ? prm[w].D_warm : 0.0f;
        q.w_warm = prm[w].warm == DD_WARM_GIVEN ? prm[w].w_warm : 0.0f;
        q.pad0 = q.pad1 = 0;
        model |= prm[w].warm == DD_WARM_MODEL;
    }
    DD_TRY(copy(c, c->params, c->h_params, sizeof(dd::WinParams) * nw, cudaMemcpyHostToDevice));
    if (model) {                                  // the model's guesses, on the device
        dd::MlpDev m;
        int dev = -1;
        if (!dd::mlp_device_view(c->warm_model, &m, &dev) || dev != c->device) return DD_ERR_ARG;
        rc = feature_counts(c, nw);
        if (rc) return rc;
        DD_TRY(dd::launch_warm(c->g, nw, c->feat_counts, c->wins, c->params, m, c->stream));
        c->stats.kernel_launches++;
    }
    DD_TRY(cudaMemsetAsync(c->sch, 0, sizeof(dd::Sched), c->stream));
    DD_TRY(dd::launch_init(c->g, nw, c->st, c->tasks, c->max_tasks, c->part, c->wins, c->params, c->jobs,
                           c->job_stride, c->sch, c->cfg.pop_k, c->cfg.queue_capacity, c->cfg.max_rounds,
                           (int32_t)trace_cap, c->stream));
    c->stats.kernel_launches++;
    dd::TraceRec* tr_dev = trace_cap > 0 ? c->trace : nullptr;
    const bool graph = !c->cfg.host_loop && !c->timing;
    dd::NvtxRange rounds("dd rounds");
    if (graph) {
        // One graph launch runs every round on the device.
        if (!c->gexec || c->g_nw != nw || c->g_key[0] != (const void*)c->ev || c->g_key[1] != (const void*)tr_dev ||
            c->g_key[2] != (const void*)c->st) {
            rc = build_graph(c, nw, tr_dev);
            if (rc) return rc;
        }
        DD_TRY(cudaGraphLaunch(c->gexec, c->stream));
    } else {
        // Host-driven rounds: launch batches, poll for the end.  With timing
        // on, one round per poll, so that every timed launch has work.
        int batch = c->timing ? 1 : 2;
        for (;;) {
            for (int b = 0; b < batch; b++) {
                DD_TRY(eval(c, nullptr, nw == 1));
                DD_TRY(dd::launch_control(c->g, nw, c->st, c->queues, c->tasks, c->max_tasks, c->part, c->err,
                                          tr_dev, c->jobs, c->job_stride, c->sch, 0, 0, c->stream));
                c->stats.kernel_launches++;
            }
            DD_TRY(copy(c, c->h_sch, c->sch, sizeof(dd::Sched), cudaMemcpyDeviceToHost));
            DD_TRY(sync(c));
            if (c->h_sch->running == 0) break;
            if (batch < 64 && !c->timing) batch *= 2;
        }
    }
    DD_TRY(copy(c, c->h_st, c->st, sizeof(dd::SolveState) * nw, cudaMemcpyDeviceToHost));
    DD_TRY(copy(c, c->h_sch, c->sch, sizeof(dd::Sched), cudaMemcpyDeviceToHost));
    std::vector<dd::TraceRec> tr((size_t)trace_cap);
    if (trace_cap > 0) DD_TRY(copy(c, tr.data(), c->trace, sizeof(dd::TraceRec) * trace_cap, cudaMemcpyDeviceToHost));
    DD_TRY(sync(c));
    if (graph) {                                  // every round ran one evaluation and one control launch
        c->stats.kernel_launches += 2 * (int64_t)c->h_sch->round;
        c->stats.eval_launches += c->h_sch->round;
    }
    int status = DD_OK;
    for (int w = 0; w < nw; w++)
        if (c->h_st[w].status != DD_OK && status == DD_OK) status = c->h_st[w].status;
    if (nw == 1 && status != DD_OK) return status;
    for (int w = 0; w < nw; w++) fill_result(c->h_st[w], evs[w], M, &out[w]);
    if (trace_len) *trace_len = c->h_st[0].trace_len;
    for (int64_t i = 0; i < trace_cap && i < c->h_st[0].trace_len; i++) {
        trace[i].D_lo = tr[i].D_lo;
        trace[i].D_hi = tr[i].D_hi;
        trace[i].D_c = tr[i].D_c;
        trace[i].leaf = tr[i].leaf;
        trace[i].Kbar = from_i128(tr[i].Kbar);
        trace[i].K_c = from_i128(tr[i].K_c);
    }
    return status;
}

}  // namespace

namespace dd {
bool d_ok(float D, float tau) {
    if (!std::isfinite(D)) return false;
    double dt = (double)D * (double)tau;
    return dt <= 0.75 && dt >= -64.0;
}

// Host checks of a window descriptor.  Event contents (coordinates in the
// frame, times in the window) are checked by the ingest kernels, which flag
// the window; the call then fails with DD_ERR_ARG.
// With two polarity planes the events must carry their polarities.
int check_events(const ::dd_events* ev, int32_t planes) {
    if (!ev || ev->n < 0 || ev->n > INT32_MAX / 2) return DD_ERR_ARG;
    if (!std::isfinite(ev->tau) || !(ev->tau > 0.0f) || !std::isfinite(ev->t0)) return DD_ERR_ARG;
    if (ev->n > 0 && (!ev->x || !ev->y || !ev->t)) return DD_ERR_ARG;
    if (planes > 1 && ev->n > 0 && !ev->p) return DD_ERR_ARG;
    return DD_OK;
}

void ctx_info(const ::dd_ctx* c, Geom* g, int32_t* threads, int32_t* eval_blocks, int32_t* max_tasks, int32_t* pop_k,
              int32_t* queue_capacity, int64_t* max_rounds) {
    *g = c->g;
    *threads = c->threads;
    *eval_blocks = c->eval_blocks;
    *max_tasks = c->max_tasks;
    *pop_k = c->cfg.pop_k;
    *queue_capacity = c->cfg.queue_capacity;
    *max_rounds = c->cfg.max_rounds;
}
cudaStream_t ctx_stream(const ::dd_ctx* c) { return c->stream; }
const ::dd_mlp* ctx_warm_model(const ::dd_ctx* c) { return c->warm_model; }
}  // namespace dd

extern "C" {

const char* dd_strerror(int status) {
    switch (status) {
        case DD_OK: return "ok";
        case DD_ERR_ARG: return "invalid argument or malformed events";
        case DD_ERR_OOM: return "out of memory";
        case DD_ERR_QUEUE_OVERFLOW: return "branch-and-bound queue overflow";
        case DD_ERR_TIMEOUT: return "branch-and-bound round limit reached";
        case DD_ERR_CUDA: return "CUDA runtime error";
        case DD_ERR_NO_DEVICE: return "no sm_103 CUDA device";
        case DD_ERR_CAPACITY: return "input exceeds a fixed capacity (allocation-free scratch or serving slot)";
        case DD_ERR_CANCELLED: return "request cancelled";
        default: return "unknown status";
    }
}

void dd_destroy(dd_ctx* c) {
    if (!c) return;
    drop_graph(c);
    release(c->ev);
    release(c->rcp);
    release(c->in_x);
    release(c->in_y);
    release(c->in_t);
    release(c->in_p);
    release(c->row_count);
    release(c->row_off);
    release(c->cursor);
    release(c->err);
    release(c->wins);
    release(c->params);
    release(c->st);
    release(c->queues);
    release(c->tasks);
    release(c->part);
    release(c->jobs);
    release(c->chunk_win);
    release(c->sch);
    release(c->macc);
    release(c->mdone);
    release(c->msums);
    release(c->keys);
    release(c->S);
    release(c->C);
    release(c->F);
    release(c->iwe);
    release(c->trace);
    release(c->feat_counts);
    release_host(c->h_st);
    release_host(c->h_tasks);
    release_host(c->h_jobs);
    release_host(c->h_sch);
    release_host(c->h_wins);
    release_host(c->h_params);
    release_host(c->h_chunks);
    release_host(c->h_err);
    for (cudaEvent_t e : c->t_ev) cudaEventDestroy(e);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

int dd_create(int32_t W, int32_t H, float foe_x, float foe_y, const dd_config* cfg, dd_ctx** out) {
    if (!out || W < 1 || H < 1 || W > 4096 || H > 4096) return DD_ERR_ARG;
    if (!std::isfinite(foe_x) || !std::isfinite(foe_y) || foe_x < 0.0f || foe_y < 0.0f || foe_x > (float)W ||
        foe_y > (float)H)
        return DD_ERR_ARG;
    dd_config k{};
    if (cfg) k = *cfg;
    if (k.pop_k < 0 || k.pop_k > dd::MAX_POP || k.queue_capacity < 0 || k.band_rows < 0 || k.threads < 0 ||
        k.max_rounds < 0)
        return DD_ERR_ARG;
    if (k.threads && (k.threads % 32 || k.threads > 512)) return DD_ERR_ARG;
    if (k.max_splits < 0 || k.max_splits > 64 || k.host_loop < 0) return DD_ERR_ARG;
    if (k.warp_to_start != 0 && k.warp_to_start != 1) return DD_ERR_ARG;
    if (k.polarity != 0 && k.polarity != 1) return DD_ERR_ARG;
    if (k.polarity && H > 2048) return DD_ERR_ARG;          // the event sort has 4096 bins
    if (!k.pop_k) k.pop_k = 1;
    if (!k.queue_capacity) k.queue_capacity = 8192;
    if (!k.max_rounds) k.max_rounds = 1 << 20;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DD_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return DD_ERR_NO_DEVICE;

    dd_ctx* c = new (std::nothrow) dd_ctx();
    if (!c) return DD_ERR_OOM;
    c->device = dev;
    c->cfg = k;
    c->threads = k.threads ? k.threads : 512;
    c->g.W = W;
    c->g.H = H;
    c->g.fx = foe_x;
    c->g.fy = foe_y;
    // Default band: about 40 KB of uint32 counts (16 rows at 640 px), so
    // that heavy tasks spread over many blocks and several blocks share an SM.
    int rows = k.band_rows ? k.band_rows : (int)(40 * 1024 / (4 * W));
    if (rows < 1) rows = 1;
    if (rows > H) rows = H;
    if ((size_t)rows * (W | 1) * 4 > 200 * 1024) rows = (int)(200 * 1024 / (4 * (W | 1)));
    if (rows < 1) {
        delete c;
        return DD_ERR_ARG;
    }
    c->g.band_rows = rows;
    c->g.planes = k.polarity ? 2 : 1;
    c->g.plane_tiles = (H + rows - 1) / rows;
    c->g.n_tiles = c->g.planes * c->g.plane_tiles;
    c->g.n_tb = dd::time_buckets(c->g.planes * H);
    c->g.max_splits = k.max_splits ? k.max_splits : 16;
    c->g.ref0 = k.warp_to_start ? 1 : 0;
    if (!k.fuse_span) k.fuse_span = 25;
    c->g.fuse_cells = k.fuse_span > 0 ? 0.01f * (float)k.fuse_span : 0.0f;
    c->cfg.fuse_span = k.fuse_span;
    c->max_tasks = 3 * k.pop_k > 64 ? 3 * k.pop_k : 64;
    c->cfg.threads = c->threads;
    c->cfg.band_rows = rows;
    c->cfg.max_splits = c->g.max_splits;

    int rc = DD_OK;
    auto A = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    const size_t M = (size_t)c->g.planes * W * H;      // image cells of one task
    A((void**)&c->sch, sizeof(dd::Sched));
    A((void**)&c->macc, sizeof(uint32_t) * (size_t)c->max_tasks * M);
    A((void**)&c->mdone, sizeof(int32_t) * (size_t)c->max_tasks * c->g.n_tiles);
    A((void**)&c->msums, sizeof(dd::Partial) * (size_t)c->max_tasks * c->g.n_tiles);
    if (rc == DD_OK && (cudaMemset(c->macc, 0, sizeof(uint32_t) * (size_t)c->max_tasks * M) != cudaSuccess ||
                        cudaMemset(c->mdone, 0, sizeof(int32_t) * (size_t)c->max_tasks * c->g.n_tiles) != cudaSuccess ||
                        cudaMemset(c->msums, 0, sizeof(dd::Partial) * (size_t)c->max_tasks * c->g.n_tiles) !=
                            cudaSuccess))
        rc = DD_ERR_CUDA;
    A((void**)&c->keys, sizeof(i128) * c->max_tasks);
    A((void**)&c->S, sizeof(unsigned long long) * c->max_tasks);
    A((void**)&c->C, sizeof(unsigned long long) * c->max_tasks);
    A((void**)&c->F, sizeof(unsigned long long) * c->max_tasks);
    if (rc == DD_OK && cudaMallocHost((void**)&c->h_tasks, sizeof(dd::Task) * c->max_tasks) != cudaSuccess)
        rc = DD_ERR_OOM;
    if (rc == DD_OK &&
        cudaMallocHost((void**)&c->h_jobs, sizeof(dd::Job) * (size_t)c->max_tasks * c->g.max_splits) != cudaSuccess)
        rc = DD_ERR_OOM;
    if (rc == DD_OK && cudaMallocHost((void**)&c->h_sch, sizeof(dd::Sched)) != cudaSuccess) rc = DD_ERR_OOM;
    if (rc == DD_OK && cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK && dd::eval_smem_setup(c->g) != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK && (c->eval_blocks = dd::eval_resident_blocks(c->g, c->threads)) <= 0) rc = DD_ERR_CUDA;
    c->g.split_target = c->eval_blocks;
    if (rc == DD_OK) rc = ensure_windows(c, 1);
    if (rc != DD_OK) {
        dd_destroy(c);
        return rc;
    }
    c->stream = c->own;
    *out = c;
    return DD_OK;
}

int dd_set_stream(dd_ctx* c, void* stream) {
    if (!c) return DD_ERR_ARG;
    c->stream = stream ? (cudaStream_t)stream : c->own;
    return DD_OK;
}

int dd_get_stats(dd_ctx* c, dd_stats* out) {
    if (!c || !out) return DD_ERR_ARG;
    *out = c->stats;
    return DD_OK;
}

int dd_reset_stats(dd_ctx* c) {
    if (!c) return DD_ERR_ARG;
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->t_ms.clear();
    return DD_OK;
}

int dd_get_launch_times(dd_ctx* c, float* ms, int32_t cap, int32_t* n) {
    if (!c || !n || cap < 0 || (cap > 0 && !ms)) return DD_ERR_ARG;
    const int32_t k = (int32_t)c->t_ms.size();
    for (int32_t i = 0; i < k && i < cap; i++) ms[i] = c->t_ms[i];
    *n = k;
    return DD_OK;
}

int dd_set_timing(dd_ctx* c, int32_t enable) {
    if (!c) return DD_ERR_ARG;
    c->timing = enable != 0;
    return DD_OK;
}

int dd_contrast(dd_ctx* c, const dd_events* ev, const float* D, int32_t nD, dd_i128* K, uint64_t* S,
                int64_t* N_in, uint32_t* iwe) {
    if (!c || nD < 0 || (nD > 0 && (!D || !K))) return DD_ERR_ARG;
    int rc = check_events(ev, c->g.planes);
    if (rc) return rc;
    for (int32_t j = 0; j < nD; j++)
        if (!d_ok(D[j], ev->tau)) return DD_ERR_ARG;
    rc = ingest(c, ev, 1);
    if (rc) return rc;
    if (nD == 0) {
        DD_TRY(copy(c, c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        return c->h_err[0] ? DD_ERR_ARG : DD_OK;
    }
    return eval_tasks(c, ev, nD, dd::TASK_POINT, D, D, K, S, N_in, iwe);
}

int dd_bound(dd_ctx* c, const dd_events* ev, const float* D_lo, const float* D_hi, int32_t n, dd_i128* Kbar,
             uint64_t* Sbar, int64_t* N_full, uint32_t* iwe) {
    if (!c || n < 0 || (n > 0 && (!D_lo || !D_hi || !Kbar))) return DD_ERR_ARG;
    int rc = check_events(ev, c->g.planes);
    if (rc) return rc;
    for (int32_t j = 0; j < n; j++)
        if (!d_ok(D_lo[j], ev->tau) || !d_ok(D_hi[j], ev->tau) || !(D_lo[j] <= D_hi[j])) return DD_ERR_ARG;
    rc = ingest(c, ev, 1);
    if (rc) return rc;
    if (n == 0) {
        DD_TRY(copy(c, c->h_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        return c->h_err[0] ? DD_ERR_ARG : DD_OK;
    }
    return eval_tasks(c, ev, n, dd::TASK_BOUND, D_lo, D_hi, Kbar, Sbar, N_full, iwe);
}

int dd_solve(dd_ctx* c, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma, dd_result* out) {
    dd_window_params p = {D_lo, D_hi, tol_D, 0, gamma};
    return solve_impl(c, ev, 1, &p, out, nullptr, 0, nullptr);
}

int dd_solve_trace(dd_ctx* c, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma,
                   dd_result* out, dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    dd_window_params p = {D_lo, D_hi, tol_D, 0, gamma};
    return solve_impl(c, ev, 1, &p, out, trace, trace_cap, trace_len);
}

int dd_solve_batch(dd_ctx* c, const dd_events* windows, int32_t n_windows, const dd_window_params* params,
                   dd_result* out) {
    return solve_impl(c, windows, n_windows, params, out, nullptr, 0, nullptr);
}

int dd_solve_window(dd_ctx* c, const dd_events* ev, const dd_window_params* p, dd_result* out,
                    dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    return solve_impl(c, ev, 1, p, out, trace, trace_cap, trace_len);
}

int dd_features(dd_ctx* c, const dd_events* windows, int32_t n_windows, float* feat) {
    if (!c || !windows || n_windows < 1 || !feat) return DD_ERR_ARG;
    for (int w = 0; w < n_windows; w++) {
        const int rc = check_events(&windows[w], c->g.planes);
        if (rc) return rc;
    }
    int rc = ingest(c, windows, n_windows);
    if (rc) return rc;
    rc = feature_counts(c, n_windows);
    if (rc) return rc;
    DD_TRY(dd::launch_feature_norm(n_windows, c->feat_counts, c->wins, feat, c->stream));
    c->stats.kernel_launches++;
    DD_TRY(copy(c, c->h_err, c->err, sizeof(int32_t) * n_windows, cudaMemcpyDeviceToHost));
    DD_TRY(sync(c));
    for (int w = 0; w < n_windows; w++)
        if (c->h_err[w]) return DD_ERR_ARG;
    return DD_OK;
}

int dd_resample(dd_ctx* c, const dd_events* in, int32_t W, int32_t H, int32_t W2, int32_t H2, float keep,
                uint64_t seed, int16_t* x_out, int16_t* y_out, float* t_out, int64_t* n_out) {
    if (!c || !n_out || W < 1 || H < 1 || W > 4096 || H > 4096 || W2 < 1 || H2 < 1 || W2 > 4096 || H2 > 4096)
        return DD_ERR_ARG;
    if (!std::isfinite(keep) || !(keep >= 0.0f) || !(keep <= 1.0f)) return DD_ERR_ARG;
    int rc = check_events(in, 1);                  // polarities are not carried over
    if (rc) return rc;
    if (in->n > 0 && (!x_out || !y_out || !t_out)) return DD_ERR_ARG;
    const int16_t* x = in->x;
    const int16_t* y = in->y;
    const float* t = in->t;
    if (!in->device_ptrs && in->n > 0) {          // host arrays: through the context's staging buffers
        rc = ensure_staging(c, in->n);
        if (rc) return rc;
        DD_TRY(copy(c, c->in_x, in->x, sizeof(int16_t) * in->n, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->in_y, in->y, sizeof(int16_t) * in->n, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->in_t, in->t, sizeof(float) * in->n, cudaMemcpyHostToDevice));
        x = c->in_x;
        y = c->in_y;
        t = c->in_t;
    }
    const int64_t nb = dd::resample_blocks(in->n);
    if (nb + 1 > c->rs_cap) {
        release(c->rs_counts);
        release(c->rs_offsets);
        release(c->rs_err);
        c->rs_cap = 0;
        const int64_t cap = nb + 1 < 64 ? 64 : nb + 1;
        DD_TRY(cudaMalloc((void**)&c->rs_counts, sizeof(int32_t) * cap));
        DD_TRY(cudaMalloc((void**)&c->rs_offsets, sizeof(int64_t) * cap));
        DD_TRY(cudaMalloc((void**)&c->rs_err, sizeof(int32_t)));
        c->rs_cap = cap;
    }
    DD_TRY(dd::launch_resample(x, y, t, in->n, W, H, W2, H2, keep, seed, x_out, y_out, t_out, c->rs_counts,
                               c->rs_offsets, c->rs_err, c->stream));
    c->stats.kernel_launches += nb ? 3 : 0;
    int64_t m = 0;
    int32_t bad = 0;
    DD_TRY(copy(c, &m, c->rs_offsets + nb, sizeof(int64_t), cudaMemcpyDeviceToHost));
    DD_TRY(copy(c, &bad, c->rs_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    DD_TRY(sync(c));
    if (bad) return DD_ERR_ARG;
    *n_out = m;
    return DD_OK;
}

int dd_stream_solve(dd_ctx* c, const dd_events* stream, double t_start, float tau, double hop, int32_t n_windows,
                    const dd_window_params* params, dd_result* out, float* ttc, int64_t* first) {
    if (!c || !stream || !params || !out || n_windows < 1 || !std::isfinite(t_start) || !std::isfinite(hop) ||
        !(hop > 0.0) || !std::isfinite(tau) || !(tau > 0.0f))
        return DD_ERR_ARG;
    if (stream->n < 0 || (stream->n > 0 && (!stream->x || !stream->y || !stream->t))) return DD_ERR_ARG;
    // The stream's windows: first event and count of each (device search,
    // or host search for host arrays, with the same binary32 test).
    std::vector<int64_t> f((size_t)n_windows), cnt((size_t)n_windows);
    std::vector<float> t0((size_t)n_windows);
    if (stream->device_ptrs) {
        int64_t* d = nullptr;
        DD_TRY(cudaMallocAsync((void**)&d, sizeof(int64_t) * 2 * n_windows + sizeof(float) * n_windows, c->stream));
        cudaError_t e = dd::launch_stream_bounds(stream->t, stream->n, t_start, hop, tau, n_windows, d,
                                                 d + n_windows, (float*)(d + 2 * n_windows), c->stream);
        c->stats.kernel_launches++;
        if (e == cudaSuccess) e = copy(c, f.data(), d, sizeof(int64_t) * n_windows, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = copy(c, cnt.data(), d + n_windows, sizeof(int64_t) * n_windows, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = copy(c, t0.data(), d + 2 * n_windows, sizeof(float) * n_windows, cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaFreeAsync(d, c->stream);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = sync(c);
        DD_TRY(e);
    } else {
        for (int32_t k = 0; k < n_windows; k++) {
            const float w0 = (float)(t_start + hop * (double)k);
            int64_t lo = 0, hi = stream->n;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (stream->t[mid] - w0 >= 0.0f) hi = mid;
                else lo = mid + 1;
            }
            int64_t a = lo, b = stream->n;
            while (a < b) {
                const int64_t mid = a + (b - a) / 2;
                if (stream->t[mid] - w0 > tau) b = mid;
                else a = mid + 1;
            }
            f[k] = lo;
            cnt[k] = a - lo;
            t0[k] = w0;
        }
    }
    std::vector<dd_events> ws((size_t)n_windows);
    std::vector<dd_window_params> ps((size_t)n_windows, *params);
    for (int32_t k = 0; k < n_windows; k++) {
        dd_events& e = ws[k];
        e.x = stream->x + f[k];
        e.y = stream->y + f[k];
        e.t = stream->t + f[k];
        e.p = stream->p ? stream->p + f[k] : nullptr;
        e.n = cnt[k];
        e.t0 = t0[k];
        e.tau = tau;
        e.device_ptrs = stream->device_ptrs;
        if (first) first[k] = f[k];
    }
    const int rc = solve_impl(c, ws.data(), n_windows, ps.data(), out, nullptr, 0, nullptr);
    if (ttc)
        for (int32_t k = 0; k < n_windows; k++)   // time to contact at the window's end: 1/D_end
            ttc[k] = out[k].status == DD_OK && out[k].D_end > 0.0f ? 1.0f / out[k].D_end : INFINITY;
    return rc;
}

int dd_check_flags(uint32_t* flags, int32_t* checked, int32_t reset) {
    if (!flags || !checked) return DD_ERR_ARG;
    DD_TRY(dd::check_flags(flags, checked, reset != 0));
    return DD_OK;
}

int dd_time_span(dd_ctx* c, const dd_events* ev, float* t0, float* tau) {
    if (!c || !ev || !t0 || !tau || ev->n < 1 || !ev->t) return DD_ERR_ARG;
    float lo = INFINITY, hi = -INFINITY;
    if (ev->device_ptrs) {
        const int32_t nb = dd::span_blocks(ev->n);
        float2* d = nullptr;
        DD_TRY(cudaMallocAsync((void**)&d, sizeof(float2) * (nb + 1), c->stream));
        float2 h;
        cudaError_t e = dd::launch_time_span(ev->t, ev->n, d, d + nb, c->stream);
        c->stats.kernel_launches += 2;
        if (e == cudaSuccess) e = copy(c, &h, d + nb, sizeof(float2), cudaMemcpyDeviceToHost);
        cudaError_t e2 = cudaFreeAsync(d, c->stream);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = sync(c);
        DD_TRY(e);
        lo = h.x;
        hi = h.y;
    } else {
        for (int64_t i = 0; i < ev->n; i++)
            if (std::isfinite(ev->t[i])) {
                lo = std::fmin(lo, ev->t[i]);
                hi = std::fmax(hi, ev->t[i]);
            }
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) return DD_ERR_ARG;
    const float span = hi - lo;                    // binary32, as the window test takes t - t0
    if (!(span > 0.0f) || !std::isfinite(span)) return DD_ERR_ARG;
    *t0 = lo;
    *tau = span;
    return DD_OK;
}

int dd_resample_foe(int32_t W, int32_t H, float foe_x, float foe_y, int32_t W2, int32_t H2, float* foe_x2,
                    float* foe_y2) {
    if (W < 1 || H < 1 || W2 < 1 || H2 < 1 || !foe_x2 || !foe_y2) return DD_ERR_ARG;
    *foe_x2 = foe_x * ((float)W2 / (float)W);
    *foe_y2 = foe_y * ((float)H2 / (float)H);
    return DD_OK;
}

int dd_set_warm_model(dd_ctx* c, dd_mlp* m) {
    if (!c) return DD_ERR_ARG;
    if (m) {
        dd::MlpDev v;
        int dev = -1;
        if (!dd::mlp_device_view(m, &v, &dev) || dev != c->device) return DD_ERR_ARG;
    }
    c->warm_model = m;
    return DD_OK;
}

}  // extern "C"
