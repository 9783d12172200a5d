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

struct dd_ctx {
    int device = 0;
    dd::Geom g{};
    dd_config cfg{};
    int threads = 512;
    int max_tasks = 0;
    cudaStream_t own = nullptr, stream = nullptr;

    dd::Ev* ev = nullptr;
    int64_t ev_cap = 0;
    float2* rcp = nullptr;        // per sorted event: 1/(x - FOE_x), 1/(y - FOE_y)
    int64_t rcp_cap = 0;
    int16_t *in_x = nullptr, *in_y = nullptr;
    float* in_t = nullptr;
    int64_t in_cap = 0;
    int32_t *row_count = nullptr, *row_off = nullptr, *cursor = nullptr, *err = nullptr;
    int32_t* work = nullptr;      // IWE unit counter of the persistent evaluation grid
    uint32_t* macc = nullptr;     // merge buffers of split IWE items (zero between uses)
    int32_t* mdone = nullptr;
    unsigned long long* mfull = nullptr;
    int eval_blocks = 0;          // resident blocks of that grid

    dd::Task* tasks = nullptr;
    dd::Partial* part = nullptr;
    i128* keys = nullptr;
    unsigned long long *S = nullptr, *C = nullptr, *F = nullptr;
    uint32_t* iwe = nullptr;
    size_t iwe_cap = 0;

    dd::SolveState* st = nullptr;
    dd::Node* queue = nullptr;   // two buffers of queue_capacity nodes
    dd::TraceRec* trace = nullptr;
    int64_t trace_cap = 0;

    // telemetry (dd_stats) and optional per-launch timing of the IWE kernel
    dd_stats stats{};
    int timing = 0;
    std::vector<cudaEvent_t> t_ev;
    size_t t_used = 0;

    // the rounds of a solve as one CUDA graph (a conditional while loop)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* g_ev = nullptr;
    const void* g_trace = nullptr;

    // pinned host staging
    dd::SolveState* h_st = nullptr;
    dd::Task* h_tasks = nullptr;
    int32_t* h_flag = nullptr;
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

bool d_ok(float D, float tau) {
    if (!std::isfinite(D)) return false;
    double dt = (double)D * (double)tau;
    return dt <= 0.75 && dt >= -64.0;
}

// Host check of a window's arguments (events are checked on the host when
// they are host arrays, and by the ingest kernel when they are device arrays).
int check_events(const dd_ctx* c, const dd_events* ev) {
    if (!ev || ev->n < 0 || ev->n > INT32_MAX / 2) return DD_ERR_ARG;
    if (!std::isfinite(ev->tau) || !(ev->tau > 0.0f) || !std::isfinite(ev->t0)) return DD_ERR_ARG;
    if (ev->n > 0 && (!ev->x || !ev->y || !ev->t)) return DD_ERR_ARG;
    if (!ev->device_ptrs) {
        for (int64_t i = 0; i < ev->n; i++) {
            float tr = ev->t[i] - ev->t0;
            if (!std::isfinite(ev->t[i]) || !(tr >= 0.0f) || !(tr <= ev->tau)) return DD_ERR_ARG;
            if (ev->x[i] < 0 || ev->x[i] >= c->g.W || ev->y[i] < 0 || ev->y[i] >= c->g.H) return DD_ERR_ARG;
        }
    }
    return DD_OK;
}

template <class T>
int grow(T** p, int64_t* cap, int64_t need) {
    if (need <= *cap) return DD_OK;
    int64_t nc = need < 1024 ? 1024 : need + need / 4;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    DD_TRY(cudaMalloc((void**)p, sizeof(T) * (size_t)nc));
    *cap = nc;
    return DD_OK;
}

cudaError_t copy(dd_ctx* c, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind);

// Upload (host arrays) or alias (device arrays) the events, then sort them by
// row into ctx->ev.  Sets ctx->err on malformed device events.
int ingest(dd_ctx* c, const dd_events* ev) {
    int rc = grow(&c->ev, &c->ev_cap, ev->n);
    if (rc) return rc;
    rc = grow(&c->rcp, &c->rcp_cap, ev->n);
    if (rc) return rc;
    const int16_t *x = ev->x, *y = ev->y;
    const float* t = ev->t;
    if (!ev->device_ptrs && ev->n > 0) {
        if (ev->n > c->in_cap) {
            cudaFree(c->in_x);
            cudaFree(c->in_y);
            cudaFree(c->in_t);
            c->in_x = c->in_y = nullptr;
            c->in_t = nullptr;
            c->in_cap = 0;
            int64_t nc = ev->n + ev->n / 4;
            DD_TRY(cudaMalloc((void**)&c->in_x, sizeof(int16_t) * nc));
            DD_TRY(cudaMalloc((void**)&c->in_y, sizeof(int16_t) * nc));
            DD_TRY(cudaMalloc((void**)&c->in_t, sizeof(float) * nc));
            c->in_cap = nc;
        }
        DD_TRY(copy(c, c->in_x, ev->x, sizeof(int16_t) * ev->n, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->in_y, ev->y, sizeof(int16_t) * ev->n, cudaMemcpyHostToDevice));
        DD_TRY(copy(c, c->in_t, ev->t, sizeof(float) * ev->n, cudaMemcpyHostToDevice));
        x = c->in_x;
        y = c->in_y;
        t = c->in_t;
    }
    DD_TRY(dd::launch_ingest(c->g, x, y, t, ev->n, ev->t0, ev->tau, c->ev, c->rcp, c->row_count, c->row_off, c->cursor,
                             c->err, c->stream));
    c->stats.kernel_launches += ev->n > 0 ? 3 : 1;
    return DD_OK;
}

dd_i128 from_i128(i128 v) {
    dd_i128 r;
    r.lo = (uint64_t)(unsigned __int128)v;
    r.hi = (int64_t)(uint64_t)((unsigned __int128)v >> 64);
    return r;
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

cudaError_t eval(dd_ctx* c, const int32_t* n_tasks_dev, int32_t n_tasks_max, float tau, uint32_t* iwe,
                 const dd::SolveState* st) {
    if (c->timing) {
        cudaError_t e = record(c);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = dd::launch_eval(c->g, c->ev, c->rcp, c->row_off, c->tasks, n_tasks_dev, n_tasks_max, tau, c->part, iwe,
                                    st, c->threads, c->stream, c->work, c->eval_blocks, c->macc, c->mdone,
                                    c->mfull);
    if (e != cudaSuccess) return e;
    c->stats.kernel_launches++;
    c->stats.eval_launches++;
    if (c->timing) return record(c);
    return cudaSuccess;
}

// Evaluate n tasks (point or bound) and copy keys/sums/images to the host.
int eval_tasks(dd_ctx* c, const dd_events* ev, int32_t n, int kind, const float* A, const float* B, dd_i128* K,
               uint64_t* S, int64_t* N, uint32_t* iwe) {
    const int64_t M = (int64_t)c->g.W * c->g.H;
    for (int32_t j0 = 0; j0 < n; j0 += c->max_tasks) {
        const int32_t m = n - j0 < c->max_tasks ? n - j0 : c->max_tasks;
        for (int32_t j = 0; j < m; j++) {
            c->h_tasks[j].D_lo = A[j0 + j];
            c->h_tasks[j].D_hi = B[j0 + j];
            c->h_tasks[j].kind = kind;
            c->h_tasks[j].splits =
                kind == dd::TASK_BOUND ? dd::bound_splits(c->g, A[j0 + j], B[j0 + j], ev->tau) : 1;
        }
        DD_TRY(copy(c, c->tasks, c->h_tasks, sizeof(dd::Task) * m, cudaMemcpyHostToDevice));
        uint32_t* iw = nullptr;
        if (iwe) {
            size_t need = (size_t)m * M;
            if (need > c->iwe_cap) {
                cudaFree(c->iwe);
                c->iwe = nullptr;
                c->iwe_cap = 0;
                DD_TRY(cudaMalloc((void**)&c->iwe, need * sizeof(uint32_t)));
                c->iwe_cap = need;
            }
            iw = c->iwe;
        }
        DD_TRY(cudaMemsetAsync(c->work, 0, sizeof(int32_t), c->stream));
        DD_TRY(eval(c, nullptr, m, ev->tau, iw, nullptr));
        DD_TRY(dd::launch_keys(c->g, c->tasks, m, c->part, c->keys, c->S, c->C, c->F, c->stream));
        c->stats.kernel_launches++;
        std::vector<i128> hk(m);
        std::vector<unsigned long long> hs(m), hc(m), hf(m);
        DD_TRY(copy(c, hk.data(), c->keys, sizeof(i128) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hs.data(), c->S, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hc.data(), c->C, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, hf.data(), c->F, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
        DD_TRY(copy(c, c->h_flag, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (iwe)
            DD_TRY(copy(c, iwe + (size_t)j0 * M, c->iwe, sizeof(uint32_t) * (size_t)m * M, cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        if (*c->h_flag) return DD_ERR_ARG;
        for (int32_t j = 0; j < m; j++) {
            K[j0 + j] = from_i128(hk[j]);
            if (S) S[j0 + j] = hs[j];
            if (N) N[j0 + j] = (int64_t)(kind == dd::TASK_POINT ? hc[j] : hf[j]);
        }
    }
    return DD_OK;
}

void drop_graph(dd_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

// Build the solve graph: a while node whose body is one round (IWE
// evaluation, then the control kernel, which clears the loop condition when
// the search is over).  Kernel arguments are baked in, so the graph is
// rebuilt when a buffer it points to is reallocated.
int build_graph(dd_ctx* c, dd::TraceRec* trace) {
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
    cudaError_t e1 = dd::launch_eval(c->g, c->ev, c->rcp, c->row_off, c->tasks, &c->st->n_tasks, c->max_tasks, 0.0f,
                                     c->part, nullptr, c->st, c->threads, c->own, c->work, c->eval_blocks, c->macc,
                                     c->mdone, c->mfull);
    cudaError_t e2 = dd::launch_control(c->g, c->st, c->queue, c->queue + c->cfg.queue_capacity, c->tasks,
                                        c->part, c->err, trace, h, 1, c->work, c->own);
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
    c->g_ev = c->ev;
    c->g_trace = trace;
    return DD_OK;
}

int solve_impl(dd_ctx* c, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma, dd_result* out,
               dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    if (!c || !out) return DD_ERR_ARG;
    int rc = check_events(c, ev);
    if (rc) return rc;
    if (!d_ok(D_lo, ev->tau) || !d_ok(D_hi, ev->tau) || !(D_lo < D_hi)) return DD_ERR_ARG;
    if (!std::isfinite(tol_D) || !(tol_D >= 0.0f) || !std::isfinite(gamma) || !(gamma >= 0.0)) return DD_ERR_ARG;
    if (trace_cap < 0 || (trace_cap > 0 && !trace)) return DD_ERR_ARG;
    if (trace_cap > c->trace_cap) {
        cudaFree(c->trace);
        c->trace = nullptr;
        c->trace_cap = 0;
        DD_TRY(cudaMalloc((void**)&c->trace, sizeof(dd::TraceRec) * trace_cap));
        c->trace_cap = trace_cap;
    }
    rc = ingest(c, ev);
    if (rc) return rc;
    const int64_t M = (int64_t)c->g.W * c->g.H;
    const i128 gamma_K = (i128)std::floor(gamma * (double)M * (double)M);
    DD_TRY(dd::launch_init(c->g, c->st, c->tasks, M, D_lo, D_hi, tol_D, ev->tau, gamma_K, c->cfg.pop_k,
                           c->cfg.queue_capacity, c->cfg.max_rounds, (int32_t)trace_cap, c->work, c->stream));
    c->stats.kernel_launches++;
    dd::TraceRec* tr_dev = trace_cap > 0 ? c->trace : nullptr;
    const bool graph = !c->cfg.host_loop && !c->timing;
    if (graph) {
        // One graph launch runs every round on the device.
        if (!c->gexec || c->g_ev != (const void*)c->ev || c->g_trace != (const void*)tr_dev) {
            rc = build_graph(c, tr_dev);
            if (rc) return rc;
        }
        DD_TRY(cudaGraphLaunch(c->gexec, c->stream));
    } else {
        // Host-driven rounds: launch batches, poll for the end.
        int batch = 2;
        for (;;) {
            for (int b = 0; b < batch; b++) {
                DD_TRY(eval(c, &c->st->n_tasks, c->max_tasks, ev->tau, nullptr, c->st));
                DD_TRY(dd::launch_control(c->g, c->st, c->queue, c->queue + c->cfg.queue_capacity, c->tasks,
                                          c->part, c->err, tr_dev, 0, 0, c->work, c->stream));
                c->stats.kernel_launches++;
            }
            DD_TRY(copy(c, c->h_flag, &c->st->phase, sizeof(int32_t), cudaMemcpyDeviceToHost));
            DD_TRY(sync(c));
            if (*c->h_flag == dd::PH_DONE) break;
            if (batch < 64) batch *= 2;
        }
    }
    DD_TRY(copy(c, c->h_st, c->st, sizeof(dd::SolveState), cudaMemcpyDeviceToHost));
    std::vector<dd::TraceRec> tr((size_t)trace_cap);
    if (trace_cap > 0) DD_TRY(copy(c, tr.data(), c->trace, sizeof(dd::TraceRec) * trace_cap, cudaMemcpyDeviceToHost));
    DD_TRY(sync(c));
    const dd::SolveState& s = *c->h_st;
    if (graph) {                                  // the loop ran rounds + 1 times
        c->stats.kernel_launches += 2 * (s.rounds + 1);
        c->stats.eval_launches += s.rounds + 1;
    }
    if (s.status != DD_OK) return s.status;
    // Sec. 4.1 retrieval and reporting (double precision, from the exact keys).
    dd_result r;
    std::memset(&r, 0, sizeof(r));
    r.D_star = s.D_hat;
    r.D_end = (float)((double)s.D_hat / (1.0 - (double)s.D_hat * (double)ev->tau));
    r.K_hat = from_i128(s.K_hat);
    r.gap_K = from_i128(s.stop_kb);
    r.contrast = (double)s.K_hat / ((double)M * (double)M);
    r.bound_gap = (double)s.stop_kb / ((double)M * (double)M);
    r.nodes_expanded = s.nodes_expanded;
    r.point_evals = s.point_evals;
    r.bound_evals = s.bound_evals;
    r.event_warps = ev->n * (s.point_evals + s.bound_evals);
    r.cell_increments = s.cells;
    r.bound_increments = s.bcells;
    r.rounds = s.rounds;
    r.max_queue = s.max_queue;
    r.status = DD_OK;
    *out = r;
    if (trace_len) *trace_len = s.trace_len;
    for (int64_t i = 0; i < trace_cap && i < s.trace_len; i++) {
        trace[i].D_lo = tr[i].D_lo;
        trace[i].D_hi = tr[i].D_hi;
        trace[i].D_c = tr[i].D_c;
        trace[i].leaf = tr[i].leaf;
        trace[i].Kbar = from_i128(tr[i].Kbar);
        trace[i].K_c = from_i128(tr[i].K_c);
    }
    return DD_OK;
}

}  // namespace

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
        case DD_ERR_CAPACITY: return "input exceeds the fixed scratch of the allocation-free entry point";
        default: return "unknown status";
    }
}

void dd_destroy(dd_ctx* c) {
    if (!c) return;
    cudaFree(c->ev);
    cudaFree(c->rcp);
    cudaFree(c->in_x);
    cudaFree(c->in_y);
    cudaFree(c->in_t);
    cudaFree(c->row_count);
    cudaFree(c->row_off);
    cudaFree(c->cursor);
    cudaFree(c->err);
    cudaFree(c->work);
    cudaFree(c->macc);
    cudaFree(c->mdone);
    cudaFree(c->mfull);
    cudaFree(c->tasks);
    cudaFree(c->part);
    cudaFree(c->keys);
    cudaFree(c->S);
    cudaFree(c->C);
    cudaFree(c->F);
    cudaFree(c->iwe);
    cudaFree(c->st);
    cudaFree(c->queue);
    cudaFree(c->trace);
    cudaFreeHost(c->h_st);
    cudaFreeHost(c->h_tasks);
    cudaFreeHost(c->h_flag);
    for (cudaEvent_t e : c->t_ev) cudaEventDestroy(e);
    drop_graph(c);
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
    if (k.threads && (k.threads % 32 || k.threads > 1024)) return DD_ERR_ARG;
    if (k.max_splits < 0 || k.max_splits > 64 || k.host_loop < 0) return DD_ERR_ARG;
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
    c->g.n_tiles = (H + rows - 1) / rows;
    c->g.n_tb = dd::time_buckets(H);
    c->g.max_splits = k.max_splits ? k.max_splits : 16;
    c->max_tasks = 3 * k.pop_k > 64 ? 3 * k.pop_k : 64;
    c->cfg.threads = c->threads;
    c->cfg.band_rows = rows;

    int rc = DD_OK;
    auto A = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    const int bins = c->g.n_tb * H;
    A((void**)&c->row_count, sizeof(int32_t) * bins);
    A((void**)&c->row_off, sizeof(int32_t) * (bins + 1));
    A((void**)&c->cursor, sizeof(int32_t) * bins);
    A((void**)&c->err, sizeof(int32_t));
    A((void**)&c->work, sizeof(int32_t));
    A((void**)&c->macc, sizeof(uint32_t) * (size_t)c->max_tasks * W * H);
    A((void**)&c->mdone, sizeof(int32_t) * (size_t)c->max_tasks * c->g.n_tiles);
    A((void**)&c->mfull, sizeof(unsigned long long) * (size_t)c->max_tasks * c->g.n_tiles);
    if (rc == DD_OK && (cudaMemset(c->macc, 0, sizeof(uint32_t) * (size_t)c->max_tasks * W * H) != cudaSuccess ||
                        cudaMemset(c->mdone, 0, sizeof(int32_t) * (size_t)c->max_tasks * c->g.n_tiles) != cudaSuccess ||
                        cudaMemset(c->mfull, 0, sizeof(unsigned long long) * (size_t)c->max_tasks * c->g.n_tiles) !=
                            cudaSuccess))
        rc = DD_ERR_CUDA;
    A((void**)&c->tasks, sizeof(dd::Task) * c->max_tasks);
    A((void**)&c->part, sizeof(dd::Partial) * (size_t)c->max_tasks * c->g.n_tiles);
    A((void**)&c->keys, sizeof(i128) * c->max_tasks);
    A((void**)&c->S, sizeof(unsigned long long) * c->max_tasks);
    A((void**)&c->C, sizeof(unsigned long long) * c->max_tasks);
    A((void**)&c->F, sizeof(unsigned long long) * c->max_tasks);
    A((void**)&c->st, sizeof(dd::SolveState));
    A((void**)&c->queue, sizeof(dd::Node) * 2 * (size_t)k.queue_capacity);
    if (rc == DD_OK && cudaMallocHost((void**)&c->h_st, sizeof(dd::SolveState)) != cudaSuccess) rc = DD_ERR_OOM;
    if (rc == DD_OK && cudaMallocHost((void**)&c->h_tasks, sizeof(dd::Task) * c->max_tasks) != cudaSuccess)
        rc = DD_ERR_OOM;
    if (rc == DD_OK && cudaMallocHost((void**)&c->h_flag, sizeof(int32_t)) != cudaSuccess) rc = DD_ERR_OOM;
    if (rc == DD_OK && cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK && dd::eval_smem_setup(c->g) != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK && (c->eval_blocks = dd::eval_resident_blocks(c->g, c->threads)) <= 0) rc = DD_ERR_CUDA;
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

int dd_contrast(dd_ctx* c, const dd_events* ev, const float* D, int32_t nD, dd_i128* K, uint64_t* S,
                int64_t* N_in, uint32_t* iwe) {
    if (!c || nD < 0 || (nD > 0 && (!D || !K))) return DD_ERR_ARG;
    int rc = check_events(c, ev);
    if (rc) return rc;
    for (int32_t j = 0; j < nD; j++)
        if (!d_ok(D[j], ev->tau)) return DD_ERR_ARG;
    rc = ingest(c, ev);
    if (rc) return rc;
    if (nD == 0) {
        DD_TRY(copy(c, c->h_flag, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        return *c->h_flag ? DD_ERR_ARG : DD_OK;
    }
    return eval_tasks(c, ev, nD, dd::TASK_POINT, D, D, K, S, N_in, iwe);
}

int dd_bound(dd_ctx* c, const dd_events* ev, const float* D_lo, const float* D_hi, int32_t n, dd_i128* Kbar,
             uint64_t* Sbar, int64_t* N_full, uint32_t* iwe) {
    if (!c || n < 0 || (n > 0 && (!D_lo || !D_hi || !Kbar))) return DD_ERR_ARG;
    int rc = check_events(c, ev);
    if (rc) return rc;
    for (int32_t j = 0; j < n; j++)
        if (!d_ok(D_lo[j], ev->tau) || !d_ok(D_hi[j], ev->tau) || !(D_lo[j] <= D_hi[j])) return DD_ERR_ARG;
    rc = ingest(c, ev);
    if (rc) return rc;
    if (n == 0) {
        DD_TRY(copy(c, c->h_flag, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        DD_TRY(sync(c));
        return *c->h_flag ? DD_ERR_ARG : DD_OK;
    }
    return eval_tasks(c, ev, n, dd::TASK_BOUND, D_lo, D_hi, Kbar, Sbar, N_full, iwe);
}

int dd_get_stats(dd_ctx* c, dd_stats* out) {
    if (!c || !out) return DD_ERR_ARG;
    *out = c->stats;
    return DD_OK;
}

int dd_reset_stats(dd_ctx* c) {
    if (!c) return DD_ERR_ARG;
    std::memset(&c->stats, 0, sizeof(c->stats));
    return DD_OK;
}

int dd_set_timing(dd_ctx* c, int32_t enable) {
    if (!c) return DD_ERR_ARG;
    c->timing = enable != 0;
    return DD_OK;
}

int dd_solve(dd_ctx* c, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma, dd_result* out) {
    return solve_impl(c, ev, D_lo, D_hi, tol_D, gamma, out, nullptr, 0, nullptr);
}

int dd_solve_trace(dd_ctx* c, const dd_events* ev, float D_lo, float D_hi, float tol_D, double gamma,
                   dd_result* out, dd_node_rec* trace, int64_t trace_cap, int64_t* trace_len) {
    return solve_impl(c, ev, D_lo, D_hi, tol_D, gamma, out, trace, trace_cap, trace_len);
}

}  // extern "C"
