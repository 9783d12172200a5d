// Serving engine: continuous batching of windows from concurrent streams.
//
// A server owns S device slots, each able to hold one window of up to E
// events with its whole search state (sorted events, row tables, queue,
// tasks, partials).  One host thread runs the loop:
//   1. admit: every request whose arrival time has passed takes a free slot;
//      device-resident events are sorted and its search starts (its first
//      jobs join the job list of the next round); host-array events are
//      first copied into the slot by an upload thread on a copy stream, so
//      the rounds of the other windows go on meanwhile, and the search starts
//      between rounds once the copy has landed;
//   2. one round over all busy slots: a single evaluation launch for the jobs
//      of every busy window, then one control block per slot;
//   3. retire: windows that finished hand back their result and free their
//      slot for the next request.
// Requests therefore join and leave between rounds while others are in
// flight: their evaluations share launches, and a result does not depend on
// which other windows shared its rounds (each window's search only reads its
// own slot).
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    dd_events ev{};
    dd_window_params p{};
    double arrival = 0.0, done_t = 0.0;
    int slot = -1;
    int state = 0;            // 0 waiting, 1 running, 2 finished
    int status = DD_OK;
    bool cancel = false;      // running: stop it at the next round
    bool cancel_sent = false; // its slot's device flag is set
    dd_result res{};
};

}  // namespace

struct dd_server {
    dd::Geom g{};
    int32_t threads = 0, eval_blocks = 0, max_tasks = 0, pop_k = 1, qcap = 0;
    int64_t max_rounds = 0;
    int S = 0;
    int64_t E = 0;
    int bins = 0, max_chunks = 0;
    bool cancel_pending = false;  // a running request was cancelled (under mu)
    bool up_stop = false;         // the upload thread ends (under mu)
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;   // host-array uploads
    std::vector<cudaEvent_t> up_ev;       // per slot: its uploaded events have landed
    std::vector<int> up_state;            // per slot: 0 none, 1 waiting for the upload thread, 2 copies
                                          // issued (under mu)
    std::deque<int> up_queue;             // slots for the upload thread (under mu)
    std::thread up_th;

    // device, per slot
    dd::Ev* ev = nullptr;
    float2* rcp = nullptr;
    int16_t *in_x = nullptr, *in_y = nullptr;
    float* in_t = nullptr;
    int8_t* in_p = nullptr;       // polarities (two planes only)
    int32_t *row_count = nullptr, *row_off = nullptr, *cursor = nullptr, *err = nullptr, *phase = nullptr;
    int32_t* chunk_zero = nullptr;
    dd::WinIn* wins = nullptr;
    dd::WinParams* params = nullptr;
    dd::SolveState* st = nullptr;
    dd::Node* queues = nullptr;
    dd::Task* tasks = nullptr;
    dd::Partial* part = nullptr;
    dd::Job* jobs = nullptr;
    int job_stride = 0;
    dd::Sched* sch = nullptr;
    int32_t* feat_counts = nullptr;    // [128], the admitted window's features
    dd::MlpDev model{};
    bool has_model = false;

    // pinned host (window descriptors and parameters staged per slot)
    int32_t* h_phase = nullptr;
    dd::SolveState* h_st = nullptr;
    dd::WinIn* h_win = nullptr;
    dd::WinParams* h_par = nullptr;

    // requests
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> waiting;      // in submission order
    std::vector<uint64_t> slot_req;    // ticket per slot, 0 = free
    uint64_t next_ticket = 1;
    bool stopping = false;
    int failed = DD_OK;
    std::thread th;

    // telemetry
    int64_t rounds = 0, admitted = 0, peak_busy = 0;
};

namespace {

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

void free_server(dd_server* s) {
    release(s->ev);
    release(s->rcp);
    release(s->in_x);
    release(s->in_y);
    release(s->in_t);
    release(s->in_p);
    release(s->row_count);
    release(s->row_off);
    release(s->cursor);
    release(s->err);
    release(s->phase);
    release(s->chunk_zero);
    release(s->wins);
    release(s->params);
    release(s->st);
    release(s->queues);
    release(s->tasks);
    release(s->part);
    release(s->jobs);
    release(s->sch);
    release(s->feat_counts);
    release_host(s->h_phase);
    release_host(s->h_st);
    release_host(s->h_win);
    release_host(s->h_par);
    if (s->stream) cudaStreamDestroy(s->stream);
    s->stream = nullptr;
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    s->copy_stream = nullptr;
    for (cudaEvent_t e : s->up_ev)
        if (e) cudaEventDestroy(e);
    s->up_ev.clear();
}

size_t slot_bytes(const dd_server* s) {
    return (size_t)s->E * (sizeof(dd::Ev) + sizeof(float2) + 2 * sizeof(int16_t) + sizeof(float) +
                           (s->g.planes > 1 ? sizeof(int8_t) : 0)) +
           sizeof(int32_t) * (3 * (size_t)s->bins + 1) + sizeof(dd::SolveState) +
           sizeof(dd::Node) * 2 * (size_t)s->qcap + sizeof(dd::Task) * (size_t)s->max_tasks +
           sizeof(dd::Partial) * (size_t)s->max_tasks + sizeof(dd::Job) * 2 * (size_t)dd::jobs_per_window(s->g, s->max_tasks);
}

int alloc_server(dd_server* s) {
    int rc = DD_OK;
    auto A = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    auto AH = [&](void** p, size_t bytes) {
        if (rc == DD_OK && cudaMallocHost(p, bytes) != cudaSuccess) rc = DD_ERR_OOM;
    };
    const size_t S = (size_t)s->S, E = (size_t)s->E;
    A((void**)&s->ev, sizeof(dd::Ev) * S * E);
    A((void**)&s->rcp, sizeof(float2) * S * E);
    A((void**)&s->in_x, sizeof(int16_t) * S * E);
    A((void**)&s->in_y, sizeof(int16_t) * S * E);
    A((void**)&s->in_t, sizeof(float) * S * E);
    if (s->g.planes > 1) A((void**)&s->in_p, sizeof(int8_t) * S * E);
    A((void**)&s->row_count, sizeof(int32_t) * S * s->bins);
    A((void**)&s->row_off, sizeof(int32_t) * S * (s->bins + 1));
    A((void**)&s->cursor, sizeof(int32_t) * S * s->bins);
    A((void**)&s->err, sizeof(int32_t) * S);
    A((void**)&s->phase, sizeof(int32_t) * S);
    A((void**)&s->chunk_zero, sizeof(int32_t) * (size_t)s->max_chunks);
    A((void**)&s->wins, sizeof(dd::WinIn) * S);
    A((void**)&s->params, sizeof(dd::WinParams) * S);
    A((void**)&s->st, sizeof(dd::SolveState) * S);
    A((void**)&s->queues, sizeof(dd::Node) * 2 * (size_t)s->qcap * S);
    A((void**)&s->tasks, sizeof(dd::Task) * (size_t)s->max_tasks * S);
    A((void**)&s->part, sizeof(dd::Partial) * (size_t)s->max_tasks * S);
    s->job_stride = (int)(S * dd::jobs_per_window(s->g, s->max_tasks));
    A((void**)&s->jobs, sizeof(dd::Job) * 2 * (size_t)s->job_stride);
    A((void**)&s->sch, sizeof(dd::Sched));
    A((void**)&s->feat_counts, sizeof(int32_t) * dd::FEATURES);
    AH((void**)&s->h_phase, sizeof(int32_t) * S);
    AH((void**)&s->h_st, sizeof(dd::SolveState) * S);
    AH((void**)&s->h_win, sizeof(dd::WinIn) * S);
    AH((void**)&s->h_par, sizeof(dd::WinParams) * S);
    if (rc) return rc;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return DD_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return DD_ERR_CUDA;
    s->up_ev.assign(S, nullptr);
    s->up_state.assign(S, 0);
    for (size_t k = 0; k < S; k++)
        if (cudaEventCreateWithFlags(&s->up_ev[k], cudaEventDisableTiming) != cudaSuccess) return DD_ERR_CUDA;
    // Every slot starts free: a finished search takes no part in a round.
    std::memset(s->h_st, 0, sizeof(dd::SolveState) * S);
    for (size_t w = 0; w < S; w++) s->h_st[w].phase = dd::PH_DONE;
    if (cudaMemcpyAsync(s->st, s->h_st, sizeof(dd::SolveState) * S, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(s->sch, 0, sizeof(dd::Sched), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->chunk_zero, 0, sizeof(int32_t) * (size_t)s->max_chunks, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->wins, 0, sizeof(dd::WinIn) * S, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    return DD_OK;
}

// Copy the host-array events of request r into slot k's input buffers on
// the copy stream (the calling thread blocks only while pageable memory is
// staged; pinned memory returns at once) and mark their arrival with the
// slot's event.
cudaError_t upload(dd_server* s, int k, const Request& r) {
    const dd_events& e = r.ev;
    const size_t off = (size_t)k * s->E;
    cudaError_t c = cudaSuccess;
    if (e.n > 0) {
        c = cudaMemcpyAsync(s->in_x + off, e.x, sizeof(int16_t) * e.n, cudaMemcpyHostToDevice, s->copy_stream);
        if (c == cudaSuccess)
            c = cudaMemcpyAsync(s->in_y + off, e.y, sizeof(int16_t) * e.n, cudaMemcpyHostToDevice, s->copy_stream);
        if (c == cudaSuccess)
            c = cudaMemcpyAsync(s->in_t + off, e.t, sizeof(float) * e.n, cudaMemcpyHostToDevice, s->copy_stream);
        if (c == cudaSuccess && s->g.planes > 1)
            c = cudaMemcpyAsync(s->in_p + off, e.p, sizeof(int8_t) * e.n, cudaMemcpyHostToDevice, s->copy_stream);
    }
    if (c == cudaSuccess) c = cudaEventRecord(s->up_ev[k], s->copy_stream);
    return c;
}

// Start the search of request r in slot k (all asynchronous on the serving
// stream): host-array events are read from the slot's input buffers, where
// the upload put them; device arrays in place.  `sharers`: the searches of
// the coming round, this one included (its first bound splits by rows to
// fill its share of the grid).
cudaError_t start_search(dd_server* s, int k, const Request& r, int sharers) {
    const dd_events& e = r.ev;
    dd::WinIn& wi = s->h_win[k];
    const size_t off = (size_t)k * s->E;
    wi.x = e.x;
    wi.y = e.y;
    wi.t = e.t;
    wi.p = s->g.planes > 1 ? e.p : nullptr;
    if (!e.device_ptrs && e.n > 0) {
        wi.x = s->in_x + off;
        wi.y = s->in_y + off;
        wi.t = s->in_t + off;
        if (s->g.planes > 1) wi.p = s->in_p + off;
    }
    wi.n = e.n;
    wi.ev_off = (int64_t)off;
    wi.t0 = e.t0;
    wi.tau = e.tau;
    wi.chunk0 = 0;
    wi.pad = 0;
    dd::WinParams& q = s->h_par[k];
    const double M = (double)s->g.W * s->g.H;
    q.gamma_K = (dd::i128)std::floor(r.p.gamma * M * M);
    q.D_lo = r.p.D_lo;
    q.D_hi = r.p.D_hi;
    q.tol = r.p.tol_D;
    q.warm = r.p.warm;
    q.D_warm = r.p.warm == DD_WARM_GIVEN ? r.p.D_warm : 0.0f;
    q.w_warm = r.p.warm == DD_WARM_GIVEN ? r.p.w_warm : 0.0f;
    q.pad0 = q.pad1 = 0;
    // The slot's staging entries are rewritten only when the slot is started
    // again, after this search has retired (a later synchronised round), so
    // these copies need no wait.
    cudaError_t c = cudaMemcpyAsync(s->wins + k, &wi, sizeof(dd::WinIn), cudaMemcpyHostToDevice, s->stream);
    if (c != cudaSuccess) return c;
    c = cudaMemcpyAsync(s->params + k, &q, sizeof(dd::WinParams), cudaMemcpyHostToDevice, s->stream);
    if (c != cudaSuccess) return c;
    const int32_t n_chunks = (int32_t)((e.n + dd::CHUNK - 1) / dd::CHUNK);
    c = dd::launch_ingest(s->g, s->wins + k, 1, s->chunk_zero, n_chunks, s->ev, s->rcp,
                          s->row_count + (size_t)k * s->bins, s->row_off + (size_t)k * (s->bins + 1),
                          s->cursor + (size_t)k * s->bins, s->err + k, s->stream);
    if (c != cudaSuccess) return c;
    if (r.p.warm == DD_WARM_MODEL) {               // the model's guess for this window
        c = cudaMemsetAsync(s->feat_counts, 0, sizeof(int32_t) * dd::FEATURES, s->stream);
        if (c != cudaSuccess) return c;
        c = dd::launch_features(s->g, s->wins + k, s->chunk_zero, n_chunks, s->ev, s->feat_counts, s->stream);
        if (c != cudaSuccess) return c;
        c = dd::launch_warm(s->g, 1, s->feat_counts, s->wins + k, s->params + k, s->model, s->stream);
        if (c != cudaSuccess) return c;
    }
    return dd::launch_init(s->g, 1, s->st, s->tasks, s->max_tasks, s->part, s->wins, s->params, s->jobs,
                           s->job_stride, s->sch, s->pop_k, s->qcap, s->max_rounds, 0, s->stream, k,
                           sharers > 1 ? sharers : 1);
}

void fill(const dd::SolveState& st, const dd_events& ev, int64_t M, dd_result* out) {
    dd_result r;
    std::memset(&r, 0, sizeof(r));
    auto pack = [](dd::i128 v) {
        dd_i128 o;
        o.lo = (uint64_t)(unsigned __int128)v;
        o.hi = (int64_t)(uint64_t)((unsigned __int128)v >> 64);
        return o;
    };
    r.D_star = st.D_hat;
    r.D_end = (float)((double)st.D_hat / (1.0 - (double)st.D_hat * (double)ev.tau));
    r.K_hat = pack(st.K_hat);
    r.gap_K = pack(st.stop_kb);
    r.contrast = (double)st.K_hat / ((double)M * (double)M);
    r.bound_gap = (double)st.stop_kb / ((double)M * (double)M);
    r.nodes_expanded = st.nodes_expanded;
    r.point_evals = st.point_evals;
    r.bound_evals = st.bound_evals;
    r.event_warps = ev.n * (st.point_evals + st.bound_evals);
    r.cell_increments = st.cells;
    r.bound_increments = st.bcells;
    r.rounds = st.rounds;
    r.max_queue = st.max_queue;
    r.status = st.status;
    r.D_warm = st.D_warm;
    r.w_warm = st.w_warm;
    *out = r;
}

void fail_all(dd_server* s, int status) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->failed = status;
    for (auto& kv : s->reqs)
        if (kv.second.state != 2) {
            kv.second.state = 2;
            kv.second.status = status;
            kv.second.done_t = now_s();
        }
    s->waiting.clear();
    s->cv.notify_all();
}

// The upload thread: copies the host-array events of admitted requests into
// their slots on the copy stream, so that the serving thread never waits for
// a copy.
void uploader(dd_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        int k = -1;
        Request r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return !s->up_queue.empty() || s->up_stop; });
            if (s->up_queue.empty()) return;
            k = s->up_queue.front();
            s->up_queue.pop_front();
            r = s->reqs[s->slot_req[k]];
        }
        const cudaError_t c = upload(s, k, r);
        if (c != cudaSuccess) {
            fail_all(s, DD_ERR_CUDA);
            return;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->up_state[k] = 2;
        s->cv.notify_all();
    }
}

void loop(dd_server* s) {
    const int64_t M = (int64_t)s->g.W * s->g.H;
    dd::EvalArgs a{};
    a.ev = s->ev;
    a.rcp = s->rcp;
    a.row_off = s->row_off;
    a.wins = s->wins;
    a.tasks = s->tasks;
    a.task_stride = s->max_tasks;
    a.jobs = s->jobs;
    a.job_stride = s->job_stride;
    a.sch = s->sch;
    a.part = s->part;
    a.iwe_out = nullptr;
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<std::pair<int, uint64_t>> starts;   // searches to start before this round
        int busy = 0, searching = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                const double t = now_s();
                for (int k = 0; k < s->S && !s->waiting.empty(); k++) {
                    if (s->slot_req[k]) continue;
                    Request& r = s->reqs[s->waiting.front()];
                    if (r.arrival > t) break;
                    const uint64_t id = s->waiting.front();
                    s->waiting.pop_front();
                    s->slot_req[k] = id;
                    r.slot = k;
                    r.state = 1;
                    s->admitted++;
                    if (!r.ev.device_ptrs && r.ev.n > 0) {   // host arrays: to the upload thread first
                        s->up_state[k] = 1;
                        s->up_queue.push_back(k);
                        s->cv.notify_all();
                    } else {
                        starts.emplace_back(k, id);
                    }
                }
                // uploads that have landed: their searches start now (or,
                // cancelled meanwhile, they finish without one)
                int uploading = 0;
                for (int k = 0; k < s->S; k++) {
                    if (s->up_state[k] == 2 && cudaEventQuery(s->up_ev[k]) == cudaSuccess) {
                        s->up_state[k] = 0;
                        Request& r = s->reqs[s->slot_req[k]];
                        if (r.cancel) {
                            std::memset(&r.res, 0, sizeof(r.res));
                            r.res.status = DD_ERR_CANCELLED;
                            r.status = DD_ERR_CANCELLED;
                            r.state = 2;
                            r.done_t = now_s();
                            s->slot_req[k] = 0;
                            s->cv.notify_all();
                        } else {
                            starts.emplace_back(k, s->slot_req[k]);
                        }
                    }
                    uploading += s->up_state[k] != 0;
                }
                busy = 0;
                searching = 0;
                for (int k = 0; k < s->S; k++) {
                    busy += s->slot_req[k] != 0;
                    searching += s->slot_req[k] != 0 && s->up_state[k] == 0;
                }
                if (searching) break;
                if (s->stopping && s->waiting.empty() && !uploading) return;
                if (uploading) {
                    // nothing to evaluate until an upload lands
                    s->cv.wait_for(lk, std::chrono::microseconds(20));
                } else if (s->waiting.empty()) {
                    s->cv.wait(lk);
                } else {
                    const double dt = s->reqs[s->waiting.front()].arrival - now_s();
                    if (dt > 0) s->cv.wait_for(lk, std::chrono::duration<double>(dt));
                }
            }
        }
        for (auto& ad : starts) {
            Request r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r = s->reqs[ad.second];
            }
            if (start_search(s, ad.first, r, searching) != cudaSuccess) {
                fail_all(s, DD_ERR_CUDA);
                return;
            }
        }
        if (busy > s->peak_busy) s->peak_busy = busy;
        // Cancelled running requests: their slots' searches stop at this
        // round's control step (the flag is written before the round, in
        // stream order).
        std::vector<int> cancels;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->cancel_pending) {
                for (int k = 0; k < s->S; k++) {
                    if (!s->slot_req[k] || s->up_state[k]) continue;   // an upload's cancel is seen as it lands
                    Request& r = s->reqs[s->slot_req[k]];
                    if (r.cancel && !r.cancel_sent) {
                        r.cancel_sent = true;
                        cancels.push_back(k);
                    }
                }
                s->cancel_pending = false;
            }
        }
        for (int k : cancels) {
            static const int32_t one = 1;
            if (cudaMemcpyAsync(reinterpret_cast<char*>(s->st + k) + offsetof(dd::SolveState, cancel), &one,
                                sizeof(int32_t), cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
                fail_all(s, DD_ERR_CUDA);
                return;
            }
        }
        // One round over every busy slot.
        if (dd::launch_eval(s->g, a, s->threads, s->eval_blocks, s->stream) != cudaSuccess ||
            dd::launch_control(s->g, s->S, s->st, s->queues, s->tasks, s->max_tasks, s->part, s->err, nullptr,
                               s->jobs, s->job_stride, s->sch, 0, 0, s->stream, 1, s->phase) != cudaSuccess ||
            cudaMemcpyAsync(s->h_phase, s->phase, sizeof(int32_t) * s->S, cudaMemcpyDeviceToHost, s->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess) {
            fail_all(s, DD_ERR_CUDA);
            return;
        }
        s->rounds++;
        // Retire finished windows.
        std::vector<int> done;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int k = 0; k < s->S; k++)
                if (s->slot_req[k] && s->up_state[k] == 0 && s->h_phase[k] == dd::PH_DONE) done.push_back(k);
        }
        for (int k : done) {
            if (cudaMemcpyAsync(s->h_st + k, s->st + k, sizeof(dd::SolveState), cudaMemcpyDeviceToHost, s->stream) !=
                cudaSuccess) {
                fail_all(s, DD_ERR_CUDA);
                return;
            }
        }
        if (!done.empty() && cudaStreamSynchronize(s->stream) != cudaSuccess) {
            fail_all(s, DD_ERR_CUDA);
            return;
        }
        if (!done.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            const double t = now_s();
            for (int k : done) {
                Request& r = s->reqs[s->slot_req[k]];
                fill(s->h_st[k], r.ev, M, &r.res);
                r.status = s->h_st[k].status;
                r.state = 2;
                r.done_t = t;
                s->slot_req[k] = 0;
            }
            s->cv.notify_all();
        }
    }
}

}  // namespace

extern "C" {

double dd_serve_clock(void) { return now_s(); }

int dd_serve_start(dd_ctx* ctx, int32_t max_slots, int64_t max_events, dd_server** out) {
    if (!ctx || !out || max_slots < 0 || max_events < 1 || max_events > INT32_MAX / 2) return DD_ERR_ARG;
    dd_server* s = new (std::nothrow) dd_server();
    if (!s) return DD_ERR_OOM;
    dd::ctx_info(ctx, &s->g, &s->threads, &s->eval_blocks, &s->max_tasks, &s->pop_k, &s->qcap, &s->max_rounds);
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return DD_ERR_NO_DEVICE;
    }
    if (const dd_mlp* m = dd::ctx_warm_model(ctx)) {
        int dev = -1;
        s->has_model = dd::mlp_device_view(m, &s->model, &dev);
    }
    s->E = max_events;
    s->bins = dd::bins_of(s->g);
    s->max_chunks = (int)((max_events + dd::CHUNK - 1) / dd::CHUNK);
    if (max_slots == 0) {
        // Slots from free device memory: at most half of it, at most 64.
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete s;
            return DD_ERR_CUDA;
        }
        const size_t per = slot_bytes(s);
        size_t n = (free_b / 2) / (per ? per : 1);
        max_slots = (int32_t)(n > 64 ? 64 : n);
        if (max_slots < 1) {
            delete s;
            return DD_ERR_OOM;
        }
    }
    s->S = max_slots;
    s->slot_req.assign(s->S, 0);
    int rc = alloc_server(s);
    if (rc) {
        free_server(s);
        delete s;
        return rc;
    }
    try {
        s->up_th = std::thread(uploader, s);
    } catch (...) {
        free_server(s);
        delete s;
        return DD_ERR_OOM;
    }
    try {
        s->th = std::thread(loop, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->up_stop = true;
            s->cv.notify_all();
        }
        s->up_th.join();
        free_server(s);
        delete s;
        return DD_ERR_OOM;
    }
    *out = s;
    return DD_OK;
}

int dd_serve_slots(dd_server* s, int32_t* slots, int64_t* max_events) {
    if (!s) return DD_ERR_ARG;
    if (slots) *slots = s->S;
    if (max_events) *max_events = s->E;
    return DD_OK;
}

int dd_serve_submit(dd_server* s, const dd_events* ev, const dd_window_params* p, double arrival_s,
                    uint64_t* ticket) {
    if (!s || !ev || !p || !ticket) return DD_ERR_ARG;
    if (ev->n < 0 || (ev->n > 0 && (!ev->x || !ev->y || !ev->t))) return DD_ERR_ARG;
    if (s->g.planes > 1 && ev->n > 0 && !ev->p) return DD_ERR_ARG;
    if (!std::isfinite(ev->tau) || !(ev->tau > 0.0f) || !std::isfinite(ev->t0)) return DD_ERR_ARG;
    auto d_ok = [&](float D) {
        if (!std::isfinite(D)) return false;
        const double dt = (double)D * (double)ev->tau;
        return dt <= 0.75 && dt >= -64.0;
    };
    if (!d_ok(p->D_lo) || !d_ok(p->D_hi) || !(p->D_lo < p->D_hi) || !(p->tol_D >= 0.0f) || !std::isfinite(p->tol_D) ||
        !(p->gamma >= 0.0) || !std::isfinite(p->gamma))
        return DD_ERR_ARG;
    if (p->warm == DD_WARM_GIVEN) {
        if (!std::isfinite(p->D_warm) || !std::isfinite(p->w_warm) || !(p->w_warm > 0.0f)) return DD_ERR_ARG;
    } else if (p->warm == DD_WARM_MODEL) {
        if (!s->has_model) return DD_ERR_ARG;
    } else if (p->warm != DD_WARM_NONE) {
        return DD_ERR_ARG;
    }
    if (ev->n > s->E) return DD_ERR_CAPACITY;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return DD_ERR_ARG;
    if (s->failed) return s->failed;
    Request r;
    r.ev = *ev;
    r.p = *p;
    r.arrival = arrival_s >= 0.0 ? arrival_s : now_s();
    const uint64_t id = s->next_ticket++;
    s->reqs[id] = r;
    s->waiting.push_back(id);
    *ticket = id;
    s->cv.notify_all();
    return DD_OK;
}

static int take(dd_server* s, uint64_t ticket, dd_result* out, double* latency_s, bool wait) {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return DD_ERR_ARG;
    if (wait) s->cv.wait(lk, [&] { return it->second.state == 2; });
    if (it->second.state != 2) return DD_PENDING;
    const int st = it->second.status;
    if (out) *out = it->second.res;
    if (latency_s) *latency_s = it->second.done_t - it->second.arrival;
    s->reqs.erase(it);
    return st;
}

int dd_serve_cancel(dd_server* s, uint64_t ticket) {
    if (!s) return DD_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return DD_ERR_ARG;
    Request& r = it->second;
    if (r.state == 0) {                           // not admitted: dropped
        for (auto q = s->waiting.begin(); q != s->waiting.end(); ++q)
            if (*q == ticket) {
                s->waiting.erase(q);
                break;
            }
        std::memset(&r.res, 0, sizeof(r.res));
        r.res.status = DD_ERR_CANCELLED;
        r.status = DD_ERR_CANCELLED;
        r.state = 2;
        r.done_t = now_s();
        s->cv.notify_all();
    } else if (r.state == 1 && !r.cancel) {       // running: the serving thread stops it
        r.cancel = true;
        s->cancel_pending = true;
        s->cv.notify_all();
    }
    return DD_OK;
}

int dd_serve_poll(dd_server* s, uint64_t ticket, dd_result* out, double* latency_s) {
    if (!s) return DD_ERR_ARG;
    return take(s, ticket, out, latency_s, false);
}

int dd_serve_wait(dd_server* s, uint64_t ticket, dd_result* out, double* latency_s) {
    if (!s) return DD_ERR_ARG;
    return take(s, ticket, out, latency_s, true);
}

int dd_serve_stats(dd_server* s, int64_t* rounds, int64_t* admitted, int64_t* peak_busy) {
    if (!s) return DD_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (rounds) *rounds = s->rounds;
    if (admitted) *admitted = s->admitted;
    if (peak_busy) *peak_busy = s->peak_busy;
    return DD_OK;
}

int dd_serve_stop(dd_server* s) {
    if (!s) return DD_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->up_stop = true;
        s->cv.notify_all();
    }
    if (s->up_th.joinable()) s->up_th.join();
    const int rc = s->failed;
    free_server(s);
    delete s;
    return rc;
}

}  // extern "C"
