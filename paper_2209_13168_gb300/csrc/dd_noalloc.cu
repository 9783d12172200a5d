// dd_contrast_noalloc: the contrast evaluation of dd_contrast for callers that
// must not allocate device memory.  Every buffer the evaluation needs beyond
// the caller's inputs and outputs lives in one file-scope device array whose
// size is fixed at build time; this file calls no cudaMalloc or cudaFree.
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr int64_t NA_MAX_EVENTS = DD_NOALLOC_MAX_EVENTS;
constexpr int NA_MAX_ROWS = 4096;   // sort bins: time buckets x rows
constexpr int NA_MAX_TASKS = 64;     // hypotheses per kernel launch (calls are chunked)
constexpr int NA_MAX_TILES = 1024;   // row bands of one frame (at most 683 for 4096 x 4096)

// Byte offsets of the sub-buffers inside the static array (each 256-aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t OFF_EV = 0;
constexpr size_t OFF_RCP = align256(OFF_EV + sizeof(dd::Ev) * NA_MAX_EVENTS);
constexpr size_t OFF_ROW_COUNT = align256(OFF_RCP + sizeof(float2) * NA_MAX_EVENTS);
constexpr size_t OFF_ROW_OFF = align256(OFF_ROW_COUNT + sizeof(int32_t) * NA_MAX_ROWS);
constexpr size_t OFF_CURSOR = align256(OFF_ROW_OFF + sizeof(int32_t) * (NA_MAX_ROWS + 1));
constexpr size_t OFF_ERR = align256(OFF_CURSOR + sizeof(int32_t) * NA_MAX_ROWS);
constexpr size_t OFF_WIN = align256(OFF_ERR + sizeof(int32_t));
constexpr size_t OFF_CHUNKS = align256(OFF_WIN + sizeof(dd::WinIn));
constexpr size_t NA_MAX_CHUNKS = (NA_MAX_EVENTS + dd::CHUNK - 1) / dd::CHUNK;
constexpr size_t OFF_SCHED = align256(OFF_CHUNKS + sizeof(int32_t) * NA_MAX_CHUNKS);
constexpr size_t OFF_JOBS = align256(OFF_SCHED + sizeof(dd::Sched));
constexpr size_t OFF_TASKS = align256(OFF_JOBS + sizeof(dd::Job) * 2 * NA_MAX_TASKS);
constexpr size_t OFF_PART = align256(OFF_TASKS + sizeof(dd::Task) * NA_MAX_TASKS);
constexpr size_t OFF_KEYS = align256(OFF_PART + sizeof(dd::Partial) * NA_MAX_TASKS);
constexpr size_t OFF_S = align256(OFF_KEYS + sizeof(dd::i128) * NA_MAX_TASKS);
constexpr size_t OFF_C = align256(OFF_S + sizeof(unsigned long long) * NA_MAX_TASKS);
constexpr size_t OFF_F = align256(OFF_C + sizeof(unsigned long long) * NA_MAX_TASKS);
constexpr size_t SCRATCH_BYTES = align256(OFF_F + sizeof(unsigned long long) * NA_MAX_TASKS);
static_assert(SCRATCH_BYTES == DD_NOALLOC_SCRATCH_BYTES, "dd.h states the static scratch size");
static_assert(sizeof(dd::Partial) == 40 && sizeof(dd::Task) == 16 && sizeof(dd::Ev) == 16, "layout");

// The scratch itself.  In host code `g_scratch` is only a stand-in symbol:
// its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_base[NA_MAX_DEVICES] = {};

// Device address of the scratch on the current device; resolved on the first
// call per device (with that device current) and cached.
int scratch_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return DD_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DD_ERR_NO_DEVICE;
        if (!(prop.major == 10 && prop.minor == 3)) return DD_ERR_NO_DEVICE;
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return DD_ERR_CUDA;
        g_base[dev] = (unsigned char*)p;
    }
    *out = g_base[dev];
    return DD_OK;
}


}  // namespace

extern "C" int dd_contrast_noalloc(int32_t W, int32_t H, float foe_x, float foe_y, const dd_events* ev,
                                   const float* D, int32_t nD, dd_i128* K, void* stream) {
    if (W < 1 || H < 1 || W > 4096 || H > 4096) return DD_ERR_ARG;
    if (!std::isfinite(foe_x) || !std::isfinite(foe_y) || foe_x < 0.0f || foe_y < 0.0f || foe_x > (float)W ||
        foe_y > (float)H)
        return DD_ERR_ARG;
    if (!ev || !ev->device_ptrs || nD < 0 || (nD > 0 && (!D || !K))) return DD_ERR_ARG;
    if (ev->n > NA_MAX_EVENTS) return DD_ERR_CAPACITY;
    // the descriptor and domain checks of dd_contrast (polarity unused)
    if (dd::check_events(ev, 1) != DD_OK) return DD_ERR_ARG;
    for (int32_t j = 0; j < nD; j++)
        if (!dd::d_ok(D[j], ev->tau)) return DD_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_NO_DEVICE;
    unsigned char* base = nullptr;
    int rc = scratch_base(dev, &base);
    if (rc) return rc;

    dd::Geom g{};
    g.W = W;
    g.H = H;
    g.fx = foe_x;
    g.fy = foe_y;
    // Bands of about 96 KB of counts: taller than dd_create's default of
    // 40 KB, because a contrast-only call has no bound tasks to split over
    // several blocks, so fewer, taller units mean fewer candidate-run set-ups
    // per hypothesis.  The keys are exact sums and do not depend on the band.
    int rows = (int)(96 * 1024 / (4 * W));
    if (rows < 1) rows = 1;
    if (rows > H) rows = H;
    g.band_rows = rows;
    g.n_tiles = (H + rows - 1) / rows;
    g.n_tb = dd::time_buckets(H);
    g.max_splits = 1;
    g.split_target = 0;
    g.ref0 = 0;
    g.planes = 1;                                 // polarity unused (Eq. 12 as the paper writes it)
    g.plane_tiles = g.n_tiles;
    if (g.n_tiles > NA_MAX_TILES) return DD_ERR_CAPACITY;
    if (dd::eval_smem_setup(g) != cudaSuccess) return DD_ERR_CUDA;

    cudaStream_t s = (cudaStream_t)stream;
    dd::Ev* ev_sorted = (dd::Ev*)(base + OFF_EV);
    float2* rcp = (float2*)(base + OFF_RCP);
    int32_t* row_count = (int32_t*)(base + OFF_ROW_COUNT);
    int32_t* row_off = (int32_t*)(base + OFF_ROW_OFF);
    int32_t* cursor = (int32_t*)(base + OFF_CURSOR);
    int32_t* err = (int32_t*)(base + OFF_ERR);
    dd::WinIn* win = (dd::WinIn*)(base + OFF_WIN);
    int32_t* chunk_win = (int32_t*)(base + OFF_CHUNKS);
    dd::Sched* sch = (dd::Sched*)(base + OFF_SCHED);
    dd::Job* jobs = (dd::Job*)(base + OFF_JOBS);
    dd::Task* tasks = (dd::Task*)(base + OFF_TASKS);
    dd::Partial* part = (dd::Partial*)(base + OFF_PART);
    dd::i128* keys = (dd::i128*)(base + OFF_KEYS);
    unsigned long long* S = (unsigned long long*)(base + OFF_S);
    unsigned long long* C = (unsigned long long*)(base + OFF_C);
    unsigned long long* F = (unsigned long long*)(base + OFF_F);

    // The window descriptor and chunk map go in from host stack buffers; the
    // ingest clears the bin counts and the error flag itself; the tasks' sums
    // are cleared before each evaluation (and again by their reader).
    dd::WinIn h_win;
    h_win.x = ev->x;
    h_win.y = ev->y;
    h_win.t = ev->t;
    h_win.p = nullptr;
    h_win.n = ev->n;
    h_win.ev_off = 0;
    h_win.t0 = ev->t0;
    h_win.tau = ev->tau;
    h_win.chunk0 = 0;
    h_win.pad = 0;
    const int32_t n_chunks = (int32_t)((ev->n + dd::CHUNK - 1) / dd::CHUNK);
    int32_t h_chunks[NA_MAX_CHUNKS];
    for (int32_t k = 0; k < n_chunks; k++) h_chunks[k] = 0;
    if (cudaMemcpyAsync(win, &h_win, sizeof(h_win), cudaMemcpyHostToDevice, s) != cudaSuccess) return DD_ERR_CUDA;
    if (n_chunks &&
        cudaMemcpyAsync(chunk_win, h_chunks, sizeof(int32_t) * n_chunks, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DD_ERR_CUDA;
    if (dd::launch_ingest(g, win, 1, chunk_win, n_chunks, ev_sorted, rcp, row_count, row_off, cursor, err, s) !=
        cudaSuccess)
        return DD_ERR_CUDA;
    dd::EvalArgs a{};
    a.ev = ev_sorted;
    a.rcp = rcp;
    a.row_off = row_off;
    a.wins = win;
    a.tasks = tasks;
    a.task_stride = NA_MAX_TASKS;
    a.jobs = jobs;
    a.job_stride = NA_MAX_TASKS;
    a.sch = sch;
    a.part = part;
    a.iwe_out = nullptr;
    dd::Task h_tasks[NA_MAX_TASKS];
    dd::Job h_jobs[NA_MAX_TASKS];
    dd::Sched h_sch;
    dd::i128 h_keys[NA_MAX_TASKS];
    int32_t h_err = 0;
    const int grid = dd::eval_resident_blocks(g, 512);
    if (grid <= 0) return DD_ERR_CUDA;
    for (int32_t j0 = 0; j0 < nD || j0 == 0; j0 += NA_MAX_TASKS) {
        const int32_t m = nD - j0 < NA_MAX_TASKS ? nD - j0 : NA_MAX_TASKS;
        if (m > 0) {
            for (int32_t j = 0; j < m; j++) {
                h_tasks[j].D_lo = h_tasks[j].D_hi = D[j0 + j];
                h_tasks[j].kind = dd::TASK_POINT;
                h_tasks[j].splits = 1;
                h_jobs[j].win = 0;
                h_jobs[j].task = j;
                h_jobs[j].split = 0;
                h_jobs[j].splits = 1;
            }
            std::memset(&h_sch, 0, sizeof(h_sch));
            h_sch.n_jobs[0] = m;
            if (cudaMemcpyAsync(tasks, h_tasks, sizeof(dd::Task) * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(jobs, h_jobs, sizeof(dd::Job) * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(sch, &h_sch, sizeof(h_sch), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return DD_ERR_CUDA;
            if (cudaMemsetAsync(part, 0, sizeof(dd::Partial) * m, s) != cudaSuccess) return DD_ERR_CUDA;
            if (dd::launch_eval(g, a, 512, grid, s) != cudaSuccess) return DD_ERR_CUDA;
            if (dd::launch_keys(g, tasks, m, part, keys, S, C, F, s) != cudaSuccess) return DD_ERR_CUDA;
            if (cudaMemcpyAsync(h_keys, keys, sizeof(dd::i128) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return DD_ERR_CUDA;
        }
        if (cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return DD_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return DD_ERR_CUDA;
        if (h_err) return DD_ERR_ARG;
        for (int32_t j = 0; j < m; j++) {
            K[j0 + j].lo = (uint64_t)(unsigned __int128)h_keys[j];
            K[j0 + j].hi = (int64_t)(uint64_t)((unsigned __int128)h_keys[j] >> 64);
        }
        if (nD == 0) break;
    }
    return DD_OK;
}
