// GB300 (sm_103a) kernels of the exact divergence estimator:
//   ingest   validate + counting-sort events by row (once per window)
//   eval     point contrast (Eqs. 11-13) and interval bound (Eqs. 14-19) on
//            shared-memory IWE tiles, one (task, row band) per block
//   keys     per-task integer keys from the per-tile partial sums
//   control  Algorithm 1 on the device: incumbent, priority queue, pruning,
//            next batch of tasks
//
// Arithmetic contract.  The warp is evaluated in IEEE binary32 with one
// rounding per operation, in this order, with no contraction into FMA:
//     g = 1/(1 - D*tau);  s = (1 - D*t)*g;  cell = floor((FOE + d*s) + 1/2).
// __fmul_rn/__fadd_rn/__fsub_rn/__frcp_rn are never contracted.  The pixel a
// warped event lands in is an integer decided by that arithmetic, and all
// later work (counts, sums of squares, keys) is exact integer arithmetic, so
// results do not depend on thread or block order.
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <cfloat>

namespace dd {

// ------------------------------------------------------------ warp (Eq. 11)

__device__ __forceinline__ float warp_g(float D, float tau) {
    return __frcp_rn(__fsub_rn(1.0f, __fmul_rn(D, tau)));
}
__device__ __forceinline__ float warp_s(float D, float t, float g) {
    return __fmul_rn(__fsub_rn(1.0f, __fmul_rn(D, t)), g);
}
// Eq. (12), pixel u covers [u - 1/2, u + 1/2).
__device__ __forceinline__ int cell_of(float foe, float d, float s) {
    return __float2int_rd(__fadd_rn(__fadd_rn(foe, __fmul_rn(d, s)), 0.5f));
}
__device__ __forceinline__ float fmin_t(float a, float b) { return a < b ? a : b; }
__device__ __forceinline__ float fmax_t(float a, float b) { return a < b ? b : a; }

// Relative widening of the per-event scale range (binary32 s(D) is monotone
// in D only up to a few ulps; 2^-19 covers the error for D*tau <= 3/4).
__device__ constexpr float WIDEN_DN = 1.0f - 0x1p-19f;
__device__ constexpr float WIDEN_UP = 1.0f + 0x1p-19f;
// Half a pixel plus a 2^-8 px margin (above the cell rounding error).
__device__ constexpr float HALF_PLUS = 0.50390625f;

// ------------------------------------------------------------------ ingest

constexpr int INGEST_THREADS = 512;
constexpr int MAX_ROWS = 4096;

__device__ __forceinline__ bool event_ok(int xi, int yi, float ti, float tr, float tau, int W, int H) {
    return isfinite(ti) && tr >= 0.0f && tr <= tau && xi >= 0 && xi < W && yi >= 0 && yi < H;
}

__global__ void __launch_bounds__(INGEST_THREADS) k_row_hist(const int16_t* __restrict__ x,
                                                             const int16_t* __restrict__ y,
                                                             const float* __restrict__ t, int64_t n,
                                                             float t0, float tau, int W, int H,
                                                             int32_t* row_count, int32_t* err) {
    __shared__ int32_t h[MAX_ROWS];
    for (int r = threadIdx.x; r < H; r += blockDim.x) h[r] = 0;
    __syncthreads();
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int xi = x[i], yi = y[i];
        float ti = t[i];
        float tr = __fsub_rn(ti, t0);
        if (!event_ok(xi, yi, ti, tr, tau, W, H)) { bad = 1; continue; }
        atomicAdd(&h[yi], 1);
    }
    if (bad) atomicOr(err, 1);
    __syncthreads();
    for (int r = threadIdx.x; r < H; r += blockDim.x)
        if (h[r]) atomicAdd(&row_count[r], h[r]);
}

// Exclusive scan of the row counts (H <= 4096) by one block.
__global__ void __launch_bounds__(1024) k_row_scan(const int32_t* row_count, int H, int32_t* row_off,
                                                   int32_t* cursor) {
    __shared__ int32_t wsum[32];
    const int per = (H + 1023) / 1024;
    int base = threadIdx.x * per;
    int local[4];
    int tot = 0;
    for (int k = 0; k < per; k++) {
        int r = base + k;
        local[k] = r < H ? row_count[r] : 0;
        tot += local[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = tot;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int s = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int excl = v - tot + (wid ? wsum[wid - 1] : 0);
    for (int k = 0; k < per; k++) {
        int r = base + k;
        if (r < H) { row_off[r] = excl; cursor[r] = excl; }
        excl += local[k];
    }
    if (threadIdx.x == 1023) row_off[H] = excl;
}

// Scatter each valid event to its row segment; a block reserves one range
// per row, so the global atomics are per (block, row).
__global__ void __launch_bounds__(INGEST_THREADS) k_row_scatter(const int16_t* __restrict__ x,
                                                                const int16_t* __restrict__ y,
                                                                const float* __restrict__ t, int64_t n,
                                                                float t0, float tau, int W, int H,
                                                                int32_t* cursor, Ev* __restrict__ out,
                                                                int64_t chunk) {
    __shared__ int32_t h[MAX_ROWS];
    __shared__ int32_t base[MAX_ROWS];
    int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int r = threadIdx.x; r < H; r += blockDim.x) h[r] = 0;
    __syncthreads();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        int xi = x[i], yi = y[i];
        float ti = t[i];
        if (event_ok(xi, yi, ti, __fsub_rn(ti, t0), tau, W, H)) atomicAdd(&h[yi], 1);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < H; r += blockDim.x) {
        base[r] = h[r] ? atomicAdd(&cursor[r], h[r]) : 0;
        h[r] = 0;
    }
    __syncthreads();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        int xi = x[i], yi = y[i];
        float ti = t[i];
        float tr = __fsub_rn(ti, t0);
        if (!event_ok(xi, yi, ti, tr, tau, W, H)) continue;
        int pos = base[yi] + atomicAdd(&h[yi], 1);
        Ev e;
        e.x = (int16_t)xi;
        e.y = (int16_t)yi;
        e.t = tr;
        out[pos] = e;
    }
}

cudaError_t launch_ingest(const Geom& g, const int16_t* x, const int16_t* y, const float* t, int64_t n,
                          float t0, float tau, Ev* out, int32_t* row_count, int32_t* row_off,
                          int32_t* cursor, int32_t* err, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(row_count, 0, sizeof(int32_t) * g.H, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        int64_t nb = (n + INGEST_THREADS - 1) / INGEST_THREADS;
        int blocks = (int)(nb < 304 ? nb : 304);
        k_row_hist<<<blocks, INGEST_THREADS, 0, s>>>(x, y, t, n, t0, tau, g.W, g.H, row_count, err);
    }
    k_row_scan<<<1, 1024, 0, s>>>(row_count, g.H, row_off, cursor);
    if (n > 0) {
        int64_t chunk = 8192;
        int blocks = (int)((n + chunk - 1) / chunk);
        k_row_scatter<<<blocks, INGEST_THREADS, 0, s>>>(x, y, t, n, t0, tau, g.W, g.H, cursor, out, chunk);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------- eval

// Rows of events that can reach tile rows [y0, y1) for any scale in
// [smin, smax] (a superset; binary64 with margins).
__device__ void tile_event_range(const Geom& g, const int32_t* row_off, double smin, double smax, int y0,
                                 int y1, int& e0, int& e1) {
    double A = (double)y0 - 0.5625 - (double)g.fy;
    double B = (double)(y1 - 1) + 0.5625 - (double)g.fy;
    double dylo = A >= 0.0 ? A / smax : A / smin;
    double dyhi = B >= 0.0 ? B / smin : B / smax;
    double rl = floor((double)g.fy + dylo) - 1.0, rh = ceil((double)g.fy + dyhi) + 1.0;
    int rlo = rl < 0.0 ? 0 : (rl > g.H - 1 ? g.H - 1 : (int)rl);
    int rhi = rh < 0.0 ? 0 : (rh > g.H - 1 ? g.H - 1 : (int)rh);
    e0 = row_off[rlo];
    e1 = row_off[rhi + 1];
}

// Eq. (16) for one event restricted to tile rows [y0, y1): walk the cells of
// the major axis (larger |offset|, ties to x); for major cell k the widened
// s-range where the major coordinate rounds to k gives the run of minor
// cells.  Identical per-cell arithmetic to a whole-frame walk; the tile only
// skips major cells whose runs cannot reach its rows.
__device__ __forceinline__ void segment_tile(const Geom& g, float dx, float dy, float sa, float sb, int xa,
                                             int ya, int xb, int yb, int y0, int y1, uint32_t* tile) {
    const int W = g.W, H = g.H;
    if (dx == 0.0f && dy == 0.0f) {
        if (xa >= 0 && xa < W && ya >= y0 && ya < y1) atomicAdd(&tile[(ya - y0) * W + xa], 1u);
        return;
    }
    if (fabsf(dx) >= fabsf(dy)) {
        int k0 = min(xa, xb), k1 = max(xa, xb);
        k0 = max(k0, 0);
        k1 = min(k1, W - 1);
        if (dy == 0.0f) {
            if (ya < y0 || ya >= y1) return;
        } else {
            float r = __frcp_rn(dy);
            float e0 = __fsub_rn(__fsub_rn((float)y0, g.fy), HALF_PLUS);
            float e1 = __fadd_rn(__fsub_rn((float)(y1 - 1), g.fy), HALF_PLUS);
            float b0 = __fmul_rn(e0, r), b1 = __fmul_rn(e1, r);
            float lo = fmax_t(fmin_t(b0, b1), sa), hi = fmin_t(fmax_t(b0, b1), sb);
            if (lo > hi) return;
            int c0 = cell_of(g.fx, dx, lo), c1 = cell_of(g.fx, dx, hi);
            k0 = max(k0, min(c0, c1) - 2);
            k1 = min(k1, max(c0, c1) + 2);
        }
        float rm = __frcp_rn(dx);
        for (int k = k0; k <= k1; k++) {
            float e = __fsub_rn((float)k, g.fx);
            float b1 = __fmul_rn(__fsub_rn(e, HALF_PLUS), rm), b2 = __fmul_rn(__fadd_rn(e, HALF_PLUS), rm);
            float lo = b1 < b2 ? b1 : b2, hi = b1 < b2 ? b2 : b1;
            if (lo < sa) lo = sa;
            if (hi > sb) hi = sb;
            if (lo > hi) continue;
            int j1 = cell_of(g.fy, dy, lo), j2 = cell_of(g.fy, dy, hi);
            int j0 = max(max(min(j1, j2), 0), y0), jn = min(min(max(j1, j2), H - 1), y1 - 1);
            for (int j = j0; j <= jn; j++) atomicAdd(&tile[(j - y0) * W + k], 1u);
        }
    } else {
        int k0 = max(max(min(ya, yb), 0), y0), k1 = min(min(max(ya, yb), H - 1), y1 - 1);
        float rm = __frcp_rn(dy);
        for (int k = k0; k <= k1; k++) {
            float e = __fsub_rn((float)k, g.fy);
            float b1 = __fmul_rn(__fsub_rn(e, HALF_PLUS), rm), b2 = __fmul_rn(__fadd_rn(e, HALF_PLUS), rm);
            float lo = b1 < b2 ? b1 : b2, hi = b1 < b2 ? b2 : b1;
            if (lo < sa) lo = sa;
            if (hi > sb) hi = sb;
            if (lo > hi) continue;
            int j1 = cell_of(g.fx, dx, lo), j2 = cell_of(g.fx, dx, hi);
            int j0 = max(min(j1, j2), 0), jn = min(max(j1, j2), W - 1);
            uint32_t* row = tile + (k - y0) * W;
            for (int j = j0; j <= jn; j++) atomicAdd(&row[j], 1u);
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One (task, tile) item: zero the tile, scatter the events that can reach its
// rows, reduce.  Writes part[task * n_tiles + tile].
__device__ __forceinline__ void eval_item(const Geom& g, const Ev* __restrict__ ev,
                                          const int32_t* __restrict__ row_off, const Task& tk, int task, int ti,
                                          float tau, Partial* __restrict__ part, uint32_t* __restrict__ iwe_out,
                                          uint32_t* tile, unsigned long long (*red)[32], int* erange) {
    const int y0 = ti * g.band_rows, y1 = min(y0 + g.band_rows, g.H);
    const int W = g.W, cnt = (y1 - y0) * W;

    for (int i = threadIdx.x; i < cnt; i += blockDim.x) tile[i] = 0u;
    if (threadIdx.x == 0) {
        double gl = 1.0 / (1.0 - (double)tk.D_lo * (double)tau);
        double gh = 1.0 / (1.0 - (double)tk.D_hi * (double)tau);
        double smin = fmin(fmin(gl, gh), 1.0) * (1.0 - 1e-5), smax = fmax(fmax(gl, gh), 1.0) * (1.0 + 1e-5);
        int e0, e1;
        tile_event_range(g, row_off, smin, smax, y0, y1, e0, e1);
        erange[0] = e0;
        erange[1] = e1;
    }
    __syncthreads();
    const int e0 = erange[0], e1 = erange[1];
    unsigned long long full = 0;

    if (tk.kind == TASK_POINT) {
        const float D = tk.D_lo, gg = warp_g(D, tau);
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const Ev v = ev[e];
            const float dx = __fsub_rn((float)v.x, g.fx), dy = __fsub_rn((float)v.y, g.fy);
            const float s = warp_s(D, v.t, gg);
            const int ux = cell_of(g.fx, dx, s), uy = cell_of(g.fy, dy, s);
            if ((unsigned)ux < (unsigned)W && uy >= y0 && uy < y1) atomicAdd(&tile[(uy - y0) * W + ux], 1u);
        }
    } else {
        const float Dl = tk.D_lo, Dh = tk.D_hi, gl = warp_g(Dl, tau), gh = warp_g(Dh, tau);
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const Ev v = ev[e];
            const float dx = __fsub_rn((float)v.x, g.fx), dy = __fsub_rn((float)v.y, g.fy);
            const float sl = warp_s(Dl, v.t, gl), sh = warp_s(Dh, v.t, gh);
            const float sa = __fmul_rn(sl < sh ? sl : sh, WIDEN_DN);
            const float sb = __fmul_rn(sl < sh ? sh : sl, WIDEN_UP);
            const int xa = cell_of(g.fx, dx, sa), ya = cell_of(g.fy, dy, sa);
            const int xb = cell_of(g.fx, dx, sb), yb = cell_of(g.fy, dy, sb);
            // Eq. (19): both end cells in the frame; counted by the tile of row ya.
            if (xa >= 0 && xa < W && ya >= 0 && ya < g.H && xb >= 0 && xb < W && yb >= 0 && yb < g.H &&
                ya >= y0 && ya < y1)
                full++;
            segment_tile(g, dx, dy, sa, sb, xa, ya, xb, yb, y0, y1, tile);
        }
    }
    __syncthreads();

    unsigned long long S = 0, C = 0;
    uint32_t* out = iwe_out ? iwe_out + (size_t)task * W * g.H + (size_t)y0 * W : nullptr;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const unsigned long long v = tile[i];
        S += v * v;
        C += v;
        if (out) out[i] = (uint32_t)v;
    }
    S = warp_sum(S);
    C = warp_sum(C);
    full = warp_sum(full);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][wid] = S; red[1][wid] = C; red[2][wid] = full; }
    __syncthreads();
    if (wid == 0) {
        S = lane < nw ? red[0][lane] : 0;
        C = lane < nw ? red[1][lane] : 0;
        full = lane < nw ? red[2][lane] : 0;
        S = warp_sum(S);
        C = warp_sum(C);
        full = warp_sum(full);
        if (lane == 0) {
            Partial p;
            p.S = S;
            p.cells = C;
            p.full = full;
            part[task * g.n_tiles + ti] = p;
        }
    }
}

// IWE evaluation of a task list.  With `work` (an item counter that is zero
// at launch), a grid of resident blocks takes (task, tile) items in turn,
// the tasks queued last (a round's bound tasks) first.  Without it, block b
// evaluates item b.  A finished search launches nothing.
__global__ void __launch_bounds__(1024) k_eval(Geom g, const Ev* __restrict__ ev,
                                               const int32_t* __restrict__ row_off,
                                               const Task* __restrict__ tasks, const int32_t* n_tasks_dev,
                                               int32_t n_tasks_host, float tau, Partial* __restrict__ part,
                                               uint32_t* __restrict__ iwe_out, const SolveState* st,
                                               int32_t* work) {
    extern __shared__ uint32_t tile[];
    __shared__ unsigned long long red[3][32];
    __shared__ int erange[2];
    __shared__ int s_item;
    if (st && st->phase == PH_DONE) return;
    const int n_tasks = n_tasks_dev ? *n_tasks_dev : n_tasks_host;
    if (st) tau = st->tau;                       // a solve keeps its tau in the state
    const int n_items = n_tasks * g.n_tiles;
    if (!work) {
        const int task = blockIdx.x / g.n_tiles;
        if (task >= n_tasks) return;
        eval_item(g, ev, row_off, tasks[task], task, blockIdx.x - task * g.n_tiles, tau, part, iwe_out, tile, red,
                  erange);
        return;
    }
    for (;;) {
        __syncthreads();                          // the previous item's readers are done
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int task = n_tasks - 1 - item / g.n_tiles;
        eval_item(g, ev, row_off, tasks[task], task, item % g.n_tiles, tau, part, iwe_out, tile, red, erange);
    }
}

int eval_resident_blocks(const Geom& g, int threads) {
    int per_sm = 0, dev = 0, sms = 0;
    size_t smem = (size_t)g.band_rows * g.W * sizeof(uint32_t);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval, threads, smem) != cudaSuccess) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return per_sm * sms;
}

// The dynamic shared-memory limit is a per-function attribute shared by all
// contexts: only ever raise it.
cudaError_t eval_smem_setup(const Geom& g) {
    static int current = 0;
    int bytes = g.band_rows * g.W * (int)sizeof(uint32_t);
    if (bytes <= current) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_eval(const Geom& g, const Ev* ev, const int32_t* row_off, const Task* tasks,
                        const int32_t* n_tasks_dev, int32_t n_tasks_max, float tau, Partial* part,
                        uint32_t* iwe_out, const SolveState* st, int threads, cudaStream_t s, int32_t* work,
                        int grid_blocks) {
    if (n_tasks_max <= 0) return cudaSuccess;
    size_t smem = (size_t)g.band_rows * g.W * sizeof(uint32_t);
    int items = n_tasks_max * g.n_tiles;
    int grid = work && grid_blocks > 0 && grid_blocks < items ? grid_blocks : items;
    k_eval<<<grid, threads, smem, s>>>(g, ev, row_off, tasks, n_tasks_dev, n_tasks_max, tau, part, iwe_out, st,
                                       work);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- keys

// Eq. (13) / Eq. (14) in integer form: K = M*S - N^2 with N = N_in for a
// point and N = N_full for a bound.
__device__ __forceinline__ i128 key_of(int64_t M, unsigned long long S, unsigned long long N) {
    return (i128)M * (i128)S - (i128)N * (i128)N;
}

__global__ void k_keys(Geom g, const Task* tasks, int32_t n_tasks, const Partial* part, i128* key,
                       unsigned long long* S_out, unsigned long long* C_out, unsigned long long* F_out) {
    const int t = blockIdx.x;
    if (t >= n_tasks) return;
    unsigned long long S = 0, C = 0, F = 0;
    for (int i = threadIdx.x; i < g.n_tiles; i += 32) {
        const Partial p = part[t * g.n_tiles + i];
        S += p.S;
        C += p.cells;
        F += p.full;
    }
    S = warp_sum(S);
    C = warp_sum(C);
    F = warp_sum(F);
    if (threadIdx.x == 0) {
        const int64_t M = (int64_t)g.W * g.H;
        const unsigned long long N = tasks[t].kind == TASK_POINT ? C : F;
        key[t] = key_of(M, S, N);
        S_out[t] = S;
        C_out[t] = C;
        F_out[t] = F;
    }
}

cudaError_t launch_keys(const Geom& g, const Task* tasks, int32_t n_tasks, const Partial* part, i128* key,
                        unsigned long long* S, unsigned long long* cells, unsigned long long* full,
                        cudaStream_t s) {
    if (n_tasks <= 0) return cudaSuccess;
    k_keys<<<n_tasks, 32, 0, s>>>(g, tasks, n_tasks, part, key, S, cells, full);
    return cudaGetLastError();
}

// ------------------------------------------------------------- Algorithm 1

__device__ __forceinline__ float centre(float lo, float hi) {
    return __fadd_rn(lo, __fmul_rn(0.5f, __fsub_rn(hi, lo)));
}

__global__ void k_init(SolveState* st, Task* tasks, int64_t M, float D_lo, float D_hi, float tol, float tau,
                       i128 gamma_K, int32_t K_pop, int32_t qcap, int64_t max_rounds, int32_t trace_cap,
                       int32_t* work) {
    if (threadIdx.x != 0) return;
    *work = 0;
    st->gamma_K = gamma_K;
    st->M = M;
    st->max_rounds = max_rounds;
    st->D_lo = D_lo;
    st->D_hi = D_hi;
    st->tol = tol;
    st->tau = tau;
    st->K_pop = K_pop;
    st->qcap = qcap;
    st->trace_cap = trace_cap;
    st->K_hat = 0;
    st->leaf_max = 0;
    st->stop_kb = 0;
    st->D_hat = centre(D_lo, D_hi);               // incumbent = centre of the domain
    st->phase = PH_INIT;
    st->status = DD_OK;
    st->n_pop = 0;
    st->q_n = 0;
    st->q_start = 0;
    st->q_cur = 0;
    st->have_leaf = 0;
    st->have_stop = 0;
    st->nodes_expanded = st->point_evals = st->bound_evals = st->cells = st->bcells = 0;
    st->rounds = st->max_queue = st->trace_len = 0;
    Task a, b;
    a.D_lo = a.D_hi = st->D_hat;
    a.kind = TASK_POINT;
    a.pad = 0;
    b.D_lo = D_lo;                                // bound of the domain (queued first)
    b.D_hi = D_hi;
    b.kind = TASK_BOUND;
    b.pad = 0;
    tasks[0] = a;
    tasks[1] = b;
    st->n_tasks = 2;
}

cudaError_t launch_init(SolveState* st, Task* tasks, int64_t M, float D_lo, float D_hi, float tol, float tau,
                        i128 gamma_K, int32_t K_pop, int32_t qcap, int64_t max_rounds, int32_t trace_cap,
                        int32_t* work, cudaStream_t s) {
    k_init<<<1, 32, 0, s>>>(st, tasks, M, D_lo, D_hi, tol, tau, gamma_K, K_pop, qcap, max_rounds, trace_cap, work);
    return cudaGetLastError();
}

// Priority order of the queue: larger Kbar first, ties to the smaller D_lo.
// Distinct queued intervals have distinct D_lo, so the order is total.
__device__ __forceinline__ bool better(const Node& a, const Node& b) {
    return a.kb > b.kb || (a.kb == b.kb && a.lo < b.lo);
}

// Number of entries of the sorted array q[0..n) that come before e.
__device__ __forceinline__ int rank_in(const Node* q, int n, const Node& e) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (better(q[mid], e)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int CTL_THREADS = 256;

// One block per search.  Consumes the keys of the round just evaluated
// (Algorithm 1: incumbent update, leaves, child bounds and their insertion),
// then dequeues the next batch (dequeue and gap test) and writes its tasks,
// or finishes.  The queue is kept sorted in priority order in one of two
// buffers: insertion is a parallel merge into the other buffer, a dequeue
// takes a prefix.
__global__ void __launch_bounds__(CTL_THREADS) k_control(Geom g, SolveState* st, Node* qa, Node* qb, Task* tasks,
                                                        const Partial* part, const int32_t* err, TraceRec* trace,
                                                        cudaGraphConditionalHandle loop, int32_t use_loop,
                                                        int32_t* work) {
    __shared__ i128 key[3 * MAX_POP];
    __shared__ unsigned long long cells[3 * MAX_POP];
    __shared__ Node kids[2 * MAX_POP + 1];
    __shared__ Node sorted_kids[2 * MAX_POP + 1];
    __shared__ int s_nk, s_stop;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (st->phase == PH_DONE) {
        if (use_loop && tid == 0) cudaGraphSetConditional(loop, 0);
        return;
    }
    if (tid == 0) *work = 0;                      // the next evaluation starts at item 0
    const int64_t M = st->M;
    const int n_tasks = st->n_tasks;

    for (int t = wid; t < n_tasks; t += nw) {
        unsigned long long S = 0, C = 0, F = 0;
        for (int i = lane; i < g.n_tiles; i += 32) {
            const Partial p = part[t * g.n_tiles + i];
            S += p.S;
            C += p.cells;
            F += p.full;
        }
        S = warp_sum(S);
        C = warp_sum(C);
        F = warp_sum(F);
        if (lane == 0) {
            key[t] = key_of(M, S, tasks[t].kind == TASK_POINT ? C : F);
            cells[t] = C;
        }
    }
    __syncthreads();

    if (tid == 0) {
        int stop = 0, nk = 0;
        if (*err) {
            st->status = DD_ERR_ARG;
            stop = 1;
        } else if (st->phase == PH_INIT) {
            st->K_hat = key[0];
            st->point_evals = 1;
            st->bound_evals = 1;
            st->cells = (int64_t)(cells[0] + cells[1]);
            st->bcells = (int64_t)cells[1];
            Node root;
            root.lo = st->D_lo;
            root.hi = st->D_hi;
            root.pad0 = root.pad1 = 0;
            root.kb = key[1];
            kids[nk++] = root;                    // the domain is queued unconditionally
            st->phase = PH_RUN;
        } else {
            const int np = st->n_pop;
            i128 K_hat = st->K_hat;
            for (int j = 0; j < np; j++) {        // incumbent update, dequeue order
                const Popped& p = st->pop[j];
                const i128 kc = key[p.t_point];
                st->nodes_expanded++;
                st->point_evals++;
                st->cells += (int64_t)cells[p.t_point];
                if (kc >= K_hat) {
                    K_hat = kc;
                    st->D_hat = p.c;
                }
            }
            st->K_hat = K_hat;
            for (int j = 0; j < np; j++) {        // leaves and child bounds
                const Popped& p = st->pop[j];
                if (st->trace_len < st->trace_cap && trace) {
                    TraceRec r;
                    r.D_lo = p.lo;
                    r.D_hi = p.hi;
                    r.D_c = p.c;
                    r.leaf = p.leaf;
                    r.Kbar = p.kb;
                    r.K_c = key[p.t_point];
                    trace[st->trace_len] = r;
                }
                st->trace_len++;
                if (p.leaf) {
                    if (!st->have_leaf || p.kb > st->leaf_max) st->leaf_max = p.kb;
                    st->have_leaf = 1;
                    continue;
                }
                st->bound_evals += 2;
                st->cells += (int64_t)(cells[p.t_left] + cells[p.t_right]);
                st->bcells += (int64_t)(cells[p.t_left] + cells[p.t_right]);
                for (int side = 0; side < 2; side++) {
                    const i128 kb = key[side ? p.t_right : p.t_left];
                    if (kb >= K_hat) {            // insertion test, end-of-round incumbent
                        Node nd;
                        nd.lo = side ? p.c : p.lo;
                        nd.hi = side ? p.hi : p.c;
                        nd.pad0 = nd.pad1 = 0;
                        nd.kb = kb;
                        kids[nk++] = nd;
                    }
                }
            }
        }
        if (!stop && st->q_n + nk > st->qcap) {
            st->status = DD_ERR_QUEUE_OVERFLOW;
            stop = 1;
        }
        s_nk = nk;
        s_stop = stop;
    }
    __syncthreads();
    const int nk = s_nk;
    int stop = s_stop;

    if (!stop) {
        // sort the new children, then merge them with the queued intervals
        for (int i = tid; i < nk; i += blockDim.x) {
            int r = 0;
            for (int j = 0; j < nk; j++) r += better(kids[j], kids[i]);
            sorted_kids[r] = kids[i];
        }
        __syncthreads();
        const Node* src = (st->q_cur ? qb : qa) + st->q_start;
        Node* dst = st->q_cur ? qa : qb;
        const int a = st->q_n;
        for (int i = tid; i < a; i += blockDim.x) {
            const Node e = src[i];
            dst[i + rank_in(sorted_kids, nk, e)] = e;
        }
        for (int j = tid; j < nk; j += blockDim.x) {
            const Node e = sorted_kids[j];
            dst[j + rank_in(src, a, e)] = e;
        }
        __syncthreads();
        if (tid == 0) {
            st->q_cur ^= 1;
            st->q_start = 0;
            st->q_n = a + nk;
            if (st->q_n > st->max_queue) st->max_queue = st->q_n;
        }
        __syncthreads();
    }

    if (tid == 0) {
        const Node* q = st->q_cur ? qb : qa;
        int np = 0;
        if (!stop) {                              // dequeue up to K_pop intervals
            const i128 K0 = st->K_hat, gK = st->gamma_K;
            while (np < st->K_pop && np < st->q_n) {
                const Node nd = q[np];
                if (nd.kb - K0 <= gK) {           // gap test
                    if (np == 0) {
                        st->have_stop = 1;
                        st->stop_kb = nd.kb;
                    }
                    break;
                }
                Popped& p = st->pop[np];
                p.lo = nd.lo;
                p.hi = nd.hi;
                p.kb = nd.kb;
                np++;
            }
            st->q_start = np;
            st->q_n -= np;
        }
        if (stop || np == 0) {
            i128 top = st->K_hat;
            if (st->have_leaf && st->leaf_max > top) top = st->leaf_max;
            if (st->have_stop && st->stop_kb > top) top = st->stop_kb;
            st->stop_kb = top - st->K_hat;        // the certificate gap_K
            st->n_pop = 0;
            st->n_tasks = 0;
            st->phase = PH_DONE;
        } else {
            st->rounds++;
            int nt = np;
            for (int j = 0; j < np; j++) {        // centre and bisection
                Popped& p = st->pop[j];
                p.c = centre(p.lo, p.hi);
                const float w = __fsub_rn(p.hi, p.lo);
                p.leaf = !(w > st->tol) || !(p.c > p.lo) || !(p.c < p.hi);
                p.t_point = j;
                Task a;
                a.D_lo = a.D_hi = p.c;
                a.kind = TASK_POINT;
                a.pad = 0;
                tasks[j] = a;
                if (!p.leaf) {
                    p.t_left = nt;
                    p.t_right = nt + 1;
                    Task l, r;
                    l.D_lo = p.lo;
                    l.D_hi = p.c;
                    l.kind = TASK_BOUND;
                    l.pad = 0;
                    r.D_lo = p.c;
                    r.D_hi = p.hi;
                    r.kind = TASK_BOUND;
                    r.pad = 0;
                    tasks[nt] = l;
                    tasks[nt + 1] = r;
                    nt += 2;
                } else {
                    p.t_left = p.t_right = -1;
                }
            }
            st->n_pop = np;
            st->n_tasks = nt;
            if (st->rounds > st->max_rounds) {
                st->status = DD_ERR_TIMEOUT;
                st->stop_kb = 0;
                st->n_tasks = 0;
                st->phase = PH_DONE;
            }
        }
        if (use_loop) cudaGraphSetConditional(loop, st->phase == PH_DONE ? 0u : 1u);
    }
}

cudaError_t launch_control(const Geom& g, SolveState* st, Node* qa, Node* qb, Task* tasks, const Partial* part,
                           const int32_t* err, TraceRec* trace, cudaGraphConditionalHandle loop, int32_t use_loop,
                           int32_t* work, cudaStream_t s) {
    k_control<<<1, CTL_THREADS, 0, s>>>(g, st, qa, qb, tasks, part, err, trace, loop, use_loop, work);
    return cudaGetLastError();
}

}  // namespace dd
