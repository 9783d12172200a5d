// GB300 (sm_103a) kernels of the exact divergence estimator:
//   ingest   validate + counting-sort events by (polarity plane, time bucket,
//            row), per window
//   eval     point contrast (Eqs. 11-13) and interval bound (Eqs. 14-19) on
//            shared-memory IWE tiles: a resident grid takes (job, row band)
//            units, a job being one task (or one split of it) of one window
//   keys     per-task integer keys from the per-task sums
//   control  Algorithm 1 on the device, one block per window: incumbent,
//            priority queue, pruning, the next round's jobs
//
// Arithmetic contract.  The warp is evaluated in IEEE binary32 with one
// rounding per operation, in this order, with no contraction into FMA:
//     g = 1/(1 - D*t_ref);  s = (1 - D*t)*g;  cell = floor((FOE + d*s) + 1/2),
// t_ref = tau (the window's end, the paper's warp) or 0 (its start).
// __fmul_rn/__fadd_rn/__fsub_rn/__frcp_rn are never contracted.  The pixel a
// warped event lands in is an integer decided by that arithmetic, and all
// later work (counts, sums of squares, keys) is exact integer arithmetic, so
// results do not depend on thread, block or launch order.
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <cfloat>
#include <mutex>

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

// Checked builds (-DDD_CHECKED, the stand-in for a memory checker): every
// index into a shared tile, a window's events, a split accumulator or the
// sorted-event output is tested first; an index out of range sets a bit of
// g_dd_check and the access is skipped (nothing traps).  Bits: 1 point and
// one-pixel tile cells, 2 segment tile cells, 4 event indices, 8 ingest
// positions, 16 accumulator and image cells.  Other builds compile the tests
// away.
#ifdef DD_CHECKED
__device__ unsigned int g_dd_check;
__device__ __forceinline__ bool dd_in(long long i, long long n, unsigned bit) {
    if (i >= 0 && i < n) return true;
    atomicOr(&g_dd_check, bit);
    return false;
}
#define DD_IN(i, n, bit) dd_in((long long)(i), (long long)(n), (bit))
#else
#define DD_IN(i, n, bit) true
#endif

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Inclusive prefix sum over the warp.
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// ------------------------------------------------------------------ ingest

constexpr int INGEST_THREADS = 512;
// Blocks per ingest chunk: each takes CHUNK / INGEST_SUB consecutive events,
// so that a window of a few chunks still spreads over many SMs.
constexpr int INGEST_SUB = 8;
static_assert(CHUNK % INGEST_SUB == 0, "sub-chunks tile a chunk");
constexpr int MAX_BINS = 4096;

__device__ __forceinline__ bool event_ok(int xi, int yi, float ti, float tr, float tau, int W, int H) {
    return isfinite(ti) && tr >= 0.0f && tr <= tau && xi >= 0 && xi < W && yi >= 0 && yi < H;
}

// Sort key of an event: (polarity plane, time bucket, row).  Bucket b holds
// the events with t*scale in [b, b+1) (binary32 product), scale = n_tb/tau.
__device__ __forceinline__ int event_key(const Geom& g, int yi, float tr, float bscale, int plane) {
    int b = __float2int_rd(__fmul_rn(tr, bscale));
    b = min(max(b, 0), g.n_tb - 1);
    return (plane * g.n_tb + b) * g.H + yi;
}

// Plane of event i: 1 for polarity p <= 0 when the planes are split.
__device__ __forceinline__ int plane_of(const Geom& g, const WinIn& win, int64_t i) {
    return g.planes > 1 && win.p[i] <= 0 ? 1 : 0;
}

// Events [i0, i1) of the sub-chunk that block b ingests: sub-chunk
// b % INGEST_SUB of chunk b / INGEST_SUB, within that chunk's window.
__device__ __forceinline__ void sub_chunk(const WinIn& win, int chunk, int sub, int64_t& i0, int64_t& i1) {
    constexpr int SUB_EVENTS = CHUNK / INGEST_SUB;
    i0 = min(win.n, (int64_t)(chunk - win.chunk0) * CHUNK + (int64_t)sub * SUB_EVENTS);
    i1 = min(win.n, i0 + SUB_EVENTS);
}

// Block b counts its sub-chunk of its window into a shared histogram of the
// window's bins, then adds it to the window's global counts.
__global__ void __launch_bounds__(INGEST_THREADS) k_row_hist(Geom g, const WinIn* __restrict__ wins,
                                                             const int32_t* __restrict__ chunk_win,
                                                             int32_t* row_count, int32_t* err) {
    __shared__ int32_t h[MAX_BINS];
    const int chunk = blockIdx.x / INGEST_SUB;
    const int w = chunk_win[chunk];
    const WinIn win = wins[w];
    const int bins = bins_of(g);
    const float bscale = __fdiv_rn((float)g.n_tb, win.tau);
    for (int r = threadIdx.x; r < bins; r += blockDim.x) h[r] = 0;
    __syncthreads();
    int64_t i0, i1;
    sub_chunk(win, chunk, blockIdx.x % INGEST_SUB, i0, i1);
    int bad = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int xi = win.x[i], yi = win.y[i];
        const float ti = win.t[i];
        const float tr = __fsub_rn(ti, win.t0);
        if (!event_ok(xi, yi, ti, tr, win.tau, g.W, g.H)) { bad = 1; continue; }
        atomicAdd(&h[event_key(g, yi, tr, bscale, plane_of(g, win, i))], 1);
    }
    if (bad) atomicOr(&err[w], 1);
    __syncthreads();
    int32_t* rc = row_count + (size_t)w * bins;
    for (int r = threadIdx.x; r < bins; r += blockDim.x)
        if (h[r]) atomicAdd(&rc[r], h[r]);
}

// Exclusive scan of one window's bin counts (at most 4096 bins), block = window.
__global__ void __launch_bounds__(1024) k_row_scan(int bins, const int32_t* row_count, int32_t* row_off,
                                                   int32_t* cursor) {
    __shared__ int32_t wsum[32];
    const int w = blockIdx.x;
    row_count += (size_t)w * bins;
    cursor += (size_t)w * bins;
    row_off += (size_t)w * (bins + 1);
    const int per = (bins + 1023) / 1024;
    int base = threadIdx.x * per;
    int local[4];
    int tot = 0;
    for (int k = 0; k < per; k++) {
        int r = base + k;
        local[k] = r < bins ? row_count[r] : 0;
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
        if (r < bins) { row_off[r] = excl; cursor[r] = excl; }
        excl += local[k];
    }
    if (threadIdx.x == 1023) row_off[bins] = excl;
}

// Scatter each valid event of the block's sub-chunk to its bin (offsets
// within the window); a block reserves one range per bin, so the global
// atomics are per (block, bin).  Also stores the reciprocals of the event's
// offsets from the FOE (used by the bound's cell walk).
__global__ void __launch_bounds__(INGEST_THREADS) k_row_scatter(Geom g, const WinIn* __restrict__ wins,
                                                                const int32_t* __restrict__ chunk_win,
                                                                int32_t* cursor, Ev* __restrict__ out,
                                                                float2* __restrict__ rcp) {
    __shared__ int32_t h[MAX_BINS];
    __shared__ int32_t base[MAX_BINS];
    const int chunk = blockIdx.x / INGEST_SUB;
    const int w = chunk_win[chunk];
    const WinIn win = wins[w];
    const int bins = bins_of(g);
    const float bscale = __fdiv_rn((float)g.n_tb, win.tau);
    int64_t i0, i1;
    sub_chunk(win, chunk, blockIdx.x % INGEST_SUB, i0, i1);
    int32_t* cur = cursor + (size_t)w * bins;
    Ev* o = out + win.ev_off;
    float2* rc = rcp + win.ev_off;
    for (int r = threadIdx.x; r < bins; r += blockDim.x) h[r] = 0;
    __syncthreads();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int xi = win.x[i], yi = win.y[i];
        const float ti = win.t[i];
        const float tr = __fsub_rn(ti, win.t0);
        if (event_ok(xi, yi, ti, tr, win.tau, g.W, g.H))
            atomicAdd(&h[event_key(g, yi, tr, bscale, plane_of(g, win, i))], 1);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < bins; r += blockDim.x) {
        base[r] = h[r] ? atomicAdd(&cur[r], h[r]) : 0;
        h[r] = 0;
    }
    __syncthreads();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int xi = win.x[i], yi = win.y[i];
        const float ti = win.t[i];
        const float tr = __fsub_rn(ti, win.t0);
        if (!event_ok(xi, yi, ti, tr, win.tau, g.W, g.H)) continue;
        const int key = event_key(g, yi, tr, bscale, plane_of(g, win, i));
        const int pos = base[key] + atomicAdd(&h[key], 1);
        if (!DD_IN(pos, win.n, 8u)) continue;
        Ev e;
        e.dx = __fsub_rn((float)xi, g.fx);
        e.dy = __fsub_rn((float)yi, g.fy);
        e.t = tr;
        e.pad = 0;
        o[pos] = e;
        rc[pos] = make_float2(__frcp_rn(e.dx), __frcp_rn(e.dy));
    }
}

cudaError_t launch_ingest(const Geom& g, const WinIn* wins_dev, int32_t n_windows, const int32_t* chunk_win_dev,
                          int32_t n_chunks, Ev* out, float2* rcp, int32_t* row_count, int32_t* row_off,
                          int32_t* cursor, int32_t* err, cudaStream_t s) {
    const int bins = bins_of(g);
    if (n_windows <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(row_count, 0, sizeof(int32_t) * bins * (size_t)n_windows, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(err, 0, sizeof(int32_t) * (size_t)n_windows, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)n_chunks * INGEST_SUB;
    if (n_chunks > 0) k_row_hist<<<blocks, INGEST_THREADS, 0, s>>>(g, wins_dev, chunk_win_dev, row_count, err);
    k_row_scan<<<n_windows, 1024, 0, s>>>(bins, row_count, row_off, cursor);
    if (n_chunks > 0) k_row_scatter<<<blocks, INGEST_THREADS, 0, s>>>(g, wins_dev, chunk_win_dev, cursor, out, rcp);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- eval

// Events of time bucket b that can reach tile rows [y0, y1) for D in
// [Dl, Dh]: the scale s(D, t) = (1 - D t)/(1 - D tau) is monotone in D and in
// t, so over the bucket's time range its extremes are at the four corners.
// An event at row y can reach the rows only if (y - FOE_y) s meets them for
// some s in that range; the rows that can are a contiguous range of the
// bucket's row-sorted events.  Binary32, each operation correctly rounded
// (relative error 2^-24; quotients as products with rounded reciprocals):
// every scale has relative error below 12 x 2^-24 on the domain
// -64 <= D tau <= 3/4, the bucket's time edges below 3 x 2^-24, and the row
// bounds (at most 4096 px) below 3 x 2^-24, all far under the margins: 1e-4
// relative on s, 1e-3 of a bucket in t (an event of bucket b has t bscale in
// [b (1 - 2^-24), (b + 1)(1 + 2^-24)), b < 8), 1/16 pixel on the band's
// edges.  A superset.
__device__ void bucket_event_range(const Geom& g, const int32_t* row_off, float Dl, float Dh, float tau,
                                   float bscale, int b, int y0, int y1, int& e0, int& e1) {
    const float rb = __frcp_rn(bscale);
    const float tl = fmaxf(0.0f, __fmul_rn((float)b - 1e-3f, rb));
    const float th = fminf(tau, __fmul_rn((float)b + 1.001f, rb));
    const float tref = warp_tref(g, tau);
    const float gl = __frcp_rn(1.0f - Dl * tref), gh = __frcp_rn(1.0f - Dh * tref);
    float smin = 3.0e38f, smax = -3.0e38f;
    for (int i = 0; i < 4; i++) {
        const float D = (i & 1) ? Dh : Dl, t = (i & 2) ? th : tl;
        const float s = (1.0f - D * t) * ((i & 1) ? gh : gl);
        smin = fminf(smin, s);
        smax = fmaxf(smax, s);
    }
    smin *= 1.0f - 1e-4f;
    smax *= 1.0f + 1e-4f;
    const float A = (float)y0 - 0.5625f - g.fy;
    const float B = (float)(y1 - 1) + 0.5625f - g.fy;
    const float dylo = A * __frcp_rn(A >= 0.0f ? smax : smin);
    const float dyhi = B * __frcp_rn(B >= 0.0f ? smin : smax);
    // The margins above exceed the few-ulp error of this arithmetic, and
    // rounding a bound that is off by less than a row outward to an integer
    // row never drops a row the exact bound admits.
    const float rl = floorf(g.fy + dylo), rh = ceilf(g.fy + dyhi);
    if (rh < 0.0f || rl > (float)(g.H - 1)) {
        e0 = e1 = 0;
        return;
    }
    const int rlo = rl < 0.0f ? 0 : (int)rl;
    const int rhi = rh > (float)(g.H - 1) ? g.H - 1 : (int)rh;
    e0 = row_off[b * g.H + rlo];
    e1 = row_off[b * g.H + rhi + 1];
}

// Eq. (16) for one event restricted to tile rows [y0, y1).  The segment is
// walked along its major axis (larger |offset| from the FOE, ties to x): for
// major cell k, the s-range where the major coordinate rounds to k (widened
// by 2^-8 px, clipped to [s_a, s_b]) gives a run of minor cells.  The walk is
// split into a set-up (seg_range: which major cells can reach the tile) and
// the per-major-cell work (seg_cell), so that a warp can spread the major
// cells of its events over its lanes.  The per-cell arithmetic is that of a
// whole-frame walk; the tile only skips major cells whose runs cannot reach
// its rows.
enum SegMode : int { SEG_NONE = 0, SEG_ONE = 1, SEG_X = 2, SEG_Y = 3 };

struct Seg {
    int mode, k0, count, addr;   // addr: the tile cell of SEG_ONE
    float dn, rm, sa, sb;        // minor offset, 1/major offset, scale range
};

__device__ __forceinline__ Seg seg_range(const Geom& g, float dx, float dy, float rdx, float rdy, float sa,
                                         float sb, int xa, int ya, int xb, int yb, int y0, int y1) {
    Seg s;
    s.mode = SEG_NONE;
    s.k0 = s.count = s.addr = 0;
    s.dn = s.rm = 0.0f;
    s.sa = sa;
    s.sb = sb;
    const int W = g.W, H = g.H;
    if (dx == 0.0f && dy == 0.0f) {               // on the FOE: one pixel for every D
        if (xa >= 0 && xa < W && ya >= y0 && ya < y1) {
            s.mode = SEG_ONE;
            s.count = 1;
            s.addr = (ya - y0) * tile_pitch(g) + xa;
        }
        return s;
    }
    if (fabsf(dx) >= fabsf(dy)) {
        int k0 = max(min(xa, xb), 0), k1 = min(max(xa, xb), W - 1);
        if (dy == 0.0f) {
            if (ya < y0 || ya >= y1) return s;
        } else {
            const float r = rdy;
            const float e0 = __fsub_rn(__fsub_rn((float)y0, g.fy), HALF_PLUS);
            const float e1 = __fadd_rn(__fsub_rn((float)(y1 - 1), g.fy), HALF_PLUS);
            const float b0 = __fmul_rn(e0, r), b1 = __fmul_rn(e1, r);
            const float lo = fmax_t(fmin_t(b0, b1), sa), hi = fmin_t(fmax_t(b0, b1), sb);
            if (lo > hi) return s;
            const int c0 = cell_of(g.fx, dx, lo), c1 = cell_of(g.fx, dx, hi);
            k0 = max(k0, min(c0, c1) - 2);
            k1 = min(k1, max(c0, c1) + 2);
        }
        if (k1 < k0) return s;
        s.mode = SEG_X;
        s.k0 = k0;
        s.count = k1 - k0 + 1;
        s.dn = dy;
        s.rm = rdx;
    } else {
        const int k0 = max(max(min(ya, yb), 0), y0), k1 = min(min(max(ya, yb), H - 1), y1 - 1);
        if (k1 < k0) return s;
        s.mode = SEG_Y;
        s.k0 = k0;
        s.count = k1 - k0 + 1;
        s.dn = dx;
        s.rm = rdy;
    }
    return s;
}

// One increment of a tile cell.  Sparse images (at most a few increments per
// cell): the sum of squares grows by 2v + 1 from the cell's previous count v
// and C counts increments (32 bits: callers fold it into 64 bits often
// enough that it cannot wrap).  Dense images (many increments per cell): the
// increment alone, the sums taken from the tile afterwards.  Undo: the
// decrement that takes back an earlier sparse increment of the same cell.
enum BumpMode : int { BUMP_SPARSE = 0, BUMP_DENSE = 1, BUMP_UNDO = 2 };
template <int MODE>
__device__ __forceinline__ void bump(uint32_t* cell, unsigned long long& S, uint32_t& C) {
    if (MODE == BUMP_DENSE) {
        atomicAdd(cell, 1u);
    } else if (MODE == BUMP_UNDO) {
        atomicSub(cell, 1u);
    } else {
        const uint32_t v = atomicAdd(cell, 1u);
        S += 2u * v + 1u;
        C++;
    }
}

template <int MODE>
__device__ __forceinline__ void seg_cell(const Geom& g, int mode, int k, float dn, float rm, float sa, float sb,
                                         int addr, int y0, int y1, uint32_t* tile, unsigned long long& S,
                                         uint32_t& C) {
    if (mode == SEG_ONE) {
        if (DD_IN(addr, (y1 - y0) * tile_pitch(g), 2u)) bump<MODE>(&tile[addr], S, C);
        return;
    }
    const bool major_x = mode == SEG_X;
    const float fm = major_x ? g.fx : g.fy, fn = major_x ? g.fy : g.fx;
    const float e = __fsub_rn((float)k, fm);
    const float b1 = __fmul_rn(__fsub_rn(e, HALF_PLUS), rm), b2 = __fmul_rn(__fadd_rn(e, HALF_PLUS), rm);
    float lo = b1 < b2 ? b1 : b2, hi = b1 < b2 ? b2 : b1;
    if (lo < sa) lo = sa;
    if (hi > sb) hi = sb;
    if (lo > hi) return;
    const int j1 = cell_of(fn, dn, lo), j2 = cell_of(fn, dn, hi);
    if (major_x) {
        const int j0 = max(max(min(j1, j2), 0), y0), jn = min(min(max(j1, j2), g.H - 1), y1 - 1);
        for (int j = j0; j <= jn; j++)
            if (DD_IN((j - y0) * tile_pitch(g) + k, (y1 - y0) * tile_pitch(g), 2u))
                bump<MODE>(&tile[(j - y0) * tile_pitch(g) + k], S, C);
    } else {
        const int j0 = max(min(j1, j2), 0), jn = min(max(j1, j2), g.W - 1);
        uint32_t* row = tile + (k - y0) * tile_pitch(g);
        for (int j = j0; j <= jn; j++)
            if (DD_IN((k - y0) * tile_pitch(g) + j, (y1 - y0) * tile_pitch(g), 2u)) bump<MODE>(&row[j], S, C);
    }
}

// Position-to-event cursor over a unit's candidate runs (erange: first
// event of each bucket's run, then each run's offset in the concatenation).
// Each thread visits increasing positions, so the cursor (the first
// position of the next run and the current run's offset from positions to
// event indices) only moves forward; positions stay below
// erange[MAX_TB + n_tb].
constexpr int MAX_TB = 8;    // time buckets of the event sort

struct Cursor {
    const int* erange;
    int cur_b, next_f, delta;
    __device__ __forceinline__ Cursor(const int* er, int) : erange(er), cur_b(0) {
        next_f = er[MAX_TB + 1];
        delta = er[0] - er[MAX_TB];
    }
    __device__ __forceinline__ int at(int f) {
        while (f >= next_f) {
            cur_b++;
            delta = erange[cur_b] - erange[MAX_TB + cur_b];
            next_f = erange[MAX_TB + cur_b + 1];
        }
        return f + delta;
    }
};



constexpr int QUEUE = 64;    // queued long-segment events per warp (a power of two, >= 63)
constexpr int MAX_WARPS = 16;   // warps of a k_eval block (at most 512 threads)

// Where one unit reads and writes.
struct UnitPtrs {
    const Ev* ev;                 // the window's sorted events
    const float2* rcp;
    const int32_t* row_off;       // the window's bin offsets
    Partial* part;                // the task's sums (atomic accumulation over its row bands)
    uint32_t* out;                // nullable: the task's image [H][W]
    uint32_t* acc;                // event-split jobs: the task's accumulator [H][W]
    int32_t* done;                // event-split jobs: finished splits per tile
    Partial* sums;                // event-split jobs: sums of the splits per tile
#ifdef DD_CHECKED
    int64_t n_ev;                 // the window's event count
#endif
};

// Dense bound images (bound_cells >= DENSE_CELLS): their increments skip the
// returned count and the tile's sums are taken in one pass afterwards.

// Eqs. (16) and (19) for the unit's share of events, positions [f_begin,
// total): Hbar into the tile, N_full into `full`, and (sparse) S and C.
// Per-warp rings of queued long segments (see bound_pass): QUEUE records of
// five words (event, s_a, s_b, both end cells' x, both end cells' y) per warp
// of the block, in dynamic shared memory after the tile (so a block's ring
// memory grows with its warps: 1,280 bytes per warp).
constexpr int QREC = 5;
struct SegQueue {
    int* rec;       // [warps * QUEUE][QREC]
    int cap;        // warps * QUEUE records
};

// Dynamic shared memory of a k_eval block: the band tile (rounded up to 16
// bytes) and the segment rings of its warps.
__host__ __device__ inline int eval_tile_words(const Geom& g) { return (g.band_rows * tile_pitch(g) + 3) & ~3; }
__host__ __device__ inline size_t eval_smem_bytes(const Geom& g, int threads);

template <int MODE>
__device__ __forceinline__ void bound_pass(const Geom& g, const UnitPtrs& p, const Task& tk, float tau, uint32_t* tile,
                                           SegQueue queue, int y0, int y1, int f_begin, int total, Cursor& cur,
                                           unsigned long long& S, unsigned long long& C, unsigned long long& full) {
    const int W = g.W, P = tile_pitch(g), rows = y1 - y0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float tref = warp_tref(g, tau);
    const float Dl = tk.D_lo, Dh = tk.D_hi, gl = warp_g(Dl, tref), gh = warp_g(Dh, tref);
    // The cells of up to 32 queued segments, one event per lane (`valid`,
    // with the end scales and end cells computed when it was queued): short
    // runs walked by their own lane, long runs spread over the warp as
    // (event, major cell) pairs.
    auto walk = [&](int e, bool valid, float sa, float sb, int xa, int ya, int xb, int yb) {
        uint32_t Ci = 0;
        Seg sg;
        sg.mode = SEG_NONE;
        sg.k0 = sg.count = sg.addr = 0;
        sg.dn = sg.rm = sg.sa = sg.sb = 0.0f;
        if (valid) {
            const Ev v = p.ev[e];
            const float2 r = p.rcp[e];
            sg = seg_range(g, v.dx, v.dy, r.x, r.y, sa, sb, xa, ya, xb, yb, y0, y1);
        }
        const int cmax = __reduce_max_sync(0xffffffffu, (unsigned)sg.count);
        if (cmax <= 4) {                       // short runs: each lane walks its own
            for (int i = 0; i < sg.count; i++)
                seg_cell<MODE>(g, sg.mode, sg.k0 + i, sg.dn, sg.rm, sg.sa, sg.sb, sg.addr, y0, y1, tile, S, Ci);
            C += Ci;
            return;
        }
        const int incl = warp_incl_scan(sg.count), excl = incl - sg.count;
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        for (int c0 = 0; c0 < tot; c0 += 32) {
            const int gi = c0 + lane;
            int o = 0;                            // owner: first lane whose inclusive sum exceeds gi
            for (int step = 16; step > 0; step >>= 1) {
                const int probe = __shfl_sync(0xffffffffu, incl, o + step - 1);
                if (probe <= gi) o += step;
            }
            const int om = __shfl_sync(0xffffffffu, sg.mode, o);
            const int ok = __shfl_sync(0xffffffffu, sg.k0 - excl, o);
            const int oa = __shfl_sync(0xffffffffu, sg.addr, o);
            const float odn = __shfl_sync(0xffffffffu, sg.dn, o);
            const float orm = __shfl_sync(0xffffffffu, sg.rm, o);
            const float osa = __shfl_sync(0xffffffffu, sg.sa, o);
            const float osb = __shfl_sync(0xffffffffu, sg.sb, o);
            if (gi < tot) seg_cell<MODE>(g, om, ok + gi, odn, orm, osa, osb, oa, y0, y1, tile, S, Ci);
        }
        C += Ci;
    };
    // Warps take 32 positions at a time, one event per lane.  A segment
    // within one pixel is counted at once; an event whose segment spans more
    // pixels is queued with its end scales and end cells (a ring of 64 entries
    // per warp; cells packed as two 16-bit halves, their range being under
    // 2^15 in magnitude), and every 32 queued events are walked together, so
    // the walk runs on full warps.
    const int qb = wid * QUEUE;
    int q_head = 0, q_tail = 0;
    auto take = [&](int i, int& e, float& sa, float& sb, int& xa, int& ya, int& xb, int& yb) {
        const int* r = queue.rec + QREC * (qb + (i & (QUEUE - 1)));
        e = r[0];
        sa = __int_as_float(r[1]);
        sb = __int_as_float(r[2]);
        const int px = r[3], py = r[4];
        xa = (int)(short)(px & 0xFFFF);
        xb = px >> 16;
        ya = (int)(short)(py & 0xFFFF);
        yb = py >> 16;
    };
    for (int base = f_begin + wid * 32; base < total; base += nw * 32) {
        const int f = base + lane;
        bool pend = false;
        int e = 0, xa = 0, xb = 0, ya = 0, yb = 0;
        float sa = 0.0f, sb = 0.0f;
        if (f < total) {
            e = cur.at(f);
            if (!DD_IN(e, p.n_ev, 4u)) e = 0;
            const Ev v = p.ev[e];
            const float dy = v.dy;
            const float sl = warp_s(Dl, v.t, gl), sh = warp_s(Dh, v.t, gh);
            sa = __fmul_rn(sl < sh ? sl : sh, WIDEN_DN);
            sb = __fmul_rn(sl < sh ? sh : sl, WIDEN_UP);
            ya = cell_of(g.fy, dy, sa);
            yb = cell_of(g.fy, dy, sb);
            // Every covered cell lies between the rows of the two end cells
            // (each cell coordinate is monotone in s).
            if (max(ya, yb) >= y0 && min(ya, yb) < y1) {
                const float dx = v.dx;
                xa = cell_of(g.fx, dx, sa);
                xb = cell_of(g.fx, dx, sb);
                const bool ya_here = (unsigned)(ya - y0) < (unsigned)rows;
                // Eq. (19): both end cells in the frame; counted by the tile of row ya.
                if ((unsigned)xa < (unsigned)W && (unsigned)xb < (unsigned)W && (unsigned)yb < (unsigned)g.H &&
                    ya_here)
                    full++;
                if (xa == xb && ya == yb) {
                    // Both ends in one pixel: each cell coordinate is monotone
                    // in s, so the segment covers that pixel only.
                    if ((unsigned)xa < (unsigned)W && ya_here) {
                        uint32_t Ci = 0;
                        if (DD_IN((ya - y0) * P + xa, rows * P, 1u)) bump<MODE>(&tile[(ya - y0) * P + xa], S, Ci);
                        C += Ci;
                    }
                } else if ((xa == xb && abs(ya - yb) == 1) || (ya == yb && abs(xa - xb) == 1)) {
                    // End cells side by side: one coordinate is constant and
                    // the other takes two adjacent values, so the segment
                    // covers exactly those two pixels (each counted where it
                    // lies in the frame and in this band).
                    uint32_t Ci = 0;
                    if ((unsigned)xa < (unsigned)W && ya_here && DD_IN((ya - y0) * P + xa, rows * P, 1u))
                        bump<MODE>(&tile[(ya - y0) * P + xa], S, Ci);
                    if ((unsigned)xb < (unsigned)W && (unsigned)(yb - y0) < (unsigned)rows &&
                        DD_IN((yb - y0) * P + xb, rows * P, 1u))
                        bump<MODE>(&tile[(yb - y0) * P + xb], S, Ci);
                    C += Ci;
                } else {
                    pend = true;
                }
            }
        }
        const unsigned pm = __ballot_sync(0xffffffffu, pend);
        if (pend) {
            int* r = queue.rec + QREC * (qb + ((q_tail + __popc(pm & ((1u << lane) - 1u))) & (QUEUE - 1)));
            r[0] = e;
            r[1] = __float_as_int(sa);
            r[2] = __float_as_int(sb);
            r[3] = (xa & 0xFFFF) | (xb << 16);
            r[4] = (ya & 0xFFFF) | (yb << 16);
        }
        q_tail += __popc(pm);
        if (q_tail - q_head >= 32) {
            __syncwarp();                         // the queued entries are visible to the warp
            take(q_head + lane, e, sa, sb, xa, ya, xb, yb);
            __syncwarp();                         // read before the next pass may overwrite
            q_head += 32;
            walk(e, true, sa, sb, xa, ya, xb, yb);
        }
    }
    while (q_tail > q_head) {                     // the rest of the queue
        const int n = min(32, q_tail - q_head);
        int e = 0, xa = 0, xb = 0, ya = 0, yb = 0;
        float sa = 0.0f, sb = 0.0f;
        __syncwarp();
        if (lane < n) take(q_head + lane, e, sa, sb, xa, ya, xb, yb);
        __syncwarp();
        q_head += n;
        walk(e, lane < n, sa, sb, xa, ya, xb, yb);
    }
}

// One unit: split `split` of `splits` of one task's row band `ti`.  The block
// scatters the events that can reach its rows into the shared tile.  Sparse
// images: each increment returns the cell's previous count v and the band's
// sum of squares grows by (v + 1)^2 - v^2 = 2v + 1, so the tile is only
// cleared afterwards; dense bound images: one pass over the tile takes S and
// C and clears it.  A split band is divided by rows when its bound's segments
// are short (bound_cells below SPLIT_ROWS_CELLS): split s owns rows
// [y0 + R s/splits, y0 + R (s + 1)/splits) of the band's R rows and counts the
// events that reach them in its own rows of the tile, so the splits share no
// cell.  With long segments (where every thin slice would read nearly all of
// the band's candidates) the band is divided by events instead: split s
// takes its share of the band's candidates, adds its tile into the L2
// accumulator, and each addition of u onto a count w adds (w + u)^2 - w^2 to
// S, so the splits' sums add up to the band's; the last split to finish
// clears the accumulated band.  The tile arrives zeroed and leaves zeroed.
__device__ __forceinline__ void eval_unit(const Geom& g, const UnitPtrs& p, const Task& tk, int ti, int split,
                                          int splits, float tau, uint32_t* tile, unsigned long long (*red)[32],
                                          int* erange, int* s_last, SegQueue queue) {
    // Unit ti is row band `band` of polarity plane `plane`: the plane's own
    // run of sorted events, its own image and its own counts.
    const int plane = ti >= g.plane_tiles ? 1 : 0, band = ti - plane * g.plane_tiles;
    const bool by_rows = splits > 1 && (!p.acc || bound_cells(g, tk.D_lo, tk.D_hi, tau) < SPLIT_ROWS_CELLS);
    const int b0 = band * g.band_rows, R = min(b0 + g.band_rows, g.H) - b0;
    const int y0 = by_rows ? b0 + (int)((long long)R * split / splits) : b0;
    const int y1 = by_rows ? b0 + (int)((long long)R * (split + 1) / splits) : b0 + R;
    const int32_t* row_off = p.row_off + (size_t)plane * g.n_tb * g.H;
    const size_t plane_off = (size_t)plane * g.W * g.H;
    const int W = g.W, P = tile_pitch(g), rows = y1 - y0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

    // erange[b] = first event of bucket b's candidate run; erange[MAX_TB + b] =
    // the run's offset in the concatenation of all runs (MAX_TB + n_tb: total).
    if (threadIdx.x < 32) {
        int e0 = 0, e1 = 0;
        if (lane < g.n_tb && y1 > y0)
            bucket_event_range(g, row_off, tk.D_lo, tk.D_hi, tau, __fdiv_rn((float)g.n_tb, tau), lane, y0, y1, e0,
                               e1);
        const int len = e1 - e0, incl = warp_incl_scan(len);
        if (lane < g.n_tb) {
            erange[lane] = e0;
            erange[MAX_TB + lane] = incl - len;
        }
        if (lane == g.n_tb - 1) erange[MAX_TB + g.n_tb] = incl;
    }
    __syncthreads();
    unsigned long long full = 0;
    const int all = erange[MAX_TB + g.n_tb];
    const int f_begin = by_rows ? 0 : (int)((long long)all * split / splits);
    const int total = by_rows ? all : (int)((long long)all * (split + 1) / splits);
    Cursor cur(erange, MAX_TB);

    unsigned long long S = 0, C = 0;
    bool dense = false;
    if (tk.kind == TASK_POINT) {
        const float D = tk.D_lo, gg = warp_g(D, warp_tref(g, tau));
        uint32_t Ct = 0;                          // at most one increment per event
#pragma unroll 4
        for (int f = f_begin + threadIdx.x; f < total; f += blockDim.x) {
            const int e = cur.at(f);
            if (!DD_IN(e, p.n_ev, 4u)) continue;
            const Ev v = p.ev[e];
            const float s = warp_s(D, v.t, gg);
            const int uy = cell_of(g.fy, v.dy, s);
            if ((unsigned)(uy - y0) >= (unsigned)rows) continue;
            const int ux = cell_of(g.fx, v.dx, s);
            if ((unsigned)ux < (unsigned)W && DD_IN((uy - y0) * P + ux, rows * P, 1u))
                bump<BUMP_SPARSE>(&tile[(uy - y0) * P + ux], S, Ct);
        }
        C = Ct;
    } else {
        dense = bound_cells(g, tk.D_lo, tk.D_hi, tau) >= DENSE_CELLS;
        if (dense)
            bound_pass<BUMP_DENSE>(g, p, tk, tau, tile, queue, y0, y1, f_begin, total, cur, S, C, full);
        else
            bound_pass<BUMP_SPARSE>(g, p, tk, tau, tile, queue, y0, y1, f_begin, total, cur, S, C, full);
    }
    __syncthreads();

    uint32_t* out = p.out ? p.out + plane_off + (size_t)y0 * W : nullptr;
    unsigned long long Cl = C;
    // Tile rows have pitch P (odd), frame rows pitch W: warps take rows, lanes
    // take columns.
    if (splits == 1 || by_rows) {
        if (out) {
            if (dense) S = Cl = 0;
            for (int r = wid; r < rows; r += nw)
                for (int c = lane; c < W; c += 32) {
                    const uint32_t v = tile[r * P + c];
                    if (DD_IN(r * W + c, rows * W, 16u)) out[r * W + c] = v;
                    tile[r * P + c] = 0u;
                    if (dense) {
                        S += (unsigned long long)v * v;
                        Cl += v;
                    }
                }
        } else {
            // The band's rows are contiguous in the tile (the padding column
            // of an odd pitch stays zero): 16-byte words, then the tail.
            const int words = rows * P, quads = words >> 2;
            uint4* t4 = reinterpret_cast<uint4*>(tile);
            if (dense) {
                S = Cl = 0;
                for (int i = threadIdx.x; i < quads; i += blockDim.x) {
                    const uint4 v = t4[i];
                    t4[i] = make_uint4(0u, 0u, 0u, 0u);
                    S += (unsigned long long)v.x * v.x + (unsigned long long)v.y * v.y +
                         (unsigned long long)v.z * v.z + (unsigned long long)v.w * v.w;
                    Cl += (unsigned long long)v.x + v.y + v.z + v.w;
                }
                for (int i = 4 * quads + threadIdx.x; i < words; i += blockDim.x) {
                    const uint32_t v = tile[i];
                    tile[i] = 0u;
                    S += (unsigned long long)v * v;
                    Cl += v;
                }
            } else {
                for (int i = threadIdx.x; i < quads; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
                for (int i = 4 * quads + threadIdx.x; i < words; i += blockDim.x) tile[i] = 0u;
            }
        }
    } else {
        uint32_t* acc = p.acc + plane_off + (size_t)y0 * W;
        // Splits of one band finish together: each starts its pass at its own
        // row so that they add into different words at a time.
        const int rot = (int)((long long)rows * split / splits);
        S = Cl = 0;
        // Four columns per lane at a time: their additions are issued
        // before any returned count is used, so the L2 round trips overlap.
        constexpr int MERGE_COLS = 4;
        for (int q = wid; q < rows; q += nw) {
            const int r = q + rot < rows ? q + rot : q + rot - rows;
            for (int c0 = lane; c0 < W; c0 += 32 * MERGE_COLS) {
                uint32_t v[MERGE_COLS], w[MERGE_COLS];
#pragma unroll
                for (int k = 0; k < MERGE_COLS; k++) {
                    const int c = c0 + 32 * k;
                    v[k] = c < W ? tile[r * P + c] : 0u;
                }
#pragma unroll
                for (int k = 0; k < MERGE_COLS; k++) {
                    const int c = c0 + 32 * k;
                    w[k] = 0u;
                    if (v[k]) {
                        tile[r * P + c] = 0u;
                        if (DD_IN(r * W + c, rows * W, 16u)) w[k] = atomicAdd(&acc[r * W + c], v[k]);
                        else v[k] = 0u;
                    }
                }
#pragma unroll
                for (int k = 0; k < MERGE_COLS; k++) {
                    S += (2ull * w[k] + v[k]) * v[k];
                    Cl += v[k];
                }
            }
        }
        __threadfence();                          // this thread's additions, before the count below
        S = warp_sum(S);
        Cl = warp_sum(Cl);
        full = warp_sum(full);
        if (lane == 0) {
            red[0][wid] = S;
            red[1][wid] = Cl;
            red[2][wid] = full;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0, f = 0;
            for (int w = 0; w < nw; w++) {
                a += red[0][w];
                b += red[1][w];
                f += red[2][w];
            }
            atomicAdd(&p.sums[ti].S, a);
            atomicAdd(&p.sums[ti].cells[0], b);
            if (f) atomicAdd(&p.sums[ti].full[0], f);
            __threadfence();
            *s_last = atomicAdd(&p.done[ti], 1) == splits - 1;
        }
        __syncthreads();
        if (!*s_last) return;                     // another split finishes the band
        __threadfence();                          // every split's additions are visible now
        for (int i = threadIdx.x; i < rows * W; i += blockDim.x) {
            if (out) out[i] = __ldcg(&acc[i]);
            acc[i] = 0u;
        }
        if (threadIdx.x == 0) {
            const unsigned long long qS = atomicExch(&p.sums[ti].S, 0ull);
            const unsigned long long qC = atomicExch(&p.sums[ti].cells[0], 0ull);
            const unsigned long long qF = atomicExch(&p.sums[ti].full[0], 0ull);
            p.done[ti] = 0;
            if (qS) atomicAdd(&p.part->S, qS);
            if (qC) atomicAdd(&p.part->cells[plane], qC);
            if (qF) atomicAdd(&p.part->full[plane], qF);
        }
        return;
    }
    // Each warp adds its share of the band's sums to the task's.
    S = warp_sum(S);
    const unsigned long long C64 = warp_sum(Cl);
    full = warp_sum(full);
    if (lane == 0) {
        if (S) atomicAdd(&p.part->S, S);
        if (C64) atomicAdd(&p.part->cells[plane], C64);
        if (full) atomicAdd(&p.part->full[plane], full);
    }
}

// The bound's work for one event (Eqs. 16 and 19 restricted to the tile rows
// [y0, y1)), as bound_pass does it, with the event's own lane walking its
// segment: from its offsets (dx, dy) and its binary32 scales at the
// interval's ends (sl, sh), the widened scale range, the end cells, N_full
// into F and the covered cells.  BUMP_UNDO takes back exactly the increments
// an earlier BUMP_SPARSE call made for the same event and interval.
template <int MODE>
__device__ __forceinline__ void bound_event(const Geom& g, const UnitPtrs& p, int e, float dx, float dy, float sl,
                                            float sh, int y0, int y1, uint32_t* tile, unsigned long long& S,
                                            uint32_t& C, uint32_t& F) {
    const int W = g.W, P = tile_pitch(g), rows = y1 - y0;
    const float sa = __fmul_rn(sl < sh ? sl : sh, WIDEN_DN);
    const float sb = __fmul_rn(sl < sh ? sh : sl, WIDEN_UP);
    const int ya = cell_of(g.fy, dy, sa), yb = cell_of(g.fy, dy, sb);
    if (max(ya, yb) < y0 || min(ya, yb) >= y1) return;
    const int xa = cell_of(g.fx, dx, sa), xb = cell_of(g.fx, dx, sb);
    const bool ya_here = (unsigned)(ya - y0) < (unsigned)rows;
    if (MODE != BUMP_UNDO && (unsigned)xa < (unsigned)W && (unsigned)xb < (unsigned)W && (unsigned)yb < (unsigned)g.H &&
        ya_here)
        F++;
    if (xa == xb && ya == yb) {
        if ((unsigned)xa < (unsigned)W && ya_here && DD_IN((ya - y0) * P + xa, rows * P, 1u))
            bump<MODE>(&tile[(ya - y0) * P + xa], S, C);
    } else if ((xa == xb && abs(ya - yb) == 1) || (ya == yb && abs(xa - xb) == 1)) {
        if ((unsigned)xa < (unsigned)W && ya_here && DD_IN((ya - y0) * P + xa, rows * P, 1u))
            bump<MODE>(&tile[(ya - y0) * P + xa], S, C);
        if ((unsigned)xb < (unsigned)W && (unsigned)(yb - y0) < (unsigned)rows && DD_IN((yb - y0) * P + xb, rows * P, 1u))
            bump<MODE>(&tile[(yb - y0) * P + xb], S, C);
    } else {
        const float2 r = p.rcp[e];
        const Seg sg = seg_range(g, dx, dy, r.x, r.y, sa, sb, xa, ya, xb, yb, y0, y1);
        for (int i = 0; i < sg.count; i++)
            seg_cell<MODE>(g, sg.mode, sg.k0 + i, sg.dn, sg.rm, sg.sa, sg.sb, sg.addr, y0, y1, tile, S, C);
    }
}

// The contrast's work for one event (Eqs. 11-12) restricted to the tile rows,
// from its offsets and its binary32 scale.
template <int MODE>
__device__ __forceinline__ void point_event(const Geom& g, float dx, float dy, float sc, int y0, int y1,
                                            uint32_t* tile, unsigned long long& S, uint32_t& C) {
    const int rows = y1 - y0, P = tile_pitch(g);
    const int uy = cell_of(g.fy, dy, sc);
    if ((unsigned)(uy - y0) >= (unsigned)rows) return;
    const int ux = cell_of(g.fx, dx, sc);
    if ((unsigned)ux < (unsigned)g.W && DD_IN((uy - y0) * P + ux, rows * P, 1u))
        bump<MODE>(&tile[(uy - y0) * P + ux], S, C);
}


// One fused unit: the three tasks of one expanded interval [lo, hi] with
// centre c -- the contrast at c (Eqs. 11-13) and the bounds over [lo, c] and
// [c, hi] (Eqs. 14-19) -- on one row band, with one pass over the events.
// Per event, the range [RN(min(s_lo, s_c, s_hi)(1 - 2^-19)),
// RN(max(s_lo, s_c, s_hi)(1 + 2^-19))] of its binary32 scales at lo, c and hi
// (computed as the tasks compute them) contains every scale the three tasks
// use: s_c itself and the widened ends of both halves (rounding is
// monotone).  Each cell coordinate is monotone in s, so when both ends of
// that range fall in one pixel, every task puts the event in that pixel and
// nowhere else: a stable event, counted once into the tile for all three (its
// increments give a common sum of squares S_C and count N_C, which is also
// each bound's N_full share).  The other events are listed as unstable; each
// task in turn adds its own increments for them on top of the common counts,
// each increment returning the cell's previous count v, so that the task's
// sum of squares is S_C + sum(2v + 1); the centre's and the left half's
// increments are taken back before the next task.  The sums, and so the keys,
// are those of three separate passes.  A band with more unstable events than
// the list holds runs as three ordinary units instead.
__device__ void eval_fused_unit(const Geom& g, const UnitPtrs& p, const Task& tp, const Task& tl, const Task& tr,
                                Partial* part_p, Partial* part_l, Partial* part_r, int ti, float tau, uint32_t* tile,
                                unsigned long long (*red)[32], int* erange, int* s_n, int* s_last, SegQueue queue) {
    const int plane = ti >= g.plane_tiles ? 1 : 0, band = ti - plane * g.plane_tiles;
    const int y0 = band * g.band_rows, y1 = min(y0 + g.band_rows, g.H);
    const int32_t* row_off = p.row_off + (size_t)plane * g.n_tb * g.H;
    const int W = g.W, P = tile_pitch(g), rows = y1 - y0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float lo = tl.D_lo, c = tp.D_lo, hi = tr.D_hi;
    if (threadIdx.x < 32) {
        int e0 = 0, e1 = 0;
        if (lane < g.n_tb)
            bucket_event_range(g, row_off, lo, hi, tau, __fdiv_rn((float)g.n_tb, tau), lane, y0, y1, e0, e1);
        const int len = e1 - e0, incl = warp_incl_scan(len);
        if (lane < g.n_tb) {
            erange[lane] = e0;
            erange[MAX_TB + lane] = incl - len;
        }
        if (lane == g.n_tb - 1) erange[MAX_TB + g.n_tb] = incl;
        if (lane == 0) *s_n = 0;
    }
    __syncthreads();
    const int total = erange[MAX_TB + g.n_tb];
    Cursor cur(erange, MAX_TB);
    const float tref = warp_tref(g, tau);
    const float glo = warp_g(lo, tref), gc = warp_g(c, tref), ghi = warp_g(hi, tref);
    int* list = queue.rec;                        // unstable events (the segment rings' memory)
    const int list_cap = QREC * queue.cap;

    // Pass over the candidates: stable events into the tile, the rest listed.
    unsigned long long SC = 0;
    uint32_t NC = 0;
    for (int base = wid * 32; base < total; base += nw * 32) {
        const int f = base + lane;
        bool uns = false;
        int e = 0;
        if (f < total) {
            e = cur.at(f);
            if (!DD_IN(e, p.n_ev, 4u)) e = 0;
            const Ev v = p.ev[e];
            const float a = warp_s(lo, v.t, glo), b = warp_s(c, v.t, gc), d = warp_s(hi, v.t, ghi);
            const float wa = __fmul_rn(fmin_t(fmin_t(a, b), d), WIDEN_DN);
            const float wb = __fmul_rn(fmax_t(fmax_t(a, b), d), WIDEN_UP);
            const int ya = cell_of(g.fy, v.dy, wa), yb = cell_of(g.fy, v.dy, wb);
            if (max(ya, yb) >= y0 && min(ya, yb) < y1) {
                const int xa = cell_of(g.fx, v.dx, wa), xb = cell_of(g.fx, v.dx, wb);
                if (xa == xb && ya == yb) {
                    if ((unsigned)xa < (unsigned)W && DD_IN((ya - y0) * P + xa, rows * P, 1u))
                        bump<BUMP_SPARSE>(&tile[(ya - y0) * P + xa], SC, NC);
                } else {
                    uns = true;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, uns);
        if (m) {
            int at = 0;
            if (lane == 0) at = atomicAdd(s_n, __popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            const int pos = at + __popc(m & ((1u << lane) - 1u));
            if (uns && pos < list_cap) list[pos] = e;
        }
    }
    __syncthreads();
    const int n = *s_n;
    if (n > list_cap) {                           // too many unstable events: three ordinary units
        const int words = rows * P;
        for (int i = threadIdx.x; i < words; i += blockDim.x) tile[i] = 0u;
        __syncthreads();
        for (int k = 0; k < 3; k++) {
            UnitPtrs q = p;
            q.part = k == 0 ? part_p : (k == 1 ? part_l : part_r);
            const Task tk = k == 0 ? tp : (k == 1 ? tl : tr);
            eval_unit(g, q, tk, ti, 0, 1, tau, tile, red, erange, s_last, queue);
            __syncthreads();
        }
        return;
    }
    // Each task's own increments for the unstable events, on top of the
    // common counts: the centre, then the left half, then the right half.  A
    // thread's first listed event stays in registers (offsets and its three
    // scales) through the five passes; further ones are read again.
    unsigned long long Sp = 0, Sl = 0, Sr = 0, Sx = 0;
    uint32_t Cp = 0, Cl = 0, Cr = 0, Fl = 0, Fr = 0, Cx = 0, Fx = 0;
    int e1 = -1;
    float ex = 0.0f, ey = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    if ((int)threadIdx.x < n) {
        e1 = list[threadIdx.x];
        const Ev v = p.ev[e1];
        ex = v.dx;
        ey = v.dy;
        s1 = warp_s(lo, v.t, glo);
        s2 = warp_s(c, v.t, gc);
        s3 = warp_s(hi, v.t, ghi);
    }
    auto each = [&](auto&& f) {
        if (e1 >= 0) f(e1, ex, ey, s1, s2, s3);
        for (int i = threadIdx.x + blockDim.x; i < n; i += blockDim.x) {
            const int e = list[i];
            const Ev v = p.ev[e];
            f(e, v.dx, v.dy, warp_s(lo, v.t, glo), warp_s(c, v.t, gc), warp_s(hi, v.t, ghi));
        }
    };
    each([&](int, float dx, float dy, float, float b, float) {
        point_event<BUMP_SPARSE>(g, dx, dy, b, y0, y1, tile, Sp, Cp);
    });
    __syncthreads();
    each([&](int, float dx, float dy, float, float b, float) {
        point_event<BUMP_UNDO>(g, dx, dy, b, y0, y1, tile, Sx, Cx);
    });
    __syncthreads();
    each([&](int e, float dx, float dy, float a, float b, float) {
        bound_event<BUMP_SPARSE>(g, p, e, dx, dy, a, b, y0, y1, tile, Sl, Cl, Fl);
    });
    __syncthreads();
    each([&](int e, float dx, float dy, float a, float b, float) {
        bound_event<BUMP_UNDO>(g, p, e, dx, dy, a, b, y0, y1, tile, Sx, Cx, Fx);
    });
    __syncthreads();
    each([&](int e, float dx, float dy, float, float b, float d) {
        bound_event<BUMP_SPARSE>(g, p, e, dx, dy, b, d, y0, y1, tile, Sr, Cr, Fr);
    });
    __syncthreads();

    // The tile leaves zeroed (its padding column stays zero): 16-byte words,
    // then the tail.
    {
        const int words = rows * P, quads = words >> 2;
        uint4* t4 = reinterpret_cast<uint4*>(tile);
        for (int i = threadIdx.x; i < quads; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = 4 * quads + threadIdx.x; i < words; i += blockDim.x) tile[i] = 0u;
    }
    // Sums of the three tasks: per warp, then per block (in the list's memory).
    unsigned long long* wsum = reinterpret_cast<unsigned long long*>(queue.rec);   // [8][MAX_WARPS]
    auto put = [&](int k, unsigned long long x) {
        x = warp_sum(x);
        if (lane == 0) wsum[k * MAX_WARPS + wid] = x;
    };
    put(0, SC + Sp);
    put(1, (unsigned long long)NC + Cp);
    put(2, SC + Sl);
    put(3, (unsigned long long)NC + Cl);
    put(4, (unsigned long long)NC + Fl);
    put(5, SC + Sr);
    put(6, (unsigned long long)NC + Cr);
    put(7, (unsigned long long)NC + Fr);
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        unsigned long long t = 0;
        for (int w = 0; w < nw; w++) t += wsum[k * MAX_WARPS + w];
        // k: 0 centre S, 1 centre N_in, then S, cells, N_full of the left (2-4) and right (5-7) halves
        Partial* q = k < 2 ? part_p : (k < 5 ? part_l : part_r);
        const int f = k < 2 ? k : (k < 5 ? k - 2 : k - 5);
        unsigned long long* dst = f == 0 ? &q->S : (f == 1 ? &q->cells[plane] : &q->full[plane]);
        if (t) atomicAdd(dst, t);
    }
}

constexpr int Q_STAGE = 256;   // queued intervals staged in shared memory for the merge

// Shared memory of one control step (one block of k_control per window).
struct __align__(16) CtlShared {
    SolveState s;
    i128 key[3 * MAX_POP];
    unsigned long long cells[3 * MAX_POP];
    Node kids[2 * MAX_POP + 1];
    Node sorted_kids[2 * MAX_POP + 1];
    Node q_stage[Q_STAGE];
    Node q_head[MAX_POP];               // the merged queue's first entries, for the dequeue
    float2 bound_iv[3 * MAX_POP];       // the next round's bound tasks' intervals
    int16_t t_fuse[3 * MAX_POP];        // per next-round task: 0 own jobs, -1 part of a fused
                                        // job, k > 0 the centre of a fused job (left half k - 1)
    int8_t t_dense[3 * MAX_POP];        // per next-round task: a dense bound that may be split
    int16_t t_jobs[3 * MAX_POP];        // per next-round task, in job order: its number of jobs
    int s_nk, s_stop;
};


__host__ __device__ inline size_t eval_smem_bytes(const Geom& g, int threads) {
    return sizeof(uint32_t) * (size_t)eval_tile_words(g) + sizeof(int) * (size_t)QREC * QUEUE * (threads / 32);
}

// IWE evaluation of the round's job list.  A grid of resident blocks takes
// units (job, row band) from a counter; block 0 clears the other parity's
// list and counter for the control blocks of this round.
__global__ void __launch_bounds__(512, 3) k_eval(Geom g, EvalArgs a) {
    extern __shared__ __align__(16) uint32_t tile[];
    __shared__ unsigned long long red[3][32];
    __shared__ int erange[2 * MAX_TB + 1];
    __shared__ int s_unit, s_last, s_n;
    Sched* sch = a.sch;
    const int par = sch->round & 1;
    const int n_units = sch->n_jobs[par] * g.n_tiles;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sch->n_jobs[par ^ 1] = 0;
        sch->work[par ^ 1] = 0;
    }
    if (n_units == 0) return;
    int32_t* work = &sch->work[par];
    const Job* jobs = a.jobs + (size_t)par * a.job_stride;
    const int tile_words = g.band_rows * tile_pitch(g);
    SegQueue queue;
    queue.rec = reinterpret_cast<int*>(tile + eval_tile_words(g));
    queue.cap = (int)(blockDim.x >> 5) * QUEUE;
    const int bins1 = bins_of(g) + 1;
    const size_t task_cells = (size_t)g.planes * g.W * g.H;
    // Block b starts with unit b; later units come from the counter, which
    // numbers them from gridDim.x on.  The counter is asked when a unit
    // starts and its answer stored only when the unit ends, so no warp waits
    // for it; the unit's own barriers order every thread's read of s_unit
    // before that store.
    if (threadIdx.x == 0) s_unit = blockIdx.x;
    for (int i = threadIdx.x; i < tile_words; i += blockDim.x) tile[i] = 0u;
    __syncthreads();
    for (;;) {
        const int u = s_unit;
        if (u >= n_units) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(work, 1);
        const int j = u / g.n_tiles, ti = u - j * g.n_tiles;
        const Job jb = jobs[j];
        const int64_t ev_off = a.wins[jb.win].ev_off;
        const float tau = a.wins[jb.win].tau;
        const Task* wt = a.tasks + (size_t)jb.win * a.task_stride;
        const Task tk = wt[jb.task];
        UnitPtrs p;
        p.ev = a.ev + ev_off;
        p.rcp = a.rcp + ev_off;
#ifdef DD_CHECKED
        p.n_ev = a.wins[jb.win].n;
#endif
        p.row_off = a.row_off + (size_t)jb.win * bins1;
        p.part = a.part + ((size_t)jb.win * a.task_stride + jb.task);
        p.out = a.iwe_out ? a.iwe_out + (size_t)jb.task * task_cells : nullptr;
        p.acc = a.mg.acc ? a.mg.acc + (size_t)jb.task * task_cells : nullptr;
        p.done = a.mg.done ? a.mg.done + (size_t)jb.task * g.n_tiles : nullptr;
        p.sums = a.mg.sums ? a.mg.sums + (size_t)jb.task * g.n_tiles : nullptr;
        if (jb.splits < 0) {                      // one expanded interval: its three tasks together
            Partial* wp = a.part + (size_t)jb.win * a.task_stride;
            eval_fused_unit(g, p, tk, wt[jb.split], wt[jb.split + 1], wp + jb.task, wp + jb.split,
                            wp + jb.split + 1, ti, tau, tile, red, erange, &s_n, &s_last, queue);
        } else {
            eval_unit(g, p, tk, ti, jb.split, max(1, jb.splits), tau, tile, red, erange, &s_last, queue);
        }
        if (threadIdx.x == 0) s_unit = gridDim.x + next;
        __syncthreads();                          // the unit is done; s_unit is set
    }
}

// The checked-build error word (always 0 in other builds); reset clears it.
cudaError_t check_flags(uint32_t* flags, int32_t* checked, bool reset) {
#ifdef DD_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_dd_check, sizeof(uint32_t));
    if (e == cudaSuccess && reset) {
        const uint32_t zero = 0;
        e = cudaMemcpyToSymbol(g_dd_check, &zero, sizeof(uint32_t));
    }
    *checked = 1;
    return e;
#else
    (void)reset;
    *flags = 0;
    *checked = 0;
    return cudaSuccess;
#endif
}

int eval_resident_blocks(const Geom& g, int threads) {
    int per_sm = 0, dev = 0, sms = 0;
    const size_t smem = eval_smem_bytes(g, threads);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval, threads, smem) != cudaSuccess) return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return per_sm * sms;
}

cudaError_t launch_eval(const Geom& g, const EvalArgs& a, int threads, int grid_blocks, cudaStream_t s) {
    if (grid_blocks <= 0) return cudaErrorInvalidValue;
    k_eval<<<grid_blocks, threads, eval_smem_bytes(g, threads), s>>>(g, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- keys

__global__ void k_keys(Geom g, const Task* tasks, int32_t n_tasks, Partial* part, i128* key,
                       unsigned long long* S_out, unsigned long long* C_out, unsigned long long* F_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tasks) return;
    const Partial p = part[t];
    part[t] = Partial{};                          // cleared for the next evaluation
    const int64_t M = (int64_t)g.W * g.H;
    key[t] = partial_key(M, p, tasks[t].kind == TASK_POINT);
    S_out[t] = p.S;
    C_out[t] = p.cells[0] + p.cells[1];
    F_out[t] = p.full[0] + p.full[1];
}

cudaError_t launch_keys(const Geom& g, const Task* tasks, int32_t n_tasks, Partial* part, i128* key,
                        unsigned long long* S, unsigned long long* cells, unsigned long long* full,
                        cudaStream_t s) {
    if (n_tasks <= 0) return cudaSuccess;
    k_keys<<<(n_tasks + 63) / 64, 64, 0, s>>>(g, tasks, n_tasks, part, key, S, cells, full);
    return cudaGetLastError();
}

__device__ __forceinline__ float centre(float lo, float hi) {
    return __fadd_rn(lo, __fmul_rn(0.5f, __fsub_rn(hi, lo)));
}

// One block per window w0 + b: the search state, the first tasks (the centre
// of the domain and the bound of the domain) and their jobs in the list the
// next evaluation reads.  `sharers`: the searches that share the rounds
// (their bound tasks split to fill 1/sharers of the grid; 0: never split).
__global__ void k_init(Geom g, int32_t sharers, int32_t w0, SolveState* st_all, Task* tasks_all,
                       int32_t task_stride, Partial* part_all, const WinIn* wins, const WinParams* params,
                       Job* jobs_all, int32_t job_stride, Sched* sch, int32_t K_pop, int32_t qcap,
                       int64_t max_rounds, int32_t trace_cap) {
    const int w = w0 + blockIdx.x;
    for (int i = threadIdx.x; i < task_stride; i += blockDim.x)   // the window's task sums start at zero
        part_all[(size_t)w * task_stride + i] = Partial{};
    if (threadIdx.x != 0) return;
    const int par = sch->round & 1;
    Job* jobs = jobs_all + (size_t)par * job_stride;
    SolveState* st = st_all + w;
    Task* tasks = tasks_all + (size_t)w * task_stride;
    const WinParams pr = params[w];
    const float tau = wins[w].tau;
    st->gamma_K = pr.gamma_K;
    st->M = (int64_t)g.W * g.H;
    st->max_rounds = max_rounds;
    st->D_lo = pr.D_lo;
    st->D_hi = pr.D_hi;
    st->tol = pr.tol;
    st->tau = tau;
    st->K_pop = K_pop;
    st->qcap = qcap;
    st->trace_cap = trace_cap;
    st->K_hat = 0;
    st->leaf_max = 0;
    st->stop_kb = 0;
    st->warm = pr.warm;
    st->D_warm = 0.0f;
    st->w_warm = 0.0f;
    // The pieces the domain enters the queue as: the domain itself, or with
    // a warm start the pieces of positive width cut at guess -/+ half-width.
    float cut[4] = {pr.D_lo, pr.D_hi, pr.D_hi, pr.D_hi};
    int n_cut = 2;
    if (pr.warm) {
        float d = pr.D_warm;                      // the guess, clamped into the domain
        if (!(d >= pr.D_lo)) d = pr.D_lo;
        if (d > pr.D_hi) d = pr.D_hi;
        float a = __fsub_rn(d, pr.w_warm), b = __fadd_rn(d, pr.w_warm);
        if (!(a >= pr.D_lo)) a = pr.D_lo;
        if (!(b <= pr.D_hi)) b = pr.D_hi;
        cut[1] = a;
        cut[2] = b;
        n_cut = 4;
        st->D_hat = d;                            // incumbent = the guess
        st->D_warm = d;
        st->w_warm = pr.w_warm;
    } else {
        st->D_hat = centre(pr.D_lo, pr.D_hi);     // incumbent = centre of the domain
    }
    st->phase = PH_INIT;
    st->status = DD_OK;
    st->cancel = 0;
    st->n_pop = 0;
    st->q_n = 0;
    st->q_start = 0;
    st->q_cur = 0;
    st->have_leaf = 0;
    st->have_stop = 0;
    st->nodes_expanded = st->point_evals = st->bound_evals = st->cells = st->bcells = 0;
    st->rounds = st->max_queue = st->trace_len = 0;
    Task a;
    a.D_lo = a.D_hi = st->D_hat;
    a.kind = TASK_POINT;
    a.splits = 1;
    tasks[0] = a;
    int nt = 1, n_jobs = 1;
    int n_pieces = 0, n_dense = 0, rank = 0;
    for (int i = 0; i + 1 < n_cut; i++)
        if (cut[i] < cut[i + 1]) {
            n_pieces++;
            n_dense += bound_cells(g, cut[i], cut[i + 1], tau) >= DENSE_CELLS;
        }
    for (int i = 0; i + 1 < n_cut; i++) {
        if (!(cut[i] < cut[i + 1])) continue;
        Task b;                                   // bound of one piece
        b.D_lo = cut[i];
        b.D_hi = cut[i + 1];
        b.kind = TASK_BOUND;
        const bool dense = bound_cells(g, b.D_lo, b.D_hi, tau) >= DENSE_CELLS;
        b.splits = sharers > 0 && dense ? fill_splits(g, g.split_target / sharers, (1 + n_pieces) * g.n_tiles,
                                                      n_dense, rank++)
                                        : 1;
        tasks[nt++] = b;
        n_jobs += b.splits;
    }
    st->n_tasks = nt;
    const int base = atomicAdd(&sch->n_jobs[par], n_jobs);
    int o = base;
    for (int t = 1; t < nt; t++)                  // bounds first (heavier)
        for (int s = 0; s < tasks[t].splits; s++) {
            Job j;
            j.win = w;
            j.task = t;
            j.split = s;
            j.splits = tasks[t].splits;
            jobs[o++] = j;
        }
    Job j;
    j.win = w;
    j.task = 0;
    j.split = 0;
    j.splits = 1;
    jobs[o] = j;
}

cudaError_t launch_init(const Geom& g, int32_t n_windows, SolveState* st, Task* tasks, int32_t task_stride,
                        Partial* part, const WinIn* wins, const WinParams* params, Job* jobs, int32_t job_stride,
                        Sched* sch, int32_t K_pop, int32_t qcap, int64_t max_rounds, int32_t trace_cap,
                        cudaStream_t s, int32_t w0, int32_t sharers) {
    if (sharers < 0) sharers = n_windows;
    k_init<<<n_windows, 32, 0, s>>>(g, sharers, w0, st, tasks, task_stride, part, wins, params, jobs, job_stride,
                                    sch, K_pop, qcap, max_rounds, trace_cap);
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

__device__ __forceinline__ i128 shfl_i128(i128 v, int src) {
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return (i128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}

__device__ __forceinline__ i128 warp_max_i128(i128 v) {
    for (int o = 16; o > 0; o >>= 1) {
        const i128 w = shfl_i128(v, threadIdx.x ^ o);
        if (w > v) v = w;
    }
    return v;
}

// One block per window.  Consumes the keys of the round just evaluated
// (Algorithm 1: incumbent update, leaves, child bounds and their insertion),
// then dequeues the next batch (dequeue and gap test) and writes its tasks
// and jobs, or finishes.  The search state is staged in shared memory;
// per-interval work runs one interval per lane of warp 0.  The queue is kept
// sorted in priority order in one of two buffers: insertion is a parallel
// merge into the other buffer, a dequeue takes a prefix.  The last block to
// finish counts the windows still searching, advances the round and sets the
// graph loop condition (with one window, its block does so directly).
__device__ __forceinline__ void control_body(const Geom& g, const CtlArgs& c, int w, CtlShared& sm) {
    SolveState& s = sm.s;
    i128* key = sm.key;
    unsigned long long* cells = sm.cells;
    Node* kids = sm.kids;
    Node* sorted_kids = sm.sorted_kids;
    Node* q_stage = sm.q_stage;
    Node* q_head = sm.q_head;
    float2* bound_iv = sm.bound_iv;
    int16_t* t_fuse = sm.t_fuse;
    int8_t* t_dense = sm.t_dense;
    int16_t* t_jobs = sm.t_jobs;
    int& s_nk = sm.s_nk;
    int& s_stop = sm.s_stop;
    const int32_t n_windows = c.n_windows, task_stride = c.task_stride, job_stride = c.job_stride;
    const int32_t use_loop = c.use_loop, split_ok = c.split_ok;
    SolveState* st_all = c.st_all;
    Node* queues = c.queues;
    Task* tasks_all = c.tasks_all;
    Partial* part_all = c.part_all;
    const int32_t* err_all = c.err_all;
    TraceRec* trace = c.trace;
    Job* jobs_all = c.jobs_all;
    Sched* sch = c.sch;
    int32_t* phase_out = c.phase_out;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int par = sch->round & 1;
    const int running = sch->running;             // searches still running after the last round
    SolveState* st = st_all + w;
    Task* tasks = tasks_all + (size_t)w * task_stride;
    Partial* part = part_all + (size_t)w * task_stride;
    Job* jobs = jobs_all + (size_t)(par ^ 1) * job_stride;
    static_assert(sizeof(SolveState) % 16 == 0, "state is copied as int4");
    for (int i = tid; i < (int)(sizeof(SolveState) / 16); i += blockDim.x)
        reinterpret_cast<int4*>(&s)[i] = reinterpret_cast<const int4*>(st)[i];
    __syncthreads();
    if (s.phase != PH_DONE) {
    Node* qa = queues + (size_t)w * 2 * s.qcap;
    Node* qb = qa + s.qcap;
    const int32_t* err = err_all + w;
    const int64_t M = s.M;
    const int n_tasks = s.n_tasks;

    // Each task's sums (accumulated by the evaluation over its row bands),
    // read and cleared for the next round.
    for (int t = tid; t < n_tasks; t += blockDim.x) {
        const Partial q = part[t];
        part[t] = Partial{};
        key[t] = partial_key(M, q, tasks[t].kind == TASK_POINT);
        cells[t] = q.cells[0] + q.cells[1];
    }
    __syncthreads();

    if (wid == 0) {
        int stop = 0, nk = 0;
        if (*err) {
            if (lane == 0) s.status = DD_ERR_ARG;
            stop = 1;
        } else if (s.cancel) {                    // the host cancelled the search between rounds
            if (lane == 0) s.status = DD_ERR_CANCELLED;
            stop = 1;
        } else if (s.phase == PH_INIT) {
            if (lane == 0) {
                s.K_hat = key[0];
                s.point_evals = 1;
                s.bound_evals = n_tasks - 1;
                s.cells = (int64_t)cells[0];
                s.bcells = 0;
                for (int t = 1; t < n_tasks; t++) {
                    s.cells += (int64_t)cells[t];
                    s.bcells += (int64_t)cells[t];
                    // the domain is queued unconditionally; warm-start pieces
                    // when their bound reaches the incumbent, as children are
                    if (s.warm && !(key[t] >= s.K_hat)) continue;
                    Node nd;
                    nd.lo = tasks[t].D_lo;
                    nd.hi = tasks[t].D_hi;
                    nd.pad0 = nd.pad1 = 0;
                    nd.kb = key[t];
                    kids[nk++] = nd;
                }
                s.phase = PH_RUN;
            }
            nk = __shfl_sync(0xffffffffu, nk, 0);
        } else {
            const int np = s.n_pop;
            // Incumbent update in dequeue order (a centre with K >= K_hat wins):
            // per chunk of 32, the chunk maximum wins if it reaches the running
            // incumbent, at the last lane attaining it.
            i128 K_hat = s.K_hat;
            float D_hat = s.D_hat;
            unsigned long long pc = 0;
            for (int base = 0; base < np; base += 32) {
                const int j = base + lane;
                const bool v = j < np;
                const i128 kc = v ? key[s.pop[j].t_point] : (i128)(-1);
                if (v) pc += cells[s.pop[j].t_point];
                const i128 m = warp_max_i128(kc);
                if (m >= K_hat) {
                    const unsigned at = __ballot_sync(0xffffffffu, v && kc == m);
                    const int last = 31 - __clz(at);
                    K_hat = m;
                    D_hat = __shfl_sync(0xffffffffu, v ? s.pop[j].c : 0.0f, last);
                }
            }
            pc = warp_sum(pc);
            // Leaves, traces, child bounds, children inserted against the
            // end-of-round incumbent.
            int nonleaf = 0, has_leaf = 0;
            i128 lmax = (i128)(-1);
            unsigned long long bc = 0;
            for (int base = 0; base < np; base += 32) {
                const int j = base + lane;
                const bool v = j < np;
                Popped p;
                if (v) p = s.pop[j];
                if (v && trace && w == 0 && s.trace_len + j < s.trace_cap) {
                    TraceRec r;
                    r.D_lo = p.lo;
                    r.D_hi = p.hi;
                    r.D_c = p.c;
                    r.leaf = p.leaf;
                    r.Kbar = p.kb;
                    r.K_c = key[p.t_point];
                    trace[s.trace_len + j] = r;
                }
                const bool leaf = v && p.leaf, split = v && !p.leaf;
                if (leaf && (!has_leaf || p.kb > lmax)) lmax = p.kb;
                has_leaf |= leaf;
                i128 kl = 0, kr = 0;
                int c = 0;
                if (split) {
                    kl = key[p.t_left];
                    kr = key[p.t_right];
                    bc += cells[p.t_left] + cells[p.t_right];
                    c = (kl >= K_hat) + (kr >= K_hat);
                }
                nonleaf += __popc(__ballot_sync(0xffffffffu, split));
                const int incl = warp_incl_scan(c);
                const int at = nk + incl - c;
                if (split) {
                    int o = at;
                    if (kl >= K_hat) {
                        Node nd;
                        nd.lo = p.lo;
                        nd.hi = p.c;
                        nd.pad0 = nd.pad1 = 0;
                        nd.kb = kl;
                        kids[o++] = nd;
                    }
                    if (kr >= K_hat) {
                        Node nd;
                        nd.lo = p.c;
                        nd.hi = p.hi;
                        nd.pad0 = nd.pad1 = 0;
                        nd.kb = kr;
                        kids[o] = nd;
                    }
                }
                nk += __shfl_sync(0xffffffffu, incl, 31);
            }
            bc = warp_sum(bc);
            has_leaf = __any_sync(0xffffffffu, has_leaf);
            lmax = warp_max_i128(lmax);
            if (lane == 0) {
                s.K_hat = K_hat;
                s.D_hat = D_hat;
                s.nodes_expanded += np;
                s.point_evals += np;
                s.bound_evals += 2 * nonleaf;
                s.cells += (int64_t)(pc + bc);
                s.bcells += (int64_t)bc;
                if (has_leaf && (!s.have_leaf || lmax > s.leaf_max)) s.leaf_max = lmax;
                s.have_leaf |= has_leaf;
                s.trace_len += np;
            }
        }
        if (!stop && s.q_n + nk > s.qcap) {
            if (lane == 0) s.status = DD_ERR_QUEUE_OVERFLOW;
            stop = 1;
        }
        if (lane == 0) {
            s_nk = nk;
            s_stop = stop;
        }
    }
    __syncthreads();
    const int nk = s_nk;
    const int stop = s_stop;

    if (!stop) {
        // sort the new children, then merge them with the queued intervals;
        // a queue that fits is staged in shared memory first, so that the
        // children's ranks are searched there instead of in global memory
        const Node* src = (s.q_cur ? qb : qa) + s.q_start;
        Node* dst = s.q_cur ? qa : qb;
        const int a = s.q_n;
        const bool staged = a <= Q_STAGE;
        // A child's rank among the children (they are distinct: popped
        // intervals are disjoint) counted by `per` threads, each over every
        // per-th child, summed within the thread group.
        int per = 1;
        while (nk > 32 && per < 32 && 2 * per * nk <= (int)blockDim.x) per *= 2;
        for (int base = 0; base < nk * per; base += blockDim.x) {
            const int i = (base + tid) / per, part = (base + tid) % per;
            int r = 0;
            if (i < nk)
                for (int j = part; j < nk; j += per) r += better(kids[j], kids[i]);
            for (int o = per / 2; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (i < nk && part == 0) sorted_kids[r] = kids[i];
        }
        if (staged)
            for (int i = tid; i < a; i += blockDim.x) q_stage[i] = src[i];
        __syncthreads();
        const Node* qs = staged ? q_stage : src;
        for (int i = tid; i < a; i += blockDim.x) {
            const Node e = qs[i];
            const int at = i + rank_in(sorted_kids, nk, e);
            dst[at] = e;
            if (at < MAX_POP) q_head[at] = e;
        }
        for (int j = tid; j < nk; j += blockDim.x) {
            const Node e = sorted_kids[j];
            const int at = j + rank_in(qs, a, e);
            dst[at] = e;
            if (at < MAX_POP) q_head[at] = e;
        }
        __syncthreads();
        if (tid == 0) {
            s.q_cur ^= 1;
            s.q_start = 0;
            s.q_n = a + nk;
            if (s.q_n > s.max_queue) s.max_queue = s.q_n;
        }
        __syncthreads();
    }

    if (wid == 0) {
        const Node* q = q_head;                   // the first entries of the queue just merged
        int np = 0;
        if (!stop) {                              // dequeue up to K_pop intervals
            const i128 K0 = s.K_hat, gK = s.gamma_K;
            const int lim = min(s.K_pop, s.q_n);
            for (int base = 0; base < lim; base += 32) {
                const int j = base + lane;
                const bool v = j < lim;
                Node nd;
                if (v) nd = q[j];
                const bool pass = v && (nd.kb - K0 > gK);   // gap test
                const unsigned fail = __ballot_sync(0xffffffffu, v && !pass);
                const int first = fail ? __ffs(fail) - 1 : 32;
                if (v && lane < first) {
                    s.pop[j].lo = nd.lo;
                    s.pop[j].hi = nd.hi;
                    s.pop[j].kb = nd.kb;
                }
                if (fail) {
                    if (base + first == 0 && lane == 0) {
                        s.have_stop = 1;
                        s.stop_kb = nd.kb;
                    }
                    np = base + first;
                    break;
                }
                np = min(lim, base + 32);
            }
            if (lane == 0) {
                s.q_start = np;
                s.q_n -= np;
            }
        }
        __syncwarp();
        if (stop || np == 0) {
            if (lane == 0) {
                i128 top = s.K_hat;
                if (s.have_leaf && s.leaf_max > top) top = s.leaf_max;
                if (s.have_stop && s.stop_kb > top) top = s.stop_kb;
                s.stop_kb = top - s.K_hat;        // the certificate gap_K
                s.n_pop = 0;
                s.n_tasks = 0;
                s.phase = PH_DONE;
            }
        } else {
            int nl_before = 0;
            for (int base = 0; base < np; base += 32) {   // centre and bisection
                const int j = base + lane;
                const bool v = j < np;
                bool split = false, fuse = false;
                if (v) {
                    Popped& p = s.pop[j];
                    p.c = centre(p.lo, p.hi);
                    const float w = __fsub_rn(p.hi, p.lo);
                    p.leaf = !(w > s.tol) || !(p.c > p.lo) || !(p.c < p.hi);
                    split = !p.leaf;
                    // narrow intervals: centre and halves evaluated by one fused job
                    fuse = split && g.fuse_cells > 0.0f && bound_cells(g, p.lo, p.hi, s.tau) - 1.0f <= g.fuse_cells;
                }
                const unsigned sb = __ballot_sync(0xffffffffu, split);
                if (v) {
                    Popped& p = s.pop[j];
                    p.t_point = j;
                    Task a;
                    a.D_lo = a.D_hi = p.c;
                    a.kind = TASK_POINT;
                    a.splits = 1;
                    tasks[j] = a;
                    t_fuse[j] = 0;
                    t_dense[j] = 0;
                    if (split) {
                        const int t = np + 2 * (nl_before + __popc(sb & ((1u << lane) - 1u)));
                        p.t_left = t;
                        p.t_right = t + 1;
                        t_fuse[j] = fuse ? (int16_t)(t + 1) : (int16_t)0;
                        t_fuse[t] = t_fuse[t + 1] = fuse ? (int16_t)-1 : (int16_t)0;
                        // dense bounds (splittable when the round is small), decided once here
                        t_dense[t] = split_ok && !fuse && bound_cells(g, p.lo, p.c, s.tau) >= DENSE_CELLS;
                        t_dense[t + 1] = split_ok && !fuse && bound_cells(g, p.c, p.hi, s.tau) >= DENSE_CELLS;
                        Task l, r;
                        l.D_lo = p.lo;
                        l.D_hi = p.c;
                        l.kind = TASK_BOUND;
                        l.splits = 1;                 // the job builder decides (fill_splits)
                        r.D_lo = p.c;
                        r.D_hi = p.hi;
                        r.kind = TASK_BOUND;
                        r.splits = 1;
                        tasks[t] = l;
                        tasks[t + 1] = r;
                        bound_iv[t] = make_float2(p.lo, p.c);
                        bound_iv[t + 1] = make_float2(p.c, p.hi);
                    } else {
                        p.t_left = p.t_right = -1;
                    }
                }
                nl_before += __popc(sb);
            }
            if (lane == 0) {
                s.rounds++;
                s.n_pop = np;
                s.n_tasks = np + 2 * nl_before;
                if (s.rounds > s.max_rounds) {
                    s.status = DD_ERR_TIMEOUT;
                    s.stop_kb = 0;
                    s.n_tasks = 0;
                    s.phase = PH_DONE;
                }
            }
        }
        __syncwarp();
        // Jobs of the next round, bound tasks first: a task of `splits` splits
        // contributes that many jobs (fill_splits for the dense bounds, ranked
        // in this loop's order; every other task has one split).
        if (s.phase != PH_DONE) {
            const int nt = s.n_tasks;
            int nd = 0, nabs = 0;                 // dense bound tasks; tasks inside fused jobs
            for (int c0 = 0; c0 < nt; c0 += 32) {
                const int q = c0 + lane, t = nt - 1 - q;
                nd += __popc(__ballot_sync(0xffffffffu, q < nt && t_dense[t]));
                nabs += __popc(__ballot_sync(0xffffffffu, q < nt && t_fuse[t] < 0));
            }
            const int units = (nt - nabs) * g.n_tiles;   // one per job and band before any split
            // the window's share of the grid: the searches still running
            // after the last round share it (all of them before the first)
            const int sharers = n_windows == 1 ? 1 : (running > 0 ? running : n_windows);
            const int target = g.split_target / sharers;
            int total = 0, seen = 0;
            for (int c0 = 0; c0 < nt; c0 += 32) {     // jobs per task, counted once
                const int q = c0 + lane, t = nt - 1 - q;
                const bool d = q < nt && t_dense[t];
                const unsigned db = __ballot_sync(0xffffffffu, d);
                const int rank = seen + __popc(db & ((1u << lane) - 1u));
                seen += __popc(db);
                const int c = q >= nt || t_fuse[t] < 0 ? 0 : (d ? fill_splits(g, target, units, nd, rank) : 1);
                if (q < nt) t_jobs[q] = (int16_t)c;
                total += __reduce_add_sync(0xffffffffu, (unsigned)c);
            }
            int base = 0;
            if (lane == 0) {
                if (n_windows == 1) {             // the only block: the list is its own
                    sch->n_jobs[par ^ 1] = total;
                } else {
                    base = atomicAdd(&sch->n_jobs[par ^ 1], total);
                }
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            __syncwarp();
            int run = 0;
            for (int c0 = 0; c0 < nt; c0 += 32) {
                const int q = c0 + lane;
                const int t = nt - 1 - q;
                const int c = q < nt ? (int)t_jobs[q] : 0;
                const int incl = warp_incl_scan(c);
                const int fz = c > 0 ? (int)t_fuse[t] : 0;
                for (int k = 0; k < c; k++) {
                    Job j;
                    j.win = w;
                    j.task = t;
                    j.split = fz > 0 ? fz - 1 : k;
                    j.splits = fz > 0 ? -1 : c;
                    jobs[base + run + incl - c + k] = j;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < (int)(sizeof(SolveState) / 16); i += blockDim.x)
        reinterpret_cast<int4*>(st)[i] = reinterpret_cast<const int4*>(&s)[i];
    } // s.phase != PH_DONE at entry
    __syncthreads();
    if (tid == 0 && phase_out) phase_out[w] = s.phase;
    if (tid == 0 && n_windows == 1) {             // the only block is the last: no ticket
        const int active = s.phase != PH_DONE ? 1 : 0;
        sch->running = active;
        sch->round += 1;
        if (use_loop) cudaGraphSetConditional(c.loop, active ? 1u : 0u);
    } else if (tid == 0) {
        __threadfence();
        if (s.phase != PH_DONE) atomicAdd(&sch->active, 1);
        if (atomicAdd(&sch->ticket, 1) == n_windows - 1) {    // the last block of the round
            __threadfence();
            const int active = atomicAdd(&sch->active, 0);
            sch->running = active;
            sch->active = 0;
            sch->ticket = 0;
            sch->round += 1;
            if (use_loop) cudaGraphSetConditional(c.loop, active > 0 ? 1u : 0u);
        }
    }
}

__global__ void __launch_bounds__(CTL_THREADS) k_control(Geom g, CtlArgs c) {
    __shared__ CtlShared sm;
    control_body(g, c, blockIdx.x, sm);
}


CtlArgs control_args(int32_t n_windows, SolveState* st, Node* queues, Task* tasks, int32_t task_stride, Partial* part,
                     const int32_t* err, TraceRec* trace, Job* jobs, int32_t job_stride, Sched* sch,
                     cudaGraphConditionalHandle loop, int32_t use_loop, int32_t split_ok, int32_t* phase_out) {
    CtlArgs c;
    c.n_windows = n_windows;
    c.st_all = st;
    c.queues = queues;
    c.tasks_all = tasks;
    c.task_stride = task_stride;
    c.part_all = part;
    c.err_all = err;
    c.trace = trace;
    c.jobs_all = jobs;
    c.job_stride = job_stride;
    c.sch = sch;
    c.loop = loop;
    c.use_loop = use_loop;
    c.split_ok = split_ok < 0 ? 1 : split_ok;
    c.phase_out = phase_out;
    return c;
}

cudaError_t launch_control(const Geom& g, int32_t n_windows, SolveState* st, Node* queues, Task* tasks,
                           int32_t task_stride, Partial* part, const int32_t* err, TraceRec* trace,
                           Job* jobs, int32_t job_stride, Sched* sch, cudaGraphConditionalHandle loop,
                           int32_t use_loop, cudaStream_t s, int32_t split_ok, int32_t* phase_out) {
    const CtlArgs c = control_args(n_windows, st, queues, tasks, task_stride, part, err, trace, jobs, job_stride, sch,
                                   loop, use_loop, split_ok, phase_out);
    k_control<<<n_windows, CTL_THREADS, 0, s>>>(g, c);
    return cudaGetLastError();
}

// Function attributes are per device: the carveout and the dynamic
// shared-memory limit of k_eval are set on the current device the first time
// it is used, and the limit only ever raised, under one lock (contexts of
// several host threads and devices share these records).
constexpr int SMEM_MAX_DEVICES = 64;
static std::mutex g_smem_mu;
static bool g_carveout[SMEM_MAX_DEVICES];
static int g_smem_bytes[SMEM_MAX_DEVICES];

cudaError_t eval_smem_setup(const Geom& g) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= SMEM_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    if (!g_carveout[dev]) {
        // One shared-memory carveout for every kernel of the library, so that
        // consecutive launches never wait for an L1 / shared reconfiguration.
        const void* fns[] = {(const void*)k_eval, (const void*)k_control, (const void*)k_init,
                             (const void*)k_keys, (const void*)k_row_hist, (const void*)k_row_scan,
                             (const void*)k_row_scatter};
        for (const void* f : fns) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
        }
        g_carveout[dev] = true;
    }
    const int bytes = (int)eval_smem_bytes(g, 32 * MAX_WARPS);   // any block size up to 512 threads
    if (bytes <= g_smem_bytes[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) g_smem_bytes[dev] = bytes;
    return e;
}

}  // namespace dd
