// Pre-passes over event streams: the paper's fast mode (Sec. 6, the resized
// and resampled sequences: the events of a window with their coordinates
// scaled to a coarser frame and a random share of them kept, compacted in
// their order), the windows of a time-sorted stream (Sec. 4.4: the stream
// taken batch by batch), and the time span of a batch (Sec. 3.3 measures a
// batch's times from its earliest event).
//
// Event i goes to the nearest coarse pixel centre, floor(x k + 1/2) with
// k = W2/W in binary32, clamped to the frame, and is kept when the top 24
// bits of SplitMix64 output i (key SplitMix64(seed, 0); Steele, Lea and
// Flood, OOPSLA 2014) fall below floor(keep 2^24).
#include "dd_internal.cuh"
#include "../../include/dd.h"

namespace dd {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_PER_THREAD = 8;
constexpr int RS_CHUNK = RS_THREADS * RS_PER_THREAD;   // events per block

__device__ __forceinline__ uint64_t sm64(uint64_t state0, uint64_t i) {
    uint64_t z = state0 + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Rs {
    const int16_t* x;
    const int16_t* y;
    const float* t;
    int64_t n;
    int32_t W, H, W2, H2;
    float kx, ky;
    uint64_t key;
    uint32_t thr;
};

__device__ __forceinline__ bool kept(const Rs& r, int64_t i) { return (uint32_t)(sm64(r.key, (uint64_t)i) >> 40) < r.thr; }

// Thread j of block b: the events [b*CHUNK + j*PER, ... + PER) in order.
// Counts kept events per block; flags events outside the fine frame.
__global__ void __launch_bounds__(RS_THREADS) k_rs_count(Rs r, int32_t* counts, int32_t* err) {
    __shared__ int32_t s[RS_THREADS / 32];
    const int64_t i0 = (int64_t)blockIdx.x * RS_CHUNK + (int64_t)threadIdx.x * RS_PER_THREAD;
    int c = 0, bad = 0;
    for (int k = 0; k < RS_PER_THREAD; k++) {
        const int64_t i = i0 + k;
        if (i >= r.n) break;
        const int xi = r.x[i], yi = r.y[i];
        bad |= !(xi >= 0 && xi < r.W && yi >= 0 && yi < r.H);
        c += kept(r, i);
    }
    if (bad) atomicOr(err, 1);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < RS_THREADS / 32; w++) t += s[w];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of nb block counts in one block; offsets[nb] = total.
__global__ void __launch_bounds__(1024) k_rs_scan(const int32_t* counts, int32_t nb, int64_t* offsets) {
    __shared__ int64_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int64_t t = 0;
    for (int k = 0; k < per && b0 + k < nb; k++) t += counts[b0 + k];
    part[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {                       // 1024 partial sums, in order
        int64_t run = 0;
        for (int k = 0; k < 1024; k++) {
            const int64_t v = part[k];
            part[k] = run;
            run += v;
        }
        offsets[nb] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int k = 0; k < per && b0 + k < nb; k++) {
        offsets[b0 + k] = run;
        run += counts[b0 + k];
    }
}

// The kept events of block b written from offsets[b], in order.
__global__ void __launch_bounds__(RS_THREADS) k_rs_write(Rs r, const int64_t* offsets, int16_t* x2, int16_t* y2,
                                                         float* t2) {
    __shared__ int32_t s[RS_THREADS / 32];
    const int64_t i0 = (int64_t)blockIdx.x * RS_CHUNK + (int64_t)threadIdx.x * RS_PER_THREAD;
    unsigned mask = 0;
    for (int k = 0; k < RS_PER_THREAD; k++) {
        const int64_t i = i0 + k;
        if (i < r.n && kept(r, i)) mask |= 1u << k;
    }
    const int c = __popc(mask);
    // block-wide exclusive scan of the per-thread counts, in thread order
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s[wid] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; w++) before += s[w];
    int64_t o = offsets[blockIdx.x] + before + incl - c;
    for (int k = 0; k < RS_PER_THREAD; k++) {
        if (!(mask >> k & 1u)) continue;
        const int64_t i = i0 + k;
        int cx = (int)floorf(__fadd_rn(__fmul_rn((float)r.x[i], r.kx), 0.5f));
        int cy = (int)floorf(__fadd_rn(__fmul_rn((float)r.y[i], r.ky), 0.5f));
        cx = cx > r.W2 - 1 ? r.W2 - 1 : cx;
        cy = cy > r.H2 - 1 ? r.H2 - 1 : cy;
        x2[o] = (int16_t)cx;
        y2[o] = (int16_t)cy;
        t2[o] = r.t[i];
        o++;
    }
}

// Window k of a time-sorted stream: the events with (t - t0_k) in [0, tau]
// (binary32 subtraction, the test ingest applies), t0_k = t_start + k hop in
// binary64 rounded to binary32.  (t - t0) is monotone in t, so both ends are
// binary searches: first[k] = first event with t - t0 >= 0, count[k] = the
// events before the first with t - t0 > tau.
__global__ void k_stream_bounds(const float* t, int64_t n, double t_start, double hop, float tau, int32_t n_windows,
                                int64_t* first, int64_t* count, float* t0_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_windows) return;
    const float t0 = (float)(t_start + hop * (double)k);
    int64_t lo = 0, hi = n;                       // first i with t[i] - t0 >= 0
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (__fsub_rn(t[mid], t0) >= 0.0f) hi = mid;
        else lo = mid + 1;
    }
    int64_t a = lo, b = n;                        // first i with t[i] - t0 > tau
    while (a < b) {
        const int64_t mid = a + (b - a) / 2;
        if (__fsub_rn(t[mid], t0) > tau) b = mid;
        else a = mid + 1;
    }
    first[k] = lo;
    count[k] = a - lo;
    t0_out[k] = t0;
}

// The time span of n timestamps: per block the least and greatest finite t
// (grid-stride), then one block over the blocks' results.  Non-finite
// timestamps are skipped here (the solver's own validation rejects them).
constexpr int SPAN_THREADS = 256;

__device__ __forceinline__ void span_reduce(float& lo, float& hi) {
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    __shared__ float s_lo[SPAN_THREADS / 32], s_hi[SPAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < SPAN_THREADS / 32; w++) {
            lo = fminf(lo, s_lo[w]);
            hi = fmaxf(hi, s_hi[w]);
        }
}

__global__ void __launch_bounds__(SPAN_THREADS) k_span_part(const float* t, int64_t n, float2* part) {
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * SPAN_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SPAN_THREADS) {
        const float v = t[i];
        if (isfinite(v)) {
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    span_reduce(lo, hi);
    if (threadIdx.x == 0) part[blockIdx.x] = make_float2(lo, hi);
}

__global__ void __launch_bounds__(SPAN_THREADS) k_span_final(const float2* part, int nb, float2* out) {
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += SPAN_THREADS) {
        lo = fminf(lo, part[i].x);
        hi = fmaxf(hi, part[i].y);
    }
    span_reduce(lo, hi);
    if (threadIdx.x == 0) *out = make_float2(lo, hi);
}

}  // namespace

int32_t span_blocks(int64_t n) {
    const int64_t b = (n + SPAN_THREADS - 1) / SPAN_THREADS;
    return (int32_t)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_time_span(const float* t, int64_t n, float2* part, float2* out, cudaStream_t s) {
    const int32_t nb = span_blocks(n);
    k_span_part<<<nb, SPAN_THREADS, 0, s>>>(t, n, part);
    k_span_final<<<1, SPAN_THREADS, 0, s>>>(part, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_stream_bounds(const float* t, int64_t n, double t_start, double hop, float tau, int32_t n_windows,
                                 int64_t* first, int64_t* count, float* t0, cudaStream_t s) {
    if (n_windows <= 0) return cudaSuccess;
    k_stream_bounds<<<(n_windows + 127) / 128, 128, 0, s>>>(t, n, t_start, hop, tau, n_windows, first, count, t0);
    return cudaGetLastError();
}

int32_t resample_blocks(int64_t n) { return (int32_t)((n + RS_CHUNK - 1) / RS_CHUNK); }

cudaError_t launch_resample(const int16_t* x, const int16_t* y, const float* t, int64_t n, int32_t W, int32_t H,
                            int32_t W2, int32_t H2, float keep, uint64_t seed, int16_t* x2, int16_t* y2, float* t2,
                            int32_t* counts, int64_t* offsets, int32_t* err, cudaStream_t s) {
    Rs r;
    r.x = x;
    r.y = y;
    r.t = t;
    r.n = n;
    r.W = W;
    r.H = H;
    r.W2 = W2;
    r.H2 = H2;
    r.kx = (float)W2 / (float)W;
    r.ky = (float)H2 / (float)H;
    r.key = 0;
    {
        // host copy of the device generator's key derivation
        uint64_t z = seed + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        r.key = z ^ (z >> 31);
    }
    r.thr = (uint32_t)floor((double)keep * 16777216.0);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int32_t nb = resample_blocks(n);
    if (nb == 0) return cudaMemsetAsync(offsets, 0, sizeof(int64_t), s);
    k_rs_count<<<nb, RS_THREADS, 0, s>>>(r, counts, err);
    k_rs_scan<<<1, 1024, 0, s>>>(counts, nb, offsets);
    k_rs_write<<<nb, RS_THREADS, 0, s>>>(r, offsets, x2, y2, t2);
    return cudaGetLastError();
}

}  // namespace dd
