// GPU version of the synthetic descent windows of synth/descent.py.
//
// Input generation only (no estimator arithmetic).  It draws the same
// counter-based SplitMix64 numbers (Steele, Lea and Flood, OOPSLA 2014) at
// the same counters and applies the same scene model in binary64, so a
// window is identical, event for event, to make_window()'s; only the order
// of events differs (points first, then noise; the estimator's results do
// not depend on event order).  Polarities (optional output) follow the same
// model: one per scene point, one per noise event.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t G = 0x9E3779B97F4A7C15ull;
constexpr int MAX_ATTEMPTS = 64;
constexpr int TRIES = 8;

__host__ __device__ inline uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t splitmix(uint64_t state0, uint64_t i) { return mix(state0 + (i + 1) * G); }
__host__ __device__ inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return splitmix(splitmix(seed, 0), stream);
}
__device__ inline double u01(uint64_t key, uint64_t ctr) {
    return (double)(splitmix(key, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

struct Params {
    int W, H;
    double fx, fy, D;
    float tau;
    int64_t n_signal, n_points, n_noise;
    uint64_t kp, kt, kn, kpol, knpol;
    int64_t base, extra, e_max;
};

// One thread per scene point: redraw the point until every one of its events
// finds an in-frame time within TRIES draws, then write its events.
__device__ inline int8_t polarity(double u) { return u < 0.5 ? (int8_t)1 : (int8_t)-1; }

__global__ void k_points(Params p, int16_t* x, int16_t* y, float* t, int8_t* pol, int32_t* failed) {
    const int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= p.n_points) return;
    const int64_t cnt = p.base + (pt < p.extra ? 1 : 0);
    const int64_t out0 = pt * p.base + (pt < p.extra ? pt : p.extra);
    const double tau = (double)p.tau;
    for (int a = 0; a < MAX_ATTEMPTS; a++) {
        const uint64_t pa = (uint64_t)pt * MAX_ATTEMPTS + a;
        const double x0 = u01(p.kp, 2 * pa) * p.W, y0 = u01(p.kp, 2 * pa + 1) * p.H;
        bool ok = true;
        for (int64_t j = 0; j < cnt && ok; j++) {
            bool found = false;
            for (int r = 0; r < TRIES && !found; r++) {
                const uint64_t ctr = ((pa * p.e_max + j) * TRIES + r);
                float tf = (float)(u01(p.kt, ctr) * tau);
                if (tf > p.tau) tf = p.tau;
                const double den = 1.0 - p.D * (double)tf;
                const double px = floor(p.fx + (x0 - p.fx) / den + 0.5), py = floor(p.fy + (y0 - p.fy) / den + 0.5);
                if (px >= 0 && px < p.W && py >= 0 && py < p.H) {
                    found = true;
                    x[out0 + j] = (int16_t)px;
                    y[out0 + j] = (int16_t)py;
                    t[out0 + j] = tf;
                }
            }
            ok = found;
        }
        if (ok) {
            if (pol) {
                const int8_t v = polarity(u01(p.kpol, (uint64_t)pt));
                for (int64_t j = 0; j < cnt; j++) pol[out0 + j] = v;
            }
            return;
        }
    }
    atomicAdd(failed, 1);
}

__global__ void k_noise(Params p, int16_t* x, int16_t* y, float* t, int8_t* pol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_noise) return;
    const uint64_t c = (uint64_t)i;
    double nx = floor(u01(p.kn, 3 * c) * p.W), ny = floor(u01(p.kn, 3 * c + 1) * p.H);
    if (nx > p.W - 1) nx = p.W - 1;
    if (ny > p.H - 1) ny = p.H - 1;
    float tf = (float)(u01(p.kn, 3 * c + 2) * (double)p.tau);
    if (tf > p.tau) tf = p.tau;
    const int64_t o = p.n_signal + i;
    x[o] = (int16_t)nx;
    y[o] = (int16_t)ny;
    t[o] = tf;
    if (pol) pol[o] = polarity(u01(p.knpol, c));
}

}  // namespace

extern "C" {

// Generate one window into device arrays x, y, t (and polarities p, when
// not null) of n_signal + n_noise entries (signal events of point p first,
// then noise), on `stream`.
// Returns 0, or -1 for bad arguments, -2 for a CUDA error, -3 if some point
// never fit in the frame.  Synchronises the stream.
int synth_window_gpu(int32_t W, int32_t H, double foe_x, double foe_y, int64_t n_signal, int64_t n_points,
                     int64_t n_noise, double D, double tau, uint64_t seed, int16_t* x, int16_t* y, float* t,
                     int8_t* pol, void* stream) {
    if (W < 1 || H < 1 || n_signal < 0 || n_noise < 0 || !(1.0 - D * tau > 0.0)) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    Params p;
    p.W = W;
    p.H = H;
    p.fx = foe_x;
    p.fy = foe_y;
    p.D = D;
    p.tau = (float)tau;
    p.n_signal = n_signal;
    p.n_noise = n_noise;
    p.kp = stream_key(seed, 1);
    p.kt = stream_key(seed, 2);
    p.kn = stream_key(seed, 3);
    p.kpol = stream_key(seed, 4);
    p.knpol = stream_key(seed, 6);
    int32_t* failed = nullptr;
    if (cudaMallocAsync((void**)&failed, sizeof(int32_t), s) != cudaSuccess) return -2;
    if (cudaMemsetAsync(failed, 0, sizeof(int32_t), s) != cudaSuccess) return -2;
    if (n_signal > 0) {
        int64_t np = n_points < 1 ? 1 : n_points;
        if (np > n_signal) np = n_signal;
        p.n_points = np;
        p.base = n_signal / np;
        p.extra = n_signal % np;
        p.e_max = p.base + (p.extra ? 1 : 0);
        k_points<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(p, x, y, t, pol, failed);
    }
    if (n_noise > 0) k_noise<<<(unsigned)((n_noise + 255) / 256), 256, 0, s>>>(p, x, y, t, pol);
    int32_t h_failed = 0;
    if (cudaMemcpyAsync(&h_failed, failed, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -2;
    if (cudaFreeAsync(failed, s) != cudaSuccess) return -2;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
    return h_failed ? -3 : 0;
}

}  // extern "C"
