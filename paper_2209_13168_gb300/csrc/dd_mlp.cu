// Learned warm start: window features, the 128-128-128-2 network (forward,
// backward, Adam), and the kernel that turns a window's features into the
// guess its search starts from.
//
// The paper starts Algorithm 1 from the centre of the domain; this network,
// trained on windows solved exactly, proposes a guess and a half-width
// instead (include/dd.h states the contract).  Everything here is small next
// to the search: the features are one pass over the window's sorted events
// (8 bytes per event), the network 66k multiply-adds per window.  It runs
// on CUDA cores in binary32 with a fixed summation order (each unit adds
// weight * input for inputs 0..127 in turn onto its bias), so a window's
// guess is reproducible bit for bit.
#include "dd_internal.cuh"
#include "../../include/dd.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

namespace dd {

namespace {

constexpr int P_W1 = 0;
constexpr int P_B1 = P_W1 + MLP_H * FEATURES;
constexpr int P_W2 = P_B1 + MLP_H;
constexpr int P_B2 = P_W2 + MLP_H * MLP_H;
constexpr int P_W3 = P_B2 + MLP_H;
constexpr int P_B3 = P_W3 + MLP_OUT * MLP_H;
constexpr int N_PARAMS = P_B3 + MLP_OUT;
static_assert(N_PARAMS == DD_MLP_PARAMS, "dd.h states the parameter count");
static_assert(FEATURES == DD_MLP_FEATURES && FEATURES == MLP_H, "one thread per feature and per unit");

constexpr float LOG2E = 1.44269504f;

__device__ __forceinline__ float bf(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Unit j of a dense layer with transposed bfloat16 weights wt[in][out].
__device__ __forceinline__ float unit(const uint16_t* wt, int n_out, const float* b, const float* x, int j) {
    float acc = b[j];
    for (int k = 0; k < MLP_H; k++) acc = __fadd_rn(acc, __fmul_rn(bf(wt[k * n_out + j]), x[k]));
    return acc;
}

// The forward pass of one sample by a block of 128 threads; x, h1, h2 and
// out in shared memory.  Every thread returns after the last barrier.
__device__ void forward(const MlpDev& m, const float* x, float* h1, float* h2, float* out) {
    const int j = threadIdx.x;
    const float a1 = unit(m.w1t, MLP_H, m.b1, x, j);
    h1[j] = a1 > 0.0f ? a1 : 0.0f;
    __syncthreads();
    const float a2 = unit(m.w2t, MLP_H, m.b2, h1, j);
    h2[j] = a2 > 0.0f ? a2 : 0.0f;
    __syncthreads();
    if (j < MLP_OUT) out[j] = unit(m.w3t, MLP_OUT, m.b3, h2, j);
    __syncthreads();
}

// ------------------------------------------------------------ features

constexpr int FEAT_THREADS = 256;

// Block c counts chunk c of its window's sorted events into the window's
// 16 x 8 bins (radial bin from the squared distance to the FOE relative to
// the farthest corner pixel centre; temporal bin from (t - t0)/tau).
__global__ void __launch_bounds__(FEAT_THREADS) k_features(Geom g, const WinIn* __restrict__ wins,
                                                           const int32_t* __restrict__ chunk_win,
                                                           const Ev* __restrict__ ev, int32_t* counts) {
    __shared__ int32_t h[FEATURES];
    for (int k = threadIdx.x; k < FEATURES; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int w = chunk_win[blockIdx.x];
    const WinIn win = wins[w];
    const float ax = g.fx, bx = __fsub_rn((float)(g.W - 1), g.fx);
    const float ay = g.fy, by = __fsub_rn((float)(g.H - 1), g.fy);
    const float cx = ax > bx ? ax : bx, cy = ay > by ? ay : by;
    const float R2 = __fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy));
    const float tsc = __fdiv_rn((float)FEAT_T, win.tau);
    const int64_t i0 = (int64_t)(blockIdx.x - win.chunk0) * CHUNK, i1 = min(win.n, i0 + CHUNK);
    const Ev* e = ev + win.ev_off;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const Ev v = e[i];
        const float dx = v.dx, dy = v.dy;
        const float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        const float u = R2 > 0.0f ? __fdiv_rn(r2, R2) : 0.0f;
        int rb = (int)floorf(__fmul_rn(__fsqrt_rn(u), (float)FEAT_R));
        rb = rb > FEAT_R - 1 ? FEAT_R - 1 : rb;
        int tb = (int)floorf(__fmul_rn(v.t, tsc));
        tb = tb < 0 ? 0 : (tb > FEAT_T - 1 ? FEAT_T - 1 : tb);
        atomicAdd(&h[rb * FEAT_T + tb], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < FEATURES; k += blockDim.x)
        if (h[k]) atomicAdd(&counts[(size_t)w * FEATURES + k], h[k]);
}

// Block w: if window w asks for the model's warm start, its features, the
// network, and the guess and half-width written into its search parameters.
__global__ void __launch_bounds__(MLP_H) k_warm(int32_t n_windows, const int32_t* __restrict__ counts,
                                                const WinIn* __restrict__ wins, WinParams* params, MlpDev m) {
    __shared__ float x[FEATURES], h1[MLP_H], h2[MLP_H], out[MLP_OUT];
    const int w = blockIdx.x;
    if (w >= n_windows || params[w].warm != DD_WARM_MODEL) return;
    const int j = threadIdx.x;
    const int64_t n = wins[w].n;
    x[j] = n > 0 ? __fdiv_rn((float)(counts[(size_t)w * FEATURES + j] * FEATURES), (float)n) : 0.0f;
    __syncthreads();
    forward(m, x, h1, h2, out);
    if (j == 0) {
        const float tau = wins[w].tau;
        float v = __fadd_rn(__fmul_rn(out[1], LOG2E), 0.5f);
        if (!(v >= -20.0f)) v = -20.0f;
        if (v > 1.0f) v = 1.0f;
        const int e = (int)floorf(v);
        params[w].D_warm = __fdiv_rn(out[0], tau);
        params[w].w_warm = __fdiv_rn(__uint_as_float((uint32_t)(e + 127) << 23), tau);
        params[w].warm = 1;
    }
}

// feat[w][k] = 128 counts[w][k] / n_w, as the warm-start kernel forms its input.
__global__ void __launch_bounds__(FEATURES) k_feature_norm(const int32_t* __restrict__ counts,
                                                           const WinIn* __restrict__ wins, float* feat) {
    const int w = blockIdx.x, j = threadIdx.x;
    const int64_t n = wins[w].n;
    feat[(size_t)w * FEATURES + j] =
        n > 0 ? __fdiv_rn((float)(counts[(size_t)w * FEATURES + j] * FEATURES), (float)n) : 0.0f;
}

// -------------------------------------------------------------- training

// Block b: forward pass of sample b, activations kept for the backward pass.
__global__ void __launch_bounds__(MLP_H) k_fwd(MlpDev m, const float* __restrict__ X, float* h1g, float* h2g,
                                               float* outg) {
    __shared__ float x[FEATURES], h1[MLP_H], h2[MLP_H], out[MLP_OUT];
    const int b = blockIdx.x, j = threadIdx.x;
    x[j] = X[(size_t)b * FEATURES + j];
    __syncthreads();
    forward(m, x, h1, h2, out);
    h1g[(size_t)b * MLP_H + j] = h1[j];
    h2g[(size_t)b * MLP_H + j] = h2[j];
    if (j < MLP_OUT) outg[(size_t)b * MLP_OUT + j] = out[j];
}

constexpr int LOSS_THREADS = 256;

// The loss (mean over B) and its gradient with respect to the outputs; one
// block, summed in a fixed order.
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(int32_t B, const float* __restrict__ out,
                                                       const float* __restrict__ u_star, float* gout, float* loss) {
    __shared__ float part[LOSS_THREADS];
    float acc = 0.0f;
    const float inv = 1.0f / (float)B;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float u = out[2 * b], l = out[2 * b + 1];
        const float e = u_star[b] - u;
        const float q = 9.0f * expf(-2.0f * l);
        acc += 0.5f * q * e * e + l;
        gout[2 * b] = -q * e * inv;
        gout[2 * b + 1] = (1.0f - q * e * e) * inv;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = part[0] * inv;
}

// Block b: gradients with respect to the hidden units of sample b (through
// the ReLUs), with the [out][in] bfloat16 weights.
__global__ void __launch_bounds__(MLP_H) k_back(const uint16_t* __restrict__ w2, const uint16_t* __restrict__ w3,
                                                const float* __restrict__ h1g, const float* __restrict__ h2g,
                                                const float* __restrict__ gout, float* g1g, float* g2g) {
    __shared__ float g2[MLP_H];
    const int b = blockIdx.x, k = threadIdx.x;
    const float go0 = gout[2 * b], go1 = gout[2 * b + 1];
    float a = bf(w3[k]) * go0 + bf(w3[MLP_H + k]) * go1;
    const float v2 = h2g[(size_t)b * MLP_H + k] > 0.0f ? a : 0.0f;
    g2[k] = v2;
    g2g[(size_t)b * MLP_H + k] = v2;
    __syncthreads();
    a = 0.0f;
    for (int j = 0; j < MLP_H; j++) a += bf(w2[j * MLP_H + k]) * g2[j];
    g1g[(size_t)b * MLP_H + k] = h1g[(size_t)b * MLP_H + k] > 0.0f ? a : 0.0f;
}

// One thread per parameter: its gradient summed over the B samples in order.
__global__ void __launch_bounds__(256) k_wgrad(int32_t B, const float* __restrict__ X, const float* __restrict__ h1,
                                               const float* __restrict__ h2, const float* __restrict__ g1,
                                               const float* __restrict__ g2, const float* __restrict__ gout,
                                               float* grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N_PARAMS) return;
    const float *gv, *av;
    int gs, as, gi, ai;
    if (p < P_B1) {
        gv = g1; gs = MLP_H; gi = p / FEATURES; av = X; as = FEATURES; ai = p % FEATURES;
    } else if (p < P_W2) {
        gv = g1; gs = MLP_H; gi = p - P_B1; av = nullptr; as = 0; ai = 0;
    } else if (p < P_B2) {
        gv = g2; gs = MLP_H; gi = (p - P_W2) / MLP_H; av = h1; as = MLP_H; ai = (p - P_W2) % MLP_H;
    } else if (p < P_W3) {
        gv = g2; gs = MLP_H; gi = p - P_B2; av = nullptr; as = 0; ai = 0;
    } else if (p < P_B3) {
        gv = gout; gs = MLP_OUT; gi = (p - P_W3) / MLP_H; av = h2; as = MLP_H; ai = (p - P_W3) % MLP_H;
    } else {
        gv = gout; gs = MLP_OUT; gi = p - P_B3; av = nullptr; as = 0; ai = 0;
    }
    float acc = 0.0f;
    if (av)
        for (int b = 0; b < B; b++) acc += gv[(size_t)b * gs + gi] * av[(size_t)b * as + ai];
    else
        for (int b = 0; b < B; b++) acc += gv[(size_t)b * gs + gi];
    grad[p] = acc;
}

__device__ __forceinline__ bool is_weight(int p, int* layer, int* o, int* i) {
    if (p < P_B1) { *layer = 0; *o = p / FEATURES; *i = p % FEATURES; return true; }
    if (p >= P_W2 && p < P_B2) { *layer = 1; *o = (p - P_W2) / MLP_H; *i = (p - P_W2) % MLP_H; return true; }
    if (p >= P_W3 && p < P_B3) { *layer = 2; *o = (p - P_W3) / MLP_H; *i = (p - P_W3) % MLP_H; return true; }
    return false;
}

struct Weights {
    uint16_t *w1, *w2, *w3;      // [out][in]
    uint16_t *w1t, *w2t, *w3t;   // [in][out]
};

__device__ __forceinline__ void store_weight(const Weights& wb, int layer, int o, int i, float v) {
    const uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    if (layer == 0) { wb.w1[o * FEATURES + i] = h; wb.w1t[i * MLP_H + o] = h; }
    else if (layer == 1) { wb.w2[o * MLP_H + i] = h; wb.w2t[i * MLP_H + o] = h; }
    else { wb.w3[o * MLP_H + i] = h; wb.w3t[i * MLP_OUT + o] = h; }
}

// One thread per parameter: an Adam step on the binary32 master value
// (lr_t carries the bias corrections), then the bfloat16 copies.
__global__ void __launch_bounds__(256) k_adam(float lr_t, const float* __restrict__ grad, float* master, float* mom,
                                              float* vel, Weights wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N_PARAMS) return;
    const float g = grad[p];
    const float m1 = 0.9f * mom[p] + 0.1f * g;
    const float v1 = 0.999f * vel[p] + 0.001f * g * g;
    mom[p] = m1;
    vel[p] = v1;
    const float v = master[p] - lr_t * m1 / (sqrtf(v1) + 1e-8f);
    master[p] = v;
    int layer, o, i;
    if (is_weight(p, &layer, &o, &i)) store_weight(wb, layer, o, i, v);
}

// bfloat16 copies of the master weights; with `export_` non-null also the
// parameters as the network evaluates them.
__global__ void __launch_bounds__(256) k_sync(const float* __restrict__ master, Weights wb, float* export_) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N_PARAMS) return;
    const float v = master[p];
    int layer, o, i;
    const bool w = is_weight(p, &layer, &o, &i);
    if (w) store_weight(wb, layer, o, i, v);
    if (export_) export_[p] = w ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

}  // namespace

cudaError_t launch_features(const Geom& g, const WinIn* wins, const int32_t* chunk_win, int32_t n_chunks,
                            const Ev* ev, int32_t* counts, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_features<<<n_chunks, FEAT_THREADS, 0, s>>>(g, wins, chunk_win, ev, counts);
    return cudaGetLastError();
}

cudaError_t launch_feature_norm(int32_t n_windows, const int32_t* counts, const WinIn* wins, float* feat,
                                cudaStream_t s) {
    if (n_windows <= 0) return cudaSuccess;
    k_feature_norm<<<n_windows, FEATURES, 0, s>>>(counts, wins, feat);
    return cudaGetLastError();
}

cudaError_t launch_warm(const Geom& g, int32_t n_windows, const int32_t* counts, const WinIn* wins,
                        WinParams* params, const MlpDev& m, cudaStream_t s) {
    (void)g;
    if (n_windows <= 0) return cudaSuccess;
    k_warm<<<n_windows, MLP_H, 0, s>>>(n_windows, counts, wins, params, m);
    return cudaGetLastError();
}

}  // namespace dd

// ------------------------------------------------------------------ model

struct dd_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* master = nullptr;        // binary32 parameters ([out][in] matrices)
    float* mom = nullptr;           // Adam moments
    float* vel = nullptr;
    float* grad = nullptr;
    float* exp = nullptr;           // export buffer (get_params)
    float* loss = nullptr;
    dd::Weights wb{};
    int64_t step = 0;
    // training activations for up to cap samples
    int32_t cap = 0;
    float *h1 = nullptr, *h2 = nullptr, *out = nullptr, *gout = nullptr, *g1 = nullptr, *g2 = nullptr;
};

namespace {

constexpr int NP = DD_MLP_PARAMS;
constexpr int B_MAX = 4096;

template <class T>
void release(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_acts(dd_mlp* m) {
    release(m->h1);
    release(m->h2);
    release(m->out);
    release(m->gout);
    release(m->g1);
    release(m->g2);
    m->cap = 0;
}

int ensure_acts(dd_mlp* m, int32_t B) {
    if (B <= m->cap) return DD_OK;
    free_acts(m);
    const size_t n = (size_t)B;
    if (cudaMalloc((void**)&m->h1, sizeof(float) * n * dd::MLP_H) != cudaSuccess ||
        cudaMalloc((void**)&m->h2, sizeof(float) * n * dd::MLP_H) != cudaSuccess ||
        cudaMalloc((void**)&m->g1, sizeof(float) * n * dd::MLP_H) != cudaSuccess ||
        cudaMalloc((void**)&m->g2, sizeof(float) * n * dd::MLP_H) != cudaSuccess ||
        cudaMalloc((void**)&m->out, sizeof(float) * n * dd::MLP_OUT) != cudaSuccess ||
        cudaMalloc((void**)&m->gout, sizeof(float) * n * dd::MLP_OUT) != cudaSuccess) {
        free_acts(m);
        return DD_ERR_OOM;
    }
    m->cap = B;
    return DD_OK;
}

dd::MlpDev view(const dd_mlp* m) {
    dd::MlpDev v;
    v.w1t = m->wb.w1t;
    v.w2t = m->wb.w2t;
    v.w3t = m->wb.w3t;
    v.b1 = m->master + dd::P_B1;
    v.b2 = m->master + dd::P_B2;
    v.b3 = m->master + dd::P_B3;
    return v;
}

int sync_weights(dd_mlp* m, float* export_) {
    dd::k_sync<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->master, m->wb, export_);
    return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}

void destroy(dd_mlp* m) {
    release(m->master);
    release(m->mom);
    release(m->vel);
    release(m->grad);
    release(m->exp);
    release(m->loss);
    release(m->wb.w1);
    release(m->wb.w2);
    release(m->wb.w3);
    release(m->wb.w1t);
    release(m->wb.w2t);
    release(m->wb.w3t);
    free_acts(m);
    delete m;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) for the initial weights.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int upload(dd_mlp* m, const float* host) {
    if (cudaMemcpyAsync(m->master, host, sizeof(float) * NP, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->mom, 0, sizeof(float) * NP, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->vel, 0, sizeof(float) * NP, m->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    int rc = sync_weights(m, nullptr);
    if (rc) return rc;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}

int grad_impl(dd_mlp* m, const float* X, const float* u_star, int32_t B, float* grad, float* loss) {
    if (B < 1 || B > B_MAX || !X || !u_star || !grad) return DD_ERR_ARG;
    int rc = ensure_acts(m, B);
    if (rc) return rc;
    const dd::MlpDev v = view(m);
    dd::k_fwd<<<B, dd::MLP_H, 0, m->stream>>>(v, X, m->h1, m->h2, m->out);
    dd::k_loss<<<1, dd::LOSS_THREADS, 0, m->stream>>>(B, m->out, u_star, m->gout, loss);
    dd::k_back<<<B, dd::MLP_H, 0, m->stream>>>(m->wb.w2, m->wb.w3, m->h1, m->h2, m->gout, m->g1, m->g2);
    dd::k_wgrad<<<(NP + 255) / 256, 256, 0, m->stream>>>(B, X, m->h1, m->h2, m->g1, m->g2, m->gout, grad);
    return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}

}  // namespace

namespace dd {
bool mlp_device_view(const ::dd_mlp* m, MlpDev* out, int* device) {
    if (!m) return false;
    *out = view(m);
    *device = m->device;
    return true;
}
}  // namespace dd

extern "C" {

int dd_mlp_create(uint64_t seed, dd_mlp** out) {
    if (!out) return DD_ERR_ARG;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
        !(prop.major == 10 && prop.minor == 3))
        return DD_ERR_NO_DEVICE;
    dd_mlp* m = new (std::nothrow) dd_mlp();
    if (!m) return DD_ERR_OOM;
    m->device = dev;
    bool ok = cudaMalloc((void**)&m->master, sizeof(float) * NP) == cudaSuccess &&
              cudaMalloc((void**)&m->mom, sizeof(float) * NP) == cudaSuccess &&
              cudaMalloc((void**)&m->vel, sizeof(float) * NP) == cudaSuccess &&
              cudaMalloc((void**)&m->grad, sizeof(float) * NP) == cudaSuccess &&
              cudaMalloc((void**)&m->exp, sizeof(float) * NP) == cudaSuccess &&
              cudaMalloc((void**)&m->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w1, 2 * dd::MLP_H * dd::FEATURES) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w1t, 2 * dd::MLP_H * dd::FEATURES) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w2, 2 * dd::MLP_H * dd::MLP_H) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w2t, 2 * dd::MLP_H * dd::MLP_H) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w3, 2 * dd::MLP_OUT * dd::MLP_H) == cudaSuccess &&
              cudaMalloc((void**)&m->wb.w3t, 2 * dd::MLP_OUT * dd::MLP_H) == cudaSuccess;
    if (!ok) {
        destroy(m);
        return DD_ERR_OOM;
    }
    // Uniform in +-sqrt(6 / fan_in) (fan_in = 128 for every layer); biases 0,
    // except the log half-width's, which starts at log(0.05).
    std::vector<float> p(NP, 0.0f);
    uint64_t s = seed;
    const float a = std::sqrt(6.0f / 128.0f);
    for (int i = 0; i < NP; i++) {
        const bool bias = (i >= dd::P_B1 && i < dd::P_W2) || (i >= dd::P_B2 && i < dd::P_W3) || i >= dd::P_B3;
        if (bias) continue;
        const float u = (float)(splitmix(s) >> 40) * (1.0f / 16777216.0f);
        p[i] = (2.0f * u - 1.0f) * a;
    }
    p[dd::P_B3 + 1] = std::log(0.05f);
    const int rc = upload(m, p.data());
    if (rc) {
        destroy(m);
        return rc;
    }
    *out = m;
    return DD_OK;
}

void dd_mlp_destroy(dd_mlp* m) {
    if (m) destroy(m);
}

int dd_mlp_set_stream(dd_mlp* m, void* stream) {
    if (!m) return DD_ERR_ARG;
    m->stream = (cudaStream_t)stream;
    return DD_OK;
}

int dd_mlp_get_params(dd_mlp* m, float* params, int64_t n) {
    if (!m || !params || n != NP) return DD_ERR_ARG;
    int rc = sync_weights(m, m->exp);
    if (rc) return rc;
    if (cudaMemcpyAsync(params, m->exp, sizeof(float) * NP, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    return DD_OK;
}

int dd_mlp_set_params(dd_mlp* m, const float* params, int64_t n) {
    if (!m || !params || n != NP) return DD_ERR_ARG;
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(params[i])) return DD_ERR_ARG;
    m->step = 0;
    return upload(m, params);
}

int dd_mlp_save(dd_mlp* m, const char* path) {
    if (!m || !path) return DD_ERR_ARG;
    std::vector<float> p(NP);
    if (cudaMemcpyAsync(p.data(), m->master, sizeof(float) * NP, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return DD_ERR_CUDA;
    unsigned char hdr[32];
    std::memset(hdr, 0, sizeof(hdr));
    std::memcpy(hdr, "DDMLP001", 8);
    const int64_t np = NP, st = m->step;
    std::memcpy(hdr + 8, &np, 8);
    std::memcpy(hdr + 16, &st, 8);
    FILE* f = std::fopen(path, "wb");
    if (!f) return DD_ERR_ARG;
    const bool ok = std::fwrite(hdr, 1, 32, f) == 32 && std::fwrite(p.data(), sizeof(float), NP, f) == (size_t)NP;
    return (std::fclose(f) == 0 && ok) ? DD_OK : DD_ERR_ARG;
}

int dd_mlp_load(dd_mlp* m, const char* path) {
    if (!m || !path) return DD_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return DD_ERR_ARG;
    unsigned char hdr[32];
    std::vector<float> p(NP);
    bool ok = std::fread(hdr, 1, 32, f) == 32;
    int64_t np = 0, st = 0;
    if (ok) {
        std::memcpy(&np, hdr + 8, 8);
        std::memcpy(&st, hdr + 16, 8);
        ok = std::memcmp(hdr, "DDMLP001", 8) == 0 && np == NP &&
             std::fread(p.data(), sizeof(float), NP, f) == (size_t)NP;
    }
    std::fclose(f);
    if (!ok) return DD_ERR_ARG;
    for (float v : p)
        if (!std::isfinite(v)) return DD_ERR_ARG;
    const int rc = upload(m, p.data());
    if (rc == DD_OK) m->step = st;
    return rc;
}

int dd_mlp_forward(dd_mlp* m, const float* X, int32_t B, float* out) {
    if (!m || B < 0 || (B > 0 && (!X || !out))) return DD_ERR_ARG;
    if (B == 0) return DD_OK;
    int rc = ensure_acts(m, B);
    if (rc) return rc;
    dd::k_fwd<<<B, dd::MLP_H, 0, m->stream>>>(view(m), X, m->h1, m->h2, out);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) return DD_ERR_CUDA;
    return DD_OK;
}

int dd_mlp_grad(dd_mlp* m, const float* X, const float* u_star, int32_t B, float* grad, float* loss) {
    if (!m || !loss) return DD_ERR_ARG;
    return grad_impl(m, X, u_star, B, grad, loss);
}

int dd_mlp_train_step(dd_mlp* m, const float* X, const float* u_star, int32_t B, float lr, float* loss) {
    if (!m || !std::isfinite(lr) || !(lr > 0.0f)) return DD_ERR_ARG;
    int rc = grad_impl(m, X, u_star, B, m->grad, loss);
    if (rc) return rc;
    m->step++;
    const double t = (double)m->step;
    const float lr_t = (float)(lr * std::sqrt(1.0 - std::pow(0.999, t)) / (1.0 - std::pow(0.9, t)));
    dd::k_adam<<<(NP + 255) / 256, 256, 0, m->stream>>>(lr_t, m->grad, m->master, m->mom, m->vel, m->wb);
    return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}

}  // extern "C"
