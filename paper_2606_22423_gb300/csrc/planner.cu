// Learned planner: a small FP32 network (4 -> 64 -> 64 -> S, ReLU) that
// predicts the log time of each scan strategy for a column from four
// features, trained on the GPU by these kernels (forward, backward, Adam).
// Every scan strategy returns the same exact result, so the planner only
// affects speed.
//
// Layout: parameters are one flat float array [W1 (4x64), b1, W2 (64x64), b2,
// W3 (64xS), b3], W_l row-major with shape (fan_in, fan_out).  Gradients of
// a weight are reduced over the batch by one thread each (no atomics, so a
// training step is deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gbscan.h"
#include "batch_kernels.cuh"

void gb_set_last_error(const char* msg);

namespace {

constexpr int kIn = 4;
constexpr int kHid = 64;
constexpr uint32_t kCkptMagic = 0x4e4c5047u;  // "GPLN"
constexpr uint32_t kCkptVersion = 1;

scan_status pfail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);
    return s;
}

scan_status pcuda(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    gb_set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA;
}

#define PL_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return pcuda(e_, #call); \
    } while (0)

// z = in W + b (and a = relu(z) when a != null); one thread per (row, unit)
__global__ void k_dense_fwd(const float* __restrict__ in, int K, const float* __restrict__ W,
                            const float* __restrict__ b, int M, int rows, float* __restrict__ z,
                            float* __restrict__ a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * M) return;
    const int n = i / M, m = i - n * M;
    float acc = b[m];
    for (int k = 0; k < K; ++k) acc = fmaf(in[n * K + k], W[k * M + m], acc);
    z[i] = acc;
    if (a) a[i] = acc > 0.f ? acc : 0.f;
}

// dY = 2 (Y - T) / count; loss partial sums into *loss (one atomic per block)
__global__ void k_mse_grad(const float* __restrict__ y, const float* __restrict__ t, int count,
                           float* __restrict__ dy, float* __restrict__ loss)
{
    __shared__ float red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (i < count) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / static_cast<float>(count);
        e = d * d / static_cast<float>(count);
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0]);
}

// dW[k][m] = sum_n in[n][k] dz[n][m] (threads k < K) and db[m] = sum_n dz[n][m] (k == K)
__global__ void k_dense_bwd_w(const float* __restrict__ in, int K, const float* __restrict__ dz, int M,
                              int rows, float* __restrict__ dW, float* __restrict__ db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (K + 1) * M) return;
    const int k = i / M, m = i - k * M;
    float acc = 0.f;
    if (k < K) {
        for (int n = 0; n < rows; ++n) acc = fmaf(in[n * K + k], dz[n * M + m], acc);
        dW[k * M + m] = acc;
    } else {
        for (int n = 0; n < rows; ++n) acc += dz[n * M + m];
        db[m] = acc;
    }
}

// dprev[n][k] = [zprev[n][k] > 0] * sum_m dz[n][m] W[k][m]
__global__ void k_dense_bwd_in(const float* __restrict__ dz, int M, const float* __restrict__ W, int K,
                               const float* __restrict__ zprev, int rows, float* __restrict__ dprev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * K) return;
    const int n = i / K, k = i - n * K;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) acc = fmaf(dz[n * M + m], W[k * M + m], acc);
    dprev[i] = zprev[i] > 0.f ? acc : 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// The first strategy (in index order) whose predicted log time is within
// `margin` of the row's minimum: with margin 0 the argmin (ties to the lower
// index); with margin > 0 predicted gains below the margin do not move the
// plan off the earlier (simpler) strategies.
__global__ void k_argmin_rows(const float* __restrict__ y, int rows, int S, float margin,
                              int32_t* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= rows) return;
    float lo = y[n * S];
    for (int s = 1; s < S; ++s) lo = fminf(lo, y[n * S + s]);
    int best = 0;
    while (best < S - 1 && y[n * S + best] > lo + margin) ++best;
    out[n] = best;
}

// Same rule on y + prior: the network predicts a correction to a prior
// estimate of each strategy's log time (the law's), row-major rows x S.
__global__ void k_argmin_rows_prior(const float* __restrict__ y, const float* __restrict__ prior, int rows,
                                    int S, float margin, int32_t* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= rows) return;
    float lo = y[n * S] + prior[n * S];
    for (int s = 1; s < S; ++s) lo = fminf(lo, y[n * S + s] + prior[n * S + s]);
    int best = 0;
    while (best < S - 1 && y[n * S + best] + prior[n * S + best] > lo + margin) ++best;
    out[n] = best;
}

// Bounds of the features the network was trained on: outside them its
// predictions are extrapolations, and the fallback decides.
struct FeatureBox {
    float lo[kIn], hi[kIn];
    int on;
};

// The fallback's choice unless the network is confident and on familiar
// ground: per row whose features lie inside the box, the strategy the network
// predicts fastest among those available (the fallback's log time below
// kUnavailable) replaces the fallback's choice only if its predicted log time
// is lower than the network's prediction for the fallback's choice by more
// than `margin`.
constexpr float kUnavailable = 29.0f;
__global__ void k_choose_guarded(const float* __restrict__ x, const float* __restrict__ y,
                                 const int32_t* __restrict__ fallback, const float* __restrict__ fallback_log_ms,
                                 int rows, int S, float margin, FeatureBox box, int32_t* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= rows) return;
    const int f = fallback[n];
    if (box.on) {
        for (int k = 0; k < kIn; ++k) {
            const float v = x[n * kIn + k];
            if (v < box.lo[k] || v > box.hi[k]) {
                out[n] = f;
                return;
            }
        }
    }
    int best = f;
    for (int s = 0; s < S; ++s) {
        if (fallback_log_ms[n * S + s] >= kUnavailable) continue;
        if (y[n * S + s] < y[n * S + best]) best = s;
    }
    out[n] = (y[n * S + best] < y[n * S + f] - margin) ? best : f;
}

inline unsigned blocks_for(long long n, int t = 256) { return static_cast<unsigned>((n + t - 1) / t); }

// splitmix64 (Steele, Lea, Flood 2014) for the deterministic initial weights
uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

struct scan_planner {
    int S = 4;
    size_t nparams = 0;
    float* d_params = nullptr;
    float* d_grads = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    int step = 0;
    int cap = 0;  // rows of the activation workspace
    float* d_ws = nullptr;
    float* d_loss = nullptr;

    size_t off_W(int l) const
    {
        const int fi[3] = {kIn, kHid, kHid}, fo[3] = {kHid, kHid, S};
        size_t o = 0;
        for (int i = 0; i < l; ++i) o += static_cast<size_t>(fi[i]) * fo[i] + fo[i];
        return o;
    }
    size_t off_b(int l) const
    {
        const int fi[3] = {kIn, kHid, kHid}, fo[3] = {kHid, kHid, S};
        return off_W(l) + static_cast<size_t>(fi[l]) * fo[l];
    }
};

namespace {

scan_status ensure_ws(scan_planner* pl, uint32_t rows)
{
    if (static_cast<int>(rows) <= pl->cap) return SCAN_OK;
    if (pl->d_ws) cudaFree(pl->d_ws);
    pl->d_ws = nullptr;
    // z1 a1 z2 a2 y dy dz2 dz1 : 6 x 64 + 2 x S floats per row
    const size_t per = 6ull * kHid + 2ull * pl->S;
    PL_CUDA(cudaMalloc(&pl->d_ws, per * rows * sizeof(float)));
    pl->cap = static_cast<int>(rows);
    return SCAN_OK;
}

struct Acts {
    float *z1, *a1, *z2, *a2, *y, *dy, *dz2, *dz1;
};

Acts acts(const scan_planner* pl)
{
    Acts a;
    float* p = pl->d_ws;
    const size_t r = static_cast<size_t>(pl->cap);
    a.z1 = p; p += r * kHid;
    a.a1 = p; p += r * kHid;
    a.z2 = p; p += r * kHid;
    a.a2 = p; p += r * kHid;
    a.dz2 = p; p += r * kHid;
    a.dz1 = p; p += r * kHid;
    a.y = p; p += r * pl->S;
    a.dy = p;
    return a;
}

void forward(const scan_planner* pl, const float* x, int rows, const Acts& a, float* y, cudaStream_t st)
{
    const float* P = pl->d_params;
    k_dense_fwd<<<blocks_for(1ll * rows * kHid), 256, 0, st>>>(x, kIn, P + pl->off_W(0), P + pl->off_b(0), kHid,
                                                              rows, a.z1, a.a1);
    k_dense_fwd<<<blocks_for(1ll * rows * kHid), 256, 0, st>>>(a.a1, kHid, P + pl->off_W(1), P + pl->off_b(1),
                                                              kHid, rows, a.z2, a.a2);
    k_dense_fwd<<<blocks_for(1ll * rows * pl->S), 256, 0, st>>>(a.a2, kHid, P + pl->off_W(2), P + pl->off_b(2),
                                                               pl->S, rows, y, nullptr);
}

void backward(const scan_planner* pl, const float* x, const float* t, int rows, const Acts& a,
              cudaStream_t st)
{
    const float* P = pl->d_params;
    float* G = pl->d_grads;
    const int S = pl->S;
    k_mse_grad<<<blocks_for(1ll * rows * S), 256, 0, st>>>(a.y, t, rows * S, a.dy, pl->d_loss);
    k_dense_bwd_w<<<blocks_for(1ll * (kHid + 1) * S), 256, 0, st>>>(a.a2, kHid, a.dy, S, rows,
                                                                   G + pl->off_W(2), G + pl->off_b(2));
    k_dense_bwd_in<<<blocks_for(1ll * rows * kHid), 256, 0, st>>>(a.dy, S, P + pl->off_W(2), kHid, a.z2, rows,
                                                                 a.dz2);
    k_dense_bwd_w<<<blocks_for(1ll * (kHid + 1) * kHid), 256, 0, st>>>(a.a1, kHid, a.dz2, kHid, rows,
                                                                      G + pl->off_W(1), G + pl->off_b(1));
    k_dense_bwd_in<<<blocks_for(1ll * rows * kHid), 256, 0, st>>>(a.dz2, kHid, P + pl->off_W(1), kHid, a.z1,
                                                                 rows, a.dz1);
    k_dense_bwd_w<<<blocks_for(1ll * (kIn + 1) * kHid), 256, 0, st>>>(x, kIn, a.dz1, kHid, rows,
                                                                     G + pl->off_W(0), G + pl->off_b(0));
}

}  // namespace

extern "C" {

scan_status scan_planner_create(uint32_t n_strategies, uint64_t seed, scan_planner** out)
{
    gb_set_last_error("");
    if (!out || n_strategies < 1 || n_strategies > 16) return pfail(SCAN_EINVAL, "bad planner shape");
    auto* pl = new (std::nothrow) scan_planner();
    if (!pl) return pfail(SCAN_ENOMEM, "host allocation failed");
    pl->S = static_cast<int>(n_strategies);
    pl->nparams = pl->off_b(2) + pl->S;
    std::vector<float> h(pl->nparams, 0.f);
    uint64_t s = seed;
    const int fi[3] = {kIn, kHid, kHid}, fo[3] = {kHid, kHid, pl->S};
    for (int l = 0; l < 3; ++l) {  // He-uniform weights, zero biases
        const float lim = std::sqrt(6.f / static_cast<float>(fi[l]));
        for (int i = 0; i < fi[l] * fo[l]; ++i) {
            const double u = static_cast<double>(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            h[pl->off_W(l) + i] = static_cast<float>((2.0 * u - 1.0) * lim);
        }
    }
    cudaError_t e = cudaMalloc(&pl->d_params, 4 * pl->nparams * sizeof(float) + 16);
    if (e != cudaSuccess) {
        delete pl;
        return pcuda(e, "cudaMalloc(planner)");
    }
    pl->d_grads = pl->d_params + pl->nparams;
    pl->d_m = pl->d_grads + pl->nparams;
    pl->d_v = pl->d_m + pl->nparams;
    pl->d_loss = pl->d_v + pl->nparams;
    e = cudaMemset(pl->d_params, 0, 4 * pl->nparams * sizeof(float) + 16);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_params, h.data(), pl->nparams * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(pl->d_params);
        delete pl;
        return pcuda(e, "planner init");
    }
    *out = pl;
    return SCAN_OK;
}

scan_status scan_planner_destroy(scan_planner* pl)
{
    if (!pl) return SCAN_OK;
    cudaDeviceSynchronize();
    if (pl->d_params) cudaFree(pl->d_params);
    if (pl->d_ws) cudaFree(pl->d_ws);
    delete pl;
    return SCAN_OK;
}

uint64_t scan_planner_param_count(const scan_planner* pl) { return pl ? pl->nparams : 0; }

scan_status scan_planner_get_params(const scan_planner* pl, float* host_params)
{
    if (!pl || !host_params) return pfail(SCAN_EINVAL, "null pointer");
    PL_CUDA(cudaMemcpy(host_params, pl->d_params, pl->nparams * sizeof(float), cudaMemcpyDeviceToHost));
    return SCAN_OK;
}

scan_status scan_planner_set_params(scan_planner* pl, const float* host_params)
{
    if (!pl || !host_params) return pfail(SCAN_EINVAL, "null pointer");
    PL_CUDA(cudaMemcpy(pl->d_params, host_params, pl->nparams * sizeof(float), cudaMemcpyHostToDevice));
    PL_CUDA(cudaMemset(pl->d_m, 0, 2 * pl->nparams * sizeof(float)));
    pl->step = 0;
    return SCAN_OK;
}

scan_status scan_planner_forward(scan_planner* pl, const float* dev_x, uint32_t rows, float* dev_y, void* stream)
{
    gb_set_last_error("");
    if (!pl || (rows && (!dev_x || !dev_y))) return pfail(SCAN_EINVAL, "null pointer");
    if (!rows) return SCAN_OK;
    scan_status s = ensure_ws(pl, rows);
    if (s != SCAN_OK) return s;
    forward(pl, dev_x, static_cast<int>(rows), acts(pl), dev_y, static_cast<cudaStream_t>(stream));
    PL_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_planner_gradients(scan_planner* pl, const float* dev_x, const float* dev_t, uint32_t rows,
                                   float* dev_grads, void* stream, float* host_loss)
{
    gb_set_last_error("");
    if (!pl || !rows || !dev_x || !dev_t) return pfail(SCAN_EINVAL, "null pointer or empty batch");
    scan_status s = ensure_ws(pl, rows);
    if (s != SCAN_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Acts a = acts(pl);
    PL_CUDA(cudaMemsetAsync(pl->d_loss, 0, sizeof(float), st));
    forward(pl, dev_x, static_cast<int>(rows), a, a.y, st);
    backward(pl, dev_x, dev_t, static_cast<int>(rows), a, st);
    PL_CUDA(cudaGetLastError());
    if (dev_grads)
        PL_CUDA(cudaMemcpyAsync(dev_grads, pl->d_grads, pl->nparams * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (host_loss) {
        PL_CUDA(cudaMemcpyAsync(host_loss, pl->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        PL_CUDA(cudaStreamSynchronize(st));
    }
    return SCAN_OK;
}

scan_status scan_planner_train_step(scan_planner* pl, const float* dev_x, const float* dev_t, uint32_t rows,
                                    float lr, void* stream, float* host_loss)
{
    scan_status s = scan_planner_gradients(pl, dev_x, dev_t, rows, nullptr, stream, host_loss);
    if (s != SCAN_OK) return s;
    pl->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, static_cast<float>(pl->step));
    const float bc2 = 1.f - std::pow(b2, static_cast<float>(pl->step));
    k_adam<<<blocks_for(static_cast<long long>(pl->nparams)), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        pl->d_params, pl->d_grads, pl->d_m, pl->d_v, static_cast<int>(pl->nparams), lr, b1, b2, 1e-8f, bc1, bc2);
    PL_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_planner_choose_margin(scan_planner* pl, const float* dev_x, uint32_t rows, float margin,
                                       int32_t* dev_choice, void* stream)
{
    if (!(margin >= 0.0f)) return pfail(SCAN_EINVAL, "margin must be >= 0");
    scan_status s = ensure_ws(pl, rows ? rows : 1);
    if (s != SCAN_OK) return s;
    const Acts a = acts(pl);
    s = scan_planner_forward(pl, dev_x, rows, a.y, stream);
    if (s != SCAN_OK || !rows) return s;
    k_argmin_rows<<<blocks_for(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(a.y, static_cast<int>(rows),
                                                                                  pl->S, margin, dev_choice);
    PL_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_planner_choose_prior(scan_planner* pl, const float* dev_x, uint32_t rows, float margin,
                                      const float* dev_prior, int32_t* dev_choice, void* stream)
{
    if (!pl || (rows && (!dev_x || !dev_prior || !dev_choice))) return pfail(SCAN_EINVAL, "null pointer");
    if (!(margin >= 0.0f)) return pfail(SCAN_EINVAL, "margin must be >= 0");
    scan_status s = ensure_ws(pl, rows ? rows : 1);
    if (s != SCAN_OK) return s;
    const Acts a = acts(pl);
    s = scan_planner_forward(pl, dev_x, rows, a.y, stream);
    if (s != SCAN_OK || !rows) return s;
    k_argmin_rows_prior<<<blocks_for(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        a.y, dev_prior, static_cast<int>(rows), pl->S, margin, dev_choice);
    PL_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_planner_choose_guarded(scan_planner* pl, const float* dev_x, uint32_t rows, float margin,
                                        const int32_t* dev_fallback, const float* dev_fallback_log_ms,
                                        const float* host_feature_box, int32_t* dev_choice, void* stream)
{
    if (!pl || (rows && (!dev_x || !dev_fallback || !dev_fallback_log_ms || !dev_choice)))
        return pfail(SCAN_EINVAL, "null pointer");
    if (!(margin >= 0.0f)) return pfail(SCAN_EINVAL, "margin must be >= 0");
    scan_status s = ensure_ws(pl, rows ? rows : 1);
    if (s != SCAN_OK) return s;
    const Acts a = acts(pl);
    s = scan_planner_forward(pl, dev_x, rows, a.y, stream);
    if (s != SCAN_OK || !rows) return s;
    FeatureBox box{};
    box.on = host_feature_box != nullptr;
    for (int k = 0; k < kIn && box.on; ++k) {
        box.lo[k] = host_feature_box[k];
        box.hi[k] = host_feature_box[kIn + k];
    }
    k_choose_guarded<<<blocks_for(rows), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        dev_x, a.y, dev_fallback, dev_fallback_log_ms, static_cast<int>(rows), pl->S, margin, box, dev_choice);
    PL_CUDA(cudaGetLastError());
    return SCAN_OK;
}

scan_status scan_planner_choose(scan_planner* pl, const float* dev_x, uint32_t rows, int32_t* dev_choice,
                                void* stream)
{
    return scan_planner_choose_margin(pl, dev_x, rows, 0.0f, dev_choice, stream);
}

scan_status scan_planner_save(const scan_planner* pl, const char* path)
{
    if (!pl || !path) return pfail(SCAN_EINVAL, "null pointer");
    std::vector<float> h(pl->nparams);
    scan_status s = scan_planner_get_params(pl, h.data());
    if (s != SCAN_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return pfail(SCAN_EINVAL, "cannot open checkpoint for writing");
    const uint32_t hdr[4] = {kCkptMagic, kCkptVersion, static_cast<uint32_t>(pl->S),
                             static_cast<uint32_t>(pl->nparams)};
    const bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
                    std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    std::fclose(f);
    return ok ? SCAN_OK : pfail(SCAN_EINVAL, "short write of checkpoint");
}

scan_status scan_planner_load(scan_planner* pl, const char* path)
{
    if (!pl || !path) return pfail(SCAN_EINVAL, "null pointer");
    FILE* f = std::fopen(path, "rb");
    if (!f) return pfail(SCAN_EINVAL, "cannot open checkpoint");
    uint32_t hdr[4] = {0, 0, 0, 0};
    std::vector<float> h(pl->nparams);
    bool ok = std::fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == kCkptMagic && hdr[1] == kCkptVersion &&
              hdr[2] == static_cast<uint32_t>(pl->S) && hdr[3] == pl->nparams &&
              std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) return pfail(SCAN_EINVAL, "checkpoint header or size does not match this planner");
    return scan_planner_set_params(pl, h.data());
}

}  // extern "C"
