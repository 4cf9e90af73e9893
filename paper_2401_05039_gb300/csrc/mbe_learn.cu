// Learned schedule: per-root features, core numbers, the 8 -> 64 -> 64 -> 1
// cost network (FP16 weights and activations, FP32 accumulation) with its
// training kernels, and the execution order it produces.
//
// The network never touches enumeration results: it only orders (and
// pre-splits) root tasks, and every order gives the same count, hash and
// nodes. The static order is the fallback when a prediction is not finite.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mbe.h"
#include "mbe_internal.h"
#include "mbe_learn.h"
#include "mbe_prep.h"
#include "mbe_runtime.h"

namespace mbe {
namespace {

constexpr int kF = 8, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH,
              kOffB3 = kOffW3 + kH, kNP = kOffB3 + 1;
static_assert(kNP == 4801, "parameter count");

constexpr unsigned kFull = 0xffffffffu;

// --------------------------------------------------------------- features
// One warp per root r: |N2(r)|, |P0|, |Q0| through the CSC lists of N(r)
// (a per-warp stamp array marks U vertices already seen for this root), and
// the sum / max of the degrees of N(r).
__global__ void root_features_kernel(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                     const int32_t *v_adj, int32_t nU, const int32_t *larger, const int32_t *core,
                                     int32_t *mark, int64_t mark_stride, int32_t *raw, float *feat)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t *stamp = mark + (int64_t)wid * mark_stride;
    for (int r = wid; r < nU; r += warps) {
        const int ro = u_off[r], d = u_off[r + 1] - ro;
        int n2 = 0, p0 = 0;
        long long sdeg = 0;
        int mdeg = 0;
        for (int j0 = 0; j0 < d; j0 += 32) {
            const int j = j0 + lane;
            const bool vj = j < d;
            const int w = vj ? u_adj[ro + j] : 0;
            const int wo = vj ? v_off[w] : 0;
            const int wd = vj ? v_off[w + 1] - wo : 0;
            sdeg += wd;
            mdeg = max(mdeg, wd);
            int incl = wd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            const int excl = incl - wd;
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                int s = 0;
#pragma unroll
                for (int b = 16; b > 0; b >>= 1) {
                    int cand = s + b;
                    int ex = __shfl_sync(kFull, excl, cand & 31);
                    if (cand < 32 && ex <= q) s = cand;
                }
                const int ws = __shfl_sync(kFull, wo, s), es = __shfl_sync(kFull, excl, s);
                if (q < total) {
                    const int u = v_adj[ws + (q - es)];
                    if (u != r && atomicExch(stamp + u, r) != r) {
                        ++n2;
                        const int du = u_off[u + 1] - u_off[u];
                        if (du > d || (du == d && u > r)) ++p0;
                    }
                }
            }
        }
        n2 = __reduce_add_sync(kFull, (unsigned)n2);
        p0 = __reduce_add_sync(kFull, (unsigned)p0);
        for (int o = 16; o > 0; o >>= 1) {
            sdeg += __shfl_xor_sync(kFull, sdeg, o);
            mdeg = max(mdeg, __shfl_xor_sync(kFull, mdeg, o));
        }
        if (lane == 0) {
            int32_t v[kF] = {d, n2, p0, n2 - p0, core[r], (int32_t)min(sdeg, (long long)INT32_MAX), mdeg,
                             d > 0 ? larger[d] : 0};
            if (d == 0)
                for (int k = 0; k < kF; ++k) v[k] = 0;
            for (int k = 0; k < kF; ++k) raw[(int64_t)r * kF + k] = v[k];
            for (int k = 0; k < 7; ++k) feat[(int64_t)r * kF + k] = d > 0 ? log1pf((float)v[k]) : 0.f;
            feat[(int64_t)r * kF + 7] = d > 0 ? (float)v[7] / (float)nU : 0.f;
        }
    }
}

// ----------------------------------------------------------- core numbers
// G as a general graph: vertex x < nU is u = x, vertex nU + v is v.
__global__ void core_init_kernel(const int32_t *u_off, const int32_t *v_off, int32_t nU, int32_t nV, int32_t *deg,
                                 int32_t *alive)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nU + nV; x += gridDim.x * blockDim.x) {
        deg[x] = x < nU ? u_off[x + 1] - u_off[x] : v_off[x - nU + 1] - v_off[x - nU];
        alive[x] = 1;
    }
}

// One peeling round at `level`: every live vertex of remaining degree <=
// level gets core number `level` and leaves, lowering its neighbours'
// degrees. A vertex whose degree drops to <= level during the round may
// leave in the same round or the next: either way at this level.
__global__ void core_peel_kernel(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                 const int32_t *v_adj, int32_t nU, int32_t nV, int32_t level, int32_t *deg,
                                 int32_t *alive, int32_t *core, int32_t *removed)
{
    int local = 0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nU + nV; x += gridDim.x * blockDim.x) {
        if (!alive[x] || deg[x] > level) continue;
        alive[x] = 0;
        core[x] = level;
        ++local;
        if (x < nU) {
            for (int k = u_off[x]; k < u_off[x + 1]; ++k) atomicSub(deg + nU + u_adj[k], 1);
        } else {
            const int v = x - nU;
            for (int k = v_off[v]; k < v_off[v + 1]; ++k) atomicSub(deg + v_adj[k], 1);
        }
    }
    if (local) atomicAdd(removed, local);
}

// ---------------------------------------------------------------- network
__device__ __forceinline__ float h2f(__half h) { return __half2float(h); }
__device__ __forceinline__ float round16(float x) { return __half2float(__float2half_rn(x)); }

// Loads the FP16 weights and FP32 biases of the network into shared memory.
struct NetSmem {
    __half w1[kH * kF];
    __half w2[kH * kH];
    __half w3[kH];
    float b1[kH], b2[kH], b3;
};

__device__ void load_net(NetSmem &n, const __half *p16, const float *p32)
{
    for (int i = threadIdx.x; i < kH * kF; i += blockDim.x) n.w1[i] = p16[kOffW1 + i];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) n.w2[i] = p16[kOffW2 + i];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        n.w3[i] = p16[kOffW3 + i];
        n.b1[i] = p32[kOffB1 + i];
        n.b2[i] = p32[kOffB2 + i];
    }
    if (threadIdx.x == 0) n.b3 = p32[kOffB3];
    __syncthreads();
}

// Forward of one sample (FP16 operands, FP32 accumulation). Optionally
// stores the FP16 input and hidden activations for the backward pass.
__device__ float forward_one(const NetSmem &n, const float *x32, __half *x16o, __half *h1o, __half *h2o)
{
    float x[kF];
#pragma unroll
    for (int i = 0; i < kF; ++i) {
        __half xh = __float2half_rn(x32[i]);
        x[i] = __half2float(xh);
        if (x16o) x16o[i] = xh;
    }
    float h1[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        float z = n.b1[j];
#pragma unroll
        for (int i = 0; i < kF; ++i) z = fmaf(h2f(n.w1[j * kF + i]), x[i], z);
        h1[j] = round16(fmaxf(z, 0.f));
        if (h1o) h1o[j] = __float2half_rn(h1[j]);
    }
    float y = n.b3;
    for (int k = 0; k < kH; ++k) {
        float z = n.b2[k];
        const __half2 *row = reinterpret_cast<const __half2 *>(n.w2 + k * kH);
#pragma unroll
        for (int j = 0; j < kH / 2; ++j) {
            float2 w = __half22float2(row[j]);
            z = fmaf(w.x, h1[2 * j], z);
            z = fmaf(w.y, h1[2 * j + 1], z);
        }
        const float h2 = round16(fmaxf(z, 0.f));
        if (h2o) h2o[k] = __float2half_rn(h2);
        y = fmaf(h2f(n.w3[k]), h2, y);
    }
    return y;
}

__global__ void mlp_predict_kernel(const __half *p16, const float *p32, const float *X, int32_t n, float *y)
{
    __shared__ NetSmem net;
    load_net(net, p16, p32);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = forward_one(net, X + (int64_t)i * kF, nullptr, nullptr, nullptr);
}

// Training forward over a minibatch (rows idx[b] of X): stores X16, H1, H2
// and dy = 2 (y - t) / B; adds the squared error sum into *loss.
__global__ void mlp_train_forward_kernel(const __half *p16, const float *p32, const float *X, const float *T,
                                         const int32_t *idx, int32_t B, __half *X16, __half *H1, __half *H2,
                                         float *dy, float *loss)
{
    __shared__ NetSmem net;
    load_net(net, p16, p32);
    float se = 0.f;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const int i = idx ? idx[b] : b;
        float y = forward_one(net, X + (int64_t)i * kF, X16 + (int64_t)b * kF, H1 + (int64_t)b * kH,
                              H2 + (int64_t)b * kH);
        float r = y - T[i];
        dy[b] = 2.f * r / (float)B;
        se += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(kFull, se, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, se);
}

// dZ2 = dy W3 [H2 > 0], dZ1 = (dZ2 W2) [H1 > 0], per sample, FP32.
__global__ void mlp_backward_kernel(const __half *p16, const __half *H1, const __half *H2, const float *dy, int32_t B,
                                    float *dZ1, float *dZ2)
{
    __shared__ __half w2[kH * kH];
    __shared__ __half w3[kH];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) w2[i] = p16[kOffW2 + i];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) w3[i] = p16[kOffW3 + i];
    __syncthreads();
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        float dz2[kH];
#pragma unroll
        for (int k = 0; k < kH; ++k) {
            dz2[k] = __half2float(H2[(int64_t)b * kH + k]) > 0.f ? dy[b] * h2f(w3[k]) : 0.f;
            dZ2[(int64_t)b * kH + k] = dz2[k];
        }
        for (int j = 0; j < kH; ++j) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kH; ++k) s = fmaf(dz2[k], h2f(w2[k * kH + j]), s);
            dZ1[(int64_t)b * kH + j] = __half2float(H1[(int64_t)b * kH + j]) > 0.f ? s : 0.f;
        }
    }
}

// Parameter gradients: one thread per parameter, summing over the batch.
__global__ void mlp_grad_kernel(const __half *X16, const __half *H1, const __half *H2, const float *dy,
                                const float *dZ1, const float *dZ2, int32_t B, float *g)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNP) return;
    float s = 0.f;
    if (p < kOffB1) { // W1[j][i]
        const int j = p / kF, i = p % kF;
        for (int b = 0; b < B; ++b) s = fmaf(dZ1[(int64_t)b * kH + j], __half2float(X16[(int64_t)b * kF + i]), s);
    } else if (p < kOffW2) { // b1[j]
        const int j = p - kOffB1;
        for (int b = 0; b < B; ++b) s += dZ1[(int64_t)b * kH + j];
    } else if (p < kOffB2) { // W2[k][j]
        const int k = (p - kOffW2) / kH, j = (p - kOffW2) % kH;
        for (int b = 0; b < B; ++b) s = fmaf(dZ2[(int64_t)b * kH + k], __half2float(H1[(int64_t)b * kH + j]), s);
    } else if (p < kOffW3) { // b2[k]
        const int k = p - kOffB2;
        for (int b = 0; b < B; ++b) s += dZ2[(int64_t)b * kH + k];
    } else if (p < kOffB3) { // W3[k]
        const int k = p - kOffW3;
        for (int b = 0; b < B; ++b) s = fmaf(dy[b], __half2float(H2[(int64_t)b * kH + k]), s);
    } else {
        for (int b = 0; b < B; ++b) s += dy[b];
    }
    g[p] = s;
}

// Adam on the FP32 master weights; the FP16 copy is re-quantised.
__global__ void mlp_adam_kernel(float *p32, __half *p16, float *m, float *v, const float *g, float lr, float b1,
                                float b2, float eps, int32_t step)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNP) return;
    const float gi = g[p];
    const float mi = b1 * m[p] + (1.f - b1) * gi;
    const float vi = b2 * v[p] + (1.f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    const float w = p32[p] - lr * mh / (sqrtf(vh) + eps);
    p32[p] = w;
    p16[p] = __float2half_rn(w);
}

__global__ void to_half_kernel(const float *p32, __half *p16, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p16[i] = __float2half_rn(p32[i]);
}

// Execution-order keys: predicted log cost quantised to 1/256, -1 for
// isolated roots; *bad is set when a prediction is not finite.
__global__ void order_keys_kernel(const float *pred, const int32_t *u_off, int32_t nU, int32_t max_key, int32_t *key,
                                  int32_t *bad)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nU; u += gridDim.x * blockDim.x) {
        if (u_off[u + 1] == u_off[u]) {
            key[u] = -1;
            continue;
        }
        const float p = pred[u];
        if (!isfinite(p)) {
            atomicOr(bad, 1);
            key[u] = 0;
            continue;
        }
        key[u] = (int32_t)fminf(fmaxf(p * 256.f, 0.f), (float)max_key);
    }
}

} // namespace

// ------------------------------------------------------------ host launchers
cudaError_t compute_core_numbers(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                 const int32_t *v_adj, int32_t nU, int32_t nV, int32_t *d_deg, int32_t *d_alive,
                                 int32_t *d_core, int32_t *d_removed, cudaStream_t s)
{
    const int n = nU + nV;
    if (n == 0) return cudaSuccess;
    int blocks = std::min(4 * 152, (n + 255) / 256);
    core_init_kernel<<<blocks, 256, 0, s>>>(u_off, v_off, nU, nV, d_deg, d_alive);
    int remaining = n, level = 0;
    for (int guard = 0; guard < 4 * n + 64 && remaining > 0; ++guard) {
        cudaError_t e = cudaMemsetAsync(d_removed, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        core_peel_kernel<<<blocks, 256, 0, s>>>(u_off, u_adj, v_off, v_adj, nU, nV, level, d_deg, d_alive, d_core,
                                                 d_removed);
        int32_t h = 0;
        e = cudaMemcpyAsync(&h, d_removed, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        if (h == 0) ++level;
        else remaining -= h;
    }
    return remaining == 0 ? cudaGetLastError() : cudaErrorUnknown;
}

cudaError_t compute_root_features(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                  const int32_t *v_adj, int32_t nU, const int32_t *d_larger, const int32_t *d_core,
                                  int32_t *d_mark, int64_t mark_stride, int32_t n_warps, int32_t *d_raw,
                                  float *d_feat, cudaStream_t s)
{
    if (nU == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_mark, 0xff, sizeof(int32_t) * (size_t)mark_stride * n_warps, s);
    if (e != cudaSuccess) return e;
    const int blocks = n_warps / 8;
    root_features_kernel<<<blocks, 256, 0, s>>>(u_off, u_adj, v_off, v_adj, nU, d_larger, d_core, d_mark,
                                                 mark_stride, d_raw, d_feat);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(d_mark, 0xff, sizeof(int32_t) * (size_t)mark_stride * n_warps, s);
    return e;
}

cudaError_t learned_order_keys(const float *d_pred, const int32_t *u_off, int32_t nU, int32_t max_key,
                               int32_t *d_key, int32_t *d_bad, cudaStream_t s)
{
    int blocks = std::max(1, std::min(4 * 152, (nU + 255) / 256));
    order_keys_kernel<<<blocks, 256, 0, s>>>(d_pred, u_off, nU, max_key, d_key, d_bad);
    return cudaGetLastError();
}

} // namespace mbe

// ------------------------------------------------------------------- model
struct mbe_model {
    int device = 0;
    float *p32 = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __half *p16 = nullptr;
    int32_t steps = 0;
    // training scratch, sized for the largest batch seen
    int32_t cap = 0;
    __half *X16 = nullptr, *H1 = nullptr, *H2 = nullptr;
    float *dy = nullptr, *dZ1 = nullptr, *dZ2 = nullptr, *loss = nullptr;
    int32_t *idx = nullptr;

    void free_scratch()
    {
        cudaFree(X16);
        cudaFree(H1);
        cudaFree(H2);
        cudaFree(dy);
        cudaFree(dZ1);
        cudaFree(dZ2);
        cudaFree(loss);
        cudaFree(idx);
        X16 = H1 = H2 = nullptr;
        dy = dZ1 = dZ2 = loss = nullptr;
        idx = nullptr;
        cap = 0;
    }
};

namespace mbe {
namespace {

int ensure_train_scratch(mbe_model *md, int32_t B)
{
    if (md->cap >= B) return MBE_OK;
    md->free_scratch();
    if (cudaMalloc(&md->X16, sizeof(__half) * (size_t)B * kF) != cudaSuccess ||
        cudaMalloc(&md->H1, sizeof(__half) * (size_t)B * kH) != cudaSuccess ||
        cudaMalloc(&md->H2, sizeof(__half) * (size_t)B * kH) != cudaSuccess ||
        cudaMalloc(&md->dy, sizeof(float) * (size_t)B) != cudaSuccess ||
        cudaMalloc(&md->dZ1, sizeof(float) * (size_t)B * kH) != cudaSuccess ||
        cudaMalloc(&md->dZ2, sizeof(float) * (size_t)B * kH) != cudaSuccess ||
        cudaMalloc(&md->loss, sizeof(float)) != cudaSuccess ||
        cudaMalloc(&md->idx, sizeof(int32_t) * (size_t)B) != cudaSuccess) {
        cudaGetLastError();
        md->free_scratch();
        return MBE_ERR_OOM;
    }
    md->cap = B;
    return MBE_OK;
}

// One minibatch: forward (storing activations), backward, parameter gradients.
cudaError_t batch_grad(mbe_model *md, const float *X, const float *T, const int32_t *d_idx, int32_t B,
                       cudaStream_t s)
{
    const int blocks = std::max(1, std::min(2 * 152, (B + 127) / 128));
    cudaError_t e = cudaMemsetAsync(md->loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    mlp_train_forward_kernel<<<blocks, 128, 0, s>>>(md->p16, md->p32, X, T, d_idx, B, md->X16, md->H1, md->H2,
                                                     md->dy, md->loss);
    mlp_backward_kernel<<<blocks, 128, 0, s>>>(md->p16, md->H1, md->H2, md->dy, B, md->dZ1, md->dZ2);
    mlp_grad_kernel<<<(kNP + 127) / 128, 128, 0, s>>>(md->X16, md->H1, md->H2, md->dy, md->dZ1, md->dZ2, B, md->g);
    return cudaGetLastError();
}

uint64_t splitmix_host(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

} // namespace

const void *model_params16(const mbe_model *md) { return md ? md->p16 : nullptr; }
const float *model_params32(const mbe_model *md) { return md ? md->p32 : nullptr; }

cudaError_t model_predict(const mbe_model *md, const float *d_feat, int32_t n, float *d_out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int blocks = std::max(1, std::min(4 * 152, (n + 127) / 128));
    mlp_predict_kernel<<<blocks, 128, 0, s>>>(md->p16, md->p32, d_feat, n, d_out);
    return cudaGetLastError();
}

} // namespace mbe

using namespace mbe;

extern "C" {

int mbe_model_create(uint64_t seed, mbe_model **out)
{
    if (!out) return MBE_ERR_INVALID_ARG;
    *out = nullptr;
    mbe_model *md = new mbe_model();
    cudaGetDevice(&md->device);
    if (cudaMalloc(&md->p32, sizeof(float) * kNP) != cudaSuccess ||
        cudaMalloc(&md->m, sizeof(float) * kNP) != cudaSuccess ||
        cudaMalloc(&md->v, sizeof(float) * kNP) != cudaSuccess ||
        cudaMalloc(&md->g, sizeof(float) * kNP) != cudaSuccess ||
        cudaMalloc(&md->p16, sizeof(__half) * kNP) != cudaSuccess) {
        cudaGetLastError();
        mbe_model_destroy(md);
        return MBE_ERR_OOM;
    }
    // Uniform(+-1/sqrt(fan_in)) weights from SplitMix64, zero biases
    std::vector<float> h(kNP, 0.f);
    uint64_t st = seed;
    auto unif = [&](float lim) { return lim * (2.f * (float)((splitmix_host(st) >> 40) * 0x1.0p-24) - 1.f); };
    for (int i = 0; i < kH * kF; ++i) h[kOffW1 + i] = unif(1.f / sqrtf((float)kF));
    for (int i = 0; i < kH * kH; ++i) h[kOffW2 + i] = unif(1.f / sqrtf((float)kH));
    for (int i = 0; i < kH; ++i) h[kOffW3 + i] = unif(1.f / sqrtf((float)kH));
    int rc = mbe_model_set_params(md, h.data());
    if (rc != MBE_OK) {
        mbe_model_destroy(md);
        return rc;
    }
    *out = md;
    return MBE_OK;
}

int mbe_model_destroy(mbe_model *md)
{
    if (!md) return MBE_OK;
    cudaFree(md->p32);
    cudaFree(md->m);
    cudaFree(md->v);
    cudaFree(md->g);
    cudaFree(md->p16);
    md->free_scratch();
    delete md;
    return MBE_OK;
}

int mbe_model_set_params(mbe_model *md, const float *host_params)
{
    if (!md || !host_params) return MBE_ERR_INVALID_ARG;
    if (cudaMemcpy(md->p32, host_params, sizeof(float) * kNP, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(md->m, 0, sizeof(float) * kNP) != cudaSuccess ||
        cudaMemset(md->v, 0, sizeof(float) * kNP) != cudaSuccess)
        return MBE_ERR_CUDA;
    to_half_kernel<<<(kNP + 255) / 256, 256>>>(md->p32, md->p16, kNP);
    md->steps = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? MBE_OK : MBE_ERR_CUDA;
}

int mbe_model_get_params(const mbe_model *md, float *host_params)
{
    if (!md || !host_params) return MBE_ERR_INVALID_ARG;
    return cudaMemcpy(host_params, md->p32, sizeof(float) * kNP, cudaMemcpyDeviceToHost) == cudaSuccess ? MBE_OK
                                                                                                       : MBE_ERR_CUDA;
}

int mbe_model_predict(const mbe_model *md, const float *d_feat, int32_t n, float *d_out, void *stream)
{
    if (!md || n < 0 || (n > 0 && (!d_feat || !d_out))) return MBE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = model_predict(md, d_feat, n, d_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

int mbe_model_loss_grad(mbe_model *md, const float *d_feat, const float *d_target, int32_t n, float *host_grad,
                        float *host_loss, void *stream)
{
    if (!md || n <= 0 || !d_feat || !d_target) return MBE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_train_scratch(md, n);
    if (rc != MBE_OK) return rc;
    cudaError_t e = batch_grad(md, d_feat, d_target, nullptr, n, s);
    float l = 0.f;
    if (e == cudaSuccess && host_grad)
        e = cudaMemcpyAsync(host_grad, md->g, sizeof(float) * kNP, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, md->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (host_loss) *host_loss = l / (float)n;
    return cuda_status(e);
}

int mbe_model_train(mbe_model *md, const float *d_feat, const float *d_target, int32_t n, int32_t epochs,
                    int32_t batch, float lr, uint64_t seed, void *stream, float *final_loss)
{
    if (!md || n <= 0 || !d_feat || !d_target || epochs < 1 || batch < 1 || !(lr > 0.f)) return MBE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t B = std::min(batch, n);
    int rc = ensure_train_scratch(md, B);
    if (rc != MBE_OK) return rc;
    int32_t *d_perm = nullptr;
    if (cudaMalloc(&d_perm, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return MBE_ERR_OOM;
    }
    std::vector<int32_t> perm((size_t)n);
    uint64_t st = seed;
    double last = 0.0;
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int32_t i = 0; i < n; ++i) perm[i] = i;
        for (int32_t i = n - 1; i > 0; --i) { // Fisher-Yates from SplitMix64
            int32_t j = (int32_t)(splitmix_host(st) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        e = cudaMemcpyAsync(d_perm, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
        double sum = 0.0;
        int32_t nb = 0;
        for (int32_t b0 = 0; b0 + B <= n && e == cudaSuccess; b0 += B) {
            e = batch_grad(md, d_feat, d_target, d_perm + b0, B, s);
            if (e != cudaSuccess) break;
            md->steps += 1;
            mlp_adam_kernel<<<(kNP + 127) / 128, 128, 0, s>>>(md->p32, md->p16, md->m, md->v, md->g, lr, 0.9f, 0.999f,
                                                               1e-8f, md->steps);
            e = cudaGetLastError();
            if (ep == epochs - 1 && e == cudaSuccess) {
                float l = 0.f;
                e = cudaMemcpyAsync(&l, md->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                sum += l / (float)B;
                ++nb;
            }
        }
        if (nb) last = sum / nb;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_perm);
    if (final_loss) *final_loss = (float)last;
    return cuda_status(e);
}

} // extern "C"
