// Small MLP for the cost model: h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2),
// y = W3 h2 + b3, loss = mean over outputs and samples of (y - t)^2, Adam.
// FP32 throughout, trained on the GPU by these kernels.
//
// Parameter vector (row-major, out x in): W1[H][F] b1[H] W2[H][H] b2[H] W3[O][H] b3[O].
// Activations are stored feature-major ([unit][sample]) so that a warp's
// stores and the gradient reductions read consecutive samples.
//
// Kernels (one thread per sample where a sample is independent):
//   mlp_forward_kernel   x -> z1, z2 (kept for backward), y       weights in shared memory
//   mlp_backward_kernel  dy = 2 (y - t) / (B O); dz2, dz1; per-block loss partials
//   mlp_outer_kernel     split-K partial sums of dW = sum_b dz_b (x) a_b (and db = sum_b dz_b)
//                        over a fixed number of sample chunks, then mlp_outer_final sums
//                        the chunks in a fixed order: gradients are bit-reproducible
//   mlp_adam_kernel      Adam (Kingma & Ba 2015, Algorithm 1), elementwise
// The dimensions are tiny (F <= 32, H <= 64, O <= 4), so plain FP32 SIMT is used;
// a tensor-core GEMM would not pay for itself at 64 x 64.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sy_internal.h"

namespace sy {

constexpr int kMlpMaxF = 32;
constexpr int kMlpMaxH = 64;
constexpr int kMlpMaxO = 4;
constexpr int kMlpThreads = 128;
constexpr int kOuterChunks = 64;  // fixed split of the samples for the gradient reductions

struct MlpLayout {
    int F, H, O;
    int64_t W1, b1, W2, b2, W3, b3, P;
};

inline MlpLayout mlp_layout(int F, int H, int O) {
    MlpLayout L;
    L.F = F;
    L.H = H;
    L.O = O;
    L.W1 = 0;
    L.b1 = L.W1 + static_cast<int64_t>(H) * F;
    L.W2 = L.b1 + H;
    L.b2 = L.W2 + static_cast<int64_t>(H) * H;
    L.W3 = L.b2 + H;
    L.b3 = L.W3 + static_cast<int64_t>(O) * H;
    L.P = L.b3 + O;
    return L;
}

struct Mlp {
    Queue* q = nullptr;
    MlpLayout L{};
    float* d_params = nullptr;
    float* d_grad = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    int64_t adam_t = 0;
    // normalisation of inputs and outputs (host copies; predict applies them)
    std::vector<float> x_mean, x_std, y_mean, y_std;
    // scratch sized for the largest batch seen
    int64_t cap = 0;
    float *d_z1 = nullptr, *d_z2 = nullptr, *d_y = nullptr, *d_dz1 = nullptr, *d_dz2 = nullptr, *d_dy = nullptr;
    float* d_partials = nullptr;  // kOuterChunks * (H*max(F,H) + H) floats
    float* d_loss_part = nullptr;
    int loss_blocks = 0;
};

namespace {

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

struct Offs {
    int F, H, O;
    int W1, b1, W2, b2, W3, b3, P;
};

Offs offs_of(const MlpLayout& L) {
    return Offs{L.F, L.H, L.O, (int)L.W1, (int)L.b1, (int)L.W2, (int)L.b2, (int)L.W3, (int)L.b3, (int)L.P};
}

__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(const float* __restrict__ params, Offs o,
                                                                  const float* __restrict__ X, int64_t B,
                                                                  float* __restrict__ Z1, float* __restrict__ Z2,
                                                                  float* __restrict__ Y) {
    extern __shared__ float w[];
    for (int i = threadIdx.x; i < o.P; i += blockDim.x) w[i] = params[i];
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < B; b += stride) {
        float x[kMlpMaxF];
#pragma unroll
        for (int i = 0; i < kMlpMaxF; ++i) x[i] = i < o.F ? X[b * o.F + i] : 0.0f;
        float h1[kMlpMaxH];
#pragma unroll
        for (int j = 0; j < kMlpMaxH; ++j) {
            float s = 0.0f;
            if (j < o.H) {
                s = w[o.b1 + j];
#pragma unroll
                for (int i = 0; i < kMlpMaxF; ++i)
                    if (i < o.F) s = fmaf(w[o.W1 + j * o.F + i], x[i], s);
                if (Z1) Z1[static_cast<int64_t>(j) * B + b] = s;
            }
            h1[j] = j < o.H ? silu(s) : 0.0f;
        }
        float y[kMlpMaxO];
#pragma unroll
        for (int k = 0; k < kMlpMaxO; ++k) y[k] = k < o.O ? w[o.b3 + k] : 0.0f;
        for (int j = 0; j < o.H; ++j) {
            float s = w[o.b2 + j];
#pragma unroll
            for (int i = 0; i < kMlpMaxH; ++i)
                if (i < o.H) s = fmaf(w[o.W2 + j * o.H + i], h1[i], s);
            if (Z2) Z2[static_cast<int64_t>(j) * B + b] = s;
            const float h = silu(s);
#pragma unroll
            for (int k = 0; k < kMlpMaxO; ++k)
                if (k < o.O) y[k] = fmaf(w[o.W3 + k * o.H + j], h, y[k]);
        }
#pragma unroll
        for (int k = 0; k < kMlpMaxO; ++k)
            if (k < o.O) Y[b * o.O + k] = y[k];
    }
}

// dy = scale (y - t), dz2 = (W3^T dy) * silu'(z2), dz1 = (W2^T dz2) * silu'(z1).
// DY, dZ2, dZ1 feature-major.  loss_part[block] = sum over the block's samples of
// sum_k (y - t)^2.
__global__ void __launch_bounds__(kMlpThreads) mlp_backward_kernel(
    const float* __restrict__ params, Offs o, const float* __restrict__ T, int64_t B, float scale,
    const float* __restrict__ Z1, const float* __restrict__ Z2, const float* __restrict__ Y, float* __restrict__ DY,
    float* __restrict__ dZ1, float* __restrict__ dZ2, float* __restrict__ loss_part) {
    extern __shared__ float w[];
    __shared__ float red[kMlpThreads];
    for (int i = threadIdx.x; i < o.P; i += blockDim.x) w[i] = params[i];
    __syncthreads();
    float loss = 0.0f;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < B; b += stride) {
        float dy[kMlpMaxO];
#pragma unroll
        for (int k = 0; k < kMlpMaxO; ++k) {
            dy[k] = 0.0f;
            if (k < o.O) {
                const float e = Y[b * o.O + k] - T[b * o.O + k];
                loss = fmaf(e, e, loss);
                dy[k] = scale * e;
                DY[static_cast<int64_t>(k) * B + b] = dy[k];
            }
        }
        float dz2[kMlpMaxH];
#pragma unroll
        for (int j = 0; j < kMlpMaxH; ++j) {
            dz2[j] = 0.0f;
            if (j < o.H) {
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < kMlpMaxO; ++k)
                    if (k < o.O) s = fmaf(w[o.W3 + k * o.H + j], dy[k], s);
                dz2[j] = s * silu_grad(Z2[static_cast<int64_t>(j) * B + b]);
                dZ2[static_cast<int64_t>(j) * B + b] = dz2[j];
            }
        }
        for (int i = 0; i < o.H; ++i) {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < kMlpMaxH; ++j)
                if (j < o.H) s = fmaf(w[o.W2 + j * o.H + i], dz2[j], s);
            dZ1[static_cast<int64_t>(i) * B + b] = s * silu_grad(Z1[static_cast<int64_t>(i) * B + b]);
        }
    }
    red[threadIdx.x] = loss;
    __syncthreads();
    for (int s = kMlpThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// Partial outer products over sample chunk blockIdx.x:
//   part[c][m][n] = sum_{b in chunk c} A[m][b] * act(Bm[n][b]),  part_bias[c][m] = sum_b A[m][b]
// A is feature-major (M x B).  Bm element (n, b) is at Bm[n * ldn + b * ldb];
// act = silu when `silu_b`, identity otherwise.
__global__ void __launch_bounds__(256) mlp_outer_kernel(const float* __restrict__ A, int M,
                                                        const float* __restrict__ Bm, int N, int64_t ldn, int64_t ldb,
                                                        bool silu_b, int64_t B, float* __restrict__ part) {
    constexpr int kTile = 32;
    __shared__ float sa[kMlpMaxH][kTile + 1];
    __shared__ float sb[kMlpMaxH][kTile + 1];
    const int64_t per = (B + kOuterChunks - 1) / kOuterChunks;
    const int64_t b0 = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t b1 = b0 + per < B ? b0 + per : B;
    const int outputs = M * N + M;
    float acc[(kMlpMaxH * kMlpMaxH + kMlpMaxH + 255) / 256];
#pragma unroll
    for (int r = 0; r < (kMlpMaxH * kMlpMaxH + kMlpMaxH + 255) / 256; ++r) acc[r] = 0.0f;
    for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
        const int cnt = static_cast<int>(b1 - t0 < kTile ? b1 - t0 : kTile);
        for (int e = threadIdx.x; e < M * kTile; e += blockDim.x) {
            const int m = e / kTile, k = e % kTile;
            sa[m][k] = k < cnt ? A[static_cast<int64_t>(m) * B + t0 + k] : 0.0f;
        }
        for (int e = threadIdx.x; e < N * kTile; e += blockDim.x) {
            const int n = e / kTile, k = e % kTile;
            float v = k < cnt ? Bm[static_cast<int64_t>(n) * ldn + (t0 + k) * ldb] : 0.0f;
            sb[n][k] = (silu_b && k < cnt) ? silu(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < (kMlpMaxH * kMlpMaxH + kMlpMaxH + 255) / 256; ++r) {
            const int out = threadIdx.x + r * 256;
            if (out < outputs) {
                float s = acc[r];
                if (out < M * N) {
                    const int m = out / N, n = out % N;
                    for (int k = 0; k < cnt; ++k) s = fmaf(sa[m][k], sb[n][k], s);
                } else {
                    const int m = out - M * N;
                    for (int k = 0; k < cnt; ++k) s += sa[m][k];
                }
                acc[r] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < (kMlpMaxH * kMlpMaxH + kMlpMaxH + 255) / 256; ++r) {
        const int out = threadIdx.x + r * 256;
        if (out < outputs) part[static_cast<int64_t>(blockIdx.x) * outputs + out] = acc[r];
    }
}

// Sum the kOuterChunks partials in chunk order; write weights to grad[w_off + m*N + n]
// and biases to grad[b_off + m].
__global__ void mlp_outer_final(const float* __restrict__ part, int M, int N, float* __restrict__ grad,
                                int64_t w_off, int64_t b_off) {
    const int outputs = M * N + M;
    for (int out = blockIdx.x * blockDim.x + threadIdx.x; out < outputs; out += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < kOuterChunks; ++c) s += part[static_cast<int64_t>(c) * outputs + out];
        if (out < M * N) grad[w_off + out] = s;
        else grad[b_off + (out - M * N)] = s;
    }
}

__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t n, float lr, float beta1, float beta2, float eps,
                                float bc1, float bc2) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void mlp_gather_kernel(const float* __restrict__ src, const int* __restrict__ perm, int64_t n, int width,
                                  float* __restrict__ dst) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n * width;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = e / width, c = e - r * width;
        dst[e] = src[static_cast<int64_t>(perm[r]) * width + c];
    }
}

Mlp* as_mlp(sy_mlp_t h) { return reinterpret_cast<Mlp*>(h); }

int blocks_for(int64_t n, int threads, int cap) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return static_cast<int>(b < cap ? b : cap);
}

sy_status ensure_scratch(Mlp* M, int64_t B) {
    if (B <= M->cap) return SY_OK;
    const MlpLayout& L = M->L;
    float** bufs[] = {&M->d_z1, &M->d_z2, &M->d_y, &M->d_dz1, &M->d_dz2, &M->d_dy};
    for (float** b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    const size_t hb = sizeof(float) * static_cast<size_t>(B) * L.H;
    const size_t ob = sizeof(float) * static_cast<size_t>(B) * L.O;
    SY_CUDA(cudaMalloc(&M->d_z1, hb));
    SY_CUDA(cudaMalloc(&M->d_z2, hb));
    SY_CUDA(cudaMalloc(&M->d_dz1, hb));
    SY_CUDA(cudaMalloc(&M->d_dz2, hb));
    SY_CUDA(cudaMalloc(&M->d_y, ob));
    SY_CUDA(cudaMalloc(&M->d_dy, ob));
    M->cap = B;
    return SY_OK;
}

// `keep` stores z1/z2 for the backward pass; the caller must have sized the
// scratch (ensure_scratch) before passing any scratch pointer as Y.
sy_status forward(Mlp* M, const float* X, int64_t B, float* Y, bool keep) {
    if (keep && B > M->cap) return fail(SY_ERR_INVALID_ARGUMENT, "MLP scratch not sized for %lld samples", (long long)B);
    const Offs o = offs_of(M->L);
    const size_t smem = sizeof(float) * static_cast<size_t>(M->L.P);
    mlp_forward_kernel<<<blocks_for(B, kMlpThreads, M->q->sm_count * 8), kMlpThreads, smem, M->q->launch>>>(
        M->d_params, o, X, B, keep ? M->d_z1 : nullptr, keep ? M->d_z2 : nullptr, Y);
    SY_CUDA(cudaGetLastError());
    ++M->q->launches;
    return SY_OK;
}

// Forward + backward on (X, T) of B samples; gradient into d_grad; loss (mean of squares)
// into *loss_out when non-null (synchronises).
sy_status loss_grad(Mlp* M, const float* X, const float* T, int64_t B, float* loss_out) {
    SY_TRY(ensure_scratch(M, B));  // before reading any scratch pointer below
    SY_TRY(forward(M, X, B, M->d_y, true));
    const MlpLayout& L = M->L;
    const Offs o = offs_of(L);
    const size_t smem = sizeof(float) * static_cast<size_t>(L.P);
    const int nb = blocks_for(B, kMlpThreads, M->loss_blocks);
    const float scale = 2.0f / (static_cast<float>(B) * static_cast<float>(L.O));
    cudaStream_t s = M->q->launch;
    mlp_backward_kernel<<<nb, kMlpThreads, smem, s>>>(M->d_params, o, T, B, scale, M->d_z1, M->d_z2, M->d_y, M->d_dy,
                                                       M->d_dz1, M->d_dz2, M->d_loss_part);
    SY_CUDA(cudaGetLastError());
    // layer 3: dW3 = dy (x) silu(z2);  layer 2: dW2 = dz2 (x) silu(z1);  layer 1: dW1 = dz1 (x) x
    const int outs3 = L.O * L.H + L.O, outs2 = L.H * L.H + L.H, outs1 = L.H * L.F + L.H;
    float* part = M->d_partials;
    mlp_outer_kernel<<<kOuterChunks, 256, 0, s>>>(M->d_dy, L.O, M->d_z2, L.H, B, 1, true, B, part);
    mlp_outer_final<<<blocks_for(outs3, 256, 64), 256, 0, s>>>(part, L.O, L.H, M->d_grad, L.W3, L.b3);
    mlp_outer_kernel<<<kOuterChunks, 256, 0, s>>>(M->d_dz2, L.H, M->d_z1, L.H, B, 1, true, B, part);
    mlp_outer_final<<<blocks_for(outs2, 256, 64), 256, 0, s>>>(part, L.H, L.H, M->d_grad, L.W2, L.b2);
    mlp_outer_kernel<<<kOuterChunks, 256, 0, s>>>(M->d_dz1, L.H, X, L.F, 1, L.F, false, B, part);
    mlp_outer_final<<<blocks_for(outs1, 256, 64), 256, 0, s>>>(part, L.H, L.F, M->d_grad, L.W1, L.b1);
    SY_CUDA(cudaGetLastError());
    M->q->launches += 7;
    if (loss_out) {
        std::vector<float> lp(nb);
        SY_CUDA(cudaMemcpyAsync(lp.data(), M->d_loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
        SY_CUDA(cudaStreamSynchronize(s));
        double tot = 0.0;
        for (float v : lp) tot += v;
        *loss_out = static_cast<float>(tot / (static_cast<double>(B) * L.O));
    }
    return SY_OK;
}

sy_status adam(Mlp* M, float lr, float beta1, float beta2, float eps) {
    M->adam_t += 1;
    const float bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(M->adam_t)));
    const float bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(M->adam_t)));
    mlp_adam_kernel<<<blocks_for(M->L.P, 256, 64), 256, 0, M->q->launch>>>(M->d_params, M->d_grad, M->d_m, M->d_v,
                                                                          M->L.P, lr, beta1, beta2, eps, bc1, bc2);
    SY_CUDA(cudaGetLastError());
    ++M->q->launches;
    return SY_OK;
}

// splitmix64 (Steele, Lea & Flood 2014) for initialisation and shuffling.
uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
struct Rng {
    uint64_t s;
    uint64_t next() { return mix64(s += 0x9e3779b97f4a7c15ull); }
    double uniform() { return static_cast<double>(next() >> 11) * (1.0 / 9007199254740992.0); }
};

void fit_norm(const float* A, int64_t n, int w, std::vector<float>* mean, std::vector<float>* stdv) {
    mean->assign(w, 0.0f);
    stdv->assign(w, 1.0f);
    for (int c = 0; c < w; ++c) {
        double s = 0.0, ss = 0.0;
        for (int64_t r = 0; r < n; ++r) s += A[r * w + c];
        const double mu = n ? s / n : 0.0;
        for (int64_t r = 0; r < n; ++r) ss += (A[r * w + c] - mu) * (A[r * w + c] - mu);
        const double sd = n > 1 ? std::sqrt(ss / n) : 1.0;
        (*mean)[c] = static_cast<float>(mu);
        (*stdv)[c] = static_cast<float>(sd > 1e-12 ? sd : 1.0);
    }
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" {

sy_status sy_mlp_create(sy_queue_t qh, int in_features, int hidden, int out_features, uint64_t seed, sy_mlp_t* out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!out) return fail(SY_ERR_NULL_POINTER, "out is NULL");
    *out = nullptr;
    if (in_features < 1 || in_features > kMlpMaxF || hidden < 1 || hidden > kMlpMaxH || out_features < 1 ||
        out_features > kMlpMaxO)
        return fail(SY_ERR_INVALID_ARGUMENT, "MLP %d-%d-%d outside 1..%d, 1..%d, 1..%d", in_features, hidden,
                    out_features, kMlpMaxF, kMlpMaxH, kMlpMaxO);
    SY_TRY(use_device(q));
    Mlp* M = new (std::nothrow) Mlp();
    if (!M) return fail(SY_ERR_OUT_OF_MEMORY, "MLP allocation failed");
    M->q = q;
    M->L = mlp_layout(in_features, hidden, out_features);
    M->loss_blocks = q->sm_count * 4;
    M->x_mean.assign(in_features, 0.0f);
    M->x_std.assign(in_features, 1.0f);
    M->y_mean.assign(out_features, 0.0f);
    M->y_std.assign(out_features, 1.0f);
    const size_t pb = sizeof(float) * static_cast<size_t>(M->L.P);
    const int64_t part_floats = kOuterChunks * (static_cast<int64_t>(hidden) * (hidden > in_features ? hidden : in_features) + hidden);
    cudaError_t e = cudaMalloc(&M->d_params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_grad, pb);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_partials, sizeof(float) * static_cast<size_t>(part_floats));
    if (e == cudaSuccess) e = cudaMalloc(&M->d_loss_part, sizeof(float) * static_cast<size_t>(M->loss_blocks));
    if (e == cudaSuccess) e = cudaMemset(M->d_m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(M->d_v, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(M->d_grad, 0, pb);
    if (e == cudaSuccess) {
        // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
        std::vector<float> p(M->L.P, 0.0f);
        Rng r{seed};
        auto fill = [&](int64_t off, int64_t count, int fan_in) {
            const double a = 1.0 / std::sqrt(static_cast<double>(fan_in));
            for (int64_t i = 0; i < count; ++i) p[off + i] = static_cast<float>((2.0 * r.uniform() - 1.0) * a);
        };
        fill(M->L.W1, static_cast<int64_t>(hidden) * in_features, in_features);
        fill(M->L.W2, static_cast<int64_t>(hidden) * hidden, hidden);
        fill(M->L.W3, static_cast<int64_t>(out_features) * hidden, hidden);
        e = cudaMemcpy(M->d_params, p.data(), pb, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        float* bufs[] = {M->d_params, M->d_grad, M->d_m, M->d_v, M->d_partials, M->d_loss_part};
        for (float* b : bufs)
            if (b) cudaFree(b);
        delete M;
        return cuda_fail(e, "sy_mlp_create");
    }
    *out = reinterpret_cast<sy_mlp_t>(M);
    return SY_OK;
}

sy_status sy_mlp_destroy(sy_mlp_t h) {
    if (!h) return SY_OK;
    Mlp* M = as_mlp(h);
    cudaSetDevice(M->q->device);
    cudaStreamSynchronize(M->q->stream);
    float* bufs[] = {M->d_params, M->d_grad, M->d_m, M->d_v, M->d_partials, M->d_loss_part,
                     M->d_z1, M->d_z2, M->d_y, M->d_dz1, M->d_dz2, M->d_dy};
    for (float* b : bufs)
        if (b) cudaFree(b);
    delete M;
    return SY_OK;
}

sy_status sy_mlp_param_count(sy_mlp_t h, int64_t* n) {
    if (!h || !n) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    *n = as_mlp(h)->L.P;
    return SY_OK;
}

sy_status sy_mlp_get_params(sy_mlp_t h, float* host, int64_t n) {
    if (!h || !host) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    Mlp* M = as_mlp(h);
    if (n != M->L.P) return fail(SY_ERR_INVALID_ARGUMENT, "n = %lld, model has %lld", (long long)n, (long long)M->L.P);
    SY_TRY(use_device(M->q));
    SY_CUDA(cudaMemcpyAsync(host, M->d_params, sizeof(float) * n, cudaMemcpyDeviceToHost, M->q->stream));
    SY_CUDA(cudaStreamSynchronize(M->q->stream));
    return SY_OK;
}

sy_status sy_mlp_get_grad(sy_mlp_t h, float* host, int64_t n) {
    if (!h || !host) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    Mlp* M = as_mlp(h);
    if (n != M->L.P) return fail(SY_ERR_INVALID_ARGUMENT, "n = %lld, model has %lld", (long long)n, (long long)M->L.P);
    SY_TRY(use_device(M->q));
    SY_CUDA(cudaMemcpyAsync(host, M->d_grad, sizeof(float) * n, cudaMemcpyDeviceToHost, M->q->stream));
    SY_CUDA(cudaStreamSynchronize(M->q->stream));
    return SY_OK;
}

sy_status sy_mlp_set_params(sy_mlp_t h, const float* host, int64_t n) {
    if (!h || !host) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    Mlp* M = as_mlp(h);
    if (n != M->L.P) return fail(SY_ERR_INVALID_ARGUMENT, "n = %lld, model has %lld", (long long)n, (long long)M->L.P);
    SY_TRY(use_device(M->q));
    SY_CUDA(cudaMemcpyAsync(M->d_params, host, sizeof(float) * n, cudaMemcpyHostToDevice, M->q->stream));
    SY_CUDA(cudaMemsetAsync(M->d_m, 0, sizeof(float) * n, M->q->stream));
    SY_CUDA(cudaMemsetAsync(M->d_v, 0, sizeof(float) * n, M->q->stream));
    SY_CUDA(cudaStreamSynchronize(M->q->stream));
    M->adam_t = 0;
    return SY_OK;
}

sy_status sy_mlp_forward(sy_mlp_t h, const float* d_X, int64_t B, float* d_Y) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    if (B < 0) return fail(SY_ERR_INVALID_ARGUMENT, "B < 0");
    if (B == 0) return SY_OK;
    if (!d_X || !d_Y) return fail(SY_ERR_NULL_POINTER, "X or Y is NULL");
    Mlp* M = as_mlp(h);
    SY_TRY(use_device(M->q));
    return forward(M, d_X, B, d_Y, false);
}

sy_status sy_mlp_backward(sy_mlp_t h, const float* d_X, const float* d_T, int64_t B, float* loss) {
    return sy_mlp_loss_grad(h, d_X, d_T, B, loss);
}

sy_status sy_mlp_loss_grad(sy_mlp_t h, const float* d_X, const float* d_T, int64_t B, float* loss) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    if (B < 1) return fail(SY_ERR_INVALID_ARGUMENT, "B < 1");
    if (!d_X || !d_T) return fail(SY_ERR_NULL_POINTER, "X or T is NULL");
    Mlp* M = as_mlp(h);
    SY_TRY(use_device(M->q));
    return loss_grad(M, d_X, d_T, B, loss);
}

sy_status sy_mlp_adam_step(sy_mlp_t h, float lr, float beta1, float beta2, float eps) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    Mlp* M = as_mlp(h);
    SY_TRY(use_device(M->q));
    return adam(M, lr, beta1, beta2, eps);
}

sy_status sy_mlp_train(sy_mlp_t h, const float* X, const float* T, int64_t n, int epochs, int batch, float lr,
                       uint64_t seed, float* final_loss) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    if (!X || !T) return fail(SY_ERR_NULL_POINTER, "X or T is NULL");
    if (n < 1 || epochs < 0 || batch < 1) return fail(SY_ERR_INVALID_ARGUMENT, "n, epochs or batch out of range");
    Mlp* M = as_mlp(h);
    const MlpLayout& L = M->L;
    SY_TRY(use_device(M->q));
    // normalisation from the training set (host), then normalised copies on the device
    fit_norm(X, n, L.F, &M->x_mean, &M->x_std);
    fit_norm(T, n, L.O, &M->y_mean, &M->y_std);
    std::vector<float> xn(static_cast<size_t>(n) * L.F), tn(static_cast<size_t>(n) * L.O);
    for (int64_t r = 0; r < n; ++r) {
        for (int c = 0; c < L.F; ++c) xn[r * L.F + c] = (X[r * L.F + c] - M->x_mean[c]) / M->x_std[c];
        for (int c = 0; c < L.O; ++c) tn[r * L.O + c] = (T[r * L.O + c] - M->y_mean[c]) / M->y_std[c];
    }
    float *dX = nullptr, *dT = nullptr, *sX = nullptr, *sT = nullptr;
    int* dperm = nullptr;
    cudaStream_t s = M->q->stream;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        if (dX) cudaFree(dX);
        if (dT) cudaFree(dT);
        if (sX) cudaFree(sX);
        if (sT) cudaFree(sT);
        if (dperm) cudaFree(dperm);
    };
    cudaError_t e = cudaMalloc(&dX, sizeof(float) * xn.size());
    if (e == cudaSuccess) e = cudaMalloc(&dT, sizeof(float) * tn.size());
    if (e == cudaSuccess) e = cudaMalloc(&sX, sizeof(float) * xn.size());
    if (e == cudaSuccess) e = cudaMalloc(&sT, sizeof(float) * tn.size());
    if (e == cudaSuccess) e = cudaMalloc(&dperm, sizeof(int) * static_cast<size_t>(n));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, xn.data(), sizeof(float) * xn.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, tn.data(), sizeof(float) * tn.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sy_mlp_train setup");
    }
    sy_status st = ensure_scratch(M, batch < n ? batch : n);
    std::vector<int> perm(n);
    Rng rng{seed};
    float last = 0.0f;
    for (int ep = 0; st == SY_OK && ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[i] = static_cast<int>(i);
        for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates
            const int64_t j = static_cast<int64_t>(rng.next() % static_cast<uint64_t>(i + 1));
            std::swap(perm[i], perm[j]);
        }
        e = cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "perm upload");
            break;
        }
        mlp_gather_kernel<<<blocks_for(n * L.F, 256, 1024), 256, 0, s>>>(dX, dperm, n, L.F, sX);
        mlp_gather_kernel<<<blocks_for(n * L.O, 256, 1024), 256, 0, s>>>(dT, dperm, n, L.O, sT);
        M->q->launches += 2;
        for (int64_t off = 0; st == SY_OK && off < n; off += batch) {
            const int64_t bsz = n - off < batch ? n - off : batch;
            const bool want = (ep == epochs - 1) && (off + batch >= n);
            st = loss_grad(M, sX + off * L.F, sT + off * L.O, bsz, want ? &last : nullptr);
            if (st == SY_OK) st = adam(M, lr, 0.9f, 0.999f, 1e-8f);
        }
    }
    cudaError_t le = cudaGetLastError();
    if (st == SY_OK && le != cudaSuccess) st = cuda_fail(le, "sy_mlp_train");
    cleanup();
    if (final_loss) *final_loss = last;
    return st;
}

sy_status sy_mlp_normalization(sy_mlp_t h, float* x_mean, float* x_std, float* y_mean, float* y_std) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    Mlp* M = as_mlp(h);
    if (x_mean) std::memcpy(x_mean, M->x_mean.data(), sizeof(float) * M->L.F);
    if (x_std) std::memcpy(x_std, M->x_std.data(), sizeof(float) * M->L.F);
    if (y_mean) std::memcpy(y_mean, M->y_mean.data(), sizeof(float) * M->L.O);
    if (y_std) std::memcpy(y_std, M->y_std.data(), sizeof(float) * M->L.O);
    return SY_OK;
}

sy_status sy_cost_model_predict(sy_mlp_t h, const float* features, int64_t n, float* pred) {
    if (!h) return fail(SY_ERR_NULL_POINTER, "model is NULL");
    if (n < 0) return fail(SY_ERR_INVALID_ARGUMENT, "n < 0");
    if (n == 0) return SY_OK;
    if (!features || !pred) return fail(SY_ERR_NULL_POINTER, "features or pred is NULL");
    Mlp* M = as_mlp(h);
    const MlpLayout& L = M->L;
    SY_TRY(use_device(M->q));
    std::vector<float> xn(static_cast<size_t>(n) * L.F);
    for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < L.F; ++c) xn[r * L.F + c] = (features[r * L.F + c] - M->x_mean[c]) / M->x_std[c];
    float *dX = nullptr, *dY = nullptr;
    cudaStream_t s = M->q->stream;
    cudaError_t e = cudaMalloc(&dX, sizeof(float) * xn.size());
    if (e == cudaSuccess) e = cudaMalloc(&dY, sizeof(float) * static_cast<size_t>(n) * L.O);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, xn.data(), sizeof(float) * xn.size(), cudaMemcpyHostToDevice, s);
    sy_status st = e == cudaSuccess ? forward(M, dX, n, dY, false) : cuda_fail(e, "sy_cost_model_predict");
    if (st == SY_OK) {
        e = cudaMemcpyAsync(pred, dY, sizeof(float) * static_cast<size_t>(n) * L.O, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "sy_cost_model_predict");
    }
    if (dX) cudaFree(dX);
    if (dY) cudaFree(dY);
    if (st != SY_OK) return st;
    for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < L.O; ++c) pred[r * L.O + c] = pred[r * L.O + c] * M->y_std[c] + M->y_mean[c];
    return SY_OK;
}

sy_status sy_cost_model_choose(sy_mlp_t h, const float* features, int n, int objective, int* best) {
    if (!h || !best) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    if (n < 1) return fail(SY_ERR_INVALID_ARGUMENT, "no candidates");
    Mlp* M = as_mlp(h);
    if (objective < 0 || objective > 2 || (objective > 0 && M->L.O < 2))
        return fail(SY_ERR_INVALID_ARGUMENT, "objective %d needs outputs (log time, log energy)", objective);
    std::vector<float> pred(static_cast<size_t>(n) * M->L.O);
    SY_TRY(sy_cost_model_predict(h, features, n, pred.data()));
    int arg = 0;
    double bestv = 0.0;
    for (int i = 0; i < n; ++i) {
        const double lt = pred[static_cast<size_t>(i) * M->L.O];
        const double le = M->L.O > 1 ? pred[static_cast<size_t>(i) * M->L.O + 1] : 0.0;
        const double v = objective == 0 ? lt : objective == 1 ? le : lt + le;  // log EDP = log t + log E
        if (i == 0 || v < bestv) {
            bestv = v;
            arg = i;
        }
    }
    *best = arg;
    return SY_OK;
}

sy_status sy_mlp_save(sy_mlp_t h, const char* path) {
    if (!h || !path) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    Mlp* M = as_mlp(h);
    std::vector<float> p(M->L.P);
    SY_TRY(sy_mlp_get_params(h, p.data(), M->L.P));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(SY_ERR_IO, "cannot open %s for writing", path);
    const int32_t hdr[4] = {0x53594d31 /* "SYM1" */, M->L.F, M->L.H, M->L.O};
    bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1;
    ok = ok && std::fwrite(M->x_mean.data(), sizeof(float), M->L.F, f) == static_cast<size_t>(M->L.F);
    ok = ok && std::fwrite(M->x_std.data(), sizeof(float), M->L.F, f) == static_cast<size_t>(M->L.F);
    ok = ok && std::fwrite(M->y_mean.data(), sizeof(float), M->L.O, f) == static_cast<size_t>(M->L.O);
    ok = ok && std::fwrite(M->y_std.data(), sizeof(float), M->L.O, f) == static_cast<size_t>(M->L.O);
    ok = ok && std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SY_OK : fail(SY_ERR_IO, "write to %s failed", path);
}

sy_status sy_mlp_load(sy_queue_t qh, const char* path, sy_mlp_t* out) {
    if (!path || !out) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(SY_ERR_IO, "cannot open %s", path);
    int32_t hdr[4];
    if (std::fread(hdr, sizeof hdr, 1, f) != 1 || hdr[0] != 0x53594d31) {
        std::fclose(f);
        return fail(SY_ERR_IO, "%s is not a saved sy MLP", path);
    }
    sy_mlp_t h = nullptr;
    sy_status st = sy_mlp_create(qh, hdr[1], hdr[2], hdr[3], 0, &h);
    if (st != SY_OK) {
        std::fclose(f);
        return st;
    }
    Mlp* M = as_mlp(h);
    std::vector<float> p(M->L.P);
    bool ok = std::fread(M->x_mean.data(), sizeof(float), hdr[1], f) == static_cast<size_t>(hdr[1]);
    ok = ok && std::fread(M->x_std.data(), sizeof(float), hdr[1], f) == static_cast<size_t>(hdr[1]);
    ok = ok && std::fread(M->y_mean.data(), sizeof(float), hdr[3], f) == static_cast<size_t>(hdr[3]);
    ok = ok && std::fread(M->y_std.data(), sizeof(float), hdr[3], f) == static_cast<size_t>(hdr[3]);
    ok = ok && std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
    std::fclose(f);
    if (!ok) {
        sy_mlp_destroy(h);
        return fail(SY_ERR_IO, "%s is truncated", path);
    }
    st = sy_mlp_set_params(h, p.data(), M->L.P);
    if (st != SY_OK) {
        sy_mlp_destroy(h);
        return st;
    }
    *out = h;
    return SY_OK;
}

}  // extern "C"
