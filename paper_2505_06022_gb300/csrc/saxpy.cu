// SAXPY, z[i] = alpha * x[i] + y[i] (paper §2 Listing 1; §3 Listing 2 runs the
// same kernel once per one_to_one chunk).
//
// HBM-bound: 12 bytes per element (two 4-byte reads, one 4-byte write), two
// flops.  Every access is a 128-bit streaming load/store (ld.global.cs /
// st.global.cs: the data is touched once, so it should not displace anything
// else in L2).  Each thread keeps kUnroll independent float4 pairs in flight;
// the grid holds at most `waves` x 2048 threads per SM (a full SM's thread slots;
// the 40-register kernel keeps 6 of 8 such blocks of 256 resident, which measured
// no slower at 2^26: 102 % of the copy) and strides over the array.
//
// The product is rounded, then the sum: __fmul_rn / __fadd_rn are never
// contracted into an FMA, so the result is fl(fl(alpha*x) + y) bit for bit.
#include <cstdint>

#include "stamp.cuh"
#include "sy_internal.h"

namespace sy {
namespace {

constexpr int kThreads = 256;  // scalar kernel and the default vector variant
constexpr int kUnroll = 4;

__device__ __forceinline__ float saxpy1(float alpha, float x, float y) {
    return __fadd_rn(__fmul_rn(alpha, x), y);
}

// Vector body over n4 float4 elements (all three pointers 16-byte aligned).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) saxpy_vec4_kernel(int64_t n4, float alpha, const float4* x,
                                                             const float4* y, float4* z, unsigned long long* stamp) {
    stamp_begin(stamp);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * THREADS;
    int64_t i = static_cast<int64_t>(blockIdx.x) * THREADS + threadIdx.x;
    // Main loop: kUnroll vectors per thread per trip, loads issued before use.
    for (; i + (kUnroll - 1) * stride < n4; i += kUnroll * stride) {
        float4 a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            a[u] = __ldcs(x + i + u * stride);
            b[u] = __ldcs(y + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            float4 r;
            r.x = saxpy1(alpha, a[u].x, b[u].x);
            r.y = saxpy1(alpha, a[u].y, b[u].y);
            r.z = saxpy1(alpha, a[u].z, b[u].z);
            r.w = saxpy1(alpha, a[u].w, b[u].w);
            __stcs(z + i + u * stride, r);
        }
    }
    for (; i < n4; i += stride) {
        float4 a = __ldcs(x + i), b = __ldcs(y + i), r;
        r.x = saxpy1(alpha, a.x, b.x);
        r.y = saxpy1(alpha, a.y, b.y);
        r.z = saxpy1(alpha, a.z, b.z);
        r.w = saxpy1(alpha, a.w, b.w);
        __stcs(z + i, r);
    }
    stamp_end(stamp);
}

// Scalar elements: [0, head) and [tail0, n).  Also the whole array when the
// pointers are not mutually aligned (head = n, tail0 = n).
__global__ void __launch_bounds__(kThreads) saxpy_scalar_kernel(int64_t n, int64_t head, int64_t tail0,
                                                                float alpha, const float* x, const float* y,
                                                                float* z, unsigned long long* stamp) {
    stamp_begin(stamp);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    const int64_t count = head + (n - tail0);
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; t < count; t += stride) {
        int64_t i = t < head ? t : tail0 + (t - head);
        z[i] = saxpy1(alpha, __ldcs(x + i), __ldcs(y + i));
    }
    stamp_end(stamp);
}

int64_t blocks_for(Queue* q, int64_t work_items, int threads, int waves) {
    int64_t want = (work_items + threads - 1) / threads;
    int64_t cap = static_cast<int64_t>(q->sm_count) * (2048 / threads) * waves;  // waves x a full SM
    if (want < 1) want = 1;
    return want < cap ? want : cap;
}

// Vector-kernel variants: threads in {128, 256, 512} x waves in {1, 2, 4}; 0 = 256 x 1.
constexpr int kSaxpyThreads[3] = {128, 256, 512};
constexpr int kSaxpyWaves[3] = {1, 2, 4};

}  // namespace

int saxpy_variant_count() { return 9; }

bool saxpy_variant_info(int variant, int* threads, int* waves) {
    if (variant < 0 || variant > 9) return false;
    const int t = variant == 0 ? 256 : kSaxpyThreads[(variant - 1) / 3];
    const int w = variant == 0 ? 1 : kSaxpyWaves[(variant - 1) % 3];
    if (threads) *threads = t;
    if (waves) *waves = w;
    return true;
}

sy_status launch_saxpy(Queue* q, int64_t n, float alpha, const float* x, const float* y, float* z) {
    return launch_saxpy_variant(q, n, alpha, x, y, z, 0);
}

sy_status launch_saxpy_variant(Queue* q, int64_t n, float alpha, const float* x, const float* y, float* z,
                               int variant) {
    int threads = 256, waves = 1;
    if (!saxpy_variant_info(variant, &threads, &waves))
        return fail(SY_ERR_INVALID_ARGUMENT, "SAXPY variant %d not in 0..%d", variant, saxpy_variant_count());
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x) & 15u;
    const uintptr_t ay = reinterpret_cast<uintptr_t>(y) & 15u;
    const uintptr_t az = reinterpret_cast<uintptr_t>(z) & 15u;
    int64_t head = n, n4 = 0, tail0 = n;
    if (ax == ay && ay == az && (ax & 3u) == 0) {
        head = static_cast<int64_t>(((16u - ax) & 15u) / 4u);
        if (head > n) head = n;
        n4 = (n - head) / 4;
        tail0 = head + 4 * n4;
    }
    if (n4 > 0) {
        const int64_t blocks = blocks_for(q, (n4 + kUnroll - 1) / kUnroll, threads, waves);
        const float4* x4 = reinterpret_cast<const float4*>(x + head);
        const float4* y4 = reinterpret_cast<const float4*>(y + head);
        float4* z4 = reinterpret_cast<float4*>(z + head);
        const unsigned g = static_cast<unsigned>(blocks);
        if (threads == 128) saxpy_vec4_kernel<128><<<g, 128, 0, q->launch>>>(n4, alpha, x4, y4, z4, q->cur_stamp);
        else if (threads == 512) saxpy_vec4_kernel<512><<<g, 512, 0, q->launch>>>(n4, alpha, x4, y4, z4, q->cur_stamp);
        else saxpy_vec4_kernel<256><<<g, 256, 0, q->launch>>>(n4, alpha, x4, y4, z4, q->cur_stamp);
        SY_CUDA(cudaGetLastError());
        ++q->launches;
        q->cur_blocks += static_cast<uint64_t>(blocks);
    }
    const int64_t scalar = head + (n - tail0);
    if (scalar > 0) {
        const int64_t blocks = blocks_for(q, scalar, kThreads, 1);
        saxpy_scalar_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, q->launch>>>(n, head, tail0, alpha, x, y,
                                                                                      z, q->cur_stamp);
        SY_CUDA(cudaGetLastError());
        ++q->launches;
        q->cur_blocks += static_cast<uint64_t>(blocks);
    }
    return SY_OK;
}

}  // namespace sy
