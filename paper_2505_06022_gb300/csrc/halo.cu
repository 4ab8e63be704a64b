// Halo exchange of split-buffer execution as one kernel per step (paper §3: before a
// chunk runs, the runtime moves the rows its range mapper reads but another chunk
// owns).  All of a step's transfers go in one launch, blockIdx.y picking the
// transfer, so the step costs one small kernel instead of one copy per transfer.
//
// Launched with programmatic dependent launch (when enabled): every block first
// waits for the previous kernel on the stream (the last chunk of the previous step,
// which wrote the rows it reads) and then lets the next launch (the first chunk of
// this step) start; that chunk waits in turn for this kernel to complete before
// reading the halo rows.
//
// Traffic: each transfer reads and writes rows * nx * sizeof(storage) bytes; the
// copy unit is the widest of 16, 4 or 2 bytes that every pointer, the pitch and the
// row width allow.
#include <cstdint>

#include "stamp.cuh"
#include "sy_internal.h"

namespace sy {
namespace {

constexpr int kHaloThreads = 256;
constexpr int kHaloMax = 32;  // transfers per launch
constexpr int64_t kHaloBlocksPerCopy = 64;

struct HaloArgs {
    const char* src[kHaloMax];
    char* dst[kHaloMax];
    int64_t rows[kHaloMax];
    int64_t pitch_bytes;
    int64_t units;  // copy units per row
    int pdl;
};

template <typename T>
__global__ void __launch_bounds__(kHaloThreads) halo_kernel(HaloArgs a) {
    if (a.pdl) {
        griddep_wait();
        griddep_launch_dependents();
    }
    const int t = blockIdx.y;
    const int64_t total = a.rows[t] * a.units;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kHaloThreads;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kHaloThreads + threadIdx.x; i < total; i += stride) {
        const int64_t r = i / a.units, u = i - r * a.units;
        const T* s = reinterpret_cast<const T*>(a.src[t] + r * a.pitch_bytes);
        T* d = reinterpret_cast<T*>(a.dst[t] + r * a.pitch_bytes);
        d[u] = s[u];
    }
}

bool aligned_to(const void* p, int64_t a) { return (reinterpret_cast<uintptr_t>(p) % static_cast<uintptr_t>(a)) == 0; }

}  // namespace

sy_status launch_halo(Queue* q, const HaloCopy* copies, int n, int64_t pitch_bytes, int64_t width_bytes,
                      bool pdl) {
    if (n <= 0 || width_bytes <= 0) return SY_OK;
    int64_t unit = 16;
    for (int64_t v : {int64_t{16}, int64_t{4}, int64_t{2}}) {
        bool ok = pitch_bytes % v == 0 && width_bytes % v == 0;
        for (int i = 0; ok && i < n; ++i) ok = aligned_to(copies[i].src, v) && aligned_to(copies[i].dst, v);
        unit = v;
        if (ok) break;
        if (v == 2) return fail(SY_ERR_INVALID_ARGUMENT, "halo rows are not aligned to 2 bytes");
    }
    const bool overlap = pdl && wave::launch_overlap_enabled();
    for (int first = 0; first < n; first += kHaloMax) {
        const int m = n - first < kHaloMax ? n - first : kHaloMax;
        HaloArgs a = {};
        int64_t most = 0;
        for (int i = 0; i < m; ++i) {
            a.src[i] = static_cast<const char*>(copies[first + i].src);
            a.dst[i] = static_cast<char*>(copies[first + i].dst);
            a.rows[i] = copies[first + i].rows;
            if (a.rows[i] > most) most = a.rows[i];
        }
        a.pitch_bytes = pitch_bytes;
        a.units = width_bytes / unit;
        a.pdl = overlap ? 1 : 0;
        int64_t bx = (most * a.units + kHaloThreads - 1) / kHaloThreads;
        if (bx > kHaloBlocksPerCopy) bx = kHaloBlocksPerCopy;
        if (bx < 1) bx = 1;
        const void* fn = unit == 16 ? reinterpret_cast<const void*>(&halo_kernel<uint4>)
                         : unit == 4 ? reinterpret_cast<const void*>(&halo_kernel<uint32_t>)
                                     : reinterpret_cast<const void*>(&halo_kernel<uint16_t>);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(bx), static_cast<unsigned>(m));
        cfg.blockDim = dim3(kHaloThreads);
        cfg.stream = q->launch;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap ? 1 : 0;
        void* params[1] = {&a};
        const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, params);
        if (e != cudaSuccess)
            return fail(SY_ERR_CUDA, "halo exchange (%d transfers, %lld blocks each): %s", m,
                        static_cast<long long>(bx), cudaGetErrorString(e));
    }
    return SY_OK;
}

}  // namespace sy
