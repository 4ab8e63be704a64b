// Wave-step launch logic (grid sizing, variant table, layout checks) and the
// FP64 discrete-energy reduction.
//
// Discrete energy of the leapfrog scheme (conserved exactly when L = L^T):
//   E^{n+1/2} = sum (u_new - u_old)^2 - c2 * sum u_new * (L u_old)
// Reduction shape is fixed (kEnergyBlocks blocks x 256 threads, each thread a
// fixed arithmetic progression of points, a fixed shared-memory tree per block,
// then one block summing the partials in a fixed tree), so the result does not
// depend on scheduling: repeated calls give identical bits.
#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "wave_kernel.cuh"

namespace sy {
namespace wave {

namespace {
std::mutex g_occ_mu;
std::unordered_map<uint64_t, int> g_occ;

int occupancy(const void* fn, int threads) {
    const uint64_t key = reinterpret_cast<uint64_t>(fn) ^ (static_cast<uint64_t>(threads) << 56);
    {
        std::lock_guard<std::mutex> lock(g_occ_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) return it->second;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, 0) != cudaSuccess || blocks < 1)
        blocks = 1;
    std::lock_guard<std::mutex> lock(g_occ_mu);
    g_occ[key] = blocks;
    return blocks;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Programmatic dependent launch of the chunk kernels; SY_PDL=0 turns it off.
bool pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("SY_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}
}  // namespace

int kernel_occupancy(const void* fn, int threads) { return occupancy(fn, threads); }
bool launch_overlap_enabled() { return pdl_enabled(); }

sy_status launch_typed(Queue* q, const WaveLaunch& w, KernelFn vec_fn, KernelFn scalar_fn, int tile_rows,
                       int threads, int span, size_t esize, Form form) {
    const int64_t rows = w.row_end - w.row_begin;
    if (rows <= 0 || w.nx == 0) return SY_OK;
    Args a;
    a.u_prev = static_cast<const char*>(w.u_prev);
    a.u_cur = static_cast<const char*>(w.u_cur);
    a.u_next = static_cast<char*>(w.u_next);
    a.ny = w.ny;
    a.nx = w.nx;
    a.pitch_bytes = w.pitch * static_cast<int64_t>(esize);
    a.row_begin = w.row_begin;
    a.row_end = w.row_end;
    a.c2 = w.c2;
    a.stamp = q->cur_stamp;
    a.pdl = 0;
    a.neg0 = -0.0f;
    if (!aligned(w.u_cur, esize) || !aligned(w.u_next, esize) || (!w.start && !aligned(w.u_prev, esize)))
        return fail(SY_ERR_INVALID_ARGUMENT, "field pointers must be aligned to the element size (%zu bytes)", esize);
    const bool vec_ok = aligned(w.u_cur, 16) && aligned(w.u_next, 16) && (w.start || aligned(w.u_prev, 16)) &&
                        (a.pitch_bytes % 16) == 0;
    if (vec_ok) {
        a.tiles_x = (w.nx + span - 1) / span;
        a.tiles = a.tiles_x * ((rows + tile_rows - 1) / tile_rows);
        (void)form;
        const int64_t wpb = threads / 32;
        int64_t blocks = (a.tiles + wpb - 1) / wpb;
        const int64_t cap = static_cast<int64_t>(occupancy(reinterpret_cast<const void*>(vec_fn), threads)) * q->sm_count;
        if (blocks > cap) blocks = cap;  // persistent: every block resident at once
        if (w.pdl && pdl_enabled()) {
            a.pdl = w.pdl;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(static_cast<unsigned>(blocks));
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = q->launch;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t e = cudaLaunchKernelEx(&cfg, vec_fn, a);
            if (e != cudaSuccess)
                return fail(SY_ERR_CUDA, "cudaLaunchKernelEx(%lld blocks x %d threads, %d-row tiles): %s (%s)",
                            static_cast<long long>(blocks), threads, tile_rows, cudaGetErrorString(e),
                            cudaGetErrorName(e));
        } else {
            vec_fn<<<static_cast<unsigned>(blocks), threads, 0, q->launch>>>(a);
        }
        q->cur_blocks += static_cast<uint64_t>(blocks);
    } else {
        a.tiles_x = 0;
        a.tiles = 0;
        const int64_t total = rows * w.nx;
        int64_t blocks = (total + 255) / 256;
        const int64_t cap = static_cast<int64_t>(q->sm_count) * 8;
        if (blocks > cap) blocks = cap;
        scalar_fn<<<static_cast<unsigned>(blocks), 256, 0, q->launch>>>(a);
        q->cur_blocks += static_cast<uint64_t>(blocks);
    }
    SY_CUDA(cudaGetLastError());
    ++q->launches;
    return SY_OK;
}

}  // namespace wave

int wave_variant_count(int, int dtype) { return dtype == SY_F32 ? wave::kVariants32 : wave::kVariants16; }

// Default per storage type and radius: the fastest variant of an exhaustive sweep at
// 8192 x 8192 on GB300 (128-thread blocks; rows per tile grow with the radius, where
// the halo re-read factor (rows + 2r) / rows matters).
int wave_default_variant(int radius, int dtype) {
    static const int kDefault[2][4] = {{1, 2, 3, 2}, {2, 2, 3, 3}};
    return kDefault[dtype == SY_F32 ? 0 : 1][radius - 1];
}

bool wave_variant_info(int radius, int dtype, int variant, int* tile_rows, int* tile_cols, int* threads) {
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0 || variant < 0 ||
        variant > wave_variant_count(radius, dtype))
        return false;
    if (variant == 0) variant = wave_default_variant(radius, dtype);
    const int V = static_cast<int>(16 / dtype_size(dtype));
    int rows, thr, cols;
    if (variant <= 8) {
        rows = wave::kTileRows[(variant - 1) % 4];
        thr = wave::kBlockThreads[(variant - 1) / 4];
        cols = 32 * V;
    } else if (variant <= 12) {  // halo lanes: 30 of a warp's 32 vectors are output
        rows = wave::kHlRows[(variant - 9) % 2];
        thr = wave::kBlockThreads[(variant - 9) / 2];
        cols = 30 * V;
    } else if (variant < wave::kMarchVariant) {  // narrow halo lanes (16-bit): 30 vectors of 4 elements
        rows = wave::kHlRows[variant - 13];
        thr = 128;
        cols = 30 * 4;
    } else {  // march (16-bit): strips of 30 vectors, segments sized per launch (nominal rows)
        rows = 32;
        thr = 128;
        cols = 30 * V;
    }
    if (tile_rows) *tile_rows = rows;
    if (threads) *threads = thr;
    if (tile_cols) *tile_cols = cols;
    return true;
}

sy_status launch_wave(Queue* q, const WaveLaunch& w) {
    int tile_rows = 0, threads = 0;
    if (!wave_variant_info(w.radius, w.dtype, w.variant, &tile_rows, nullptr, &threads))
        return fail(SY_ERR_INVALID_ARGUMENT, "bad stencil variant %d", w.variant);
    const int v = w.variant == 0 ? wave_default_variant(w.radius, w.dtype) : w.variant;
    const wave::Form form = v == wave::kMarchVariant && w.dtype != SY_F32 ? wave::Form::March
                            : v >= 13                                     ? wave::Form::Narrow
                            : v >= 9                                      ? wave::Form::Halo
                                                                          : wave::Form::Tile;
    switch (w.dtype) {
        case SY_F32: return wave::launch_f32(q, w, tile_rows, threads, form);
        case SY_BF16: return wave::launch_bf16(q, w, tile_rows, threads, form);
        case SY_F16: return wave::launch_f16(q, w, tile_rows, threads, form);
    }
    return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", w.dtype);
}

// ---------------------------------------------------------------------------
// FP64 discrete energy
// ---------------------------------------------------------------------------
namespace energy {

constexpr int kThreads = 256;

// FP64 weights of the order-2r second difference (exact rationals rounded once).
template <int R>
__device__ __forceinline__ double c0x2_64() {
    return R == 1 ? -4.0 : R == 2 ? -5.0 : R == 3 ? -49.0 / 9.0 : -205.0 / 36.0;
}
template <int R>
__device__ __forceinline__ double wk64(int k) {
    if (R == 1) return 1.0;
    if (R == 2) return k == 1 ? 4.0 / 3.0 : -1.0 / 12.0;
    if (R == 3) return k == 1 ? 1.5 : k == 2 ? -3.0 / 20.0 : 1.0 / 90.0;
    return k == 1 ? 8.0 / 5.0 : k == 2 ? -1.0 / 5.0 : k == 3 ? 8.0 / 315.0 : -1.0 / 560.0;
}

struct EArgs {
    const char* u_new;
    const char* u_old;
    int64_t ny, nx, pitch_bytes;
};

template <typename S, int R>
__global__ void __launch_bounds__(kThreads) energy_partials_kernel(EArgs a, double* partials) {
    using T = wave::Traits<S>;
    auto at = [&](const char* base, int64_t i, int64_t j) -> double {
        if (i < 0 || i >= a.ny || j < 0 || j >= a.nx) return 0.0;
        return static_cast<double>(T::load1(base + i * a.pitch_bytes + j * static_cast<int64_t>(sizeof(S))));
    };
    double kin = 0.0, pot = 0.0;
    const int64_t total = a.ny * a.nx;
    const int64_t stride = static_cast<int64_t>(kEnergyBlocks) * kThreads;
    // point p = i * nx + j; the thread's points advance by `stride`, so (i, j) moves by
    // (di, dj) per trip: one division per thread instead of two per point
    const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t di = stride / a.nx, dj = stride - di * a.nx;
    int64_t i = p0 / a.nx, j = p0 - i * a.nx;
    for (int64_t p = p0; p < total; p += stride, i += di, j += dj) {
        if (j >= a.nx) {
            j -= a.nx;
            ++i;
        }
        const double un = at(a.u_new, i, j), uo = at(a.u_old, i, j);
        double lap = __dmul_rn(c0x2_64<R>(), uo);
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            double vert = __dadd_rn(at(a.u_old, i - k, j), at(a.u_old, i + k, j));
            double horz = __dadd_rn(at(a.u_old, i, j - k), at(a.u_old, i, j + k));
            lap = __dadd_rn(lap, __dmul_rn(wk64<R>(k), __dadd_rn(vert, horz)));
        }
        const double d = __dsub_rn(un, uo);
        kin = __dadd_rn(kin, __dmul_rn(d, d));
        pot = __dadd_rn(pot, __dmul_rn(un, lap));
    }
    __shared__ double sk[kThreads], sp[kThreads];
    sk[threadIdx.x] = kin;
    sp[threadIdx.x] = pot;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] = __dadd_rn(sk[threadIdx.x], sk[threadIdx.x + s]);
            sp[threadIdx.x] = __dadd_rn(sp[threadIdx.x], sp[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sk[0];
        partials[2 * blockIdx.x + 1] = sp[0];
    }
}

// One block of kEnergyBlocks threads; partials holds 2 * kEnergyBlocks doubles.
__global__ void __launch_bounds__(kEnergyBlocks) energy_final_kernel(const double* partials, double c2,
                                                                     double* out3) {
    __shared__ double sk[kEnergyBlocks], sp[kEnergyBlocks];
    sk[threadIdx.x] = partials[2 * threadIdx.x];
    sp[threadIdx.x] = partials[2 * threadIdx.x + 1];
    __syncthreads();
    for (int s = kEnergyBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] = __dadd_rn(sk[threadIdx.x], sk[threadIdx.x + s]);
            sp[threadIdx.x] = __dadd_rn(sp[threadIdx.x], sp[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out3[0] = __dsub_rn(sk[0], __dmul_rn(c2, sp[0]));
        out3[1] = sk[0];
        out3[2] = sp[0];
    }
}

template <typename S>
void launch_partials(int radius, EArgs a, double* partials, cudaStream_t s) {
    switch (radius) {
        case 1: energy_partials_kernel<S, 1><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        case 2: energy_partials_kernel<S, 2><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        case 3: energy_partials_kernel<S, 3><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        default: energy_partials_kernel<S, 4><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
    }
}

}  // namespace energy

namespace {

// Both energy kernels on `stream`: partials (2 * kEnergyBlocks doubles) then the
// three results (energy, kinetic, potential) into out3 (device).
sy_status launch_energy_on(cudaStream_t stream, const sy_stencil_params* p, const void* u_new, const void* u_old,
                           double* partials, double* out3) {
    const size_t esize = dtype_size(p->dtype);
    if ((reinterpret_cast<uintptr_t>(u_new) % esize) || (reinterpret_cast<uintptr_t>(u_old) % esize))
        return fail(SY_ERR_INVALID_ARGUMENT, "field pointers must be aligned to the element size");
    energy::EArgs a;
    a.u_new = static_cast<const char*>(u_new);
    a.u_old = static_cast<const char*>(u_old);
    a.ny = p->ny;
    a.nx = p->nx;
    a.pitch_bytes = p->pitch * static_cast<int64_t>(esize);
    switch (p->dtype) {
        case SY_F32: energy::launch_partials<float>(p->radius, a, partials, stream); break;
        case SY_BF16: energy::launch_partials<__nv_bfloat16>(p->radius, a, partials, stream); break;
        default: energy::launch_partials<__half>(p->radius, a, partials, stream); break;
    }
    SY_CUDA(cudaGetLastError());
    energy::energy_final_kernel<<<1, kEnergyBlocks, 0, stream>>>(partials, static_cast<double>(p->c2), out3);
    SY_CUDA(cudaGetLastError());
    return SY_OK;
}

}  // namespace

sy_status launch_energy_final(cudaStream_t stream, const double* partials, double c2, double* out3) {
    energy::energy_final_kernel<<<1, kEnergyBlocks, 0, stream>>>(partials, c2, out3);
    SY_CUDA(cudaGetLastError());
    return SY_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free energy reduction (sy_wave_energy_static)
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory where they need the energy: code
// issuing work while a stream is captured into a CUDA graph in global mode
// (cudaMalloc is not permitted then), applications whose own allocator owns all
// device memory, and loops that must never hit the device-wide synchronisation
// cudaMalloc/cudaFree can cause.  For them the per-block partial sums live in
// this module-scope array instead of the queue's scratch.  Size: 2 x
// kEnergyBlocks doubles = 16 KiB, held by every GPU that loads the library until
// the process exits.  Host code must not pass the array's name to a kernel (on
// the host it names a stand-in, not device memory): it uses the address that
// cudaGetSymbolAddress returns for the current device, looked up once per device.
constexpr int kStaticEnergyDoubles = 2 * kEnergyBlocks;
static __device__ __align__(256) double g_energy_partials_static[kStaticEnergyDoubles];
// The reduction's shape is fixed: it always writes 2 x kEnergyBlocks partial sums,
// whatever the grid size, so the array's size is checked once, here.
static_assert(2 * kEnergyBlocks <= kStaticEnergyDoubles, "static energy scratch too small for the reduction");

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of the static partials on the current device (set up on the
// first call per device).
sy_status static_partials(double** out) {
    int dev = -1;
    SY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SY_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_energy_partials_static);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_energy_partials_static)");
        g_static_addr[dev] = ptr;
    }
    *out = static_cast<double*>(g_static_addr[dev]);
    return SY_OK;
}
}  // namespace

sy_status launch_wave_energy(Queue* q, const sy_stencil_params* p, const void* u_new, const void* u_old,
                             double* partials, int n_partials, double* out3_device) {
    if (n_partials != kEnergyBlocks) return fail(SY_ERR_INVALID_ARGUMENT, "energy partials must be %d", kEnergyBlocks);
    SY_TRY(launch_energy_on(q->launch, p, u_new, u_old, partials, out3_device));
    q->launches += 2;
    return SY_OK;
}

}  // namespace sy

extern "C" sy_status sy_wave_energy_static(void* cuda_stream, const sy_stencil_params* p, const void* u_new,
                                           const void* u_old, double* out3) {
    using namespace sy;
    SY_TRY(stencil_param_checks(p));
    if (!out3) return fail(SY_ERR_NULL_POINTER, "out3 is NULL");
    if (reinterpret_cast<uintptr_t>(out3) % alignof(double))
        return fail(SY_ERR_INVALID_ARGUMENT, "out3 must be 8-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (p->ny == 0 || p->nx == 0) {
        SY_CUDA(cudaMemsetAsync(out3, 0, 3 * sizeof(double), stream));
        return SY_OK;
    }
    if (!u_new || !u_old) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    double* partials = nullptr;
    SY_TRY(static_partials(&partials));
    return launch_energy_on(stream, p, u_new, u_old, partials, out3);
}
