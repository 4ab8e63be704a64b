// Launch logic of the 3D wave step: layout checks, the variant table, and the
// choice of plane-segment length that gives every persistent warp the same
// number of tasks; and the FP64 discrete energy of the 3D scheme,
//   E^{n+1/2} = sum (u_new - u_old)^2 - c2 * sum u_new * (L u_old),
// with the fixed reduction shape of the 2D one (kEnergyBlocks x 256 threads, fixed
// trees), so repeated calls give identical bits.
#include "wave3d_tma.cuh"

namespace sy {
namespace wave3 {

namespace {
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
}  // namespace

// Planes per segment: minimises the busiest worker's plane loads, rounds x (seg + R)
// (a segment's first 2R planes are re-read, mostly from L2, where the previous
// segment's worker has just read them); ties go to the longer segment.  A worker
// is a warp (warp-column kernel) or a block (slab and TMA kernels).
int64_t choose_seg(int64_t tiles_xy, int64_t planes, int64_t workers, int R) {
    int64_t best = planes, best_cost = -1;
    const int64_t hi = planes < 64 ? planes : 64;
    for (int64_t seg = 1; seg <= hi; ++seg) {
        const int64_t segs = (planes + seg - 1) / seg;
        const int64_t rounds = (tiles_xy * segs + workers - 1) / workers;
        const int64_t cost = rounds * (seg + R);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && seg > best)) {
            best = seg;
            best_cost = cost;
        }
    }
    return best;
}

sy_status launch3_typed(Queue* q, const WaveLaunch3& w, KernelFn3 vec_fn, KernelFn3 scalar_fn, int rows, int threads,
                        int V, size_t esize) {
    const int64_t planes = w.z_end - w.z_begin;
    if (planes <= 0 || w.ny == 0 || w.nx == 0) return SY_OK;
    Args3 a;
    a.u_prev = static_cast<const char*>(w.u_prev);
    a.u_cur = static_cast<const char*>(w.u_cur);
    a.u_next = static_cast<char*>(w.u_next);
    a.nz = w.nz;
    a.ny = w.ny;
    a.nx = w.nx;
    a.pitch_bytes = w.pitch * static_cast<int64_t>(esize);
    a.plane_bytes = w.plane * static_cast<int64_t>(esize);
    a.z_begin = w.z_begin;
    a.z_end = w.z_end;
    a.c2 = w.c2;
    a.stamp = q->cur_stamp;
    a.pdl = 0;
    a.neg0 = -0.0f;
    if (!aligned(w.u_cur, esize) || !aligned(w.u_next, esize) || (!w.start && !aligned(w.u_prev, esize)))
        return fail(SY_ERR_INVALID_ARGUMENT, "field pointers must be aligned to the element size (%zu bytes)", esize);
    const bool vec_ok = aligned(w.u_cur, 16) && aligned(w.u_next, 16) && (w.start || aligned(w.u_prev, 16)) &&
                        (a.pitch_bytes % 16) == 0 && (a.plane_bytes % 16) == 0;
    if (vec_ok) {
        const int64_t span = 32 * static_cast<int64_t>(V);
        const bool slab = rows < 0;
        const int64_t tile_rows = slab ? -rows : rows;
        a.tiles_x = (w.nx + span - 1) / span;
        a.tiles_y = (w.ny + tile_rows - 1) / tile_rows;
        // a task is one warp's (warp-column kernel) or one block's (slab kernel)
        const int64_t tasks_per_block = slab ? 1 : threads / 32;
        const int64_t cap = static_cast<int64_t>(wave::kernel_occupancy(reinterpret_cast<const void*>(vec_fn),
                                                                        threads)) * q->sm_count;
        a.seg = choose_seg(a.tiles_x * a.tiles_y, planes, cap * tasks_per_block, w.radius);
        a.segs = (planes + a.seg - 1) / a.seg;
        a.tasks = a.tiles_x * a.tiles_y * a.segs;
        int64_t blocks = (a.tasks + tasks_per_block - 1) / tasks_per_block;
        if (blocks > cap) blocks = cap;  // persistent: every block resident at once
        if (w.pdl && wave::launch_overlap_enabled()) {
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
            SY_CUDA(cudaLaunchKernelEx(&cfg, vec_fn, a));
        } else {
            vec_fn<<<static_cast<unsigned>(blocks), threads, 0, q->launch>>>(a);
        }
        q->cur_blocks += static_cast<uint64_t>(blocks);
    } else {
        a.tiles_x = a.tiles_y = a.seg = a.segs = a.tasks = 0;
        const int64_t total = planes * w.ny * w.nx;
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

namespace energy3 {

constexpr int kThreads = 256;

// FP64 weights: 3 w_0 and w_k of the order-2r second difference (rationals rounded once).
template <int R>
__device__ __forceinline__ double c0x3_64() {
    return R == 1 ? -6.0 : R == 2 ? -7.5 : R == 3 ? -49.0 / 6.0 : -205.0 / 24.0;
}
template <int R>
__device__ __forceinline__ double wk64(int k) {
    if (R == 1) return 1.0;
    if (R == 2) return k == 1 ? 4.0 / 3.0 : -1.0 / 12.0;
    if (R == 3) return k == 1 ? 1.5 : k == 2 ? -3.0 / 20.0 : 1.0 / 90.0;
    return k == 1 ? 8.0 / 5.0 : k == 2 ? -1.0 / 5.0 : k == 3 ? 8.0 / 315.0 : -1.0 / 560.0;
}

struct EArgs3 {
    const char* u_new;
    const char* u_old;
    int64_t nz, ny, nx, pitch_bytes, plane_bytes;
};

template <typename S, int R>
__global__ void __launch_bounds__(kThreads) energy3_partials_kernel(EArgs3 a, double* partials) {
    using T = Traits<S>;
    auto at = [&](const char* base, int64_t z, int64_t y, int64_t x) -> double {
        if (z < 0 || z >= a.nz || y < 0 || y >= a.ny || x < 0 || x >= a.nx) return 0.0;
        return static_cast<double>(
            T::load1(base + z * a.plane_bytes + y * a.pitch_bytes + x * static_cast<int64_t>(sizeof(S))));
    };
    double kin = 0.0, pot = 0.0;
    const int64_t per_plane = a.ny * a.nx;
    const int64_t total = a.nz * per_plane;
    const int64_t stride = static_cast<int64_t>(kEnergyBlocks) * kThreads;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; p < total; p += stride) {
        const int64_t z = p / per_plane;
        const int64_t rem = p - z * per_plane;
        const int64_t y = rem / a.nx, x = rem - y * a.nx;
        const double un = at(a.u_new, z, y, x), uo = at(a.u_old, z, y, x);
        double lap = __dmul_rn(c0x3_64<R>(), uo);
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            const double vert = __dadd_rn(at(a.u_old, z, y - k, x), at(a.u_old, z, y + k, x));
            const double horz = __dadd_rn(at(a.u_old, z, y, x - k), at(a.u_old, z, y, x + k));
            const double depth = __dadd_rn(at(a.u_old, z - k, y, x), at(a.u_old, z + k, y, x));
            lap = __dadd_rn(lap, __dmul_rn(wk64<R>(k), __dadd_rn(__dadd_rn(vert, horz), depth)));
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

template <typename S>
void launch_partials(int radius, EArgs3 a, double* partials, cudaStream_t s) {
    switch (radius) {
        case 1: energy3_partials_kernel<S, 1><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        case 2: energy3_partials_kernel<S, 2><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        case 3: energy3_partials_kernel<S, 3><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
        default: energy3_partials_kernel<S, 4><<<kEnergyBlocks, kThreads, 0, s>>>(a, partials); break;
    }
}

}  // namespace energy3
}  // namespace wave3

sy_status launch_wave3d_energy(Queue* q, const sy_stencil3d_params* p, const void* u_new, const void* u_old,
                               double* partials, double* out3_device) {
    const size_t esize = dtype_size(p->dtype);
    if ((reinterpret_cast<uintptr_t>(u_new) % esize) || (reinterpret_cast<uintptr_t>(u_old) % esize))
        return fail(SY_ERR_INVALID_ARGUMENT, "field pointers must be aligned to the element size");
    wave3::energy3::EArgs3 a;
    a.u_new = static_cast<const char*>(u_new);
    a.u_old = static_cast<const char*>(u_old);
    a.nz = p->nz;
    a.ny = p->ny;
    a.nx = p->nx;
    a.pitch_bytes = p->pitch * static_cast<int64_t>(esize);
    a.plane_bytes = p->plane * static_cast<int64_t>(esize);
    switch (p->dtype) {
        case SY_F32: wave3::energy3::launch_partials<float>(p->radius, a, partials, q->launch); break;
        case SY_BF16: wave3::energy3::launch_partials<__nv_bfloat16>(p->radius, a, partials, q->launch); break;
        default: wave3::energy3::launch_partials<__half>(p->radius, a, partials, q->launch); break;
    }
    SY_CUDA(cudaGetLastError());
    SY_TRY(launch_energy_final(q->launch, partials, static_cast<double>(p->c2), out3_device));
    q->launches += 2;
    return SY_OK;
}

namespace {
// The default variant per storage class and radius: the fastest of a sweep at 512^3 on
// GB300 (FP32 radius 1 / 2 / 4: 5.3e11 / 4.2e11 / 2.2e11 updates/s; BF16 radius 1 / 2 / 4:
// 9.4e11 / 6.0e11 / 2.5e11).  Warp columns of one row except FP32 radius 2 (two rows):
// the register queue, (2r+1) x rows vectors per lane, sets how many warps stay resident;
// 16-bit radius 2 and 4 run them in blocks of 256 threads.  The slab and TMA variants
// measured slower (see their kernels), except 16-bit radius 4, where TMA strips of 32
// rows tie with the default (2.53e11).
constexpr int kDefaultVariant3[2][4] = {{1, 2, 1, 1}, {1, 4, 1, 4}};

enum class Form3 { column, slab, tma };

// Resolved variant -> (rows, threads, form).
bool variant3(int radius, int dtype, int variant, int* rows, int* threads, Form3* form) {
    const int v = variant == 0 ? kDefaultVariant3[dtype == SY_F32 ? 0 : 1][radius - 1] : variant;
    if (v <= wave3::kColumnVariants3) {
        const int* table = radius <= 2 ? wave3::kRows12 : wave3::kRows34;
        *rows = table[(v - 1) % 3];
        *threads = wave3::kThreads3[(v - 1) / 3];
        *form = Form3::column;
    } else if (v <= wave3::kColumnVariants3 + 2) {
        *rows = wave3::kSlabWarps * (v - wave3::kColumnVariants3);
        *threads = wave3::kSlabWarps * 32;
        *form = Form3::slab;
    } else {
        *rows = 2 * wave3::kTmaWarps * (v - wave3::kColumnVariants3 - 2);  // strips of 16 or 32 rows
        *threads = wave3::kTmaWarps * 32;
        *form = Form3::tma;
    }
    return true;
}
}  // namespace

static_assert(kWave3dVariants == wave3::kVariants3, "the ABI's 3D variant count is the kernel table's");

bool wave3d_variant_info(int radius, int dtype, int variant, int* tile_rows, int* threads) {
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0 || variant < 0 || variant > wave3::kVariants3)
        return false;
    int rows = 0, thr = 0;
    Form3 form = Form3::column;
    variant3(radius, dtype, variant, &rows, &thr, &form);
    if (tile_rows) *tile_rows = rows;
    if (threads) *threads = thr;
    return true;
}

sy_status launch_wave3d(Queue* q, const WaveLaunch3& w) {
    int rows = 0, threads = 0;
    Form3 form = Form3::column;
    if (!wave3d_variant_info(w.radius, w.dtype, w.variant, nullptr, nullptr))
        return fail(SY_ERR_INVALID_ARGUMENT, "bad 3D stencil variant %d", w.variant);
    variant3(w.radius, w.dtype, w.variant, &rows, &threads, &form);
    if (form == Form3::tma) {
        const size_t es = dtype_size(w.dtype);
        const bool tma_ok = wave3::aligned(w.u_cur, 16) && wave3::aligned(w.u_next, 16) &&
                            (w.start || wave3::aligned(w.u_prev, 16)) &&
                            (w.pitch * es) % 16 == 0 && (w.plane * es) % 16 == 0 &&
                            // TMA coordinates are 32-bit
                            w.nz + 64 < (int64_t{1} << 31) && w.ny + 64 < (int64_t{1} << 31) &&
                            w.nx + 64 < (int64_t{1} << 31);
        const int64_t planes = w.z_end - w.z_begin;
        if (planes <= 0 || w.ny == 0 || w.nx == 0) return SY_OK;
        if (tma_ok) {
            switch (w.dtype) {
                case SY_F32: return wave3::launch3_tma_f32(q, w, rows);
                case SY_BF16: return wave3::launch3_tma_bf16(q, w, rows);
                case SY_F16: return wave3::launch3_tma_f16(q, w, rows);
            }
        }
        rows = 1;  // unaligned layouts and fields of 2^31 planes, rows or columns: the column family
        threads = 128;
        form = Form3::column;
    }
    if (form == Form3::slab) rows = -rows;
    switch (w.dtype) {
        case SY_F32: return wave3::launch3_f32(q, w, rows, threads);
        case SY_BF16: return wave3::launch3_bf16(q, w, rows, threads);
        case SY_F16: return wave3::launch3_f16(q, w, rows, threads);
    }
    return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", w.dtype);
}

}  // namespace sy
