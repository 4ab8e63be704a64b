// Launch logic of the 3D wave step: layout checks, the variant table, and the
// choice of plane-segment length that gives every persistent warp the same
// number of tasks.
#include "wave3d_kernel.cuh"

namespace sy {
namespace wave3 {

namespace {
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Planes per segment: minimises the busiest warp's plane loads, rounds x (seg + R)
// (a segment's first 2R planes are re-read, mostly from L2, where the previous
// segment's warp has just read them); ties go to the longer segment.
int64_t choose_seg(int64_t tiles_xy, int64_t planes, int64_t nwarps, int R) {
    int64_t best = planes, best_cost = -1;
    const int64_t hi = planes < 64 ? planes : 64;
    for (int64_t seg = 1; seg <= hi; ++seg) {
        const int64_t segs = (planes + seg - 1) / seg;
        const int64_t rounds = (tiles_xy * segs + nwarps - 1) / nwarps;
        const int64_t cost = rounds * (seg + R);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && seg > best)) {
            best = seg;
            best_cost = cost;
        }
    }
    return best;
}
}  // namespace

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
    if (!aligned(w.u_cur, esize) || !aligned(w.u_next, esize) || (!w.start && !aligned(w.u_prev, esize)))
        return fail(SY_ERR_INVALID_ARGUMENT, "field pointers must be aligned to the element size (%zu bytes)", esize);
    const bool vec_ok = aligned(w.u_cur, 16) && aligned(w.u_next, 16) && (w.start || aligned(w.u_prev, 16)) &&
                        (a.pitch_bytes % 16) == 0 && (a.plane_bytes % 16) == 0;
    if (vec_ok) {
        const int64_t span = 32 * static_cast<int64_t>(V);
        a.tiles_x = (w.nx + span - 1) / span;
        a.tiles_y = (w.ny + rows - 1) / rows;
        const int64_t wpb = threads / 32;
        const int64_t cap = static_cast<int64_t>(wave::kernel_occupancy(reinterpret_cast<const void*>(vec_fn),
                                                                        threads)) * q->sm_count;
        a.seg = choose_seg(a.tiles_x * a.tiles_y, planes, cap * wpb, w.radius);
        a.segs = (planes + a.seg - 1) / a.seg;
        a.tasks = a.tiles_x * a.tiles_y * a.segs;
        int64_t blocks = (a.tasks + wpb - 1) / wpb;
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

}  // namespace wave3

bool wave3d_variant_info(int radius, int dtype, int variant, int* tile_rows, int* threads) {
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0 || variant < 0 || variant > wave3::kVariants3)
        return false;
    int rows, thr;
    if (variant == 0) {
        // Default per radius: the fastest tile of a sweep at 512^3 (FP32) on GB300.
        // One-row tiles win at radius 1: the register queue ((2r+1) x rows vectors
        // per lane) sets how many warps stay resident, and the extra halo rows
        // ((rows + 2r) / rows) come from L2.
        static const int kDefault[4] = {1, 2, 2, 2};
        rows = kDefault[radius - 1];
        thr = 128;
    } else {
        const int* table = radius <= 2 ? wave3::kRows12 : wave3::kRows34;
        rows = table[(variant - 1) % 3];
        thr = wave3::kThreads3[(variant - 1) / 3];
    }
    if (tile_rows) *tile_rows = rows;
    if (threads) *threads = thr;
    return true;
}

sy_status launch_wave3d(Queue* q, const WaveLaunch3& w) {
    int rows = 0, threads = 0;
    if (!wave3d_variant_info(w.radius, w.dtype, w.variant, &rows, &threads))
        return fail(SY_ERR_INVALID_ARGUMENT, "bad 3D stencil variant %d", w.variant);
    switch (w.dtype) {
        case SY_F32: return wave3::launch3_f32(q, w, rows, threads);
        case SY_BF16: return wave3::launch3_bf16(q, w, rows, threads);
        case SY_F16: return wave3::launch3_f16(q, w, rows, threads);
    }
    return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", w.dtype);
}

}  // namespace sy
