// Host side of the 3D leapfrog step: argument checks, one launch per chunk of
// planes (each timed like the 2D chunks), the start form, and the variant table.
#include "sy_internal.h"

namespace sy {

sy_status stencil3d_param_checks(const sy_stencil3d_params* p) {
    if (!p) return fail(SY_ERR_NULL_POINTER, "params is NULL");
    if (p->nz < 0 || p->ny < 0 || p->nx < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative grid size");
    if (p->pitch < p->nx)
        return fail(SY_ERR_INVALID_ARGUMENT, "pitch %lld < nx %lld", (long long)p->pitch, (long long)p->nx);
    if (p->plane < p->ny * p->pitch)
        return fail(SY_ERR_INVALID_ARGUMENT, "plane stride %lld < ny x pitch = %lld", (long long)p->plane,
                    (long long)(p->ny * p->pitch));
    if (p->radius < 1 || p->radius > 4) return fail(SY_ERR_INVALID_ARGUMENT, "radius %d not in 1..4", p->radius);
    if (dtype_size(p->dtype) == 0) return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", p->dtype);
    if (p->variant < 0 || p->variant > kWave3dVariants)
        return fail(SY_ERR_INVALID_ARGUMENT, "variant %d not in 0..%d", p->variant, kWave3dVariants);
    return SY_OK;
}

sy_status stencil3d_common(Queue* q, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                           void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                           sy_event* chunk_events, bool start, bool reverse) {
    SY_TRY(stencil3d_param_checks(p));
    if ((p->nz == 0 || p->ny == 0 || p->nx == 0) && n_chunks == 0) return SY_OK;
    SY_TRY(validate_chunks(p->nz, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    if (!u_cur || !u_next || (!start && !u_prev)) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    const size_t bytes = static_cast<size_t>(p->nz) * static_cast<size_t>(p->plane) * dtype_size(p->dtype);
    if (ranges_overlap(u_next, bytes, u_cur, bytes)) return fail(SY_ERR_ALIAS, "u_next overlaps u_cur");
    if (!start && u_next != u_prev && ranges_overlap(u_next, bytes, u_prev, bytes))
        return fail(SY_ERR_ALIAS, "u_next partially overlaps u_prev");
    SY_TRY(use_device(q));
    for (int i = 0; i < n_chunks; ++i) {
        const int c = reverse ? n_chunks - 1 - i : i;
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, chunk_events ? &chunk_events[c] : nullptr, &rec));
        WaveLaunch3 w;
        w.nz = p->nz;
        w.ny = p->ny;
        w.nx = p->nx;
        w.pitch = p->pitch;
        w.plane = p->plane;
        w.radius = p->radius;
        w.dtype = p->dtype;
        w.variant = p->variant;
        w.c2 = start ? 0.5f * p->c2 : p->c2;
        w.start = start;
        w.u_prev = start ? u_cur : u_prev;
        w.u_cur = u_cur;
        w.u_next = u_next;
        w.z_begin = chunks[c].begin;
        w.z_end = chunks[c].end;
        w.pdl = i == 0 ? 1 : 2;  // the first launch waits for the previous step; the rest overlap it
        SY_TRY(launch_wave3d(q, w));
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}

}  // namespace sy

using namespace sy;

extern "C" {

sy_status sy_stencil3d_step(sy_queue_t qh, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                            void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                            sy_event* chunk_events) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return stencil3d_common(q, p, u_prev, u_cur, u_next, chunks, n_chunks, halo_radius, chunk_events, false);
}

sy_status sy_stencil3d_start(sy_queue_t qh, const sy_stencil3d_params* p, const void* u0, void* u_m1,
                             const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* chunk_events) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return stencil3d_common(q, p, nullptr, u0, u_m1, chunks, n_chunks, halo_radius, chunk_events, true);
}

sy_status sy_stencil3d_step_planes(sy_queue_t qh, const sy_stencil3d_params* p, const void* u_prev,
                                   const void* u_cur, void* u_next, int64_t plane_begin, int64_t plane_end,
                                   int halo_radius, int start, sy_event* ev) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil3d_param_checks(p));
    if (plane_begin < 0 || plane_end < plane_begin || plane_end > p->nz)
        return fail(SY_ERR_BAD_CHUNKS, "planes [%lld, %lld) outside [0, %lld)", (long long)plane_begin,
                    (long long)plane_end, (long long)p->nz);
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    if (!u_cur || !u_next || (!start && !u_prev)) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    const size_t bytes = static_cast<size_t>(p->nz) * static_cast<size_t>(p->plane) * dtype_size(p->dtype);
    if (ranges_overlap(u_next, bytes, u_cur, bytes)) return fail(SY_ERR_ALIAS, "u_next overlaps u_cur");
    if (!start && u_next != u_prev && ranges_overlap(u_next, bytes, u_prev, bytes))
        return fail(SY_ERR_ALIAS, "u_next partially overlaps u_prev");
    SY_TRY(use_device(q));
    EventRecord* rec = nullptr;
    SY_TRY(begin_event(q, ev, &rec));
    WaveLaunch3 w;
    w.nz = p->nz;
    w.ny = p->ny;
    w.nx = p->nx;
    w.pitch = p->pitch;
    w.plane = p->plane;
    w.radius = p->radius;
    w.dtype = p->dtype;
    w.variant = p->variant;
    w.c2 = start ? 0.5f * p->c2 : p->c2;
    w.start = start != 0;
    w.u_prev = start ? u_cur : u_prev;
    w.u_cur = u_cur;
    w.u_next = u_next;
    w.z_begin = plane_begin;
    w.z_end = plane_end;
    w.pdl = 0;
    SY_TRY(launch_wave3d(q, w));
    return end_event(q, rec);
}

sy_status sy_wave3d_energy(sy_queue_t qh, const sy_stencil3d_params* p, const void* u_new, const void* u_old,
                           double* energy, double* kinetic, double* potential) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil3d_param_checks(p));
    if (!energy) return fail(SY_ERR_NULL_POINTER, "energy out is NULL");
    if (p->nz == 0 || p->ny == 0 || p->nx == 0) {
        *energy = 0.0;
        if (kinetic) *kinetic = 0.0;
        if (potential) *potential = 0.0;
        return SY_OK;
    }
    if (!u_new || !u_old) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    SY_TRY(use_device(q));
    void* scratch = nullptr;
    SY_TRY(queue_scratch(q, sizeof(double) * (2 * kEnergyBlocks + 3), &scratch));
    double* partials = static_cast<double*>(scratch);
    double* out3 = partials + 2 * kEnergyBlocks;
    SY_TRY(launch_wave3d_energy(q, p, u_new, u_old, partials, out3));
    double host[3];
    SY_CUDA(cudaMemcpyAsync(host, out3, sizeof host, cudaMemcpyDeviceToHost, q->stream));
    SY_CUDA(cudaStreamSynchronize(q->stream));
    *energy = host[0];
    if (kinetic) *kinetic = host[1];
    if (potential) *potential = host[2];
    return SY_OK;
}

sy_status sy_stencil3d_variant_count(int radius, int dtype, int* count) {
    clear_error();
    if (!count) return fail(SY_ERR_NULL_POINTER, "count is NULL");
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0)
        return fail(SY_ERR_INVALID_ARGUMENT, "radius %d / dtype %d", radius, dtype);
    *count = kWave3dVariants;
    return SY_OK;
}

sy_status sy_stencil3d_variant_info(int radius, int dtype, int variant, int* tile_rows, int* threads) {
    clear_error();
    if (!wave3d_variant_info(radius, dtype, variant, tile_rows, threads))
        return fail(SY_ERR_INVALID_ARGUMENT, "radius %d / dtype %d / variant %d", radius, dtype, variant);
    return SY_OK;
}

}  // extern "C"
