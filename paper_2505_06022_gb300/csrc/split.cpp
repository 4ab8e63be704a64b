// Split-buffer execution: every chunk keeps its rows in a buffer of its own, as a
// chunk placed on another device would (paper §3: the runtime splits a kernel
// across devices and infers from the range mappers which data must be moved
// before each chunk runs).
//
// Local layout of chunk c = [a, b): halo_lo rows above (global rows a - halo_lo ..
// a - 1), then its own b - a rows, then halo_hi rows below; halo_lo =
// min(h, a) and halo_hi = min(h, ny - b) for halo radius h, so a local buffer
// starts or ends exactly at the domain edge where the chunk does, and the
// kernel's zero ghosts beyond the local buffer are the domain's Dirichlet zeros.
//
// Transfers: the neighbourhood range mapper of chunk c reads [a - h, b + h)
// clipped to the domain; the rows of that region it does not write belong to
// other chunks and are copied from their owners' buffers before the step (each
// run of rows with one owner is one transfer; a chunk shorter than h makes a
// region span several owners).  One halo-exchange kernel does all of a step's
// transfers; it and the chunk kernels overlap their launches (programmatic
// dependent launch), each waiting for its predecessor before reading.
#include <vector>

#include "sy_internal.h"

using namespace sy;

namespace {

struct Layout {
    int64_t halo_lo, halo_hi, rows;
};

Layout layout_of(int64_t ny, const sy_chunk& c, int h) {
    Layout L;
    L.halo_lo = c.begin < h ? c.begin : h;
    L.halo_hi = ny - c.end < h ? ny - c.end : h;
    L.rows = L.halo_lo + (c.end - c.begin) + L.halo_hi;
    return L;
}

int owner_of(const sy_chunk* chunks, int n, int64_t row) {
    int lo = 0, hi = n - 1;  // chunks tile [0, ny) in order
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (chunks[mid].begin <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

sy_status transfers(int64_t ny, const sy_chunk* chunks, int n, int h, std::vector<sy_transfer>* out) {
    out->clear();
    for (int c = 0; c < n; ++c) {
        sy_chunk region;
        SY_TRY(sy_rm_neighbourhood(chunks[c], h, ny, &region));
        // the parts of the read region outside [begin, end): above, then below
        const int64_t parts[2][2] = {{region.begin, chunks[c].begin}, {chunks[c].end, region.end}};
        for (const auto& part : parts) {
            int64_t row = part[0];
            while (row < part[1]) {
                const int src = owner_of(chunks, n, row);
                const int64_t stop = chunks[src].end < part[1] ? chunks[src].end : part[1];
                out->push_back(sy_transfer{src, c, row, stop});
                row = stop;
            }
        }
    }
    return SY_OK;
}

}  // namespace

extern "C" {

sy_status sy_rm_transfers(int64_t ny, const sy_chunk* chunks, int n_chunks, int halo_radius, sy_transfer* out,
                          int max_out, int* n_out) {
    if (!n_out) return fail(SY_ERR_NULL_POINTER, "n_out is NULL");
    if (halo_radius < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative halo radius");
    SY_TRY(validate_chunks(ny, chunks, n_chunks));
    std::vector<sy_transfer> t;
    SY_TRY(transfers(ny, chunks, n_chunks, halo_radius, &t));
    *n_out = static_cast<int>(t.size());
    if (!out) return SY_OK;  // size query
    if (max_out < static_cast<int>(t.size()))
        return fail(SY_ERR_INVALID_ARGUMENT, "out holds %d transfers, need %zu", max_out, t.size());
    for (size_t i = 0; i < t.size(); ++i) out[i] = t[i];
    return SY_OK;
}

sy_status sy_split_layout(int64_t ny, const sy_chunk* chunks, int n_chunks, int halo_radius, int chunk,
                          int64_t* halo_lo, int64_t* halo_hi, int64_t* local_rows) {
    SY_TRY(validate_chunks(ny, chunks, n_chunks));
    if (chunk < 0 || chunk >= n_chunks) return fail(SY_ERR_INVALID_ARGUMENT, "chunk %d out of range", chunk);
    if (halo_radius < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative halo radius");
    const Layout L = layout_of(ny, chunks[chunk], halo_radius);
    if (halo_lo) *halo_lo = L.halo_lo;
    if (halo_hi) *halo_hi = L.halo_hi;
    if (local_rows) *local_rows = L.rows;
    return SY_OK;
}

}  // extern "C"

namespace {

sy_status split_common(Queue* q, const sy_stencil_params* p, void* const* local_prev, void* const* local_cur,
                       void* const* local_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                       sy_event* chunk_events, bool start) {
    SY_TRY(stencil_param_checks(p));
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    if ((!start && !local_prev) || !local_cur || !local_next) return fail(SY_ERR_NULL_POINTER, "buffer list is NULL");
    const size_t es = dtype_size(p->dtype);
    const size_t pb = static_cast<size_t>(p->pitch) * es;
    std::vector<Layout> lay(n_chunks);
    for (int c = 0; c < n_chunks; ++c) {
        lay[c] = layout_of(p->ny, chunks[c], halo_radius);
        if ((!start && !local_prev[c]) || !local_cur[c] || !local_next[c])
            return fail(SY_ERR_NULL_POINTER, "chunk %d: buffer is NULL", c);
        const size_t bytes = static_cast<size_t>(lay[c].rows) * pb;
        if (ranges_overlap(local_next[c], bytes, local_cur[c], bytes))
            return fail(SY_ERR_ALIAS, "chunk %d: u_next overlaps u_cur", c);
        if (!start && local_next[c] != local_prev[c] && ranges_overlap(local_next[c], bytes, local_prev[c], bytes))
            return fail(SY_ERR_ALIAS, "chunk %d: u_next partially overlaps u_prev", c);
    }
    SY_TRY(use_device(q));
    // 1. halo rows of u_cur from their owners (inferred from the range mappers), all
    //    of the step's transfers in one kernel
    std::vector<sy_transfer> t;
    SY_TRY(transfers(p->ny, chunks, n_chunks, halo_radius, &t));
    std::vector<HaloCopy> copies;
    copies.reserve(t.size());
    for (const sy_transfer& x : t) {
        const int64_t src_row = x.row_begin - chunks[x.src].begin + lay[x.src].halo_lo;
        const int64_t dst_row = x.row_begin - chunks[x.dst].begin + lay[x.dst].halo_lo;
        copies.push_back(HaloCopy{static_cast<const char*>(local_cur[x.src]) + src_row * pb,
                                  static_cast<char*>(local_cur[x.dst]) + dst_row * pb, x.row_end - x.row_begin});
    }
    SY_TRY(launch_halo(q, copies.data(), static_cast<int>(copies.size()), static_cast<int64_t>(pb),
                       p->nx * static_cast<int64_t>(es), true));
    // 2. each chunk steps its own rows of a local grid of halo_lo + len + halo_hi rows
    for (int c = 0; c < n_chunks; ++c) {
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, chunk_events ? &chunk_events[c] : nullptr, &rec));
        WaveLaunch w;
        w.ny = lay[c].rows;
        w.nx = p->nx;
        w.pitch = p->pitch;
        w.radius = p->radius;
        w.dtype = p->dtype;
        w.variant = p->variant;
        w.c2 = start ? 0.5f * p->c2 : p->c2;
        w.start = start;
        w.u_prev = start ? local_cur[c] : local_prev[c];
        w.u_cur = local_cur[c];
        w.u_next = local_next[c];
        w.row_begin = lay[c].halo_lo;
        w.row_end = lay[c].halo_lo + (chunks[c].end - chunks[c].begin);
        // the first chunk waits for the halo exchange (or, with none, the previous step);
        // the others start once it has, so both are complete before they read
        w.pdl = c == 0 ? 1 : 2;
        SY_TRY(launch_wave(q, w));
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}

}  // namespace

extern "C" {

sy_status sy_stencil_step_split(sy_queue_t qh, const sy_stencil_params* p, void* const* local_prev,
                                void* const* local_cur, void* const* local_next, const sy_chunk* chunks,
                                int n_chunks, int halo_radius, sy_event* chunk_events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return split_common(q, p, local_prev, local_cur, local_next, chunks, n_chunks, halo_radius, chunk_events,
                        false);
}

sy_status sy_stencil_start_split(sy_queue_t qh, const sy_stencil_params* p, void* const* local_u0,
                                 void* const* local_um1, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                 sy_event* chunk_events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return split_common(q, p, nullptr, local_u0, local_um1, chunks, n_chunks, halo_radius, chunk_events, true);
}

sy_status sy_stencil_step_rows(sy_queue_t qh, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                               void* u_next, int64_t row_begin, int64_t row_end, int halo_radius, int start,
                               sy_event* ev) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (row_begin < 0 || row_end < row_begin || row_end > p->ny)
        return fail(SY_ERR_BAD_CHUNKS, "rows [%lld, %lld) outside [0, %lld)", (long long)row_begin,
                    (long long)row_end, (long long)p->ny);
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    if (!u_cur || !u_next || (!start && !u_prev)) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    const size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(p->pitch) * dtype_size(p->dtype);
    if (ranges_overlap(u_next, bytes, u_cur, bytes)) return fail(SY_ERR_ALIAS, "u_next overlaps u_cur");
    if (!start && u_next != u_prev && ranges_overlap(u_next, bytes, u_prev, bytes))
        return fail(SY_ERR_ALIAS, "u_next partially overlaps u_prev");
    SY_TRY(use_device(q));
    EventRecord* rec = nullptr;
    SY_TRY(begin_event(q, ev, &rec));
    WaveLaunch w;
    w.ny = p->ny;
    w.nx = p->nx;
    w.pitch = p->pitch;
    w.radius = p->radius;
    w.dtype = p->dtype;
    w.variant = p->variant;
    w.c2 = start ? 0.5f * p->c2 : p->c2;
    w.start = start != 0;
    w.u_prev = start ? u_cur : u_prev;
    w.u_cur = u_cur;
    w.u_next = u_next;
    w.row_begin = row_begin;
    w.row_end = row_end;
    w.pdl = 0;
    SY_TRY(launch_wave(q, w));
    return end_event(q, rec);
}

}  // extern "C"
