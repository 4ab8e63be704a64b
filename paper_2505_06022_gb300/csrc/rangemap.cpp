// Range mappers on 3D boxes and the transfers a chunk list implies (paper §3:
// the runtime infers data movement from the range mapper of each accessor).
#include "sy_internal.h"

namespace sy {
namespace {

bool empty(const sy_box& b) {
    for (int d = 0; d < 3; ++d)
        if (b.lo[d] >= b.hi[d]) return true;
    return false;
}

int64_t volume(const sy_box& b) {
    if (empty(b)) return 0;
    int64_t v = 1;
    for (int d = 0; d < 3; ++d) v *= b.hi[d] - b.lo[d];
    return v;
}

sy_box intersect(const sy_box& a, const sy_box& b) {
    sy_box r;
    for (int d = 0; d < 3; ++d) {
        r.lo[d] = a.lo[d] > b.lo[d] ? a.lo[d] : b.lo[d];
        r.hi[d] = a.hi[d] < b.hi[d] ? a.hi[d] : b.hi[d];
    }
    return r;
}

sy_status check_mapper(const sy_range_mapper* rm, const int64_t* extent) {
    if (!rm || !extent) return fail(SY_ERR_NULL_POINTER, "range mapper or extent is NULL");
    if (rm->kind < SY_RM_ONE_TO_ONE || rm->kind > SY_RM_FIXED)
        return fail(SY_ERR_INVALID_ARGUMENT, "unknown range mapper kind %d", rm->kind);
    if (rm->kind == SY_RM_SLICE && (rm->dim < 0 || rm->dim > 2))
        return fail(SY_ERR_INVALID_ARGUMENT, "slice dimension %d not in 0..2", rm->dim);
    for (int d = 0; d < 3; ++d) {
        if (extent[d] < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative extent");
        if (rm->kind == SY_RM_NEIGHBOURHOOD && rm->radius[d] < 0)
            return fail(SY_ERR_INVALID_ARGUMENT, "negative neighbourhood radius");
    }
    return SY_OK;
}

sy_box apply(const sy_range_mapper& rm, const sy_box& chunk, const int64_t* extent) {
    sy_box out;
    for (int d = 0; d < 3; ++d) {
        int64_t lo = chunk.lo[d], hi = chunk.hi[d];
        if (rm.kind == SY_RM_NEIGHBOURHOOD) {
            lo -= rm.radius[d];
            hi += rm.radius[d];
        } else if (rm.kind == SY_RM_ALL || (rm.kind == SY_RM_SLICE && rm.dim == d)) {
            lo = 0;
            hi = extent[d];
        } else if (rm.kind == SY_RM_FIXED) {
            lo = rm.fixed.lo[d];
            hi = rm.fixed.hi[d];
        }
        out.lo[d] = lo < 0 ? 0 : lo;
        out.hi[d] = hi > extent[d] ? extent[d] : hi;
    }
    return out;
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" {

sy_status sy_rm_box(const sy_range_mapper* rm, const sy_box* chunk, const int64_t* extent, sy_box* out) {
    clear_error();
    SY_TRY(check_mapper(rm, extent));
    if (!chunk || !out) return fail(SY_ERR_NULL_POINTER, "chunk or out is NULL");
    *out = apply(*rm, *chunk, extent);
    return SY_OK;
}

sy_status sy_rm_box_transfers(const sy_range_mapper* rm, const sy_box* chunks, int n, const int64_t* extent,
                              sy_box_transfer* out, int max_out, int* n_out) {
    clear_error();
    SY_TRY(check_mapper(rm, extent));
    if (!chunks || !n_out || (max_out > 0 && !out)) return fail(SY_ERR_NULL_POINTER, "null pointer");
    if (n < 1) return fail(SY_ERR_BAD_CHUNKS, "no chunks");
    // The chunks must tile the buffer: each non-empty and inside it, pairwise
    // disjoint, and their volumes adding up to the buffer's.
    sy_box whole;
    for (int d = 0; d < 3; ++d) {
        whole.lo[d] = 0;
        whole.hi[d] = extent[d];
    }
    int64_t total = 0;
    for (int c = 0; c < n; ++c) {
        const sy_box& b = chunks[c];
        if (empty(b) || volume(intersect(b, whole)) != volume(b))
            return fail(SY_ERR_BAD_CHUNKS, "chunk %d is empty or outside the buffer", c);
        for (int e = 0; e < c; ++e)
            if (!empty(intersect(b, chunks[e]))) return fail(SY_ERR_BAD_CHUNKS, "chunks %d and %d overlap", e, c);
        total += volume(b);
    }
    if (total != volume(whole)) return fail(SY_ERR_BAD_CHUNKS, "chunks do not cover the buffer");
    int count = 0;
    for (int dst = 0; dst < n; ++dst) {
        const sy_box need = apply(*rm, chunks[dst], extent);
        for (int src = 0; src < n; ++src) {
            if (src == dst) continue;
            const sy_box box = intersect(need, chunks[src]);
            if (empty(box)) continue;
            if (count < max_out) {
                out[count].src = src;
                out[count].dst = dst;
                out[count].box = box;
            }
            ++count;
        }
    }
    *n_out = count;
    if (count > max_out)
        return fail(SY_ERR_INVALID_ARGUMENT, "%d transfers, room for %d", count, max_out);
    return SY_OK;
}

}  // extern "C"
