// Exhaustive autotuner and cost-model features.
//
// The tuner times every candidate configuration of a kernel on the caller's
// buffers -- tile variant x chunk count for the 2D and 3D stencils, launch
// variant x chunk count for SAXPY -- using the launches' own device timestamps (no event
// records between launches), and reports the median of `reps` timed runs after
// one warm-up run.  A run's time is the span from the first chunk's first block
// to the last chunk's last block.  It is both the fallback of the learned cost
// model and the baseline its regret is measured against.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sy_internal.h"

using namespace sy;

namespace {

// Device span (ms) of launches issued back to back on one stream: first block
// start of the first to last block end of the last.  Launches on one stream
// complete in order, so the last one having finished means all have.
sy_status span_ms(Queue* q, const std::vector<sy_event>& evs, double* ms) {
    *ms = 0.0;
    if (evs.empty()) return SY_OK;
    const EventRecord& r0 = q->ring[evs.front() % kEventRing];
    const EventRecord& r1 = q->ring[evs.back() % kEventRing];
    if (r0.id != evs.front() || r1.id != evs.back()) return fail(SY_ERR_INVALID_ARGUMENT, "stale tuning events");
    unsigned long long a[4], b[4];
    SY_CUDA(cudaMemcpyAsync(a, q->d_stamps + 4ull * r0.slot, sizeof a, cudaMemcpyDeviceToHost, q->aux));
    SY_CUDA(cudaMemcpyAsync(b, q->d_stamps + 4ull * r1.slot, sizeof b, cudaMemcpyDeviceToHost, q->aux));
    SY_CUDA(cudaStreamSynchronize(q->aux));
    if (b[2] != r1.expected) return fail(SY_ERR_NOT_READY, "tuning run has not completed");
    const unsigned long long start = ~a[0], end = b[1];
    *ms = end > start ? static_cast<double>(end - start) * 1e-6 : 0.0;
    return SY_OK;
}

double median(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

sy_status validate_counts(const int* counts, int n_counts, int64_t rows) {
    if (n_counts < 1 || !counts) return fail(SY_ERR_INVALID_ARGUMENT, "no chunk counts");
    for (int i = 0; i < n_counts; ++i)
        if (counts[i] < 1 || counts[i] > rows)
            return fail(SY_ERR_INVALID_ARGUMENT, "chunk count %d not in 1..%lld", counts[i], (long long)rows);
    return SY_OK;
}

}  // namespace

extern "C" {

sy_status sy_saxpy_variant_count(int* count) {
    if (!count) return fail(SY_ERR_NULL_POINTER, "count is NULL");
    *count = saxpy_variant_count();
    return SY_OK;
}

sy_status sy_saxpy_variant_info(int variant, int* threads, int* waves) {
    if (!saxpy_variant_info(variant, threads, waves))
        return fail(SY_ERR_INVALID_ARGUMENT, "SAXPY variant %d not in 0..%d", variant, saxpy_variant_count());
    return SY_OK;
}

sy_status sy_saxpy_config(sy_queue_t qh, int64_t n, float alpha, const float* x, const float* y, float* z,
                          int variant, const sy_chunk* chunks, int n_chunks, sy_event* events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (n < 0) return fail(SY_ERR_INVALID_ARGUMENT, "n = %lld < 0", (long long)n);
    if (!saxpy_variant_info(variant, nullptr, nullptr))
        return fail(SY_ERR_INVALID_ARGUMENT, "SAXPY variant %d not in 0..%d", variant, saxpy_variant_count());
    if (n == 0 && n_chunks == 0) return SY_OK;
    if (!x || !y || !z) return fail(SY_ERR_NULL_POINTER, "x, y and z must be non-NULL");
    const size_t bytes = static_cast<size_t>(n) * sizeof(float);
    if ((z != x && ranges_overlap(z, bytes, x, bytes)) || (z != y && ranges_overlap(z, bytes, y, bytes)))
        return fail(SY_ERR_ALIAS, "z partially overlaps x or y");
    SY_TRY(validate_chunks(n, chunks, n_chunks));
    SY_TRY(use_device(q));
    for (int c = 0; c < n_chunks; ++c) {
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, events ? &events[c] : nullptr, &rec));
        const int64_t a = chunks[c].begin, len = chunks[c].end - a;
        SY_TRY(launch_saxpy_variant(q, len, alpha, x + a, y + a, z + a, variant));
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}

sy_status sy_tune_stencil(sy_queue_t qh, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                          void* u_next, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                          int max_out, int* n_out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (!out || !n_out) return fail(SY_ERR_NULL_POINTER, "out or n_out is NULL");
    if (reps < 1) return fail(SY_ERR_INVALID_ARGUMENT, "reps < 1");
    if (p->ny < 1 || p->nx < 1) return fail(SY_ERR_INVALID_ARGUMENT, "empty grid");
    SY_TRY(validate_counts(chunk_counts, n_counts, p->ny));
    const int nv = wave_variant_count(p->radius, p->dtype);
    if (max_out < nv * n_counts) return fail(SY_ERR_INVALID_ARGUMENT, "out holds %d, need %d", max_out, nv * n_counts);
    *n_out = 0;
    std::vector<sy_chunk> chunks;
    for (int ci = 0; ci < n_counts; ++ci) {
        const int k = chunk_counts[ci];
        chunks.resize(k);
        SY_TRY(sy_split_rows(p->ny, k, chunks.data()));
        for (int v = 1; v <= nv; ++v) {
            sy_stencil_params pv = *p;
            pv.variant = v;
            std::vector<double> runs;
            std::vector<sy_event> evs(k);
            for (int r = 0; r <= reps; ++r) {  // run 0 warms up
                SY_TRY(stencil_common(q, &pv, u_prev, u_cur, u_next, chunks.data(), k, p->radius, evs.data(), false));
                SY_CUDA(cudaStreamSynchronize(q->stream));
                double ms = 0.0;
                SY_TRY(span_ms(q, evs, &ms));
                if (r > 0) runs.push_back(ms);
            }
            sy_tune_record& rec = out[(*n_out)++];
            rec.variant = v;
            wave_variant_info(p->radius, p->dtype, v, &rec.tile_rows, &rec.tile_cols, &rec.threads);
            rec.chunks = k;
            rec.ms = median(runs);
        }
    }
    return SY_OK;
}

sy_status sy_tune_saxpy(sy_queue_t qh, int64_t n, const float* x, const float* y, float* z, const int* chunk_counts,
                        int n_counts, int reps, sy_tune_record* out, int max_out, int* n_out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!out || !n_out) return fail(SY_ERR_NULL_POINTER, "out or n_out is NULL");
    if (reps < 1 || n < 1) return fail(SY_ERR_INVALID_ARGUMENT, "reps < 1 or n < 1");
    SY_TRY(validate_counts(chunk_counts, n_counts, n));
    const int nv = saxpy_variant_count();
    if (max_out < nv * n_counts) return fail(SY_ERR_INVALID_ARGUMENT, "out holds %d, need %d", max_out, nv * n_counts);
    *n_out = 0;
    std::vector<sy_chunk> chunks;
    for (int ci = 0; ci < n_counts; ++ci) {
        const int k = chunk_counts[ci];
        chunks.resize(k);
        SY_TRY(sy_split_rows(n, k, chunks.data()));
        for (int v = 1; v <= nv; ++v) {
            std::vector<double> runs;
            std::vector<sy_event> evs(k);
            for (int r = 0; r <= reps; ++r) {
                SY_TRY(sy_saxpy_config(qh, n, 1.5f, x, y, z, v, chunks.data(), k, evs.data()));
                SY_CUDA(cudaStreamSynchronize(q->stream));
                double ms = 0.0;
                SY_TRY(span_ms(q, evs, &ms));
                if (r > 0) runs.push_back(ms);
            }
            sy_tune_record& rec = out[(*n_out)++];
            rec.variant = v;
            int threads = 0, waves = 0;
            saxpy_variant_info(v, &threads, &waves);
            rec.tile_rows = waves;
            rec.tile_cols = 4;
            rec.threads = threads;
            rec.chunks = k;
            rec.ms = median(runs);
        }
    }
    return SY_OK;
}

sy_status sy_tune_stencil3d(sy_queue_t qh, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                            void* u_next, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                            int max_out, int* n_out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil3d_param_checks(p));
    if (!out || !n_out) return fail(SY_ERR_NULL_POINTER, "out or n_out is NULL");
    if (reps < 1) return fail(SY_ERR_INVALID_ARGUMENT, "reps < 1");
    if (p->nz < 1 || p->ny < 1 || p->nx < 1) return fail(SY_ERR_INVALID_ARGUMENT, "empty grid");
    SY_TRY(validate_counts(chunk_counts, n_counts, p->nz));
    const int nv = kWave3dVariants;
    if (max_out < nv * n_counts) return fail(SY_ERR_INVALID_ARGUMENT, "out holds %d, need %d", max_out, nv * n_counts);
    *n_out = 0;
    std::vector<sy_chunk> chunks;
    for (int ci = 0; ci < n_counts; ++ci) {
        const int k = chunk_counts[ci];
        chunks.resize(k);
        SY_TRY(sy_split_rows(p->nz, k, chunks.data()));
        for (int v = 1; v <= nv; ++v) {
            sy_stencil3d_params pv = *p;
            pv.variant = v;
            std::vector<double> runs;
            std::vector<sy_event> evs(k);
            for (int r = 0; r <= reps; ++r) {  // run 0 warms up
                SY_TRY(stencil3d_common(q, &pv, u_prev, u_cur, u_next, chunks.data(), k, p->radius, evs.data(),
                                        false));
                SY_CUDA(cudaStreamSynchronize(q->stream));
                double ms = 0.0;
                SY_TRY(span_ms(q, evs, &ms));
                if (r > 0) runs.push_back(ms);
            }
            sy_tune_record& rec = out[(*n_out)++];
            rec.variant = v;
            wave3d_variant_info(p->radius, p->dtype, v, &rec.tile_rows, &rec.threads);
            rec.tile_cols = 32 * static_cast<int32_t>(16 / dtype_size(p->dtype));
            rec.chunks = k;
            rec.ms = median(runs);
        }
    }
    return SY_OK;
}

sy_status sy_tune_exhaustive(sy_queue_t q, int kind, const void* params, int64_t n, const void* in0, const void* in1,
                             void* out_buf, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                             int max_out, int* n_out, int* best) {
    if (!best || !n_out) return fail(SY_ERR_NULL_POINTER, "best or n_out is NULL");
    sy_status st;
    switch (kind) {
        case SY_TUNE_SAXPY:
            st = sy_tune_saxpy(q, n, static_cast<const float*>(in0), static_cast<const float*>(in1),
                               static_cast<float*>(out_buf), chunk_counts, n_counts, reps, out, max_out, n_out);
            break;
        case SY_TUNE_STENCIL:
            if (!params) return fail(SY_ERR_NULL_POINTER, "params is NULL");
            st = sy_tune_stencil(q, static_cast<const sy_stencil_params*>(params), in0, in1, out_buf, chunk_counts,
                                 n_counts, reps, out, max_out, n_out);
            break;
        case SY_TUNE_STENCIL3D:
            if (!params) return fail(SY_ERR_NULL_POINTER, "params is NULL");
            st = sy_tune_stencil3d(q, static_cast<const sy_stencil3d_params*>(params), in0, in1, out_buf,
                                   chunk_counts, n_counts, reps, out, max_out, n_out);
            break;
        default: return fail(SY_ERR_INVALID_ARGUMENT, "unknown tuning kind %d", kind);
    }
    if (st != SY_OK) return st;
    int b = 0;
    for (int i = 1; i < *n_out; ++i)
        if (out[i].ms < out[b].ms) b = i;
    *best = b;
    return SY_OK;
}

sy_status sy_cost_features(const sy_cost_query* cq, float* out) {
    if (!cq || !out) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    if (cq->kind != 0 && cq->kind != 1) return fail(SY_ERR_INVALID_ARGUMENT, "kind %d", cq->kind);
    if (cq->ny < 1 || cq->nx < 1 || cq->tile_rows < 1 || cq->tile_cols < 1 || cq->threads < 1 || cq->chunks < 1)
        return fail(SY_ERR_INVALID_ARGUMENT, "non-positive size in cost query");
    const size_t es = cq->kind == 0 ? 4 : dtype_size(cq->dtype);
    if (!es) return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", cq->dtype);
    const double r = cq->kind == 0 ? 0.0 : static_cast<double>(cq->radius);
    const double points = static_cast<double>(cq->ny) * static_cast<double>(cq->nx);
    const double bpp = cq->kind == 0 ? 12.0 : 3.0 * static_cast<double>(es);  // algorithmic bytes per point
    const double fpp = cq->kind == 0 ? 2.0 : 4.0 * r + 4.0;                   // flops per point
    const double tiles = cq->kind == 0
                             ? points / (4.0 * cq->threads)
                             : std::ceil(static_cast<double>(cq->nx) / cq->tile_cols) *
                                   std::ceil(static_cast<double>(cq->ny) / cq->tile_rows);
    out[0] = static_cast<float>(cq->kind);
    out[1] = static_cast<float>(std::log2(bpp));
    out[2] = static_cast<float>(fpp);
    out[3] = static_cast<float>(r);
    out[4] = static_cast<float>(std::log2(static_cast<double>(cq->ny)));
    out[5] = static_cast<float>(std::log2(static_cast<double>(cq->nx)));
    out[6] = static_cast<float>(std::log2(points));
    out[7] = static_cast<float>(std::log2(static_cast<double>(cq->tile_rows)));
    out[8] = static_cast<float>(std::log2(static_cast<double>(cq->threads)));
    out[9] = static_cast<float>(std::log2(static_cast<double>(cq->chunks)));
    out[10] = static_cast<float>(std::log2(points * bpp));
    out[11] = static_cast<float>(cq->kind == 0 ? 1.0 : (cq->tile_rows + 2.0 * r) / cq->tile_rows);
    out[12] = static_cast<float>(std::log2(tiles > 1.0 ? tiles : 1.0));
    return SY_OK;
}

}  // extern "C"
