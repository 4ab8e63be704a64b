// sy_wave_run: a whole leapfrog simulation (Taylor start + n chunked steps)
// captured once into a CUDA graph and replayed.  The chunked launches are the
// same ones sy_stencil_start / sy_stencil_step issue; capturing them removes the
// host's per-launch cost and the gaps between stream launches, and the
// per-chunk timestamps keep working inside the graph (their slots are zeroed
// by the graph's first node on every replay).
#include <cstring>

#include "sy_internal.h"

namespace sy {
namespace {

bool same_params(const sy_stencil_params& a, const sy_stencil_params& b) {
    return a.ny == b.ny && a.nx == b.nx && a.pitch == b.pitch && a.radius == b.radius && a.dtype == b.dtype &&
           a.c2 == b.c2 && a.variant == b.variant;
}

bool cache_hit(const RunGraph& g, const sy_stencil_params* p, const void* u0, void* ua, void* ub, int64_t steps,
               const sy_chunk* chunks, int n_chunks, int halo, bool events) {
    if (!g.valid || !same_params(g.p, *p) || g.u0 != u0 || g.ua != ua || g.ub != ub || g.steps != steps ||
        g.halo != halo || g.events != events || static_cast<int>(g.chunks.size()) != n_chunks)
        return false;
    for (int c = 0; c < n_chunks; ++c)
        if (g.chunks[c].begin != chunks[c].begin || g.chunks[c].end != chunks[c].end) return false;
    return true;
}

// Issue the launches of a run on q->launch.  Fills prev/cur with the buffers
// holding u^{steps-1} and u^{steps}.
sy_status issue_run(Queue* q, const sy_stencil_params* p, const void* u0, void* ua, void* ub, int64_t steps,
                    const sy_chunk* chunks, int n_chunks, int halo, bool events, const void** prev,
                    const void** cur) {
    std::vector<sy_event> ev(events ? n_chunks : 0);
    sy_event* evp = events ? ev.data() : nullptr;
    // start: u_a = u^{-1}
    SY_TRY(stencil_common(q, p, nullptr, u0, ua, chunks, n_chunks, halo, evp, true));
    const void* pv = ua;  // u^{-1}
    const void* cv = u0;  // u^0
    if (steps >= 1) {     // u^1 over u^{-1} in u_a (in place)
        SY_TRY(stencil_common(q, p, ua, u0, ua, chunks, n_chunks, halo, evp, false));
        pv = u0;
        cv = ua;
    }
    if (steps >= 2) {  // u^2 into u_b, so that u0 is never written
        SY_TRY(stencil_common(q, p, u0, ua, ub, chunks, n_chunks, halo, evp, false));
        pv = ua;
        cv = ub;
    }
    for (int64_t s = 2; s < steps; ++s) {  // then in place, alternating u_a / u_b
        void* nv = const_cast<void*>(pv);
        SY_TRY(stencil_common(q, p, pv, cv, nv, chunks, n_chunks, halo, evp, false));
        pv = cv;
        cv = nv;
    }
    *prev = pv;
    *cur = cv;
    return SY_OK;
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" sy_status sy_wave_run(sy_queue_t qh, const sy_stencil_params* p, const void* u0, void* u_a, void* u_b,
                                 int64_t steps, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                 sy_event* events, const void** prev_out, const void** cur_out) {
    Queue* q;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (steps < 0) return fail(SY_ERR_INVALID_ARGUMENT, "steps = %lld < 0", (long long)steps);
    if (!u0 || !u_a || !u_b) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    const size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(p->pitch) * dtype_size(p->dtype);
    if (ranges_overlap(u0, bytes, u_a, bytes) || ranges_overlap(u0, bytes, u_b, bytes) ||
        ranges_overlap(u_a, bytes, u_b, bytes))
        return fail(SY_ERR_ALIAS, "u0, u_a and u_b must not overlap");
    if (p->ny == 0 || p->nx == 0) return fail(SY_ERR_INVALID_ARGUMENT, "empty grid");
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    const bool want = events != nullptr;
    const uint64_t timed = static_cast<uint64_t>(steps + 1) * static_cast<uint64_t>(n_chunks);
    if (want && timed > kGraphStampSlots)
        return fail(SY_ERR_INVALID_ARGUMENT, "%llu timed launches exceed %u per run (pass events = NULL)",
                    (unsigned long long)timed, kGraphStampSlots);
    SY_TRY(use_device(q));

    RunGraph& g = q->run;
    if (!cache_hit(g, p, u0, u_a, u_b, steps, chunks, n_chunks, halo_radius, want)) {
        if (g.exec) {
            SY_CUDA(cudaStreamSynchronize(q->stream));
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        g.valid = false;
        // The capture stream must not start before earlier work on the queue: the
        // graph is launched on q->stream, so capture-time ordering is not needed,
        // but the capture itself issues nothing until launch.
        q->capturing = true;
        q->next_graph_slot = 0;
        q->capture_expected.clear();
        q->launch = q->aux;
        const uint64_t launches0 = q->launches;
        cudaError_t e = cudaStreamBeginCapture(q->aux, cudaStreamCaptureModeThreadLocal);
        sy_status st = SY_OK;
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
        if (st == SY_OK && want) {
            e = cudaMemsetAsync(q->d_stamps + 4ull * kStreamStampSlots, 0,
                                4ull * timed * sizeof(unsigned long long), q->aux);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(stamps)");
        }
        const void *pv = nullptr, *cv = nullptr;
        if (st == SY_OK) st = issue_run(q, p, u0, u_a, u_b, steps, chunks, n_chunks, halo_radius, want, &pv, &cv);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(q->aux, &graph);
        if (st == SY_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
        q->launch = q->stream;
        q->capturing = false;
        const uint64_t per_replay = q->launches - launches0;
        q->launches = launches0;
        if (st == SY_OK) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != SY_OK) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            return st;
        }
        g.valid = true;
        g.p = *p;
        g.u0 = u0;
        g.ua = u_a;
        g.ub = u_b;
        g.steps = steps;
        g.halo = halo_radius;
        g.events = want;
        g.chunks.assign(chunks, chunks + n_chunks);
        g.expected = q->capture_expected;
        g.launches = per_replay;
        g.prev_out = pv;
        g.cur_out = cv;
    }
    SY_CUDA(cudaGraphLaunch(g.exec, q->stream));
    q->launches += g.launches;
    if (want) {
        std::lock_guard<std::mutex> lock(q->mu);
        for (size_t i = 0; i < g.expected.size(); ++i) {
            const uint32_t slot = kStreamStampSlots + static_cast<uint32_t>(i);
            const uint64_t id = q->next_event++;
            EventRecord& r = q->ring[id % kEventRing];
            r.id = id;
            r.slot = slot;
            r.expected = g.expected[i];
            r.window = q->open_window;
            q->slot_owner[slot] = id;
            events[i] = id;
        }
    }
    if (prev_out) *prev_out = g.prev_out;
    if (cur_out) *cur_out = g.cur_out;
    return SY_OK;
}
