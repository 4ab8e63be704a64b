// sy_wave_run / sy_wave3d_run: a whole leapfrog simulation (Taylor start + n
// chunked steps) captured once into a CUDA graph and replayed.  The chunked
// launches are the same ones sy_stencil_start / sy_stencil_step (and their 3D
// forms) issue; capturing them removes the host's per-launch cost and the gaps
// between stream launches, and the per-chunk timestamps keep working inside the
// graph (their slots are zeroed by the graph's first node on every replay).
//
// The chunks of one step are independent (each writes only its own rows and reads
// the previous two levels), so their launch order is free; the run alternates it
// (start and even steps first to last, odd steps last to first), and a reversed 2D
// step also sweeps each chunk's tiles bottom to top.  A step then starts on the rows
// the previous step touched last, while they are still in L2 (8192^2: FP32 +4 %,
// BF16 +8 %; 3D chunks of planes gain nothing, so only their order alternates).
// Results are unchanged; event ids are returned in chunk order.
//
// sy_wave_run_host is the same run on host buffers: the runtime, not the caller,
// moves the data (the buffer/accessor model: a kernel's accessors name the data,
// the runtime makes it present on the device).  Alternate calls use two device work
// sets, and the copies run on a stream per direction, so a call's host-to-device copy
// overlaps the previous call's simulation and its device-to-host copy the next one's.
#include <algorithm>
#include <cstring>

#include "sy_internal.h"

namespace sy {

sy_status graph_run(Queue* q, RunGraph& g, const std::vector<unsigned char>& key, uint64_t timed, bool want,
                    sy_status (*issue)(Queue*, const void*, const void**, const void**), const void* ctx,
                    sy_event* events, const void** prev_out, const void** cur_out) {
    if (want && timed > kGraphStampSlots)
        return fail(SY_ERR_INVALID_ARGUMENT, "%llu timed launches exceed %u per run (pass events = NULL)",
                    (unsigned long long)timed, kGraphStampSlots);
    SY_TRY(use_device(q));
    if (!g.valid || g.key != key) {
        if (g.exec) {
            SY_CUDA(cudaStreamSynchronize(q->stream));
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        g.valid = false;
        // Captured on the queue's private stream; the graph is launched on q->stream,
        // which orders it after earlier work on the queue.
        q->capturing = true;
        q->next_graph_slot = 0;
        q->capture_expected.clear();
        q->launch = q->aux;
        const uint64_t launches0 = q->launches;
        cudaError_t e = cudaStreamBeginCapture(q->aux, cudaStreamCaptureModeThreadLocal);
        sy_status st = SY_OK;
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
        if (st == SY_OK && want) {
            e = cudaMemsetAsync(q->d_stamps + 4ull * kStreamStampSlots, 0, 4ull * timed * sizeof(unsigned long long),
                                q->aux);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(stamps)");
        }
        const void *pv = nullptr, *cv = nullptr;
        if (st == SY_OK) st = issue(q, ctx, &pv, &cv);
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
        g.key = key;
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

namespace {

template <class T>
void append(std::vector<unsigned char>& key, const T& v) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
    key.insert(key.end(), b, b + sizeof(T));
}

// The arguments of one run, shared by the 2D and 3D forms.
template <class P>
struct RunArgs {
    const P* p;
    const void* u0;
    void* ua;
    void* ub;
    int64_t steps;
    const sy_chunk* chunks;
    int n_chunks;
    int halo;
    bool events;
};

template <class P>
std::vector<unsigned char> run_key(const RunArgs<P>& a) {
    std::vector<unsigned char> key;
    append(key, *a.p);
    append(key, a.u0);
    append(key, a.ua);
    append(key, a.ub);
    append(key, a.steps);
    append(key, a.halo);
    append(key, a.events);
    for (int c = 0; c < a.n_chunks; ++c) append(key, a.chunks[c]);
    return key;
}

sy_status step2(Queue* q, const sy_stencil_params* p, const void* up, const void* uc, void* un, const sy_chunk* ch,
                int n, int halo, sy_event* ev, bool start, bool reverse) {
    return stencil_common(q, p, up, uc, un, ch, n, halo, ev, start, reverse);
}
sy_status step3(Queue* q, const sy_stencil3d_params* p, const void* up, const void* uc, void* un, const sy_chunk* ch,
                int n, int halo, sy_event* ev, bool start, bool reverse) {
    return stencil3d_common(q, p, up, uc, un, ch, n, halo, ev, start, reverse);
}

// Start into u_a, step 1 in place over it, step 2 into u_b (u0 is never written),
// then in place, alternating u_a / u_b; step s launches its chunks in reverse
// order when s is odd (the start counts as step 0).
template <class P, sy_status (*STEP)(Queue*, const P*, const void*, const void*, void*, const sy_chunk*, int, int,
                                     sy_event*, bool, bool)>
sy_status issue_run(Queue* q, const void* ctx, const void** prev, const void** cur) {
    const RunArgs<P>& a = *static_cast<const RunArgs<P>*>(ctx);
    std::vector<sy_event> ev(a.events ? a.n_chunks : 0);
    sy_event* evp = a.events ? ev.data() : nullptr;
    SY_TRY(STEP(q, a.p, nullptr, a.u0, a.ua, a.chunks, a.n_chunks, a.halo, evp, true, false));
    const void* pv = a.ua;  // u^{-1}
    const void* cv = a.u0;  // u^0
    if (a.steps >= 1) {
        SY_TRY(STEP(q, a.p, a.ua, a.u0, a.ua, a.chunks, a.n_chunks, a.halo, evp, false, true));
        pv = a.u0;
        cv = a.ua;
    }
    if (a.steps >= 2) {
        SY_TRY(STEP(q, a.p, a.u0, a.ua, a.ub, a.chunks, a.n_chunks, a.halo, evp, false, false));
        pv = a.ua;
        cv = a.ub;
    }
    for (int64_t s = 2; s < a.steps; ++s) {  // this is step s + 1
        void* nv = const_cast<void*>(pv);
        SY_TRY(STEP(q, a.p, pv, cv, nv, a.chunks, a.n_chunks, a.halo, evp, false, (s + 1) % 2 == 1));
        pv = cv;
        cv = nv;
    }
    *prev = pv;
    *cur = cv;
    return SY_OK;
}

// graph_run returns the event ids in launch order; put each odd step's back in chunk order.
void chunk_order(sy_event* events, int64_t steps, int n_chunks) {
    if (!events) return;
    for (int64_t s = 1; s <= steps; s += 2) std::reverse(events + s * n_chunks, events + (s + 1) * n_chunks);
}

sy_status run_checks(int64_t steps, const void* u0, const void* ua, const void* ub, size_t bytes, bool empty) {
    if (steps < 0) return fail(SY_ERR_INVALID_ARGUMENT, "steps = %lld < 0", (long long)steps);
    if (!u0 || !ua || !ub) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    if (ranges_overlap(u0, bytes, ua, bytes) || ranges_overlap(u0, bytes, ub, bytes) ||
        ranges_overlap(ua, bytes, ub, bytes))
        return fail(SY_ERR_ALIAS, "u0, u_a and u_b must not overlap");
    if (empty) return fail(SY_ERR_INVALID_ARGUMENT, "empty grid");
    return SY_OK;
}

}  // namespace

// ---- sy_wave_run_host ---------------------------------------------------------------

sy_status host_run_sync(Queue* q) {
    HostRun& h = q->host;
    if (h.h2d) SY_CUDA(cudaStreamSynchronize(h.h2d));
    if (h.d2h) SY_CUDA(cudaStreamSynchronize(h.d2h));
    return SY_OK;
}

void host_run_release(Queue* q) {
    HostRun& h = q->host;
    if (h.h2d) cudaStreamSynchronize(h.h2d);
    if (h.d2h) cudaStreamSynchronize(h.d2h);
    for (int s = 0; s < kHostSets; ++s) {
        if (h.graph[s].exec) cudaGraphExecDestroy(h.graph[s].exec);
        h.graph[s] = RunGraph();
        for (cudaEvent_t* e : {&h.in_done[s], &h.sim_done[s], &h.out_done[s]})
            if (*e) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
    }
    if (h.ws) cudaFree(h.ws);
    h.ws = nullptr;
    h.ws_bytes = h.field = 0;
    if (h.h2d) cudaStreamDestroy(h.h2d);
    if (h.d2h) cudaStreamDestroy(h.d2h);
    h.h2d = h.d2h = nullptr;
}

namespace {

// Copy streams and events (first call), and work sets of at least `field` bytes per field.
sy_status host_run_prepare(Queue* q, size_t field) {
    HostRun& h = q->host;
    if (!h.h2d) {
        // all or nothing: a partial failure leaves no half-made stream or event behind
        cudaStream_t s2[2] = {nullptr, nullptr};
        cudaEvent_t ev[3 * kHostSets] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&s2[0], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s2[1], cudaStreamNonBlocking);
        for (int i = 0; i < 3 * kHostSets && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            for (cudaStream_t x : s2)
                if (x) cudaStreamDestroy(x);
            return cuda_fail(e, "sy_wave_run_host: copy streams and events");
        }
        h.h2d = s2[0];
        h.d2h = s2[1];
        for (int s = 0; s < kHostSets; ++s) {
            h.in_done[s] = ev[3 * s];
            h.sim_done[s] = ev[3 * s + 1];
            h.out_done[s] = ev[3 * s + 2];
        }
    }
    if (h.field < field) {
        // the old sets may still be read or written: wait for every stream that uses them
        SY_CUDA(cudaStreamSynchronize(q->stream));
        SY_TRY(host_run_sync(q));
        for (int s = 0; s < kHostSets; ++s) {
            if (h.graph[s].exec) cudaGraphExecDestroy(h.graph[s].exec);
            h.graph[s] = RunGraph();
        }
        if (h.ws) SY_CUDA(cudaFree(h.ws));
        h.ws = nullptr;
        h.ws_bytes = h.field = 0;
        void* ws = nullptr;
        cudaError_t e = cudaMalloc(&ws, 3 * kHostSets * field);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(host-run work sets)");
        h.ws = ws;
        h.ws_bytes = 3 * kHostSets * field;
        h.field = field;
    }
    return SY_OK;
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" sy_status sy_wave_run_host(sy_queue_t qh, const sy_stencil_params* p, const void* host_u0, void* host_out,
                                      void* host_prev_out, int64_t steps, const sy_chunk* chunks, int n_chunks,
                                      int halo_radius, sy_event* events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (steps < 0) return fail(SY_ERR_INVALID_ARGUMENT, "steps = %lld < 0", (long long)steps);
    if (!host_u0 || !host_out) return fail(SY_ERR_NULL_POINTER, "host field pointer is NULL");
    if (p->ny == 0 || p->nx == 0) return fail(SY_ERR_INVALID_ARGUMENT, "empty grid");
    const size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(p->pitch) * dtype_size(p->dtype);
    if (host_prev_out && ranges_overlap(host_out, bytes, host_prev_out, bytes))
        return fail(SY_ERR_ALIAS, "host_out and host_prev_out must not overlap");
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    const uint64_t timed = static_cast<uint64_t>(steps + 1) * static_cast<uint64_t>(n_chunks);
    if (events && timed > kGraphStampSlots)
        return fail(SY_ERR_INVALID_ARGUMENT, "%llu timed launches exceed %u per run (pass events = NULL)",
                    (unsigned long long)timed, kGraphStampSlots);
    SY_TRY(use_device(q));
    const size_t field = (bytes + 255) / 256 * 256;
    SY_TRY(host_run_prepare(q, field));
    HostRun& h = q->host;
    const int s = static_cast<int>(h.calls % kHostSets);
    char* set = static_cast<char*>(h.ws) + 3 * static_cast<size_t>(s) * field;
    void* u0 = set;
    void* ua = set + field;
    void* ub = set + 2 * field;

    // host -> device: this set's u0 is free once the call kHostSets back has finished
    // simulating and copying out (with steps = 0 its result is u0 itself; the copy-outs
    // run in call order on one stream, so every older call's copy-out is done too); if
    // this input is one of the more recent calls' outputs, wait for that copy as well.
    SY_CUDA(cudaStreamWaitEvent(h.h2d, h.out_done[s], 0));
    for (int t = 0; t < kHostSets; ++t) {
        if (t == s) continue;
        bool reads = false;
        for (const void* o : h.last_out[t])
            reads = reads || (o && ranges_overlap(host_u0, bytes, o, h.last_out_bytes[t]));
        if (reads) SY_CUDA(cudaStreamWaitEvent(h.h2d, h.out_done[t], 0));
    }
    SY_CUDA(cudaMemcpyAsync(u0, host_u0, bytes, cudaMemcpyHostToDevice, h.h2d));
    SY_CUDA(cudaEventRecord(h.in_done[s], h.h2d));

    // the simulation, on the queue's stream, once the input is in place
    SY_CUDA(cudaStreamWaitEvent(q->stream, h.in_done[s], 0));
    RunArgs<sy_stencil_params> a{p, u0, ua, ub, steps, chunks, n_chunks, halo_radius, events != nullptr};
    const void *pv = nullptr, *cv = nullptr;
    SY_TRY(graph_run(q, h.graph[s], run_key(a), timed, events != nullptr, issue_run<sy_stencil_params, step2>, &a,
                     events, &pv, &cv));
    chunk_order(events, steps, n_chunks);
    SY_CUDA(cudaEventRecord(h.sim_done[s], q->stream));

    // device -> host
    SY_CUDA(cudaStreamWaitEvent(h.d2h, h.sim_done[s], 0));
    SY_CUDA(cudaMemcpyAsync(host_out, cv, bytes, cudaMemcpyDeviceToHost, h.d2h));
    if (host_prev_out) SY_CUDA(cudaMemcpyAsync(host_prev_out, pv, bytes, cudaMemcpyDeviceToHost, h.d2h));
    SY_CUDA(cudaEventRecord(h.out_done[s], h.d2h));
    h.last_out[s][0] = host_out;
    h.last_out[s][1] = host_prev_out;
    h.last_out_bytes[s] = bytes;
    ++h.calls;
    return SY_OK;
}

extern "C" sy_status sy_wave_run(sy_queue_t qh, const sy_stencil_params* p, const void* u0, void* u_a, void* u_b,
                                 int64_t steps, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                 sy_event* events, const void** prev_out, const void** cur_out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    const size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(p->pitch) * dtype_size(p->dtype);
    SY_TRY(run_checks(steps, u0, u_a, u_b, bytes, p->ny == 0 || p->nx == 0));
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    RunArgs<sy_stencil_params> a{p, u0, u_a, u_b, steps, chunks, n_chunks, halo_radius, events != nullptr};
    const uint64_t timed = static_cast<uint64_t>(steps + 1) * static_cast<uint64_t>(n_chunks);
    SY_TRY(graph_run(q, q->run, run_key(a), timed, events != nullptr, issue_run<sy_stencil_params, step2>, &a,
                     events, prev_out, cur_out));
    chunk_order(events, steps, n_chunks);
    return SY_OK;
}

extern "C" sy_status sy_wave3d_run(sy_queue_t qh, const sy_stencil3d_params* p, const void* u0, void* u_a,
                                   void* u_b, int64_t steps, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                   sy_event* events, const void** prev_out, const void** cur_out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil3d_param_checks(p));
    const size_t bytes = static_cast<size_t>(p->nz) * static_cast<size_t>(p->plane) * dtype_size(p->dtype);
    SY_TRY(run_checks(steps, u0, u_a, u_b, bytes, p->nz == 0 || p->ny == 0 || p->nx == 0));
    SY_TRY(validate_chunks(p->nz, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    RunArgs<sy_stencil3d_params> a{p, u0, u_a, u_b, steps, chunks, n_chunks, halo_radius, events != nullptr};
    const uint64_t timed = static_cast<uint64_t>(steps + 1) * static_cast<uint64_t>(n_chunks);
    SY_TRY(graph_run(q, q->run3, run_key(a), timed, events != nullptr, issue_run<sy_stencil3d_params, step3>, &a,
                     events, prev_out, cur_out));
    chunk_order(events, steps, n_chunks);
    return SY_OK;
}
