// Host runtime of libsy: status/errors, the queue (one device + one in-order
// stream, paper §2 Listing 1), per-launch events, NVML energy metering (paper §4
// Listing 3), range mappers and chunk validation (paper §3 Listing 2), and the
// argument checking of every compute entry point before its kernels launch.
#include <dlfcn.h>

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "sy_internal.h"

namespace sy {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;

sy_status fail(sy_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

sy_status cuda_fail(cudaError_t e, const char* what) {
    return fail(SY_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { t_last_error.clear(); }

bool fault_enabled(const char* name) {
    const char* env = getenv("SY_FAULT");
    if (!env || !*env) return false;
    std::string all(env);
    size_t pos = 0;
    while (pos <= all.size()) {
        size_t comma = all.find(',', pos);
        std::string tok = all.substr(pos, comma == std::string::npos ? std::string::npos : comma - pos);
        if (tok == name) return true;
        if (comma == std::string::npos) break;
        pos = comma + 1;
    }
    return false;
}

// ---------------------------------------------------------------------------
// NVML, loaded at run time (no link-time dependency)
// ---------------------------------------------------------------------------
namespace nvml {
typedef int ret_t;
typedef void* device_t;
static std::once_flag g_once;
static bool g_ok = false;
static ret_t (*p_init)(void) = nullptr;
static ret_t (*p_by_pci)(const char*, device_t*) = nullptr;
static ret_t (*p_energy)(device_t, unsigned long long*) = nullptr;

static void* g_handle = nullptr;

// SY_NVML_LIB names another library exporting the same NVML entry points (a test
// double); by default the driver's libnvidia-ml.so.1.
static void load() {
    if (fault_enabled("nvml_missing")) return;
    const char* path = getenv("SY_NVML_LIB");
    void* h = dlopen(path && *path ? path : "libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    g_handle = h;
    p_init = reinterpret_cast<ret_t (*)(void)>(dlsym(h, "nvmlInit_v2"));
    p_by_pci = reinterpret_cast<ret_t (*)(const char*, device_t*)>(dlsym(h, "nvmlDeviceGetHandleByPciBusId_v2"));
    p_energy = reinterpret_cast<ret_t (*)(device_t, unsigned long long*)>(
        dlsym(h, "nvmlDeviceGetTotalEnergyConsumption"));
    if (!p_init || !p_by_pci || !p_energy) return;
    if (p_init() != 0) return;
    g_ok = true;
}

bool available() {
    std::call_once(g_once, load);
    return g_ok && !fault_enabled("nvml_missing");
}

void* symbol(const char* name) { return available() ? dlsym(g_handle, name) : nullptr; }

static bool device_for(int cuda_device, device_t* out) {
    if (!available()) return false;
    char bus[64] = {0};
    if (cudaDeviceGetPCIBusId(bus, sizeof bus, cuda_device) != cudaSuccess) return false;
    return p_by_pci(bus, out) == 0;
}

static bool energy_mj(device_t d, uint64_t* mj) {
    if (!available() || !d) return false;
    unsigned long long v = 0;
    if (p_energy(d, &v) != 0) return false;
    *mj = static_cast<uint64_t>(v);
    return true;
}
}  // namespace nvml

static double host_seconds() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// queue
// ---------------------------------------------------------------------------
Queue* as_queue(sy_queue_t q) { return reinterpret_cast<Queue*>(q); }

sy_status check_queue(sy_queue_t q, Queue** out) {
    if (!q) return fail(SY_ERR_NULL_POINTER, "queue is NULL");
    *out = as_queue(q);
    return SY_OK;
}

sy_status use_device(Queue* q) {
    int cur = -1;
    SY_CUDA(cudaGetDevice(&cur));
    if (cur != q->device) SY_CUDA(cudaSetDevice(q->device));
    return SY_OK;
}

sy_status queue_scratch(Queue* q, size_t bytes, void** out) {
    if (q->scratch_bytes < bytes) {
        if (q->scratch) {
            SY_CUDA(cudaStreamSynchronize(q->stream));
            SY_CUDA(cudaFree(q->scratch));
            q->scratch = nullptr;
            q->scratch_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&q->scratch, bytes);
        if (e != cudaSuccess) {
            q->scratch = nullptr;
            return cuda_fail(e, "cudaMalloc(queue scratch)");
        }
        q->scratch_bytes = bytes;
    }
    *out = q->scratch;
    return SY_OK;
}

sy_status begin_event(Queue* q, sy_event* want, EventRecord** rec) {
    *rec = nullptr;
    q->cur_stamp = nullptr;
    q->cur_blocks = 0;
    if (!want) return SY_OK;
    uint32_t slot;
    if (q->capturing) {
        if (q->next_graph_slot >= kGraphStampSlots)
            return fail(SY_ERR_INVALID_ARGUMENT, "more than %u timed launches in one captured run", kGraphStampSlots);
        slot = kStreamStampSlots + q->next_graph_slot++;
        q->capture_expected.push_back(0);
        q->cur_stamp = q->d_stamps + 4ull * slot;
        *want = 0;  // ids are issued per replay
        return SY_OK;
    }
    slot = q->next_stream_slot;
    q->next_stream_slot = (q->next_stream_slot + 1) % kStreamStampSlots;
    std::lock_guard<std::mutex> lock(q->mu);
    if (slot % kStampPage == 0) {  // zero the page this slot opens, ahead of its launches
        SY_CUDA(cudaMemsetAsync(q->d_stamps + 4ull * slot, 0, 4ull * kStampPage * sizeof(unsigned long long),
                                q->launch));
        for (uint32_t i = slot; i < slot + kStampPage; ++i) q->slot_owner[i] = 0;
    }
    uint64_t id = q->next_event++;
    EventRecord& r = q->ring[id % kEventRing];
    r.id = id;
    r.slot = slot;
    r.expected = 0;
    r.window = q->open_window;
    q->slot_owner[slot] = id;
    q->cur_stamp = q->d_stamps + 4ull * slot;
    *want = id;
    *rec = &r;
    return SY_OK;
}

sy_status end_event(Queue* q, EventRecord* rec) {
    if (q->capturing && q->cur_stamp) q->capture_expected.back() = q->cur_blocks;
    if (rec) rec->expected = q->cur_blocks;
    q->cur_stamp = nullptr;
    q->cur_blocks = 0;
    return SY_OK;
}

static sy_status find_event(Queue* q, sy_event ev, EventRecord** out) {
    if (ev == 0 || ev >= q->next_event || q->next_event - ev > kEventRing)
        return fail(SY_ERR_INVALID_ARGUMENT, "event %llu is not a live event of this queue",
                    static_cast<unsigned long long>(ev));
    EventRecord& r = q->ring[ev % kEventRing];
    if (r.id != ev || q->slot_owner[r.slot] != ev)
        return fail(SY_ERR_INVALID_ARGUMENT, "event %llu was recycled", (unsigned long long)ev);
    *out = &r;
    return SY_OK;
}

// Copy stamp slots [lo, hi) to the host (a snapshot: launches may still run).
static sy_status read_stamps(Queue* q, uint32_t lo, uint32_t hi, std::vector<unsigned long long>* out) {
    out->assign(4ull * (hi - lo), 0ull);
    if (hi <= lo) return SY_OK;
    SY_CUDA(cudaMemcpyAsync(out->data(), q->d_stamps + 4ull * lo, out->size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, q->aux));
    SY_CUDA(cudaStreamSynchronize(q->aux));
    return SY_OK;
}

static sy_status stamp_ms(const EventRecord& r, const unsigned long long* slot, double* ms) {
    if (r.expected == 0) {  // nothing launched (e.g. an empty range): zero time
        *ms = 0.0;
        return SY_OK;
    }
    if (slot[2] != r.expected)
        return fail(SY_ERR_NOT_READY, "event %llu: %llu of %llu blocks finished", (unsigned long long)r.id,
                    slot[2], (unsigned long long)r.expected);
    unsigned long long start = ~slot[0], end = slot[1];
    *ms = end > start ? static_cast<double>(end - start) * 1e-6 : 0.0;
    return SY_OK;
}

// ---------------------------------------------------------------------------
// checks
// ---------------------------------------------------------------------------
bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
    if (abytes == 0 || bbytes == 0) return false;
    uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

sy_status validate_chunks(int64_t n, const sy_chunk* chunks, int n_chunks) {
    if (n_chunks < 1) return fail(SY_ERR_BAD_CHUNKS, "chunk list is empty");
    if (!chunks) return fail(SY_ERR_NULL_POINTER, "chunk list is NULL");
    int64_t expect = 0;
    for (int c = 0; c < n_chunks; ++c) {
        if (chunks[c].begin != expect)
            return fail(SY_ERR_BAD_CHUNKS, "chunk %d begins at %lld, expected %lld", c, (long long)chunks[c].begin,
                        (long long)expect);
        if (chunks[c].end <= chunks[c].begin)
            return fail(SY_ERR_BAD_CHUNKS, "chunk %d [%lld, %lld) is empty or reversed", c,
                        (long long)chunks[c].begin, (long long)chunks[c].end);
        expect = chunks[c].end;
    }
    if (expect != n)
        return fail(SY_ERR_BAD_CHUNKS, "chunks end at %lld, range has %lld", (long long)expect, (long long)n);
    return SY_OK;
}

size_t dtype_size(int dtype) {
    switch (dtype) {
        case SY_F32: return 4;
        case SY_BF16:
        case SY_F16: return 2;
        default: return 0;
    }
}

}  // namespace sy

using namespace sy;

// ---- stencil argument checks and chunked launches (shared by step/start/run) ----
sy_status sy::stencil_param_checks(const sy_stencil_params* p) {
    if (!p) return fail(SY_ERR_NULL_POINTER, "params is NULL");
    if (p->ny < 0 || p->nx < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative grid size");
    if (p->pitch < p->nx) return fail(SY_ERR_INVALID_ARGUMENT, "pitch %lld < nx %lld", (long long)p->pitch,
                                      (long long)p->nx);
    if (p->radius < 1 || p->radius > 4) return fail(SY_ERR_INVALID_ARGUMENT, "radius %d not in 1..4", p->radius);
    if (dtype_size(p->dtype) == 0) return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", p->dtype);
    if (p->variant < 0 || p->variant > wave_variant_count(p->radius, p->dtype))
        return fail(SY_ERR_INVALID_ARGUMENT, "variant %d not in 0..%d", p->variant,
                    wave_variant_count(p->radius, p->dtype));
    return SY_OK;
}

sy_status sy::stencil_common(Queue* q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                                void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                sy_event* chunk_events, bool start, bool reverse) {
    SY_TRY(stencil_param_checks(p));
    if (p->ny == 0 || p->nx == 0) {
        if (n_chunks == 0) return SY_OK;
    }
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < stencil radius %d", halo_radius, p->radius);
    if (!u_cur || !u_next || (!start && !u_prev)) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(p->pitch) * dtype_size(p->dtype);
    if (ranges_overlap(u_next, bytes, u_cur, bytes)) return fail(SY_ERR_ALIAS, "u_next overlaps u_cur");
    if (!start && u_next != u_prev && ranges_overlap(u_next, bytes, u_prev, bytes))
        return fail(SY_ERR_ALIAS, "u_next partially overlaps u_prev");
    SY_TRY(use_device(q));
    for (int i = 0; i < n_chunks; ++i) {
        const int c = reverse ? n_chunks - 1 - i : i;
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, chunk_events ? &chunk_events[c] : nullptr, &rec));
        WaveLaunch w;
        w.ny = p->ny;
        w.nx = p->nx;
        w.pitch = p->pitch;
        w.radius = p->radius;
        w.dtype = p->dtype;
        w.variant = p->variant;
        w.c2 = start ? 0.5f * p->c2 : p->c2;
        w.start = start;
        w.u_prev = start ? u_cur : u_prev;
        w.u_cur = u_cur;
        w.u_next = u_next;
        w.row_begin = chunks[c].begin;
        w.row_end = chunks[c].end;
        w.pdl = i == 0 ? 1 : 2;  // the first launch waits for the previous step; the rest overlap it
        w.reverse = reverse;     // a reversed step also sweeps each chunk bottom to top
        SY_TRY(launch_wave(q, w));
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}


// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* sy_status_string(sy_status s) {
    switch (s) {
        case SY_OK: return "SY_OK";
        case SY_ERR_INVALID_ARGUMENT: return "SY_ERR_INVALID_ARGUMENT";
        case SY_ERR_NULL_POINTER: return "SY_ERR_NULL_POINTER";
        case SY_ERR_ALIAS: return "SY_ERR_ALIAS";
        case SY_ERR_BAD_CHUNKS: return "SY_ERR_BAD_CHUNKS";
        case SY_ERR_HALO_TOO_SMALL: return "SY_ERR_HALO_TOO_SMALL";
        case SY_ERR_UNSUPPORTED: return "SY_ERR_UNSUPPORTED";
        case SY_ERR_CUDA: return "SY_ERR_CUDA";
        case SY_ERR_NVML_UNAVAILABLE: return "SY_ERR_NVML_UNAVAILABLE";
        case SY_ERR_TIMEOUT: return "SY_ERR_TIMEOUT";
        case SY_ERR_OUT_OF_MEMORY: return "SY_ERR_OUT_OF_MEMORY";
        case SY_ERR_NOT_READY: return "SY_ERR_NOT_READY";
        case SY_ERR_IO: return "SY_ERR_IO";
        case SY_ERR_NVML: return "SY_ERR_NVML";
    }
    return "SY_ERR_UNKNOWN";
}

const char* sy_last_error(void) { return t_last_error.c_str(); }

int sy_abi_version(void) { return SY_ABI_VERSION; }

// ---- queue ---------------------------------------------------------------------
sy_status sy_queue_create(int device, void* cuda_stream, sy_queue_t* out) {
    if (!out) return fail(SY_ERR_NULL_POINTER, "out is NULL");
    *out = nullptr;
    int count = 0;
    SY_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return fail(SY_ERR_INVALID_ARGUMENT, "device %d out of range (%d devices)", device, count);
    Queue* q = new (std::nothrow) Queue();
    if (!q) return fail(SY_ERR_OUT_OF_MEMORY, "queue allocation failed");
    q->device = device;
    q->ring.resize(kEventRing);
    q->slot_owner.assign(kStampSlots, 0);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&q->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            q->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
            q->owned = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&q->d_stamps, 4ull * kStampSlots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(q->d_stamps, 0, 4ull * kStampSlots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&q->d_flags, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(q->d_flags, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        if (q->d_stamps) cudaFree(q->d_stamps);
        if (q->d_flags) cudaFree(q->d_flags);
        if (q->aux) cudaStreamDestroy(q->aux);
        if (q->owned) cudaStreamDestroy(q->stream);
        delete q;
        return cuda_fail(e, "sy_queue_create");
    }
    q->launch = q->stream;
    nvml::device_t d = nullptr;
    if (nvml::device_for(device, &d)) {
        q->nvml_device = d;
        q->energy_ok = nvml::energy_mj(d, &q->energy_at_create);
    }
    *out = reinterpret_cast<sy_queue_t>(q);
    return SY_OK;
}

sy_status sy_queue_destroy(sy_queue_t qh) {
    if (!qh) return SY_OK;
    Queue* q = as_queue(qh);
    cudaSetDevice(q->device);
    cudaStreamSynchronize(q->stream);
    host_run_release(q);
    if (q->run.exec) cudaGraphExecDestroy(q->run.exec);
    if (q->run3.exec) cudaGraphExecDestroy(q->run3.exec);
    if (q->scratch) cudaFree(q->scratch);
    if (q->d_stamps) cudaFree(q->d_stamps);
    if (q->d_flags) cudaFree(q->d_flags);
    if (q->aux) cudaStreamDestroy(q->aux);
    if (q->owned) cudaStreamDestroy(q->stream);
    delete q;
    return SY_OK;
}

sy_status sy_queue_sync(sy_queue_t qh) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(use_device(q));
    SY_CUDA(cudaStreamSynchronize(q->stream));
    SY_TRY(host_run_sync(q));
    unsigned int flags = 0;
    SY_CUDA(cudaMemcpy(&flags, q->d_flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags) {
        SY_CUDA(cudaMemset(q->d_flags, 0, sizeof flags));
        return fail(SY_ERR_TIMEOUT, "a kernel's bounded wait gave up (flags 0x%x); its outputs are invalid", flags);
    }
    return SY_OK;
}

sy_status sy_queue_stream(sy_queue_t qh, void** stream) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!stream) return fail(SY_ERR_NULL_POINTER, "stream out is NULL");
    *stream = q->stream;
    return SY_OK;
}

sy_status sy_queue_launch_count(sy_queue_t qh, uint64_t* launches) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!launches) return fail(SY_ERR_NULL_POINTER, "launches out is NULL");
    *launches = q->launches;
    return SY_OK;
}

// ---- events and energy ------------------------------------------------------------
sy_status sy_event_elapsed(sy_queue_t qh, sy_event ev, double* ms) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!ms) return fail(SY_ERR_NULL_POINTER, "ms out is NULL");
    EventRecord* r = nullptr;
    SY_TRY(find_event(q, ev, &r));
    SY_TRY(use_device(q));
    std::vector<unsigned long long> st;
    SY_TRY(read_stamps(q, r->slot, r->slot + 1, &st));
    return stamp_ms(*r, st.data(), ms);
}

sy_status sy_events_elapsed(sy_queue_t qh, const sy_event* evs, int n, double* ms) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (n < 0) return fail(SY_ERR_INVALID_ARGUMENT, "n = %d < 0", n);
    if (n == 0) return SY_OK;
    if (!evs || !ms) return fail(SY_ERR_NULL_POINTER, "events or ms is NULL");
    SY_TRY(use_device(q));
    std::vector<EventRecord*> recs(n);
    for (int i = 0; i < n; ++i) SY_TRY(find_event(q, evs[i], &recs[i]));
    std::vector<unsigned long long> st;
    SY_TRY(read_stamps(q, 0, kStampSlots, &st));
    for (int i = 0; i < n; ++i) SY_TRY(stamp_ms(*recs[i], st.data() + 4ull * recs[i]->slot, &ms[i]));
    return SY_OK;
}

sy_status sy_energy_read(sy_queue_t qh, uint64_t* mj) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!mj) return fail(SY_ERR_NULL_POINTER, "millijoules out is NULL");
    if (!q->nvml_device || !nvml::energy_mj(q->nvml_device, mj))
        return fail(SY_ERR_NVML_UNAVAILABLE, "NVML energy counter unavailable for device %d", q->device);
    return SY_OK;
}

sy_status sy_device_energy(sy_queue_t qh, double* joules) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!joules) return fail(SY_ERR_NULL_POINTER, "joules out is NULL");
    uint64_t now = 0;
    if (!q->energy_ok || !nvml::energy_mj(q->nvml_device, &now))
        return fail(SY_ERR_NVML_UNAVAILABLE, "NVML energy counter unavailable for device %d", q->device);
    *joules = static_cast<double>(now - q->energy_at_create) * 1e-3;
    return SY_OK;
}

sy_status sy_meter_begin(sy_queue_t qh) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(use_device(q));
    if (q->open_window >= 0) return fail(SY_ERR_INVALID_ARGUMENT, "a metering window is already open");
    SY_CUDA(cudaStreamSynchronize(q->stream));
    uint64_t e0 = 0;
    bool ok = q->nvml_device && nvml::energy_mj(q->nvml_device, &e0);
    std::lock_guard<std::mutex> lock(q->mu);
    q->windows.push_back(Window{});
    q->windows.back().have_energy = ok;
    q->open_window = static_cast<int64_t>(q->windows.size()) - 1;
    q->window_e0 = e0;
    q->window_t0 = host_seconds();
    return SY_OK;
}

sy_status sy_meter_end(sy_queue_t qh, double* joules, double* seconds) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(use_device(q));
    if (q->open_window < 0) return fail(SY_ERR_INVALID_ARGUMENT, "no metering window is open");
    SY_CUDA(cudaStreamSynchronize(q->stream));
    double t1 = host_seconds();
    uint64_t e1 = 0;
    std::lock_guard<std::mutex> lock(q->mu);
    Window& w = q->windows[q->open_window];
    w.seconds = t1 - q->window_t0;
    w.have_energy = w.have_energy && nvml::energy_mj(q->nvml_device, &e1);
    w.joules = w.have_energy ? static_cast<double>(e1 - q->window_e0) * 1e-3 : 0.0;
    w.closed = true;
    q->open_window = -1;
    if (seconds) *seconds = w.seconds;
    if (joules) *joules = w.have_energy ? w.joules : -1.0;
    if (!w.have_energy)
        return fail(SY_ERR_NVML_UNAVAILABLE, "NVML energy counter unavailable for device %d", q->device);
    return SY_OK;
}

sy_status sy_kernel_energy(sy_queue_t qh, sy_event ev, double* joules) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!joules) return fail(SY_ERR_NULL_POINTER, "joules out is NULL");
    EventRecord* r = nullptr;
    SY_TRY(find_event(q, ev, &r));
    if (r->window < 0 || r->window >= static_cast<int64_t>(q->windows.size()) || !q->windows[r->window].closed)
        return fail(SY_ERR_NOT_READY, "event %llu was not issued inside a closed metering window",
                    (unsigned long long)ev);
    const Window& w = q->windows[r->window];
    if (!w.have_energy) return fail(SY_ERR_NVML_UNAVAILABLE, "window has no energy reading");
    double ms = 0.0;
    SY_TRY(sy_event_elapsed(qh, ev, &ms));
    double watts = w.seconds > 0 ? w.joules / w.seconds : 0.0;
    *joules = watts * ms * 1e-3;
    return SY_OK;
}

sy_status sy_chunk_stats_read(sy_queue_t qh, const sy_stencil_params* p, const sy_chunk* chunks,
                              const sy_event* events, int n, sy_chunk_stats* out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (n < 0) return fail(SY_ERR_INVALID_ARGUMENT, "n = %d < 0", n);
    if (n == 0) return SY_OK;
    if (!chunks || !events || !out) return fail(SY_ERR_NULL_POINTER, "chunks, events or out is NULL");
    std::vector<double> ms(static_cast<size_t>(n));
    SY_TRY(sy_events_elapsed(qh, events, n, ms.data()));
    const double es = static_cast<double>(dtype_size(p->dtype));
    for (int c = 0; c < n; ++c) {
        const double updates = static_cast<double>(chunks[c].end - chunks[c].begin) * static_cast<double>(p->nx);
        out[c].ms = ms[c];
        out[c].updates = updates;
        out[c].bytes = 3.0 * es * updates;  // algorithmic: read u^n and u^{n-1}, write u^{n+1}
        double j = -1.0;
        if (sy_kernel_energy(qh, events[c], &j) != SY_OK) j = -1.0;  // no closed metering window
        out[c].joules = j;
    }
    clear_error();
    return SY_OK;
}

sy_status sy_chunk_energy_replay(sy_queue_t qh, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                                 void* u_next, const sy_chunk* chunks, int n_chunks, int c, int halo_radius,
                                 double min_seconds, int min_reps, double* joules, double* ms, int* reps) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (!joules || !ms || !reps) return fail(SY_ERR_NULL_POINTER, "joules, ms or reps is NULL");
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (c < 0 || c >= n_chunks) return fail(SY_ERR_INVALID_ARGUMENT, "chunk %d not in 0..%d", c, n_chunks - 1);
    if (min_reps < 1 || !(min_seconds >= 0.0) || min_seconds > 600.0)
        return fail(SY_ERR_INVALID_ARGUMENT, "min_reps = %d, min_seconds = %g", min_reps, min_seconds);
    *joules = -1.0;
    *ms = 0.0;
    *reps = 0;
    if (q->open_window >= 0) return fail(SY_ERR_INVALID_ARGUMENT, "a metering window is already open");
    const int64_t a = chunks[c].begin, b = chunks[c].end;
    // argument checks and a warm-up (occupancy lookups, first-touch) outside the window
    for (int i = 0; i < 2; ++i) SY_TRY(sy_stencil_step_rows(qh, p, u_prev, u_cur, u_next, a, b, halo_radius, 0, nullptr));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SY_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    const sy_status meter = sy_meter_begin(qh);
    sy_status st = SY_OK;
    int n = 0;
    const double t0 = host_seconds();
    ce = cudaEventRecord(e0, q->stream);
    if (ce != cudaSuccess) st = cuda_fail(ce, "cudaEventRecord");
    while (st == SY_OK && (n < min_reps || host_seconds() - t0 < min_seconds)) {
        for (int i = 0; i < 32 && st == SY_OK; ++i, ++n)
            st = sy_stencil_step_rows(qh, p, u_prev, u_cur, u_next, a, b, halo_radius, 0, nullptr);
        if (st == SY_OK) {
            ce = cudaStreamSynchronize(q->stream);
            if (ce != cudaSuccess) st = cuda_fail(ce, "cudaStreamSynchronize");
        }
    }
    if (st == SY_OK) {
        ce = cudaEventRecord(e1, q->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float el = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&el, e0, e1);
        if (ce != cudaSuccess) st = cuda_fail(ce, "cudaEventElapsedTime");
        *ms = static_cast<double>(el) / n;
        *reps = n;
    }
    double j = -1.0, secs = 0.0;
    sy_status mend = SY_OK;
    if (meter == SY_OK) mend = sy_meter_end(qh, &j, &secs);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SY_OK) return st;
    if (meter != SY_OK) return meter;
    if (mend != SY_OK) return mend;
    *joules = j / n;
    return SY_OK;
}

// ---- range mappers ---------------------------------------------------------------------
sy_status sy_split_rows(int64_t n, int k, sy_chunk* out) {
    if (!out) return fail(SY_ERR_NULL_POINTER, "out is NULL");
    if (n < 0 || k < 1) return fail(SY_ERR_INVALID_ARGUMENT, "split of %lld rows into %d chunks", (long long)n, k);
    int64_t base = n / k, extra = n % k, row = 0;
    for (int c = 0; c < k; ++c) {
        int64_t len = base + (c < extra ? 1 : 0);
        out[c].begin = row;
        out[c].end = row + len;
        row += len;
    }
    return SY_OK;
}

sy_status sy_rm_one_to_one(sy_chunk chunk, sy_chunk* region) {
    if (!region) return fail(SY_ERR_NULL_POINTER, "region is NULL");
    *region = chunk;
    return SY_OK;
}

sy_status sy_rm_neighbourhood(sy_chunk chunk, int radius, int64_t n, sy_chunk* region) {
    if (!region) return fail(SY_ERR_NULL_POINTER, "region is NULL");
    if (radius < 0) return fail(SY_ERR_INVALID_ARGUMENT, "negative radius %d", radius);
    int64_t lo = chunk.begin - radius, hi = chunk.end + radius;
    region->begin = lo < 0 ? 0 : lo;
    region->end = hi > n ? n : hi;
    return SY_OK;
}

sy_status sy_chunks_validate(int64_t n, const sy_chunk* chunks, int n_chunks) {
    return validate_chunks(n, chunks, n_chunks);
}

// ---- SAXPY -------------------------------------------------------------------------------
static sy_status saxpy_checks(int64_t n, const float* x, const float* y, float* z) {
    if (n < 0) return fail(SY_ERR_INVALID_ARGUMENT, "n = %lld < 0", (long long)n);
    if (n == 0) return SY_OK;
    if (!x || !y || !z) return fail(SY_ERR_NULL_POINTER, "x, y and z must be non-NULL");
    size_t bytes = static_cast<size_t>(n) * sizeof(float);
    if ((z != x && ranges_overlap(z, bytes, x, bytes)) || (z != y && ranges_overlap(z, bytes, y, bytes)))
        return fail(SY_ERR_ALIAS, "z partially overlaps x or y");
    return SY_OK;
}

sy_status sy_saxpy(sy_queue_t qh, int64_t n, float alpha, const float* x, const float* y, float* z, sy_event* ev) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(saxpy_checks(n, x, y, z));
    SY_TRY(use_device(q));
    EventRecord* rec = nullptr;
    SY_TRY(begin_event(q, ev, &rec));
    if (n > 0) SY_TRY(launch_saxpy(q, n, alpha, x, y, z));
    return end_event(q, rec);
}

sy_status sy_saxpy_split(sy_queue_t qh, int64_t n, float alpha, const float* x, const float* y, float* z,
                         const sy_chunk* chunks, int n_chunks, sy_event* events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(saxpy_checks(n, x, y, z));
    if (n == 0 && n_chunks == 0) return SY_OK;
    SY_TRY(validate_chunks(n, chunks, n_chunks));
    SY_TRY(use_device(q));
    for (int c = 0; c < n_chunks; ++c) {
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, events ? &events[c] : nullptr, &rec));
        int64_t a = chunks[c].begin, len = chunks[c].end - a;
        SY_TRY(launch_saxpy(q, len, alpha, x + a, y + a, z + a));  // one_to_one: [a, b) -> [a, b)
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}

// ---- stencil ------------------------------------------------------------------------------
sy_status sy_stencil_step(sy_queue_t qh, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                          void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                          sy_event* chunk_events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return stencil_common(q, p, u_prev, u_cur, u_next, chunks, n_chunks, halo_radius, chunk_events, false);
}

sy_status sy_stencil_start(sy_queue_t qh, const sy_stencil_params* p, const void* u0, void* u_m1,
                           const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* chunk_events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    return stencil_common(q, p, nullptr, u0, u_m1, chunks, n_chunks, halo_radius, chunk_events, true);
}

sy_status sy_stencil_multistep(sy_queue_t qh, const sy_stencil_params* p, int T, const void* u_prev,
                               const void* u_cur, void* out_prev, void* out_cur, const sy_chunk* chunks, int n_chunks,
                               int halo_radius, sy_event* chunk_events) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (T != 2 && T != 4) return fail(SY_ERR_INVALID_ARGUMENT, "T = %d not in {2, 4}", T);
    if (p->ny == 0 || p->nx == 0) {
        if (n_chunks == 0) return SY_OK;
    }
    SY_TRY(validate_chunks(p->ny, chunks, n_chunks));
    if (halo_radius < T * p->radius)
        return fail(SY_ERR_HALO_TOO_SMALL, "halo radius %d < T x radius = %d", halo_radius, T * p->radius);
    if (!u_prev || !u_cur || !out_prev || !out_cur) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    const size_t es = dtype_size(p->dtype);
    const int64_t pb = p->pitch * static_cast<int64_t>(es);
    const uintptr_t all = reinterpret_cast<uintptr_t>(u_prev) | reinterpret_cast<uintptr_t>(u_cur) |
                          reinterpret_cast<uintptr_t>(out_prev) | reinterpret_cast<uintptr_t>(out_cur);
    if ((all % 16) || (pb % 16))
        return fail(SY_ERR_INVALID_ARGUMENT, "temporal blocking needs 16-byte aligned rows (base and pitch)");
    const size_t bytes = static_cast<size_t>(p->ny) * static_cast<size_t>(pb);
    const void* in[2] = {u_prev, u_cur};
    const void* outs[2] = {out_prev, out_cur};
    for (const void* o : outs)
        for (const void* i : in)
            if (ranges_overlap(o, bytes, i, bytes))
                return fail(SY_ERR_ALIAS, "outputs must not overlap the inputs (other chunks read them)");
    if (ranges_overlap(out_prev, bytes, out_cur, bytes)) return fail(SY_ERR_ALIAS, "out_prev overlaps out_cur");
    SY_TRY(use_device(q));
    const int fault = fault_enabled("tb_timeout") ? 1 : 0;
    for (int c = 0; c < n_chunks; ++c) {
        EventRecord* rec = nullptr;
        SY_TRY(begin_event(q, chunk_events ? &chunk_events[c] : nullptr, &rec));
        TBLaunch w;
        w.ny = p->ny;
        w.nx = p->nx;
        w.pitch_bytes = pb;
        w.radius = p->radius;
        w.dtype = p->dtype;
        w.T = T;
        w.c2 = p->c2;
        w.u_prev = u_prev;
        w.u_cur = u_cur;
        w.out_prev = out_prev;
        w.out_cur = out_cur;
        w.row_begin = chunks[c].begin;
        w.row_end = chunks[c].end;
        w.fault = fault;
        w.pdl = c == 0 ? 1 : 2;
        SY_TRY(launch_tb(q, w));
        SY_TRY(end_event(q, rec));
    }
    return SY_OK;
}

sy_status sy_stencil_variant_count(int radius, int dtype, int* count) {
    if (!count) return fail(SY_ERR_NULL_POINTER, "count is NULL");
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0)
        return fail(SY_ERR_INVALID_ARGUMENT, "radius %d / dtype %d unsupported", radius, dtype);
    *count = wave_variant_count(radius, dtype);
    return SY_OK;
}

sy_status sy_stencil_default_variant(int radius, int dtype, int* variant) {
    if (!variant) return fail(SY_ERR_NULL_POINTER, "variant is NULL");
    if (radius < 1 || radius > 4 || dtype_size(dtype) == 0)
        return fail(SY_ERR_INVALID_ARGUMENT, "bad radius %d or dtype %d", radius, dtype);
    *variant = wave_default_variant(radius, dtype);
    return SY_OK;
}

sy_status sy_stencil_variant_info(int radius, int dtype, int variant, int* tile_rows, int* tile_cols,
                                  int* threads) {
    if (!wave_variant_info(radius, dtype, variant, tile_rows, tile_cols, threads))
        return fail(SY_ERR_INVALID_ARGUMENT, "no variant %d for radius %d dtype %d", variant, radius, dtype);
    return SY_OK;
}

sy_status sy_wave_energy(sy_queue_t qh, const sy_stencil_params* p, const void* u_new, const void* u_old,
                         double* energy, double* kinetic, double* potential) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (!energy) return fail(SY_ERR_NULL_POINTER, "energy out is NULL");
    if (p->ny == 0 || p->nx == 0) {
        *energy = 0.0;
        if (kinetic) *kinetic = 0.0;
        if (potential) *potential = 0.0;
        return SY_OK;
    }
    if (!u_new || !u_old) return fail(SY_ERR_NULL_POINTER, "field pointer is NULL");
    SY_TRY(use_device(q));
    void* scratch = nullptr;
    size_t need = sizeof(double) * (2 * kEnergyBlocks + 3);
    SY_TRY(queue_scratch(q, need, &scratch));
    double* partials = static_cast<double*>(scratch);
    double* out3 = partials + 2 * kEnergyBlocks;
    SY_TRY(launch_wave_energy(q, p, u_new, u_old, partials, kEnergyBlocks, out3));
    double host[3];
    SY_CUDA(cudaMemcpyAsync(host, out3, sizeof host, cudaMemcpyDeviceToHost, q->stream));
    SY_CUDA(cudaStreamSynchronize(q->stream));
    *energy = host[0];
    if (kinetic) *kinetic = host[1];
    if (potential) *potential = host[2];
    return SY_OK;
}

}  // extern "C"
