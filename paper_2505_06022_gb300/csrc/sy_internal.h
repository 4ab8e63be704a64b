// Internal declarations shared by libsy's translation units.  Not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "sy.h"

namespace sy {

// ---- errors ------------------------------------------------------------------
sy_status fail(sy_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
sy_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define SY_CUDA(call)                                             \
    do {                                                          \
        cudaError_t sy_e_ = (call);                               \
        if (sy_e_ != cudaSuccess) return ::sy::cuda_fail(sy_e_, #call); \
    } while (0)

#define SY_TRY(expr)                        \
    do {                                    \
        sy_status sy_s_ = (expr);           \
        if (sy_s_ != SY_OK) return sy_s_;   \
    } while (0)

// Host-side fault injection for tests: SY_FAULT=<name>[,<name>...].
bool fault_enabled(const char* name);

// ---- queue -----------------------------------------------------------------------
struct EventRecord {
    cudaEvent_t start = nullptr;
    cudaEvent_t stop = nullptr;
    uint64_t id = 0;       // 0 = slot unused
    int64_t window = -1;   // metering window the kernel was issued in
};

struct Window {
    double joules = 0.0;
    double seconds = 0.0;
    bool closed = false;
    bool have_energy = false;
};

constexpr uint64_t kEventRing = 65536;

struct Queue {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owned = false;
    int sm_count = 0;
    uint64_t launches = 0;
    std::mutex mu;
    // events
    std::vector<EventRecord> ring;
    uint64_t next_event = 1;
    // energy
    void* nvml_device = nullptr;
    bool energy_ok = false;
    uint64_t energy_at_create = 0;
    int64_t open_window = -1;
    uint64_t window_e0 = 0;
    double window_t0 = 0.0;
    std::vector<Window> windows;
    // scratch owned by the queue (allocated on first use)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
};

Queue* as_queue(sy_queue_t q);
sy_status check_queue(sy_queue_t q, Queue** out);
// Ensure the queue's device is current on this thread.
sy_status use_device(Queue* q);
// Scratch of at least `bytes` (device memory owned by the queue).
sy_status queue_scratch(Queue* q, size_t bytes, void** out);

// Event bracketing of one launch.  begin_event records the start event (when
// `want` is non-null) and returns the slot; end_event records the stop event.
sy_status begin_event(Queue* q, sy_event* want, EventRecord** rec);
sy_status end_event(Queue* q, EventRecord* rec);

// ---- checks ------------------------------------------------------------------------
bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes);
sy_status validate_chunks(int64_t n, const sy_chunk* chunks, int n_chunks);
size_t dtype_size(int dtype);

// ---- kernel launchers (implemented in the .cu files) -----------------------------
sy_status launch_saxpy(Queue* q, int64_t n, float alpha, const float* x, const float* y, float* z);

struct WaveLaunch {
    int64_t ny, nx, pitch;
    int radius;
    int dtype;
    int variant;
    float c2;        // coefficient of L u (c2, or c2/2 for the start)
    bool start;      // Taylor start: u + c2 * L u, no u_prev
    const void* u_prev;
    const void* u_cur;
    void* u_next;
    int64_t row_begin, row_end;
};
sy_status launch_wave(Queue* q, const WaveLaunch& w);
int wave_variant_count(int radius, int dtype);
bool wave_variant_info(int radius, int dtype, int variant, int* tile_rows, int* tile_cols, int* threads);

sy_status launch_wave_energy(Queue* q, const sy_stencil_params* p, const void* u_new, const void* u_old,
                             double* partials, int n_partials, double* out3_device);
constexpr int kEnergyBlocks = 1024;

}  // namespace sy
