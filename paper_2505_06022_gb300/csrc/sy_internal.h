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

namespace nvml {
// True once NVML is loaded and initialised (libnvidia-ml.so.1, or SY_NVML_LIB).
bool available();
// An entry point of the loaded NVML library, or nullptr.
void* symbol(const char* name);
}  // namespace nvml

// ---- device-side kernel timestamps -----------------------------------------------
// Each timed launch owns one stamp slot of 4 x u64 in device memory, zeroed before
// use: [0] = ~(earliest block start), [1] = latest block end (both %globaltimer, ns),
// [2] = blocks finished, [3] = spare.  Blocks stamp with atomics, so timing a launch
// adds no operation to the stream and does not separate consecutive kernels.
constexpr uint32_t kStampSlots = 65536;
constexpr uint32_t kStreamStampSlots = 49152;  // ring for directly issued launches
constexpr uint32_t kStampPage = 1024;          // the ring is zeroed page by page ahead of use
constexpr uint32_t kGraphStampSlots = kStampSlots - kStreamStampSlots;
constexpr uint64_t kEventRing = 65536;

struct EventRecord {
    uint64_t id = 0;        // 0 = unused
    uint32_t slot = 0;      // stamp slot
    uint64_t expected = 0;  // blocks that stamp the slot when the launch has finished
    int64_t window = -1;    // metering window the launch was issued in
};

struct Window {
    double joules = 0.0;
    double seconds = 0.0;
    bool closed = false;
    bool have_energy = false;
};

// A cached whole-simulation graph (sy_wave_run, sy_wave3d_run): valid for the
// exact call it was captured for, identified by the bytes of its arguments.
struct RunGraph {
    bool valid = false;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> expected;  // per graph stamp slot
    uint64_t launches = 0;           // kernel launches per replay
    const void* prev_out = nullptr;
    const void* cur_out = nullptr;
};

// Work sets of sy_wave_run_host: call k uses set k mod kHostSets, so a call's input
// copy waits only for the copy-out of the call kHostSets back.
constexpr int kHostSets = 3;

struct HostRun {
    void* ws = nullptr;  // kHostSets sets x 3 fields of `field` bytes (owned)
    size_t ws_bytes = 0;
    size_t field = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;  // owned copy streams
    // per set: host->device copy done, simulation done, device->host copies done
    cudaEvent_t in_done[kHostSets] = {};
    cudaEvent_t sim_done[kHostSets] = {};
    cudaEvent_t out_done[kHostSets] = {};
    RunGraph graph[kHostSets];
    uint64_t calls = 0;
    // per set: the host ranges its latest call writes (u^{steps}, u^{steps-1})
    const void* last_out[kHostSets][2] = {};
    size_t last_out_bytes[kHostSets] = {};
};

struct Queue {
    int device = 0;
    cudaStream_t stream = nullptr;  // the queue's stream (owned or borrowed)
    cudaStream_t launch = nullptr;  // where launchers enqueue: `stream`, or `aux` while capturing
    cudaStream_t aux = nullptr;     // owned: graph capture and timestamp reads
    bool owned = false;
    int sm_count = 0;
    uint64_t launches = 0;
    std::mutex mu;
    // events and timestamps
    std::vector<EventRecord> ring;
    uint64_t next_event = 1;
    unsigned long long* d_stamps = nullptr;
    std::vector<uint64_t> slot_owner;  // event id that last used each slot
    uint32_t next_stream_slot = 0;
    bool capturing = false;
    uint32_t next_graph_slot = 0;           // relative to kStreamStampSlots while capturing
    std::vector<uint64_t> capture_expected;
    // the launch being issued: launchers stamp `cur_stamp` and add their blocks
    unsigned long long* cur_stamp = nullptr;
    uint64_t cur_blocks = 0;
    // energy
    void* nvml_device = nullptr;
    bool energy_ok = false;
    uint64_t energy_at_create = 0;
    int64_t open_window = -1;
    uint64_t window_e0 = 0;
    double window_t0 = 0.0;
    std::vector<Window> windows;
    // error flags kernels with bounded waits set (bit 0: a wait timed out); read and
    // cleared by sy_queue_sync
    unsigned int* d_flags = nullptr;
    // scratch owned by the queue (allocated on first use)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    RunGraph run;    // sy_wave_run
    RunGraph run3;   // sy_wave3d_run
    // sy_wave_run_host: two device work sets (u0, u_a, u_b each) used by alternate
    // calls, one cached graph per set, and copy streams for each direction, so that
    // one call's copies overlap the neighbouring calls' simulations.
    HostRun host;
};

// Waits for / releases what sy_wave_run_host created on the queue (run.cpp).
sy_status host_run_sync(Queue* q);
void host_run_release(Queue* q);

Queue* as_queue(sy_queue_t q);
sy_status check_queue(sy_queue_t q, Queue** out);
// Ensure the queue's device is current on this thread.
sy_status use_device(Queue* q);
// Scratch of at least `bytes` (device memory owned by the queue).
sy_status queue_scratch(Queue* q, size_t bytes, void** out);

// Event bracketing of one logical launch (one or more kernels stamping one slot).
// begin_event assigns a stamp slot when `want` is non-null; the launchers then
// pass q->cur_stamp to their kernels and add their grid sizes to q->cur_blocks;
// end_event closes the record.
sy_status begin_event(Queue* q, sy_event* want, EventRecord** rec);
sy_status end_event(Queue* q, EventRecord* rec);

// ---- checks ------------------------------------------------------------------------
bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes);
sy_status validate_chunks(int64_t n, const sy_chunk* chunks, int n_chunks);
size_t dtype_size(int dtype);

// ---- kernel launchers (implemented in the .cu files) -----------------------------
sy_status launch_saxpy(Queue* q, int64_t n, float alpha, const float* x, const float* y, float* z);
sy_status launch_saxpy_variant(Queue* q, int64_t n, float alpha, const float* x, const float* y, float* z,
                               int variant);
int saxpy_variant_count();
bool saxpy_variant_info(int variant, int* threads, int* waves);

struct WaveLaunch {
    int64_t ny, nx, pitch;
    int radius;
    int dtype;
    int variant;
    float c2;        // coefficient of L u (c2, or c2/2 for the start)
    bool start;      // Taylor start: u + c2 * L u, no u_prev
    int pdl;         // overlap with the previous launch: 0 none, 1 first chunk of a step, 2 later chunk
    const void* u_prev;
    const void* u_cur;
    void* u_next;
    int64_t row_begin, row_end;
    bool reverse = false;  // visit the chunk's tiles last to first (same results)
};
sy_status launch_wave(Queue* q, const WaveLaunch& w);
namespace wave {
// Resident blocks per SM of a kernel at `threads` threads (cached per kernel).
int kernel_occupancy(const void* fn, int threads);
// Programmatic dependent launch between chunk kernels (SY_PDL=0 turns it off).
bool launch_overlap_enabled();
}  // namespace wave

// Halo exchange of split-buffer execution (halo.cu): copy `rows` rows of
// width_bytes each, consecutive rows pitch_bytes apart, from src to dst, for every
// entry, in one launch per 32 entries; pdl = wait for the previous kernel inside the
// launch and let the next one start early (when programmatic launch is enabled).
struct HaloCopy {
    const void* src;
    void* dst;
    int64_t rows;
};
sy_status launch_halo(Queue* q, const HaloCopy* copies, int n, int64_t pitch_bytes, int64_t width_bytes, bool pdl);

// One chunk of planes of the 3D step (wave3d_*.cu).
struct WaveLaunch3 {
    int64_t nz, ny, nx, pitch, plane;  // elements
    int radius;
    int dtype;
    int variant;
    float c2;
    bool start;
    int pdl;
    const void* u_prev;
    const void* u_cur;
    void* u_next;
    int64_t z_begin, z_end;
};
sy_status launch_wave3d(Queue* q, const WaveLaunch3& w);
bool wave3d_variant_info(int radius, int dtype, int variant, int* tile_rows, int* threads);
constexpr int kWave3dVariants = 10;
sy_status stencil3d_param_checks(const sy_stencil3d_params* p);
// reverse: launch the chunks last to first (chunk_events[c] still belongs to chunk c).
sy_status stencil3d_common(Queue* q, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                           void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                           sy_event* chunk_events, bool start, bool reverse = false);

// Replays (capturing on first use) the graph of a whole run.  `key` identifies
// the call; `issue` enqueues its launches on q->launch and reports the buffers
// holding u^{steps-1} and u^{steps}; `timed` = stamped launches per replay.
sy_status graph_run(Queue* q, RunGraph& g, const std::vector<unsigned char>& key, uint64_t timed, bool want,
                    sy_status (*issue)(Queue*, const void*, const void**, const void**), const void* ctx,
                    sy_event* events, const void** prev_out, const void** cur_out);
// Argument checks and one launch per chunk, shared by sy_stencil_step/start/run;
// reverse: launch the chunks last to first (chunk_events[c] still belongs to chunk c).
sy_status stencil_common(Queue* q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                         void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                         sy_event* chunk_events, bool start, bool reverse = false);
sy_status stencil_param_checks(const sy_stencil_params* p);
int wave_variant_count(int radius, int dtype);
// The variant (1..count) that variant 0 stands for.
int wave_default_variant(int radius, int dtype);
bool wave_variant_info(int radius, int dtype, int variant, int* tile_rows, int* tile_cols, int* threads);

// Temporal blocking (tb.cu): T steps per pass for rows [row_begin, row_end).
struct TBLaunch {
    int64_t ny, nx, pitch_bytes;
    int radius, dtype, T;
    float c2;
    const void* u_prev;
    const void* u_cur;
    void* out_prev;
    void* out_cur;
    int64_t row_begin, row_end;
    int fault;  // host-injected fault for tests
    int pdl;
};
sy_status launch_tb(Queue* q, const TBLaunch& w);

sy_status launch_wave_energy(Queue* q, const sy_stencil_params* p, const void* u_new, const void* u_old,
                             double* partials, int n_partials, double* out3_device);
constexpr int kEnergyBlocks = 1024;
// Second stage of the fixed-shape FP64 energy reduction: sums 2 x kEnergyBlocks
// partials (kinetic, potential) and writes (kin - c2 pot, kin, pot) to out3.
sy_status launch_energy_final(cudaStream_t stream, const double* partials, double c2, double* out3);
// The 3D energy: first stage (wave3d.cu) then launch_energy_final, on q->launch.
sy_status launch_wave3d_energy(Queue* q, const sy_stencil3d_params* p, const void* u_new, const void* u_old,
                               double* partials, double* out3_device);

}  // namespace sy
