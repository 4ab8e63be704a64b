/*
 * sy.h -- C ABI of libsy: range-mapped data-parallel kernels for one GB300
 * (sm_103a) GPU, with per-kernel timing and energy metering.
 *
 * The programming model follows the paper's SYCL extensions:
 *   - a queue stands for one device and one in-order stream (paper §2, Listing 1:
 *     kernels are submitted to a queue bound to a device);
 *   - a submission is a parallel_for over an index range whose accessors state
 *     which buffers it reads and writes (paper §2, Listing 1);
 *   - a range mapper ties a chunk of the execution range to the data the chunk
 *     touches, and the runtime splits a kernel into chunks (paper §3, Listing 2);
 *   - each submission yields an event whose kernel energy can be queried, and the
 *     device energy can be queried as a whole (paper §4, Listing 3).
 *
 * General rules (every entry point):
 *   - Every call returns sy_status; SY_OK is 0.  No C++ exception crosses the ABI.
 *     On failure, sy_last_error() returns a thread-local message.
 *   - "device pointer" arguments are CUDA global-memory addresses on the queue's
 *     device, owned by the caller; the library never frees them.  "host pointer"
 *     arguments are ordinary host memory.
 *   - Launches are asynchronous on the queue's stream unless a call says it
 *     synchronises.  Inputs must stay valid until the work has completed.
 *   - Argument checks (null pointers, sizes, aliasing, chunk lists) happen on the
 *     host before anything is launched; a rejected call launches nothing.
 *   - All kernels are hand-written CUDA for sm_103a; there is no CPU fallback.
 *     SY_ERR_CUDA reports a CUDA runtime error (message in sy_last_error()).
 *   - A queue is not safe for concurrent calls: calls taking the same queue (or a
 *     plan or model made on it) must not overlap in time -- issue them from one
 *     host thread or serialise them.  Different queues may be driven from
 *     different threads at once; the library's shared tables are locked.
 */
#ifndef SY_H
#define SY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define SY_ABI_VERSION 1

typedef enum sy_status {
    SY_OK = 0,
    SY_ERR_INVALID_ARGUMENT = 1, /* a size, radius, dtype or option is out of range */
    SY_ERR_NULL_POINTER = 2,     /* a required pointer is NULL */
    SY_ERR_ALIAS = 3,            /* buffers overlap in a way the call forbids */
    SY_ERR_BAD_CHUNKS = 4,       /* chunk list does not tile the range in order */
    SY_ERR_HALO_TOO_SMALL = 5,   /* declared halo radius < stencil radius */
    SY_ERR_UNSUPPORTED = 6,      /* feature unavailable on this device / system */
    SY_ERR_CUDA = 7,             /* CUDA runtime error */
    SY_ERR_NVML_UNAVAILABLE = 8, /* NVML missing or energy counter unsupported */
    SY_ERR_TIMEOUT = 9,          /* a bounded device-side wait gave up */
    SY_ERR_OUT_OF_MEMORY = 10,   /* library-internal allocation failed */
    SY_ERR_NOT_READY = 11,       /* queried work has not completed */
    SY_ERR_IO = 12,              /* file read/write failed */
    SY_ERR_NVML = 13             /* an NVML call failed (return code in sy_last_error()) */
} sy_status;

/* Storage type of a field.  Arithmetic is always FP32 (energy: FP64). */
typedef enum sy_dtype { SY_F32 = 0, SY_BF16 = 1, SY_F16 = 2 } sy_dtype;

typedef struct sy_queue_s* sy_queue_t;

/* Event id of one submitted kernel (0 = none).  Valid for the queue that issued
 * it until 65536 newer events have been issued on that queue. */
typedef uint64_t sy_event;

/* A half-open sub-range [begin, end) of an execution range (rows for 2D). */
typedef struct sy_chunk {
    int64_t begin;
    int64_t end;
} sy_chunk;

/* ------------------------------------------------------------------------- */
/* Status and errors                                                          */
/* ------------------------------------------------------------------------- */

const char* sy_status_string(sy_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* sy_last_error(void);
int sy_abi_version(void);

/* ------------------------------------------------------------------------- */
/* Queue (paper §2, Listing 1: a queue bound to one GPU device)               */
/* ------------------------------------------------------------------------- */

/* Borrow the legacy default stream (the runtime's cudaStreamLegacy handle); the
 * stream handle 0 cannot be used for this because NULL requests an owned stream. */
#define SY_STREAM_LEGACY ((void*)0x1)

/* Create a queue on CUDA device `device`.  `cuda_stream` is a cudaStream_t to
 * borrow (never destroyed by the library), SY_STREAM_LEGACY for the legacy
 * default stream, or NULL to create an owned non-blocking stream.  The queue remembers the device energy counter at
 * creation (for sy_device_energy) when NVML is available. */
sy_status sy_queue_create(int device, void* cuda_stream, sy_queue_t* out);
sy_status sy_queue_destroy(sy_queue_t q);
/* Block until all work submitted to the queue has completed (including the
 * host copies of sy_wave_run_host).  Returns
 * SY_ERR_TIMEOUT (once) if a kernel's bounded wait gave up since the last sync. */
sy_status sy_queue_sync(sy_queue_t q);
/* The cudaStream_t the queue submits to. */
sy_status sy_queue_stream(sy_queue_t q, void** cuda_stream);
/* Number of kernel launches this queue has issued so far. */
sy_status sy_queue_launch_count(sy_queue_t q, uint64_t* launches);

/* ------------------------------------------------------------------------- */
/* Events: per-kernel time and energy (paper §4, Listing 3)                   */
/* ------------------------------------------------------------------------- */

/* Device time of an event's launch in milliseconds: from the first block's start
 * to the last block's end, read from %globaltimer stamps the kernels themselves
 * write (no operation is added to the stream, so timing does not slow the
 * launches down).  Returns SY_ERR_NOT_READY if the launch has not completed. */
sy_status sy_event_elapsed(sy_queue_t q, sy_event ev, double* ms);

/* Device times of n events at once (one copy of the timestamp ring); ms receives
 * n values.  Fails with SY_ERR_NOT_READY if any of them has not completed. */
sy_status sy_events_elapsed(sy_queue_t q, const sy_event* events, int n, double* ms);

/* Raw NVML total-energy counter of the queue's device, in millijoules
 * (nvmlDeviceGetTotalEnergyConsumption).  SY_ERR_NVML_UNAVAILABLE if NVML cannot
 * be loaded or the counter is unsupported. */
sy_status sy_energy_read(sy_queue_t q, uint64_t* millijoules);

/* Device energy in joules since the queue was created (paper §4, Listing 3:
 * the queue's whole-device energy query).  Includes every process's work on the GPU. */
sy_status sy_device_energy(sy_queue_t q, double* joules);

/* Metering window.  sy_meter_begin synchronises the queue and samples the energy
 * counter and the host clock; sy_meter_end synchronises again and samples them
 * again, returning the energy (J) and wall time (s) of the window.  Kernels
 * issued inside a closed window get an energy attribution (below).  The counter
 * updates at a coarse period, so windows should last well beyond it (about
 * 100 ms or more on current drivers). */
sy_status sy_meter_begin(sy_queue_t q);
sy_status sy_meter_end(sy_queue_t q, double* joules, double* seconds);

/* Energy of one kernel (paper §4, Listing 3: the energy query on a kernel's event):
 * the average device power of the closed metering window the kernel ran in,
 * times the kernel's device time.  SY_ERR_NOT_READY if the kernel was not
 * issued inside a window that has since been closed. */
sy_status sy_kernel_energy(sy_queue_t q, sy_event ev, double* joules);


/* ------------------------------------------------------------------------- */
/* SAXPY (paper §2 Listing 1; §3 Listing 2 with one_to_one range mappers)     */
/* ------------------------------------------------------------------------- */

/* z[i] = alpha * x[i] + y[i] for i in [0, n), evaluated as two FP32 roundings
 * fl(fl(alpha * x[i]) + y[i]) (no fused multiply-add).  x, y, z: device
 * pointers to n floats.  z may be exactly x or exactly y (in place) but must not
 * partially overlap either.  Any alignment is accepted (16-byte aligned
 * pointers take the vector path).  n == 0 is a no-op.  `ev` (nullable) receives
 * the event of the launch. */
sy_status sy_saxpy(sy_queue_t q, int64_t n, float alpha, const float* x, const float* y, float* z, sy_event* ev);

/* The same kernel split into chunks (paper §3, Listing 2): chunk c covers
 * [chunks[c].begin, chunks[c].end) with one_to_one range mappers, one launch per
 * chunk.  The chunks must tile [0, n) in order; events (nullable) receives
 * n_chunks event ids. */
sy_status sy_saxpy_split(sy_queue_t q, int64_t n, float alpha, const float* x, const float* y, float* z,
                         const sy_chunk* chunks, int n_chunks, sy_event* events);

/* ------------------------------------------------------------------------- */
/* Range mappers and splitting (paper §3)                                     */
/* ------------------------------------------------------------------------- */

/* Even split of [0, n) into k chunks; the first n % k chunks are one longer.
 * out: host array of k chunks.  k >= 1, n >= 0. */
sy_status sy_split_rows(int64_t n, int k, sy_chunk* out);

/* one_to_one range mapper: chunk [begin, end) touches exactly [begin, end). */
sy_status sy_rm_one_to_one(sy_chunk chunk, sy_chunk* region);

/* neighbourhood range mapper of radius r: chunk [begin, end) of a domain of n
 * rows reads [begin - r, end + r) clipped to [0, n). */
sy_status sy_rm_neighbourhood(sy_chunk chunk, int radius, int64_t n, sy_chunk* region);

/* SY_OK when chunks tile [0, n) in order with no empty chunk, else
 * SY_ERR_BAD_CHUNKS. */
sy_status sy_chunks_validate(int64_t n, const sy_chunk* chunks, int n_chunks);

/* ------------------------------------------------------------------------- */
/* 2D leapfrog wave stencil (range-split, neighbourhood range mappers)        */
/* ------------------------------------------------------------------------- */
/* The field is row-major: element (i, j), 0 <= i < ny, 0 <= j < nx, lives at
 * index i * pitch + j; a field buffer holds ny * pitch elements of its dtype.
 * Points outside the grid are zero (Dirichlet-zero ghosts).
 *
 *   L u_ij  = 2 w_0 u_ij + sum_{k=1..r} w_k ((u_{i-k,j} + u_{i+k,j}) + (u_{i,j-k} + u_{i,j+k}))
 *   u^{n+1} = (2 u^n - u^{n-1}) + c2 * L u^n
 *
 * with w the order-2r central second-difference weights (r = 1: 1, -2, 1;
 * r = 2: -1/12, 4/3, -5/2, ...; Fornberg 1988) rounded once to FP32, evaluated
 * in FP32 in exactly this order, and the result rounded once to the storage
 * type (round to nearest even).  16-bit values are widened exactly to FP32. */

typedef struct sy_stencil_params {
    int64_t ny;      /* rows (>= 0) */
    int64_t nx;      /* columns (>= 0) */
    int64_t pitch;   /* elements between row starts (>= nx) */
    int32_t radius;  /* stencil radius r, 1..4 */
    int32_t dtype;   /* sy_dtype of all three fields */
    float c2;        /* (c dt / dx)^2 */
    int32_t variant; /* kernel tile variant, 0 = library default (see sy_stencil_variant_count) */
} sy_stencil_params;

/* One leapfrog step, split into row chunks with a neighbourhood range mapper of
 * radius halo_radius: chunk c writes rows [begin, end) of u_next and reads rows
 * [begin - r, end + r) (clipped) of u_cur and rows [begin, end) of u_prev; one
 * launch per chunk, in list order, on the queue's stream.
 *   u_prev, u_cur: device pointers (read); u_next: device pointer (written).
 *   u_next may be exactly u_prev (in place) but must not overlap u_cur, nor
 *   partially overlap u_prev.
 *   chunks: host array tiling [0, ny) in order (SY_ERR_BAD_CHUNKS otherwise).
 *   halo_radius < radius gives SY_ERR_HALO_TOO_SMALL.
 *   chunk_events (nullable): n_chunks event ids, one per chunk launch.
 * Results do not depend on the chunking: any valid chunk list gives the same
 * bits. */
sy_status sy_stencil_step(sy_queue_t q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                          void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                          sy_event* chunk_events);

/* Per-chunk statistics of one stepped chunk list (the events sy_stencil_step
 * returned for `chunks`, in order): device time, algorithmic bytes (read u^n and
 * u^{n-1}, write u^{n+1}: 3 x sizeof(storage) per point), grid-point updates and
 * energy (sy_kernel_energy; -1 when the launch lies in no closed metering
 * window or NVML is unavailable).  SY_ERR_NOT_READY until the launches complete. */
typedef struct sy_chunk_stats {
    double ms;
    double bytes;
    double joules;
    double updates;
} sy_chunk_stats;
sy_status sy_chunk_stats_read(sy_queue_t q, const sy_stencil_params* p, const sy_chunk* chunks,
                              const sy_event* events, int n, sy_chunk_stats* out);

/* Measured energy of one chunk's step kernel (the metering mode of the paper's
 * per-kernel energy query, §4 Listing 3): the launch sy_stencil_step issues for
 * chunks[c] (same variant, range mapper and halo rules) is replayed back to back
 * inside one NVML metering window lasting at least min_seconds and min_reps
 * launches; *joules and *ms are the window's energy and the launches' device time
 * (CUDA events on the queue's stream) divided by the *reps launches.  The window
 * holds nothing else, so this measures the chunk, unlike sy_kernel_energy, which
 * attributes a shared window's average power by time.  Idle power is not
 * subtracted.  u_next is overwritten each time (from the same inputs unless it
 * aliases u_prev); the queue is synchronised; no metering window may be open.
 * NVML's counter ticks every ~100 ms on GB300, so min_seconds >= 0.5 gives a
 * resolution of a few percent.  SY_ERR_NVML_UNAVAILABLE (with *ms and *reps set,
 * *joules = -1) when the counter cannot be read. */
sy_status sy_chunk_energy_replay(sy_queue_t q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                                 void* u_next, const sy_chunk* chunks, int n_chunks, int c, int halo_radius,
                                 double min_seconds, int min_reps, double* joules, double* ms, int* reps);

/* Taylor start for zero initial velocity: u_m1 = u0 + (c2 / 2) * L u0, evaluated
 * as fl(u0 + fl((c2/2) * L u0)) with L as above (bit-identical to a step with c2
 * halved and u_prev = u_cur = u0).  u_m1 must not overlap u0.  Same chunk rules
 * as sy_stencil_step. */
sy_status sy_stencil_start(sy_queue_t q, const sy_stencil_params* p, const void* u0, void* u_m1,
                           const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* chunk_events);

/* A whole simulation in one call: the Taylor start from u0, then `steps` leapfrog
 * steps, each split into the chunks as in sy_stencil_step.  The launches are
 * captured into a CUDA graph on the first call and the graph is replayed by later
 * calls with identical arguments (one cached graph per queue; changing any
 * argument re-captures).  u0 (device, read) is never written; u_a and u_b
 * (device) are work fields that receive the results: on return *prev_out and
 * *cur_out (nullable) name the buffers (u0, u_a or u_b) holding u^{steps-1} and
 * u^{steps}.  u0, u_a, u_b must not overlap.  events (nullable) receives
 * (steps + 1) * n_chunks ids -- the start's chunks, then each step's, in chunk
 * order -- valid until the next sy_wave_run on this queue (at most 16384 per run;
 * pass NULL beyond).  The chunks of a step are independent, so the run orders
 * them for cache reuse: odd steps launch the chunks last to first and sweep each
 * chunk's rows bottom to top, so that a step starts on the rows the previous step
 * touched last (results are identical to any other order). */
sy_status sy_wave_run(sy_queue_t q, const sy_stencil_params* p, const void* u0, void* u_a, void* u_b, int64_t steps,
                      const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* events, const void** prev_out,
                      const void** cur_out);

/* sy_wave_run on host memory: the runtime moves the data, as the paper's
 * buffer/accessor model has it (§2 Listing 1, §3: a kernel names the data it
 * accesses and the runtime makes it present where the kernel runs).  The call
 * copies host_u0 (ny x pitch elements of p's storage type, the device layout)
 * into device memory the queue owns, runs the Taylor start and `steps` chunked
 * steps exactly as sy_wave_run does (same launches, same cached-graph replay,
 * same results), and copies u^{steps} into host_out and, when host_prev_out is
 * not NULL, u^{steps-1} into host_prev_out (each ny x pitch elements).
 *   - Asynchronous: the call returns once the work is enqueued.  host_u0 must
 *     stay unchanged, and host_out / host_prev_out must not be read, until
 *     sy_queue_sync(q) returns.  With pinned host memory (cudaHostAlloc or
 *     cudaHostRegister) the copies are asynchronous; pageable memory works, but
 *     its copies synchronise with the host.
 *   - Consecutive calls overlap: calls rotate through three device work sets of
 *     three fields each (allocated on the first call and when a larger grid
 *     arrives, freed by sy_queue_destroy), and the copies run on one stream per
 *     direction, so a call's input copy overlaps the earlier calls' simulations and
 *     its output copy the later calls', and an input copy waits only for the
 *     output copy of the call three back.  A call whose host_u0 overlaps an
 *     earlier call's outputs waits for those copies first, so feeding a result
 *     back in is safe.
 *   - host_out and host_prev_out must not overlap each other (SY_ERR_ALIAS);
 *     host_u0 may equal host_out (it is read before the result is written).
 *   - events as in sy_wave_run (valid until the next whole run on this queue);
 *     other errors as in sy_wave_run. */
sy_status sy_wave_run_host(sy_queue_t q, const sy_stencil_params* p, const void* host_u0, void* host_out,
                           void* host_prev_out, int64_t steps, const sy_chunk* chunks, int n_chunks, int halo_radius,
                           sy_event* events);

/* Temporal blocking: T leapfrog steps (T = 2 or 4; radius 1 to 4) in one pass over
 * memory.  Each chunk reads u^{n-1} (u_prev) and u^n (u_cur) with a halo of T x r
 * rows (halo_radius >= T * radius) and writes u^{n+T-1} (out_prev) and u^{n+T}
 * (out_cur) for its rows; the intermediate steps are recomputed on the halo in
 * shared memory instead of being written and re-read.  Tiles are staged by TMA
 * (rows must be 16-byte aligned: base pointers and pitch).  Results are
 * bit-identical to T calls of sy_stencil_step.  The outputs must not overlap the
 * inputs or each other (chunks read each other's input rows while writing).
 * The kernel's waits are bounded: if one gives up, the next sy_queue_sync returns
 * SY_ERR_TIMEOUT and the outputs are invalid.  Fields of 2^31 rows or columns or
 * more (the copies' coordinates are 32-bit) are refused with SY_ERR_UNSUPPORTED. */
sy_status sy_stencil_multistep(sy_queue_t q, const sy_stencil_params* p, int T, const void* u_prev,
                               const void* u_cur, void* out_prev, void* out_cur, const sy_chunk* chunks, int n_chunks,
                               int halo_radius, sy_event* chunk_events);

/* Number of tile variants for a (radius, dtype); variant ids are 1..count
 * (0 always means the default).  tile_rows / tile_cols / threads (nullable)
 * describe variant `variant`: a warp tile of tile_rows x tile_cols output points,
 * `threads` per block.  tile_cols = 32 x (16 / element size) is the register
 * tile whose outer lanes load the columns beside it; tile_cols = 30 x (16 /
 * element size) is the halo-lane form, whose two outer lanes hold those columns
 * instead of producing output (no edge registers, 1/16 of the lanes idle).
 * Variants 1-8: register tiles of 2/4/8/16 rows x 128/256 threads; 9-12:
 * halo-lane tiles of 4/8 rows x 128/256 threads; for 16-bit storage also 13-14:
 * narrow halo-lane tiles (4 elements, 8 bytes, a lane: tile_cols = 120) of 4/8
 * rows x 128 threads, which hold half the registers per tile row, and 15: the march
 * form (each warp walks a strip of tile_cols columns down a segment of rows, rows
 * copied into shared memory by TMA; tile_rows = 32 is nominal: the segment length
 * is chosen per launch so that every resident warp takes one segment). */
sy_status sy_stencil_variant_count(int radius, int dtype, int* count);
/* The variant (1..count) that variant 0 stands for at this radius and storage. */
sy_status sy_stencil_default_variant(int radius, int dtype, int* variant);
sy_status sy_stencil_variant_info(int radius, int dtype, int variant, int* tile_rows, int* tile_cols,
                                  int* threads);

/* Discrete energy of the leapfrog scheme, conserved exactly when L is symmetric:
 *   E^{n+1/2} = sum (u_new - u_old)^2 - c2 * sum u_new * (L u_old)
 * summed over the whole grid in FP64 (fields widened exactly; L with FP64
 * weights).  The reduction has a fixed shape, so repeated calls give identical
 * bits.  Synchronises the queue; energy, kinetic (sum of squares) and potential
 * (sum u_new * L u_old) are host pointers, the last two nullable.  Uses a
 * scratch buffer the queue allocates on first use. */
sy_status sy_wave_energy(sy_queue_t q, const sy_stencil_params* p, const void* u_new, const void* u_old,
                         double* energy, double* kinetic, double* potential);

/* ------------------------------------------------------------------------- */
/* Data transfers inferred from range mappers; split-buffer execution           */
/* ------------------------------------------------------------------------- */
/* paper §3: the runtime splits a kernel across devices and uses the range
 * mappers to infer the data transfers each chunk needs before it runs.  For the
 * neighbourhood mapper of halo radius h, chunk c = [a, b) reads [a - h, b + h)
 * clipped to [0, ny); the rows it does not write are moved from the chunks that
 * write them, one transfer per run of rows with a single owner. */
typedef struct sy_transfer {
    int32_t src;       /* chunk that owns (writes) the rows */
    int32_t dst;       /* chunk that reads them */
    int64_t row_begin; /* global rows [row_begin, row_end) */
    int64_t row_end;
} sy_transfer;

/* All transfers for a chunk list, in order of destination chunk (rows above, then
 * below).  out = NULL only counts (*n_out). */
sy_status sy_rm_transfers(int64_t ny, const sy_chunk* chunks, int n_chunks, int halo_radius, sy_transfer* out,
                          int max_out, int* n_out);

/* Local buffer of chunk c in split-buffer mode: halo_lo = min(h, begin) rows above
 * its own rows, halo_hi = min(h, ny - end) rows below; local_rows = halo_lo +
 * (end - begin) + halo_hi rows of p->pitch elements.  (Each pointer nullable.) */
sy_status sy_split_layout(int64_t ny, const sy_chunk* chunks, int n_chunks, int halo_radius, int chunk,
                          int64_t* halo_lo, int64_t* halo_hi, int64_t* local_rows);

/* One step with every chunk's fields in buffers of its own (the layout above), as
 * chunks on separate devices would hold them: first the inferred halo rows of
 * u_cur are copied between the chunks' buffers (one halo-exchange kernel for all
 * transfers), then each chunk's rows are stepped; consecutive launches overlap
 * (programmatic dependent launch, SY_PDL=0 turns it off), each waiting for its
 * predecessor's writes before it reads.  local_prev / local_cur / local_next: arrays of n_chunks
 * device pointers; p describes the global grid.  Aliasing rules per chunk as in
 * sy_stencil_step.  Bit-identical to sy_stencil_step on one shared buffer. */
sy_status sy_stencil_step_split(sy_queue_t q, const sy_stencil_params* p, void* const* local_prev,
                                void* const* local_cur, void* const* local_next, const sy_chunk* chunks,
                                int n_chunks, int halo_radius, sy_event* chunk_events);
/* One chunk on its own: step rows [row_begin, row_end) of the grid in p, reading
 * [row_begin - r, row_end + r) clipped (the neighbourhood range mapper), with no
 * requirement that other chunks exist -- the kernel a device runs on the chunk it
 * holds (its halo rows having been brought in by the caller).  start != 0 runs the
 * Taylor start instead (u_prev unused).  Same aliasing rules as sy_stencil_step. */
sy_status sy_stencil_step_rows(sy_queue_t q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                               void* u_next, int64_t row_begin, int64_t row_end, int halo_radius, int start,
                               sy_event* ev);
/* The Taylor start in split-buffer mode (halos of u0 refreshed first). */
sy_status sy_stencil_start_split(sy_queue_t q, const sy_stencil_params* p, void* const* local_u0,
                                 void* const* local_um1, const sy_chunk* chunks, int n_chunks, int halo_radius,
                                 sy_event* chunk_events);

/* ------------------------------------------------------------------------- */
/* Batched stencils: many independent, unevenly sized grids in one launch     */
/* ------------------------------------------------------------------------- */
/* Each grid is advanced with the stencil of sy_stencil_step over its whole row
 * range (one chunk).  One persistent launch steps every grid once: the warps
 * stride over the concatenated tile list of all grids, so small and large grids
 * share the GPU instead of paying one launch each.  A run of steps can be
 * captured into a CUDA graph and replayed.  Results are bit-identical to
 * stepping every grid with sy_stencil_step. */
typedef struct sy_batch_grid {
    int64_t ny;     /* rows (>= 1) */
    int64_t nx;     /* columns (>= 1) */
    int64_t pitch;  /* elements between row starts (>= nx); pitch * sizeof(dtype) % 16 == 0 */
    int32_t radius; /* 1..4 */
    float c2;       /* (c dt / dx)^2 */
    void* u_a;      /* device, 16-byte aligned, ny * pitch elements: u^{n-1} (or u^{-1} after the start) */
    void* u_b;      /* device, 16-byte aligned, ny * pitch elements: u^n (or u^0 before the start) */
} sy_batch_grid;

typedef struct sy_batch_plan_s* sy_batch_plan_t;

/* Build a plan over n_grids (1..4096) grids of one dtype.  tile_rows: tile height
 * of the warp tiles, 2, 4 or 8 for every grid (one launch per step, each grid's
 * radius chosen at run time), or 0 for per-radius launches: the grids of each
 * radius get a kernel compiled for that radius (its own register budget, the
 * single-field default tile height), and the launches of a step overlap.  The grids' buffers must not overlap each
 * other.  The plan copies the descriptors to the device; the buffers stay owned by
 * the caller and must outlive the plan. */
sy_status sy_stencil_batch_plan(sy_queue_t q, const sy_batch_grid* grids, int n_grids, int dtype, int tile_rows,
                                sy_batch_plan_t* out);
/* Totals of a plan (each pointer nullable): warp tiles, grid points, blocks of the
 * persistent launches of one step. */
sy_status sy_stencil_batch_info(sy_batch_plan_t plan, int64_t* total_tiles, int64_t* points, int* blocks);
/* Taylor start for every grid: u_a = u_b + (c2/2) L u_b (one launch). */
sy_status sy_stencil_batch_start(sy_batch_plan_t plan, int timed);
/* One leapfrog step of every grid (one launch).  parity 0: u_a <- step(u_a, u_b);
 * parity 1: u_b <- step(u_b, u_a).  timed != 0 records the launch's device time
 * (read with sy_stencil_batch_times, index 0). */
sy_status sy_stencil_batch_step(sy_batch_plan_t plan, int parity, int timed);
/* Capture `steps` consecutive steps, parities 0, 1, 0, ... into a CUDA graph owned
 * by the plan (replacing any earlier capture).  Every launch is timed. */
sy_status sy_stencil_batch_capture(sy_batch_plan_t plan, int64_t steps);
/* The same `steps` steps as ONE cooperative launch (the cross-step form): every
 * block of a co-resident grid walks the classes' tiles of a step, then meets the
 * others at a grid-wide barrier before the next step.  One kernel carries every
 * radius (with the per-class tile heights), so its register budget is that of
 * the radius-4 tiles.  The barrier's wait is bounded (about 1 s): if it gives up,
 * the next sy_queue_sync returns SY_ERR_TIMEOUT and the fields are invalid.
 * Needs a per-class plan (tile_rows = 0) and a device with cooperative launch
 * (SY_ERR_UNSUPPORTED otherwise); replaces any earlier capture, replayed by
 * sy_stencil_batch_run with the same parity rules; its one launch is timed
 * (sy_stencil_batch_times index 1). */
sy_status sy_stencil_batch_capture_persistent(sy_batch_plan_t plan, int64_t steps);
/* Replay the captured steps on the queue's stream.  Each replay starts at parity
 * 0, so with an even step count consecutive replays continue the simulation; after
 * a replay of an odd count u_a holds the newest field. */
sy_status sy_stencil_batch_run(sy_batch_plan_t plan);
/* Device times (ms) of the plan's timed launches: index 0 = the last timed
 * sy_stencil_batch_start/step, index 1 + s = step s of the last replay. */
sy_status sy_stencil_batch_times(sy_batch_plan_t plan, double* ms, int n);
sy_status sy_stencil_batch_destroy(sy_batch_plan_t plan);

/* ------------------------------------------------------------------------- */
/* Learned cost model: a 3-layer MLP trained on the GPU by the library's kernels */
/* ------------------------------------------------------------------------- */
/* Not in the paper (whose SYnergy layer picks device frequencies by model-driven
 * energy targets, §4): here a small MLP predicts (log time, log energy) of a
 * kernel configuration from its features, and the dispatcher takes the argmin.
 *   h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3   (FP32)
 *   loss = mean over samples and outputs of (y - t)^2, Adam (Kingma & Ba 2015).
 * Parameter vector: W1[H][F] b1[H] W2[H][H] b2[H] W3[O][H] b3[O] (row-major,
 * out x in).  Limits: F <= 32, H <= 64, O <= 4.  The model's weights and
 * training scratch are device buffers owned by the handle. */
typedef struct sy_mlp_s* sy_mlp_t;

/* New model, weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from `seed`, biases 0,
 * identity normalisation. */
sy_status sy_mlp_create(sy_queue_t q, int in_features, int hidden, int out_features, uint64_t seed, sy_mlp_t* out);
sy_status sy_mlp_destroy(sy_mlp_t m);
sy_status sy_mlp_param_count(sy_mlp_t m, int64_t* n);
/* Host copies of the parameters / of the last gradient (n = param count). */
sy_status sy_mlp_get_params(sy_mlp_t m, float* host, int64_t n);
sy_status sy_mlp_get_grad(sy_mlp_t m, float* host, int64_t n);
/* Replace the parameters (and reset Adam's moments). */
sy_status sy_mlp_set_params(sy_mlp_t m, const float* host, int64_t n);
/* Raw forward (no normalisation): d_X device B x F (row-major), d_Y device B x O. */
sy_status sy_mlp_forward(sy_mlp_t m, const float* d_X, int64_t B, float* d_Y);
/* Forward + backward on device d_X (B x F), d_T (B x O): the gradient of the loss
 * goes into the model's gradient buffer; *loss (nullable, host) receives the loss
 * (and then the call synchronises).  The reduction over samples has a fixed shape,
 * so the gradient is bit-reproducible. */
sy_status sy_mlp_loss_grad(sy_mlp_t m, const float* d_X, const float* d_T, int64_t B, float* loss);
/* The backward pass under its own name: identical to sy_mlp_loss_grad. */
sy_status sy_mlp_backward(sy_mlp_t m, const float* d_X, const float* d_T, int64_t B, float* loss);
/* One Adam step with the current gradient. */
sy_status sy_mlp_adam_step(sy_mlp_t m, float lr, float beta1, float beta2, float eps);
/* Train on host arrays X (n x F) and T (n x O): the inputs and targets are
 * normalised to zero mean / unit variance per column (kept in the model), then
 * `epochs` passes of Adam (beta 0.9 / 0.999, eps 1e-8) over minibatches of
 * `batch` samples in an order shuffled per epoch from `seed`.  *final_loss
 * (nullable) = loss of the last minibatch (normalised units). */
sy_status sy_mlp_train(sy_mlp_t m, const float* X, const float* T, int64_t n, int epochs, int batch, float lr,
                       uint64_t seed, float* final_loss);
/* The model's normalisation vectors (each nullable; F, F, O, O floats). */
sy_status sy_mlp_normalization(sy_mlp_t m, float* x_mean, float* x_std, float* y_mean, float* y_std);
/* Predictions in target units for n host feature rows (n x F) -> pred (n x O). */
sy_status sy_cost_model_predict(sy_mlp_t m, const float* features, int64_t n, float* pred);
/* Index of the candidate (row of features, n x F) with the smallest predicted
 * objective: 0 = time (output 0), 1 = energy (output 1), 2 = energy-delay product
 * (sum of the two log outputs). */
sy_status sy_cost_model_choose(sy_mlp_t m, const float* features, int n, int objective, int* best);
/* Save / load a model (parameters and normalisation) as a small binary file. */
sy_status sy_mlp_save(sy_mlp_t m, const char* path);
sy_status sy_mlp_load(sy_queue_t q, const char* path, sy_mlp_t* out);

/* ------------------------------------------------------------------------- */
/* Exhaustive autotuner and cost-model features                                 */
/* ------------------------------------------------------------------------- */
/* One measured candidate.  Stencil: variant = tile variant (tile_rows x
 * tile_cols warp tiles, `threads` per block).  SAXPY: variant = launch variant,
 * tile_rows = waves of blocks per SM, tile_cols = 4 (floats per access),
 * threads per block.  ms = median device time of one run over all chunks. */
typedef struct sy_tune_record {
    int32_t variant;
    int32_t tile_rows;
    int32_t tile_cols;
    int32_t threads;
    int32_t chunks;
    double ms;
} sy_tune_record;

/* Time every tile variant x chunk count of one stencil step on the caller's
 * buffers (same rules as sy_stencil_step; halo = radius): one warm-up run and
 * `reps` timed runs per candidate, device timestamps, median.  out holds at
 * least variant_count x n_counts records; *n_out receives how many were written.
 * Synchronises the queue after every run. */
sy_status sy_tune_stencil(sy_queue_t q, const sy_stencil_params* p, const void* u_prev, const void* u_cur,
                          void* u_next, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                          int max_out, int* n_out);
/* The same for SAXPY over n floats (z = 1.5 x + y), launch variant x chunk count. */
sy_status sy_tune_saxpy(sy_queue_t q, int64_t n, const float* x, const float* y, float* z, const int* chunk_counts,
                        int n_counts, int reps, sy_tune_record* out, int max_out, int* n_out);
/* SAXPY launch variants: 1..count; variant 0 is the default of sy_saxpy. */
sy_status sy_saxpy_variant_count(int* count);
sy_status sy_saxpy_variant_info(int variant, int* threads, int* waves);
/* sy_saxpy_split with an explicit launch variant (what a tuner or the cost model chose). */
sy_status sy_saxpy_config(sy_queue_t q, int64_t n, float alpha, const float* x, const float* y, float* z,
                          int variant, const sy_chunk* chunks, int n_chunks, sy_event* events);

/* A candidate configuration described for the cost model. */
typedef struct sy_cost_query {
    int32_t kind;      /* 0 = SAXPY, 1 = stencil step */
    int32_t dtype;     /* storage (SAXPY: SY_F32) */
    int32_t radius;    /* stencil radius (SAXPY: 0) */
    int64_t ny, nx;    /* grid (SAXPY: ny = 1, nx = n) */
    int32_t tile_rows; /* as in sy_tune_record */
    int32_t tile_cols;
    int32_t threads;
    int32_t chunks;
} sy_cost_query;
#define SY_COST_FEATURES 13
/* The model's input features of a candidate (SY_COST_FEATURES floats): kind,
 * log2 bytes/point, flops/point, radius, log2 ny, log2 nx, log2 points,
 * log2 tile_rows, log2 threads, log2 chunks, log2 total bytes, halo read factor
 * (tile_rows + 2r) / tile_rows, log2 tile count. */
sy_status sy_cost_features(const sy_cost_query* query, float* out);

/* ------------------------------------------------------------------------- */
/* Energy targets by frequency scaling (paper §4: a queue given the target    */
/* MIN_EDP runs at the clock frequency that minimises the energy-delay        */
/* product; frequencies are set through NVML on NVIDIA GPUs).                 */
/*                                                                            */
/* Device selection here is by NVML index, so that the host logic runs       */
/* without a GPU; sy_clock_nvml_index maps a CUDA ordinal to it.              */
/* Changing clocks alters a device-wide setting that outlives the process and */
/* every other user of the GPU inherits; sy_clock_lock, sy_clock_unlock and   */
/* sy_clock_sweep therefore refuse with SY_ERR_UNSUPPORTED, before any NVML   */
/* call, unless the environment variable SY_CLOCK_CONTROL is "1".             */
/* ------------------------------------------------------------------------- */
typedef enum sy_energy_target {
    SY_TARGET_MIN_TIME = 0,   /* minimise t */
    SY_TARGET_MIN_ENERGY = 1, /* minimise E */
    SY_TARGET_MIN_EDP = 2,    /* minimise E * t (the paper's MIN_EDP) */
    SY_TARGET_MIN_ED2P = 3    /* minimise E * t^2 */
} sy_energy_target;

/* One measured (or predicted) operating point of a kernel or region. */
typedef struct sy_freq_point {
    uint32_t sm_mhz; /* SM (graphics) clock the point was taken at */
    double seconds;  /* time of the measured work, > 0 */
    double joules;   /* energy of the measured work, >= 0 */
} sy_freq_point;

/* Index of the point that minimises the target's objective.  Ties go to the
 * higher clock, then to the lower index.  SY_ERR_INVALID_ARGUMENT for n < 1, an
 * unknown target, or a time <= 0, energy < 0 or a non-finite value. */
sy_status sy_clock_choose(int target, const sy_freq_point* points, int n, int* index);

/* NVML index of CUDA device `cuda_device` (matched by PCI bus id). */
sy_status sy_clock_nvml_index(int cuda_device, uint32_t* nvml_index);

/* Read-only: the memory clock the device runs at and the SM clocks NVML
 * supports with it, highest first (at most `cap` written, *n = how many exist). */
sy_status sy_clock_supported(uint32_t nvml_index, uint32_t* mem_mhz, uint32_t* sm_mhz, int cap, int* n);

/* Read-only: current and maximum SM clock. */
sy_status sy_clock_current(uint32_t nvml_index, uint32_t* sm_mhz, uint32_t* sm_max_mhz);

/* Lock the SM clock to `sm_mhz` (one of sy_clock_supported's values, else
 * SY_ERR_INVALID_ARGUMENT), and release the lock.  Gated as described above;
 * SY_ERR_NVML if NVML refuses (e.g. no permission). */
sy_status sy_clock_lock(uint32_t nvml_index, uint32_t sm_mhz);
sy_status sy_clock_unlock(uint32_t nvml_index);

/* Called by sy_clock_sweep with the clock locked at sm_mhz: runs the work and
 * reports its time and energy; returns 0 on success, anything else aborts. */
typedef int (*sy_measure_fn)(void* ctx, uint32_t sm_mhz, double* seconds, double* joules);

/* Per-kernel frequency selection by measurement: for each of the n candidate
 * clocks in order, lock it, call `measure`, and record the point in
 * points[i]; then release the lock (always, also after a failure) and choose
 * by `target` (*best = index into points).  Gated as described above.  Every
 * candidate is validated before the first lock.  A failing measure returns
 * SY_ERR_INVALID_ARGUMENT with the lock already released. */
sy_status sy_clock_sweep(uint32_t nvml_index, const uint32_t* sm_mhz, int n, sy_measure_fn measure, void* ctx,
                         int target, sy_freq_point* points, int* best);

/* ------------------------------------------------------------------------- */
/* Range mappers on boxes (paper §3: a range mapper ties the chunk of the     */
/* execution range a device runs to the part of a buffer it accesses, and the */
/* runtime infers the data transfers from it; the paper names one_to_one, the */
/* other kinds are this library's).                                           */
/* ------------------------------------------------------------------------- */
/* A box is [lo[d], hi[d]) in each of 3 dimensions, dimension 0 the slowest (a
 * 1D or 2D range uses extent 1 in the dimensions it lacks).  Empty when
 * lo[d] >= hi[d] in some dimension. */
typedef struct sy_box {
    int64_t lo[3];
    int64_t hi[3];
} sy_box;

typedef enum sy_rm_kind {
    SY_RM_ONE_TO_ONE = 0,    /* the chunk itself */
    SY_RM_NEIGHBOURHOOD = 1, /* the chunk grown by radius[d] on both sides of dimension d */
    SY_RM_SLICE = 2,         /* the chunk with dimension `dim` widened to the whole buffer */
    SY_RM_ALL = 3,           /* the whole buffer */
    SY_RM_FIXED = 4          /* the box `fixed` */
} sy_rm_kind;

typedef struct sy_range_mapper {
    int32_t kind;      /* sy_rm_kind */
    int32_t dim;       /* SY_RM_SLICE: 0..2 */
    int64_t radius[3]; /* SY_RM_NEIGHBOURHOOD: >= 0 */
    sy_box fixed;      /* SY_RM_FIXED */
} sy_range_mapper;

/* The part of a buffer of `extent` (3 sizes >= 0) that a kernel over `chunk`
 * accesses under the mapper, clipped to [0, extent).  SY_ERR_INVALID_ARGUMENT
 * for an unknown kind, a negative radius or extent, or dim outside 0..2. */
sy_status sy_rm_box(const sy_range_mapper* rm, const sy_box* chunk, const int64_t* extent, sy_box* out);

/* One transfer: `box` (inside chunk src's own box) must reach chunk dst. */
typedef struct sy_box_transfer {
    int32_t src, dst;
    sy_box box;
} sy_box_transfer;

/* Transfers a kernel with this mapper needs when chunk c holds exactly the
 * current values of its own box: for each dst, then each src != dst, the
 * non-empty intersection of rm(chunk_dst) with chunk_src.  The n chunks must
 * tile the buffer (non-empty, disjoint, covering [0, extent)), else
 * SY_ERR_BAD_CHUNKS.  *n_out = how many exist; more than max_out gives
 * SY_ERR_INVALID_ARGUMENT (out then holds the first max_out). */
sy_status sy_rm_box_transfers(const sy_range_mapper* rm, const sy_box* chunks, int n, const int64_t* extent,
                              sy_box_transfer* out, int max_out, int* n_out);

/* ------------------------------------------------------------------------- */
/* Leapfrog step on a 3D grid (a second workload), chunked along planes: a    */
/* chunk is a range of planes [begin, end) and reads the planes the            */
/* neighbourhood range mapper (radius along dimension 0) gives it.            */
/*   L u = 3 w_0 u + sum_{m=1..r} w_m ( ((u[z][y-m][x] + u[z][y+m][x])         */
/*                   + (u[z][y][x-m] + u[z][y][x+m])) + (u[z-m][y][x] + u[z+m][y][x]) ) */
/*   u^{n+1} = (2 u^n - u^{n-1}) + c2 * L u^n;  start u^{-1} = u^0 + (c2/2) L u^0 */
/* with the weights, ghosts, rounding and storage rules of sy_stencil_step.   */
/* ------------------------------------------------------------------------- */
typedef struct sy_stencil3d_params {
    int64_t nz, ny, nx; /* grid: nz planes of ny rows of nx points */
    int64_t pitch;      /* elements from one row to the next, >= nx */
    int64_t plane;      /* elements from one plane to the next, >= ny * pitch */
    int32_t radius;     /* 1..4 */
    int32_t dtype;      /* storage, sy_dtype */
    float c2;           /* (c dt / dx)^2; stable for c2 * 12 * sum_k |w_k| <= 4 */
    int32_t variant;    /* 0 = default tile, 1..sy_stencil3d_variant_count */
} sy_stencil3d_params;

/* One step of every chunk (chunks = plane ranges tiling [0, nz) in order; one
 * launch each).  Fields are device buffers of nz x plane elements (caller-owned);
 * padding is read but never written.  u_next may be u_prev (in place), must not
 * overlap u_cur.  The
 * fast path needs 16-byte aligned pointers, row and plane strides; other
 * element-aligned layouts take a one-point-per-thread kernel.  Events as in
 * sy_stencil_step. */
sy_status sy_stencil3d_step(sy_queue_t q, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                            void* u_next, const sy_chunk* chunks, int n_chunks, int halo_radius,
                            sy_event* chunk_events);
/* Taylor start: u_m1 = u0 + (c2/2) L u0. */
sy_status sy_stencil3d_start(sy_queue_t q, const sy_stencil3d_params* p, const void* u0, void* u_m1,
                             const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* chunk_events);
/* One chunk of planes on its own: step planes [plane_begin, plane_end) of the
 * grid in p, reading the planes the neighbourhood range mapper gives them, with
 * no requirement that other chunks exist -- the kernel a device runs on the
 * chunk it holds (its halo planes brought in by the caller).  start != 0 runs
 * the Taylor start (u_prev unused).  Same aliasing rules as sy_stencil3d_step. */
sy_status sy_stencil3d_step_planes(sy_queue_t q, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                                   void* u_next, int64_t plane_begin, int64_t plane_end, int halo_radius, int start,
                                   sy_event* ev);
/* Start + `steps` steps as one cached CUDA graph, as sy_wave_run (odd steps
 * launch the chunks of planes last to first; each chunk's tiles in their usual
 * order). */
sy_status sy_wave3d_run(sy_queue_t q, const sy_stencil3d_params* p, const void* u0, void* u_a, void* u_b,
                        int64_t steps, const sy_chunk* chunks, int n_chunks, int halo_radius, sy_event* events,
                        const void** prev_out, const void** cur_out);
/* Discrete energy of the 3D scheme, E^{n+1/2} = sum (u_new - u_old)^2 - c2 *
 * sum u_new * (L u_old), in FP64 with a fixed reduction shape (as sy_wave_energy,
 * whose scratch buffer it shares). */
sy_status sy_wave3d_energy(sy_queue_t q, const sy_stencil3d_params* p, const void* u_new, const void* u_old,
                           double* energy, double* kinetic, double* potential);
/* Tile variants 1-6: rows of a warp's tile (1, 2, 4) x threads per block (128,
 * 256); variants 7-8: a block of 8 warps marching a strip of 8 or 16 rows with
 * the strip's centre plane in shared memory (tile_rows reports the strip,
 * threads 256); variants 9-10: the same strips with every plane copied into a
 * shared-memory ring by TMA ahead of use; variant 0 is the default. */
sy_status sy_stencil3d_variant_count(int radius, int dtype, int* count);
sy_status sy_stencil3d_variant_info(int radius, int dtype, int variant, int* tile_rows, int* threads);

/* Exhaustive tuner of the 3D step (as sy_tune_stencil): its tile variants x chunk counts (plane chunks). */
sy_status sy_tune_stencil3d(sy_queue_t q, const sy_stencil3d_params* p, const void* u_prev, const void* u_cur,
                            void* u_next, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                            int max_out, int* n_out);
/* Exhaustive search over every candidate of one kernel kind, the baseline the
 * cost model's regret is measured against: kind SY_TUNE_SAXPY (n elements;
 * in0 = x, in1 = y, out_buf = z; params unused), SY_TUNE_STENCIL (params = a
 * sy_stencil_params; in0 = u_prev, in1 = u_cur, out_buf = u_next) or
 * SY_TUNE_STENCIL3D (params = a sy_stencil3d_params; same buffers).  Records as
 * the per-kind tuners above; *best = index of the fastest record. */
#define SY_TUNE_SAXPY 0
#define SY_TUNE_STENCIL 1
#define SY_TUNE_STENCIL3D 2
sy_status sy_tune_exhaustive(sy_queue_t q, int kind, const void* params, int64_t n, const void* in0, const void* in1,
                             void* out_buf, const int* chunk_counts, int n_counts, int reps, sy_tune_record* out,
                             int max_out, int* n_out, int* best);

/* Checkpoint / resume of a 2D simulation: the two time levels the recurrence
 * needs and the step count.  Save synchronises the queue and writes u_prev, u_cur
 * (rows without pitch padding) and `step` to `path`; load checks that the file
 * holds the grid, storage, radius and c2 of p (else SY_ERR_INVALID_ARGUMENT),
 * fills u_prev, u_cur (any pitch) and *step, and synchronises.  Stepping on from
 * a loaded checkpoint gives the bits of an uninterrupted run.  SY_ERR_IO for
 * unreadable, foreign or truncated files. */
sy_status sy_checkpoint_save(sy_queue_t q, const char* path, const sy_stencil_params* p, const void* u_prev,
                             const void* u_cur, int64_t step);
sy_status sy_checkpoint_load(sy_queue_t q, const char* path, const sy_stencil_params* p, void* u_prev, void* u_cur,
                             int64_t* step);

/* Allocation-free form of sy_wave_energy.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * moment they need the energy -- code issuing work while a stream is being
 * captured into a CUDA graph in global mode (cudaMalloc is not permitted then),
 * applications whose own allocator owns all device memory, and loops that must
 * never hit the device-wide synchronisation cudaMalloc/cudaFree can cause.  It
 * allocates nothing and synchronises nothing:
 *   - The per-block partial sums live in one fixed module-scope device array of
 *     2 x 1024 doubles (16 KiB), which every GPU that loads the library holds
 *     until the process exits.  The reduction has a fixed shape that uses exactly
 *     that many for any grid size (checked when the library is compiled), so no
 *     grid is too large for it.
 *   - It runs on the calling thread's current device, on `cuda_stream` (a
 *     cudaStream_t; NULL = the legacy default stream), with no queue.
 *   - out3 (device, 3 doubles, caller-owned) receives energy, kinetic and
 *     potential, as sy_wave_energy computes them (same kernels, same order).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and keeps it for the life of the process, per device
 *     ordinal; make that first call before any stream capture.  The address
 *     belongs to the device's primary context: calling this from another context
 *     (one created with the driver API), or after cudaDeviceReset, is not
 *     supported.
 *   - Every call shares the one array and leaves its partial sums there; each
 *     call overwrites all of them before reading, so nothing needs clearing, but
 *     calls that overlap on the GPU (different streams, or a graph replayed
 *     concurrently) race on it and must be serialised by the caller. */
sy_status sy_wave_energy_static(void* cuda_stream, const sy_stencil_params* p, const void* u_new, const void* u_old,
                                double* out3);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* SY_H */
