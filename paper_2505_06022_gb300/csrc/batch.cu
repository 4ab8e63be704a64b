// Batched leapfrog steps over many independent, unevenly sized grids: one
// persistent launch advances every grid by one step, and a run of steps is
// captured into a CUDA graph.
//
// Work list: the warp tiles of all grids, concatenated in plan order (each grid's
// tiles in row-major order), stored once per plan as a table of packed (grid,
// tile column, tile row) entries.  A persistent grid of SMs x occupancy blocks
// strides over that table; a warp reads its next entry one tile ahead (a
// broadcast load that is in flight while the current tile computes), so moving to
// another grid costs no search and no division, and runs the same tile code as
// the single-field kernel (wave_tile).  Grids of every size therefore share the
// GPU in one launch instead of paying one launch (and one partially filled last
// wave) per grid.
//
// Buffers: grid g owns u_a and u_b.  A step with parity 0 reads u_a (u^{n-1})
// and u_b (u^n) and writes u^{n+1} over u_a; parity 1 swaps the roles.  The
// Taylor start writes u^{-1} = start(u_b) into u_a.
#include <mutex>
#include <new>
#include <vector>

#include "tma.cuh"
#include "wave_kernel.cuh"

namespace sy {

struct BatchGridDev {
    char* ua;
    char* ub;
    int64_t ny, nx, pitch_bytes;
    int64_t tiles_x;
    int32_t radius;
    float c2;
    float neg0;  // -0.0f (the packed products' addend, a run-time value)
};

// A group of grids stepped by one persistent launch: every grid of the plan
// (radius chosen per grid at run time), or, in per-radius mode, the grids of one
// radius (a kernel compiled for that radius, with its own register budget).
struct BatchClass {
    int radius = 0;           // 0 = mixed radii
    int64_t desc_off = 0;     // first descriptor of the class in d_desc
    int64_t tile_off = 0;     // first entry of the class in d_tiles
    int n = 0;                // grids in the class
    int64_t tiles = 0;
    int blocks = 0;           // persistent grid size of the class's launch
};

struct BatchPlan {
    Queue* q = nullptr;
    int dtype = 0;
    int tile_rows = 4;
    int n_grids = 0;
    int64_t total_tiles = 0;
    int64_t points = 0;
    std::vector<BatchClass> classes;
    BatchGridDev* d_desc = nullptr;
    uint64_t* d_tiles = nullptr;             // packed work list, class by class
    unsigned long long* d_stamps = nullptr;  // slot 0: last direct launch; 1..: graph launches
    int64_t stamp_slots = 0;
    std::vector<uint64_t> expected;          // blocks per stamped launch (index = slot)
    cudaGraphExec_t exec = nullptr;
    int64_t graph_steps = 0;
    uint64_t graph_launches = 0;
    int blocks = 0;                          // persistent grid size
    int threads = 128;
    unsigned* d_sync = nullptr;              // cross-step form: [0] barrier arrivals, [1] abort flag
    int persistent_blocks = 0;               // cross-step form: co-resident grid of its launch
};

namespace {

constexpr int kBatchThreads = 128;
constexpr int kMaxBatchGrids = 4096;  // grid index: 12 bits of a work-list entry

// Work-list entry: grid index within its class (bits 52..63), tile row (bits 20..51),
// tile column (bits 0..19).
constexpr int kTileXBits = 20, kTileYBits = 32;
__host__ __device__ __forceinline__ uint64_t pack_tile(int64_t g, int64_t tx, int64_t ty) {
    return (static_cast<uint64_t>(g) << (kTileXBits + kTileYBits)) | (static_cast<uint64_t>(ty) << kTileXBits) |
           static_cast<uint64_t>(tx);
}

template <typename S, int R, int RY, bool START, bool CG = false>
__device__ __forceinline__ void batch_tile(const BatchGridDev& G, int parity, int64_t tx, int64_t ty, int lane) {
    wave::Args a;
    const bool swap = (parity & 1) != 0;
    a.u_prev = swap ? G.ub : G.ua;
    a.u_cur = START ? G.ub : (swap ? G.ua : G.ub);
    a.u_next = START ? G.ua : (swap ? G.ub : G.ua);
    a.ny = G.ny;
    a.nx = G.nx;
    a.pitch_bytes = G.pitch_bytes;
    a.row_begin = 0;
    a.row_end = G.ny;
    a.tiles_x = G.tiles_x;
    a.tiles = 0;
    a.c2 = START ? 0.5f * G.c2 : G.c2;
    a.stamp = nullptr;
    a.pdl = 0;
    a.neg0 = G.neg0;
    wave::wave_tile<S, R, RY, START, false, CG>(a, tx, ty, lane);
}

// Tile height of the per-radius kernels: FP32 4/4/8/4 rows for r = 1..4, 16-bit 4/4/8/8.
// The single-field defaults, except FP32 radius 1, where the batch's smaller grids run
// 1.3 % faster on 4-row tiles than on the single field's 2 (64 uneven grids, 100 steps;
// 2-row tiles for radius 2 or 4 measured 1.3 % and 5.8 % slower).
template <typename S, int R>
struct ClassRows {
    static constexpr int value = sizeof(S) == 4 ? (R == 3 ? 8 : 4) : (R <= 2 ? 4 : 8);
};

// RFIX = 0: grids of any radius, dispatched per grid at run time, RY-row tiles (one
// kernel carries every radius, so its register budget is that of the largest
// branch).  RFIX = 1..4: every grid has that radius, ClassRows tiles.
// pdl as in the single-field kernel: 1 = wait for the previous launch first, 2 = an
// independent launch of the same step; with either, completion implies the
// predecessor's completion.
template <typename S, int RFIX, int RY, bool START>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BatchGridDev* __restrict__ grids,
                                                              const uint64_t* __restrict__ work, int64_t total_tiles,
                                                              int parity, unsigned long long* stamp, int pdl) {
    static_assert(RFIX != 0 || RY != 0, "a mixed-radius kernel needs a tile height");
    if (pdl == 1) griddep_wait();
    if (pdl) griddep_launch_dependents();
    stamp_begin(stamp);
    const int lane = threadIdx.x & 31;
    const int64_t warps_per_block = blockDim.x >> 5;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * warps_per_block;
    int64_t t = static_cast<int64_t>(blockIdx.x) * warps_per_block + (threadIdx.x >> 5);
    uint64_t cur = t < total_tiles ? __ldg(work + t) : 0;
    for (; t < total_tiles; t += nwarps) {
        const uint64_t next = t + nwarps < total_tiles ? __ldg(work + t + nwarps) : 0;
        const int g = static_cast<int>(cur >> (kTileXBits + kTileYBits));
        const int64_t ty = static_cast<int64_t>((cur >> kTileXBits) & ((1ull << kTileYBits) - 1));
        const int64_t tx = static_cast<int64_t>(cur & ((1ull << kTileXBits) - 1));
        const BatchGridDev& G = grids[g];
        if (RFIX) {
            batch_tile<S, RFIX ? RFIX : 1, ClassRows<S, RFIX ? RFIX : 1>::value, START>(G, parity, tx, ty, lane);
        } else {
            switch (G.radius) {
                case 1: batch_tile<S, 1, RY ? RY : 4, START>(G, parity, tx, ty, lane); break;
                case 2: batch_tile<S, 2, RY ? RY : 4, START>(G, parity, tx, ty, lane); break;
                case 3: batch_tile<S, 3, RY ? RY : 4, START>(G, parity, tx, ty, lane); break;
                default: batch_tile<S, 4, RY ? RY : 4, START>(G, parity, tx, ty, lane); break;
            }
        }
        cur = next;
    }
    stamp_end(stamp);
    if (pdl && threadIdx.x == 0) griddep_wait();
}

// ---- cross-step form: a whole run in one launch ----------------------------------
// Every step of every class in one cooperative launch (all blocks co-resident): each
// step walks the classes' work lists in turn, with the tile heights of the per-class
// kernels, and a grid-wide barrier separates consecutive steps.  One kernel carries
// every radius, so its register budget is that of the radius-4 tiles.  Fields are
// written by one step and read by the next within the launch, so every load goes
// through L2 (ld.global.cg), made coherent by the barrier's fences.  The barrier's
// wait is bounded: a block that gives up sets the queue's error flag and an abort
// flag that releases the others, and every block returns (sy_queue_sync then reports
// SY_ERR_TIMEOUT and the fields are invalid).
struct PersistClass {
    int64_t desc_off, tile_off, tiles;
    int radius;
};

struct PersistArgs {
    const BatchGridDev* grids;
    const uint64_t* work;
    PersistClass cls[4];
    int n_cls;
    int64_t steps;
    unsigned* barrier;  // arrivals; zeroed before the launch
    unsigned* abort;    // set by a block whose wait gave up; zeroed before the launch
    unsigned* err;      // the queue's error flags (bit 0: a bounded wait gave up)
    int fault;          // host-injected for tests: 1 = block 0 never arrives at the first barrier
    unsigned long long* stamp;
};

template <typename S, int R>
__device__ __forceinline__ void persist_class(const BatchGridDev* __restrict__ grids, const uint64_t* __restrict__ work,
                                              int64_t tiles, int parity, int64_t w, int64_t nwarps, int lane) {
    for (int64_t t = w; t < tiles; t += nwarps) {
        const uint64_t e = __ldg(work + t);
        const int g = static_cast<int>(e >> (kTileXBits + kTileYBits));
        const int64_t ty = static_cast<int64_t>((e >> kTileXBits) & ((1ull << kTileYBits) - 1));
        const int64_t tx = static_cast<int64_t>(e & ((1ull << kTileXBits) - 1));
        batch_tile<S, R, ClassRows<S, R>::value, false, true>(grids[g], parity, tx, ty, lane);
    }
}

// Grid-wide barrier after step s: true when every block arrived, false if the wait
// gave up (or another block's did).
__device__ __forceinline__ bool persist_barrier(const PersistArgs& a, int64_t s) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // this block's writes of step s, before its arrival
        if (!(a.fault == 1 && s == 0 && blockIdx.x == 0)) atomicAdd(a.barrier, 1u);
        const unsigned target = static_cast<unsigned>(s + 1) * gridDim.x;
        const long long t0 = clock64();
        for (;;) {
            unsigned v, ab;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.barrier) : "memory");
            if (v >= target) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(a.abort) : "memory");
            if (ab || clock64() - t0 > tma::kWaitCycles) {
                atomicOr(a.err, 1u);
                atomicExch(a.abort, 1u);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename S>
__global__ void __launch_bounds__(kBatchThreads) batch_persistent_kernel(PersistArgs a) {
    stamp_begin(a.stamp);
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * wpb;
    const int64_t w = static_cast<int64_t>(blockIdx.x) * wpb + (threadIdx.x >> 5);
    for (int64_t s = 0; s < a.steps; ++s) {
        const int parity = static_cast<int>(s & 1);
        for (int c = 0; c < a.n_cls; ++c) {
            const PersistClass& K = a.cls[c];
            const BatchGridDev* G = a.grids + K.desc_off;
            const uint64_t* W = a.work + K.tile_off;
            switch (K.radius) {
                case 1: persist_class<S, 1>(G, W, K.tiles, parity, w, nwarps, lane); break;
                case 2: persist_class<S, 2>(G, W, K.tiles, parity, w, nwarps, lane); break;
                case 3: persist_class<S, 3>(G, W, K.tiles, parity, w, nwarps, lane); break;
                default: persist_class<S, 4>(G, W, K.tiles, parity, w, nwarps, lane); break;
            }
        }
        if (s + 1 < a.steps && !persist_barrier(a, s)) return;  // block-uniform
    }
    stamp_end(a.stamp);
}

using PersistFn = void (*)(PersistArgs);

PersistFn persist_fn(int dtype) {
    switch (dtype) {
        case SY_F32: return batch_persistent_kernel<float>;
        case SY_BF16: return batch_persistent_kernel<__nv_bfloat16>;
        default: return batch_persistent_kernel<__half>;
    }
}

using BatchFn = void (*)(const BatchGridDev*, const uint64_t*, int64_t, int, unsigned long long*, int);

// radius 1..4: the class kernel of that radius (per-radius plans); radius 0: the
// mixed-radius kernel with tile_rows-row tiles (2, 4 or 8).
template <typename S, bool START>
BatchFn pick_batch(int tile_rows, int radius) {
    switch (radius) {
        case 1: return batch_kernel<S, 1, 0, START>;
        case 2: return batch_kernel<S, 2, 0, START>;
        case 3: return batch_kernel<S, 3, 0, START>;
        case 4: return batch_kernel<S, 4, 0, START>;
    }
    switch (tile_rows) {
        case 2: return batch_kernel<S, 0, 2, START>;
        case 8: return batch_kernel<S, 0, 8, START>;
        default: return batch_kernel<S, 0, 4, START>;
    }
}

// Tile height a grid of radius r gets: per-radius mode (tile_rows == 0) uses ClassRows,
// a uniform plan tile_rows.
int rows_for(int tile_rows, int radius, size_t es) {
    if (tile_rows) return tile_rows;
    if (es == 4) return radius == 3 ? 8 : 4;  // as ClassRows
    return radius <= 2 ? 4 : 8;
}

BatchFn batch_fn(int dtype, int tile_rows, int radius, bool start) {
    switch (dtype) {
        case SY_F32: return start ? pick_batch<float, true>(tile_rows, radius) : pick_batch<float, false>(tile_rows, radius);
        case SY_BF16:
            return start ? pick_batch<__nv_bfloat16, true>(tile_rows, radius)
                         : pick_batch<__nv_bfloat16, false>(tile_rows, radius);
        default:
            return start ? pick_batch<__half, true>(tile_rows, radius) : pick_batch<__half, false>(tile_rows, radius);
    }
}

BatchPlan* as_plan(sy_batch_plan_t p) { return reinterpret_cast<BatchPlan*>(p); }

// One step (or the start) of every grid: one persistent launch per class, on
// q->launch; the first waits for the previous launch, later classes of the same step
// overlap it.  `slot` < 0 means untimed.
sy_status launch_batch(BatchPlan* P, bool start, int parity, int64_t slot) {
    Queue* q = P->q;
    unsigned long long* stamp = slot >= 0 ? P->d_stamps + 4 * slot : nullptr;
    uint64_t blocks = 0;
    for (size_t c = 0; c < P->classes.size(); ++c) {
        const BatchClass& K = P->classes[c];
        if (K.tiles == 0) continue;
        BatchFn fn = batch_fn(P->dtype, P->tile_rows, K.radius, start);
        const int pdl = c == 0 ? 1 : 2;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(K.blocks));
        cfg.blockDim = dim3(P->threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = q->launch;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SY_CUDA(cudaLaunchKernelEx(&cfg, fn, static_cast<const BatchGridDev*>(P->d_desc + K.desc_off),
                                   static_cast<const uint64_t*>(P->d_tiles + K.tile_off), K.tiles, parity, stamp,
                                   pdl));
        ++q->launches;
        blocks += static_cast<uint64_t>(K.blocks);
    }
    if (slot >= 0) P->expected[slot] = blocks;
    return SY_OK;
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" {

sy_status sy_stencil_batch_plan(sy_queue_t qh, const sy_batch_grid* grids, int n_grids, int dtype, int tile_rows,
                                sy_batch_plan_t* out) {
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    if (!out) return fail(SY_ERR_NULL_POINTER, "out is NULL");
    *out = nullptr;
    if (n_grids < 1 || n_grids > kMaxBatchGrids)
        return fail(SY_ERR_INVALID_ARGUMENT, "n_grids = %d not in 1..%d", n_grids, kMaxBatchGrids);
    if (!grids) return fail(SY_ERR_NULL_POINTER, "grids is NULL");
    const size_t esize = dtype_size(dtype);
    if (!esize) return fail(SY_ERR_INVALID_ARGUMENT, "unknown dtype %d", dtype);
    if (tile_rows != 0 && tile_rows != 2 && tile_rows != 4 && tile_rows != 8)
        return fail(SY_ERR_INVALID_ARGUMENT, "tile_rows %d not in {0, 2, 4, 8}", tile_rows);
    const int V = static_cast<int>(16 / esize);
    // validation first, in the caller's order
    for (int g = 0; g < n_grids; ++g) {
        const sy_batch_grid& G = grids[g];
        if (G.ny < 1 || G.nx < 1 || G.pitch < G.nx)
            return fail(SY_ERR_INVALID_ARGUMENT, "grid %d: bad size %lld x %lld (pitch %lld)", g, (long long)G.ny,
                        (long long)G.nx, (long long)G.pitch);
        if (G.radius < 1 || G.radius > 4) return fail(SY_ERR_INVALID_ARGUMENT, "grid %d: radius %d", g, G.radius);
        if (!G.u_a || !G.u_b) return fail(SY_ERR_NULL_POINTER, "grid %d: field pointer is NULL", g);
        const int64_t pb = G.pitch * static_cast<int64_t>(esize);
        if ((reinterpret_cast<uintptr_t>(G.u_a) | reinterpret_cast<uintptr_t>(G.u_b)) % 16 || pb % 16)
            return fail(SY_ERR_INVALID_ARGUMENT,
                        "grid %d: batched fields need 16-byte aligned rows (base and pitch); use sy_stencil_step", g);
        const size_t bytes = static_cast<size_t>(G.ny) * static_cast<size_t>(pb);
        if (ranges_overlap(G.u_a, bytes, G.u_b, bytes)) return fail(SY_ERR_ALIAS, "grid %d: u_a overlaps u_b", g);
        for (int h = 0; h < g; ++h) {  // grids must not share memory (they are updated concurrently)
            const size_t hb = static_cast<size_t>(grids[h].ny) * grids[h].pitch * esize;
            if (ranges_overlap(G.u_a, bytes, grids[h].u_a, hb) || ranges_overlap(G.u_a, bytes, grids[h].u_b, hb) ||
                ranges_overlap(G.u_b, bytes, grids[h].u_a, hb) || ranges_overlap(G.u_b, bytes, grids[h].u_b, hb))
                return fail(SY_ERR_ALIAS, "grids %d and %d overlap", h, g);
        }
    }
    // classes: per radius (tile_rows == 0) or one mixed class; descriptors class by class
    std::vector<BatchClass> classes;
    std::vector<BatchGridDev> desc;
    std::vector<uint64_t> work;
    desc.reserve(n_grids);
    const int radii_lo = tile_rows == 0 ? 1 : 0, radii_hi = tile_rows == 0 ? 4 : 0;
    int64_t total_tiles = 0, points = 0;
    for (int r = radii_lo; r <= radii_hi; ++r) {
        BatchClass K;
        K.radius = r;
        K.desc_off = static_cast<int64_t>(desc.size());
        K.tile_off = static_cast<int64_t>(work.size());
        for (int g = 0; g < n_grids; ++g) {
            const sy_batch_grid& G = grids[g];
            if (r != 0 && G.radius != r) continue;
            BatchGridDev D;
            D.ua = static_cast<char*>(G.u_a);
            D.ub = static_cast<char*>(G.u_b);
            D.ny = G.ny;
            D.nx = G.nx;
            D.pitch_bytes = G.pitch * static_cast<int64_t>(esize);
            D.tiles_x = (G.nx + 32 * V - 1) / (32 * V);
            D.radius = G.radius;
            D.c2 = G.c2;
            D.neg0 = -0.0f;
            const int rows = rows_for(tile_rows, G.radius, esize);
            const int64_t tiles_y = (G.ny + rows - 1) / rows;
            if (D.tiles_x >= (int64_t(1) << kTileXBits) || tiles_y >= (int64_t(1) << kTileYBits))
                return fail(SY_ERR_INVALID_ARGUMENT, "grid %d: %lld x %lld is too large for a batched plan", g,
                            (long long)G.ny, (long long)G.nx);
            for (int64_t ty = 0; ty < tiles_y; ++ty)
                for (int64_t tx = 0; tx < D.tiles_x; ++tx) work.push_back(pack_tile(K.n, tx, ty));
            K.tiles += D.tiles_x * tiles_y;
            points += G.ny * G.nx;
            desc.push_back(D);
            ++K.n;
        }
        if (K.n) {
            total_tiles += K.tiles;
            classes.push_back(K);
        }
    }
    const int64_t tiles = total_tiles;
    SY_TRY(use_device(q));
    BatchPlan* P = new (std::nothrow) BatchPlan();
    if (!P) return fail(SY_ERR_OUT_OF_MEMORY, "plan allocation failed");
    P->q = q;
    P->dtype = dtype;
    P->tile_rows = tile_rows;
    P->n_grids = n_grids;
    P->total_tiles = tiles;
    P->points = points;
    P->classes = classes;
    cudaError_t e = cudaMalloc(&P->d_desc, sizeof(BatchGridDev) * desc.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_desc, desc.data(), sizeof(BatchGridDev) * desc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_tiles, sizeof(uint64_t) * work.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_tiles, work.data(), sizeof(uint64_t) * work.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        P->stamp_slots = 1;
        e = cudaMalloc(&P->d_stamps, 4 * sizeof(unsigned long long));
        P->expected.assign(1, 0);
    }
    for (BatchClass& K : P->classes) {  // persistent grid per class, sized for its step kernel
        int occ = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, reinterpret_cast<const void*>(batch_fn(dtype, tile_rows, K.radius, false)), kBatchThreads, 0);
        if (occ < 1) occ = 1;
        const int64_t want = (K.tiles + kBatchThreads / 32 - 1) / (kBatchThreads / 32);
        const int64_t cap = static_cast<int64_t>(occ) * q->sm_count;
        K.blocks = static_cast<int>(want < cap ? want : cap);
        if (K.blocks < 1) K.blocks = 1;
    }
    if (e != cudaSuccess) {
        if (P->d_desc) cudaFree(P->d_desc);
        if (P->d_tiles) cudaFree(P->d_tiles);
        if (P->d_stamps) cudaFree(P->d_stamps);
        delete P;
        return cuda_fail(e, "sy_stencil_batch_plan");
    }
    P->blocks = 0;
    for (const BatchClass& K : P->classes) P->blocks += K.blocks;
    *out = reinterpret_cast<sy_batch_plan_t>(P);
    return SY_OK;
}

sy_status sy_stencil_batch_info(sy_batch_plan_t ph, int64_t* total_tiles, int64_t* points, int* blocks) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    if (total_tiles) *total_tiles = P->total_tiles;
    if (points) *points = P->points;
    if (blocks) *blocks = P->blocks;
    return SY_OK;
}

sy_status sy_stencil_batch_start(sy_batch_plan_t ph, int timed) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    SY_TRY(use_device(P->q));
    if (timed) SY_CUDA(cudaMemsetAsync(P->d_stamps, 0, 4 * sizeof(unsigned long long), P->q->launch));
    return launch_batch(P, true, 0, timed ? 0 : -1);
}

sy_status sy_stencil_batch_step(sy_batch_plan_t ph, int parity, int timed) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    SY_TRY(use_device(P->q));
    if (timed) SY_CUDA(cudaMemsetAsync(P->d_stamps, 0, 4 * sizeof(unsigned long long), P->q->launch));
    return launch_batch(P, false, parity, timed ? 0 : -1);
}

sy_status sy_stencil_batch_capture(sy_batch_plan_t ph, int64_t steps) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    if (steps < 1 || steps > (1 << 20)) return fail(SY_ERR_INVALID_ARGUMENT, "steps = %lld", (long long)steps);
    Queue* q = P->q;
    SY_TRY(use_device(q));
    SY_CUDA(cudaStreamSynchronize(q->stream));
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (P->stamp_slots < steps + 1) {
        SY_CUDA(cudaFree(P->d_stamps));
        P->d_stamps = nullptr;
        SY_CUDA(cudaMalloc(&P->d_stamps, 4 * sizeof(unsigned long long) * static_cast<size_t>(steps + 1)));
        P->stamp_slots = steps + 1;
    }
    P->expected.assign(static_cast<size_t>(steps + 1), 0);
    const uint64_t launches0 = q->launches;
    q->launch = q->aux;
    cudaError_t e = cudaStreamBeginCapture(q->aux, cudaStreamCaptureModeThreadLocal);
    sy_status st = e == cudaSuccess ? SY_OK : cuda_fail(e, "cudaStreamBeginCapture");
    if (st == SY_OK) {
        e = cudaMemsetAsync(P->d_stamps + 4, 0, 4 * sizeof(unsigned long long) * static_cast<size_t>(steps), q->aux);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
    }
    for (int64_t s = 0; st == SY_OK && s < steps; ++s) st = launch_batch(P, false, static_cast<int>(s & 1), 1 + s);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(q->aux, &graph);
    if (st == SY_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
    q->launch = q->stream;
    P->graph_launches = q->launches - launches0;
    q->launches = launches0;
    if (st == SY_OK) {
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != SY_OK) {
        if (P->exec) cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
        return st;
    }
    P->graph_steps = steps;
    return SY_OK;
}

sy_status sy_stencil_batch_run(sy_batch_plan_t ph) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    if (!P->exec) return fail(SY_ERR_INVALID_ARGUMENT, "no captured run: call sy_stencil_batch_capture first");
    SY_TRY(use_device(P->q));
    SY_CUDA(cudaGraphLaunch(P->exec, P->q->stream));
    P->q->launches += P->graph_launches;
    return SY_OK;
}

sy_status sy_stencil_batch_times(sy_batch_plan_t ph, double* ms, int n) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    if (n < 0 || n > P->stamp_slots) return fail(SY_ERR_INVALID_ARGUMENT, "n = %d not in 0..%lld", n,
                                                 (long long)P->stamp_slots);
    if (n && !ms) return fail(SY_ERR_NULL_POINTER, "ms is NULL");
    SY_TRY(use_device(P->q));
    std::vector<unsigned long long> st(4 * static_cast<size_t>(n));
    if (n) {
        SY_CUDA(cudaMemcpyAsync(st.data(), P->d_stamps, st.size() * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, P->q->aux));
        SY_CUDA(cudaStreamSynchronize(P->q->aux));
    }
    for (int i = 0; i < n; ++i) {
        const unsigned long long* s = &st[4 * static_cast<size_t>(i)];
        if (P->expected[i] == 0) {
            ms[i] = 0.0;
            continue;
        }
        if (s[2] != P->expected[i]) return fail(SY_ERR_NOT_READY, "batch launch %d has not completed", i);
        const unsigned long long start = ~s[0], end = s[1];
        ms[i] = end > start ? static_cast<double>(end - start) * 1e-6 : 0.0;
    }
    return SY_OK;
}

sy_status sy_stencil_batch_destroy(sy_batch_plan_t ph) {
    if (!ph) return SY_OK;
    BatchPlan* P = as_plan(ph);
    cudaSetDevice(P->q->device);
    cudaStreamSynchronize(P->q->stream);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->d_desc) cudaFree(P->d_desc);
    if (P->d_tiles) cudaFree(P->d_tiles);
    if (P->d_stamps) cudaFree(P->d_stamps);
    if (P->d_sync) cudaFree(P->d_sync);
    delete P;
    return SY_OK;
}

sy_status sy_stencil_batch_capture_persistent(sy_batch_plan_t ph, int64_t steps) {
    if (!ph) return fail(SY_ERR_NULL_POINTER, "plan is NULL");
    BatchPlan* P = as_plan(ph);
    if (steps < 1 || steps > (1 << 20)) return fail(SY_ERR_INVALID_ARGUMENT, "steps = %lld", (long long)steps);
    if (P->tile_rows != 0)
        return fail(SY_ERR_INVALID_ARGUMENT, "the cross-step form needs a per-class plan (tile_rows = 0)");
    if (P->classes.size() > 4) return fail(SY_ERR_INVALID_ARGUMENT, "more than 4 radius classes");
    Queue* q = P->q;
    SY_TRY(use_device(q));
    int coop = 0;
    SY_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, q->device));
    if (!coop) return fail(SY_ERR_UNSUPPORTED, "the device does not support cooperative launches");
    PersistFn fn = persist_fn(P->dtype);
    int occ = 0;
    SY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(fn), kBatchThreads, 0));
    if (occ < 1) return fail(SY_ERR_UNSUPPORTED, "the cross-step kernel does not fit on an SM");
    int64_t blocks = static_cast<int64_t>(occ) * q->sm_count;  // every block co-resident
    int64_t most_tiles = 0;
    for (const BatchClass& K : P->classes) most_tiles = K.tiles > most_tiles ? K.tiles : most_tiles;
    const int64_t want = (most_tiles + kBatchThreads / 32 - 1) / (kBatchThreads / 32);
    if (blocks > want) blocks = want < 1 ? 1 : want;
    if (static_cast<uint64_t>(steps) * static_cast<uint64_t>(blocks) >= (1ull << 31))
        return fail(SY_ERR_INVALID_ARGUMENT, "steps x blocks too large for the step barrier's counter");
    SY_CUDA(cudaStreamSynchronize(q->stream));
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (!P->d_sync) SY_CUDA(cudaMalloc(&P->d_sync, 2 * sizeof(unsigned)));
    if (P->stamp_slots < 2) {
        SY_CUDA(cudaFree(P->d_stamps));
        P->d_stamps = nullptr;
        SY_CUDA(cudaMalloc(&P->d_stamps, 4 * sizeof(unsigned long long) * 2));
        P->stamp_slots = 2;
    }
    P->expected.assign(2, 0);
    P->expected[1] = static_cast<uint64_t>(blocks);
    PersistArgs a = {};
    a.grids = P->d_desc;
    a.work = P->d_tiles;
    a.n_cls = static_cast<int>(P->classes.size());
    for (int c = 0; c < a.n_cls; ++c) {
        const BatchClass& K = P->classes[c];
        a.cls[c] = PersistClass{K.desc_off, K.tile_off, K.tiles, K.radius};
    }
    a.steps = steps;
    a.barrier = P->d_sync;
    a.abort = P->d_sync + 1;
    a.err = q->d_flags;
    a.fault = fault_enabled("batch_barrier_timeout") ? 1 : 0;
    a.stamp = P->d_stamps + 4;
    q->launch = q->aux;
    cudaError_t e = cudaStreamBeginCapture(q->aux, cudaStreamCaptureModeThreadLocal);
    sy_status st = e == cudaSuccess ? SY_OK : cuda_fail(e, "cudaStreamBeginCapture");
    if (st == SY_OK) {
        e = cudaMemsetAsync(P->d_stamps + 4, 0, 4 * sizeof(unsigned long long), q->aux);
        if (e == cudaSuccess) e = cudaMemsetAsync(P->d_sync, 0, 2 * sizeof(unsigned), q->aux);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
    }
    if (st == SY_OK) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(blocks));
        cfg.blockDim = dim3(kBatchThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = q->aux;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, fn, a);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaLaunchKernelEx(cooperative)");
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(q->aux, &graph);
    if (st == SY_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
    q->launch = q->stream;
    if (st == SY_OK) {
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != SY_OK) {
        if (P->exec) cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
        return st;
    }
    P->graph_steps = steps;
    P->graph_launches = 1;
    P->persistent_blocks = static_cast<int>(blocks);
    return SY_OK;
}

}  // extern "C"
