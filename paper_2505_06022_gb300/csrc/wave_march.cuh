// Streaming ("march") form of the wave step for 16-bit storage.
//
// A warp owns a strip of 30*V output columns (V = 8 elements a lane) and a segment of
// rows of the chunk, and walks down the segment two rows a step.  The rows arrive in
// shared memory by TMA (cp.async.bulk.tensor.2d, completion counted on one mbarrier
// per ring slot): a step copies two rows of u^n, 32*V columns wide (the strip and V
// columns on each side: lanes 0 and 31 hold the neighbouring columns and store
// nothing), and the two rows of u^{n-1} it writes, the strip only.  kDepth slots per
// warp keep that many steps in flight ahead of the arithmetic.  Points outside the
// grid arrive as zeros (the copy's out-of-bounds fill): those are the Dirichlet
// ghosts, so no lane tests a bound before it reads.
//
// Each lane widens its 8 elements of every u^n row once, into a rolling window of the
// 2r+2 rows around the step's two output rows (FP32, in registers; the loop is
// unrolled over a whole turn of the window so that every window slot is a
// compile-time register): the vertical neighbours come from the window, the
// horizontal ones from the adjacent lanes by shuffles.  Against the register-tile
// kernel this reads the r halo rows above and below a tile once per segment instead
// of once per tile, and widens every element once instead of once per use.  Measured
// slower than the tiles all the same (more control instructions per row and a
// dependency chain along the walk); it is kept as a tuner candidate.
//
// Arithmetic: the canonical operation order of the tile kernel (update2 with packed
// additions and packed products), so results are bit-identical to it.
//
// Bounded waits: a wait on a slot gives up after ~1 s (tma::kWaitCycles); the warp
// then sets the queue's error flag, waits (again bounded) for the copies it still has
// in flight, and stops; every warp still reaches the block's final barrier.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "tma.cuh"
#include "wave_kernel.cuh"

namespace sy {
namespace wave {
namespace march {

constexpr int kWarps = 4;                // warps per block, each marching its own strip
constexpr int kThreads = 32 * kWarps;
constexpr int kRowsPerStep = 2;          // rows a step copies and computes (one wait, one vote)
constexpr int kDepth = 4;                // ring slots per warp: kDepth * kRowsPerStep rows in flight
constexpr int kRowBytes = 512;           // one u^n row copy (32 x 8 elements); a u^{n-1} row takes 480
constexpr int kSlot = 2 * kRowsPerStep * kRowBytes;  // u^n rows, then u^{n-1} rows
constexpr int kPrevOff = kRowsPerStep * kRowBytes;
constexpr int kMinSegment = 8;           // rows; the segment length is otherwise chosen per launch

template <typename S>
struct Geo {
    static_assert(sizeof(S) == 2, "the march form is for 16-bit storage");
    static constexpr int V = 8;                              // elements a lane (16 bytes)
    static constexpr int SPAN = 32 * V;                      // columns of a u^n row copy
    static constexpr int OUT = 30 * V;                       // output columns of a strip
    static constexpr unsigned CUR_TX = SPAN * sizeof(S);     // 512 bytes
    static constexpr unsigned PREV_TX = OUT * sizeof(S);     // 480 bytes
    static constexpr int SMEM = kWarps * kDepth * (kSlot + 8);
    static_assert(CUR_TX == kRowBytes && PREV_TX <= kRowBytes, "slot layout");
};

struct MArgs {
    char* u_next;
    int64_t ny, nx, pitch_bytes;
    int64_t row_begin, row_end;
    int64_t strips;  // strips of 30*V output columns
    int64_t seg;     // rows per segment
    int64_t tasks;   // strips x segments, segment-major
    float c2;
    float neg0;                  // -0.0f (see mul2_rn)
    unsigned int* err;           // error flags (bit 0: a wait timed out)
    unsigned long long* stamp;   // timestamp slot or null
    int fault;                   // host-injected fault for tests: 1 = never issue the first copy
    int pdl;                     // as in Args
};

// Blocks an SM the kernel is compiled for: the window is (2r+2) x 8 FP32 registers a
// lane, so radius 3-4 gets 168 registers (3 blocks), radius 1-2 128 (4 blocks).
template <int R>
struct MinBlocks {
    static constexpr int value = R >= 3 ? 3 : 4;
};

// Unroll period (in steps) of the window: the smallest P with P * G a multiple of the
// window's 2r + G rows, so that every window slot is a compile-time register.
template <int R, int G>
struct Period {
    static constexpr int WN = 2 * R + G;
    static constexpr int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }
    static constexpr int value = WN / gcd(G, WN);
};

template <typename S, int R, bool START, bool REV>
__global__ void __launch_bounds__(kThreads, MinBlocks<R>::value)
    wave_march_kernel(const __grid_constant__ CUtensorMap map_cur, const __grid_constant__ CUtensorMap map_prev,
                      MArgs a) {
    using Ge = Geo<S>;
    using Tr = Traits<S>;
    constexpr int V = Ge::V;
    constexpr int G = kRowsPerStep;
    constexpr int WN = 2 * R + G;            // window rows: the step's G output rows and r each side
    constexpr int P = Period<R, G>::value;   // steps per unroll period
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* ring = smem + warp * kDepth * kSlot;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kWarps * kDepth * kSlot) + warp * kDepth;

    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    if (lane == 0) {
        for (int s = 0; s < kDepth; ++s) tma::mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kWarps;
    uint32_t n = 0;  // ring position: steps this warp has consumed
    bool ok = true;
    bool first_copy = true;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * kWarps + warp; t < a.tasks && ok; t += nwarps) {
        const int64_t tt = REV ? a.tasks - 1 - t : t;
        const int64_t sg = tt / a.strips, tx = tt - sg * a.strips;
        const int64_t y0 = a.row_begin + sg * a.seg;
        const int rows = static_cast<int>((y0 + a.seg < a.row_end ? y0 + a.seg : a.row_end) - y0);
        // u^n rows y0 - r + m for m < rows + 2r, G a step: step s copies m = sG .. sG + G - 1
        // and computes the output rows o = sG - 2r + g (g < G) that lie in [0, rows)
        const int steps = (rows + 2 * R + G - 1) / G;
        const int xo = static_cast<int>(tx * Ge::OUT);        // first output column (lane 1's)
        const int xs = xo - V;                                 // first copied column (lane 0's)
        // lane 0: the copies of step s into the slot of ring position n + s (only rows that
        // the chunk's range mapper reads: u^n rows below y0 + rows + r are not copied)
        auto issue = [&](int s) {
            const uint32_t k = n + static_cast<uint32_t>(s);
            unsigned char* slot = ring + (k % kDepth) * kSlot;
            uint64_t* bar = &bars[k % kDepth];
            int ncur = rows + 2 * R - s * G;
            ncur = ncur < G ? ncur : G;
            int o0 = s * G - 2 * R, nprev = 0;  // output rows of the step: [o0, o0 + G) within [0, rows)
            if (!START) {
                const int lo = o0 > 0 ? o0 : 0, hi = o0 + G < rows ? o0 + G : rows;
                nprev = hi > lo ? hi - lo : 0;
                o0 = lo;
            }
            tma::fence_proxy_async();  // this slot's earlier reads, ordered by __syncwarp, come first
            tma::mbar_expect_tx(bar, ncur * Ge::CUR_TX + nprev * Ge::PREV_TX);
            if (first_copy && a.fault == 1) {
                first_copy = false;  // never issued: the wait on this slot runs out
                return;
            }
            first_copy = false;
            for (int g = 0; g < ncur; ++g)
                tma::load_2d(slot + g * kRowBytes, &map_cur, xs, static_cast<int>(y0 - R + s * G + g), bar);
            // u^{n-1} row o goes to prev slot position o - (sG - 2r)
            for (int g = 0; g < nprev; ++g)
                tma::load_2d(slot + kPrevOff + (o0 + g - (s * G - 2 * R)) * kRowBytes, &map_prev, xo,
                             static_cast<int>(y0 + o0 + g), bar);
        };
        if (lane == 0) {
            const int first = steps < kDepth ? steps : kDepth;
            for (int s = 0; s < first; ++s) issue(s);
        }
        const int64_t out_x = static_cast<int64_t>(xo) + static_cast<int64_t>(lane - 1) * V;
        const bool out_lane = lane >= 1 && lane <= 30 && out_x < a.nx;
        const int nvalid = out_lane ? static_cast<int>(a.nx - out_x < V ? a.nx - out_x : V) : 0;
        // row y0 of the lane's columns (lanes that store nothing keep the row start)
        char* out_row = a.u_next + y0 * a.pitch_bytes + (out_lane ? out_x * static_cast<int64_t>(sizeof(S)) : 0);
        float win[WN][V];  // win[m % WN] = u^n row y0 - r + m, widened
        int failed = -1;
        for (int sb = 0; sb < steps && failed < 0; sb += P) {
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int s = sb + j;
                if (s >= steps) break;
                const uint32_t k = n + static_cast<uint32_t>(s);
                const unsigned char* slot = ring + (k % kDepth) * kSlot;
                const bool got = tma::mbar_wait_bounded(&bars[k % kDepth], (k / kDepth) & 1u);
                if (!__all_sync(kFull, got)) {
                    failed = s;
                    break;
                }
                uint4 c[G], pv[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    c[g] = *reinterpret_cast<const uint4*>(slot + g * kRowBytes + lane * 16);
                    pv[g] = make_uint4(0u, 0u, 0u, 0u);
                    if (!START && out_lane && s * G - 2 * R + g >= 0)
                        pv[g] = *reinterpret_cast<const uint4*>(slot + kPrevOff + g * kRowBytes + (lane - 1) * 16);
                }
                __syncwarp();  // every lane has read the slot
                if (lane == 0 && s + kDepth < steps) issue(s + kDepth);
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < V; ++e) win[(j * G + g) % WN][e] = Tr::elem(c[g], e);
                if (s * G + G - 1 < 2 * R) continue;  // window warm-up: no output row complete yet
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int o = s * G - 2 * R + g;  // output row (relative to y0)
                    // centre row m = o + r, in window slot (j G + g - r) mod WN
                    const float(&cen)[V] = win[(j * G + g - R + 2 * WN) % WN];
                    float ext[V + 2 * R];  // columns out_x - r .. out_x + V + r - 1
#pragma unroll
                    for (int e = 0; e < V; ++e) ext[R + e] = cen[e];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        ext[R - d] = __shfl_up_sync(kFull, cen[V - d], 1);
                        ext[R + V - 1 + d] = __shfl_down_sync(kFull, cen[d - 1], 1);
                    }
                    float out[V];
#pragma unroll
                    for (int e = 0; e < V; e += 2) {
                        float2 vert[R], horz[R];
#pragma unroll
                        for (int d = 1; d <= R; ++d) {
                            const float(&up_row)[V] = win[(j * G + g - R - d + 2 * WN) % WN];
                            const float(&dn_row)[V] = win[(j * G + g - R + d + 2 * WN) % WN];
                            vert[d - 1] = add2_rn(make_float2(up_row[e], up_row[e + 1]),
                                                  make_float2(dn_row[e], dn_row[e + 1]));
                            horz[d - 1] = horz2<R>(ext, e, d);
                        }
                        const float2 upv =
                            START ? make_float2(0.0f, 0.0f) : make_float2(Tr::elem(pv[g], e), Tr::elem(pv[g], e + 1));
                        const float2 r2 =
                            update2<R, START, true>(make_float2(cen[e], cen[e + 1]), upv, vert, horz, a.c2, a.neg0);
                        out[e] = r2.x;
                        out[e + 1] = r2.y;
                    }
                    if (out_lane && o >= 0 && o < rows) {
                        char* dst = out_row + static_cast<int64_t>(o) * a.pitch_bytes;
                        if (nvalid == V) {
                            Vec16::st_cs(dst, Tr::pack(out));
                        } else {
#pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (e < nvalid) Tr::store1(dst + e * static_cast<int64_t>(sizeof(S)), out[e]);
                        }
                    }
                }
            }
        }
        if (failed >= 0) {
            // let this warp's copies still in flight land before its shared memory is released
            if (lane == 0) {
                atomicOr(a.err, 1u);
                const int last = failed + kDepth < steps ? failed + kDepth : steps;  // steps issued
                for (int s = failed; s < last; ++s) {
                    const uint32_t k = n + static_cast<uint32_t>(s);
                    tma::mbar_wait_bounded(&bars[k % kDepth], (k / kDepth) & 1u);
                }
            }
            __syncwarp();
            ok = false;
        }
        n += static_cast<uint32_t>(steps);
    }
    stamp_end(a.stamp);
    if (a.pdl && threadIdx.x == 0) griddep_wait();
}

// ---- host ----------------------------------------------------------------------
template <typename S>
sy_status make_row_map(const void* base, int64_t ny, int64_t nx, int64_t pitch_bytes, int box_cols, CUtensorMap* map) {
    auto enc = tma::encoder();
    if (!enc) return fail(SY_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch_bytes)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), 1u};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SY_ERR_INVALID_ARGUMENT, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return SY_OK;
}

template <typename S, int R, bool START, bool REV>
sy_status launch_march_k(Queue* q, const WaveLaunch& w) {
    using Ge = Geo<S>;
    auto kern = wave_march_kernel<S, R, START, REV>;
    static std::once_flag once;
    static int occ = 0;
    static cudaError_t occ_err = cudaSuccess;
    std::call_once(once, [&] {
        occ_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Ge::SMEM);
        if (occ_err == cudaSuccess)
            occ_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, Ge::SMEM);
    });
    if (occ_err != cudaSuccess) return cuda_fail(occ_err, "march kernel attributes");
    if (occ < 1) return fail(SY_ERR_UNSUPPORTED, "the march kernel does not fit on an SM");
    const int64_t rows = w.row_end - w.row_begin;
    const int64_t pb = w.pitch * static_cast<int64_t>(sizeof(S));
    CUtensorMap mc, mp;
    SY_TRY(make_row_map<S>(w.u_cur, w.ny, w.nx, pb, Ge::SPAN, &mc));
    if (START) mp = mc;
    else SY_TRY(make_row_map<S>(w.u_prev, w.ny, w.nx, pb, Ge::OUT, &mp));
    MArgs a;
    a.u_next = static_cast<char*>(w.u_next);
    a.ny = w.ny;
    a.nx = w.nx;
    a.pitch_bytes = pb;
    a.row_begin = w.row_begin;
    a.row_end = w.row_end;
    a.strips = (w.nx + Ge::OUT - 1) / Ge::OUT;
    // one segment per resident warp where the chunk allows: segments of equal length,
    // as many per strip as the grid's warps divided among the strips
    const int64_t warps = static_cast<int64_t>(occ) * q->sm_count * kWarps;
    int64_t per_strip = warps / a.strips;
    if (per_strip < 1) per_strip = 1;
    int64_t seg = (rows + per_strip - 1) / per_strip;
    if (seg < kMinSegment) seg = kMinSegment;
    a.seg = seg;
    a.tasks = a.strips * ((rows + seg - 1) / seg);
    a.c2 = w.c2;
    a.neg0 = -0.0f;
    a.err = q->d_flags;
    a.stamp = q->cur_stamp;
    a.fault = fault_enabled("march_timeout") ? 1 : 0;
    a.pdl = 0;
    int64_t blocks = (a.tasks + kWarps - 1) / kWarps;
    const int64_t cap = static_cast<int64_t>(occ) * q->sm_count;
    if (blocks > cap) blocks = cap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = Ge::SMEM;
    cfg.stream = q->launch;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (w.pdl && launch_overlap_enabled()) {
        a.pdl = w.pdl;
        cfg.numAttrs = 1;
    }
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mc, mp, a);
    if (e != cudaSuccess)
        return fail(SY_ERR_CUDA, "march kernel (%lld blocks x %d threads, %lld-row segments): %s",
                    static_cast<long long>(blocks), kThreads, static_cast<long long>(seg), cudaGetErrorString(e));
    ++q->launches;
    q->cur_blocks += static_cast<uint64_t>(blocks);
    return SY_OK;
}

template <typename S, int R>
sy_status launch_march_r(Queue* q, const WaveLaunch& w) {
    if (w.start) return launch_march_k<S, R, true, false>(q, w);
    return w.reverse ? launch_march_k<S, R, false, true>(q, w) : launch_march_k<S, R, false, false>(q, w);
}

// Layouts whose rows are not 16-byte aligned, and fields of 2^31 rows or columns or
// more, go to the tile kernel's launcher (which takes the scalar kernel for the
// unaligned ones).
template <typename S>
sy_status launch_march(Queue* q, const WaveLaunch& w) {
    if (w.row_end <= w.row_begin || w.nx == 0) return SY_OK;
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec_ok = a16(w.u_cur) && a16(w.u_next) && (w.start || a16(w.u_prev)) &&
                        (w.pitch * static_cast<int64_t>(sizeof(S))) % 16 == 0;
    // TMA coordinates are 32-bit: taller or wider fields take the tile kernel too
    const bool coords_ok = w.ny + 64 < (int64_t{1} << 31) && w.nx + 64 < (int64_t{1} << 31);
    if (!vec_ok || !coords_ok) return launch_dtype<S>(q, w, 4, 128, Form::Tile);
    switch (w.radius) {
        case 1: return launch_march_r<S, 1>(q, w);
        case 2: return launch_march_r<S, 2>(q, w);
        case 3: return launch_march_r<S, 3>(q, w);
        default: return launch_march_r<S, 4>(q, w);
    }
}

}  // namespace march
}  // namespace wave
}  // namespace sy
