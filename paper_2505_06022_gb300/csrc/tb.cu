// Temporal blocking: T leapfrog steps per pass over HBM.
//
// A block owns a tile of BY x BX output points of a row chunk.  TMA
// (cp.async.bulk.tensor.2d, completion counted on an mbarrier) copies the
// tile's u^n and u^{n-1} with a halo of T*r rows and PAD >= T*r columns into
// shared memory; points outside the grid arrive as zeros (the copy's
// out-of-bounds fill), which are the Dirichlet ghosts.  The block then advances
// T steps in shared memory over shrinking regions -- step k computes u^{n+k}
// on the tile grown by (T-k)*r, recomputing the halo instead of re-reading it
// from HBM -- and writes u^{n+T-1} and u^{n+T} for the tile.  HBM traffic is two
// reads and two writes per point per pass: 16/T bytes per FP32 update instead
// of 12.  Every point is computed with the single-step operation order and
// rounded to storage after every step, so results are bit-identical to T calls
// of the single-step kernel.
//
// Blocks are persistent, several per SM: while one block computes, the copies
// of the others' next tiles are in flight (each block issues its next tile's
// copies as soon as it has written its current one; kStages = 2 would instead
// double-buffer within a block).  Every wait on an mbarrier is bounded by a clock limit; on
// expiry the block sets an error flag, waits (again bounded) for its own
// copies in flight, and returns; the host reports SY_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "tma.cuh"
#include "wave_kernel.cuh"

namespace sy {
namespace tb {

constexpr int kThreads = 256;  // 8 warps: one row-lane each
constexpr int BY = 32;
// Tiles in shared memory per block.  With 2 the next tile's copy overlaps the
// block's own compute; with 1 the block's footprint halves and 2.5x as many
// blocks fit an SM, whose computing blocks hide the others' copies -- measured
// faster (T = 4: 9.8e11 -> 1.13e12 updates/s FP32, 1.20e12 -> 1.34e12 BF16).
constexpr int kStages = 1;

struct TBArgs {
    char* out_prev;  // u^{n+T-1}
    char* out_cur;   // u^{n+T}
    int64_t ny, nx, pitch_bytes;
    int64_t row_begin, row_end;
    int64_t tiles_x, tiles;
    float c2;
    unsigned int* err;           // error flags (bit 0: a wait timed out)
    unsigned long long* stamp;   // timestamp slot or null
    int fault;                   // host-injected fault for tests: 1 = never issue the first copy
    int pdl;                     // as in wave::Args
    float neg0;                  // -0.0f, set by the host: the packed products' addend (wave::mul2_rn)
};

template <typename S, int R, int T>
struct Geo {
    static constexpr int ES = sizeof(S);
    static constexpr int VEC = 16 / ES;                                     // elements per 16 bytes
    static constexpr int PAD = ((T * R + VEC - 1) / VEC) * VEC;             // 16-byte aligned x halo
    static constexpr int W = 32 * VEC;                                      // box / row width: one warp's span
    static constexpr int BX = W - 2 * PAD;                                  // output columns of a tile
    static constexpr int H = BY + 2 * T * R;                                // box height
    static constexpr int BUF = ((W * H * ES + 127) / 128) * 128;            // one field, 128-byte aligned
    static constexpr int SMEM = 2 * kStages * BUF + 2 * 8;                  // stages x 2 fields + 2 barriers
    static constexpr unsigned TX = 2u * W * H * ES;                         // bytes a stage receives
    static_assert(BX > 0 && BX % VEC == 0, "tile width");
};

using tma::kWaitCycles;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait_bounded;

template <typename S>
__device__ __forceinline__ float ld_s(const S* buf, int idx);
template <>
__device__ __forceinline__ float ld_s<float>(const float* buf, int idx) { return buf[idx]; }
template <>
__device__ __forceinline__ float ld_s<__nv_bfloat16>(const __nv_bfloat16* buf, int idx) {
    return __uint_as_float(static_cast<uint32_t>(__bfloat16_as_ushort(buf[idx])) << 16);
}
template <>
__device__ __forceinline__ float ld_s<__half>(const __half* buf, int idx) { return __half2float(buf[idx]); }

template <typename S>
__device__ __forceinline__ S to_s(float v);
template <>
__device__ __forceinline__ float to_s<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_s<__half>(float v) { return __float2half_rn(v); }

// One step over buffer rows [k*R, H - k*R) and every column of the W-wide
// buffers: X holds u^m, Y holds u^{m-1} and receives u^{m+1}.  A row is exactly
// one warp wide: lane g owns the 16-byte column group g, and each warp owns a
// contiguous run of rows; the 2R+1 rows of its group around the current row
// stay in registers (a rolling window), and the horizontal neighbours come from
// lanes g-1 and g+1 by shuffles (zeros beyond the buffer's outer columns).  Results
// in the outer PAD columns are computed from partial neighbourhoods, but the
// needed region of step k, [PAD - (T-k)R, PAD + BX + (T-k)R), lies inside
// [k R, W - k R) where every value is exact (PAD >= T R).  Points outside the grid
// are set to zero (interior tiles skip the test).
// The 16-bit rows of tb_step: the same walk, but the window holds the 2R+1 rows
// widened to FP32 (each element widened once, when its row enters the window,
// instead of once per use), and the products as well as the additions are paired.
template <typename S, int R>
__device__ __forceinline__ void tb_rows16(const uint4* X, uint4* Y, int r0, int r1, int y_buf0, int x_buf0,
                                          bool interior, int64_t ny, int64_t nx, float c2, float neg0) {
    using Tr = wave::Traits<S>;
    constexpr int V = Tr::V;
    constexpr int NG = 32;
    constexpr int W = 2 * R + 1;
    const int g = threadIdx.x & 31;
    float win[W][V];  // win[i % W] = row r0 - R + i, widened
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) {
        const uint4 v = X[(r0 - R + d) * NG + g];
#pragma unroll
        for (int e = 0; e < V; ++e) win[d][e] = Tr::elem(v, e);
    }
    const uint4* xrow = X + (r0 + R) * NG + g;  // row r + R of group g
    const uint4* yrow = Y + r0 * NG + g;
    uint4* orow = Y + r0 * NG + g;
    for (int rb = r0; rb < r1; rb += W) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int r = rb + j;
            if (r >= r1) break;
            {
                const uint4 v = xrow[(r - r0) * NG];
#pragma unroll
                for (int e = 0; e < V; ++e) win[(j + 2 * R) % W][e] = Tr::elem(v, e);
            }
            const uint4 pv = yrow[(r - r0) * NG];
            const float(&cen)[V] = win[(j + R) % W];
            float ext[V + 2 * R];  // columns g*V - R .. g*V + V + R - 1
#pragma unroll
            for (int e = 0; e < V; ++e) ext[R + e] = cen[e];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const float from_left = __shfl_up_sync(wave::kFull, cen[V - d], 1);
                const float from_right = __shfl_down_sync(wave::kFull, cen[d - 1], 1);
                ext[R - d] = g == 0 ? 0.0f : from_left;
                ext[R + V - 1 + d] = g == 31 ? 0.0f : from_right;
            }
            float out[V];
#pragma unroll
            for (int e = 0; e < V; e += 2) {
                float2 vert[R], horz[R];
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    const float(&wu)[V] = win[(j + R - d) % W];
                    const float(&wd)[V] = win[(j + R + d) % W];
                    vert[d - 1] = wave::add2_rn(make_float2(wu[e], wu[e + 1]), make_float2(wd[e], wd[e + 1]));
                    horz[d - 1] = wave::horz2<R>(ext, e, d);
                }
                const float2 o = wave::update2<R, false, true>(make_float2(cen[e], cen[e + 1]),
                                                               make_float2(Tr::elem(pv, e), Tr::elem(pv, e + 1)), vert,
                                                               horz, c2, neg0);
                out[e] = o.x;
                out[e + 1] = o.y;
            }
            if (!interior) {  // ghosts outside the grid stay zero
                const int64_t gy = static_cast<int64_t>(y_buf0) + r;
                const bool row_in = gy >= 0 && gy < ny;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const int64_t gx = static_cast<int64_t>(x_buf0) + g * V + e;
                    if (!row_in || gx < 0 || gx >= nx) out[e] = 0.0f;
                }
            }
            orow[(r - r0) * NG] = Tr::pack(out);
        }
    }
}

template <typename S, int R, int T>
__device__ __forceinline__ void tb_step(const uint4* X, uint4* Y, int k, int y_buf0, int x_buf0, bool interior,
                                        int64_t ny, int64_t nx, float c2, float neg0) {
    using G = Geo<S, R, T>;
    using Tr = wave::Traits<S>;
    constexpr int V = Tr::V;
    constexpr int NG = 32;                     // 16-byte groups per row = lanes
    constexpr int NRL = kThreads / 32;         // row lanes = warps
    const int g = threadIdx.x & 31, rl = threadIdx.x >> 5;
    const int r_lo = k * R, r_hi = G::H - k * R;
    const int per = (r_hi - r_lo + NRL - 1) / NRL;
    const int r0 = r_lo + rl * per;
    const int r1 = r0 + per < r_hi ? r0 + per : r_hi;
    if (r0 >= r1) return;  // warp-uniform
    if constexpr (sizeof(S) == 2) {
        tb_rows16<S, R>(X, Y, r0, r1, y_buf0, x_buf0, interior, ny, nx, c2, neg0);
        return;
    }
    // rolling window of the 2R+1 rows around the current one: row r0 - R + i lives in
    // win[i % W]; the loop is unrolled by W rows so that every slot index is a
    // compile-time constant and the window moves without register copies
    constexpr int W = 2 * R + 1;
    uint4 win[W];
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) win[d] = X[(r0 - R + d) * NG + g];
    const uint4* xrow = X + (r0 + R) * NG + g;  // row r + R of group g
    const uint4* yrow = Y + r0 * NG + g;
    uint4* orow = Y + r0 * NG + g;
    for (int rb = r0; rb < r1; rb += W) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int r = rb + j;
            if (r >= r1) break;
            win[(j + 2 * R) % W] = xrow[(r - r0) * NG];
            const uint4 pv = yrow[(r - r0) * NG];
            const uint4& cen = win[(j + R) % W];
            float ext[V + 2 * R];  // columns g*V - R .. g*V + V + R - 1
#pragma unroll
            for (int e = 0; e < V; ++e) ext[R + e] = Tr::elem(cen, e);
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const float from_left = __shfl_up_sync(wave::kFull, ext[R + V - d], 1);
                const float from_right = __shfl_down_sync(wave::kFull, ext[R + d - 1], 1);
                ext[R - d] = g == 0 ? 0.0f : from_left;
                ext[R + V - 1 + d] = g == 31 ? 0.0f : from_right;
            }
            float out[V];
            if constexpr (sizeof(S) == 2) {  // 16-bit storage: pair the additions and the products
#pragma unroll
                for (int e = 0; e < V; e += 2) {
                    float2 vert[R], horz[R];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        const uint4& wu = win[(j + R - d) % W];
                        const uint4& wd = win[(j + R + d) % W];
                        vert[d - 1] = wave::add2_rn(make_float2(Tr::elem(wu, e), Tr::elem(wu, e + 1)),
                                                    make_float2(Tr::elem(wd, e), Tr::elem(wd, e + 1)));
                        horz[d - 1] = wave::horz2<R>(ext, e, d);
                    }
                    const float2 o = wave::update2<R, false, true>(make_float2(ext[R + e], ext[R + e + 1]),
                                                                   make_float2(Tr::elem(pv, e), Tr::elem(pv, e + 1)),
                                                                   vert, horz, c2, neg0);
                    out[e] = o.x;
                    out[e + 1] = o.y;
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    float vert[R], horz[R];
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        vert[d - 1] = __fadd_rn(Tr::elem(win[(j + R - d) % W], e), Tr::elem(win[(j + R + d) % W], e));
                        horz[d - 1] = __fadd_rn(ext[R + e - d], ext[R + e + d]);
                    }
                    out[e] = wave::update<R, false>(ext[R + e], Tr::elem(pv, e), vert, horz, c2);
                }
            }
            if (!interior) {  // ghosts outside the grid stay zero
                const int64_t gy = static_cast<int64_t>(y_buf0) + r;
                const bool row_in = gy >= 0 && gy < ny;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const int64_t gx = static_cast<int64_t>(x_buf0) + g * V + e;
                    if (!row_in || gx < 0 || gx >= nx) out[e] = 0.0f;
                }
            }
            orow[(r - r0) * NG] = Tr::pack(out);
        }
    }
}

// Blocks an SM the kernel is compiled for (its register budget): a tile's shared
// memory admits 5 blocks at radius 1 and 3-4 at radius 2, and the unrolled row window
// would otherwise take a few registers more than 4 (radius 1) or 3 (radius 2) blocks
// leave, which cost 16-bit radius-1 passes a quarter of their resident warps.
template <int R>
struct TbMinBlocks {
    static constexpr int value = R == 1 ? 4 : (R == 2 ? 3 : 2);
};

template <typename S, int R, int T>
__global__ void __launch_bounds__(kThreads, TbMinBlocks<R>::value) wave_tb_kernel(const __grid_constant__ CUtensorMap map_prev,
                                                           const __grid_constant__ CUtensorMap map_cur, TBArgs a) {
    using G = Geo<S, R, T>;
    using Tr = wave::Traits<S>;
    constexpr int V = Tr::V;
    constexpr int NG = G::W / V;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kStages * G::BUF);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kThreads / 32;

    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // copies of tile t into stage s: u^n box into field 0, u^{n-1} box into field 1
    auto issue = [&](int64_t t, int s, bool skip) {
        const int64_t ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
        const int x = static_cast<int>(tx * G::BX) - G::PAD;
        const int y = static_cast<int>(a.row_begin + ty * BY) - T * R;
        unsigned char* base = smem + 2 * s * G::BUF;
        tma::fence_proxy_async();  // earlier generic writes to this stage
        mbar_expect_tx(&bars[s], G::TX);
        if (!skip) {
            tma::load_2d(base, &map_cur, x, y, &bars[s]);
            tma::load_2d(base + G::BUF, &map_prev, x, y, &bars[s]);
        }
    };

    int64_t t = blockIdx.x;
    unsigned uses0 = 0u, uses1 = 0u;
    if (t < a.tiles && tid == 0) issue(t, 0, a.fault == 1);
    for (int it = 0; t < a.tiles; ++it, t += gridDim.x) {
        const int s = kStages == 2 ? (it & 1) : 0;
        const int64_t tn = t + gridDim.x;
        if (kStages == 2 && tn < a.tiles && tid == 0) issue(tn, s ^ 1, false);
        const unsigned par = (s ? uses1 : uses0) & 1u;
        // every thread waits (acquiring the copied data); the block decides together
        const bool ok = mbar_wait_bounded(&bars[s], par);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(a.err, 1u);
                // let this block's own copies land before its shared memory is released
                mbar_wait_bounded(&bars[s], par);
                if (kStages == 2 && tn < a.tiles) mbar_wait_bounded(&bars[s ^ 1], (s ? uses0 : uses1) & 1u);
            }
            return;  // the whole block returns: no barrier below is left half-reached
        }
        if (s) ++uses1;
        else ++uses0;
        uint4* X = reinterpret_cast<uint4*>(smem + 2 * s * G::BUF);  // u^{m}
        uint4* Y = reinterpret_cast<uint4*>(smem + 2 * s * G::BUF + G::BUF);  // u^{m-1} -> u^{m+1}
        const int64_t ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
        const int64_t y0 = a.row_begin + ty * BY, x0 = tx * G::BX;
        const int y_buf0 = static_cast<int>(y0) - T * R;  // global row of buffer row 0
        const int x_buf0 = static_cast<int>(x0) - G::PAD;  // global column of buffer column 0
        const bool interior = y_buf0 >= 0 && y_buf0 + G::H <= a.ny && x_buf0 >= 0 && x_buf0 + G::W <= a.nx;

#pragma unroll 1
        for (int k = 1; k <= T; ++k) {
            tb_step<S, R, T>(X, Y, k, y_buf0, x_buf0, interior, a.ny, a.nx, a.c2, a.neg0);
            __syncthreads();
            uint4* tmp = X;  // u^{m+1} is now in Y
            X = Y;
            Y = tmp;
        }
        // X = u^{n+T} and Y = u^{n+T-1} on the tile: write the tile's rows of the chunk,
        // one 16-byte group per thread (element stores at the right edge of the grid)
        constexpr int TG = G::BX / V;  // groups per tile row
        for (int idx = tid; idx < BY * TG; idx += kThreads) {
            const int i = idx / TG, gg = idx - i * TG;
            const int64_t gy = y0 + i;
            const int64_t gx = x0 + static_cast<int64_t>(gg) * V;
            if (gy >= a.row_end || gx >= a.nx) continue;
            const int bidx = (T * R + i) * NG + G::PAD / V + gg;
            char* oc = a.out_cur + gy * a.pitch_bytes + gx * G::ES;
            char* op = a.out_prev + gy * a.pitch_bytes + gx * G::ES;
            if (gx + V <= a.nx) {
                *reinterpret_cast<uint4*>(oc) = X[bidx];
                *reinterpret_cast<uint4*>(op) = Y[bidx];
            } else {
                const S* xs = reinterpret_cast<const S*>(&X[bidx]);
                const S* ys = reinterpret_cast<const S*>(&Y[bidx]);
                for (int e = 0; e < V && gx + e < a.nx; ++e) {
                    reinterpret_cast<S*>(oc)[e] = xs[e];
                    reinterpret_cast<S*>(op)[e] = ys[e];
                }
            }
        }
        (void)lane;
        (void)warp;
        (void)kWarps;
        __syncthreads();  // the stage is free for the next copy into it
        if (kStages == 1 && tn < a.tiles && tid == 0) issue(tn, 0, false);
    }
    stamp_end(a.stamp);
    if (a.pdl && tid == 0) griddep_wait();
}

// ---- host ----------------------------------------------------------------------
template <typename S, int R, int T>
sy_status make_map(const void* base, int64_t ny, int64_t nx, int64_t pitch_bytes, CUtensorMap* map) {
    using G = Geo<S, R, T>;
    auto enc = tma::encoder();
    if (!enc) return fail(SY_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    const CUtensorMapDataType dt = sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch_bytes)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(G::W), static_cast<cuuint32_t>(G::H)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SY_ERR_INVALID_ARGUMENT, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return SY_OK;
}

template <typename S, int R, int T>
sy_status launch_tb(Queue* q, const TBLaunch& w) {
    using G = Geo<S, R, T>;
    // the tile copies' coordinates are 32-bit
    if (w.ny + BY + 2 * T * R >= (int64_t{1} << 31) || w.nx + G::W >= (int64_t{1} << 31))
        return fail(SY_ERR_UNSUPPORTED, "temporal blocking supports fields of fewer than 2^31 rows and columns");
    auto kern = wave_tb_kernel<S, R, T>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(tb smem)");
    CUtensorMap mp, mc;
    sy_status st = make_map<S, R, T>(w.u_prev, w.ny, w.nx, w.pitch_bytes, &mp);
    if (st == SY_OK) st = make_map<S, R, T>(w.u_cur, w.ny, w.nx, w.pitch_bytes, &mc);
    if (st != SY_OK) return st;
    TBArgs a;
    a.out_prev = static_cast<char*>(w.out_prev);
    a.out_cur = static_cast<char*>(w.out_cur);
    a.ny = w.ny;
    a.nx = w.nx;
    a.pitch_bytes = w.pitch_bytes;
    a.row_begin = w.row_begin;
    a.row_end = w.row_end;
    a.tiles_x = (w.nx + G::BX - 1) / G::BX;
    a.tiles = a.tiles_x * ((w.row_end - w.row_begin + BY - 1) / BY);
    a.c2 = w.c2;
    a.err = q->d_flags;
    a.stamp = q->cur_stamp;
    a.fault = w.fault;
    a.pdl = w.pdl;
    a.neg0 = -0.0f;
    if (a.tiles == 0) return SY_OK;
    int occ = 0;
    SY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, G::SMEM));
    if (occ < 1) return fail(SY_ERR_UNSUPPORTED, "temporal-blocking kernel does not fit on an SM");
    int64_t blocks = static_cast<int64_t>(occ) * q->sm_count;
    if (blocks > a.tiles) blocks = a.tiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = q->launch;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = w.pdl ? 1 : 0;
    SY_CUDA(cudaLaunchKernelEx(&cfg, kern, mp, mc, a));
    ++q->launches;
    q->cur_blocks += static_cast<uint64_t>(blocks);
    return SY_OK;
}

template <typename S, int T>
sy_status launch_r(Queue* q, const TBLaunch& w) {
    switch (w.radius) {
        case 1: return launch_tb<S, 1, T>(q, w);
        case 2: return launch_tb<S, 2, T>(q, w);
        case 3: return launch_tb<S, 3, T>(q, w);
        case 4: return launch_tb<S, 4, T>(q, w);
        default: return fail(SY_ERR_UNSUPPORTED, "temporal blocking supports radius 1 to 4 (asked %d)", w.radius);
    }
}

template <typename S>
sy_status launch_T(Queue* q, const TBLaunch& w) {
    switch (w.T) {
        case 2: return launch_r<S, 2>(q, w);
        case 4: return launch_r<S, 4>(q, w);
        default: return fail(SY_ERR_UNSUPPORTED, "temporal blocking supports T = 2 and 4 (asked %d)", w.T);
    }
}

}  // namespace tb

sy_status launch_tb(Queue* q, const TBLaunch& w) {
    switch (w.dtype) {
        case SY_F32: return tb::launch_T<float>(q, w);
        case SY_BF16: return tb::launch_T<__nv_bfloat16>(q, w);
        default: return tb::launch_T<__half>(q, w);
    }
}

}  // namespace sy
