// Leapfrog wave step on a 3D grid (radius-r star stencil, Dirichlet-zero ghosts)
// for one chunk of planes of a field laid out plane by plane, row by row.
// Included by wave3d_f32.cu, wave3d_bf16.cu and wave3d_f16.cu.
//
//   L u = 3 w_0 u + sum_{m=1..r} w_m ( ((u_{z,y-m,x} + u_{z,y+m,x}) + (u_{z,y,x-m} + u_{z,y,x+m}))
//                                      + (u_{z-m,y,x} + u_{z+m,y,x}) )
//   u^{n+1} = (2 u^n - u^{n-1}) + c2 * L u^n          (start: u^{-1} = u^0 + (c2/2) L u^0)
//
// Every operation is an explicit round-to-nearest FP32 intrinsic in exactly this
// order; 16-bit storage is widened exactly and the result rounded once.
//
// Vector kernel (16-byte aligned rows), HBM-bound at 3 x sizeof(S) bytes per point:
//   * A warp owns a column of tiles: 32*V columns x RY rows, marched through a
//     segment of consecutive planes.  It keeps the tile's rows of the 2r+1 planes
//     z-r .. z+r in registers (a queue shifted by one plane per step), so each
//     plane of u^n is read once per segment; per plane it loads one new plane of
//     the tile, the r rows above and below the tile (L2 hits: the neighbouring
//     tiles read them too), the tile of u^{n-1} and, in lanes 0 and 31, the r
//     columns beyond the warp's span.
//   * Horizontal neighbours come from the adjacent lanes by warp shuffles.
//   * Tasks (tile column x plane segment) are numbered x fastest, then y, then
//     segment; persistent warps stride over them, so the warps in flight work on
//     neighbouring tiles of the same few segments and the halo rows they share
//     are still in L2.  The host sizes the segments so that every warp gets the
//     same number of tasks.
// Scalar kernel: rows that are not 16-byte aligned; one point per thread.
#pragma once

#include "wave_kernel.cuh"

namespace sy {
namespace wave3 {

using wave::kFull;
using wave::Traits;
using wave::wk;

// 3 w_0 rounded once to FP32: r = 1: -6, r = 2: -15/2, r = 3: -49/6, r = 4: -205/24.
template <int R>
__device__ __forceinline__ float c0x3();
template <>
__device__ __forceinline__ float c0x3<1>() { return -6.0f; }
template <>
__device__ __forceinline__ float c0x3<2>() { return -7.5f; }
template <>
__device__ __forceinline__ float c0x3<3>() { return static_cast<float>(-49.0 / 6.0); }
template <>
__device__ __forceinline__ float c0x3<4>() { return static_cast<float>(-205.0 / 24.0); }

struct Args3 {
    const char* u_prev;  // unused by the start kernel
    const char* u_cur;
    char* u_next;
    int64_t nz, ny, nx, pitch_bytes, plane_bytes;
    int64_t z_begin, z_end;    // the chunk's planes
    int64_t tiles_x, tiles_y;  // warp tiles per plane
    int64_t seg, segs;         // planes per segment, segments in the chunk
    int64_t tasks;             // tiles_x * tiles_y * segs
    float c2;                  // coefficient of L u
    unsigned long long* stamp;
    int pdl;  // as in the 2D kernel: 0 none, 1 wait for the predecessor first, 2 independent chunk
    float neg0;  // -0.0f, set by the host: the packed products' addend (wave::mul2_rn)
};

template <int R, bool START>
__device__ __forceinline__ float update3(float u, float up, const float (&vert)[R], const float (&horz)[R],
                                         const float (&depth)[R], float c2) {
    float acc = __fmul_rn(c0x3<R>(), u);
#pragma unroll
    for (int d = 1; d <= R; ++d)
        acc = __fadd_rn(acc, __fmul_rn(wk<R>(d), __fadd_rn(__fadd_rn(vert[d - 1], horz[d - 1]), depth[d - 1])));
    if (START) return __fadd_rn(u, __fmul_rn(c2, acc));
    return __fadd_rn(__fsub_rn(__fmul_rn(2.0f, u), up), __fmul_rn(c2, acc));
}

// update3 for two neighbouring points, additions paired (wave::add2_rn) and products
// paired as FMAs with the run-time -0 addend neg0 (wave::mul2_rn): bit-identical to
// update3.
template <int R, bool START>
__device__ __forceinline__ float2 update3_2(float2 u, float2 up, const float2 (&vert)[R], const float2 (&horz)[R],
                                            const float2 (&depth)[R], float c2, float neg0) {
    using wave::add2_rn;
    using wave::mul2_rn;
    float2 acc = mul2_rn(c0x3<R>(), u, neg0);
#pragma unroll
    for (int d = 1; d <= R; ++d)
        acc = add2_rn(acc, mul2_rn(wk<R>(d), add2_rn(add2_rn(vert[d - 1], horz[d - 1]), depth[d - 1]), neg0));
    if (START) return add2_rn(u, mul2_rn(c2, acc, neg0));
    return add2_rn(wave::inertia2(u, up), mul2_rn(c2, acc, neg0));
}

// One row of a lane's V points: c is the row itself, up[d-1] / dn[d-1] the rows d
// above / below, zm[d-1] / zp[d-1] the same row d planes before / after, pv its
// u^{n-1}; edge[d-1] the column d beyond the warp's span (lane 0: left, lane 31:
// right).  Horizontal neighbours inside the span come from the adjacent lanes.
template <typename S, int R, bool START>
__device__ __forceinline__ void row_update(const uint4& c, const uint4 (&up)[R], const uint4 (&dn)[R],
                                           const uint4 (&zm)[R], const uint4 (&zp)[R], const uint4& pv,
                                           const float (&edge)[R], int lane, float c2, float neg0,
                                           float (&out)[Traits<S>::V]) {
    using T = Traits<S>;
    constexpr int V = T::V;
    float ext[V + 2 * R];  // ext[m] holds column x0 - R + m
#pragma unroll
    for (int e = 0; e < V; ++e) ext[R + e] = T::elem(c, e);
#pragma unroll
    for (int d = 1; d <= R; ++d) {
        const float from_left = __shfl_up_sync(kFull, ext[R + V - d], 1);
        const float from_right = __shfl_down_sync(kFull, ext[R + d - 1], 1);
        ext[R - d] = lane == 0 ? edge[d - 1] : from_left;
        ext[R + V - 1 + d] = lane == 31 ? edge[d - 1] : from_right;
    }
    if constexpr (sizeof(S) == 2) {  // 16-bit storage: pair the additions and the products
#pragma unroll
        for (int e = 0; e < V; e += 2) {
            float2 vert[R], horz[R], depth[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                vert[d - 1] = wave::add2_rn(make_float2(T::elem(up[d - 1], e), T::elem(up[d - 1], e + 1)),
                                            make_float2(T::elem(dn[d - 1], e), T::elem(dn[d - 1], e + 1)));
                horz[d - 1] = wave::horz2<R>(ext, e, d);
                depth[d - 1] = wave::add2_rn(make_float2(T::elem(zm[d - 1], e), T::elem(zm[d - 1], e + 1)),
                                             make_float2(T::elem(zp[d - 1], e), T::elem(zp[d - 1], e + 1)));
            }
            const float2 u2 = START ? make_float2(0.0f, 0.0f) : make_float2(T::elem(pv, e), T::elem(pv, e + 1));
            const float2 o = update3_2<R, START>(make_float2(ext[R + e], ext[R + e + 1]), u2, vert, horz, depth, c2, neg0);
            out[e] = o.x;
            out[e + 1] = o.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            float vert[R], horz[R], depth[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                vert[d - 1] = __fadd_rn(T::elem(up[d - 1], e), T::elem(dn[d - 1], e));
                horz[d - 1] = __fadd_rn(ext[R + e - d], ext[R + e + d]);
                depth[d - 1] = __fadd_rn(T::elem(zm[d - 1], e), T::elem(zp[d - 1], e));
            }
            out[e] = update3<R, START>(ext[R + e], START ? 0.0f : T::elem(pv, e), vert, horz, depth, c2);
        }
    }
}

// One warp's task: tile (tx, ty) through the planes of segment sg.  CHECK = false
// is the interior form: every row the tile reads lies in [0, ny) and every lane's
// V columns in [0, nx) (planes are always checked against [0, nz)).
template <typename S, int R, int RY, bool START, bool CHECK>
__device__ __forceinline__ void column_impl(const Args3& a, int64_t tx, int64_t ty, int64_t sg, int lane) {
    using T = Traits<S>;
    constexpr int V = T::V;
    constexpr int64_t ES = sizeof(S);
    static_assert(R <= V, "radius must not exceed the vector width");
    const int64_t pb = a.pitch_bytes, zb = a.plane_bytes;
    const int64_t x0 = (tx * 32 + lane) * V;
    const int64_t y0 = ty * RY;
    const int64_t za = a.z_begin + sg * a.seg;
    const int64_t ze = za + a.seg < a.z_end ? za + a.seg : a.z_end;
    const bool col_in = !CHECK || x0 < a.nx;
    const int nvalid = !CHECK ? V : (col_in ? static_cast<int>(a.nx - x0 < V ? a.nx - x0 : V) : 0);
    const bool masked = CHECK && nvalid < V;
    const char* cur_col = a.u_cur + x0 * ES;  // plane 0, row 0, this lane's columns
    auto row_in = [&](int64_t y) { return !CHECK || (y >= 0 && y < a.ny); };
    auto load_cur = [&](int64_t z, int64_t y) -> uint4 {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (z >= 0 && z < a.nz && col_in && row_in(y)) {
            v = __ldg(reinterpret_cast<const uint4*>(cur_col + z * zb + y * pb));
            if (masked) T::mask(v, nvalid);
        }
        return v;
    };

    // q[m][k]: row y0 + k of plane z - R + m
    uint4 q[2 * R + 1][RY];
#pragma unroll
    for (int m = 1; m <= 2 * R; ++m)
#pragma unroll
        for (int k = 0; k < RY; ++k) q[m][k] = load_cur(za - R + (m - 1), y0 + k);

    // lanes 0 and 31 read the R columns beyond the warp's span, one element each
    const bool edge_lane = lane == 0 || lane == 31;
    const int64_t edge_col0 = lane == 0 ? x0 - 1 : x0 + V;  // column at distance 1; d steps outwards
    const int64_t edge_step = lane == 0 ? -1 : 1;

    for (int64_t z = za; z < ze; ++z) {
#pragma unroll
        for (int m = 0; m < 2 * R; ++m)
#pragma unroll
            for (int k = 0; k < RY; ++k) q[m][k] = q[m + 1][k];
#pragma unroll
        for (int k = 0; k < RY; ++k) q[2 * R][k] = load_cur(z + R, y0 + k);
        // yh[d-1]: row y0 - d;  yh[R + d - 1]: row y0 + RY - 1 + d   (plane z)
        uint4 yh[2 * R];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            yh[d - 1] = load_cur(z, y0 - d);
            yh[R + d - 1] = load_cur(z, y0 + RY - 1 + d);
        }
        uint4 prev[START ? 1 : RY];
        if (!START) {
            const char* pbase = a.u_prev + z * zb + y0 * pb + x0 * ES;
#pragma unroll
            for (int k = 0; k < RY; ++k) {
                prev[k] = make_uint4(0u, 0u, 0u, 0u);
                if (col_in && row_in(y0 + k)) prev[k] = __ldcs(reinterpret_cast<const uint4*>(pbase + k * pb));
            }
        }
        float edge[RY][R];  // edge[k][d-1]: column x0 - d (lane 0) or x0 + V - 1 + d (lane 31)
        const char* ebase = a.u_cur + z * zb + y0 * pb;
#pragma unroll
        for (int k = 0; k < RY; ++k)
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const int64_t col = edge_col0 + (d - 1) * edge_step;
                edge[k][d - 1] = 0.0f;
                if (edge_lane && row_in(y0 + k) && col >= 0 && col < a.nx)
                    edge[k][d - 1] = T::load1(ebase + k * pb + col * ES);
            }

        char* nbase = a.u_next + z * zb + y0 * pb + x0 * ES;
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            uint4 up[R], dn[R], zm[R], zp[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const int up_row = k - d, dn_row = k + d;
                up[d - 1] = up_row >= 0 ? q[R][up_row >= 0 ? up_row : 0] : yh[(-up_row - 1) < R ? (-up_row - 1) : 0];
                dn[d - 1] = dn_row < RY ? q[R][dn_row < RY ? dn_row : 0]
                                        : yh[R + (dn_row - RY < R ? dn_row - RY : 0)];
                zm[d - 1] = q[R - d][k];
                zp[d - 1] = q[R + d][k];
            }
            float out[V];
            row_update<S, R, START>(q[R][k], up, dn, zm, zp, prev[START ? 0 : k], edge[k], lane, a.c2, a.neg0, out);
            if (col_in && row_in(y0 + k)) {
                char* dst = nbase + k * pb;
                if (!CHECK || nvalid == V) {
                    __stcs(reinterpret_cast<uint4*>(dst), T::pack(out));
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (e < nvalid) T::store1(dst + e * ES, out[e]);
                }
            }
        }
    }
}

template <typename S, int R, int RY, bool START>
__device__ __forceinline__ void column(const Args3& a, int64_t tx, int64_t ty, int64_t sg, int lane) {
    constexpr int V = Traits<S>::V;
    const int64_t y0 = ty * RY;
    const bool interior = (y0 - R >= 0) && (y0 + RY + R <= a.ny) && ((tx + 1) * 32 * V <= a.nx);
    if (interior) column_impl<S, R, RY, START, false>(a, tx, ty, sg, lane);
    else column_impl<S, R, RY, START, true>(a, tx, ty, sg, lane);
}

// Register cap per tile height (blocks of 256 threads that must fit an SM): the
// kernel is latency-bound when few warps are resident, and its loads of a plane are
// consumed in the same step, so resident warps are what keeps HBM busy.  Radius 1
// gets 64 / 85 / 128 registers for 1 / 2 / 4 rows, radius 2 one step less, 16-bit
// radius 3-4 128 for one row (the rest uncapped).  The 1-row FP32 forms and the 1-row 16-bit radius-1 form
// fit without spilling; the FP32 radius-1 forms of 2 and 4 rows and several 16-bit
// forms spill up to about 150 bytes a thread.  Measured at 512^3, resident warps
// still win: raising the 16-bit radius-2 one-row cap to 128 registers (no spill,
// 16 warps an SM instead of 24) ran 5 % slower, and loading the next plane's HBM
// rows one plane ahead (two planes in flight per warp for 2 x rows more vectors a
// lane) ran 6-30 % slower for every storage type and radius 1-4.  16-bit radius 3-4
// one-row columns are held to 2 blocks of 256 (128 registers; uncapped 180 / 210, one
// block of 256 an SM): BF16 radius 4 2.5e11 -> 2.7e11 updates/s.  The same cap on FP32
// radius 4 (168 -> 128 registers, a 28-byte spill) ran 8 % slower, so FP32 radius 3-4
// stay uncapped.
template <int R, int RY, int ES>
struct MinBlocks3 {
    static constexpr int value = R == 1   ? (RY == 1 ? 4 : RY == 2 ? 3 : 2)
                                 : R == 2 ? (RY == 1 ? 3 : RY == 2 ? 2 : 1)
                                          : (RY == 1 && ES == 2 ? 2 : 1);
};

template <typename S, int R, int RY, bool START>
__global__ void __launch_bounds__(256, MinBlocks3<R, RY, sizeof(S)>::value) wave3d_vec_kernel(Args3 a) {
    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    const int lane = threadIdx.x & 31;
    const int64_t warps_per_block = blockDim.x >> 5;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * warps_per_block;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * warps_per_block + (threadIdx.x >> 5); t < a.tasks;
         t += nwarps) {
        const int64_t rest = t / a.tiles_x;
        const int64_t tx = t - rest * a.tiles_x;
        const int64_t sg = rest / a.tiles_y;
        const int64_t ty = rest - sg * a.tiles_y;
        column<S, R, RY, START>(a, tx, ty, sg, lane);
    }
    stamp_end(a.stamp);
    if (a.pdl && threadIdx.x == 0) griddep_wait();
}

// Slab form (radius 2-4 pays for it): a block of 8 warps marches a strip of
// RB = 8*RYW consecutive rows (warp w owns rows w*RYW ..) through the planes of a
// segment together.  Each warp keeps its rows' plane queue in registers as above,
// but the rows above and below a row come from a shared-memory slab holding the
// centre plane of the whole strip plus its R-row halo (loaded by the first and
// last warp), so a strip reads 2R halo rows per plane instead of every warp
// reading 2R.  The slab is double-buffered by plane: one barrier per plane.
constexpr int kSlabWarps = 8;

template <int R, int RYW>
struct Slab {
    static constexpr int RB = kSlabWarps * RYW;                   // rows of the strip
    static constexpr int SR = RB + 2 * R;                         // slab rows (with halo)
    static constexpr int BYTES = 2 * SR * 32 * sizeof(uint4);     // two planes of slab
};

template <typename S, int R, int RYW, bool START, bool CHECK>
__device__ __forceinline__ void strip_impl(const Args3& a, int64_t tx, int64_t tb, int64_t sg, uint4* slab,
                                           int warp, int lane) {
    using T = Traits<S>;
    using SL = Slab<R, RYW>;
    constexpr int V = T::V;
    constexpr int64_t ES = sizeof(S);
    const int64_t pb = a.pitch_bytes, zb = a.plane_bytes;
    const int64_t x0 = (tx * 32 + lane) * V;
    const int64_t yb = tb * SL::RB;          // first row of the strip
    const int64_t y0 = yb + warp * RYW;      // this warp's first row
    const int64_t za = a.z_begin + sg * a.seg;
    const int64_t ze = za + a.seg < a.z_end ? za + a.seg : a.z_end;
    const bool col_in = !CHECK || x0 < a.nx;
    const int nvalid = !CHECK ? V : (col_in ? static_cast<int>(a.nx - x0 < V ? a.nx - x0 : V) : 0);
    const bool masked = CHECK && nvalid < V;
    const char* cur_col = a.u_cur + x0 * ES;
    auto row_in = [&](int64_t y) { return !CHECK || (y >= 0 && y < a.ny); };
    auto load_cur = [&](int64_t z, int64_t y) -> uint4 {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (z >= 0 && z < a.nz && col_in && row_in(y)) {
            v = __ldg(reinterpret_cast<const uint4*>(cur_col + z * zb + y * pb));
            if (masked) T::mask(v, nvalid);
        }
        return v;
    };
    uint4 q[2 * R + 1][RYW];  // q[m][k]: row y0 + k of plane z - R + m
#pragma unroll
    for (int m = 1; m <= 2 * R; ++m)
#pragma unroll
        for (int k = 0; k < RYW; ++k) q[m][k] = load_cur(za - R + (m - 1), y0 + k);
    const bool edge_lane = lane == 0 || lane == 31;
    const int64_t edge_col0 = lane == 0 ? x0 - 1 : x0 + V;
    const int64_t edge_step = lane == 0 ? -1 : 1;

    for (int64_t z = za; z < ze; ++z) {
#pragma unroll
        for (int m = 0; m < 2 * R; ++m)
#pragma unroll
            for (int k = 0; k < RYW; ++k) q[m][k] = q[m + 1][k];
#pragma unroll
        for (int k = 0; k < RYW; ++k) q[2 * R][k] = load_cur(z + R, y0 + k);
        // slab row j holds strip row j - R of plane z
        uint4* sl = slab + ((z - za) & 1) * (SL::SR * 32);
#pragma unroll
        for (int k = 0; k < RYW; ++k) sl[(R + warp * RYW + k) * 32 + lane] = q[R][k];
        if (warp == 0) {
#pragma unroll
            for (int d = 1; d <= R; ++d) sl[(R - d) * 32 + lane] = load_cur(z, yb - d);
        } else if (warp == kSlabWarps - 1) {
#pragma unroll
            for (int d = 1; d <= R; ++d) sl[(R + SL::RB - 1 + d) * 32 + lane] = load_cur(z, yb + SL::RB - 1 + d);
        }
        uint4 prev[START ? 1 : RYW];
        if (!START) {
            const char* pbase = a.u_prev + z * zb + y0 * pb + x0 * ES;
#pragma unroll
            for (int k = 0; k < RYW; ++k) {
                prev[k] = make_uint4(0u, 0u, 0u, 0u);
                if (col_in && row_in(y0 + k)) prev[k] = __ldcs(reinterpret_cast<const uint4*>(pbase + k * pb));
            }
        }
        float edge[RYW][R];
        const char* ebase = a.u_cur + z * zb + y0 * pb;
#pragma unroll
        for (int k = 0; k < RYW; ++k)
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const int64_t col = edge_col0 + (d - 1) * edge_step;
                edge[k][d - 1] = 0.0f;
                if (edge_lane && row_in(y0 + k) && col >= 0 && col < a.nx)
                    edge[k][d - 1] = T::load1(ebase + k * pb + col * ES);
            }
        __syncthreads();  // the strip's plane z is in the slab (the other buffer is still being read by none)

        char* nbase = a.u_next + z * zb + y0 * pb + x0 * ES;
#pragma unroll
        for (int k = 0; k < RYW; ++k) {
            uint4 up[R], dn[R], zm[R], zp[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const int ru = k - d, rd = k + d;  // rows relative to this warp's first row
                up[d - 1] = ru >= 0 ? q[R][ru >= 0 ? ru : 0] : sl[(R + warp * RYW + ru) * 32 + lane];
                dn[d - 1] = rd < RYW ? q[R][rd < RYW ? rd : 0] : sl[(R + warp * RYW + rd) * 32 + lane];
                zm[d - 1] = q[R - d][k];
                zp[d - 1] = q[R + d][k];
            }
            float out[V];
            row_update<S, R, START>(q[R][k], up, dn, zm, zp, prev[START ? 0 : k], edge[k], lane, a.c2, a.neg0, out);
            if (col_in && row_in(y0 + k)) {
                char* dst = nbase + k * pb;
                if (!CHECK || nvalid == V) {
                    __stcs(reinterpret_cast<uint4*>(dst), T::pack(out));
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (e < nvalid) T::store1(dst + e * ES, out[e]);
                }
            }
        }
    }
    __syncthreads();  // the slab is free for the block's next task
}

// Tasks are (tile column, strip, segment), x fastest; persistent blocks stride over them.
template <typename S, int R, int RYW, bool START>
__global__ void __launch_bounds__(kSlabWarps * 32) wave3d_slab_kernel(Args3 a) {
    __shared__ uint4 slab[Slab<R, RYW>::BYTES / sizeof(uint4)];
    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int V = Traits<S>::V;
    constexpr int RB = Slab<R, RYW>::RB;
    for (int64_t t = blockIdx.x; t < a.tasks; t += gridDim.x) {  // block-uniform
        const int64_t rest = t / a.tiles_x;
        const int64_t tx = t - rest * a.tiles_x;
        const int64_t sg = rest / a.tiles_y;
        const int64_t tb = rest - sg * a.tiles_y;
        const int64_t yb = tb * RB;
        const bool interior = (yb - R >= 0) && (yb + RB + R <= a.ny) && ((tx + 1) * 32 * V <= a.nx);
        if (interior) strip_impl<S, R, RYW, START, false>(a, tx, tb, sg, slab, warp, lane);
        else strip_impl<S, R, RYW, START, true>(a, tx, tb, sg, slab, warp, lane);
    }
    stamp_end(a.stamp);
    if (a.pdl && threadIdx.x == 0) griddep_wait();
}

// One point per thread; any element-aligned layout.
template <typename S, int R, bool START>
__global__ void __launch_bounds__(256) wave3d_scalar_kernel(Args3 a) {
    using T = Traits<S>;
    stamp_begin(a.stamp);
    const int64_t planes = a.z_end - a.z_begin;
    const int64_t per_plane = a.ny * a.nx;
    const int64_t total = planes * per_plane;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < total; p += stride) {
        const int64_t z = a.z_begin + p / per_plane;
        const int64_t r = p - (z - a.z_begin) * per_plane;
        const int64_t y = r / a.nx;
        const int64_t x = r - y * a.nx;
        auto at = [&](int64_t zz, int64_t yy, int64_t xx) -> float {
            if (zz < 0 || zz >= a.nz || yy < 0 || yy >= a.ny || xx < 0 || xx >= a.nx) return 0.0f;
            return T::load1(a.u_cur + zz * a.plane_bytes + yy * a.pitch_bytes + xx * static_cast<int64_t>(sizeof(S)));
        };
        float vert[R], horz[R], depth[R];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            vert[d - 1] = __fadd_rn(at(z, y - d, x), at(z, y + d, x));
            horz[d - 1] = __fadd_rn(at(z, y, x - d), at(z, y, x + d));
            depth[d - 1] = __fadd_rn(at(z - d, y, x), at(z + d, y, x));
        }
        const int64_t off = z * a.plane_bytes + y * a.pitch_bytes + x * static_cast<int64_t>(sizeof(S));
        const float up = START ? 0.0f : T::load1_cs(a.u_prev + off);
        T::store1(a.u_next + off, update3<R, START>(at(z, y, x), up, vert, horz, depth, a.c2));
    }
    stamp_end(a.stamp);
}

using KernelFn3 = void (*)(Args3);

// Warp-column variants 1-6: tile heights {1, 2, 4} (the register queue holds
// (2r+1) x RY vectors) x {128, 256} threads, variant v = (rows[(v-1) % 3],
// threads[(v-1) / 3]).  Slab variants 7-8: strips of 8 x {1, 2} rows, 256 threads.
constexpr int kRows12[3] = {1, 2, 4};
constexpr int kRows34[3] = {1, 2, 4};
constexpr int kThreads3[2] = {128, 256};
constexpr int kColumnVariants3 = 6;
constexpr int kVariants3 = 10;  // + TMA variants 9-10 (wave3d_tma.cuh): strips of 8 x {2, 4} rows

// rows < 0: the slab kernel with strips of -rows rows
template <typename S, int R, bool START>
KernelFn3 pick_vec3(int rows) {
    switch (rows) {
        case 1: return wave3d_vec_kernel<S, R, 1, START>;
        case 2: return wave3d_vec_kernel<S, R, 2, START>;
        case 4: return wave3d_vec_kernel<S, R, 4, START>;
        case -8: return wave3d_slab_kernel<S, R, 1, START>;
        default: return wave3d_slab_kernel<S, R, 2, START>;
    }
}

// rows > 0: warp-column kernel with rows-row tiles; rows < 0: slab kernel, strips of -rows rows.
sy_status launch3_typed(Queue* q, const WaveLaunch3& w, KernelFn3 vec_fn, KernelFn3 scalar_fn, int rows, int threads,
                        int V, size_t esize);

template <typename S, int R>
sy_status launch3_r(Queue* q, const WaveLaunch3& w, int rows, int threads) {
    KernelFn3 vec = w.start ? pick_vec3<S, R, true>(rows) : pick_vec3<S, R, false>(rows);
    KernelFn3 sca = w.start ? wave3d_scalar_kernel<S, R, true> : wave3d_scalar_kernel<S, R, false>;
    return launch3_typed(q, w, vec, sca, rows, threads, Traits<S>::V, sizeof(S));
}

template <typename S>
sy_status launch3_dtype(Queue* q, const WaveLaunch3& w, int rows, int threads) {
    switch (w.radius) {
        case 1: return launch3_r<S, 1>(q, w, rows, threads);
        case 2: return launch3_r<S, 2>(q, w, rows, threads);
        case 3: return launch3_r<S, 3>(q, w, rows, threads);
        default: return launch3_r<S, 4>(q, w, rows, threads);
    }
}

sy_status launch3_f32(Queue* q, const WaveLaunch3& w, int rows, int threads);
sy_status launch3_bf16(Queue* q, const WaveLaunch3& w, int rows, int threads);
sy_status launch3_f16(Queue* q, const WaveLaunch3& w, int rows, int threads);

}  // namespace wave3
}  // namespace sy
