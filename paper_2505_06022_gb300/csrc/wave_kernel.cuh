// Leapfrog wave step kernels (radius-r star stencil, Dirichlet-zero ghosts) for
// one row chunk of a row-major field.  Included by wave_f32.cu, wave_bf16.cu and
// wave_f16.cu, one storage type each.
//
//   L u_ij  = 2 w_0 u_ij + sum_{k=1..r} w_k ((u_{i-k,j} + u_{i+k,j}) + (u_{i,j-k} + u_{i,j+k}))
//   u^{n+1} = (2 u^n - u^{n-1}) + c2 * L u^n          (start: u^{-1} = u^0 + (c2/2) L u^0)
//
// Every operation is an explicit round-to-nearest FP32 intrinsic in exactly this
// order, so no FMA contraction can change a bit; 16-bit storage is widened
// exactly and the result rounded once (round to nearest even).
//
// Vector kernel (16-byte aligned rows): HBM-bound, 3 x sizeof(S) bytes per point.
//   * A warp owns a tile of 32*V columns x RY rows (V = 16 / sizeof(S)); lane l
//     owns the V columns [x0, x0+V) and marches down the RY rows.
//   * All loads of a tile are issued before any arithmetic: RY+2r rows of u_cur
//     (halo rows included, read through the non-coherent path: u_cur is never
//     written during the step), RY rows of u_prev and the two warp-edge vectors
//     per row, each a single 128-bit access.  u_prev/u_next are streamed
//     (ld.global.cs / st.global.cs: touched once), u_cur keeps default caching
//     so that the halo rows re-read by the tile below hit in L2.
//   * Horizontal neighbours come from the adjacent lanes by warp shuffles; only
//     lanes 0 and 31 load the r columns beyond the warp's span.
//   * Warps stride over the tiles of the chunk in row-major tile order, so the
//     tiles in flight at any moment form a narrow band of rows and the halo rows
//     are still in L2 when they are read again.
// Scalar kernel: any layout whose rows are not 16-byte aligned; one point per
// thread, same arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "stamp.cuh"
#include "sy_internal.h"

namespace sy {
namespace wave {

constexpr unsigned kFull = 0xffffffffu;

// ---- weights: the order-2r central second difference, rounded once to FP32 ----
// r = 1: 1, -2, 1;  r = 2: -1/12, 4/3, -5/2;  r = 3: 1/90, -3/20, 3/2, -49/18;
// r = 4: -1/560, 8/315, -1/5, 8/5, -205/72 (Fornberg 1988).  c0x2 = 2 w_0 (the
// centre weight of the 2D star counts once per axis).
template <int R>
__device__ __forceinline__ float c0x2();
template <>
__device__ __forceinline__ float c0x2<1>() { return -4.0f; }
template <>
__device__ __forceinline__ float c0x2<2>() { return -5.0f; }
template <>
__device__ __forceinline__ float c0x2<3>() { return static_cast<float>(-49.0 / 9.0); }
template <>
__device__ __forceinline__ float c0x2<4>() { return static_cast<float>(-205.0 / 36.0); }

template <int R>
__device__ __forceinline__ float wk(int k);
template <>
__device__ __forceinline__ float wk<1>(int) { return 1.0f; }
template <>
__device__ __forceinline__ float wk<2>(int k) {
    return k == 1 ? static_cast<float>(4.0 / 3.0) : static_cast<float>(-1.0 / 12.0);
}
template <>
__device__ __forceinline__ float wk<3>(int k) {
    return k == 1 ? 1.5f : (k == 2 ? static_cast<float>(-3.0 / 20.0) : static_cast<float>(1.0 / 90.0));
}
template <>
__device__ __forceinline__ float wk<4>(int k) {
    return k == 1   ? static_cast<float>(8.0 / 5.0)
           : k == 2 ? static_cast<float>(-1.0 / 5.0)
           : k == 3 ? static_cast<float>(8.0 / 315.0)
                    : static_cast<float>(-1.0 / 560.0);
}

// ---- storage traits: a 16-byte unit holds V elements -----------------------------
template <typename S>
struct Traits;

__device__ __forceinline__ uint32_t word(const uint4& r, int i) {
    return i == 0 ? r.x : (i == 1 ? r.y : (i == 2 ? r.z : r.w));
}
__device__ __forceinline__ void set_word(uint4& r, int i, uint32_t v) {
    if (i == 0) r.x = v;
    else if (i == 1) r.y = v;
    else if (i == 2) r.z = v;
    else r.w = v;
}
__device__ __forceinline__ uint32_t word(const uint2& r, int i) { return i == 0 ? r.x : r.y; }
__device__ __forceinline__ void set_word(uint2& r, int i, uint32_t v) {
    if (i == 0) r.x = v;
    else r.y = v;
}

// 16- and 8-byte global accesses of one lane's vector.
struct Vec16 {
    using T = uint4;
    __device__ static __forceinline__ uint4 zero() { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ static __forceinline__ uint4 ld(const char* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
    __device__ static __forceinline__ uint4 ld_cs(const char* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
    __device__ static __forceinline__ uint4 ld_cg(const char* p) { return __ldcg(reinterpret_cast<const uint4*>(p)); }
    __device__ static __forceinline__ void st_cs(char* p, uint4 v) { __stcs(reinterpret_cast<uint4*>(p), v); }
};
struct Vec8 {
    using T = uint2;
    __device__ static __forceinline__ uint2 zero() { return make_uint2(0u, 0u); }
    __device__ static __forceinline__ uint2 ld(const char* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
    __device__ static __forceinline__ uint2 ld_cs(const char* p) { return __ldcs(reinterpret_cast<const uint2*>(p)); }
    __device__ static __forceinline__ uint2 ld_cg(const char* p) { return __ldcg(reinterpret_cast<const uint2*>(p)); }
    __device__ static __forceinline__ void st_cs(char* p, uint2 v) { __stcs(reinterpret_cast<uint2*>(p), v); }
};

template <>
struct Traits<float> {
    static constexpr int V = 4;
    using Mem = Vec16;
    __device__ static __forceinline__ float elem(const uint4& r, int e) { return __uint_as_float(word(r, e)); }
    // zero elements e >= nvalid
    __device__ static __forceinline__ void mask(uint4& r, int nvalid) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (e >= nvalid) set_word(r, e, 0u);
    }
    __device__ static __forceinline__ uint4 pack(const float (&v)[V]) {
        return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                          __float_as_uint(v[3]));
    }
    __device__ static __forceinline__ float load1(const char* p) { return __ldg(reinterpret_cast<const float*>(p)); }
    __device__ static __forceinline__ float load1_cg(const char* p) {
        return __ldcg(reinterpret_cast<const float*>(p));
    }
    __device__ static __forceinline__ float load1_cs(const char* p) {
        return __ldcs(reinterpret_cast<const float*>(p));
    }
    __device__ static __forceinline__ void store1(char* p, float v) { *reinterpret_cast<float*>(p) = v; }
};

template <>
struct Traits<__nv_bfloat16> {
    static constexpr int V = 8;
    using Mem = Vec16;
    __device__ static __forceinline__ float elem(const uint4& r, int e) {
        uint32_t w = word(r, e >> 1);
        return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
    }
    __device__ static __forceinline__ void mask(uint4& r, int nvalid) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (e >= nvalid) set_word(r, e >> 1, word(r, e >> 1) & ((e & 1) ? 0x0000ffffu : 0xffff0000u));
    }
    __device__ static __forceinline__ uint32_t bits(float v) {
        return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
    // two elements per conversion (cvt.rn.bf16x2.f32: each half rounded to nearest even)
    __device__ static __forceinline__ uint32_t pair(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    __device__ static __forceinline__ uint4 pack(const float (&v)[V]) {
        return make_uint4(pair(v[0], v[1]), pair(v[2], v[3]), pair(v[4], v[5]), pair(v[6], v[7]));
    }
    __device__ static __forceinline__ float load1(const char* p) {
        return __uint_as_float(static_cast<uint32_t>(__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
    }
    __device__ static __forceinline__ float load1_cg(const char* p) {
        return __uint_as_float(static_cast<uint32_t>(__ldcg(reinterpret_cast<const unsigned short*>(p))) << 16);
    }
    __device__ static __forceinline__ float load1_cs(const char* p) {
        return __uint_as_float(static_cast<uint32_t>(__ldcs(reinterpret_cast<const unsigned short*>(p))) << 16);
    }
    __device__ static __forceinline__ void store1(char* p, float v) {
        *reinterpret_cast<unsigned short*>(p) = static_cast<unsigned short>(bits(v));
    }
};

template <>
struct Traits<__half> {
    static constexpr int V = 8;
    using Mem = Vec16;
    __device__ static __forceinline__ float elem(const uint4& r, int e) {
        uint32_t w = word(r, e >> 1);
        unsigned short h = static_cast<unsigned short>((e & 1) ? (w >> 16) : (w & 0xffffu));
        return __half2float(__ushort_as_half(h));
    }
    __device__ static __forceinline__ void mask(uint4& r, int nvalid) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (e >= nvalid) set_word(r, e >> 1, word(r, e >> 1) & ((e & 1) ? 0x0000ffffu : 0xffff0000u));
    }
    __device__ static __forceinline__ uint32_t bits(float v) {
        return static_cast<uint32_t>(__half_as_ushort(__float2half_rn(v)));
    }
    // two elements per conversion (cvt.rn.f16x2.f32: each half rounded to nearest even)
    __device__ static __forceinline__ uint32_t pair(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    __device__ static __forceinline__ uint4 pack(const float (&v)[V]) {
        return make_uint4(pair(v[0], v[1]), pair(v[2], v[3]), pair(v[4], v[5]), pair(v[6], v[7]));
    }
    __device__ static __forceinline__ float load1(const char* p) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    __device__ static __forceinline__ float load1_cg(const char* p) {
        return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p))));
    }
    __device__ static __forceinline__ float load1_cs(const char* p) {
        return __half2float(__ushort_as_half(__ldcs(reinterpret_cast<const unsigned short*>(p))));
    }
    __device__ static __forceinline__ void store1(char* p, float v) {
        *reinterpret_cast<unsigned short*>(p) = static_cast<unsigned short>(bits(v));
    }
};

// 16-bit storage, 4 elements (8 bytes) a lane: the narrow form of the tile kernel.
// Same element conversions as Traits<S>; half the registers per row of a tile.
template <typename S>
struct Narrow {
    static_assert(sizeof(S) == 2, "the narrow form is for 16-bit storage");
    static constexpr int V = 4;
    using Mem = Vec8;
    __device__ static __forceinline__ float elem(const uint2& r, int e) {
        // element e is half (e & 1) of word e >> 1: the 16-byte form's conversion of that word
        return Traits<S>::elem(make_uint4(word(r, e >> 1), 0u, 0u, 0u), e & 1);
    }
    __device__ static __forceinline__ void mask(uint2& r, int nvalid) {
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (e >= nvalid) set_word(r, e >> 1, word(r, e >> 1) & ((e & 1) ? 0x0000ffffu : 0xffff0000u));
    }
    __device__ static __forceinline__ uint2 pack(const float (&v)[V]) {
        return make_uint2(Traits<S>::pair(v[0], v[1]), Traits<S>::pair(v[2], v[3]));
    }
    __device__ static __forceinline__ float load1(const char* p) { return Traits<S>::load1(p); }
    __device__ static __forceinline__ float load1_cg(const char* p) { return Traits<S>::load1_cg(p); }
    __device__ static __forceinline__ void store1(char* p, float v) { Traits<S>::store1(p, v); }
};

template <typename S, bool NARROW>
struct TileTraits {
    using type = Traits<S>;
};
template <typename S>
struct TileTraits<S, true> {
    using type = Narrow<S>;
};

struct Args {
    const char* u_prev;  // unused by the start kernel
    const char* u_cur;
    char* u_next;
    int64_t ny, nx, pitch_bytes;
    int64_t row_begin, row_end;
    int64_t tiles_x, tiles;  // vector kernel: tiles per row band, total tiles
    float c2;                // coefficient of L u
    unsigned long long* stamp;  // timestamp slot of this launch, or null
    // Launch overlap with the previous kernel on the stream (programmatic dependent
    // launch): 0 = none; 1 = first chunk of a step: wait for the predecessor before
    // touching memory; 2 = later chunk of the same step: independent of the chunks
    // before it (disjoint rows written, earlier steps' buffers read), no entry wait.
    // With 1 or 2 the block's first thread also waits at exit, so that a launch's
    // completion implies its predecessor's and the chain is transitive.
    int pdl;
    // -0.0f, set by the host: the addend that turns a packed FMA into a packed
    // product (see mul2_rn); a run-time value, so the code generator cannot fold it.
    float neg0;
};

// One output point from its neighbourhood, in the canonical operation order.
template <int R, bool START>
__device__ __forceinline__ float update(float u, float up, const float (&vert)[R], const float (&horz)[R], float c2) {
    float acc = __fmul_rn(c0x2<R>(), u);
#pragma unroll
    for (int d = 1; d <= R; ++d) acc = __fadd_rn(acc, __fmul_rn(wk<R>(d), __fadd_rn(vert[d - 1], horz[d - 1])));
    if (START) return __fadd_rn(u, __fmul_rn(c2, acc));
    return __fadd_rn(__fsub_rn(__fmul_rn(2.0f, u), up), __fmul_rn(c2, acc));
}

// The same update for two neighbouring points at once.  The additions use
// Blackwell's packed FP32 add (add.rn.f32x2, written as PTX: each half one IEEE
// round-to-nearest addition, bit-identical to __fadd_rn); a - b is evaluated as
// a + (-b), which IEEE 754 defines to be the same operation.  Scalar multiplies are
// never contracted in the translation units that use this (built with -fmad=false).
__device__ __forceinline__ float2 add2_rn(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// a - b for two points (sub.rn.f32x2: each half one IEEE round-to-nearest
// subtraction, bit-identical to __fsub_rn).
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Scalar products of two points (the form the 3D and temporally blocked kernels use).
__device__ __forceinline__ float2 mul2_scalar(float w, float2 x) {
    return make_float2(__fmul_rn(w, x.x), __fmul_rn(w, x.y));
}

// w * x for two points as one packed FMA, fma.rn.f32x2(w, x, neg0) with neg0 = -0.0:
// each half is the exact product plus -0 rounded once, which is the rounded product
// for every input (x + -0 = x for x != 0, +0 + -0 = +0, -0 + -0 = -0), so it is
// bit-identical to __fmul_rn.  The addend is a run-time argument: a packed multiply
// (mul.rn.f32x2), or an FMA with a literal -0 addend, was measured to change results
// at radius 2-4 (the product came out fused with the addition that follows it),
// while an addend whose value is unknown at compile time leaves nothing to fold.
__device__ __forceinline__ float2 mul2_rn(float w, float2 x, float neg0) {
    float2 d;
    asm("{\n\t.reg .b64 pw, px, pz, pd;\n\t"
        "mov.b64 pw, {%2, %2};\n\tmov.b64 px, {%3, %4};\n\tmov.b64 pz, {%5, %5};\n\t"
        "fma.rn.f32x2 pd, pw, px, pz;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(w), "f"(x.x), "f"(x.y), "f"(neg0));
    return d;
}

// Horizontal pair sums (u_{j-d} + u_{j+d}) of the points j = e, e+1 from a row held as
// ext[m] = column x0 - R + m.  A packed add takes its operands from aligned register
// pairs; the pair (ext[R+e-d], ext[R+e+1-d]) starts at an even index only when R - d is
// even, so for odd R - d the two sums are scalar additions (same rounding, no register
// copies to re-pair the operands).
template <int R, int N>
__device__ __forceinline__ float2 horz2(const float (&ext)[N], int e, int d) {
    if ((R - d) % 2 == 0)
        return add2_rn(make_float2(ext[R + e - d], ext[R + e + 1 - d]), make_float2(ext[R + e + d], ext[R + e + 1 + d]));
    return make_float2(__fadd_rn(ext[R + e - d], ext[R + e + d]), __fadd_rn(ext[R + e + 1 - d], ext[R + e + 1 + d]));
}

// 2u - u_prev for two points: 2u = u + u exactly (a power-of-two scaling), and the
// subtraction as in update(); bit-identical to (2 * u) - up evaluated per point.
__device__ __forceinline__ float2 inertia2(float2 u, float2 up) { return sub2_rn(add2_rn(u, u), up); }

// PMUL: the products as packed FMAs with the run-time -0 addend neg0 (mul2_rn);
// otherwise scalar (neg0 unused).  Bit-identical either way.
template <bool PMUL>
__device__ __forceinline__ float2 mul2(float w, float2 x, float neg0) {
    if constexpr (PMUL) return mul2_rn(w, x, neg0);
    else return mul2_scalar(w, x);
}

template <int R, bool START, bool PMUL = false>
__device__ __forceinline__ float2 update2(float2 u, float2 up, const float2 (&vert)[R], const float2 (&horz)[R],
                                          float c2, float neg0 = 0.0f) {
    float2 acc = mul2<PMUL>(c0x2<R>(), u, neg0);
#pragma unroll
    for (int d = 1; d <= R; ++d) acc = add2_rn(acc, mul2<PMUL>(wk<R>(d), add2_rn(vert[d - 1], horz[d - 1]), neg0));
    if (START) return add2_rn(u, mul2<PMUL>(c2, acc, neg0));
    return add2_rn(inertia2(u, up), mul2<PMUL>(c2, acc, neg0));
}

// Loads of a tile's vectors.  Within one launch u^n is never written, so it is read
// through the non-coherent path and u^{n-1} streamed; a kernel that steps several
// times in one launch (CG = true) writes what its later steps read, so it loads
// through L2 only (ld.global.cg), which a grid-wide barrier with fences makes
// coherent.
template <typename M, bool CG>
__device__ __forceinline__ typename M::T load_cur_vec(const char* p) {
    return CG ? M::ld_cg(p) : M::ld(p);
}
template <typename M, bool CG>
__device__ __forceinline__ typename M::T load_prev_vec(const char* p) {
    return CG ? M::ld_cg(p) : M::ld_cs(p);
}

// Columns of output per warp tile: 32 lanes x V, or, with halo lanes, the 30 inner
// lanes' (lanes 0 and 31 only load the columns beside the tile).
template <typename S, bool HL, bool NARROW = false>
__host__ __device__ constexpr int tile_span() {
    return (HL ? 30 : 32) * TileTraits<S, NARROW>::type::V;
}

// One warp's tile: columns [(tx*32 + lane)*V, +V) of each lane, rows
// [row_begin + ty*RY, +RY) of the chunk [row_begin, row_end), for a field laid
// out as in `a`.  CHECK = false is the interior form, valid when every row the
// tile reads or writes lies inside the grid and the chunk's range mapper and
// every lane's V columns lie inside [0, nx): no per-row predicates then.
// HL (halo lanes): lane l covers columns [(tx*30 + l - 1)*V, +V); the outer lanes 0
// and 31 hold the columns beside the tile's 30*V and store nothing, so the inner
// lanes take every horizontal neighbour by a shuffle and no lane keeps edge
// vectors in registers.  A lane's columns outside [0, nx) read as zero (the
// Dirichlet ghosts).
// NARROW: 16-bit storage with 4 elements (8 bytes) a lane instead of 8, a warp
// covering 128 columns (with halo lanes: 120): half the registers per tile row.
template <typename S, int R, int RY, bool START, bool CHECK, bool HL = false, bool CG = false, bool NARROW = false>
__device__ __forceinline__ void wave_tile_impl(const Args& a, int64_t tx, int64_t ty, int lane) {
    using T = typename TileTraits<S, NARROW>::type;
    using M = typename T::Mem;
    using VecT = typename M::T;
    constexpr int V = T::V;
    constexpr int64_t ES = sizeof(S);
    static_assert(R <= V, "radius must not exceed the vector width");
    const int64_t pb = a.pitch_bytes;
    const int64_t x0 = HL ? (tx * 30 + lane - 1) * V : (tx * 32 + lane) * V;
    const int64_t y0 = a.row_begin + ty * RY;
    const bool col_in = !CHECK || (x0 < a.nx && (!HL || x0 >= 0));
    const int nvalid = !CHECK ? V : (col_in ? static_cast<int>(a.nx - x0 < V ? a.nx - x0 : V) : 0);
    const bool stores = !HL || (lane >= 1 && lane <= 30);
    const char* cur_base = a.u_cur + (y0 - R) * pb + x0 * ES;  // row y0 - R
    const char* prev_base = a.u_prev + y0 * pb + x0 * ES;

    // ---- loads: everything for the tile is in flight before any arithmetic ----
    VecT cur[RY + 2 * R];
#pragma unroll
    for (int k = 0; k < RY + 2 * R; ++k) {
        cur[k] = M::zero();
        if (!CHECK) {
            cur[k] = load_cur_vec<M, CG>(cur_base + k * pb);
        } else {
            const int64_t row = y0 - R + k;
            if (col_in && row >= 0 && row < a.ny && row < a.row_end + R)
                cur[k] = load_cur_vec<M, CG>(cur_base + k * pb);
        }
    }
    VecT prev[START ? 1 : RY];
    if (!START) {
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            prev[k] = M::zero();
            if (!CHECK || (col_in && y0 + k < a.row_end))
                prev[k] = load_prev_vec<M, CG>(prev_base + k * pb);
        }
    }
    // warp edges: lane 0 fetches the columns left of the warp, lane 31 those right of
    // it: the whole neighbouring vector per row, or, for 16-bit storage at radius 1, the
    // one column as a scalar (one value per row instead of a vector that every lane
    // holds registers for; the 8-point vectors' unpacked arithmetic needs them more).
    // Measured at 8192^2 with 4-row tiles: BF16 +1 %, FP16 +5 %; at radius 3-4 the R
    // scalar loads per row cost more than they save (10-26 % slower with 8-row tiles).
    constexpr bool kScalarEdge = !HL && sizeof(S) == 2 && R == 1;
    VecT edge[(kScalarEdge || HL) ? 1 : RY];
    float edge1[kScalarEdge ? RY : 1][R];  // edge1[k][d-1]: column x0 - d (lane 0) or x0 + V - 1 + d (lane 31)
    if constexpr (HL) {
        // no edge loads: lanes 0 and 31 are the edges
    } else if constexpr (kScalarEdge) {
        const bool edge_lane = lane == 0 || lane == 31;
        const int64_t col0 = lane == 0 ? x0 - 1 : x0 + V;
        const int64_t step = lane == 0 ? -1 : 1;
        const char* erow = a.u_cur + y0 * pb;
#pragma unroll
        for (int k = 0; k < RY; ++k)
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const int64_t col = col0 + (d - 1) * step;
                edge1[k][d - 1] = 0.0f;
                if (edge_lane && (!CHECK || y0 + k < a.row_end) && col >= 0 && col < a.nx)
                    edge1[k][d - 1] = CG ? T::load1_cg(erow + k * pb + col * ES) : T::load1(erow + k * pb + col * ES);
            }
    } else {
        const int64_t xe = lane == 0 ? x0 - V : x0 + V;
        const bool edge_lane = (lane == 0 && xe >= 0) || (lane == 31 && xe < a.nx);
        const int edge_valid = lane == 0 ? V : static_cast<int>(a.nx - xe < V ? a.nx - xe : V);
        const char* edge_base = a.u_cur + y0 * pb + xe * ES;
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            edge[k] = M::zero();
            if (edge_lane && (!CHECK || y0 + k < a.row_end))
                edge[k] = load_cur_vec<M, CG>(edge_base + k * pb);
        }
        if (lane == 31 && edge_valid < V) {
#pragma unroll
            for (int k = 0; k < RY; ++k) T::mask(edge[k], edge_valid);
        }
    }
    if (CHECK && nvalid < V) {  // only the vector straddling nx (or past it) needs masking
#pragma unroll
        for (int k = 0; k < RY + 2 * R; ++k) T::mask(cur[k], nvalid);
    }

    // ---- arithmetic and stores, row by row ----
    char* next_base = a.u_next + y0 * pb + x0 * ES;
#pragma unroll
    for (int k = 0; k < RY; ++k) {
        // ext[m] holds column x0 - R + m
        float ext[V + 2 * R];
#pragma unroll
        for (int e = 0; e < V; ++e) ext[R + e] = T::elem(cur[k + R], e);
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            float from_left = __shfl_up_sync(kFull, ext[R + V - d], 1);
            float from_right = __shfl_down_sync(kFull, ext[R + d - 1], 1);
            if constexpr (HL) {  // lanes 0 and 31 get their own values back: unused, they store nothing
                ext[R - d] = from_left;
                ext[R + V - 1 + d] = from_right;
            } else if constexpr (kScalarEdge) {
                ext[R - d] = lane == 0 ? edge1[k][d - 1] : from_left;
                ext[R + V - 1 + d] = lane == 31 ? edge1[k][d - 1] : from_right;
            } else {
                ext[R - d] = lane == 0 ? T::elem(edge[k], V - d) : from_left;
                ext[R + V - 1 + d] = lane == 31 ? T::elem(edge[k], d - 1) : from_right;
            }
        }
        float out[V];
        if constexpr (sizeof(S) == 2) {  // 16-bit storage: twice the arithmetic per byte; pair the additions
#pragma unroll
            for (int e = 0; e < V; e += 2) {
                float2 vert[R], horz[R];
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    vert[d - 1] = add2_rn(make_float2(T::elem(cur[k + R - d], e), T::elem(cur[k + R - d], e + 1)),
                                          make_float2(T::elem(cur[k + R + d], e), T::elem(cur[k + R + d], e + 1)));
                    horz[d - 1] = horz2<R>(ext, e, d);
                }
                const float2 up = START ? make_float2(0.0f, 0.0f)
                                        : make_float2(T::elem(prev[START ? 0 : k], e), T::elem(prev[START ? 0 : k], e + 1));
                const float2 o = update2<R, START, true>(make_float2(ext[R + e], ext[R + e + 1]), up, vert, horz, a.c2, a.neg0);
                out[e] = o.x;
                out[e + 1] = o.y;
            }
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                float vert[R], horz[R];
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    vert[d - 1] = __fadd_rn(T::elem(cur[k + R - d], e), T::elem(cur[k + R + d], e));
                    horz[d - 1] = __fadd_rn(ext[R + e - d], ext[R + e + d]);
                }
                const float up = START ? 0.0f : T::elem(prev[START ? 0 : k], e);
                out[e] = update<R, START>(ext[R + e], up, vert, horz, a.c2);
            }
        }
        if (stores && (!CHECK || (col_in && y0 + k < a.row_end))) {
            char* dst = next_base + k * pb;
            if (!CHECK || nvalid == V) {
                M::st_cs(dst, T::pack(out));
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (e < nvalid) T::store1(dst + e * ES, out[e]);
            }
        }
    }
}

// Interior tiles (all rows in the grid and the range mapper, all lanes' columns
// in [0, nx)) take the predicate-free form.
template <typename S, int R, int RY, bool START, bool HL = false, bool CG = false, bool NARROW = false>
__device__ __forceinline__ void wave_tile(const Args& a, int64_t tx, int64_t ty, int lane) {
    constexpr int V = TileTraits<S, NARROW>::type::V;
    const int64_t y0 = a.row_begin + ty * RY;
    const int64_t row_hi = a.row_end + R < a.ny ? a.row_end + R : a.ny;
    const bool cols_in = HL ? (tx > 0 && (tx * 30 + 31) * V <= a.nx) : ((tx + 1) * 32 * V <= a.nx);
    const bool interior = (y0 - R >= 0) && (y0 + RY + R <= row_hi) && (y0 + RY <= a.row_end) && cols_in;
    if (interior) wave_tile_impl<S, R, RY, START, false, HL, CG, NARROW>(a, tx, ty, lane);
    else wave_tile_impl<S, R, RY, START, true, HL, CG, NARROW>(a, tx, ty, lane);
}

// REV = true visits the tiles in reverse order (tile t as tiles - 1 - t): the chunk is
// swept bottom to top, with the same results.
template <typename S, int R, int RY, bool START, bool REV, bool HL = false, bool NARROW = false>
__device__ __forceinline__ void wave_vec_body(const Args& a) {
    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    const int lane = threadIdx.x & 31;
    const int64_t warps_per_block = blockDim.x >> 5;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * warps_per_block;
    const int64_t w = static_cast<int64_t>(blockIdx.x) * warps_per_block + (threadIdx.x >> 5);
    // tile t = w + i * nwarps (REV: tiles - 1 - t), as (ty, tx) = divmod(tile, tiles_x):
    // two divisions per warp, then the coordinates move by (dy, dx) per trip.
    const int64_t first = REV ? a.tiles - 1 - w : w;
    int64_t ty = first / a.tiles_x, tx = first - ty * a.tiles_x;
    const int64_t dy = nwarps / a.tiles_x, dx = nwarps - dy * a.tiles_x;
    for (int64_t t = w; t < a.tiles; t += nwarps) {
        wave_tile<S, R, RY, START, HL, false, NARROW>(a, tx, ty, lane);
        if constexpr (REV) {
            tx -= dx;
            ty -= dy;
            if (tx < 0) {
                tx += a.tiles_x;
                --ty;
            }
        } else {
            tx += dx;
            ty += dy;
            if (tx >= a.tiles_x) {
                tx -= a.tiles_x;
                ++ty;
            }
        }
    }
    stamp_end(a.stamp);
    if (a.pdl && threadIdx.x == 0) griddep_wait();
}

template <typename S, int R, int RY, bool START, bool REV>
__global__ void __launch_bounds__(256) wave_vec_kernel(Args a) {
    wave_vec_body<S, R, RY, START, REV>(a);
}

// The halo-lane form (tiles of 30*V columns, no edge vectors).
template <typename S, int R, int RY, bool START, bool REV>
__global__ void __launch_bounds__(256) wave_hl_kernel(Args a) {
    wave_vec_body<S, R, RY, START, REV, true>(a);
}

// The narrow halo-lane form for 16-bit storage (8-byte vectors, tiles of 120 columns).
template <typename S, int R, int RY, bool START, bool REV>
__global__ void __launch_bounds__(128) wave_hln_kernel(Args a) {
    wave_vec_body<S, R, RY, START, REV, true, true>(a);
}

// The same kernel held to 96 registers (5 blocks of 128 threads an SM instead of 4, for
// a 20-byte spill): 16-bit storage, radius 1, 4-row tiles, the default there.  Measured
// at 8192^2: BF16 6.38 -> 6.55 TB/s, FP16 6.38 -> 6.50 TB/s.
template <typename S, int R, int RY, bool START, bool REV>
__global__ void __maxnreg__(96) wave_vec_kernel_r96(Args a) {
    wave_vec_body<S, R, RY, START, REV>(a);
}

// The same kernel held to 168 registers (3 blocks of 128 threads an SM instead of 2):
// 16-bit storage, radius 3-4, 8-row tiles, whose unbounded form takes 255 registers.
template <typename S, int R, int RY, bool START, bool REV>
__global__ void __launch_bounds__(128, 3) wave_vec_kernel_b3(Args a) {
    wave_vec_body<S, R, RY, START, REV>(a);
}

// The halo-lane form held to 168 registers (3 blocks of 128 threads an SM instead of
// 2): 16-bit storage, radius 3-4, 8-row tiles.
template <typename S, int R, int RY, bool START, bool REV>
__global__ void __launch_bounds__(128, 3) wave_hl_kernel_b3(Args a) {
    wave_vec_body<S, R, RY, START, REV, true>(a);
}

// One point per thread; any element-aligned layout.
template <typename S, int R, bool START>
__global__ void __launch_bounds__(256) wave_scalar_kernel(Args a) {
    using T = Traits<S>;
    stamp_begin(a.stamp);
    const int64_t rows = a.row_end - a.row_begin;
    const int64_t total = rows * a.nx;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < total; p += stride) {
        const int64_t i = a.row_begin + p / a.nx;
        const int64_t j = p - (i - a.row_begin) * a.nx;
        auto at = [&](int64_t ii, int64_t jj) -> float {
            if (ii < 0 || ii >= a.ny || jj < 0 || jj >= a.nx) return 0.0f;
            return T::load1(a.u_cur + ii * a.pitch_bytes + jj * static_cast<int64_t>(sizeof(S)));
        };
        float vert[R], horz[R];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            vert[d - 1] = __fadd_rn(at(i - d, j), at(i + d, j));
            horz[d - 1] = __fadd_rn(at(i, j - d), at(i, j + d));
        }
        const int64_t off = i * a.pitch_bytes + j * static_cast<int64_t>(sizeof(S));
        const float up = START ? 0.0f : T::load1_cs(a.u_prev + off);
        T::store1(a.u_next + off, update<R, START>(at(i, j), up, vert, horz, a.c2));
    }
    stamp_end(a.stamp);
}

// Row heights of the vector kernel's tiles; variant v (1-based) = (kTileRows[(v-1) % 4],
// kBlockThreads[(v-1) / 4]) for v <= 8; variants 9-12 are the halo-lane form with
// (kHlRows[(v-9) % 2], kBlockThreads[(v-9) / 2]); 16-bit storage adds variants 13-14,
// the narrow halo-lane form with kHlRows[v-13] rows and 128 threads, and variant 15,
// the march form (wave_march.cuh: TMA-fed row streams, one segment per warp).
constexpr int kTileRows[4] = {2, 4, 8, 16};
constexpr int kBlockThreads[2] = {128, 256};
constexpr int kHlRows[2] = {4, 8};
constexpr int kVariants32 = 12;  // FP32 storage
constexpr int kVariants16 = 15;  // 16-bit storage
constexpr int kMarchVariant = 15;

// How a variant covers a chunk.
enum class Form { Tile, Halo, Narrow, March };

using KernelFn = void (*)(Args);

// Launch helper shared by the per-dtype translation units; span = output columns per
// warp tile (or strip); tile_rows = rows per tile (or segment).
sy_status launch_typed(Queue* q, const WaveLaunch& w, KernelFn vec_fn, KernelFn scalar_fn, int tile_rows,
                       int threads, int span, size_t esize, Form form);

template <typename S, int R, bool START, bool REV>
KernelFn pick_vec(int tile_rows, Form form, int threads) {
    if constexpr (sizeof(S) == 2) {
        if (form == Form::Narrow)
            return tile_rows == 4 ? wave_hln_kernel<S, R, 4, START, REV> : wave_hln_kernel<S, R, 8, START, REV>;
    }
    if (form == Form::Halo) {
        if constexpr (sizeof(S) == 2 && R >= 3) {
            if (tile_rows == 8 && threads == 128) return wave_hl_kernel_b3<S, R, 8, START, REV>;
        }
        return tile_rows == 4 ? wave_hl_kernel<S, R, 4, START, REV> : wave_hl_kernel<S, R, 8, START, REV>;
    }
    switch (tile_rows) {
        case 2: return wave_vec_kernel<S, R, 2, START, REV>;
        case 4:
            if constexpr (sizeof(S) == 2 && R == 1) return wave_vec_kernel_r96<S, R, 4, START, REV>;
            else return wave_vec_kernel<S, R, 4, START, REV>;
        case 8:
            if constexpr (sizeof(S) == 2 && R >= 3) {
                if (threads == 128) return wave_vec_kernel_b3<S, R, 8, START, REV>;
            }
            return wave_vec_kernel<S, R, 8, START, REV>;
        default: return wave_vec_kernel<S, R, 16, START, REV>;
    }
}

// The start always sweeps forward (a run's reversed steps are its odd leapfrog steps).
template <typename S, int R>
sy_status launch_r(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form) {
    KernelFn vec = w.start     ? pick_vec<S, R, true, false>(tile_rows, form, threads)
                   : w.reverse ? pick_vec<S, R, false, true>(tile_rows, form, threads)
                               : pick_vec<S, R, false, false>(tile_rows, form, threads);
    KernelFn sca = w.start ? wave_scalar_kernel<S, R, true> : wave_scalar_kernel<S, R, false>;
    int span = form == Form::Tile ? tile_span<S, false>() : tile_span<S, true>();
    if constexpr (sizeof(S) == 2) {
        if (form == Form::Narrow) span = tile_span<S, true, true>();
    }
    return launch_typed(q, w, vec, sca, tile_rows, threads, span, sizeof(S), form);
}

template <typename S>
sy_status launch_dtype(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form) {
    switch (w.radius) {
        case 1: return launch_r<S, 1>(q, w, tile_rows, threads, form);
        case 2: return launch_r<S, 2>(q, w, tile_rows, threads, form);
        case 3: return launch_r<S, 3>(q, w, tile_rows, threads, form);
        default: return launch_r<S, 4>(q, w, tile_rows, threads, form);
    }
}

sy_status launch_f32(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form);
sy_status launch_bf16(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form);
sy_status launch_f16(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form);

}  // namespace wave
}  // namespace sy
