// TMA form of the 3D step (variants 9-10): a block of 8 warps marches a strip of
// RB = 8*RYW rows through the planes of a segment, with every plane it reads
// copied into shared memory by TMA ahead of use.
//
//   * A plane slot holds the strip's rows plus R halo rows above and below, 32
//     16-byte column groups wide: lane g owns group g; groups 0 and 31 are the x
//     halo (their results are discarded), so a tile writes 30 groups.  Points
//     outside the grid arrive as zeros (the copy's out-of-bounds fill), which are
//     the Dirichlet ghosts.
//   * A ring of 2R+1+kTmaAhead slots holds planes z-R .. z+R and the planes
//     copied ahead; each slot completes on its own mbarrier.  Per plane the block
//     computes plane z entirely from shared memory (vertical and depth
//     neighbours) and warp shuffles (horizontal), then waits for plane z+1+R, and
//     one barrier both frees the slot of plane z-R, into which the elected thread
//     copies plane z+R+kTmaAhead+1, and publishes the next plane to every warp.  u^{n-1} is read straight from global memory one plane ahead.
//   * Every wait is bounded; on expiry the block sets an error flag, waits
//     (bounded) for its copies in flight and returns; the host reports SY_ERR_TIMEOUT.
#pragma once

#include <mutex>

#include "tma.cuh"
#include "wave3d_kernel.cuh"

namespace sy {
namespace wave3 {

constexpr int kTmaWarps = 8;
constexpr int kTmaAhead = 2;  // planes copied beyond the one the current step needs last

template <typename S, int R, int RYW>
struct TmaGeo {
    static constexpr int V = Traits<S>::V;
    static constexpr int W = 32 * V;                       // box width in elements: 32 groups
    static constexpr int BX = W - 2 * V;                   // output columns of a tile
    static constexpr int RB = kTmaWarps * RYW;             // output rows of a strip
    static constexpr int H = RB + 2 * R;                   // box height
    static constexpr int ROW_U4 = 32;                      // uint4 per slot row
    static constexpr int SLOT_U4 = H * ROW_U4;
    static constexpr int SLOT = SLOT_U4 * 16;              // bytes per plane slot (= box bytes)
    static constexpr int NS = 2 * R + 1 + kTmaAhead;       // ring slots
    static constexpr int SMEM = NS * SLOT + NS * 8 + NS * 4;
    static_assert(R <= V, "radius must not exceed the vector width");
    static_assert(W * sizeof(S) == 512, "a slot row is 32 groups of 16 bytes");
};

template <typename S, int R, int RYW, bool START>
__global__ void __launch_bounds__(kTmaWarps * 32) wave3d_tma_kernel(const __grid_constant__ CUtensorMap map_cur,
                                                                    Args3 a, unsigned* err, int fault) {
    using G = TmaGeo<S, R, RYW>;
    using T = Traits<S>;
    constexpr int V = T::V;
    constexpr int64_t ES = sizeof(S);
    extern __shared__ __align__(128) unsigned char smem[];
    uint4* slots = reinterpret_cast<uint4*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::NS * G::SLOT);
    unsigned* fills = reinterpret_cast<unsigned*>(smem + G::NS * G::SLOT + G::NS * 8);  // fills issued per slot
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (a.pdl == 1) griddep_wait();
    if (a.pdl) griddep_launch_dependents();
    stamp_begin(a.stamp);
    if (tid == 0) {
        for (int s = 0; s < G::NS; ++s) {
            tma::mbar_init(&bars[s], 1);
            fills[s] = 0u;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int64_t pb = a.pitch_bytes, zb = a.plane_bytes;
    bool first_copy = true;
    for (int64_t t = blockIdx.x; t < a.tasks; t += gridDim.x) {  // block-uniform
        const int64_t rest = t / a.tiles_x;
        const int64_t tx = t - rest * a.tiles_x;
        const int64_t sg = rest / a.tiles_y;
        const int64_t tb = rest - sg * a.tiles_y;
        const int x_box = static_cast<int>(tx * G::BX) - V;  // column of group 0
        const int64_t yb = tb * G::RB;
        const int64_t za = a.z_begin + sg * a.seg;
        const int64_t ze = za + a.seg < a.z_end ? za + a.seg : a.z_end;
        const int64_t base = za - R;   // plane held by slot 0
        const int64_t last = ze - 1 + R;  // last plane this task reads
        auto slot_of = [&](int64_t p) { return static_cast<int>((p - base) % G::NS); };
        auto issue = [&](int64_t p) {  // elected thread only
            const int s = slot_of(p);
            ++fills[s];
            if (p < 0 || p >= a.nz) {  // a plane outside the grid: ghosts, zeros (no copy)
                uint4* d = slots + s * G::SLOT_U4;
                for (int i = 0; i < G::SLOT_U4; ++i) d[i] = make_uint4(0u, 0u, 0u, 0u);
                tma::mbar_expect_tx(&bars[s], 0u);  // arrival with release: the zeros are visible to waiters
                return;
            }
            tma::fence_proxy_async();  // earlier generic reads of this slot come first
            tma::mbar_expect_tx(&bars[s], G::SLOT);
            if (!(fault && first_copy))
                tma::load_3d(slots + s * G::SLOT_U4, &map_cur, x_box, static_cast<int>(yb - R), static_cast<int>(p),
                             &bars[s]);
            first_copy = false;
        };
        auto wait = [&](int64_t p) { const int s = slot_of(p); return tma::mbar_wait_bounded(&bars[s], (fills[s] - 1u) & 1u); };

        int64_t issued = za + R + kTmaAhead < last ? za + R + kTmaAhead : last;  // last plane issued so far
        if (tid == 0)
            for (int64_t p = za - R; p <= issued; ++p) issue(p);
        __syncthreads();  // fills[] visible to every waiter

        // u^{n-1} of this warp's rows, one plane ahead
        const int64_t x0 = x_box + static_cast<int64_t>(lane) * V;
        const bool useful = lane >= 1 && lane <= 30 && x0 < a.nx;
        const int nvalid = useful ? static_cast<int>(a.nx - x0 < V ? a.nx - x0 : V) : 0;
        const int64_t y0 = yb + warp * RYW;
        uint4 pv[RYW];
        auto load_prev = [&](int64_t z) {
#pragma unroll
            for (int k = 0; k < RYW; ++k) {
                pv[k] = make_uint4(0u, 0u, 0u, 0u);
                if (!START && useful && y0 + k < a.ny)
                    pv[k] = __ldcs(reinterpret_cast<const uint4*>(a.u_prev + z * zb + (y0 + k) * pb + x0 * ES));
            }
        };
        load_prev(za);

        bool ok = true;
        for (int64_t p = za - R; p <= za + R; ++p) ok = wait(p) && ok;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(err, 1u);
                for (int64_t p = za - R; p <= issued; ++p) wait(p);  // let this block's copies land
            }
            stamp_end(a.stamp);
            if (a.pdl && tid == 0) griddep_wait();
            return;  // the whole block returns: no barrier below is left half-reached
        }
        for (int64_t z = za; z < ze; ++z) {
            // planes z-R .. z+R are in place (the barrier ending the previous step saw them)
            uint4 cur_pv[RYW];
#pragma unroll
            for (int k = 0; k < RYW; ++k) cur_pv[k] = pv[k];
            if (z + 1 < ze) load_prev(z + 1);

            const uint4* cz = slots + slot_of(z) * G::SLOT_U4;
            char* nbase = a.u_next + z * zb;
#pragma unroll
            for (int k = 0; k < RYW; ++k) {
                const int row = R + warp * RYW + k;  // slot row of output row y0 + k
                uint4 up[R], dn[R], zm[R], zp[R];
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    up[d - 1] = cz[(row - d) * G::ROW_U4 + lane];
                    dn[d - 1] = cz[(row + d) * G::ROW_U4 + lane];
                    zm[d - 1] = slots[slot_of(z - d) * G::SLOT_U4 + row * G::ROW_U4 + lane];
                    zp[d - 1] = slots[slot_of(z + d) * G::SLOT_U4 + row * G::ROW_U4 + lane];
                }
                const float no_edge[R] = {};
                float out[V];
                row_update<S, R, START>(cz[row * G::ROW_U4 + lane], up, dn, zm, zp, cur_pv[k], no_edge, lane, a.c2,
                                        a.neg0, out);
                if (useful && y0 + k < a.ny) {
                    char* dst = nbase + (y0 + k) * pb + x0 * ES;
                    if (nvalid == V) {
                        __stcs(reinterpret_cast<uint4*>(dst), T::pack(out));
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e)
                            if (e < nvalid) T::store1(dst + e * ES, out[e]);
                    }
                }
            }
            // one barrier per step: every read of plane z-R's slot is done, and plane z+1+R
            // (needed next) has landed for every thread
            if (z + 1 < ze) ok = wait(z + 1 + R);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    atomicOr(err, 1u);
                    for (int64_t p = z + 1 - R; p <= issued; ++p) wait(p);  // let this block's copies land
                }
                stamp_end(a.stamp);
                if (a.pdl && tid == 0) griddep_wait();
                return;
            }
            if (issued < last) {
                ++issued;  // = z + R + kTmaAhead + 1, into the slot plane z - R held
                if (tid == 0) issue(issued);
            }
        }
        __syncthreads();  // the slots are free for the block's next task
    }
    stamp_end(a.stamp);
    if (a.pdl && tid == 0) griddep_wait();
}

int64_t choose_seg(int64_t tiles_xy, int64_t planes, int64_t workers, int R);

template <typename S, int R, int RYW, bool START>
sy_status launch_tma(Queue* q, const WaveLaunch3& w) {
    using G = TmaGeo<S, R, RYW>;
    auto kern = wave3d_tma_kernel<S, R, RYW, START>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(3D TMA smem)");
    auto enc = tma::encoder();
    if (!enc) return fail(SY_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    const int64_t es = sizeof(S);
    CUtensorMap map;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(w.nx), static_cast<cuuint64_t>(w.ny),
                                static_cast<cuuint64_t>(w.nz)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(w.pitch * es), static_cast<cuuint64_t>(w.plane * es)};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(G::W), static_cast<cuuint32_t>(G::H), 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(&map, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                           const_cast<void*>(w.u_cur), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(SY_ERR_INVALID_ARGUMENT, "cuTensorMapEncodeTiled (3D) failed (%d)", static_cast<int>(r));
    Args3 a;
    a.u_prev = static_cast<const char*>(w.u_prev);
    a.u_cur = static_cast<const char*>(w.u_cur);
    a.u_next = static_cast<char*>(w.u_next);
    a.nz = w.nz;
    a.ny = w.ny;
    a.nx = w.nx;
    a.pitch_bytes = w.pitch * es;
    a.plane_bytes = w.plane * es;
    a.z_begin = w.z_begin;
    a.z_end = w.z_end;
    a.c2 = w.c2;
    a.stamp = q->cur_stamp;
    a.pdl = 0;
    a.neg0 = -0.0f;
    const int64_t planes = w.z_end - w.z_begin;
    a.tiles_x = (w.nx + G::BX - 1) / G::BX;
    a.tiles_y = (w.ny + G::RB - 1) / G::RB;
    int occ = 0;
    SY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaWarps * 32, G::SMEM));
    if (occ < 1) return fail(SY_ERR_UNSUPPORTED, "3D TMA kernel does not fit on an SM");
    const int64_t cap = static_cast<int64_t>(occ) * q->sm_count;
    a.seg = choose_seg(a.tiles_x * a.tiles_y, planes, cap, R);
    a.segs = (planes + a.seg - 1) / a.seg;
    a.tasks = a.tiles_x * a.tiles_y * a.segs;
    const int64_t blocks = a.tasks < cap ? a.tasks : cap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(kTmaWarps * 32);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = q->launch;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (w.pdl && wave::launch_overlap_enabled()) {
        a.pdl = w.pdl;
        cfg.numAttrs = 1;
    }
    SY_CUDA(cudaLaunchKernelEx(&cfg, kern, map, a, q->d_flags, fault_enabled("w3_timeout") ? 1 : 0));
    ++q->launches;
    q->cur_blocks += static_cast<uint64_t>(blocks);
    return SY_OK;
}

// rows: the strip height, 16 or 32
template <typename S, int R>
sy_status launch_tma_r(Queue* q, const WaveLaunch3& w, int rows) {
    if (rows == 16) return w.start ? launch_tma<S, R, 2, true>(q, w) : launch_tma<S, R, 2, false>(q, w);
    return w.start ? launch_tma<S, R, 4, true>(q, w) : launch_tma<S, R, 4, false>(q, w);
}

template <typename S>
sy_status launch_tma_dtype(Queue* q, const WaveLaunch3& w, int rows) {
    switch (w.radius) {
        case 1: return launch_tma_r<S, 1>(q, w, rows);
        case 2: return launch_tma_r<S, 2>(q, w, rows);
        case 3: return launch_tma_r<S, 3>(q, w, rows);
        default: return launch_tma_r<S, 4>(q, w, rows);
    }
}

sy_status launch3_tma_f32(Queue* q, const WaveLaunch3& w, int rows);
sy_status launch3_tma_bf16(Queue* q, const WaveLaunch3& w, int rows);
sy_status launch3_tma_f16(Queue* q, const WaveLaunch3& w, int rows);

}  // namespace wave3
}  // namespace sy
