// 3D wave-step kernel instantiations for f32 storage (all radii, tile heights,
// step and start forms).  The kernels themselves are in wave3d_kernel.cuh.
#include "wave3d_kernel.cuh"

namespace sy {
namespace wave3 {

sy_status launch3_f32(Queue* q, const WaveLaunch3& w, int rows, int threads) {
    return launch3_dtype<float>(q, w, rows, threads);
}

}  // namespace wave3
}  // namespace sy
