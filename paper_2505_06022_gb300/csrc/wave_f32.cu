// Wave-step kernel instantiations for f32 storage (all radii, tile heights,
// step and start forms).  The kernels themselves are in wave_kernel.cuh.
#include "wave_kernel.cuh"

namespace sy {
namespace wave {

sy_status launch_f32(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form) {
    return launch_dtype<float>(q, w, tile_rows, threads, form);
}

}  // namespace wave
}  // namespace sy
