// Wave-step kernel instantiations for f16 storage (all radii, tile heights,
// step and start forms, and the march form).  The kernels themselves are in wave_kernel.cuh.
#include "wave_kernel.cuh"
#include "wave_march.cuh"

namespace sy {
namespace wave {

sy_status launch_f16(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form) {
    if (form == Form::March) return march::launch_march<__half>(q, w);
    return launch_dtype<__half>(q, w, tile_rows, threads, form);
}

}  // namespace wave
}  // namespace sy
