// Wave-step kernel instantiations for bf16 storage (all radii, tile heights,
// step and start forms, and the march form).  The kernels themselves are in wave_kernel.cuh.
#include "wave_kernel.cuh"
#include "wave_march.cuh"

namespace sy {
namespace wave {

sy_status launch_bf16(Queue* q, const WaveLaunch& w, int tile_rows, int threads, Form form) {
    if (form == Form::March) return march::launch_march<__nv_bfloat16>(q, w);
    return launch_dtype<__nv_bfloat16>(q, w, tile_rows, threads, form);
}

}  // namespace wave
}  // namespace sy
