// TMA form of the 3D step for f32 storage (all radii, strips of 8 and 16 rows, step
// and start forms).  The kernel is in wave3d_tma.cuh.
#include "wave3d_tma.cuh"

namespace sy {
namespace wave3 {

sy_status launch3_tma_f32(Queue* q, const WaveLaunch3& w, int rows) { return launch_tma_dtype<float>(q, w, rows); }

}  // namespace wave3
}  // namespace sy
