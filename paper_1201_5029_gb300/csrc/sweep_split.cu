// Split-FP32 instances of the fused stage sweep (every model x stencil).
#include "sweep.cuh"

namespace pycool {
cudaError_t launch_sweep_split(int model, int stencil, int vx, int tma, const LaunchTable& t, int grid,
                               cudaStream_t s) {
  return launch_sweep_impl<PREC_SPLIT>(model, stencil, vx, tma, t, grid, s);
}
}  // namespace pycool
