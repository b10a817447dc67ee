// Split-DD instances of the persistent evolve kernel, 13-point stencil (every model).
#include "persist.cuh"

namespace pycool {
cudaError_t launch_persist_dd_wide(int model, int stencil, int vx, const PParams& p, int grid,
                                   cudaStream_t s, int* bps) {
  return launch_persist_impl<PREC_DD, true>(model, stencil, vx, p, grid, s, bps);
}
}  // namespace pycool
