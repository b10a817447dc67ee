// Split-DD instances of the persistent evolve kernel (every model x stencil).
#include "persist.cuh"

namespace pycool {
cudaError_t launch_persist_dd(int model, int stencil, int vx, const PParams& p, int grid,
                              cudaStream_t s, int* bps) {
  return launch_persist_impl<PREC_DD>(model, stencil, vx, p, grid, s, bps);
}
}  // namespace pycool
