// eik_cells_f64r.cu -- FP64 replace-mode instantiations of the persistent
// cell kernel (the polish fallback; default worker shapes only).
#include "eik_cells_launch.cuh"

namespace eik {

cudaError_t launch_cells_f64_replace(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                                     int* grid_out, int& launches) {
  switch (n) {
    case 4: return launch_cells_t<double, 4, true, false>(p, sms, st, grid_out, launches, 0);
    case 8: return launch_cells_t<double, 8, true, false>(p, sms, st, grid_out, launches, 0);
    case 16: return launch_cells_t<double, 16, true, false>(p, sms, st, grid_out, launches, 0);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace eik
