// eik_cells_f64.cu -- FP64 min-mode instantiations of the persistent cell
// kernel (the sweeps of the FP64 mode and the monotone polish), and the
// dispatch over value type, mode, cell size and worker shape.
#include "eik_cells_launch.cuh"

namespace eik {

cudaError_t launch_cells_f32(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                             int* grid_out, int& launches, int wpc);
cudaError_t launch_cells_f64_replace(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                                     int* grid_out, int& launches);

cudaError_t launch_cells(bool fp64, bool replace, int n, const CellKernelParams& p, int sms,
                         cudaStream_t st, int* grid_out, int& launches, int wpc) {
  if (!fp64) {
    if (replace) return cudaErrorInvalidValue;
    return launch_cells_f32(n, p, sms, st, grid_out, launches, wpc);
  }
  if (replace) return launch_cells_f64_replace(n, p, sms, st, grid_out, launches);
  switch (n) {
    case 4: return launch_cells_t<double, 4, false, true>(p, sms, st, grid_out, launches, wpc);
    case 8: return launch_cells_t<double, 8, false, true>(p, sms, st, grid_out, launches, wpc);
    case 16: return launch_cells_t<double, 16, false, true>(p, sms, st, grid_out, launches, wpc);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace eik
