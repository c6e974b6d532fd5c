// eik_cells_f64.cu -- FP64 instantiations of the persistent cell kernel:
// monotone (min) sweeps of the FP64 mode and replace-mode polishing sweeps.
#include "eik_cells_launch.cuh"

namespace eik {

cudaError_t launch_cells_f32(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                             int* grid_out, int& launches);
void cells_shape_f32(int n, int* threads, int* smem, int* workers);

cudaError_t launch_cells(bool fp64, bool replace, int n, const CellKernelParams& p, int sms,
                         cudaStream_t st, int* grid_out, int& launches) {
  if (!fp64) {
    if (replace) return cudaErrorInvalidValue;
    return launch_cells_f32(n, p, sms, st, grid_out, launches);
  }
  if (replace) {
    switch (n) {
      case 4: return launch_cells_t<double, 4, true>(p, sms, st, grid_out, launches);
      case 8: return launch_cells_t<double, 8, true>(p, sms, st, grid_out, launches);
      case 16: return launch_cells_t<double, 16, true>(p, sms, st, grid_out, launches);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (n) {
    case 4: return launch_cells_t<double, 4, false>(p, sms, st, grid_out, launches);
    case 8: return launch_cells_t<double, 8, false>(p, sms, st, grid_out, launches);
    case 16: return launch_cells_t<double, 16, false>(p, sms, st, grid_out, launches);
    default: return cudaErrorInvalidValue;
  }
}

void cells_kernel_shape(bool fp64, int n, int* threads, int* smem, int* workers) {
  if (!fp64) {
    cells_shape_f32(n, threads, smem, workers);
    return;
  }
  switch (n) {
    case 4: shape_t<double, 4>(threads, smem, workers); break;
    case 8: shape_t<double, 8>(threads, smem, workers); break;
    default: shape_t<double, 16>(threads, smem, workers); break;
  }
}

}  // namespace eik
