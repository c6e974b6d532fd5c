// eik_cells_f32.cu -- FP32 instantiations of the persistent cell kernel
// (bulk sweeps of the FP32 + FP64-polish precision mode).
#include "eik_cells_launch.cuh"

namespace eik {

cudaError_t launch_cells_f32(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                             int* grid_out, int& launches) {
  switch (n) {
    case 4: return launch_cells_t<float, 4, false>(p, sms, st, grid_out, launches);
    case 8: return launch_cells_t<float, 8, false>(p, sms, st, grid_out, launches);
    case 16: return launch_cells_t<float, 16, false>(p, sms, st, grid_out, launches);
    default: return cudaErrorInvalidValue;
  }
}

void cells_shape_f32(int n, int* threads, int* smem, int* workers) {
  switch (n) {
    case 4: shape_t<float, 4>(threads, smem, workers); break;
    case 8: shape_t<float, 8>(threads, smem, workers); break;
    default: shape_t<float, 16>(threads, smem, workers); break;
  }
}

}  // namespace eik
