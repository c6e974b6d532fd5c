// eik_cells_f32.cu -- FP32 instantiations of the persistent cell kernel
// (bulk sweeps of the FP32 + FP64-polish precision mode).
#include "eik_cells_launch.cuh"

namespace eik {

cudaError_t launch_cells_f32(int n, const CellKernelParams& p, int sms, cudaStream_t st,
                             int* grid_out, int& launches, int wpc) {
  switch (n) {
    case 4: return launch_cells_t<float, 4, false, true>(p, sms, st, grid_out, launches, wpc);
    case 8: return launch_cells_t<float, 8, false, true>(p, sms, st, grid_out, launches, wpc);
    case 16: return launch_cells_t<float, 16, false, true>(p, sms, st, grid_out, launches, wpc);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace eik
