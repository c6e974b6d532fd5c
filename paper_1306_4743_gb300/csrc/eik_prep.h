// eik_prep.h -- descriptors and launchers of the streaming kernels in
// eik_prep.cu (internal to libeik.so).
#pragma once
#include "eik_internal.h"

namespace eik {

// Init of one instance for the bulk pass.
struct PrepInstance {
  const float* F;
  const uint8_t* mask;
  const double* q;
  double h;
  void* u;        // padded values of the bulk pass (float or double)
  void* s;        // cell-blocked slowness of the bulk pass
  void* s64;      // cell-blocked FP64 slowness for the polish, or null
  long long px, py, pz;
  int nx, ny, nz;
  int ncx, ncy, ncz;
  int cell_base, ncells;
  int n;
};

// FP32 -> FP64 hand-over of one instance.
struct PolishInstance {
  const uint8_t* mask;   // exit nodes take q exactly, not its FP32 rounding
  const double* q;
  const void* u32;
  void* u64;
  const void* s64;
  long long px32, px64, py, pz;
  int nx, ny, nz;
  int ncx, ncy, ncz;
  int cell_base, ncells;
  int n;
};

// Residual check and copy-out of one instance.
struct FinalInstance {
  const uint8_t* mask;   // exit nodes are copied out as q exactly
  const double* q;
  const void* u64;
  const void* s64;
  double* out;
  long long px64, py, pz;
  int nx, ny, nz;
  int ncx, ncy, ncz;
  int n;
};

cudaError_t launch_bulk_init(const PrepInstance* d_pi, int count, long long max_padded,
                             long long max_cellnodes, long long max_nodes, int max_cells,
                             int total_cells, CellArrays cells, Control* ctl, int* n_src, bool fp64,
                             int n, double width_factor, double kappa_rel, int sms,
                             cudaStream_t st);
cudaError_t launch_polish_prep(const PolishInstance* d_pi, int count, long long max_padded64,
                               long long max_nodes, int max_cells, int total_cells,
                               CellArrays cells, Control* ctl, int sms, cudaStream_t st);
cudaError_t launch_fallback_prep(const PolishInstance* d_pi, const FinalInstance* d_fi, int count,
                                 long long max_rows, int max_cells, int total_cells,
                                 CellArrays cells, Control* ctl, double kappa, int sms,
                                 cudaStream_t st);
// max_rows: the largest ny * nz of the launch.  after_fallback: the pass
// after the replace-mode fallback (a no-op on the device unless it ran);
// otherwise the final pass of the FP64 path.
cudaError_t launch_residual_extract(const FinalInstance* d_fi, int count, long long max_rows,
                                    Control* ctl, bool after_fallback, double kappa, int sms,
                                    cudaStream_t st);

// Persistent cell kernels (eik_cells_f32.cu / eik_cells_f64.cu).
cudaError_t launch_cells(bool fp64, bool replace, int n, const CellKernelParams& p, int sms,
                         cudaStream_t st, int* grid_out);

// Shared memory bytes and threads of the cell kernel for (type, n).
void cells_kernel_shape(bool fp64, int n, int* threads, int* smem_bytes, int* workers);

}  // namespace eik
