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

// Block schedule of the streaming kernels.  Their blocks are spread over the
// instances of a launch in proportion to each instance's work, so a batch of
// uneven grids launches no idle blocks and no block needs a division of a
// 64-bit index: a block takes kRowsPerBlock rows (fixed j, k) of one
// instance, one warp per row with its lanes striding over i (rows of small
// grids are short), or kCellsPerBlock cells.
//   rows of the padded bulk array   py * pz       (row length px of the pass)
//   rows of the padded FP64 array   py * pz       (px64)
//   grid rows                       ny * nz       (nx)
//   rows of the cell-blocked array  (n ncy) * (n ncz)   (n ncx)
//   cells                           ncells
enum SegKind { kSegPadB = 0, kSegPad64, kSegRows, kSegCellRows, kSegCells, kNumSegKinds };
constexpr int kRowsPerBlock = 32;
constexpr int kCellsPerBlock = 16;  // 8 warps, 2 cells each

// Work of one instance in the units above.
struct SegSizes {
  long long units[kNumSegKinds];
};

// seg table on the device: (count + 1) ints per kind, seg[k (count + 1) + t]
// = first block of instance t, ... + count = total blocks of kind k; the
// host keeps the totals for the launch sizes.
struct Segments {
  const int* dev;
  int count;
  int total[kNumSegKinds];
};

// Fills host_seg ((count + 1) * kNumSegKinds ints) and totals.
void make_segments(int count, const SegSizes* sizes, int* host_seg, int* totals);
size_t segment_table_bytes(int count);

// Every launcher adds the number of kernels it launched to `launches`.
cudaError_t launch_bulk_init(const PrepInstance* d_pi, const Segments& seg, int total_cells,
                             CellArrays cells, Control* ctl, int* n_src, bool fp64, int n,
                             double width_factor, double kappa_rel, cudaStream_t st,
                             int& launches);
// lift: the FP32 result is raised by this fraction of itself (see
// eik_opts.polish_lift) on its way to the FP64 polish array.
cudaError_t launch_polish_prep(const PolishInstance* d_pi, const Segments& seg, int total_cells,
                               CellArrays cells, Control* ctl, float lift, cudaStream_t st,
                               int& launches);
cudaError_t launch_fallback_prep(const PolishInstance* d_pi, const FinalInstance* d_fi,
                                 const Segments& seg, int total_cells, CellArrays cells,
                                 Control* ctl, double kappa, cudaStream_t st, int& launches);
// after_fallback: the pass after the replace-mode fallback (a no-op on the
// device unless it ran); otherwise the final pass of the FP64 path.
cudaError_t launch_residual_extract(const FinalInstance* d_fi, const Segments& seg, Control* ctl,
                                    bool after_fallback, double kappa, cudaStream_t st,
                                    int& launches);

// Persistent cell kernels (eik_cells_f32.cu / eik_cells_f64.cu /
// eik_cells_f64r.cu).  wpc: warps per worker for 16^3 cells (4, 6 or 8;
// 0 = 6); replace-mode kernels always use the default shape.
cudaError_t launch_cells(bool fp64, bool replace, int n, const CellKernelParams& p, int sms,
                         cudaStream_t st, int* grid_out, int& launches, int wpc);

}  // namespace eik
