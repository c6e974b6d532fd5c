// eik_cells_launch.cuh -- launch configuration of the persistent cell kernel
// per (value type, cell size, worker shape): a worker is one warp for n <= 8
// and WPC warps for n = 16 (4, 6 or 8; default 6: one thread per node of the
// largest plane, 192 nodes, so a plane step is one node deep); grid = SM count
// x resident CTAs per SM, at most two per SM by default.
#pragma once
#include "eik_cells.cuh"
#include "eik_prep.h"

namespace eik {

template <int N>
struct WorkerShape;
template <>
struct WorkerShape<4> { static constexpr int WPC = 1, WORKERS = 8; };
template <>
struct WorkerShape<8> { static constexpr int WPC = 1, WORKERS = 4; };
template <>
struct WorkerShape<16> { static constexpr int WPC = 6, WORKERS = 1; };

template <typename T, int N, int WORKERS>
constexpr int cells_smem_bytes() {
  using G = Geo<T, N>;
  return G::HEAD_BYTES + WORKERS * G::WORKER_BYTES;
}

template <typename T, int N, int WPC, int WORKERS, bool REPLACE>
cudaError_t launch_cells_shape(const CellKernelParams& p, int sms, cudaStream_t st,
                               int* grid_out, int& launches) {
  constexpr int threads = WPC * 32 * WORKERS;
  constexpr int smem = cells_smem_bytes<T, N, WORKERS>();
  auto kern = cells_kernel<T, N, WPC, WORKERS, REPLACE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = sms * per_sm;
  if (p.max_ctas > 0) {
    if (p.max_ctas < grid) grid = p.max_ctas;
  } else if (per_sm > 2) {
    // Enough workers for the cells of a few buckets; more only add waiting
    // workers whose polling slows the queue atomics of the working ones.
    grid = sms * 2;
  }
  if (grid_out) *grid_out = grid;
  kern<<<grid, threads, smem, st>>>(p);
  ++launches;
  return cudaGetLastError();
}

// wpc: warps per worker for n = 16 (4, 6 or 8; 0 = 6); ignored for n <= 8.
// WITH_SHAPES = false instantiates the default shape only.
template <typename T, int N, bool REPLACE, bool WITH_SHAPES>
cudaError_t launch_cells_t(const CellKernelParams& p, int sms, cudaStream_t st, int* grid_out,
                           int& launches, int wpc) {
  if constexpr (N == 16 && WITH_SHAPES) {
    if (wpc == 4) return launch_cells_shape<T, 16, 4, 1, REPLACE>(p, sms, st, grid_out, launches);
    if (wpc == 8) return launch_cells_shape<T, 16, 8, 1, REPLACE>(p, sms, st, grid_out, launches);
  }
  return launch_cells_shape<T, N, WorkerShape<N>::WPC, WorkerShape<N>::WORKERS, REPLACE>(
      p, sms, st, grid_out, launches);
}

}  // namespace eik
