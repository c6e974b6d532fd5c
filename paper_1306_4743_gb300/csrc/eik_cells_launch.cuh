// eik_cells_launch.cuh -- launch configuration of the persistent cell kernel
// per (value type, cell size): a worker is one warp for n <= 8 and six warps
// for n = 16, one thread per node of the largest plane (192 nodes), so a
// plane step is one node deep (measured: 4 warps 20.6 ms, 6 warps 18.8 ms,
// 8 warps 18.9 ms on the 257^3 FP64 solve); grid = SM count x resident CTAs
// per SM, at most two per SM by default.
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

template <typename T, int N>
constexpr int cells_smem_bytes() {
  using G = Geo<T, N>;
  return G::HEAD_BYTES + WorkerShape<N>::WORKERS * G::WORKER_BYTES;
}

template <typename T, int N, bool REPLACE>
cudaError_t launch_cells_t(const CellKernelParams& p, int sms, cudaStream_t st, int* grid_out,
                           int& launches) {
  constexpr int WPC = WorkerShape<N>::WPC, WORKERS = WorkerShape<N>::WORKERS;
  constexpr int threads = WPC * 32 * WORKERS;
  constexpr int smem = cells_smem_bytes<T, N>();
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

template <typename T, int N>
void shape_t(int* threads, int* smem, int* workers) {
  *threads = WorkerShape<N>::WPC * 32 * WorkerShape<N>::WORKERS;
  *smem = cells_smem_bytes<T, N>();
  *workers = WorkerShape<N>::WORKERS;
}

}  // namespace eik
