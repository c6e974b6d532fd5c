// eik_internal.h -- data layout shared by the host runtime and the kernels
// of libeik.so (not part of the public C ABI).
//
// Device layout of one grid ("instance"):
//   u  padded value array of (px, py, pz) elements, node (i,j,k) stored at
//      (x, y, z) = (i+1, j+1, k+1); every other element (the one-node ghost
//      layer outside the grid, Sec. 1.1, and the filler of partial cells)
//      holds +inf and is never written.  The padding lets a tensor-map (TMA)
//      box of a cell plus its one-node halo start on a 16-byte boundary.
//   s  cell-blocked slowness s = h / F, n^3 contiguous values per cell, local
//      node (a,b,c) at a + n*(b + n*c).  Exit nodes (Q') and filler nodes
//      hold +inf: a node whose s is +inf is fixed and never recomputed.
// Cells of all instances of a launch are numbered globally; cell state,
// key and preferred-direction arrays are indexed by the global cell id.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eik {

// Dial bucket ring: 4096 buckets, each a lock-free stack of cells.
constexpr int kNumBuckets = 4096;
constexpr unsigned kBucketMask = kNumBuckets - 1;

// Cell state bits.
constexpr unsigned kStQueued = 1u;   // in exactly one bucket stack
constexpr unsigned kStRunning = 2u;  // being swept by one worker
constexpr unsigned kStDirty = 4u;    // new inflow data arrived after the last load

// Counters, in device memory (unsigned long long each).
enum CounterIndex {
  kCntVisits = 0,
  kCntSweeps,
  kCntUpdates,
  kCntPushes,
  kCntMaxSweeps,  // largest sweep count of one visit (atomicMax)
  kNumCounters
};

// One grid of a launch, as the kernels see it.
struct Instance {
  void* u;               // padded values (float or double)
  const void* s;         // cell-blocked slowness (same type as u)
  long long px, py, pz;  // padded extents in elements
  int nx, ny, nz;        // grid nodes
  int ncx, ncy, ncz;     // cells per axis
  int cell_base;         // global id of the first cell
  int ncells;
  double kappa;          // change threshold of Sec. 6.4
};

// Queue and solver control words, one block in device memory.
struct Control {
  unsigned cur;        // absolute index of the lowest possibly non-empty bucket
  int active;          // cells QUEUED or RUNNING
  int queued;          // cells sitting in a bucket stack
  int status;          // first error code (EIK_*), 0 = fine
  unsigned progress;   // retired cell visits
  int n_sources;       // exit nodes seen by the init kernel
  float base;          // key of bucket 0
  float inv_width;     // 1 / bucket width
  double sum_s;        // sum of s over non-exit nodes (bucket width estimate)
  unsigned long long n_s;          // number of terms in sum_s
  unsigned long long min_q_ord;    // ordered bits of min q (double)
  unsigned long long umax_bits;    // ordered bits of the largest finite u
  unsigned long long resid_bits;   // bits of the largest residual (>= 0)
  unsigned long long nonfinite;
  unsigned long long counters[2][kNumCounters];  // [bulk, polish]
  int bad_input;       // an input failed validation
  int pad[3];
};

struct CellArrays {
  unsigned* key;                 // ordered bits of the float cell value (Eq. 3)
  unsigned* state;               // kSt* bits
  unsigned* dir;                 // preferred sweep directions, 8 bits
  int* inst;                     // instance of each cell
  unsigned* next;                // stack links: next cell + 1, 0 = end
  unsigned long long* heads;     // [kNumBuckets] (tag << 32) | (top cell + 1)
};

struct CellKernelParams {
  const Instance* inst;
  const CUtensorMap* tmaps;      // one per instance, 64-byte aligned
  CellArrays cells;
  Control* ctl;
  const unsigned short* plane_tab;  // packed (a | b << 5 | c << 10), by plane
  const int* plane_off;             // plane start offsets, 3(n-1)+2 entries
  unsigned long long spin_cap_ns;
  int max_sweeps;
  int pass;                         // 0 = bulk counters, 1 = polish counters
};

}  // namespace eik
