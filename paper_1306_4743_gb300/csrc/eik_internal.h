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

// Dial bucket ring: 4096 buckets, each 32 lock-free stacks of cells.
constexpr int kNumBuckets = 4096;
constexpr unsigned kBucketMask = kNumBuckets - 1;
constexpr int kSubStackBits = 5;
constexpr int kSubStacks = 1 << kSubStackBits;
// device bytes of the queue: sub-stack heads, then counts and run counts
constexpr unsigned long long kQueueBytes = (unsigned long long)kNumBuckets * (kSubStacks * 8 + 8);

// Cell state bits.
constexpr unsigned kStQueued = 1u;   // in exactly one bucket stack
constexpr unsigned kStRunning = 2u;  // being swept by one worker
constexpr unsigned kStDirty = 4u;    // new inflow data arrived after the last load

// Cell direction word: bits 0-7 preferred sweep directions, bits 8-13 the
// faces whose halo values changed since the cell was last staged, bit 16
// set once a visit of the cell has converged (its interior is then a fixed
// point for the halo it saw, so the next visit need only restart at the
// flagged faces).
constexpr unsigned kDirMask = 0xffu;
constexpr int kFaceShift = 8;
constexpr unsigned kDirVisited = 1u << 16;

// Counters, in device memory (unsigned long long each).
enum CounterIndex {
  kCntVisits = 0,
  kCntSweeps,
  kCntUpdates,
  kCntPushes,
  kCntMaxSweeps,  // largest sweep count of one visit (atomicMax)
  kCntBusyNs,     // sum over visits of pop-to-retire time (ns)
  kCntStageNs,    // ... of which: TMA staging
  kCntSweepNs,    //               sweeps
  kCntFlagNs,     //               write-back and flags
  kCntPopNs,      // time spent in the pop loop (waiting included)
  kCntRevisits,   // visits of a cell that had converged before
  kCntRevisitSweeps,   // ... their sweeps
  kCntRevisitUpdates,  // ... their node updates
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
  double kappa;          // change threshold of Sec. 6.3 (early sweep terminations)
};

// Queue and solver control words, one block in device memory.  The words
// that every waiting worker polls sit on cache lines of their own so that
// the polling does not queue behind the atomics of working workers.
struct Control {
  alignas(128) unsigned cur;  // absolute index of the bucket being processed
  alignas(128) int active;    // cells QUEUED or RUNNING
  alignas(128) int queued;    // cells sitting in a bucket stack
  alignas(128) int status;    // first error code (EIK_*), 0 = fine
  alignas(128) unsigned progress;  // retired cell visits
  alignas(128) float base;    // key of bucket 0
  double kappa_bulk;          // change threshold of the FP32 bulk pass
  float inv_width;            // 1 / bucket width
  int n_sources;              // exit nodes seen by the init kernel
  int bad_input;              // an input failed validation
  double sum_inv_s;           // sum of 1 / s = F / h over non-exit nodes
  double sum_s;               // sum of s = h / F over the same nodes
  unsigned long long n_s;     // number of terms in sum_inv_s
  unsigned long long min_q_ord;    // ordered bits of min q (double)
  unsigned long long umax_bits;    // ordered bits of the largest finite u
                                   // (of the lifted start, during the polish)
  unsigned long long final_umax_bits;  // ... of the final u
  unsigned long long resid_bits;   // bits of the largest final residual (>= 0)
  unsigned long long check_bits;   // bits of the largest (Lambda(u) - u) after
                                   // the monotone polish (> 0: u below the fixed point)
  unsigned long long nonfinite;
  unsigned long long counters[3][kNumCounters];  // [bulk, polish, polish fallback]
};

struct CellArrays {
  unsigned* key;                 // ordered bits of the float cell value (Eq. 3)
  unsigned* state;               // kSt* bits
  unsigned* dir;                 // preferred sweep directions, 8 bits
  int* inst;                     // instance of each cell
  unsigned* next;                // stack links: next cell + 1, 0 = end
  unsigned long long* heads;     // [kNumBuckets][kSubStacks] (tag << 32) | (top cell + 1)
  int* cnt;                      // [kNumBuckets] cells in a bucket (raised before linking)
  int* run;                      // [kNumBuckets] cells taken from a bucket, not retired
  // Polish schedule (dependency graph read off the FP32 result):
  int* deps;                     // upwind neighbours still to finish a first visit
  unsigned* down;                // bits 0-5: downwind faces; bit 8: first visit done
  // Level order of each cell's nodes, read off the FP32 result (polish):
  // lev_perm[g * n^3 ...] the cell's node indices sorted by level,
  // lev_off[g * (kMaxLevels + 1) + l] the first entry of level l, and
  // lev_depth[g] the number of levels (0: no table, sweep as usual).
  unsigned short* lev_perm;
  unsigned short* lev_off;
  int* lev_depth;
};

// Longest chain of in-cell upwind neighbours a level table can hold.
constexpr int kMaxLevels = 255;

struct CellKernelParams {
  const Instance* inst;
  const CUtensorMap* tmaps;      // one per instance, 64-byte aligned
  CellArrays cells;
  Control* ctl;
  const unsigned short* plane_tab;  // in-cell node index a + n (b + n c), by plane
  const int* plane_off;             // plane start offsets, 3(n-1)+2 entries
  unsigned long long spin_cap_ns;
  int max_sweeps;
  int pass;                         // counter set: 0 bulk, 1 polish, 2 fallback
  int max_ctas;                     // grid limit (0 = every co-resident CTA)
  int kappa_from_ctl;               // 1: take kappa from ctl->kappa_bulk
  int relaxed;                      // 1: move past a bucket once its stack is empty
  int gated;                        // 1: polish schedule (cells wait for deps == 0)
  int cell_key;                     // 0: Eq. 3 cell values, 1: Eq. 4 (no reset on pop)
  int use_levels;                   // 1: start each visit with a pass in level order
};

}  // namespace eik
