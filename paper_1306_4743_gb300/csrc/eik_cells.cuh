// eik_cells.cuh -- the persistent cell kernel: the GPU restatement of the
// parallel Heap-Cell Method's main loop (Alg. 1 and Alg. 3).
//
// A worker (one warp for n <= 8, a group of WPC warps for n = 16) repeats:
//   1. pop a cell from the lowest non-empty Dial bucket (Alg. 3; the
//      cell value is reset to +inf and its preferred directions are taken),
//   2. stage the cell and its one-node face halo of u into shared memory with
//      one TMA tensor box, and the cell's slowness with one bulk copy (the
//      domain c~ = c U N(c) of Sec. 4),
//   3. sweep the cell with the modified Locking Sweeping update of Alg. 2:
//      preferred directions first, then the standard loop of 8 directions,
//      until one whole sweep changes no value by more than kappa; each
//      sweep direction advances over the planes i+j+k = C of the Detrixhe
//      ordering (Sec. 3), whose nodes do not depend on each other,
//   4. write the changed values back, and for each face with changed border
//      values flag the neighbouring cell (the "currently downwind" rule of
//      Sec. 4) with the smallest such value as its new cell value (Eq. 3)
//      and the directions that sweep away from this cell,
//   5. retire the cell (re-queue it if it was flagged while running) and
//      decrement the active count after the flags (Sec. 5).
// The kernel returns when no cell is queued or running.
//
// Min mode (REPLACE = false): u <- min(u, Lambda(u)), the monotone update of
// Alg. 2.  Replace mode (REPLACE = true, the FP64 polish): u <- Lambda(u) at
// every non-fixed node, so a value may also rise; a change counts when it
// exceeds kappa + 2^-50 |u|.
#pragma once
#include "eik_device.cuh"

namespace eik {

// Standard loop of the 8 sweep directions.  Direction code d sweeps i
// downward when bit 0 is set, j by bit 1, k by bit 2; this is the ordering
// (+++), (-++), (--+), (+-+), (++-), (-+-), (---), (+--).
static __constant__ int kStdOrder[8] = {0, 1, 3, 2, 4, 5, 7, 6};

// a < b for stored values (>= 0: the FP64 compare runs on the integer pipe)
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool vlt(double a, double b) { return dlt_nn(a, b); }

// Per-node bits of the staged cell: written back, changed by more than
// kappa (flags the neighbour cell), active (to be recomputed, Alg. 2).  One
// 32-bit word per node: sub-word shared-memory accesses cost about twice
// the latency of word accesses, and these bits sit on the sweep's
// critical path.
// The active bit sits alone in byte 0 and the others in byte 1, so that a
// neighbour is activated by a single byte store, without reading the word
// (two threads of one plane step may activate the same neighbour; they store
// the same byte, and the neighbour's own bits are written only by the thread
// that updates it, on another plane step).
constexpr unsigned kActive = 0x4u, kWritten = 0x100u, kBig = 0x200u;

__device__ __forceinline__ void activate_node(unsigned* chg, int nb) {
  reinterpret_cast<unsigned char*>(chg + nb)[0] = (unsigned char)kActive;
}

template <typename T, int N>
struct Geo {
  static constexpr int ES = (int)sizeof(T);
  // TMA box width: smallest multiple of 16 bytes covering the N+2 halo row
  static constexpr int BX = (((N + 2) * ES + 15) / 16) * 16 / ES;
  static constexpr int BY = N + 2;
  static constexpr int BZ = N + 2;
  static constexpr int SY = BX;
  static constexpr int SZ = BX * BY;
  static constexpr int N3 = N * N * N;
  static constexpr int NPLANES = 3 * (N - 1) + 1;
  // most nodes on one plane i + j + k = C
  static constexpr int max_plane() {
    int best = 0;
    for (int C = 0; C < NPLANES; ++C) {
      int c = 0;
      for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a)
          if (C - a - b >= 0 && C - a - b < N) ++c;
      best = c > best ? c : best;
    }
    return best;
  }
  static constexpr int MAXPLANE = max_plane();
  static constexpr int UBYTES = BX * BY * BZ * ES;
  static constexpr int SBYTES = N3 * ES;
  static constexpr int align128(int b) { return (b + 127) / 128 * 128; }
  // per-worker shared memory: u tile | s tile | change flags | plane list |
  // mbarrier + scratch
  static constexpr int OFF_S = align128(UBYTES);
  static constexpr int OFF_CHG = OFF_S + align128(SBYTES);
  // active-node list of one plane (at most N^2 nodes lie on a plane)
  static constexpr int OFF_LIST = OFF_CHG + align128(N3 * 4);
  // FP64 only: the cell's level table (node order, level starts), staged
  // with the cell for the level pass of a first polish visit
  static constexpr int PERM_BYTES = ES == 8 ? align128(N3 * 2) : 0;
  static constexpr int LOFF_BYTES = ES == 8 ? align128((kMaxLevels + 1) * 2) : 0;
  static constexpr int OFF_PERM = OFF_LIST + align128(N * N * 2);
  static constexpr int OFF_LOFF = OFF_PERM + PERM_BYTES;
  static constexpr int OFF_BAR = OFF_LOFF + LOFF_BYTES;
  static constexpr int WORKER_BYTES = OFF_BAR + 256;
  // CTA-wide: plane table | plane offsets
  static constexpr int TAB_BYTES = align128(N3 * 2);
  static constexpr int OFFS_BYTES = align128((NPLANES + 1) * 4);
  static constexpr int HEAD_BYTES = TAB_BYTES + OFFS_BYTES;
};

template <int WPC>
__device__ __forceinline__ void worker_sync(int worker) {
  if constexpr (WPC == 1) {
    __syncwarp();
  } else {
    bar_sync_named(1 + worker, WPC * 32);
  }
}
template <int WPC>
__device__ __forceinline__ bool worker_any(int worker, bool pred) {
  if constexpr (WPC == 1) {
    return __any_sync(0xffffffffu, pred) != 0;
  } else {
    return bar_red_or(1 + worker, WPC * 32, pred);
  }
}

// Alg. 2 for one node si = i + n (j + n k) of the staged cell that is active: clear
// its active bit, recompute it from its six neighbours (Eq. 2), store a
// lower value (min mode) or any new value (replace mode), and on a change
// by more than the threshold activate the neighbours that may now use it.
// `left` counts, per axis (bits 0-9 x, 10-19 y, 20-29 z), the activations of
// neighbours on the plane the sweep has just left (at most one per node and
// axis, and a thread takes at most 2 (3n - 2) nodes of a sweep, so a field
// cannot overflow).  `hi` packs the largest in-grid local index per axis
// (bits 0-7 x, 8-15 y, 16-23 z): the filler of a partial cell is never
// activated (it is fixed; a filler node left behind a sweep would cost one
// more sweep to clear).
template <typename T, int N, bool REPLACE>
__device__ __forceinline__ void update_node(T* __restrict__ U, const T* __restrict__ S,
                                            unsigned* __restrict__ chg, int si, int fx, int fy,
                                            int fz, int hi, T kappa, unsigned& n_updates,
                                            unsigned& left) {
  using G = Geo<T, N>;
  const int i = si % N, j = (si / N) % N, k = si / (N * N);
  const T s = S[si];
  unsigned c1 = chg[si] & ~kActive;  // the node is no longer active (Alg. 2)
  auto activate = [&](int nb) { activate_node(chg, nb); };
  if (vlt(s, tinf<T>())) {
    const int t = (i + 1) + G::SY * (j + 1) + G::SZ * (k + 1);
    const T v = U[t];
    const T xm = U[t - 1], xp = U[t + 1];
    const T ym = U[t - G::SY], yp = U[t + G::SY];
    const T zm = U[t - G::SZ], zp = U[t + G::SZ];
    const T nv = local_solve(nmin(xm, xp), nmin(ym, yp), nmin(zm, zp), s);
    ++n_updates;
    bool big;
    if constexpr (!REPLACE) {
      const bool lower = vlt(nv, v);
      if constexpr (sizeof(T) == 8) {
        big = drop_exceeds(nv, v, (float)kappa);
      } else {
        big = vlt(nv, v - kappa);
      }
      if (lower) {
        U[t] = nv;
        c1 |= big ? (kWritten | kBig) : kWritten;
      }
    } else {
      big = nv != v && fabs(nv - v) > kappa + fabs(v) * (T)8.8817841970012523e-16;
      if (nv != v) {
        U[t] = nv;
        c1 |= big ? (kWritten | kBig) : kWritten;
      }
    }
    if (big) {
      // Alg. 2: neighbours (in this cell) that may now use the new
      // value become active; neighbours in other cells are reached through
      // the face flags.  In min mode a neighbour y can use the new value only
      // if it is below y's own value.  (Also requiring it to be below y's
      // other neighbour on that axis activates fewer nodes, but the extra
      // loads and compares on every changed node cost more in the sweeps
      // than the saved updates: 257^3 FP64 16.5 against 15.3 ms.)  The
      // neighbour on the side the sweep came from lies on the previous plane.
      auto uses = [&](T y) { return REPLACE || vlt(nv, y); };
      if (i > 0 && uses(xm)) {
        activate(si - 1);
        left += fx == 0 ? 1u : 0u;
      }
      if (i < (hi & 0xff) && uses(xp)) {
        activate(si + 1);
        left += fx != 0 ? 1u : 0u;
      }
      if (j > 0 && uses(ym)) {
        activate(si - N);
        left += fy == 0 ? (1u << 10) : 0u;
      }
      if (j < ((hi >> 8) & 0xff) && uses(yp)) {
        activate(si + N);
        left += fy != 0 ? (1u << 10) : 0u;
      }
      if (k > 0 && uses(zm)) {
        activate(si - N * N);
        left += fz == 0 ? (1u << 20) : 0u;
      }
      if (k < (hi >> 16) && uses(zp)) {
        activate(si + N * N);
        left += fz != 0 ? (1u << 20) : 0u;
      }
    }
  }
  chg[si] = c1;
}

// Level-pass helpers (min mode, Alg. 2).  During the level pass bits 16-31
// of a node's flag word hold the step in which the pass took it (kNotTaken
// before, and for the filler of partial cells, which is in no level).  take_node: no other
// thread writes node si's flag word in this step: record the step, clear the
// active bit, recompute the node from its six neighbours (Eq. 2), store a
// lower value and mark a change by more than kappa (kBig).
constexpr int kStepShift = 16;
constexpr unsigned kNotTaken = 0xffffu;

template <typename T, int N>
__device__ __forceinline__ void take_node(T* __restrict__ U, const T* __restrict__ S,
                                          unsigned* __restrict__ chg, int si, T kappa,
                                          unsigned step, unsigned& n_updates) {
  using G = Geo<T, N>;
  unsigned c1 = (chg[si] & ~kActive & 0xffffu) | (step << kStepShift);
  const T s = S[si];
  if (vlt(s, tinf<T>())) {
    const int i = si % N, j = (si / N) % N, k = si / (N * N);
    const int t = (i + 1) + G::SY * (j + 1) + G::SZ * (k + 1);
    const T v = U[t];
    const T nv = local_solve(nmin(U[t - 1], U[t + 1]), nmin(U[t - G::SY], U[t + G::SY]),
                             nmin(U[t - G::SZ], U[t + G::SZ]), s);
    ++n_updates;
    if (vlt(nv, v)) {
      U[t] = nv;
      c1 |= drop_exceeds(nv, v, (float)kappa) ? (kWritten | kBig) : kWritten;
    }
  }
  chg[si] = c1;
}

// After the level pass, in parallel over the cell: a node x taken in step
// sx read the values its neighbours had then.  A neighbour y taken in the
// same or a later step, with a change above kappa, that x may now use (y
// below x and below x's other neighbour on that axis) leaves x active for
// the sweeps.  (The same test as waking y's users right after y's step, done
// once for all nodes: the final values of x and of x's other neighbour are
// the ones x kept since its step or that the wake would have compared
// with, so no step of the pass waits for it.)  Each thread writes only its
// own nodes' active bytes; the bits it reads of other words do not change.
template <typename T, int N, int WPC>
__device__ __forceinline__ void level_check(const T* __restrict__ U, unsigned* __restrict__ chg,
                                            int tid) {
  using G = Geo<T, N>;
  constexpr int NT = WPC * 32;
  for (int e = tid; e < G::N3; e += NT) {
    const unsigned sx = chg[e] >> kStepShift;
    if (sx == kNotTaken) continue;
    const int i = e % N, j = (e / N) % N, k = e / (N * N);
    const bool in[6] = {i > 0, i < N - 1, j > 0, j < N - 1, k > 0, k < N - 1};
    const int dn[3] = {1, N, N * N};
    unsigned later = 0;  // bit d: the neighbour on side d changed in a step >= sx
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (!in[d]) continue;
      const unsigned cy = chg[e + ((d & 1) ? dn[d >> 1] : -dn[d >> 1])];
      if ((cy & kBig) && (cy >> kStepShift) >= sx) later |= 1u << d;
    }
    if (!later) continue;
    const int t = (i + 1) + G::SY * (j + 1) + G::SZ * (k + 1);
    const int dt[3] = {1, G::SY, G::SZ};
    const T v = U[t];
    bool act = false;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (!((later >> d) & 1u)) continue;
      const int o = (d & 1) ? dt[d >> 1] : -dt[d >> 1];
      const T uy = U[t + o];
      act = act || (vlt(uy, v) && vlt(uy, U[t - o]));
    }
    if (act) activate_node(chg, e);
  }
}

// One pass over a cell's nodes in the level order of its table (see
// polish_levels_kernel; the filler is in no level): level by level, every
// node of a level is taken (a first visit starts with no node active), in
// steps of UNR nodes a thread split by a barrier.  A node's FP32 upwind
// neighbours have smaller levels, so where the FP64 values keep the FP32
// order one pass settles the cell; level_check then leaves active the nodes
// whose FP64 inflow came from a node taken in the same or a later step.
// perm and loff are the staged table (node indices, level starts).
template <typename T, int N, int WPC>
__device__ __forceinline__ void level_pass(T* __restrict__ U, const T* __restrict__ S,
                                           unsigned* __restrict__ chg,
                                           const unsigned short* __restrict__ perm,
                                           const unsigned short* __restrict__ loff, int depth,
                                           int tid, int worker, T kappa, unsigned& n_updates) {
  constexpr int NT = WPC * 32;
  constexpr int UNR = 2;
  unsigned step = 0;
  for (int l = 0; l < depth; ++l) {
    const int lo = loff[l], hi = loff[l + 1];
    for (int c0 = lo; c0 < hi; c0 += UNR * NT, ++step) {
#pragma unroll
      for (int h = 0; h < UNR; ++h) {
        const int e = c0 + tid + h * NT;
        if (e < hi) take_node<T, N>(U, S, chg, (int)perm[e], kappa, step, n_updates);
      }
      worker_sync<WPC>(worker);
    }
  }
  level_check<T, N, WPC>(U, chg, tid);
  worker_sync<WPC>(worker);
}

// Worker-wide sums of the three packed per-axis counts of left-behind
// activations; returns the bit of the axis with the most (the lowest axis on
// a tie), or 0 when no activation was left behind.  `ws` is 3 * WPC ints of
// worker scratch.
template <int WPC>
__device__ __forceinline__ unsigned worker_most_left_axis(int worker, int tid, unsigned packed,
                                                          int* ws) {
  unsigned c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = __reduce_add_sync(0xffffffffu, (packed >> (10 * a)) & 1023u);
  if constexpr (WPC > 1) {
    if ((tid & 31) == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) ws[3 * (tid >> 5) + a] = (int)c[a];
    }
    worker_sync<WPC>(worker);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      unsigned t = 0;
#pragma unroll
      for (int w = 0; w < WPC; ++w) t += (unsigned)ws[3 * w + a];
      c[a] = t;
    }
  }
  if ((c[0] | c[1] | c[2]) == 0u) return 0u;
  int best = 0;
  if (c[1] > c[best]) best = 1;
  if (c[2] > c[best]) best = 2;
  return 1u << best;
}

// First and last plane (in the order of direction `dir`) that hold an
// active node; first > last when no node is active.  `ws` is 2 * WPC ints
// of worker scratch.
template <int N, int WPC>
__device__ __forceinline__ void active_planes(const unsigned* __restrict__ chg, int dir,
                                              int tid, int worker, int* ws, int& first,
                                              int& last) {
  constexpr int NT = WPC * 32, N3 = N * N * N;
  const int fx = (dir & 1) ? N - 1 : 0;
  const int fy = (dir & 2) ? N - 1 : 0;
  const int fz = (dir & 4) ? N - 1 : 0;
  int lo = 1 << 20, hi = -1;
  for (int e = tid * 4; e < N3; e += NT * 4) {
    const uint4 w = *reinterpret_cast<const uint4*>(chg + e);
    const unsigned wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!(wd[q] & kActive)) continue;
      const int idx = e + q;
      const int pl = ((idx % N) ^ fx) + (((idx / N) % N) ^ fy) + ((idx / (N * N)) ^ fz);
      lo = pl < lo ? pl : lo;
      hi = pl > hi ? pl : hi;
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if constexpr (WPC > 1) {
    const int wwarp = tid >> 5;
    if ((tid & 31) == 0) {
      ws[wwarp] = lo;
      ws[WPC + wwarp] = hi;
    }
    worker_sync<WPC>(worker);
#pragma unroll
    for (int w2 = 0; w2 < WPC; ++w2) {
      lo = ws[w2] < lo ? ws[w2] : lo;
      hi = ws[WPC + w2] > hi ? ws[WPC + w2] : hi;
    }
  }
  first = lo;
  last = hi;
}

// One directional sweep of a staged cell over planes first.. of the order
// of `dir`, where `last` is the last plane holding a node that was active
// when the sweep began.  A node's six neighbours lie on the planes just
// before and just after its own, so a node activated on the next plane is
// swept later in this same sweep; past `last`, a plane with no active node
// ends the sweep, as no later plane can hold one.  Returns (worker-wide)
// the bit of the axis along which the most nodes on planes just left were
// activated (those nodes are still active afterwards), or 0 when none was:
// then another sweep would change nothing, so the cell has converged one
// sweep earlier than the plain "until a sweep changes nothing" test would
// find.  The next sweep reverses that one axis.
//
// COMPACT (one-warp workers): the active nodes of each plane are first
// gathered into a list by ballot and the lanes then take list entries, so
// the warp issues a node's arithmetic only for nodes that need it.  This
// matters for FP64, whose narrow pipe costs the same per warp instruction
// however few lanes are active.
template <typename T, int N, int WPC, bool REPLACE, bool COMPACT>
__device__ __forceinline__ unsigned sweep_cell(T* __restrict__ U, const T* __restrict__ S,
                                               unsigned* __restrict__ chg,
                                               const unsigned short* __restrict__ tab,
                                               const int* __restrict__ off,
                                               unsigned short* __restrict__ list, int dir,
                                               int first, int last, int hi, int tid, int worker,
                                               T kappa, unsigned& n_updates, int* ws) {
  using G = Geo<T, N>;
  constexpr int NT = WPC * 32;
  // Nodes of one plane do not depend on each other: a thread takes up to UNR
  // of them (so their loads and arithmetic overlap) and every plane fits one
  // pass of the worker.
  constexpr int UNR = (G::MAXPLANE + NT - 1) / NT;
  static_assert(G::MAXPLANE <= UNR * NT, "a plane must fit one pass of the worker");
  static_assert(!COMPACT || WPC == 1, "the gathered list is per warp");
  constexpr unsigned kNone = 0xffffu;  // node indices are below 4096
  const int fx = (dir & 1) ? N - 1 : 0;
  const int fy = (dir & 2) ? N - 1 : 0;
  const int fz = (dir & 4) ? N - 1 : 0;
  // n is a power of two, so the index of a node in the order of direction
  // `dir` is the table's index with i, j, k reflected: one XOR
  const unsigned dmask = (unsigned)(fx + N * (fy + N * fz));
  // A plane's nodes are packed into the lowest slots (a small plane keeps
  // few warps busy, which matters for FP64 whose pipe is paid per warp
  // instruction).  Loading the plane's entries at its start measured
  // faster than loading them two planes ahead: a barrier waits for loads
  // still in flight.
  unsigned left = 0;
  // FP32 with one thread per (j, k) pencil of a 16^3 cell (8 warps): a
  // thread's node on plane C is (C - j - k, j, k) in the sweep's reflected
  // coordinates, computed instead of read from the plane table (one
  // dependent shared load less per plane step; measured ~5% faster bulk
  // sweeps than 6 warps with the table.  FP64 stays with the packed table:
  // its narrow pipe is paid per warp instruction, and small planes then keep
  // fewer warps busy)
  constexpr bool PENCILS = sizeof(T) == 4 && N == 16 && NT == 256;
  for (int C = first; C < G::NPLANES; ++C) {
    unsigned cur[UNR];
    if constexpr (PENCILS) {
      const int jr = tid & 15, kr = tid >> 4, ir = C - jr - kr;
      cur[0] = (ir >= 0 && ir < 16) ? ((unsigned)(ir + 16 * jr + 256 * kr) ^ dmask) : kNone;
    } else {
      const int b0 = off[C], e1 = off[C + 1];
#pragma unroll
      for (int h = 0; h < UNR; ++h) {
        const int e = b0 + tid + h * NT;
        cur[h] = e < e1 ? ((unsigned)tab[e] ^ dmask) : kNone;
      }
    }
    // the active bits of all of this thread's nodes first (Alg. 2),
    // so that their loads overlap
    bool act[UNR];
#pragma unroll
    for (int h = 0; h < UNR; ++h)
      act[h] = cur[h] != kNone && (chg[cur[h] & (unsigned)(G::N3 - 1)] & kActive);
    bool any;
    if constexpr (!COMPACT) {
      bool did = false;
#pragma unroll
      for (int h = 0; h < UNR; ++h) {
        if (!act[h]) continue;
        did = true;
        update_node<T, N, REPLACE>(U, S, chg, (int)cur[h], fx, fy, fz, hi, kappa, n_updates,
                                   left);
      }
      // also ends the plane; before the last initially active plane the
      // sweep cannot end, so a plain barrier does (bar.sync costs about half
      // a bar.red.or)
      if (C < last) {
        worker_sync<WPC>(worker);
        any = true;
      } else {
        any = worker_any<WPC>(worker, did);
      }
    } else {
      // gather the plane's active nodes
      const int lane = tid & 31;
      const unsigned below = (1u << lane) - 1u;
      int total = 0;
#pragma unroll
      for (int h = 0; h < UNR; ++h) {
        const unsigned m = __ballot_sync(0xffffffffu, act[h]);
        if (act[h]) list[total + __popc(m & below)] = (unsigned short)cur[h];
        total += __popc(m);
      }
      __syncwarp();
      for (int x0 = tid; x0 < total; x0 += UNR * NT) {
#pragma unroll
        for (int h = 0; h < UNR; ++h) {
          const int x = x0 + h * NT;
          if (x >= total) break;
          update_node<T, N, REPLACE>(U, S, chg, (int)list[x], fx, fy, fz, hi, kappa, n_updates,
                                     left);
        }
      }
      any = total > 0;
      worker_sync<WPC>(worker);
    }
    if (!any && C >= last) break;
  }
  return worker_most_left_axis<WPC>(worker, tid, left, ws);
}

template <typename T, int N, int WPC, int WORKERS, bool REPLACE>
__global__ void __launch_bounds__(WPC * 32 * WORKERS)
    cells_kernel(const CellKernelParams p) {
  using G = Geo<T, N>;
  constexpr int NT = WPC * 32;
  extern __shared__ __align__(128) unsigned char smem[];
  // Nothing queued (the replace-mode fallback after a passing check, or all
  // work already done): leave at once, as one block.
  if (__syncthreads_and(ld_acquire_s32(&p.ctl->active) <= 0)) return;
  unsigned short* tab = reinterpret_cast<unsigned short*>(smem);
  int* off = reinterpret_cast<int*>(smem + G::TAB_BYTES);
  for (int e = threadIdx.x; e < G::N3; e += blockDim.x) tab[e] = p.plane_tab[e];
  for (int e = threadIdx.x; e <= G::NPLANES; e += blockDim.x) off[e] = p.plane_off[e];

  const int worker = threadIdx.x / NT;
  const int tid = threadIdx.x % NT;
  const int lane = tid & 31;
  const int wwarp = tid >> 5;
  unsigned char* wbase = smem + G::HEAD_BYTES + worker * G::WORKER_BYTES;
  T* U = reinterpret_cast<T*>(wbase);
  T* S = reinterpret_cast<T*>(wbase + G::OFF_S);
  unsigned* chg = reinterpret_cast<unsigned*>(wbase + G::OFF_CHG);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(wbase + G::OFF_BAR);
  // scratch: [0] cell, [1] direction word, [2..7] face keys, [12..23] plane
  // range, [32..49] per-axis counts of left-behind activations
  int* wshared = reinterpret_cast<int*>(wbase + G::OFF_BAR + 16);
  unsigned short* list = reinterpret_cast<unsigned short*>(wbase + G::OFF_LIST);
  constexpr bool COMPACT = sizeof(T) == 8 && WPC == 1;

  if (tid == 0) mbar_init(bar, 1);
  fence_proxy_async_smem();
  __syncthreads();

  Control* ctl = p.ctl;
  const CellArrays& cells = p.cells;
  unsigned phase = 0;
  unsigned slot = 0;  // ring slot of the bucket the current cell came from
  unsigned long long n_visits = 0, n_sweeps = 0, n_pushes = 0, busy_ns = 0, n_revisits = 0;
  unsigned long long rv_sweeps = 0, rv_upd = 0;
  unsigned long long pop_ns = 0, stage_ns = 0, sweep_ns = 0, flag_ns = 0;
  unsigned n_updates = 0;
  unsigned long long upd_total = 0;
  int max_sweeps_seen = 0;

  for (;;) {
    // ---- 1. pop --------------------------------------------------------
    int cell = -1;
    unsigned pref = 0;  // direction word as taken: preferred dirs, faces, visited
    unsigned long long t_pop0 = 0;
    if (tid == 0) t_pop0 = global_timer_ns();
    if (wwarp == 0) {
      cell = queue_pop_warp(cells, ctl, p.spin_cap_ns, lane, &slot, p.relaxed != 0,
                            (unsigned)(blockIdx.x * WORKERS + worker) * 7u);
      if (lane == 0 && cell >= 0) {
        // V^c <- +inf (Alg. 1); the Eq. 4 variant keeps it (Sec. 6.8)
        if (p.cell_key == 0) atomicExch(cells.key + cell, kKeyInf);
        pref = atomicAnd(cells.dir + cell, kDirVisited);  // take dirs and faces
      }
      pref = __shfl_sync(0xffffffffu, pref, 0);
      if constexpr (WPC > 1) {
        if (lane == 0) {
          wshared[0] = cell;
          wshared[1] = (int)pref;
        }
      }
    }
    if constexpr (WPC > 1) {
      worker_sync<WPC>(worker);
      cell = wshared[0];
      pref = (unsigned)wshared[1];
      worker_sync<WPC>(worker);
    }
    if (cell < 0) break;
    unsigned long long t_pop = 0;
    if (tid == 0) {
      t_pop = global_timer_ns();
      pop_ns += t_pop - t_pop0;
    }

    const int ii = cells.inst[cell];
    const Instance I = p.inst[ii];
    const int lc = cell - I.cell_base;
    const int cx = lc % I.ncx;
    const int cy = (lc / I.ncx) % I.ncy;
    const int cz = lc / (I.ncx * I.ncy);
    const T kappa = (T)(p.kappa_from_ctl ? ctl->kappa_bulk : I.kappa);
    // largest in-grid local index per axis (the rest of a partial cell is filler)
    const int hi_ext = (min(N, I.nx - N * cx) - 1) | ((min(N, I.ny - N * cy) - 1) << 8) |
                       ((min(N, I.nz - N * cz) - 1) << 16);

    // ---- 2. stage cell + halo ------------------------------------------
    // (and, for the level pass of the polish, the cell's level table)
    // The level pass serves first visits: a revisit starts from a few
    // flagged face nodes, and walking all levels for them (two barriers a
    // level) cost more than sweeping from those faces.
    int lev_depth = 0;
    if constexpr (!REPLACE && sizeof(T) == 8)
      if (p.use_levels && !(pref & kDirVisited)) lev_depth = cells.lev_depth[cell];
    fence_proxy_async_smem();
    worker_sync<WPC>(worker);
    if (tid == 0) {
      fence_proxy_async_global();
      const unsigned lev_bytes = lev_depth > 0 ? (unsigned)(G::N3 * 2 + (kMaxLevels + 1) * 2) : 0u;
      mbar_arrive_expect_tx(bar, (unsigned)(G::UBYTES + G::SBYTES) + lev_bytes);
      tma_load_3d(U, p.tmaps + ii, N * cx, N * cy, N * cz, bar);
      bulk_load(S, static_cast<const T*>(I.s) + (size_t)lc * G::N3, (unsigned)G::SBYTES, bar);
      if (lev_bytes) {
        bulk_load(wbase + G::OFF_PERM, cells.lev_perm + (size_t)cell * G::N3,
                  (unsigned)(G::N3 * 2), bar);
        bulk_load(wbase + G::OFF_LOFF, cells.lev_off + (size_t)cell * (kMaxLevels + 1),
                  (unsigned)((kMaxLevels + 1) * 2), bar);
      }
    }
    // On a first visit every node starts active, except with a level table,
    // whose pass takes every non-fixed node anyway.  After a converged visit
    // only the halo can have changed (a cell's nodes have one writer, the
    // cell), so only the nodes on the faces flagged since then start active.
    const bool revisit = (pref & kDirVisited) != 0;
    const unsigned faces = (pref >> kFaceShift) & 0x3fu;
    {
      const unsigned fill =
          revisit ? 0u : (lev_depth > 0 ? (kNotTaken << kStepShift) : (unsigned)kActive);
      for (int e = tid * 4; e < G::N3; e += NT * 4)
        *reinterpret_cast<uint4*>(chg + e) = make_uint4(fill, fill, fill, fill);
    }
    {
      unsigned long long spins = 0;
      while (!mbar_try_wait(bar, phase)) {
        if (++spins > (1ull << 26)) {
          set_status(ctl, EIK_ETIMEOUT);
          // wait once more, bounded, for the copies in flight
          for (unsigned long long r = 0; r < (1ull << 26) && !mbar_try_wait(bar, phase); ++r) {
          }
          return;
        }
      }
    }
    phase ^= 1u;
    unsigned* fmin = reinterpret_cast<unsigned*>(wshared + 2);  // [6] halo face minima
    if constexpr (!REPLACE) {
      if (tid < 6) fmin[tid] = 0xffffffffu;
    }
    worker_sync<WPC>(worker);
    // Min mode: the smallest halo value of each face (as ordered float
    // bits), to start with the sweep direction that runs away from the
    // lower face on each axis.
    if constexpr (!REPLACE) {
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int axis = f >> 1, side = (f & 1) ? N + 1 : 0;
        unsigned m = 0xffffffffu;
        for (int q = tid; q < N * N; q += NT) {
          const int a = q % N + 1, b = q / N + 1;
          const int t = axis == 0 ? side + G::SY * a + G::SZ * b
                      : axis == 1 ? a + G::SY * side + G::SZ * b
                                  : a + G::SY * b + G::SZ * side;
          float v;
          if constexpr (sizeof(T) == 8) v = f32_of_f64_nn(U[t]);
          else v = U[t];
          const unsigned vb = __float_as_uint(v);
          m = vb < m ? vb : m;
        }
        m = __reduce_min_sync(0xffffffffu, m);
        if ((tid & 31) == 0 && m != 0xffffffffu) atomicMin(fmin + f, m);
      }
    }
    if (revisit) {
      // a flagged face's nodes restart; in min mode only those whose halo
      // neighbour is below them, as no other can take a lower value from it
      for (int f = 0; f < 6; ++f) {
        if (!((faces >> f) & 1u)) continue;
        const int axis = f >> 1, side = (f & 1) ? N - 1 : 0;
        const int step = axis == 0 ? 1 : axis == 1 ? G::SY : G::SZ;
        for (int q = tid; q < N * N; q += NT) {
          const int a = q % N, b = q / N;
          int i, j, k;
          if (axis == 0) { i = side; j = a; k = b; }
          else if (axis == 1) { i = a; j = side; k = b; }
          else { i = a; j = b; k = side; }
          const int e = i + N * (j + N * k);
          const int t = (i + 1) + G::SY * (j + 1) + G::SZ * (k + 1);
          const bool in_grid =
              i <= (hi_ext & 0xff) && j <= ((hi_ext >> 8) & 0xff) && k <= (hi_ext >> 16);
          if (in_grid && (REPLACE || vlt(U[side ? t + step : t - step], U[t]))) chg[e] = kActive;
        }
      }
      worker_sync<WPC>(worker);
    }
    unsigned long long t_sw = 0;
    if (tid == 0) {
      t_sw = global_timer_ns();
      stage_ns += t_sw - t_pop;
    }

    // ---- 3. sweeps -----------------------------------------------------
    // Min mode: first the direction that leaves the lower halo face behind
    // on each axis (the cell's inflow side; upward on an axis without halo
    // values) if it is a preferred direction, else the first preferred one
    // (in the standard order); then each next sweep reverses the one axis
    // along which the last one left the most active nodes behind (reversing
    // every such axis took more sweeps: a CPU model of first visits of 16^3
    // cells gave 3.5 against 2.9 sweeps on the 257^3 oscillatory field and
    // 13.9 against 8.6 on a 129^3 barrier field).  Replace mode: every
    // preferred direction, then the standard loop.  A sweep
    // covers only the planes from the first one holding an active node.
    int nsw = 0;
    bool converged = false;
    bool all_active = !revisit;  // every node active: no need to look
    int dlast = -1;
    unsigned lm = 0;
    if constexpr (!REPLACE && sizeof(T) == 8) {
      // polish: one pass in the level order read off the FP32 result first;
      // the sweeps below only pick up what it left active
      if (lev_depth > 0) {
        level_pass<T, N, WPC>(U, S, chg,
                              reinterpret_cast<const unsigned short*>(wbase + G::OFF_PERM),
                              reinterpret_cast<const unsigned short*>(wbase + G::OFF_LOFF),
                              lev_depth, tid, worker, kappa, n_updates);
        ++nsw;
        all_active = false;
      }
    }
    auto run = [&](int d) {
      int first = 0, last = G::NPLANES - 1;
      if (!all_active) active_planes<N, WPC>(chg, d, tid, worker, wshared + 12, first, last);
      all_active = false;
      dlast = d;
      if (first > last) {
        lm = 0;  // nothing active: converged without a sweep
        return;
      }
      lm = sweep_cell<T, N, WPC, REPLACE, COMPACT>(U, S, chg, tab, off, list, d, first, last,
                                                   hi_ext, tid, worker, kappa, n_updates,
                                                   wshared + 32);
      ++nsw;
    };
    if constexpr (!REPLACE) {
      // min mode: the direction leaving the lower halo face behind on each
      // axis with halo values (upward where neither face has one), when it
      // is a preferred direction or none is given; else the first preferred
      worker_sync<WPC>(worker);  // fmin complete
      int d0 = 0;
#pragma unroll
      for (int axis = 0; axis < 3; ++axis)
        if (fmin[2 * axis + 1] < fmin[2 * axis]) d0 |= 1 << axis;
      if (!converged && (((pref >> d0) & 1u) || !(pref & kDirMask))) {
        run(d0);
        if (!lm) converged = true;
      } else {
        for (int r = 0; r < 8 && !converged; ++r) {
          const int d = kStdOrder[r];
          if (!((pref >> d) & 1u)) continue;  // bits 0-7: preferred directions
          run(d);
          if (!lm) converged = true;
          break;
        }
      }
    } else {
      for (int r = 0; r < 8 && !converged; ++r) {
        const int d = kStdOrder[r];
        if (!((pref >> d) & 1u)) continue;  // bits 0-7: preferred directions
        run(d);
        if (!lm) converged = true;
      }
    }
    for (int r = 0; !converged; r = (r + 1) & 7) {
      if (nsw >= p.max_sweeps) break;
      run((!REPLACE && dlast >= 0) ? (dlast ^ (int)lm) : kStdOrder[r]);
      if (!lm) converged = true;
    }
    upd_total += n_updates;
    if (revisit) rv_upd += n_updates;
    n_updates = 0;
    if (tid == 0) {
      if (converged) atomicOr(cells.dir + cell, kDirVisited);
      else atomicAnd(cells.dir + cell, ~kDirVisited);
    }
    if (!converged) {
      if constexpr (REPLACE) {
        if (tid == 0) atomicOr(cells.state + cell, kStDirty);  // visit again later
      } else {
        if (tid == 0) set_status(ctl, EIK_ENOCONV);
      }
    }

    unsigned long long t_fl = 0;
    if (tid == 0) {
      t_fl = global_timer_ns();
      sweep_ns += t_fl - t_sw;
    }
    // ---- 4. flag keys, write back, flag downwind neighbours -------------
    T* gu = static_cast<T*>(I.u);
    const long long px = I.px, pxy = I.px * I.py;
    const long long g0 = (long long)(N * cx + 1) + px * (N * cy + 1) + pxy * (N * cz + 1);
    unsigned* fkey = reinterpret_cast<unsigned*>(wshared + 2);  // [6]
    for (int f = wwarp; f < 6; f += WPC) {
      const int axis = f >> 1, upper = f & 1;
      const int ncoord = (axis == 0 ? cx : axis == 1 ? cy : cz) + (upper ? 1 : -1);
      const int nlim = axis == 0 ? I.ncx : axis == 1 ? I.ncy : I.ncz;
      unsigned m = 0xffffffffu, mx = 0u;  // smallest / largest key of the flagging values
      if (ncoord >= 0 && ncoord < nlim) {  // warp-uniform
        for (int q = lane; q < N * N; q += 32) {
          const int a = q % N, b = q / N;
          int i, j, k;
          if (axis == 0) { i = upper ? N - 1 : 0; j = a; k = b; }
          else if (axis == 1) { i = a; j = upper ? N - 1 : 0; k = b; }
          else { i = a; j = b; k = upper ? N - 1 : 0; }
          if (chg[i + N * (j + N * k)] & kBig) {
            const int t = (i + 1) + G::SY * (j + 1) + G::SZ * (k + 1);
            const int step = axis == 0 ? 1 : axis == 1 ? G::SY : G::SZ;
            const T vi = U[t];
            const T vj = U[upper ? t + step : t - step];  // halo value
            // Min mode: only a border value below its neighbour's can be
            // used by the neighbour, and the (possibly stale) halo value is
            // never below the neighbour's current one, so this test misses
            // no inflow.  Replace mode: values may also rise, so every
            // change is passed on.
            if (REPLACE || vi < vj) {
              const unsigned kk = key_of(vi);
              m = kk < m ? kk : m;
              mx = kk > mx ? kk : mx;
            }
          }
        }
        m = __reduce_min_sync(0xffffffffu, m);
        if (p.cell_key == 1) {
          // Eq. 4: the largest flagging value plus the travel time over half
          // a cell and a node, (n h + h) / 2, at the speed of the
          // neighbour's centre node: (n + 1) / 2 times its s = h / F.
          mx = __reduce_max_sync(0xffffffffu, mx);
          if (lane == 0 && m != 0xffffffffu) {
            const int nlc = axis == 0 ? lc + (upper ? 1 : -1)
                          : axis == 1 ? lc + (upper ? I.ncx : -I.ncx)
                                      : lc + (upper ? I.ncx * I.ncy : -I.ncx * I.ncy);
            const int bx = nlc % I.ncx, by = (nlc / I.ncx) % I.ncy, bz = nlc / (I.ncx * I.ncy);
            // centre of the cell's nodes inside the grid (edge cells are partial)
            const int ci = min(N, I.nx - N * bx) / 2, cj = min(N, I.ny - N * by) / 2,
                      ck = min(N, I.nz - N * bz) / 2;
            const T sc = static_cast<const T*>(I.s)[(size_t)nlc * G::N3 + ci + N * (cj + N * ck)];
            if (sc < tinf<T>())  // an exit node at the centre keeps the Eq. 3 value
              m = key_of((float)(float_of_ord(mx) + 0.5f * (float)(N + 1) * (float)sc));
          }
        }
      }
      if (lane == 0) fkey[f] = m;
    }
    worker_sync<WPC>(worker);
    for (int e = tid; e < G::N3; e += NT) {
      if (chg[e] & kWritten) {
        const int i = e % N, j = (e / N) % N, k = e / (N * N);
        gu[g0 + i + px * j + pxy * k] = U[(i + 1) + G::SY * (j + 1) + G::SZ * (k + 1)];
      }
    }
    __threadfence();
    worker_sync<WPC>(worker);
    if (wwarp == 0 && lane < 6) {
      // one lane per face: the six flag sequences run concurrently
      __threadfence();
      const int f = lane;
      const unsigned m = fkey[f];
      if (m != 0xffffffffu) {
        const int axis = f >> 1, upper = f & 1;
        const int ncoord = (axis == 0 ? cx : axis == 1 ? cy : cz) + (upper ? 1 : -1);
        const int ncx2 = axis == 0 ? ncoord : cx;
        const int ncy2 = axis == 1 ? ncoord : cy;
        const int ncz2 = axis == 2 ? ncoord : cz;
        const unsigned nb = (unsigned)(I.cell_base + ncx2 + I.ncx * (ncy2 + I.ncy * ncz2));
        // directions that sweep away from this cell into the neighbour
        const unsigned bit = 1u << axis;
        unsigned dirs = 0;
        for (int d = 0; d < 8; ++d)
          if (((d & bit) != 0) == (upper == 0)) dirs |= 1u << d;
        // the neighbour sees the change on its opposite face
        dirs |= 1u << (kFaceShift + 2 * axis + (upper ^ 1));
        flag_cell(cells, ctl, nb, m, dirs, &n_pushes, p.gated != 0);
      }
      if (p.gated) {
        // first visit done: release downwind neighbours whose last upwind
        // dependency this was
        const unsigned dn = (lane == 0) ? atomicOr(cells.down + cell, 0x100u) : 0u;
        const unsigned dl = __shfl_sync(0x3fu, dn, 0);
        if (!(dl & 0x100u) && ((dl >> f) & 1u)) {
          const int axis = f >> 1, upper = f & 1;
          const int ncoord = (axis == 0 ? cx : axis == 1 ? cy : cz) + (upper ? 1 : -1);
          const int ncx2 = axis == 0 ? ncoord : cx;
          const int ncy2 = axis == 1 ? ncoord : cy;
          const int ncz2 = axis == 2 ? ncoord : cz;
          const unsigned nb = (unsigned)(I.cell_base + ncx2 + I.ncx * (ncy2 + I.ncy * ncz2));
          if (atomicSub(cells.deps + nb, 1) == 1) {
            const unsigned kb = ld_relaxed_u32(cells.key + nb);
            flag_cell(cells, ctl, nb, kb, 0u, &n_pushes, false);
          }
        }
      }
    }
    if (wwarp == 0) __syncwarp();
    if (tid == 0) flag_ns += global_timer_ns() - t_fl;

    // ---- 5. retire -------------------------------------------------------
    if (tid == 0) {
      retire_cell(cells, ctl, (unsigned)cell, slot, &n_pushes);
      busy_ns += global_timer_ns() - t_pop;
      ++n_visits;
      if (revisit) ++n_revisits;
      // the watchdog only needs to see that visits complete: publish every 8th
      if ((n_visits & 7u) == 1u) atomicAdd(&ctl->progress, 8u);
      n_sweeps += (unsigned long long)nsw;
      if (revisit) rv_sweeps += (unsigned long long)nsw;
      if (nsw > max_sweeps_seen) max_sweeps_seen = nsw;
    }
  }

  // counters
  unsigned long long* cnt = ctl->counters[p.pass];
  if (upd_total) atomicAdd(cnt + kCntUpdates, upd_total);
  if (rv_upd) atomicAdd(cnt + kCntRevisitUpdates, rv_upd);
  if (tid == 0) {
    if (n_visits) atomicAdd(cnt + kCntVisits, n_visits);
    if (n_sweeps) atomicAdd(cnt + kCntSweeps, n_sweeps);
    if (n_revisits) atomicAdd(cnt + kCntRevisits, n_revisits);
    if (rv_sweeps) atomicAdd(cnt + kCntRevisitSweeps, rv_sweeps);
    if (max_sweeps_seen) atomicMax(cnt + kCntMaxSweeps, (unsigned long long)max_sweeps_seen);
    if (busy_ns) atomicAdd(cnt + kCntBusyNs, busy_ns);
    atomicAdd(cnt + kCntPopNs, pop_ns);
    atomicAdd(cnt + kCntStageNs, stage_ns);
    atomicAdd(cnt + kCntSweepNs, sweep_ns);
    atomicAdd(cnt + kCntFlagNs, flag_ns);
  }
  if (n_pushes) atomicAdd(cnt + kCntPushes, n_pushes);
}

}  // namespace eik
