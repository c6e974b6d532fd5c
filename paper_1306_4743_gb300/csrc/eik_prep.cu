// eik_prep.cu -- streaming kernels around the persistent cell kernel:
// grid initialisation (the set-up steps of Alg. 3, with the LSM initialisation of Sec. 4),
// cell-value initialisation, queue seeding, the FP32 -> FP64 hand-over of
// the polish, the FP64 residual check and the copy-out to the caller layout.
#include "eik_device.cuh"
#include "eik_prep.h"

namespace eik {

namespace {

// Block-wide reductions (every thread of the block calls them; the result
// is valid in thread 0), so that a streaming kernel makes one atomic per
// block on the shared control words instead of one per warp.
template <typename V, typename Op>
__device__ __forceinline__ V block_reduce(V v, Op op) {
  __shared__ V part[32];
  for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // part[] may still be read by a previous call
  if ((threadIdx.x & 31) == 0) part[w] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 1; k < nw; ++k) v = op(v, part[k]);
  return v;
}
struct MaxOp {
  template <typename V> __device__ V operator()(V a, V b) const { return a > b ? a : b; }
};
struct MinOp {
  template <typename V> __device__ V operator()(V a, V b) const { return a < b ? a : b; }
};
struct SumOp {
  template <typename V> __device__ V operator()(V a, V b) const { return a + b; }
};

__device__ __forceinline__ void block_max_u64(unsigned long long v, unsigned long long* dst) {
  v = block_reduce(v, MaxOp());
  if (threadIdx.x == 0 && v) atomicMax(dst, v);
}

// This block's instance and first unit (row or cell) under the block
// schedule `seg` of one work kind: the last instance whose first block is
// not after blockIdx.x.
struct BlockWork {
  int inst;
  long long first;
};
__device__ __forceinline__ BlockWork block_work(const int* __restrict__ seg, int count, int per) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(seg + mid) <= b) lo = mid;
    else hi = mid;
  }
  BlockWork w;
  w.inst = lo;
  w.first = (long long)(b - __ldg(seg + lo)) * per;
  return w;
}

// Cell values of the cells that hold an exit node (Sec. 4: V^c = min q over
// the cell's exit nodes).  The LSM initialisation also marks the grid
// neighbours of exit nodes active; a neighbour across a cell face lies in
// another cell, which must be queued as well (an exit value never changes,
// so no face flag would reach that cell otherwise).
__device__ __forceinline__ void mark_exit_cells(const CellArrays& c, int cell_base, int ncx, int ncy,
                                                int ncz, int N, int lc, int a, int b, int cc,
                                                int cx, int cy, int cz, unsigned kq) {
  atomicMin(c.key + cell_base + lc, kq);
  if (a == 0 && cx > 0) atomicMin(c.key + cell_base + lc - 1, kq);
  if (a == N - 1 && cx + 1 < ncx) atomicMin(c.key + cell_base + lc + 1, kq);
  if (b == 0 && cy > 0) atomicMin(c.key + cell_base + lc - ncx, kq);
  if (b == N - 1 && cy + 1 < ncy) atomicMin(c.key + cell_base + lc + ncx, kq);
  if (cc == 0 && cz > 0) atomicMin(c.key + cell_base + lc - ncx * ncy, kq);
  if (cc == N - 1 && cz + 1 < ncz) atomicMin(c.key + cell_base + lc + ncx * ncy, kq);
}

__global__ void reset_cells_kernel(const PrepInstance* __restrict__ pi, const int* __restrict__ seg,
                                   int count, CellArrays c) {
  const BlockWork w = block_work(seg, count, kCellsPerBlock);
  const PrepInstance P = pi[w.inst];
  const long long lc = w.first + threadIdx.x;
  if (threadIdx.x < kCellsPerBlock && lc < P.ncells) {
    const int g = P.cell_base + (int)lc;
    c.key[g] = kKeyInf;
    c.state[g] = 0u;
    c.dir[g] = 0u;
    c.inst[g] = w.inst;
    c.next[g] = 0u;
  }
}

// Smallest exit value over the launch, exit-node counts, q validation.  The
// solver works on u - q_min internally (the system is shift invariant), so
// every stored value is >= 0 and orders like its bit pattern.
__global__ void minq_kernel(const PrepInstance* __restrict__ pi, const int* __restrict__ seg,
                            int count, Control* ctl, int* n_src) {
  const BlockWork w = block_work(seg, count, kRowsPerBlock);
  const PrepInstance P = pi[w.inst];
  const long long rows = (long long)P.ny * P.nz;
  unsigned long long minq = ~0ull;
  int nsrc = 0, bad = 0;
  // the block's rows are one contiguous run of mask bytes [lo, hi): read it
  // in 16-byte words where aligned (exit nodes are rare, so almost every
  // word is zero and the pass is this read), bytes at the two ends
  const long long lo = w.first * P.nx;
  const long long hi = (w.first + kRowsPerBlock < rows ? w.first + kRowsPerBlock : rows) * P.nx;
  auto take = [&](long long e) {
    const double qv = P.q[e];
    if (!isfinite(qv)) bad = 1;
    ++nsrc;
    const unsigned long long o = ord_of_double(qv);
    minq = o < minq ? o : minq;
  };
  const uintptr_t base = reinterpret_cast<uintptr_t>(P.mask);
  long long a0 = lo + (long long)((16u - ((base + (uintptr_t)lo) & 15u)) & 15u);
  if (a0 > hi) a0 = hi;
  long long a1 = a0 + ((hi - a0) & ~15ll);
  for (long long e = lo + threadIdx.x; e < a0; e += blockDim.x)
    if (P.mask[e]) take(e);
  for (long long e = a1 + threadIdx.x; e < hi; e += blockDim.x)
    if (P.mask[e]) take(e);
  const uint4* m4 = reinterpret_cast<const uint4*>(P.mask + a0);
  const long long nv = (a1 - a0) >> 4;
  for (long long v = threadIdx.x; v < nv; v += blockDim.x) {
    const uint4 m = __ldg(m4 + v);
    if ((m.x | m.y | m.z | m.w) == 0u) continue;
    for (int t = 0; t < 16; ++t)
      if (P.mask[a0 + 16 * v + t]) take(a0 + 16 * v + t);
  }
  nsrc = block_reduce(nsrc, SumOp());
  bad = block_reduce(bad, MaxOp());
  minq = block_reduce(minq, MinOp());
  if (threadIdx.x == 0) {
    if (nsrc) atomicAdd(n_src + w.inst, nsrc);
    if (bad) atomicExch(&ctl->bad_input, 1);
    if (minq != ~0ull) atomicMin(&ctl->min_q_ord, minq);
  }
}

__device__ __forceinline__ double q_base(const Control* ctl) {
  const double b = double_of_ord(ctl->min_q_ord);
  return isfinite(b) ? b : 0.0;
}

// Padded u: +inf everywhere except exit nodes, which hold q - q_min.
template <typename T>
__global__ void init_u_kernel(const PrepInstance* __restrict__ pi, const int* __restrict__ seg,
                              int count, const Control* ctl) {
  const BlockWork w = block_work(seg, count, kRowsPerBlock);
  const PrepInstance P = pi[w.inst];
  const double qb = q_base(ctl);
  T* u = static_cast<T*>(P.u);
  const long long rows = P.py * P.pz;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long r = w.first + (threadIdx.x >> 5); r < w.first + kRowsPerBlock && r < rows;
       r += nw) {
    const int y = (int)(r % P.py), z = (int)(r / P.py);
    const bool inside = y >= 1 && y <= P.ny && z >= 1 && z <= P.nz;
    const long long lrow = inside ? (long long)P.nx * ((y - 1) + (long long)P.ny * (z - 1)) : 0;
    T* urow = u + r * P.px;
    for (int x = lane; x < P.px; x += 32) {
      T v = tinf<T>();
      if (inside && x >= 1 && x <= P.nx && P.mask[lrow + x - 1]) v = (T)(P.q[lrow + x - 1] - qb);
      urow[x] = v;
    }
  }
}

// |v - lam| for stored values v, lam >= 0 (finite v), from the distance of
// their bit patterns: D steps of v's ulp, exact when both lie in one binade
// and at most twice the true distance across a binade boundary (an upper
// bound, which keeps the fallback test conservative).  Integer pipe and
// FP32 only; +inf when lam is +inf or D does not fit 32 bits.
__device__ __forceinline__ double resid_nn(double v, double lam) {
  const long long iv = __double_as_longlong(v), il = __double_as_longlong(lam);
  const unsigned long long D = (unsigned long long)(iv > il ? iv - il : il - iv);
  if (D == 0ull) return 0.0;
  if (il >= 0x7ff0000000000000ll || (D >> 32)) return CUDART_INF;
  const int ev = (int)(iv >> 52) > 0 ? (int)(iv >> 52) : 1;
  const int pe = ev - 1075 + 127;  // ulp(v) = 2^(ev - 1075) as a float exponent
  if (pe < 1) return 0.0;          // below 2^-126: negligible
  return f64_of_f32_nn(__uint2float_ru((unsigned)D) * __int_as_float(pe << 23));
}

// s = h / F in FP64 from an FP32 reciprocal r and two FMA corrections
// q <- q + r (h - q F): each multiplies the relative error by ~2^-24, so
// from q0 = h r the result is within an ulp of the correctly rounded
// quotient, with five FP64 instructions instead of a division.
__device__ __forceinline__ double slowness(double h, float f) {
  // f and 1/f widened on the integer pipe while both are normal floats
  const float rf = __frcp_rn(f);
  double fd, r;
  if (__builtin_expect(f >= 1.17549435e-38f && f <= 8.50705917e37f, 1)) {
    fd = f64_of_f32_nn(f);
    r = f64_of_f32_nn(rf);
  } else {
    fd = (double)f;
    r = (double)rf;
  }
  const double q0 = h * r;
  const double q1 = fma(fma(-q0, fd, h), r, q0);
  return fma(fma(-q1, fd, h), r, q1);
}

// Cell-blocked slowness s = h / F (FP64, then rounded to T), +inf
// at exit and filler nodes; cell values V^c = min q over exit nodes in the
// cell (Sec. 4, initialisation of cell values), also given to cells that
// hold a grid neighbour of an exit node; input validation.
template <typename T>
__global__ void init_s_kernel(const PrepInstance* __restrict__ pi, const int* __restrict__ seg,
                              int count, CellArrays c, Control* ctl) {
  const BlockWork w = block_work(seg, count, kRowsPerBlock);
  const PrepInstance P = pi[w.inst];
  const int N = P.n, N3 = N * N * N, lg = __ffs(N) - 1, nm = N - 1;
  T* s = static_cast<T*>(P.s);
  double* s64 = static_cast<double*>(P.s64);
  const int ey = N * P.ncy, ex = N * P.ncx;  // extents covered by the cells
  const long long rows = (long long)ey * N * P.ncz;
  const double qb = q_base(ctl);
  const float inv_h = (float)(1.0 / P.h);
  float acc = 0.0f;   // sum of 1 / s = F / h (bucket width): FP32 is plenty
  float accs = 0.0f;  // sum of s (dispersion of s, bulk threshold)
  unsigned long long cnt = 0;
  int bad = 0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long r = w.first + (threadIdx.x >> 5); r < w.first + kRowsPerBlock && r < rows;
       r += nw) {
    const int j = (int)(r % ey), k = (int)(r / ey);
    const int b = j & nm, cc = k & nm, cy = j >> lg, cz = k >> lg;
    const bool row_in = j < P.ny && k < P.nz;
    const long long lrow = row_in ? (long long)P.nx * (j + (long long)P.ny * k) : 0;
    for (int i = lane; i < ex; i += 32) {
      const int a = i & nm, cx = i >> lg;
      const int lc = cx + P.ncx * (cy + P.ncy * cz);
      const long long e = (long long)lc * N3 + a + N * (b + N * cc);
      double sv = CUDART_INF;  // filler nodes of partial edge cells stay fixed
      if (row_in && i < P.nx) {
        const long long lin = lrow + i;
        if (P.mask[lin]) {
          mark_exit_cells(c, P.cell_base, P.ncx, P.ncy, P.ncz, N, lc, a, b, cc, cx, cy, cz,
                          key_of((T)(P.q[lin] - qb)));
        } else {
          const float f = P.F[lin];
          if (!(f > 0.0f) || isinf(f)) {
            bad = 1;
          } else {
            sv = slowness(P.h, f);
            acc += f * inv_h;
            accs += f32_of_f64_nn(sv);
            ++cnt;
          }
        }
      }
      if constexpr (sizeof(T) == 8) s[e] = (T)sv;
      else s[e] = f32_of_f64_rn(sv);
      if (s64) s64[e] = sv;
    }
  }
  acc = block_reduce(acc, SumOp());
  accs = block_reduce(accs, SumOp());
  cnt = block_reduce(cnt, SumOp());
  bad = block_reduce(bad, MaxOp());
  if (threadIdx.x == 0) {
    if (cnt) {
      atomicAdd(&ctl->sum_inv_s, (double)acc);
      atomicAdd(&ctl->sum_s, (double)accs);
      atomicAdd(&ctl->n_s, cnt);
    }
    if (bad) atomicExch(&ctl->bad_input, 1);
  }
}

// Validation verdict, queue origin and bucket width.
__global__ void setup_bulk_kernel(Control* ctl, const int* n_src, int count, int n,
                                  double width_factor, double kappa_rel) {
  if (threadIdx.x || blockIdx.x) return;
  int ok = !ctl->bad_input;
  for (int t = 0; t < count; ++t)
    if (n_src[t] <= 0) ok = 0;
  if (!ok) {
    set_status(ctl, EIK_EINVAL);
    return;
  }
  // The slowness the front advances at: the harmonic mean of s, h / mean(F).
  // (The arithmetic mean is dominated by the slowest nodes: on a field with
  // 30% of its nodes at F = 0.01 it is ~30 h, and buckets that wide let cells
  // far ahead of the front in the fast regions start early and be revisited.)
  const double s_front = ctl->sum_inv_s > 0.0 ? (double)ctl->n_s / ctl->sum_inv_s : 1.0;
  double width = width_factor * (double)n * s_front;
  if (!(width > 0.0) || !isfinite(width)) width = 1.0;
  ctl->base = 0.0f;  // values are stored relative to q_min
  ctl->inv_width = (float)(1.0 / width);
  // change threshold of the FP32 bulk pass in polish mode, in units of
  // (cell edge x front slowness).  Stopping early only leaves values high;
  // the polish starts above the fixed point either way, so the threshold
  // trades bulk visits against polish work.  kappa_rel = 0 chooses it from
  // the dispersion of s, r = mean(s) mean(1 / s) >= 1: 3e-3 r^2, at most 1.
  // Where s is nearly uniform (r ~ 1) a fine bulk leaves the polish least to
  // do; where it spreads widely (r ~ 22 with 30% of the nodes 100x slower)
  // fronts reach cells along faster detours again and again, each time with
  // a full FP32 revisit for a small drop, and a coarse bulk that leaves those
  // drops to the polish measured 26% faster (513^3 barrier field).
  if (!(kappa_rel > 0.0)) {
    double r = 1.0;
    if (ctl->n_s > 0 && ctl->sum_inv_s > 0.0)
      r = (ctl->sum_s / (double)ctl->n_s) * (ctl->sum_inv_s / (double)ctl->n_s);
    if (!(r >= 1.0) || !isfinite(r)) r = 1.0;
    kappa_rel = fmin(3e-3 * r * r, 1.0);
  }
  ctl->kappa_bulk = kappa_rel * (double)n * s_front;
  ctl->cur = 0u;
  ctl->active = 0;
  ctl->queued = 0;
}

// Queue every cell that holds an exit node (the first step of Alg. 1).
__global__ void seed_sources_kernel(int total_cells, CellArrays c, Control* ctl, int pass) {
  if (ctl->status) return;
  unsigned long long pushes = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_cells;
       g += gridDim.x * blockDim.x) {
    if (c.key[g] != kKeyInf) {
      c.state[g] = kStQueued;
      atomicAdd(&ctl->active, 1);
      __threadfence();
      queue_push(c, ctl, (unsigned)g, &pushes);
    }
  }
  if (pushes) atomicAdd(&ctl->counters[pass][kCntPushes], pushes);
}

// FP32 result -> FP64 padded array of the polish; largest finite value.
__global__ void convert_u_kernel(const PolishInstance* __restrict__ pi, const int* __restrict__ seg,
                                 int count, Control* ctl, float lift) {
  const BlockWork w = block_work(seg, count, kRowsPerBlock);
  const PolishInstance P = pi[w.inst];
  const double qb = q_base(ctl);
  const float* u32 = static_cast<const float*>(P.u32);
  double* u64 = static_cast<double*>(P.u64);
  const long long rows = P.py * P.pz;
  unsigned long long mx = 0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long r = w.first + (threadIdx.x >> 5); r < w.first + kRowsPerBlock && r < rows;
       r += nw) {
    const int y = (int)(r % P.py), z = (int)(r / P.py);
    const bool inside = y >= 1 && y <= P.ny && z >= 1 && z <= P.nz;
    const long long lrow = inside ? (long long)P.nx * ((y - 1) + (long long)P.ny * (z - 1)) : 0;
    const float* row32 = u32 + r * P.px32;
    double* row64 = u64 + r * P.px64;
    constexpr int R = 4;  // loads of R nodes per lane in flight at once
    for (int x0 = lane; x0 < P.px64; x0 += 32 * R) {
      unsigned char mk[R];
      float w32[R];
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int x = x0 + 32 * h;
        mk[h] = 0;
        w32[h] = 0.0f;
        if (inside && x >= 1 && x <= P.nx) {
          mk[h] = __ldg(P.mask + lrow + x - 1);
          w32[h] = __ldg(row32 + x);
        }
      }
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int x = x0 + 32 * h;
        if (x >= P.px64) break;
        double v = CUDART_INF;
        if (inside && x >= 1 && x <= P.nx) {
          const long long lin = lrow + x - 1;
          if (mk[h]) {
            v = P.q[lin] - qb;
          } else {
            // Lift the FP32 value above the FP64 fixed point: its rounding
            // error grows at most ~2^-24 u per node along a characteristic (u
            // is stored relative to q_min), so the default lift of 2^-11 u
            // covers paths of up to 2^13 nodes.  The monotone FP64 sweeps
            // then descend to the fixed point.  The lift is formed in FP32
            // (its own rounding, 2^-24 u, is far inside the margin) and
            // widened on the integer pipe: no FP64 instruction per node.
            v = f64_of_f32_nn(w32[h] * lift);
          }
          if (isfinite(v)) {
            const unsigned long long o = ord_of_double(v);
            mx = o > mx ? o : mx;
          }
        }
        row64[x] = v;
      }
    }
  }
  block_max_u64(mx, &ctl->umax_bits);
}

// Polish cell values: the smallest value of the cell's non-fixed nodes, so
// that the polish visits cells in the causal order of the FP32 result.
// A gated launch runs only when the monotone polish left some u below the
// fixed point (check > threshold): the replace-mode fallback.
__device__ __forceinline__ bool fallback_needed(const Control* ctl, double kappa) {
  const double check = __longlong_as_double((long long)ctl->check_bits);
  const double umax = double_of_ord(ctl->umax_bits);
  return check > 4.0 * kappa + 1e-13 * fmax(fabs(umax), 1.0);
}

__global__ void polish_keys_kernel(const PolishInstance* __restrict__ pi,
                                   const int* __restrict__ seg, int count, CellArrays c,
                                   const Control* ctl, int gated, double kappa) {
  if (gated && (ctl->status || !fallback_needed(ctl, kappa))) return;
  const BlockWork w = block_work(seg, count, kCellsPerBlock);
  const PolishInstance P = pi[w.inst];
  const int N = P.n, N3 = N * N * N;
  const double* u64 = static_cast<const double*>(P.u64);
  const double* s64 = static_cast<const double*>(P.s64);
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const long long end = w.first + kCellsPerBlock < P.ncells ? w.first + kCellsPerBlock : P.ncells;
  for (int lc = (int)w.first + (threadIdx.x >> 5); lc < end; lc += warps) {
    const int cx = lc % P.ncx, cy = (lc / P.ncx) % P.ncy, cz = lc / (P.ncx * P.ncy);
    double m = CUDART_INF;
    int at = 0;
    for (int r = lane; r < N3; r += 32) {
      if (!(s64[(long long)lc * N3 + r] < CUDART_INF)) continue;
      const int a = r % N, b = (r / N) % N, cc = r / (N * N);
      const long long x = (long long)N * cx + a + 1, y = (long long)N * cy + b + 1,
                      z = (long long)N * cz + cc + 1;
      const double v = u64[x + P.px64 * (y + P.py * z)];
      if (v < m) {
        m = v;
        at = r;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double mo = __shfl_xor_sync(0xffffffffu, m, o);
      const int ao = __shfl_xor_sync(0xffffffffu, at, o);
      if (mo < m || (mo == m && ao < at)) {
        m = mo;
        at = ao;
      }
    }
    if (lane == 0) {
      const int g = P.cell_base + lc;
      c.key[g] = key_of(m);
      c.state[g] = 0u;
      // first sweep: away from the cell's smallest FP32 value (its upwind side)
      const int a = at % N, b = (at / N) % N, cc = at / (N * N);
      const int d = (a >= N / 2 ? 1 : 0) | (b >= N / 2 ? 2 : 0) | (cc >= N / 2 ? 4 : 0);
      c.dir[g] = 1u << d;
      c.next[g] = 0u;
    }
  }
}

// Dependency graph of the polish, read off the FP32 result.  Across each
// face, B feeds C when some border node of C (not fixed) has a larger value
// than its neighbour in B.  An edge B -> C is kept only when B's cell value
// is below C's (ties: lower cell id), so the kept graph is acyclic; deps[C]
// counts kept incoming edges, down[C] marks kept outgoing faces.  A cell is
// queued once deps[C] reaches 0; an edge that was dropped is still honoured
// by the flag protocol, which re-queues C if B's later values reach it.
__global__ void polish_graph_kernel(const PolishInstance* __restrict__ pi,
                                    const int* __restrict__ seg, int count, CellArrays c) {
  const BlockWork w = block_work(seg, count, kCellsPerBlock);
  const PolishInstance P = pi[w.inst];
  const int N = P.n, N3 = N * N * N;
  const double* u64 = static_cast<const double*>(P.u64);
  const double* s64 = static_cast<const double*>(P.s64);
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const long long sy = P.px64, sz = P.px64 * P.py;
  const long long end = w.first + kCellsPerBlock < P.ncells ? w.first + kCellsPerBlock : P.ncells;
  for (int lc = (int)w.first + (threadIdx.x >> 5); lc < end; lc += warps) {
    const int cx = lc % P.ncx, cy = (lc / P.ncx) % P.ncy, cz = lc / (P.ncx * P.ncy);
    const int g = P.cell_base + lc;
    const unsigned kc = c.key[g];
    int deps = 0;
    unsigned down = 0;
    for (int f = 0; f < 6; ++f) {
      const int axis = f >> 1, upper = f & 1;
      const int ncoord = (axis == 0 ? cx : axis == 1 ? cy : cz) + (upper ? 1 : -1);
      const int nlim = axis == 0 ? P.ncx : axis == 1 ? P.ncy : P.ncz;
      if (ncoord < 0 || ncoord >= nlim) continue;
      const int nlc = axis == 0 ? lc + (upper ? 1 : -1)
                    : axis == 1 ? lc + (upper ? P.ncx : -P.ncx)
                                : lc + (upper ? P.ncx * P.ncy : -P.ncx * P.ncy);
      bool in = false, out = false;
      for (int q = lane; q < N * N; q += 32) {
        const int a = q % N, b = q / N;
        int i, j, k;
        if (axis == 0) { i = upper ? N - 1 : 0; j = a; k = b; }
        else if (axis == 1) { i = a; j = upper ? N - 1 : 0; k = b; }
        else { i = a; j = b; k = upper ? N - 1 : 0; }
        const long long gi = (long long)N * cx + i, gj = (long long)N * cy + j,
                        gk = (long long)N * cz + k;
        if (gi >= P.nx || gj >= P.ny || gk >= P.nz) continue;
        // neighbour node across the face, in cell nlc
        int i2 = i, j2 = j, k2 = k;
        if (axis == 0) i2 = upper ? 0 : N - 1;
        else if (axis == 1) j2 = upper ? 0 : N - 1;
        else k2 = upper ? 0 : N - 1;
        const long long gi2 = gi + (axis == 0 ? (upper ? 1 : -1) : 0);
        const long long gj2 = gj + (axis == 1 ? (upper ? 1 : -1) : 0);
        const long long gk2 = gk + (axis == 2 ? (upper ? 1 : -1) : 0);
        if (gi2 >= P.nx || gj2 >= P.ny || gk2 >= P.nz) continue;
        const double uc = u64[(gi + 1) + sy * (gj + 1) + sz * (gk + 1)];
        const double ub = u64[(gi2 + 1) + sy * (gj2 + 1) + sz * (gk2 + 1)];
        const bool c_free = s64[(long long)lc * N3 + i + N * (j + N * k)] < CUDART_INF;
        const bool b_free = s64[(long long)nlc * N3 + i2 + N * (j2 + N * k2)] < CUDART_INF;
        if (c_free && ub < uc) in = true;
        if (b_free && uc < ub) out = true;
      }
      in = __any_sync(0xffffffffu, in);
      out = __any_sync(0xffffffffu, out);
      const int gb = P.cell_base + nlc;
      const unsigned kb = c.key[gb];
      const bool b_first = kb < kc || (kb == kc && gb < g);
      if (in && b_first) ++deps;
      if (out && !b_first) down |= 1u << f;
    }
    if (lane == 0) {
      c.deps[g] = deps;
      c.down[g] = down;
    }
  }
}

// Level order of each cell's nodes for the first polish visit: a node's
// in-cell upwind neighbours under the FP32 result (the smaller neighbour
// on an axis, if below the node; both on an FP32 tie) come first.  Levels
// are the layers of Kahn's topological order: level 0 holds the nodes with
// no in-cell upwind neighbour, and a node joins the layer after the one in
// which its last upwind neighbour was taken (so level = longest upwind
// chain).  Each layer is appended to the node list in shared memory and
// becomes a run of lev_perm; lev_off[l] is where layer l starts.  The
// filler of partial cells is in no layer (lev_off[depth] counts the cell's
// grid nodes); exit nodes are in layer 0, where the pass takes them without
// computing (their s is +inf).  One block per cell; cells deeper than
// kMaxLevels - 1 get no table (lev_depth 0).
__global__ void polish_levels_kernel(const PolishInstance* __restrict__ pi, int total_cells,
                                     CellArrays c) {
  __shared__ unsigned char up[4096];   // bit 2a: -axis a neighbour upwind, 2a + 1: +axis a
  __shared__ unsigned indeg[1024];     // upwind neighbours not yet taken, a byte per node
  __shared__ unsigned short lst[4096];  // nodes in level order
  __shared__ unsigned short offs[kMaxLevels + 1];
  __shared__ int tail;
  for (int g = blockIdx.x; g < total_cells; g += gridDim.x) {
    const PolishInstance P = pi[c.inst[g]];
    const int N = P.n, N3 = N * N * N, lg = __ffs(N) - 1, nm = N - 1;
    const float* u32 = static_cast<const float*>(P.u32);
    const double* s64 = static_cast<const double*>(P.s64);
    const long long sy = P.px32, sz = P.px32 * P.py;
    const int lc = g - P.cell_base;
    const int cx = lc % P.ncx, cy = (lc / P.ncx) % P.ncy, cz = lc / (P.ncx * P.ncy);
    if (threadIdx.x == 0) tail = 0;
    for (int w = threadIdx.x; w < (N3 + 3) / 4; w += blockDim.x) indeg[w] = 0u;
    __syncthreads();
    for (int r = threadIdx.x; r < N3; r += blockDim.x) {
      const int a = r & nm, b = (r >> lg) & nm, cc = r >> (2 * lg);
      // the filler of a partial cell lies outside the grid; it holds +inf, so
      // it is no node's upwind neighbour either
      const bool filler = N * cx + a >= P.nx || N * cy + b >= P.ny || N * cz + cc >= P.nz;
      unsigned m = 0;
      if (!filler && s64[(long long)lc * N3 + r] < CUDART_INF) {
        const long long t = (long long)(N * cx + a + 1) + sy * (N * cy + b + 1) + sz * (N * cz + cc + 1);
        const float v = u32[t];
        const int co[3] = {a, b, cc};
        const long long st[3] = {1, sy, sz};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          const float lo = u32[t - st[ax]], hi = u32[t + st[ax]];
          if (co[ax] > 0 && lo < v && lo <= hi) m |= 1u << (2 * ax);
          if (co[ax] < N - 1 && hi < v && hi <= lo) m |= 1u << (2 * ax + 1);
        }
      }
      up[r] = (unsigned char)m;
      if (m) {
        atomicAdd(&indeg[r >> 2], (unsigned)__popc(m) << (8 * (r & 3)));
      } else if (!filler) {
        const unsigned act = __activemask();  // warp-aggregated append
        const int leader = __ffs(act) - 1, lane = threadIdx.x & 31;
        int base = 0;
        if (lane == leader) base = atomicAdd(&tail, __popc(act));
        base = __shfl_sync(act, base, leader);
        lst[base + __popc(act & ((1u << lane) - 1u))] = (unsigned short)r;
      }
    }
    __syncthreads();
    // layer by layer: taking a node releases the neighbours it is upwind of
    int lo = 0, depth = 0;
    bool ok = true;
    for (;;) {
      const int hi = tail;  // this layer: lst[lo, hi)
      if (hi == lo) break;
      if (depth >= kMaxLevels) {
        ok = false;
        break;
      }
      if (threadIdx.x == 0) offs[depth] = (unsigned short)lo;
      ++depth;
      __syncthreads();  // everyone has read tail before the appends below
      for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        const int x = lst[e];
        const int co[3] = {x & nm, (x >> lg) & nm, x >> (2 * lg)};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          const int step = 1 << (lg * ax);
          // x is the -ax neighbour of y = x + step (y's bit 2 ax) and the
          // +ax neighbour of y = x - step (y's bit 2 ax + 1)
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const bool inside = side == 0 ? co[ax] < N - 1 : co[ax] > 0;
            if (!inside) continue;
            const int y = side == 0 ? x + step : x - step;
            if (!((up[y] >> (2 * ax + side)) & 1u)) continue;
            const unsigned sh = 8 * (y & 3);
            const unsigned old = atomicSub(&indeg[y >> 2], 1u << sh);
            if (((old >> sh) & 0xffu) == 1u) lst[atomicAdd(&tail, 1)] = (unsigned short)y;
          }
        }
      }
      lo = hi;
      __syncthreads();  // the next layer is complete
    }
    if (threadIdx.x == 0) c.lev_depth[g] = ok ? depth : 0;
    if (ok) {
      unsigned short* off = c.lev_off + (size_t)g * (kMaxLevels + 1);
      for (int l = threadIdx.x; l < depth; l += blockDim.x) off[l] = offs[l];
      if (threadIdx.x == 0) off[depth] = (unsigned short)lo;
      unsigned short* perm = c.lev_perm + (size_t)g * N3;
      for (int e = threadIdx.x; e < lo; e += blockDim.x) perm[e] = lst[e];
    }
    __syncthreads();  // shared arrays are reused by the next cell
  }
}

// Queue the cells that wait for nothing.
__global__ void seed_ready_kernel(int total_cells, CellArrays c, Control* ctl) {
  if (ctl->status) return;
  unsigned long long pushes = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_cells;
       g += gridDim.x * blockDim.x) {
    if (c.deps[g] == 0) {
      c.state[g] = kStQueued;
      atomicAdd(&ctl->active, 1);
      __threadfence();
      queue_push(c, ctl, (unsigned)g, &pushes);
    }
  }
  if (pushes) atomicAdd(&ctl->counters[1][kCntPushes], pushes);
}

__global__ void setup_polish_kernel(Control* ctl, int gated, double kappa) {
  if (threadIdx.x || blockIdx.x) return;
  if (ctl->status) return;
  if (gated && !fallback_needed(ctl, kappa)) return;
  if (gated) {  // the final statistics are taken again after the fallback
    ctl->resid_bits = 0ull;
    ctl->final_umax_bits = 0ull;
    ctl->nonfinite = 0ull;
  }
  const double umax = double_of_ord(ctl->umax_bits);
  double width = 1.0 / (double)ctl->inv_width;
  const double span = umax - (double)ctl->base;
  if (isfinite(span) && span / width > kNumBuckets / 2) width = span / (kNumBuckets / 2);
  ctl->inv_width = (float)(1.0 / width);
  ctl->cur = 0u;
  ctl->active = 0;
  ctl->queued = 0;
  ctl->progress = 0u;
}

// Queue every cell for the polish.
__global__ void seed_all_kernel(int total_cells, CellArrays c, Control* ctl, int pass, int gated,
                                double kappa) {
  if (ctl->status) return;
  if (gated && !fallback_needed(ctl, kappa)) return;
  unsigned long long pushes = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_cells;
       g += gridDim.x * blockDim.x) {
    c.state[g] = kStQueued;
    atomicAdd(&ctl->active, 1);
    __threadfence();
    queue_push(c, ctl, (unsigned)g, &pushes);
  }
  if (pushes) atomicAdd(&ctl->counters[pass][kCntPushes], pushes);
}

// max |u - Lambda(u)| over non-exit grid nodes (FP64), count of non-finite
// values, largest finite value, and the copy-out to the caller's layout.
// Lambda is the sweeps' FP64 local solve (eik_selftest_local_solve pins it
// to the direct FP64 closed forms): with `sqrt(double)` this pass was FP64-
// pipe bound at ~1.6 ms per 257^3 grid.
// MODE 0 (after the monotone polish) also records the residual as the
// fallback check; MODE 1 is the final pass of the FP64 path; MODE 2 runs
// only when the replace-mode fallback ran, and redoes MODE 0's final part.
// Blocks take grid rows (fixed j, k) and threads the i of a row.
template <int MODE>
__global__ void residual_extract_kernel(const FinalInstance* __restrict__ fi,
                                        const int* __restrict__ seg, int count, Control* ctl,
                                        double kappa) {
  if (MODE == 2 && (ctl->status || !fallback_needed(ctl, kappa))) return;
  const BlockWork w = block_work(seg, count, kRowsPerBlock);
  const FinalInstance P = fi[w.inst];
  const double qb = q_base(ctl);
  const bool shift = qb != 0.0;
  const double* u = static_cast<const double*>(P.u64);
  const double* s = static_cast<const double*>(P.s64);
  const int lg = __ffs(P.n) - 1, nm = P.n - 1;
  const long long N3 = 1ll << (3 * lg);
  const long long sy = P.px64, sz = P.px64 * P.py;
  const int rows = P.ny * P.nz;
  unsigned long long rmax = 0, umax = 0, nbad = 0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = (int)w.first + (threadIdx.x >> 5); row < w.first + kRowsPerBlock && row < rows;
       row += nw) {
    const int j = row % P.ny, k = row / P.ny;
    const long long rbase = (long long)row * P.nx;
    const long long tbase = 1 + sy * (j + 1) + sz * (k + 1);
    const long long cbase = (long long)P.ncx * ((j >> lg) + (long long)P.ncy * (k >> lg));
    const int in_cell = ((j & nm) << lg) + ((k & nm) << (2 * lg));
    for (int i = lane; i < P.nx; i += 32) {
      const long long t = tbase + i;
      const double v = u[t];
      const long long e = rbase + i;
      P.out[e] = P.mask[e] ? P.q[e] : (shift ? v + qb : v);
      // finiteness and the exit test on the bit patterns (stored values and
      // s are >= 0): each FP64 compare costs a slot of the narrow FP64 pipe,
      // which this pass is bound by
      if ((__double_as_longlong(v) & 0x7ff0000000000000ll) == 0x7ff0000000000000ll) {
        ++nbad;
        continue;
      }
      const unsigned long long o = ord_of_double(v);
      umax = o > umax ? o : umax;
      const double sv = s[(cbase + (i >> lg)) * N3 + (i & nm) + in_cell];
      if (dbits(sv) >= dbits(CUDART_INF)) continue;  // exit node
      const double ax = nmin(u[t - 1], u[t + 1]);
      const double ay = nmin(u[t - sy], u[t + sy]);
      const double az = nmin(u[t - sz], u[t + sz]);
      const double lam = local_solve(ax, ay, az, sv);
      // A value left below the fixed point (lift too small) or above it (a
      // flag skipped on the FP32 error bound) both show here and send the
      // solve to the replace-mode fallback.
      const unsigned long long rb = (unsigned long long)__double_as_longlong(resid_nn(v, lam));
      rmax = rb > rmax ? rb : rmax;
    }
  }
  rmax = block_reduce(rmax, MaxOp());
  umax = block_reduce(umax, MaxOp());
  nbad = block_reduce(nbad, SumOp());
  if (threadIdx.x == 0) {
    if (MODE == 0 && rmax) atomicMax(&ctl->check_bits, rmax);
    if (rmax) atomicMax(&ctl->resid_bits, rmax);
    if (umax) atomicMax(&ctl->final_umax_bits, umax);
    if (nbad) atomicAdd(&ctl->nonfinite, nbad);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: block schedule and launchers.
size_t segment_table_bytes(int count) {
  return (size_t)kNumSegKinds * (size_t)(count + 1) * sizeof(int);
}

void make_segments(int count, const SegSizes* sizes, int* host_seg, int* totals) {
  const long long per[kNumSegKinds] = {kRowsPerBlock, kRowsPerBlock, kRowsPerBlock,
                                       kRowsPerBlock, kCellsPerBlock};
  for (int k = 0; k < kNumSegKinds; ++k) {
    int* t = host_seg + (size_t)k * (count + 1);
    long long acc = 0;
    for (int i = 0; i < count; ++i) {
      t[i] = (int)acc;
      const long long u = sizes[i].units[k];
      acc += (u + per[k] - 1) / per[k];
    }
    t[count] = (int)acc;
    totals[k] = (int)acc;
  }
}

static inline const int* seg_of(const Segments& g, int kind) {
  return g.dev + (size_t)kind * (g.count + 1);
}
static inline unsigned blocks_of(const Segments& g, int kind) {
  return (unsigned)(g.total[kind] > 0 ? g.total[kind] : 1);
}

cudaError_t launch_bulk_init(const PrepInstance* d_pi, const Segments& g, int total_cells,
                             CellArrays cells, Control* ctl, int* n_src, bool fp64, int n,
                             double width_factor, double kappa_rel, cudaStream_t st,
                             int& launches) {
  const int c = g.count;
  launches += 6;
  reset_cells_kernel<<<blocks_of(g, kSegCells), 256, 0, st>>>(d_pi, seg_of(g, kSegCells), c, cells);
  minq_kernel<<<blocks_of(g, kSegRows), 256, 0, st>>>(d_pi, seg_of(g, kSegRows), c, ctl, n_src);
  if (fp64) {
    init_u_kernel<double><<<blocks_of(g, kSegPadB), 256, 0, st>>>(d_pi, seg_of(g, kSegPadB), c, ctl);
    init_s_kernel<double><<<blocks_of(g, kSegCellRows), 256, 0, st>>>(
        d_pi, seg_of(g, kSegCellRows), c, cells, ctl);
  } else {
    init_u_kernel<float><<<blocks_of(g, kSegPadB), 256, 0, st>>>(d_pi, seg_of(g, kSegPadB), c, ctl);
    init_s_kernel<float><<<blocks_of(g, kSegCellRows), 256, 0, st>>>(
        d_pi, seg_of(g, kSegCellRows), c, cells, ctl);
  }
  setup_bulk_kernel<<<1, 32, 0, st>>>(ctl, n_src, c, n, width_factor, kappa_rel);
  seed_sources_kernel<<<(unsigned)((total_cells + 255) / 256), 256, 0, st>>>(total_cells, cells,
                                                                            ctl, 0);
  return cudaGetLastError();
}

cudaError_t launch_polish_prep(const PolishInstance* d_pi, const Segments& g, int total_cells,
                               CellArrays cells, Control* ctl, float lift, cudaStream_t st,
                               int& launches) {
  const int c = g.count;
  launches += cells.lev_depth ? 6 : 5;
  convert_u_kernel<<<blocks_of(g, kSegPad64), 256, 0, st>>>(d_pi, seg_of(g, kSegPad64), c, ctl,
                                                             1.0f + lift);
  polish_keys_kernel<<<blocks_of(g, kSegCells), 256, 0, st>>>(d_pi, seg_of(g, kSegCells), c, cells,
                                                              ctl, 0, 0.0);
  polish_graph_kernel<<<blocks_of(g, kSegCells), 256, 0, st>>>(d_pi, seg_of(g, kSegCells), c,
                                                               cells);
  if (cells.lev_depth)
    polish_levels_kernel<<<(unsigned)total_cells, 256, 0, st>>>(d_pi, total_cells, cells);
  setup_polish_kernel<<<1, 32, 0, st>>>(ctl, 0, 0.0);
  seed_ready_kernel<<<(unsigned)((total_cells + 255) / 256), 256, 0, st>>>(total_cells, cells,
                                                                          ctl);
  return cudaGetLastError();
}

cudaError_t launch_fallback_prep(const PolishInstance* d_pi, const FinalInstance* d_fi,
                                 const Segments& g, int total_cells, CellArrays cells,
                                 Control* ctl, double kappa, cudaStream_t st, int& launches) {
  const int c = g.count;
  launches += 4;
  residual_extract_kernel<0><<<blocks_of(g, kSegRows), 256, 0, st>>>(d_fi, seg_of(g, kSegRows), c,
                                                                     ctl, kappa);
  polish_keys_kernel<<<blocks_of(g, kSegCells), 256, 0, st>>>(d_pi, seg_of(g, kSegCells), c, cells,
                                                              ctl, 1, kappa);
  setup_polish_kernel<<<1, 32, 0, st>>>(ctl, 1, kappa);
  seed_all_kernel<<<(unsigned)((total_cells + 255) / 256), 256, 0, st>>>(total_cells, cells, ctl,
                                                                        2, 1, kappa);
  return cudaGetLastError();
}

cudaError_t launch_residual_extract(const FinalInstance* d_fi, const Segments& g, Control* ctl,
                                    bool after_fallback, double kappa, cudaStream_t st,
                                    int& launches) {
  const int c = g.count;
  launches += 1;
  if (after_fallback)
    residual_extract_kernel<2><<<blocks_of(g, kSegRows), 256, 0, st>>>(d_fi, seg_of(g, kSegRows),
                                                                       c, ctl, kappa);
  else
    residual_extract_kernel<1><<<blocks_of(g, kSegRows), 256, 0, st>>>(d_fi, seg_of(g, kSegRows),
                                                                       c, ctl, kappa);
  return cudaGetLastError();
}

}  // namespace eik
