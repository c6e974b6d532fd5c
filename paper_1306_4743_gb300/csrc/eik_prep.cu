// eik_prep.cu -- streaming kernels around the persistent cell kernel:
// grid initialisation (Alg. 3 l.1-4 with the LSM initialisation of Sec. 4),
// cell-value initialisation, queue seeding, the FP32 -> FP64 hand-over of
// the polish, the FP64 residual check and the copy-out to the caller layout.
#include "eik_device.cuh"
#include "eik_prep.h"

namespace eik {

namespace {

__device__ __forceinline__ void block_max_u64(unsigned long long v, unsigned long long* dst) {
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(dst, v);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void reset_cells_kernel(const PrepInstance* __restrict__ pi, int count, CellArrays c) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const PrepInstance P = pi[ii];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P.ncells;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = P.cell_base + (int)e;
    c.key[g] = kKeyInf;
    c.state[g] = 0u;
    c.dir[g] = 0u;
    c.inst[g] = ii;
    c.next[g] = 0u;
  }
}

// Padded u: +inf everywhere except exit nodes, which hold q.
template <typename T>
__global__ void init_u_kernel(const PrepInstance* __restrict__ pi, int count) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const PrepInstance P = pi[ii];
  T* u = static_cast<T*>(P.u);
  const long long total = P.px * P.py * P.pz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e % P.px, y = (e / P.px) % P.py, z = e / (P.px * P.py);
    T v = tinf<T>();
    if (x >= 1 && x <= P.nx && y >= 1 && y <= P.ny && z >= 1 && z <= P.nz) {
      const long long lin = (x - 1) + P.nx * ((y - 1) + (long long)P.ny * (z - 1));
      if (P.mask[lin]) v = (T)P.q[lin];
    }
    u[e] = v;
  }
}

// Cell-blocked slowness s = h / F (FP64 division, then rounded to T), +inf
// at exit and filler nodes; cell values V^c = min q over exit nodes in the
// cell (Sec. 4, initialisation of cell values), also given to cells that
// hold a grid neighbour of an exit node; input validation.
template <typename T>
__global__ void init_s_kernel(const PrepInstance* __restrict__ pi, int count, CellArrays c,
                              Control* ctl, int* n_src) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const PrepInstance P = pi[ii];
  const int N = P.n, N3 = N * N * N;
  T* s = static_cast<T*>(P.s);
  double* s64 = static_cast<double*>(P.s64);
  const long long total = (long long)P.ncells * N3;
  double acc = 0.0;
  unsigned long long cnt = 0;
  int bad = 0, nsrc = 0;
  unsigned long long minq = ~0ull;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int lc = (int)(e / N3), r = (int)(e % N3);
    const int a = r % N, b = (r / N) % N, cc = r / (N * N);
    const int cx = lc % P.ncx, cy = (lc / P.ncx) % P.ncy, cz = lc / (P.ncx * P.ncy);
    const long long i = (long long)N * cx + a, j = (long long)N * cy + b, k = (long long)N * cz + cc;
    double sv = CUDART_INF;
    if (i < P.nx && j < P.ny && k < P.nz) {
      const long long lin = i + P.nx * (j + (long long)P.ny * k);
      if (P.mask[lin]) {
        const double qv = P.q[lin];
        if (!isfinite(qv)) bad = 1;
        ++nsrc;
        const unsigned kq = key_of((T)qv);
        atomicMin(c.key + P.cell_base + lc, kq);
        // The LSM initialisation marks the grid neighbours of exit nodes
        // active; a neighbour across a cell face lies in another cell, which
        // must be queued as well (an exit value never changes, so no face
        // flag would reach that cell otherwise).
        if (a == 0 && cx > 0) atomicMin(c.key + P.cell_base + lc - 1, kq);
        if (a == N - 1 && cx + 1 < P.ncx) atomicMin(c.key + P.cell_base + lc + 1, kq);
        if (b == 0 && cy > 0) atomicMin(c.key + P.cell_base + lc - P.ncx, kq);
        if (b == N - 1 && cy + 1 < P.ncy) atomicMin(c.key + P.cell_base + lc + P.ncx, kq);
        if (cc == 0 && cz > 0) atomicMin(c.key + P.cell_base + lc - P.ncx * P.ncy, kq);
        if (cc == N - 1 && cz + 1 < P.ncz)
          atomicMin(c.key + P.cell_base + lc + P.ncx * P.ncy, kq);
        const unsigned long long o = ord_of_double(qv);
        minq = o < minq ? o : minq;
      } else {
        const float f = P.F[lin];
        if (!(f > 0.0f) || isinf(f)) {
          bad = 1;
        } else {
          sv = P.h / (double)f;
          acc += sv;
          ++cnt;
        }
      }
    }
    s[e] = (T)sv;
    if (s64) s64[e] = sv;
  }
  acc = warp_sum(acc);
  for (int o = 16; o; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    nsrc += __shfl_xor_sync(0xffffffffu, nsrc, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, minq, o);
    minq = w < minq ? w : minq;
  }
  if ((threadIdx.x & 31) == 0) {
    if (cnt) {
      atomicAdd(&ctl->sum_s, acc);
      atomicAdd(&ctl->n_s, cnt);
    }
    if (nsrc) atomicAdd(n_src + ii, nsrc);
    if (bad) atomicExch(&ctl->bad_input, 1);
    if (minq != ~0ull) atomicMin(&ctl->min_q_ord, minq);
  }
}

// Validation verdict, queue origin and bucket width.
__global__ void setup_bulk_kernel(Control* ctl, const int* n_src, int count, int n,
                                  double width_factor) {
  if (threadIdx.x || blockIdx.x) return;
  int ok = !ctl->bad_input;
  for (int t = 0; t < count; ++t)
    if (n_src[t] <= 0) ok = 0;
  if (!ok) {
    set_status(ctl, EIK_EINVAL);
    return;
  }
  const double qmin = double_of_ord(ctl->min_q_ord);
  const double mean_s = ctl->n_s ? ctl->sum_s / (double)ctl->n_s : 1.0;
  double width = width_factor * (double)n * mean_s;
  if (!(width > 0.0) || !isfinite(width)) width = 1.0;
  ctl->base = __double2float_rd(qmin);
  ctl->inv_width = (float)(1.0 / width);
  ctl->cur = 0u;
  ctl->active = 0;
  ctl->queued = 0;
}

// Queue every cell that holds an exit node (Alg. 1 l.2).
__global__ void seed_sources_kernel(int total_cells, CellArrays c, Control* ctl) {
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
  if (pushes) atomicAdd(&ctl->counters[0][kCntPushes], pushes);
}

// FP32 result -> FP64 padded array of the polish; largest finite value.
__global__ void convert_u_kernel(const PolishInstance* __restrict__ pi, int count, Control* ctl) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const PolishInstance P = pi[ii];
  const float* u32 = static_cast<const float*>(P.u32);
  double* u64 = static_cast<double*>(P.u64);
  const long long total = P.px64 * P.py * P.pz;
  unsigned long long mx = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long x = e % P.px64, y = (e / P.px64) % P.py, z = e / (P.px64 * P.py);
    double v = CUDART_INF;
    if (x >= 1 && x <= P.nx && y >= 1 && y <= P.ny && z >= 1 && z <= P.nz) {
      const long long lin = (x - 1) + P.nx * ((y - 1) + (long long)P.ny * (z - 1));
      v = P.mask[lin] ? P.q[lin] : (double)u32[x + P.px32 * (y + P.py * z)];
      if (isfinite(v)) {
        const unsigned long long o = ord_of_double(v);
        mx = o > mx ? o : mx;
      }
    }
    u64[e] = v;
  }
  block_max_u64(mx, &ctl->umax_bits);
}

// Polish cell values: the smallest value of the cell's non-fixed nodes, so
// that the polish visits cells in the causal order of the FP32 result.
__global__ void polish_keys_kernel(const PolishInstance* __restrict__ pi, int count,
                                   CellArrays c) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const PolishInstance P = pi[ii];
  const int N = P.n, N3 = N * N * N;
  const double* u64 = static_cast<const double*>(P.u64);
  const double* s64 = static_cast<const double*>(P.s64);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int lc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; lc < P.ncells; lc += warps) {
    const int cx = lc % P.ncx, cy = (lc / P.ncx) % P.ncy, cz = lc / (P.ncx * P.ncy);
    double m = CUDART_INF;
    for (int r = lane; r < N3; r += 32) {
      if (!(s64[(long long)lc * N3 + r] < CUDART_INF)) continue;
      const int a = r % N, b = (r / N) % N, cc = r / (N * N);
      const long long x = (long long)N * cx + a + 1, y = (long long)N * cy + b + 1,
                      z = (long long)N * cz + cc + 1;
      const double v = u64[x + P.px64 * (y + P.py * z)];
      m = v < m ? v : m;
    }
    for (int o = 16; o; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      const int g = P.cell_base + lc;
      c.key[g] = key_of(m);
      c.state[g] = 0u;
      c.dir[g] = 0u;
      c.next[g] = 0u;
    }
  }
}

__global__ void setup_polish_kernel(Control* ctl) {
  if (threadIdx.x || blockIdx.x) return;
  if (ctl->status) return;
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
__global__ void seed_all_kernel(int total_cells, CellArrays c, Control* ctl) {
  if (ctl->status) return;
  unsigned long long pushes = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_cells;
       g += gridDim.x * blockDim.x) {
    c.state[g] = kStQueued;
    atomicAdd(&ctl->active, 1);
    __threadfence();
    queue_push(c, ctl, (unsigned)g, &pushes);
  }
  if (pushes) atomicAdd(&ctl->counters[1][kCntPushes], pushes);
}

// max |u - Lambda(u)| over non-exit grid nodes (FP64), count of non-finite
// values, largest finite value; then copy-out to the caller's layout.
__global__ void residual_extract_kernel(const FinalInstance* __restrict__ fi, int count,
                                        Control* ctl) {
  const int ii = blockIdx.y;
  if (ii >= count) return;
  const FinalInstance P = fi[ii];
  const double* u = static_cast<const double*>(P.u64);
  const double* s = static_cast<const double*>(P.s64);
  const int N = P.n, N3 = N * N * N;
  const long long total = (long long)P.nx * P.ny * P.nz;
  const long long sy = P.px64, sz = P.px64 * P.py;
  unsigned long long rmax = 0, umax = 0, nbad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % P.nx, j = (e / P.nx) % P.ny, k = e / ((long long)P.nx * P.ny);
    const long long t = (i + 1) + sy * (j + 1) + sz * (k + 1);
    const double v = u[t];
    P.out[e] = v;
    if (!isfinite(v)) {
      ++nbad;
      continue;
    }
    const unsigned long long o = ord_of_double(v);
    umax = o > umax ? o : umax;
    const long long cx = i / N, cy = j / N, cz = k / N;
    const long long lc = cx + P.ncx * (cy + (long long)P.ncy * cz);
    const double sv = s[lc * N3 + (i % N) + N * ((j % N) + N * (k % N))];
    if (!(sv < CUDART_INF)) continue;  // exit node
    const double ax = fmin(u[t - 1], u[t + 1]);
    const double ay = fmin(u[t - sy], u[t + sy]);
    const double az = fmin(u[t - sz], u[t + sz]);
    const double r = fabs(v - local_solve(ax, ay, az, sv));
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
    rmax = rb > rmax ? rb : rmax;
  }
  block_max_u64(rmax, &ctl->resid_bits);
  block_max_u64(umax, &ctl->umax_bits);
  for (int o = 16; o; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
  if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(&ctl->nonfinite, nbad);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers.
static dim3 stream_grid(long long work, int count, int sms) {
  long long blocks = (work + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return dim3((unsigned)blocks, (unsigned)count, 1);
}

cudaError_t launch_bulk_init(const PrepInstance* d_pi, int count, long long max_padded,
                             long long max_cellnodes, int max_cells, int total_cells,
                             CellArrays cells, Control* ctl, int* n_src, bool fp64, int n,
                             double width_factor, int sms, cudaStream_t st) {
  reset_cells_kernel<float><<<stream_grid(max_cells, count, sms), 256, 0, st>>>(d_pi, count, cells);
  if (fp64) {
    init_u_kernel<double><<<stream_grid(max_padded, count, sms), 256, 0, st>>>(d_pi, count);
    init_s_kernel<double>
        <<<stream_grid(max_cellnodes, count, sms), 256, 0, st>>>(d_pi, count, cells, ctl, n_src);
  } else {
    init_u_kernel<float><<<stream_grid(max_padded, count, sms), 256, 0, st>>>(d_pi, count);
    init_s_kernel<float>
        <<<stream_grid(max_cellnodes, count, sms), 256, 0, st>>>(d_pi, count, cells, ctl, n_src);
  }
  setup_bulk_kernel<<<1, 32, 0, st>>>(ctl, n_src, count, n, width_factor);
  seed_sources_kernel<<<(unsigned)((total_cells + 255) / 256), 256, 0, st>>>(total_cells, cells,
                                                                            ctl);
  return cudaGetLastError();
}

cudaError_t launch_polish_prep(const PolishInstance* d_pi, int count, long long max_padded64,
                               int max_cells, int total_cells, CellArrays cells, Control* ctl,
                               int sms, cudaStream_t st) {
  convert_u_kernel<<<stream_grid(max_padded64, count, sms), 256, 0, st>>>(d_pi, count, ctl);
  {
    long long warps = max_cells;
    long long blocks = (warps * 32 + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    polish_keys_kernel<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, st>>>(d_pi, count,
                                                                              cells);
  }
  setup_polish_kernel<<<1, 32, 0, st>>>(ctl);
  seed_all_kernel<<<(unsigned)((total_cells + 255) / 256), 256, 0, st>>>(total_cells, cells, ctl);
  return cudaGetLastError();
}

cudaError_t launch_residual_extract(const FinalInstance* d_fi, int count, long long max_nodes,
                                    Control* ctl, int sms, cudaStream_t st) {
  residual_extract_kernel<<<stream_grid(max_nodes, count, sms), 256, 0, st>>>(d_fi, count, ctl);
  return cudaGetLastError();
}

}  // namespace eik
