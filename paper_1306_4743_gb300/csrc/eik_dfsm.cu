// eik_dfsm.cu -- eik_dfsm_solve: whole-grid Fast Sweeping in the plane
// ordering of Detrixhe et al. (Sec. 2-3: each of the 8 sweep directions
// visits the planes i + j + k = C of that direction in order, and the nodes
// of one plane, which do not depend on each other, are updated in parallel).
// This is the synchronous parallel sweeping method the paper compares pHCM
// with (its DFSM), run on the whole grid as one cooperative persistent
// kernel with a device-wide barrier between planes.  In a sweep direction
// every node's upwind neighbours lie on earlier planes and its downwind ones
// on later planes, as in the lexicographic loops of FSM, so each sweep
// produces exactly the values of the FSM sweep of the same direction.
//
// FP64 values, the same local solve as the cell sweeps; the standard order
// of the 8 directions; a sweep counts the nodes lowered by more than kappa
// and the largest such decrease (the statistics of Tables 5-6), and the
// iteration ends after the first sweep that lowers no value by more than
// kappa.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "eik.h"
#include "eik_device.cuh"

namespace {

using eik::dbits;

struct DfsmCtl {
  unsigned count;      // blocks arrived at the current barrier
  unsigned gen;        // barrier generation
  int status;          // EIK_OK or EIK_ETIMEOUT
  int pad;
  unsigned long long changed[2];  // per-sweep count, double-buffered by parity
  unsigned long long maxdrop[2];  // per-sweep largest drop (bits), same
};

__constant__ int kDfsmOrder[8] = {0, 1, 3, 2, 4, 5, 7, 6};

// Device-wide barrier of a cooperative launch: the last block to arrive
// starts the next generation.  Waits are bounded: a block that waits longer
// than the cap sets EIK_ETIMEOUT, and every block then leaves.
__device__ bool grid_barrier(DfsmCtl* c, unsigned long long cap_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = eik::ld_acquire_u32(&c->gen);
    __threadfence();
    if (atomicAdd(&c->count, 1u) == gridDim.x - 1) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      const unsigned long long t0 = eik::global_timer_ns();
      unsigned spins = 0;
      while (eik::ld_acquire_u32(&c->gen) == g) {
        if (++spins > 64u) {
          if (eik::global_timer_ns() - t0 > cap_ns || *(volatile int*)&c->status) {
            atomicCAS(&c->status, 0, (int)EIK_ETIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&c->status == 0;
}

__global__ void dfsm_init(long long nx, long long ny, long long nz, double h, const float* F,
                          const uint8_t* mask, const double* q, double* u, double* s) {
  const long long px = nx + 2, pxy = px * (ny + 2);
  const long long padded = pxy * (nz + 2);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long t = t0; t < padded; t += stride) {
    const long long i = t % px - 1, j = (t / px) % (ny + 2) - 1, k = t / pxy - 1;
    double v = CUDART_INF;
    if (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz) {
      const long long e = i + nx * (j + ny * k);
      if (mask[e]) v = q[e];
    }
    u[t] = v;
  }
  const long long n = nx * ny * nz;
  for (long long e = t0; e < n; e += stride) s[e] = mask[e] ? CUDART_INF : h / (double)F[e];
}

struct DfsmArgs {
  double* u;
  const double* s;
  long long nx, ny, nz;
  double kappa;
  long long max_sweeps;
  DfsmCtl* ctl;
  unsigned long long* stats;  // per sweep: changed count, largest drop (bits)
  unsigned long long cap_ns;
};

__global__ void __launch_bounds__(256) dfsm_kernel(const DfsmArgs a) {
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  const long long px = nx + 2, pxy = px * (ny + 2);
  const long long pencils = ny * nz;
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nplanes = nx + ny + nz - 2;
  const float kf = (float)a.kappa;
  for (long long sw = 0; sw < a.max_sweeps; ++sw) {
    const int d = kDfsmOrder[sw & 7];
    unsigned long long nchg = 0, drop = 0;
    for (long long C = 0; C < nplanes; ++C) {
      // each thread owns pencils (j', k') in the direction's coordinates
      // and takes the node i' = C - j' - k' of each on plane C
      for (long long p = gtid; p < pencils; p += gthreads) {
        const long long jf = p % ny, kf2 = p / ny;
        const long long i_f = C - jf - kf2;
        if (i_f < 0 || i_f >= nx) continue;
        const long long i = (d & 1) ? nx - 1 - i_f : i_f;
        const long long j = (d & 2) ? ny - 1 - jf : jf;
        const long long k = (d & 4) ? nz - 1 - kf2 : kf2;
        const double sv = a.s[i + nx * (j + ny * k)];
        if (!(sv < CUDART_INF)) continue;  // exit node
        const long long t = (i + 1) + px * (j + 1) + pxy * (k + 1);
        const double v = a.u[t];
        const double nv = eik::local_solve(eik::nmin(a.u[t - 1], a.u[t + 1]),
                                           eik::nmin(a.u[t - px], a.u[t + px]),
                                           eik::nmin(a.u[t - pxy], a.u[t + pxy]), sv);
        if (eik::dlt_nn(nv, v)) {
          a.u[t] = nv;
          if (eik::drop_exceeds(nv, v, kf)) {
            ++nchg;
            const double dv = (dbits(v) >= dbits(CUDART_INF)) ? CUDART_INF : v - nv;
            const unsigned long long db = (unsigned long long)dbits(dv);
            drop = db > drop ? db : drop;
          }
        }
      }
      if (!grid_barrier(a.ctl, a.cap_ns)) return;
    }
    // the sweep's statistics, then every block reads the total
    for (int o = 16; o; o >>= 1) {
      nchg += __shfl_xor_sync(0xffffffffu, nchg, o);
      const unsigned long long od = __shfl_xor_sync(0xffffffffu, drop, o);
      drop = od > drop ? od : drop;
    }
    if ((threadIdx.x & 31) == 0) {
      if (nchg) atomicAdd(&a.ctl->changed[sw & 1], nchg);
      if (drop) atomicMax(&a.ctl->maxdrop[sw & 1], drop);
    }
    if (!grid_barrier(a.ctl, a.cap_ns)) return;
    const unsigned long long total = *(volatile unsigned long long*)&a.ctl->changed[sw & 1];
    if (gtid == 0) {
      a.stats[2 * sw] = total;
      a.stats[2 * sw + 1] = *(volatile unsigned long long*)&a.ctl->maxdrop[sw & 1];
      a.ctl->changed[(sw + 1) & 1] = 0;  // the next sweep's slots
      a.ctl->maxdrop[(sw + 1) & 1] = 0;
    }
    if (total == 0) {
      if (gtid == 0) a.stats[2 * a.max_sweeps] = (unsigned long long)(sw + 1);
      return;
    }
    // the resets above must land before the next sweep's atomics
    if (!grid_barrier(a.ctl, a.cap_ns)) return;
  }
  if (gtid == 0) a.stats[2 * a.max_sweeps] = (unsigned long long)a.max_sweeps;
}

// Smallest exit value, number of exits and of invalid speeds.  The
// smallest q is kept as an order-preserving 64-bit key of a signed double.
__device__ __forceinline__ unsigned long long skey(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unskey(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

__global__ void dfsm_check(long long n, const float* F, const uint8_t* mask, const double* q,
                           unsigned long long* out) {  // [qmin key, exits, bad]
  unsigned long long km = ~0ull, ne = 0, nb = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    if (mask[e]) {
      ++ne;
      if (!isfinite(q[e])) ++nb;
      const unsigned long long k = skey(q[e]);
      km = k < km ? k : km;
    }
    if (!(F[e] > 0.0f) || !isfinite(F[e])) ++nb;
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, km, o);
    km = ok < km ? ok : km;
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out, km);
    if (ne) atomicAdd(out + 1, ne);
    if (nb) atomicAdd(out + 2, nb);
  }
}

__global__ void dfsm_shift(long long padded, double* u, const unsigned long long* qk) {
  const double b = unskey(*qk);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < padded;
       t += (long long)gridDim.x * blockDim.x)
    if (u[t] < CUDART_INF) u[t] -= b;
}

__global__ void dfsm_copyout(long long nx, long long ny, long long nz, const double* u,
                             const uint8_t* mask, const double* q,
                             const unsigned long long* qk, double* out) {
  const double b = unskey(*qk);
  const long long px = nx + 2, pxy = px * (ny + 2), n = nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % nx, j = (e / nx) % ny, k = e / (nx * ny);
    out[e] = mask[e] ? q[e] : u[(i + 1) + px * (j + 1) + pxy * (k + 1)] + b;
  }
}

}  // namespace

extern "C" int eik_dfsm_solve_device(const int64_t dims[3], double h, const float* F_dev,
                                     const uint8_t* src_mask_dev, const double* q_dev,
                                     double tol, int64_t max_sweeps, double* u_out_dev,
                                     void* stream, int64_t* sweeps,
                                     int64_t* changed_per_sweep, double* max_drop_per_sweep,
                                     eik_stats* stats) {
  if (!dims || !F_dev || !src_mask_dev || !q_dev || !u_out_dev || !(h > 0.0) ||
      !(tol >= 0.0) || max_sweeps < 1 || max_sweeps > (1 << 20))
    return EIK_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > (1 << 24)) return EIK_EINVAL;
  const long long nx = dims[0], ny = dims[1], nz = dims[2];
  const long long n = nx * ny * nz;
  const long long padded = (nx + 2) * (ny + 2) * (nz + 2);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EIK_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EIK_ECUDA;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return EIK_ECUDA;
  // one allocation: u (padded) | s | control | per-sweep statistics | check words
  const size_t off_s = (size_t)padded * 8;
  const size_t off_ctl = off_s + (size_t)n * 8;
  const size_t off_stats = off_ctl + 256;
  const size_t off_chk = off_stats + ((size_t)(2 * max_sweeps + 1) * 8 + 255) / 256 * 256;
  const size_t bytes = off_chk + 64;
  unsigned char* A = nullptr;
  if (cudaMalloc(&A, bytes) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ENOMEM;
  }
  int rc = EIK_OK;
  double* u = reinterpret_cast<double*>(A);
  double* s = reinterpret_cast<double*>(A + off_s);
  DfsmCtl* ctl = reinterpret_cast<DfsmCtl*>(A + off_ctl);
  unsigned long long* dstats = reinterpret_cast<unsigned long long*>(A + off_stats);
  unsigned long long* chk = reinterpret_cast<unsigned long long*>(A + off_chk);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  unsigned long long hchk[3] = {0, 0, 0};
  std::vector<unsigned long long> hst;
  int grid = 0;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = EIK_ECUDA;
      break;
    }
    const unsigned long long init_chk[3] = {~0ull, 0, 0};
    if (cudaMemsetAsync(A + off_ctl, 0, off_chk - off_ctl, st) != cudaSuccess ||
        cudaMemcpyAsync(chk, init_chk, sizeof(init_chk), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
      rc = EIK_ECUDA;
      break;
    }
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, (long long)sms * 8);
    dfsm_check<<<std::max(blocks, 1u), 256, 0, st>>>(n, F_dev, src_mask_dev, q_dev, chk);
    if (cudaMemcpyAsync(hchk, chk, sizeof(hchk), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = EIK_ECUDA;
      break;
    }
    if (hchk[1] == 0 || hchk[2] != 0) {
      rc = EIK_EINVAL;
      break;
    }
    cudaEventRecord(e0, st);
    const unsigned pblocks =
        (unsigned)std::min<long long>((padded + 255) / 256, (long long)sms * 8);
    dfsm_init<<<pblocks, 256, 0, st>>>(nx, ny, nz, h, F_dev, src_mask_dev, q_dev, u, s);
    dfsm_shift<<<pblocks, 256, 0, st>>>(padded, u, chk);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfsm_kernel, 256, 0) !=
            cudaSuccess ||
        per_sm < 1) {
      rc = EIK_ECUDA;
      break;
    }
    grid = sms * std::min(per_sm, 2);
    DfsmArgs args;
    args.u = u;
    args.s = s;
    args.nx = nx;
    args.ny = ny;
    args.nz = nz;
    args.kappa = tol;
    args.max_sweeps = max_sweeps;
    args.ctl = ctl;
    args.stats = dstats;
    args.cap_ns = 5000000000ull;
    void* kargs[] = {&args};
    if (cudaLaunchCooperativeKernel((const void*)dfsm_kernel, dim3(grid), dim3(256), kargs, 0,
                                    st) != cudaSuccess) {
      rc = EIK_ECUDA;
      break;
    }
    dfsm_copyout<<<std::max(blocks, 1u), 256, 0, st>>>(nx, ny, nz, u, src_mask_dev, q_dev, chk,
                                                       u_out_dev);
    cudaEventRecord(e1, st);
    hst.resize((size_t)(2 * max_sweeps + 1));
    int status = 0;
    if (cudaMemcpyAsync(hst.data(), dstats, hst.size() * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = EIK_ECUDA;
      break;
    }
    if (status) {
      rc = status;
      break;
    }
    const long long nsw = (long long)hst[2 * max_sweeps];
    if (sweeps) *sweeps = nsw;
    for (long long w = 0; w < nsw; ++w) {
      if (changed_per_sweep) changed_per_sweep[w] = (int64_t)hst[2 * w];
      if (max_drop_per_sweep) {
        double dv;
        memcpy(&dv, &hst[2 * w + 1], 8);
        max_drop_per_sweep[w] = dv;
      }
    }
    if (nsw >= max_sweeps && hst[2 * (max_sweeps - 1)] != 0) rc = EIK_ENOCONV;
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      stats->seconds = ms * 1e-3;
      stats->sweeps = (uint64_t)nsw;
      stats->node_updates = (uint64_t)nsw * (uint64_t)(n - (long long)hchk[1]);
      stats->nodes = (uint64_t)n;
      stats->precision_used = EIK_FP64;
      stats->kernel_launches = 4;
      stats->grid_ctas = grid;
    }
  } while (false);
  if (rc == EIK_ECUDA) cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(A);
  return rc;
}
