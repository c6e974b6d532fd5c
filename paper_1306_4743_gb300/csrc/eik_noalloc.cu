// eik_noalloc.cu -- eik_solve_device_noalloc: an FP64 solve that allocates
// no memory at all.  It serves callers that cannot call cudaMalloc during a
// solve: programs whose own caching allocator has reserved the device memory
// up front (a cudaMalloc would fail or force that allocator to release
// blocks), latency-critical loops where an allocation can stall behind a
// device-wide synchronisation, and plug-in code whose host framework only
// lets it use memory handed to it.  The paper has no counterpart.
//
// The working memory of the solve lives in one file-scope device array of
// fixed size, kNoallocScratchBytes.  Every device that loads the library
// holds that array until the process exits.  Host code must not use the
// array's name as a device address (in host code it names a host-side
// stand-in); the address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and passed to the
// kernels from then on.  The call waits for its stream before it returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "eik.h"
#include "eik_internal.h"
#include "eik_prep.h"

using namespace eik;

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)EIK_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocCellN = 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct DeviceSlot {
  bool ready;
  unsigned char* scratch;  // device address of g_noalloc_scratch on this device
  int sms;
};

std::mutex g_mutex;  // the host staging below and the per-device slots
DeviceSlot g_slots[kMaxDevices];
EncodeTiledFn g_encode = nullptr;

// Host staging of the small tables of one call (no allocation: static).
alignas(256) unsigned char g_host_small[64 * 1024];
Control g_host_ctl;

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }
size_t take(size_t& cursor, size_t bytes) {
  const size_t at = up(cursor, 256);
  cursor = at + up(bytes, 256);
  return at;
}

// First call on a device: look up the scratch address with the device
// current, plus the SM count and the tensor-map encoder.
int setup_device(int dev, DeviceSlot** out) {
  if (dev < 0 || dev >= kMaxDevices) return EIK_EINVAL;
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                           cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return EIK_ECUDA;
      }
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    s.scratch = static_cast<unsigned char*>(p);
    s.sms = sms;
    s.ready = true;
  }
  *out = &s;
  return EIK_OK;
}

#define CKN(x)                 \
  do {                         \
    if ((x) != cudaSuccess) {  \
      cudaGetLastError();      \
      return EIK_ECUDA;        \
    }                          \
  } while (0)

}  // namespace

extern "C" int eik_solve_device_noalloc(const int64_t dims[3], double h, const float* F_dev,
                                        const uint8_t* src_mask_dev, const double* q_dev,
                                        double tol, double* u_out_dev, void* stream,
                                        eik_stats* stats) {
  if (!dims || !F_dev || !src_mask_dev || !q_dev || !u_out_dev) return EIK_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > (1 << 24)) return EIK_EINVAL;
  if (!(h > 0.0) || isinf(h) || !(tol >= 0.0) || isinf(tol)) return EIK_EINVAL;
  // A grid needs more than 16 bytes of scratch per node (padded FP64 u and
  // FP64 slowness), so anything above kNoallocScratchBytes / 16 nodes cannot
  // fit.  This bound is checked before the node count is formed (the edges
  // alone allow 2^72 nodes); every size below then stays far inside 64 bits.
  if ((long long)dims[0] * dims[1] > (long long)(kNoallocScratchBytes / 16) / dims[2])
    return EIK_EBUDGET;
  const int n = kNoallocCellN, n3 = n * n * n, np = 3 * (n - 1) + 1;
  const int nx = (int)dims[0], ny = (int)dims[1], nz = (int)dims[2];
  const int ncx = (nx + n - 1) / n, ncy = (ny + n - 1) / n, ncz = (nz + n - 1) / n;
  const long long ncells = (long long)ncx * ncy * ncz;
  const int bx = ((n + 2) * 8 + 15) / 16 * 16 / 8;
  long long px = (long long)n * (ncx - 1) + bx;
  if (px < nx + 2) px = nx + 2;
  px = (long long)up((size_t)px, 8);
  const long long py = (long long)n * ncy + 2, pz = (long long)n * ncz + 2;
  const long long nodes = (long long)nx * ny * nz;

  // layout of the scratch: the same arrays an ordinary FP64 solve uses
  size_t cur = 0;
  const size_t off_u = take(cur, (size_t)(px * py * pz) * 8);
  const size_t off_s = take(cur, (size_t)ncells * n3 * 8);
  const size_t off_key = take(cur, (size_t)ncells * 4);
  const size_t off_state = take(cur, (size_t)ncells * 4);
  const size_t off_dir = take(cur, (size_t)ncells * 4);
  const size_t off_inst = take(cur, (size_t)ncells * 4);
  const size_t off_next = take(cur, (size_t)ncells * 4);
  const size_t off_deps = take(cur, (size_t)ncells * 4);
  const size_t off_down = take(cur, (size_t)ncells * 4);
  const size_t off_heads = take(cur, (size_t)kQueueBytes);
  const size_t small_begin = up(cur, 256);
  const size_t off_ctl = take(cur, sizeof(Control));
  const size_t off_nsrc = take(cur, 4);
  const size_t off_instance = take(cur, sizeof(Instance));
  const size_t off_tmap = take(cur, sizeof(CUtensorMap));
  const size_t off_prep = take(cur, sizeof(PrepInstance));
  const size_t off_fin = take(cur, sizeof(FinalInstance));
  const size_t off_seg = take(cur, segment_table_bytes(1));
  const size_t off_tab = take(cur, (size_t)n3 * 2);
  const size_t off_off = take(cur, (size_t)(np + 1) * 4);
  const size_t small_end = up(cur, 256);
  if (small_end > kNoallocScratchBytes) return EIK_EBUDGET;  // grid too large for the scratch
  if (small_end - small_begin > sizeof(g_host_small)) return EIK_EBUDGET;

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  CKN(cudaGetDevice(&dev));
  DeviceSlot* slot = nullptr;
  int rc = setup_device(dev, &slot);
  if (rc) return rc;
  unsigned char* A = slot->scratch;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // host-side small tables
  memset(g_host_small, 0, small_end - small_begin);
  auto hp = [&](size_t off) { return g_host_small + (off - small_begin); };
  Control* hctl = reinterpret_cast<Control*>(hp(off_ctl));
  hctl->min_q_ord = ~0ull;
  Instance* hi = reinterpret_cast<Instance*>(hp(off_instance));
  hi->u = A + off_u;
  hi->s = A + off_s;
  hi->px = px;
  hi->py = py;
  hi->pz = pz;
  hi->nx = nx;
  hi->ny = ny;
  hi->nz = nz;
  hi->ncx = ncx;
  hi->ncy = ncy;
  hi->ncz = ncz;
  hi->cell_base = 0;
  hi->ncells = (int)ncells;
  hi->kappa = tol;
  {
    const cuuint64_t gdim[3] = {(cuuint64_t)px, (cuuint64_t)py, (cuuint64_t)pz};
    const cuuint64_t gstride[2] = {(cuuint64_t)(px * 8), (cuuint64_t)(px * py * 8)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)(n + 2), (cuuint32_t)(n + 2)};
    const cuuint32_t es[3] = {1, 1, 1};
    if (g_encode(reinterpret_cast<CUtensorMap*>(hp(off_tmap)), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                 A + off_u, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return EIK_ECUDA;
  }
  PrepInstance* pi = reinterpret_cast<PrepInstance*>(hp(off_prep));
  pi->F = F_dev;
  pi->mask = src_mask_dev;
  pi->q = q_dev;
  pi->h = h;
  pi->u = A + off_u;
  pi->s = A + off_s;
  pi->s64 = nullptr;
  pi->px = px;
  pi->py = py;
  pi->pz = pz;
  pi->nx = nx;
  pi->ny = ny;
  pi->nz = nz;
  pi->ncx = ncx;
  pi->ncy = ncy;
  pi->ncz = ncz;
  pi->cell_base = 0;
  pi->ncells = (int)ncells;
  pi->n = n;
  FinalInstance* fi = reinterpret_cast<FinalInstance*>(hp(off_fin));
  fi->mask = src_mask_dev;
  fi->q = q_dev;
  fi->u64 = A + off_u;
  fi->s64 = A + off_s;
  fi->out = u_out_dev;
  fi->px64 = px;
  fi->py = py;
  fi->pz = pz;
  fi->nx = nx;
  fi->ny = ny;
  fi->nz = nz;
  fi->ncx = ncx;
  fi->ncy = ncy;
  fi->ncz = ncz;
  fi->n = n;
  {
    unsigned short* tab = reinterpret_cast<unsigned short*>(hp(off_tab));
    int* off = reinterpret_cast<int*>(hp(off_off));
    int t = 0;
    for (int C = 0; C < np; ++C) {
      off[C] = t;
      for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b) {
          const int a = C - b - c;
          if (a >= 0 && a < n) tab[t++] = (unsigned short)(a + n * (b + n * c));
        }
    }
    off[np] = t;
  }

  Segments segs;
  {
    SegSizes sz;
    sz.units[kSegPadB] = py * pz;
    sz.units[kSegPad64] = py * pz;
    sz.units[kSegRows] = (long long)ny * nz;
    sz.units[kSegCellRows] = (long long)n * ncy * n * ncz;
    sz.units[kSegCells] = ncells;
    make_segments(1, &sz, reinterpret_cast<int*>(hp(off_seg)), segs.total);
    segs.dev = reinterpret_cast<const int*>(A + off_seg);
    segs.count = 1;
  }

  // Everything the solve reads before writing starts from these copies and
  // zero fills, so the contents left by the previous call do not matter.
  CKN(cudaMemcpyAsync(A + small_begin, g_host_small, small_end - small_begin,
                      cudaMemcpyHostToDevice, st));
  CKN(cudaMemsetAsync(A + off_heads, 0, (size_t)kQueueBytes, st));

  CellArrays cells;
  cells.key = reinterpret_cast<unsigned*>(A + off_key);
  cells.state = reinterpret_cast<unsigned*>(A + off_state);
  cells.dir = reinterpret_cast<unsigned*>(A + off_dir);
  cells.inst = reinterpret_cast<int*>(A + off_inst);
  cells.next = reinterpret_cast<unsigned*>(A + off_next);
  cells.heads = reinterpret_cast<unsigned long long*>(A + off_heads);
  cells.cnt = reinterpret_cast<int*>(A + off_heads + (size_t)kNumBuckets * kSubStacks * 8);
  cells.run = cells.cnt + kNumBuckets;
  cells.deps = reinterpret_cast<int*>(A + off_deps);
  cells.down = reinterpret_cast<unsigned*>(A + off_down);
  cells.lev_perm = nullptr;  // FP64 only: no level tables
  cells.lev_off = nullptr;
  cells.lev_depth = nullptr;
  Control* dctl = reinterpret_cast<Control*>(A + off_ctl);

  int launches = 0;
  CKN(launch_bulk_init(reinterpret_cast<const PrepInstance*>(A + off_prep), segs, (int)ncells,
                       cells, dctl, reinterpret_cast<int*>(A + off_nsrc), true, n, 0.5, 0.0, st,
                       launches));
  CellKernelParams p;
  memset(&p, 0, sizeof(p));
  p.inst = reinterpret_cast<const Instance*>(A + off_instance);
  p.tmaps = reinterpret_cast<const CUtensorMap*>(A + off_tmap);
  p.cells = cells;
  p.ctl = dctl;
  p.plane_tab = reinterpret_cast<const unsigned short*>(A + off_tab);
  p.plane_off = reinterpret_cast<const int*>(A + off_off);
  p.spin_cap_ns = 5000000000ull;
  p.max_sweeps = 4096;
  p.pass = 0;
  p.max_ctas = 0;
  p.kappa_from_ctl = 0;
  p.relaxed = 1;
  p.gated = 0;
  p.cell_key = 0;
  p.use_levels = 0;
  int grid = 0;
  CKN(launch_cells(true, false, n, p, slot->sms, st, &grid, launches, 0));
  CKN(launch_residual_extract(reinterpret_cast<const FinalInstance*>(A + off_fin), segs, dctl,
                              false, 0.0, st, launches));
  CKN(cudaMemcpyAsync(&g_host_ctl, dctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));

  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->cell_visits = g_host_ctl.counters[0][kCntVisits];
    stats->sweeps = g_host_ctl.counters[0][kCntSweeps];
    stats->node_updates = g_host_ctl.counters[0][kCntUpdates];
    stats->queue_pushes = g_host_ctl.counters[0][kCntPushes];
    stats->nonfinite = g_host_ctl.nonfinite;
    stats->nodes = (uint64_t)nodes;
    stats->cell_n_used = n;
    stats->precision_used = EIK_FP64;
    memcpy(&stats->residual_max, &g_host_ctl.resid_bits, 8);
    stats->kernel_launches = (uint64_t)launches;
    stats->grid_ctas = grid;
  }
  if (g_host_ctl.status) return g_host_ctl.status;
  if (g_host_ctl.nonfinite) return EIK_ENOCONV;
  return EIK_OK;
}
