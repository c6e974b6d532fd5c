// eik_api.cu -- host runtime and C ABI of libeik.so (declared in
// include/eik.h): contexts, device memory, tensor maps, the launch sequence
// of one (batched) solve, statistics, and the serving queue.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "eik.h"
#include "eik_internal.h"
#include "eik_prep.h"
#include "eik_serve.h"

using namespace eik;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int box_width(int n, int es) { return (((n + 2) * es + 15) / 16) * 16 / es; }

long long padded_x(int nx, int n, int ncx, int es) {
  long long need = (long long)n * (ncx - 1) + box_width(n, es);
  if (need < nx + 2) need = nx + 2;
  return (long long)align_up((size_t)need, 8);
}

}  // namespace

// ---------------------------------------------------------------------------
// Context.
struct eik_ctx {
  eik_opts opts;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  EncodeTiledFn encode = nullptr;
  // execution slot of the synchronous calls
  Exec main;
  // execution slot of the captured device-batch graph (its staging is only
  // written while capturing, so a replay uploads the captured tables)
  Exec gexec;
  // plane tables, per cell size (index 0: n=4, 1: n=8, 2: n=16)
  unsigned short* d_tab[3] = {nullptr, nullptr, nullptr};
  int* d_off[3] = {nullptr, nullptr, nullptr};
  // serving
  ServeState* serve = nullptr;
  // autotune results: log2(nodes) bucket -> worker shape
  struct Tuned {
    int n, ctas, wpc;
  };
  std::map<int, Tuned> tuned;
  unsigned long long tune_generation = 0;  // bumped by every eik_autotune
};

namespace {

int size_index(int n) { return n == 4 ? 0 : n == 8 ? 1 : n == 16 ? 2 : -1; }

cudaError_t ensure_plane_table(eik_ctx* ctx, int n) {
  const int si = size_index(n);
  if (ctx->d_tab[si]) return cudaSuccess;
  const int n3 = n * n * n, np = 3 * (n - 1) + 1;
  std::vector<unsigned short> tab;
  std::vector<int> off(np + 1, 0);
  tab.reserve(n3);
  for (int C = 0; C < np; ++C) {
    off[C] = (int)tab.size();
    for (int c = 0; c < n; ++c)
      for (int b = 0; b < n; ++b) {
        const int a = C - b - c;
        if (a >= 0 && a < n) tab.push_back((unsigned short)(a + n * (b + n * c)));
      }
  }
  off[np] = (int)tab.size();
  cudaError_t e = cudaMalloc(&ctx->d_tab[si], n3 * sizeof(unsigned short));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&ctx->d_off[si], (np + 1) * sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(ctx->d_tab[si], tab.data(), n3 * sizeof(unsigned short), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(ctx->d_off[si], off.data(), (np + 1) * sizeof(int), cudaMemcpyHostToDevice);
}

// Layout of one instance inside a launch.
struct InstPlan {
  int nx, ny, nz;
  double h;
  int ncx, ncy, ncz, ncells, cell_base;
  long long px_b, px64, py, pz;
  size_t off_ub, off_sb, off_u64, off_s64, off_F, off_mask, off_q, off_out;
  long long nodes;
};

// Sub-allocation of the arena for one launch.
struct LaunchPlan {
  int count = 0;
  int n = 8;
  bool polish = false;  // FP32 bulk + FP64 polish
  std::vector<InstPlan> inst;
  int total_cells = 0, max_cells = 0;
  long long max_padded_b = 0, max_padded64 = 0, max_cellnodes = 0, max_nodes = 0;
  long long max_rows = 0;  // largest ny * nz
  size_t off_lev_perm = 0, off_lev_off = 0, off_lev_depth = 0;  // polish only
  size_t off_key, off_state, off_dir, off_inst, off_next, off_deps, off_down, off_heads, off_ctl,
      off_nsrc;
  size_t off_inst_b, off_inst64, off_tmap_b, off_tmap64, off_prep, off_pol, off_fin, off_seg;
  std::vector<int> seg;  // block schedule of the streaming kernels (host copy)
  int seg_total[kNumSegKinds] = {0, 0, 0, 0, 0};
  size_t total = 0;
  size_t small_begin = 0, small_end = 0;  // tables copied from the host in one go
};

size_t take(size_t& cursor, size_t bytes) {
  const size_t at = align_up(cursor, 256);
  cursor = at + align_up(bytes, 256);
  return at;
}

int size_bucket(long long nodes) {
  int lg = 0;
  while ((1ll << (lg + 1)) <= nodes) ++lg;
  return lg;
}

int choose_cell_n(eik_ctx* ctx, long long nodes) {
  if (ctx->opts.cell_n) return ctx->opts.cell_n;
  auto it = ctx->tuned.find(size_bucket(nodes));
  if (it != ctx->tuned.end()) return it->second.n;
  // built-in size table: 16^3 cells from ~128^3 nodes up (fewer, longer
  // visits keep the queue latency small against the sweeping), else 8^3
  return nodes >= (1ll << 21) ? 16 : 8;
}

void make_plan(LaunchPlan& L, int count, const int64_t* dims, const double* h, int n, bool polish,
               bool host_io) {
  L.count = count;
  L.n = n;
  L.polish = polish;
  L.inst.resize(count);
  const int es_b = polish ? 4 : 8;
  size_t cur = 0;
  int cells = 0;
  for (int t = 0; t < count; ++t) {
    InstPlan& I = L.inst[t];
    I.nx = (int)dims[3 * t];
    I.ny = (int)dims[3 * t + 1];
    I.nz = (int)dims[3 * t + 2];
    I.h = h[t];
    I.ncx = (I.nx + n - 1) / n;
    I.ncy = (I.ny + n - 1) / n;
    I.ncz = (I.nz + n - 1) / n;
    I.ncells = I.ncx * I.ncy * I.ncz;
    I.cell_base = cells;
    cells += I.ncells;
    I.py = (long long)n * I.ncy + 2;
    I.pz = (long long)n * I.ncz + 2;
    I.px_b = padded_x(I.nx, n, I.ncx, es_b);
    I.px64 = padded_x(I.nx, n, I.ncx, 8);
    I.nodes = (long long)I.nx * I.ny * I.nz;
    const long long cn = (long long)I.ncells * n * n * n;
    I.off_ub = take(cur, (size_t)(I.px_b * I.py * I.pz) * es_b);
    I.off_sb = take(cur, (size_t)cn * es_b);
    if (polish) {
      I.off_u64 = take(cur, (size_t)(I.px64 * I.py * I.pz) * 8);
      I.off_s64 = take(cur, (size_t)cn * 8);
    } else {
      I.off_u64 = I.off_ub;
      I.off_s64 = I.off_sb;
    }
    if (host_io) {
      I.off_F = take(cur, (size_t)I.nodes * 4);
      I.off_mask = take(cur, (size_t)I.nodes);
      I.off_q = take(cur, (size_t)I.nodes * 8);
      I.off_out = take(cur, (size_t)I.nodes * 8);
    } else {
      I.off_F = I.off_mask = I.off_q = I.off_out = 0;
    }
    L.max_cells = std::max(L.max_cells, I.ncells);
    L.max_padded_b = std::max(L.max_padded_b, I.px_b * I.py * I.pz);
    L.max_padded64 = std::max(L.max_padded64, I.px64 * I.py * I.pz);
    L.max_cellnodes = std::max(L.max_cellnodes, cn);
    L.max_nodes = std::max(L.max_nodes, I.nodes);
    L.max_rows = std::max(L.max_rows, (long long)I.ny * I.nz);
  }
  L.total_cells = cells;
  L.off_key = take(cur, (size_t)cells * 4);
  L.off_state = take(cur, (size_t)cells * 4);
  L.off_dir = take(cur, (size_t)cells * 4);
  L.off_inst = take(cur, (size_t)cells * 4);
  L.off_next = take(cur, (size_t)cells * 4);
  L.off_deps = take(cur, (size_t)cells * 4);
  L.off_down = take(cur, (size_t)cells * 4);
  if (polish) {
    L.off_lev_perm = take(cur, (size_t)cells * n * n * n * 2);
    L.off_lev_off = take(cur, (size_t)cells * (kMaxLevels + 1) * 2);
    L.off_lev_depth = take(cur, (size_t)cells * 4);
  }
  L.off_heads = take(cur, (size_t)kQueueBytes);  // heads, then counts and run counts
  // small tables, filled on the host and copied in one transfer
  L.small_begin = align_up(cur, 256);
  L.off_ctl = take(cur, sizeof(Control));
  L.off_nsrc = take(cur, (size_t)count * 4);
  L.off_inst_b = take(cur, (size_t)count * sizeof(Instance));
  L.off_inst64 = take(cur, (size_t)count * sizeof(Instance));
  L.off_tmap_b = take(cur, (size_t)count * sizeof(CUtensorMap));
  L.off_tmap64 = take(cur, (size_t)count * sizeof(CUtensorMap));
  L.off_prep = take(cur, (size_t)count * sizeof(PrepInstance));
  L.off_pol = take(cur, (size_t)count * sizeof(PolishInstance));
  L.off_fin = take(cur, (size_t)count * sizeof(FinalInstance));
  L.off_seg = take(cur, segment_table_bytes(count));
  L.small_end = align_up(cur, 256);
  {
    std::vector<SegSizes> sz(count);
    for (int t = 0; t < count; ++t) {
      const InstPlan& I = L.inst[t];
      sz[t].units[kSegPadB] = I.py * I.pz;
      sz[t].units[kSegPad64] = I.py * I.pz;
      sz[t].units[kSegRows] = (long long)I.ny * I.nz;
      sz[t].units[kSegCellRows] = (long long)n * I.ncy * n * I.ncz;
      sz[t].units[kSegCells] = I.ncells;
    }
    L.seg.assign(segment_table_bytes(count) / sizeof(int), 0);
    make_segments(count, sz.data(), L.seg.data(), L.seg_total);
  }
  L.total = L.small_end;
}

int ensure_arena(Exec& ex, size_t bytes, size_t limit) {
  if (limit && bytes > limit) return EIK_EBUDGET;
  if (bytes <= ex.arena_size) return EIK_OK;
  if (ex.arena) {
    cudaStreamSynchronize(ex.stream);
    cudaFree(ex.arena);
    ex.arena = nullptr;
    ex.arena_size = 0;
    if (ex.graph) {  // it points into the old arena
      cudaGraphExecDestroy(ex.graph);
      ex.graph = nullptr;
      ex.graph_key.clear();
    }
  }
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  if (limit && want > limit) want = bytes;
  if (cudaMalloc(&ex.arena, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&ex.arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      return EIK_ENOMEM;
    }
    want = bytes;
  }
  ex.arena_size = want;
  return EIK_OK;
}

int ensure_pinned(char** buf, size_t* have, size_t bytes) {
  if (bytes <= *have) return EIK_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *have = 0;
  if (cudaMallocHost(buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ENOMEM;
  }
  *have = bytes;
  return EIK_OK;
}

int encode_map(eik_ctx* ctx, CUtensorMap* map, void* base, int es, long long px, long long py,
               long long pz, int n) {
  const cuuint64_t gdim[3] = {(cuuint64_t)px, (cuuint64_t)py, (cuuint64_t)pz};
  const cuuint64_t gstride[2] = {(cuuint64_t)(px * es), (cuuint64_t)(px * py * es)};
  const cuuint32_t box[3] = {(cuuint32_t)box_width(n, es), (cuuint32_t)(n + 2),
                             (cuuint32_t)(n + 2)};
  const cuuint32_t estride[3] = {1, 1, 1};
  CUresult r = ctx->encode(map, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           3, base, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? EIK_OK : EIK_ECUDA;
}

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) {               \
      cudaGetLastError();                  \
      return EIK_ECUDA;                    \
    }                                      \
  } while (0)

// Each edge in [1, 2^24] and at most 2^34 nodes in all; the node count is
// bounded before it is formed (d0 d1 <= 2^48 fits, d0 d1 d2 might not).
bool valid_dims(const int64_t* d) {
  for (int a = 0; a < 3; ++a)
    if (d[a] < 1 || d[a] > (1 << 24)) return false;
  return (long long)d[0] * d[1] <= (1ll << 34) / d[2];
}

// The device address of a page-locked host buffer (cudaHostAlloc or
// cudaHostRegister), else nullptr.  Kernels read such a buffer in place
// over the CPU-GPU link, so the solve need not copy what it only samples
// (q, read at exit nodes only) or reads once (F); the result can be written
// straight into it.  Pageable memory is always copied.
const void* pinned_alias(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

}  // namespace

// Launch sequence of one batched solve.  IO arrays are host pointers when
// host_io, else device pointers.
int eik_launch_batch(eik_ctx* ctx, Exec& ex, int count, const int64_t* dims, const double* h,
                     const float* const* F, const uint8_t* const* mask, const double* const* q,
                     double tol, double* const* u_out, bool host_io, cudaStream_t st,
                     bool async_out, Launch& Lr, size_t arena_limit, int n_override) {
  if (!ctx || count < 1 || !dims || !h || !F || !mask || !q || !u_out) return EIK_EINVAL;
  if (!(tol >= 0.0) || isinf(tol)) return EIK_EINVAL;
  long long nodes_total = 0, nodes_max = 0;
  for (int t = 0; t < count; ++t) {
    if (!valid_dims(dims + 3 * t)) return EIK_EINVAL;
    if (!(h[t] > 0.0) || isinf(h[t])) return EIK_EINVAL;
    if (!F[t] || !mask[t] || !q[t] || !u_out[t]) return EIK_EINVAL;
    const long long nd = (long long)dims[3 * t] * dims[3 * t + 1] * dims[3 * t + 2];
    nodes_total += nd;
    nodes_max = std::max(nodes_max, nd);
  }
  const bool polish = ctx->opts.precision == EIK_FP32_POLISH;
  const int n = n_override ? n_override : choose_cell_n(ctx, nodes_max);
  if (size_index(n) < 0) return EIK_EINVAL;
  CK(cudaSetDevice(ctx->device));
  CK(ensure_plane_table(ctx, n));

  LaunchPlan L;
  make_plan(L, count, dims, h, n, polish, host_io);
  if (L.total_cells > (1 << 30)) return EIK_EINVAL;
  int rc = ensure_arena(ex, L.total, arena_limit);
  if (rc) return rc;
  rc = ensure_pinned(&ex.h_small, &ex.h_small_size, L.small_end - L.small_begin);
  if (rc) return rc;
  rc = ensure_pinned(&ex.h_ctl, &ex.h_ctl_size, sizeof(Control));
  if (rc) return rc;
  Lr = Launch();
  Lr.count = count;
  Lr.n = n;
  Lr.polish = polish;
  Lr.host_io = host_io;
  Lr.async_out = async_out && host_io;
  Lr.nodes_total = nodes_total;
  Lr.outs.assign(u_out, u_out + count);
  // page-locked host inputs are read in place, and a page-locked output is
  // written in place by the final kernel (eik_cancel of such a request on
  // the device waits for its batch)
  std::vector<const float*> Fd(count, nullptr);
  std::vector<const double*> Qd(count, nullptr);
  std::vector<double*> Od(count, nullptr);
  if (host_io) {
    for (int t = 0; t < count; ++t) {
      Fd[t] = static_cast<const float*>(pinned_alias(F[t]));
      Qd[t] = static_cast<const double*>(pinned_alias(q[t]));
      Od[t] = static_cast<double*>(const_cast<void*>(pinned_alias(u_out[t])));
    }
  }
  Lr.direct.assign(count, 0);
  for (int t = 0; t < count; ++t) Lr.direct[t] = Od[t] ? 1 : 0;
  if (Lr.async_out) {
    size_t ob = 0;
    for (int t = 0; t < count; ++t) {
      Lr.out_off.push_back(ob);
      Lr.out_nodes.push_back(L.inst[t].nodes);
      if (!Od[t]) ob += align_up((size_t)L.inst[t].nodes * 8, 256);
    }
    if (ob) {
      rc = ensure_pinned(&ex.h_out, &ex.h_out_size, ob);
      if (rc) return rc;
    }
  }
  char* A = ex.arena;

  // host-side small tables
  char* hs = ex.h_small;
  memset(hs, 0, L.small_end - L.small_begin);
  auto hptr = [&](size_t off) { return hs + (off - L.small_begin); };
  Control* hctl = reinterpret_cast<Control*>(hptr(L.off_ctl));
  hctl->min_q_ord = ~0ull;
  Instance* hib = reinterpret_cast<Instance*>(hptr(L.off_inst_b));
  Instance* hi64 = reinterpret_cast<Instance*>(hptr(L.off_inst64));
  CUtensorMap* htb = reinterpret_cast<CUtensorMap*>(hptr(L.off_tmap_b));
  CUtensorMap* ht64 = reinterpret_cast<CUtensorMap*>(hptr(L.off_tmap64));
  PrepInstance* hp = reinterpret_cast<PrepInstance*>(hptr(L.off_prep));
  PolishInstance* hpol = reinterpret_cast<PolishInstance*>(hptr(L.off_pol));
  FinalInstance* hfin = reinterpret_cast<FinalInstance*>(hptr(L.off_fin));
  const int es_b = polish ? 4 : 8;
  for (int t = 0; t < count; ++t) {
    const InstPlan& I = L.inst[t];
    Instance& b = hib[t];
    b.u = A + I.off_ub;
    b.s = A + I.off_sb;
    b.px = I.px_b;
    b.py = I.py;
    b.pz = I.pz;
    b.nx = I.nx;
    b.ny = I.ny;
    b.nz = I.nz;
    b.ncx = I.ncx;
    b.ncy = I.ncy;
    b.ncz = I.ncz;
    b.cell_base = I.cell_base;
    b.ncells = I.ncells;
    b.kappa = polish ? 0.0 : tol;
    Instance& d = hi64[t];
    d = b;
    d.u = A + I.off_u64;
    d.s = A + I.off_s64;
    d.px = I.px64;
    d.kappa = tol;
    rc = encode_map(ctx, &htb[t], b.u, es_b, I.px_b, I.py, I.pz, n);
    if (rc) return rc;
    if (polish) {
      rc = encode_map(ctx, &ht64[t], d.u, 8, I.px64, I.py, I.pz, n);
      if (rc) return rc;
    }
    PrepInstance& P = hp[t];
    P.F = host_io ? (Fd[t] ? Fd[t] : reinterpret_cast<const float*>(A + I.off_F)) : F[t];
    P.mask = host_io ? reinterpret_cast<const uint8_t*>(A + I.off_mask) : mask[t];
    P.q = host_io ? (Qd[t] ? Qd[t] : reinterpret_cast<const double*>(A + I.off_q)) : q[t];
    P.h = I.h;
    P.u = b.u;
    P.s = A + I.off_sb;
    P.s64 = polish ? (void*)(A + I.off_s64) : nullptr;
    P.px = I.px_b;
    P.py = I.py;
    P.pz = I.pz;
    P.nx = I.nx;
    P.ny = I.ny;
    P.nz = I.nz;
    P.ncx = I.ncx;
    P.ncy = I.ncy;
    P.ncz = I.ncz;
    P.cell_base = I.cell_base;
    P.ncells = I.ncells;
    P.n = n;
    PolishInstance& Q = hpol[t];
    Q.mask = P.mask;
    Q.q = P.q;
    Q.u32 = b.u;
    Q.u64 = A + I.off_u64;
    Q.s64 = A + I.off_s64;
    Q.px32 = I.px_b;
    Q.px64 = I.px64;
    Q.py = I.py;
    Q.pz = I.pz;
    Q.nx = I.nx;
    Q.ny = I.ny;
    Q.nz = I.nz;
    Q.ncx = I.ncx;
    Q.ncy = I.ncy;
    Q.ncz = I.ncz;
    Q.cell_base = I.cell_base;
    Q.ncells = I.ncells;
    Q.n = n;
    FinalInstance& Fi = hfin[t];
    Fi.mask = P.mask;
    Fi.q = P.q;
    Fi.u64 = A + I.off_u64;
    Fi.s64 = A + I.off_s64;
    Fi.out = host_io ? (Od[t] ? Od[t] : reinterpret_cast<double*>(A + I.off_out)) : u_out[t];
    Fi.px64 = I.px64;
    Fi.py = I.py;
    Fi.pz = I.pz;
    Fi.nx = I.nx;
    Fi.ny = I.ny;
    Fi.nz = I.nz;
    Fi.ncx = I.ncx;
    Fi.ncy = I.ncy;
    Fi.ncz = I.ncz;
    Fi.n = n;
  }

  memcpy(hptr(L.off_seg), L.seg.data(), L.seg.size() * sizeof(int));
  Segments segs;
  segs.dev = reinterpret_cast<const int*>(A + L.off_seg);
  segs.count = count;
  for (int k = 0; k < kNumSegKinds; ++k) segs.total[k] = L.seg_total[k];

  // inputs and tables to the device
  if (host_io) {
    for (int t = 0; t < count; ++t) {
      const InstPlan& I = L.inst[t];
      if (!Fd[t])
        CK(cudaMemcpyAsync(A + I.off_F, F[t], (size_t)I.nodes * 4, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(A + I.off_mask, mask[t], (size_t)I.nodes, cudaMemcpyHostToDevice, st));
      if (!Qd[t])
        CK(cudaMemcpyAsync(A + I.off_q, q[t], (size_t)I.nodes * 8, cudaMemcpyHostToDevice, st));
    }
  }
  CK(cudaMemcpyAsync(A + L.small_begin, hs, L.small_end - L.small_begin, cudaMemcpyHostToDevice,
                     st));
  CK(cudaMemsetAsync(A + L.off_heads, 0, (size_t)kQueueBytes, st));

  CellArrays cells;
  cells.key = reinterpret_cast<unsigned*>(A + L.off_key);
  cells.state = reinterpret_cast<unsigned*>(A + L.off_state);
  cells.dir = reinterpret_cast<unsigned*>(A + L.off_dir);
  cells.inst = reinterpret_cast<int*>(A + L.off_inst);
  cells.next = reinterpret_cast<unsigned*>(A + L.off_next);
  cells.heads = reinterpret_cast<unsigned long long*>(A + L.off_heads);
  cells.cnt = reinterpret_cast<int*>(A + L.off_heads + (size_t)kNumBuckets * kSubStacks * 8);
  cells.run = cells.cnt + kNumBuckets;
  cells.deps = reinterpret_cast<int*>(A + L.off_deps);
  cells.down = reinterpret_cast<unsigned*>(A + L.off_down);
  cells.lev_perm = polish ? reinterpret_cast<unsigned short*>(A + L.off_lev_perm) : nullptr;
  cells.lev_off = polish ? reinterpret_cast<unsigned short*>(A + L.off_lev_off) : nullptr;
  cells.lev_depth = polish ? reinterpret_cast<int*>(A + L.off_lev_depth) : nullptr;
  Control* dctl = reinterpret_cast<Control*>(A + L.off_ctl);

  CK(cudaEventRecord(ex.ev[0], st));
  int nl = 0;  // kernels enqueued
  double wf = ctx->opts.bucket_width > 0 ? ctx->opts.bucket_width : 0.25;
  CK(launch_bulk_init(reinterpret_cast<const PrepInstance*>(A + L.off_prep), segs, L.total_cells,
                      cells, dctl, reinterpret_cast<int*>(A + L.off_nsrc), !polish, n, wf,
                      ctx->opts.bulk_kappa_rel, st, nl));

  CellKernelParams p;
  p.inst = reinterpret_cast<const Instance*>(A + L.off_inst_b);
  p.tmaps = reinterpret_cast<const CUtensorMap*>(A + L.off_tmap_b);
  p.cells = cells;
  p.ctl = dctl;
  p.plane_tab = ctx->d_tab[size_index(n)];
  p.plane_off = ctx->d_off[size_index(n)];
  p.spin_cap_ns = ctx->opts.spin_cap_us * 1000ull;
  p.max_sweeps = ctx->opts.max_sweeps_per_visit;
  p.pass = 0;
  p.max_ctas = ctx->opts.max_ctas;
  int wpc = ctx->opts.warps_per_cell;
  if (!p.max_ctas && !ctx->opts.cell_n && !wpc) {
    auto it = ctx->tuned.find(size_bucket(nodes_max));
    if (it != ctx->tuned.end()) {
      p.max_ctas = it->second.ctas;
      wpc = it->second.wpc;
    }
  }
  if (n != 16) wpc = 0;
  // default shapes per pass: the FP32 bulk sweeps 16^3 cells with 8 warps
  // (one thread per (j, k) pencil, planes computed instead of read from the
  // table: measured ~5% faster than 6 warps), FP64 sweeps with 6 warps
  const int wpc_bulk = wpc ? wpc : (n == 16 && polish ? 8 : 0);
  p.kappa_from_ctl = polish ? 1 : 0;
  p.relaxed = ctx->opts.queue_order;
  p.gated = 0;
  p.cell_key = ctx->opts.cell_key;
  p.use_levels = 0;
  CK(cudaEventRecord(ex.ev[1], st));
  int grid_ctas = 0;
  CK(launch_cells(!polish, false, n, p, ctx->sms, st, &grid_ctas, nl, wpc_bulk));
  CK(cudaEventRecord(ex.ev[2], st));
  if (polish) {
    const float lift = ctx->opts.polish_lift != 0.0 ? (float)ctx->opts.polish_lift : 0x1p-11f;
    CK(launch_polish_prep(reinterpret_cast<const PolishInstance*>(A + L.off_pol), segs,
                          L.total_cells, cells, dctl, lift, st, nl));
    p.inst = reinterpret_cast<const Instance*>(A + L.off_inst64);
    p.tmaps = reinterpret_cast<const CUtensorMap*>(A + L.off_tmap64);
    p.pass = 1;
    p.kappa_from_ctl = 0;
    p.gated = 1;
    p.use_levels = 1;
    CK(cudaEventRecord(ex.ev[3], st));
    // monotone FP64 sweeps down from the lifted FP32 result
    CK(launch_cells(true, false, n, p, ctx->sms, st, nullptr, nl, wpc));
    CK(cudaEventRecord(ex.ev[4], st));
    // fallback, gated on the device: if some u ended below the fixed point
    // (lift too small), polish again with replace-mode sweeps
    CK(launch_fallback_prep(reinterpret_cast<const PolishInstance*>(A + L.off_pol),
                            reinterpret_cast<const FinalInstance*>(A + L.off_fin), segs,
                            L.total_cells, cells, dctl, tol, st, nl));
    p.pass = 2;
    p.gated = 0;
    p.use_levels = 0;
    CK(launch_cells(true, true, n, p, ctx->sms, st, nullptr, nl, 0));
  }
  CK(launch_residual_extract(reinterpret_cast<const FinalInstance*>(A + L.off_fin), segs, dctl,
                             polish, tol, st, nl));
  CK(cudaEventRecord(ex.ev[5], st));
  Control* hres = reinterpret_cast<Control*>(ex.h_ctl);
  CK(cudaMemcpyAsync(hres, dctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  if (host_io) {
    for (int t = 0; t < count; ++t) {
      if (Od[t]) continue;  // written in place by the final kernel
      const InstPlan& I = L.inst[t];
      void* dst = Lr.async_out ? (void*)(ex.h_out + Lr.out_off[t]) : (void*)u_out[t];
      CK(cudaMemcpyAsync(dst, A + I.off_out, (size_t)I.nodes * 8, cudaMemcpyDeviceToHost, st));
    }
  }
  Lr.hres = hres;
  Lr.grid = grid_ctas;
  Lr.launches = nl;
  Lr.wpc = n == 16 ? (wpc_bulk ? wpc_bulk : 6) : 1;
  return EIK_OK;
}

int eik_finish_batch(eik_ctx* ctx, Exec& ex, Launch& Lr, eik_stats* stats) {
  (void)ctx;
  const Control* hres = Lr.hres;
  const bool polish = Lr.polish;
  const int n = Lr.n;
  const int grid_ctas = Lr.grid;
  const long long nodes_total = Lr.nodes_total;
  if (Lr.async_out) {
    for (int t = 0; t < Lr.count; ++t)
      if (!Lr.direct[t])
        memcpy(Lr.outs[t], ex.h_out + Lr.out_off[t], (size_t)Lr.out_nodes[t] * 8);
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ex.ev[0], ex.ev[5]);
    stats->seconds = ms * 1e-3;
    cudaEventElapsedTime(&ms, ex.ev[1], ex.ev[2]);
    stats->seconds_bulk = ms * 1e-3;
    cudaEventElapsedTime(&ms, ex.ev[0], ex.ev[1]);
    stats->seconds_stage[0] = ms * 1e-3;
    if (polish) {
      cudaEventElapsedTime(&ms, ex.ev[3], ex.ev[4]);
      stats->seconds_polish = ms * 1e-3;
      cudaEventElapsedTime(&ms, ex.ev[2], ex.ev[3]);
      stats->seconds_stage[1] = ms * 1e-3;
      cudaEventElapsedTime(&ms, ex.ev[4], ex.ev[5]);
      stats->seconds_stage[2] = ms * 1e-3;
    } else {
      cudaEventElapsedTime(&ms, ex.ev[2], ex.ev[5]);
      stats->seconds_stage[2] = ms * 1e-3;
    }
    stats->cell_visits = hres->counters[0][kCntVisits];
    stats->sweeps = hres->counters[0][kCntSweeps];
    stats->node_updates = hres->counters[0][kCntUpdates];
    stats->polish_visits = hres->counters[1][kCntVisits] + hres->counters[2][kCntVisits];
    stats->polish_sweeps = hres->counters[1][kCntSweeps] + hres->counters[2][kCntSweeps];
    stats->polish_node_updates = hres->counters[1][kCntUpdates] + hres->counters[2][kCntUpdates];
    stats->queue_pushes = hres->counters[0][kCntPushes] + hres->counters[1][kCntPushes] +
                          hres->counters[2][kCntPushes];
    stats->nonfinite = hres->nonfinite;
    stats->nodes = (uint64_t)nodes_total;
    stats->cell_n_used = n;
    stats->kernel_launches = (uint64_t)Lr.launches;
    stats->warps_per_cell_used = Lr.wpc;
    stats->grid_ctas = grid_ctas;
    stats->fallback_used = hres->counters[2][kCntPushes] > 0;
    stats->fallback_visits = hres->counters[2][kCntVisits];
    stats->busy_seconds_bulk = hres->counters[0][kCntBusyNs] * 1e-9;
    stats->busy_seconds_polish = hres->counters[1][kCntBusyNs] * 1e-9;
    for (int ps = 0; ps < 2; ++ps) {
      stats->phase_seconds[ps][0] = hres->counters[ps][kCntPopNs] * 1e-9;
      stats->phase_seconds[ps][1] = hres->counters[ps][kCntStageNs] * 1e-9;
      stats->phase_seconds[ps][2] = hres->counters[ps][kCntSweepNs] * 1e-9;
      stats->phase_seconds[ps][3] = hres->counters[ps][kCntFlagNs] * 1e-9;
      stats->revisits[ps] = hres->counters[ps][kCntRevisits];
      stats->revisit_sweeps[ps] = hres->counters[ps][kCntRevisitSweeps];
      stats->revisit_updates[ps] = hres->counters[ps][kCntRevisitUpdates];
    }
    for (int ps = 0; ps < 3; ++ps) stats->max_visit_sweeps[ps] = hres->counters[ps][kCntMaxSweeps];
    stats->precision_used = polish ? EIK_FP32_POLISH : EIK_FP64;
    stats->bulk_kappa = polish ? hres->kappa_bulk : 0.0;
    double r;
    unsigned long long rb = hres->resid_bits;
    memcpy(&r, &rb, 8);
    stats->residual_max = r;
    unsigned long long ub = hres->final_umax_bits;
    ub = (ub & 0x8000000000000000ull) ? (ub & 0x7fffffffffffffffull) : ~ub;
    memcpy(&r, &ub, 8);
    double qb;
    unsigned long long qo = hres->min_q_ord;
    qo = (qo & 0x8000000000000000ull) ? (qo & 0x7fffffffffffffffull) : ~qo;
    memcpy(&qb, &qo, 8);
    stats->u_max = hres->final_umax_bits ? r + qb : 0.0;
  }
  if (hres->status) return hres->status;
  if (hres->nonfinite) return EIK_ENOCONV;
  return EIK_OK;
}

int eik_run_batch(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                  const float* const* F, const uint8_t* const* mask, const double* const* q,
                  double tol, double* const* u_out, bool host_io, cudaStream_t st,
                  eik_stats* stats, int n_override) {
  if (!ctx) return EIK_EINVAL;
  Launch L;
  int rc = eik_launch_batch(ctx, ctx->main, count, dims, h, F, mask, q, tol, u_out, host_io, st,
                            false, L, ctx->opts.hbm_budget_bytes, n_override);
  if (rc) {
    if (rc == EIK_ECUDA) cudaStreamSynchronize(st);
    return rc;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ECUDA;
  }
  return eik_finish_batch(ctx, ctx->main, L, stats);
}

size_t eik_plan_bytes(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                      bool host_io) {
  long long nodes_max = 0;
  for (int t = 0; t < count; ++t)
    nodes_max = std::max(nodes_max, (long long)dims[3 * t] * dims[3 * t + 1] * dims[3 * t + 2]);
  LaunchPlan L;
  make_plan(L, count, dims, h, choose_cell_n(ctx, nodes_max),
            ctx->opts.precision == EIK_FP32_POLISH, host_io);
  return L.total;
}

namespace eik {
int exec_init(Exec& e, bool own_stream) {
  if (own_stream) {
    if (cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
    e.own_stream = true;
  }
  for (int i = 0; i < 6; ++i) {
    if (cudaEventCreate(&e.ev[i]) != cudaSuccess) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
  }
  return EIK_OK;
}
void exec_free(Exec& e) {
  if (e.stream) cudaStreamSynchronize(e.stream);
  if (e.graph) cudaGraphExecDestroy(e.graph);
  delete e.graph_launch;
  if (e.arena) cudaFree(e.arena);
  if (e.h_small) cudaFreeHost(e.h_small);
  if (e.h_out) cudaFreeHost(e.h_out);
  if (e.h_ctl) cudaFreeHost(e.h_ctl);
  for (int i = 0; i < 6; ++i)
    if (e.ev[i]) cudaEventDestroy(e.ev[i]);
  if (e.own_stream && e.stream) cudaStreamDestroy(e.stream);
  cudaGetLastError();
  e = Exec();
}
}  // namespace eik

// ---------------------------------------------------------------------------
// C ABI.
extern "C" {

int eik_opts_default(eik_opts* o) {
  if (!o) return EIK_EINVAL;
  memset(o, 0, sizeof(*o));
  o->device = 0;
  o->precision = EIK_FP32_POLISH;
  o->cell_n = 0;
  o->hbm_budget_bytes = 0;
  o->spin_cap_us = 5000000ull;
  o->bucket_width = 0.25;
  o->max_sweeps_per_visit = 4096;
  o->bulk_kappa_rel = 0.0;  // chosen from the field
  o->queue_order = 1;
  o->use_graphs = 1;
  return EIK_OK;
}

int eik_struct_sizes(size_t* opts_bytes, size_t* stats_bytes) {
  if (opts_bytes) *opts_bytes = sizeof(eik_opts);
  if (stats_bytes) *stats_bytes = sizeof(eik_stats);
  return EIK_OK;
}

const char* eik_strerror(int s) {
  switch (s) {
    case EIK_OK: return "ok";
    case EIK_EINVAL: return "invalid argument";
    case EIK_ENOMEM: return "out of memory";
    case EIK_EBUDGET: return "device memory budget exceeded";
    case EIK_ECUDA: return "CUDA error";
    case EIK_ETIMEOUT: return "device wait limit reached without progress";
    case EIK_ENOCONV: return "cell sweeps did not converge";
    case EIK_ECANCELLED: return "request cancelled";
    case EIK_EQUEUE: return "device queue inconsistency";
    case EIK_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

int eik_create(eik_ctx** out, const eik_opts* opts) {
  if (!out) return EIK_EINVAL;
  *out = nullptr;
  eik_opts o;
  if (opts) {
    o = *opts;
  } else {
    eik_opts_default(&o);
  }
  if (o.precision != EIK_FP64 && o.precision != EIK_FP32_POLISH) return EIK_EINVAL;
  if (o.cell_n != 0 && size_index(o.cell_n) < 0) return EIK_EINVAL;
  if (o.max_ctas < 0 || o.queue_order < 0 || o.queue_order > 1 || o.cell_key < 0 ||
      o.cell_key > 1 ||
      !(o.warps_per_cell == 0 || o.warps_per_cell == 4 || o.warps_per_cell == 6 ||
        o.warps_per_cell == 8))
    return EIK_EINVAL;
  if (o.max_sweeps_per_visit <= 0) o.max_sweeps_per_visit = 4096;
  if (!(o.bulk_kappa_rel >= 0.0) || isinf(o.bulk_kappa_rel)) return EIK_EINVAL;
  if (!(o.polish_lift > -0.5 && o.polish_lift < 1.0)) return EIK_EINVAL;
  if (!(o.bucket_width > 0.0)) o.bucket_width = 0.25;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    return EIK_ECUDA;
  }
  eik_ctx* c = new (std::nothrow) eik_ctx();
  if (!c) return EIK_ENOMEM;
  c->opts = o;
  c->device = o.device;
  if (cudaSetDevice(o.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return EIK_ECUDA;
  }
  c->main.stream = c->stream;
  if (exec_init(c->main, false) != EIK_OK) {
    eik_destroy(c);
    return EIK_ECUDA;
  }
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qres;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &qres) != cudaSuccess ||
      qres != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    eik_destroy(c);
    return EIK_ECUDA;
  }
  c->encode = reinterpret_cast<EncodeTiledFn>(fn);
  *out = c;
  return EIK_OK;
}

int eik_destroy(eik_ctx* c) {
  if (!c) return EIK_OK;
  cudaSetDevice(c->device);
  if (c->serve) serve_destroy(c->serve);
  if (c->stream) cudaStreamSynchronize(c->stream);
  exec_free(c->main);
  exec_free(c->gexec);
  for (int i = 0; i < 3; ++i) {
    if (c->d_tab[i]) cudaFree(c->d_tab[i]);
    if (c->d_off[i]) cudaFree(c->d_off[i]);
  }
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return EIK_OK;
}

int eik_solve(eik_ctx* ctx, const int64_t dims[3], double h, const float* F,
              const uint8_t* src_mask, const double* q, double tol, double* u_out,
              eik_stats* stats) {
  if (!ctx) return EIK_EINVAL;
  return eik_run_batch(ctx, 1, dims, &h, &F, &src_mask, &q, tol, &u_out, true, ctx->stream,
                       stats, 0);
}

int eik_solve_device(eik_ctx* ctx, const int64_t dims[3], double h, const float* F_dev,
                     const uint8_t* src_mask_dev, const double* q_dev, double tol,
                     double* u_out_dev, void* stream, eik_stats* stats) {
  if (!ctx) return EIK_EINVAL;
  return eik_run_batch(ctx, 1, dims, &h, &F_dev, &src_mask_dev, &q_dev, tol, &u_out_dev, false,
                       reinterpret_cast<cudaStream_t>(stream), stats, 0);
}

int eik_autotune(eik_ctx* ctx, const int64_t dims[3], double h, const float* F,
                 const uint8_t* src_mask, const double* q, double tol, int* best_n,
                 int* best_ctas) {
  if (!ctx || !dims || !F || !src_mask || !q || !valid_dims(dims)) return EIK_EINVAL;
  const long long nodes = (long long)dims[0] * dims[1] * dims[2];
  double* u = static_cast<double*>(malloc((size_t)nodes * sizeof(double)));
  if (!u) return EIK_ENOMEM;
  const eik_opts saved = ctx->opts;
  // worker shapes: (cell size, warps per 16^3 cell; 0 = the default shape of
  // each pass)
  const int cands[6][2] = {{4, 0}, {8, 0}, {16, 0}, {16, 4}, {16, 6}, {16, 8}};
  double best = 1e300;
  int bn = 0, bc = 0, bw = 0, rc = EIK_OK;
  for (int ci = 0; ci < 6 && rc == EIK_OK; ++ci) {
    const int n = cands[ci][0];
    if (n == 4 && nodes > (1ll << 22)) continue;  // many small cells: queue-bound
    for (int per_sm = 1; per_sm <= 2; ++per_sm) {
      ctx->opts.cell_n = n;
      ctx->opts.max_ctas = per_sm * ctx->sms;
      ctx->opts.warps_per_cell = cands[ci][1];
      double t = 0.0;
      for (int rep = 0; rep < 2 && rc == EIK_OK; ++rep) {  // first run warms up
        eik_stats st;
        rc = eik_solve(ctx, dims, h, F, src_mask, q, tol, u, &st);
        t = st.seconds;
      }
      if (rc == EIK_OK && t < best) {
        best = t;
        bn = n;
        bc = per_sm * ctx->sms;
        bw = cands[ci][1];
      }
    }
  }
  ctx->opts = saved;
  free(u);
  if (rc != EIK_OK) return rc;
  ctx->tuned[size_bucket(nodes)] = eik_ctx::Tuned{bn, bc, bw};
  ++ctx->tune_generation;  // a captured batch graph may hold the old choice
  if (best_n) *best_n = bn;
  if (best_ctas) *best_ctas = bc;
  return EIK_OK;
}

int eik_solve_batch(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                    const float* const* F, const uint8_t* const* src_mask,
                    const double* const* q, double tol, double* const* u_out, eik_stats* stats) {
  if (!ctx) return EIK_EINVAL;
  return eik_run_batch(ctx, count, dims, h, F, src_mask, q, tol, u_out, true, ctx->stream, stats,
                       0);
}

int eik_solve_batch_device(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                           const float* const* F_dev, const uint8_t* const* src_mask_dev,
                           const double* const* q_dev, double tol, double* const* u_out_dev,
                           void* stream, eik_stats* stats) {
  if (!ctx) return EIK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!ctx->opts.use_graphs || count < 1 || !dims || !h || !F_dev || !src_mask_dev || !q_dev ||
      !u_out_dev)
    return eik_run_batch(ctx, count, dims, h, F_dev, src_mask_dev, q_dev, tol, u_out_dev, false,
                         st, stats, 0);
  // The whole launch sequence of this batch is captured once as a CUDA graph
  // and replayed while every argument is the same (same grids, buffers and
  // options: the arena layout and the tensor maps then match too).
  Exec& ex = ctx->gexec;
  if (!ex.ev[0] && exec_init(ex, false) != EIK_OK) return EIK_ECUDA;
  std::vector<unsigned long long> key;
  key.push_back((unsigned long long)count);
  unsigned long long tb;
  memcpy(&tb, &tol, 8);
  key.push_back(tb);
  key.push_back((unsigned long long)(uintptr_t)st);
  key.push_back(ctx->tune_generation);
  for (int t = 0; t < count; ++t) {
    for (int a = 0; a < 3; ++a) key.push_back((unsigned long long)dims[3 * t + a]);
    unsigned long long hb;
    memcpy(&hb, &h[t], 8);
    key.push_back(hb);
    key.push_back((unsigned long long)(uintptr_t)F_dev[t]);
    key.push_back((unsigned long long)(uintptr_t)src_mask_dev[t]);
    key.push_back((unsigned long long)(uintptr_t)q_dev[t]);
    key.push_back((unsigned long long)(uintptr_t)u_out_dev[t]);
  }
  if (!(ex.graph && key == ex.graph_key && ex.graph_launch)) {
    // first call with these arguments: run it plainly (this also sizes the
    // arena and staging), then capture the same sequence for later calls
    Launch plain;
    int rc = eik_launch_batch(ctx, ex, count, dims, h, F_dev, src_mask_dev, q_dev, tol, u_out_dev,
                              false, st, false, plain, ctx->opts.hbm_budget_bytes, 0);
    if (rc != EIK_OK) {
      cudaStreamSynchronize(st);
      cudaGetLastError();
      return rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
    rc = eik_finish_batch(ctx, ex, plain, stats);
    if (rc != EIK_OK) return rc;
    if (ex.graph) {
      cudaGraphExecDestroy(ex.graph);
      ex.graph = nullptr;
    }
    ex.graph_key.clear();
    if (!ex.graph_launch) ex.graph_launch = new (std::nothrow) Launch();
    if (!ex.graph_launch) return EIK_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return EIK_OK;  // graphs unavailable on this stream: stay with plain launches
    }
    const int lrc = eik_launch_batch(ctx, ex, count, dims, h, F_dev, src_mask_dev, q_dev, tol,
                                     u_out_dev, false, st, false, *ex.graph_launch,
                                     ctx->opts.hbm_budget_bytes, 0);
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (lrc != EIK_OK || ce != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return EIK_OK;
    }
    const cudaError_t ie = cudaGraphInstantiate(&ex.graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      ex.graph = nullptr;
      return EIK_OK;
    }
    ex.graph_key = key;
    return EIK_OK;
  }
  if (cudaGraphLaunch(ex.graph, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ECUDA;
  }
  return eik_finish_batch(ctx, ex, *ex.graph_launch, stats);
}

}  // extern "C"

eik::ServeState*& eik_serve_slot(eik_ctx* ctx) { return ctx->serve; }
size_t eik_ctx_budget(eik_ctx* ctx) { return ctx->opts.hbm_budget_bytes; }
unsigned long long eik_ctx_batch_nodes(eik_ctx* ctx) {
  return ctx->opts.serve_batch_nodes ? ctx->opts.serve_batch_nodes : (64ull << 20);
}
