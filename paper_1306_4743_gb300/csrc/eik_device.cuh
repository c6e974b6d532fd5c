// eik_device.cuh -- device helpers of libeik.so: PTX wrappers (TMA, mbarrier,
// proxy fences, acquire loads), ordered float keys, the device Dial bucket
// queue that replaces the cell heap of Alg. 1 / Alg. 3, and the local solve
// of Eq. 2.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "eik.h"
#include "eik_internal.h"

namespace eik {

// ---------------------------------------------------------------------------
// Small PTX wrappers.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  (void)state;
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// 3D tiled tensor load (TMA) of one box into shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
      "r"(smem_u32(bar))
      : "memory");
}
// Contiguous bulk copy global -> shared (both 16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Barrier over the `nthreads` threads of named barrier `id` with an OR
// reduction of a predicate.
__device__ __forceinline__ bool bar_red_or(int id, int nthreads, bool pred) {
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(out)
      : "r"((unsigned)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void bar_sync_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// Order-preserving maps between floats and unsigned integers, so that the
// cell value of Eq. 3 can be lowered with an integer atomicMin.
__host__ __device__ __forceinline__ unsigned ord_of_float(float f) {
#ifdef __CUDA_ARCH__
  unsigned u = __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of_ord(unsigned o) {
  unsigned u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}
__device__ __forceinline__ unsigned long long ord_of_double(double d) {
  unsigned long long u = __double_as_longlong(d);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double double_of_ord(unsigned long long o) {
  unsigned long long u = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double(u);
}
// Cell keys are floats rounded toward -inf from the value they stand for.
__device__ __forceinline__ unsigned key_of(float v) { return ord_of_float(v); }
__device__ __forceinline__ unsigned key_of(double v) { return ord_of_float(__double2float_rd(v)); }

constexpr unsigned kKeyInf = 0xFF800000u;  // ord_of_float(+inf)

__device__ __forceinline__ void set_status(Control* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

// ---------------------------------------------------------------------------
// Local solve of Eq. 2 at one node: the root U of
//   sum_d max(U - a_d, 0)^2 = s^2,   a_d = min of the two axis-d neighbours,
// taken with 1, 2 or 3 terms after sorting a1 <= a2 <= a3.  Shifted form
// (U = a1 + w, b = a_d - a1) keeps every term of the size of s; in the
// branch that uses it, each discriminant is >= s^2 in exact arithmetic:
//   2 terms: 2s^2 - b^2 with 0 <= b < s
//   3 terms: 3s^2 - (b2^2 + b3^2 + (b3 - b2)^2) >= s^2 on the 3-term region.
// FP32 variant: a discriminant below 2^-10 * 3s^2 in the 3-term branch is
// recomputed in FP64 (the near-cancellation guard; it cannot fire except
// through rounding of the inputs).
__device__ __forceinline__ float local_solve(float ax, float ay, float az, float s) {
  const float lo = fminf(ax, ay), hi = fmaxf(ax, ay);
  const float a1 = fminf(lo, az), mid = fmaxf(lo, az);
  const float a2 = fminf(hi, mid), a3 = fmaxf(hi, mid);
  const float u1 = a1 + s;
  if (u1 <= a2) return u1;  // also covers a1 = +inf (returns +inf)
  const float s2 = s * s;
  const float b = a2 - a1;
  const float u2 = a1 + 0.5f * (b + sqrtf(fmaxf(2.0f * s2 - b * b, 0.0f)));
  if (u2 <= a3) return u2;
  const float b3 = a3 - a1, e = b3 - b;
  float d3 = 3.0f * s2 - (b * b + b3 * b3 + e * e);
  if (d3 < 0.0029296875f * s2) {  // 2^-10 * 3 s^2
    const double bd = (double)a2 - (double)a1, b3d = (double)a3 - (double)a1;
    const double ed = b3d - bd, sd = (double)s;
    const double dd = 3.0 * sd * sd - (bd * bd + b3d * b3d + ed * ed);
    return a1 + (float)((bd + b3d + sqrt(fmax(dd, 0.0))) / 3.0);
  }
  return a1 + (b + b3 + sqrtf(d3)) * (1.0f / 3.0f);
}

__device__ __forceinline__ double local_solve(double ax, double ay, double az, double s) {
  const double lo = fmin(ax, ay), hi = fmax(ax, ay);
  const double a1 = fmin(lo, az), mid = fmax(lo, az);
  const double a2 = fmin(hi, mid), a3 = fmax(hi, mid);
  const double u1 = a1 + s;
  if (u1 <= a2) return u1;
  const double s2 = s * s;
  const double b = a2 - a1;
  const double u2 = a1 + 0.5 * (b + sqrt(fmax(2.0 * s2 - b * b, 0.0)));
  if (u2 <= a3) return u2;
  const double b3 = a3 - a1, e = b3 - b;
  const double d3 = 3.0 * s2 - (b * b + b3 * b3 + e * e);
  return a1 + (b + b3 + sqrt(fmax(d3, 0.0))) / 3.0;
}

template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return CUDART_INF_F; }
template <>
__device__ __forceinline__ double tinf<double>() { return CUDART_INF; }

// ---------------------------------------------------------------------------
// Device Dial bucket queue.
//
// Bucket b (an absolute, ever-growing index) holds cells whose key lies in
// [base + b/inv_width, base + (b+1)/inv_width); it lives in ring slot
// b mod kNumBuckets as a lock-free stack (Treiber stack with a 32-bit ABA
// tag in the head word).  `cur` is a lower bound of the lowest non-empty
// bucket: a push lowers it with atomicMin, a worker that finds bucket `cur`
// empty moves it to the next non-empty bucket and re-checks the buckets it
// skipped, so a push that raced the move is not stranded.  Within a bucket
// the order is arbitrary, as is the order among cells of equal priority in
// the paper; the final values do not depend on it (Sec. 4, cell values).

__device__ __forceinline__ void stack_push(const CellArrays& c, unsigned slot, unsigned cell) {
  unsigned long long* head = c.heads + slot;
  unsigned long long old = ld_relaxed_u64(head);
  for (;;) {
    c.next[cell] = (unsigned)(old & 0xffffffffull);
    __threadfence();
    const unsigned long long nw = (((old >> 32) + 1ull) << 32) | (unsigned long long)(cell + 1u);
    const unsigned long long prev = atomicCAS(head, old, nw);
    if (prev == old) return;
    old = prev;
  }
}

// Returns the popped cell or -1 when the stack is empty.
__device__ __forceinline__ int stack_pop(const CellArrays& c, unsigned slot) {
  unsigned long long* head = c.heads + slot;
  unsigned long long old = ld_acquire_u64(head);
  for (;;) {
    const unsigned top = (unsigned)(old & 0xffffffffull);
    if (top == 0) return -1;
    const unsigned cell = top - 1u;
    const unsigned nxt = ld_relaxed_u32(c.next + cell);
    const unsigned long long nw = (((old >> 32) + 1ull) << 32) | (unsigned long long)nxt;
    const unsigned long long prev = atomicCAS(head, old, nw);
    if (prev == old) {
      __threadfence();
      return (int)cell;
    }
    old = prev;
  }
}

__device__ __forceinline__ unsigned bucket_of(const Control* ctl, float keyf, unsigned cur) {
  if (!(keyf < CUDART_INF_F)) return cur;  // no usable key: take it soon
  float f = (keyf - ctl->base) * ctl->inv_width;
  if (!(f > 0.0f)) f = 0.0f;
  if (f > 1.0e9f) f = 1.0e9f;
  unsigned b = (unsigned)f;
  if (b > cur + (unsigned)(kNumBuckets - 1)) b = cur + (unsigned)(kNumBuckets - 1);
  return b;
}

// Insert a QUEUED cell into the bucket of its key.
__device__ __forceinline__ void queue_push(const CellArrays& c, Control* ctl, unsigned cell,
                                           unsigned long long* pushes) {
  const unsigned cur = ld_relaxed_u32(&ctl->cur);
  const float keyf = float_of_ord(ld_relaxed_u32(c.key + cell));
  const unsigned b = bucket_of(ctl, keyf, cur);
  atomicAdd(&ctl->queued, 1);
  stack_push(c, b & kBucketMask, cell);
  atomicMin(&ctl->cur, b);
  ++*pushes;
}

// Warp-collective pop (all 32 lanes of the calling warp).  Returns a cell
// whose state is now RUNNING, or -1 when the solve is finished or failed.
static __device__ int queue_pop_warp(const CellArrays& c, Control* ctl, unsigned long long spin_cap_ns,
                              int lane) {
  unsigned last_prog = 0xffffffffu;
  unsigned long long t_idle = 0;
  unsigned backoff = 32;
  for (;;) {
    int stop = 0, cell = -1;
    unsigned cur = 0;
    if (lane == 0) {
      stop = (ld_acquire_s32(&ctl->status) != 0) || (ld_acquire_s32(&ctl->active) <= 0);
      if (!stop) {
        cur = ld_acquire_u32(&ctl->cur);
        cell = stack_pop(c, cur & kBucketMask);
        if (cell >= 0) {
          atomicSub(&ctl->queued, 1);
          // QUEUED -> RUNNING (drops DIRTY: this visit loads the newest data)
          unsigned st = ld_relaxed_u32(c.state + cell);
          for (;;) {
            if (!(st & kStQueued)) {
              set_status(ctl, EIK_EQUEUE);
              cell = -1;
              stop = 1;
              break;
            }
            const unsigned prev = atomicCAS(c.state + cell, st, kStRunning);
            if (prev == st) break;
            st = prev;
          }
          __threadfence();
        }
      }
    }
    stop = __shfl_sync(0xffffffffu, stop, 0);
    if (stop) return -1;
    cell = __shfl_sync(0xffffffffu, cell, 0);
    if (cell >= 0) return cell;
    cur = __shfl_sync(0xffffffffu, cur, 0);

    // Bucket `cur` is empty.  Look further only if some cell is queued.
    int queued = 0;
    if (lane == 0) queued = ld_acquire_s32(&ctl->queued);
    queued = __shfl_sync(0xffffffffu, queued, 0);
    if (queued > 0) {
      int found = kNumBuckets;
      for (int base = 1; base < kNumBuckets && found == kNumBuckets; base += 128) {
        unsigned m = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int o = base + r * 32 + lane;
          const bool ne = o < kNumBuckets &&
                          (unsigned)(ld_relaxed_u64(c.heads + ((cur + (unsigned)o) & kBucketMask)) &
                                     0xffffffffull) != 0u;
          const unsigned bal = __ballot_sync(0xffffffffu, ne);
          if (bal && m == 0) m = (unsigned)(base + r * 32 + __ffs(bal) - 1);
        }
        if (m) found = (int)m;
      }
      if (found < kNumBuckets) {
        if (lane == 0) {
          if (atomicCAS(&ctl->cur, cur, cur + (unsigned)found) == cur) {
            __threadfence();
            for (int o = 0; o < found; ++o) {
              const unsigned sl = (cur + (unsigned)o) & kBucketMask;
              if ((unsigned)(ld_acquire_u64(c.heads + sl) & 0xffffffffull) != 0u) {
                atomicMin(&ctl->cur, cur + (unsigned)o);
                break;
              }
            }
          }
        }
        __syncwarp();
        backoff = 32;
        continue;
      }
    }
    // Nothing to take: wait for running cells, with a no-progress limit.
    int timed_out = 0;
    if (lane == 0) {
      const unsigned prog = ld_acquire_u32(&ctl->progress);
      const unsigned long long now = global_timer_ns();
      if (prog != last_prog) {
        last_prog = prog;
        t_idle = now;
      } else if (now - t_idle > spin_cap_ns) {
        set_status(ctl, EIK_ETIMEOUT);
        timed_out = 1;
      }
    }
    timed_out = __shfl_sync(0xffffffffu, timed_out, 0);
    if (timed_out) return -1;
    __nanosleep(backoff);
    if (backoff < 1024) backoff *= 2;
  }
}

// Tell cell `nb` that a neighbour changed its inflow border (Alg. 2 lines 8-14
// and Alg. 3 lines 20-28): lower its cell value (Eq. 3), add preferred
// directions, and queue it unless it is queued or dirty already.  A running
// cell is marked DIRTY and re-queues itself when its visit ends.  The
// caller has made its new border values visible (__threadfence) before.
__device__ __forceinline__ void flag_cell(const CellArrays& c, Control* ctl, unsigned nb,
                                          unsigned key, unsigned dirbits,
                                          unsigned long long* pushes) {
  atomicMin(c.key + nb, key);
  atomicOr(c.dir + nb, dirbits);
  const unsigned old = atomicOr(c.state + nb, kStDirty);
  if ((old & (kStQueued | kStRunning | kStDirty)) == 0u) {
    atomicAdd(&ctl->active, 1);
    atomicOr(c.state + nb, kStQueued);
    __threadfence();
    queue_push(c, ctl, nb, pushes);
  }
}

// End of a visit: RUNNING -> IDLE, or RUNNING|DIRTY -> QUEUED with a re-push.
// The active count drops only after every flag of this visit (Sec. 5: the
// counter is decremented after processing so no worker quits early).
__device__ __forceinline__ void retire_cell(const CellArrays& c, Control* ctl, unsigned cell,
                                            unsigned long long* pushes) {
  unsigned st = ld_relaxed_u32(c.state + cell);
  unsigned nw;
  for (;;) {
    nw = (st & kStDirty) ? kStQueued : 0u;
    const unsigned prev = atomicCAS(c.state + cell, st, nw);
    if (prev == st) break;
    st = prev;
  }
  if (nw == kStQueued) {
    __threadfence();
    queue_push(c, ctl, cell, pushes);
  } else {
    __threadfence();
    atomicSub(&ctl->active, 1);
  }
  atomicAdd(&ctl->progress, 1u);
}

}  // namespace eik
