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
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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
// 64-bit compare-and-swap with release (acquire) ordering at GPU scope.
__device__ __forceinline__ unsigned long long cas_release_u64(unsigned long long* p,
                                                              unsigned long long cmp,
                                                              unsigned long long val) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(cmp), "l"(val)
               : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long cas_acquire_u64(unsigned long long* p,
                                                              unsigned long long cmp,
                                                              unsigned long long val) {
  unsigned long long old;
  asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(cmp), "l"(val)
               : "memory");
  return old;
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
// Square root on the special-function unit (about 2 ulp): the FP32 bulk
// pass only has to land close to the fixed point; the FP64 polish settles it.
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float local_solve(float ax, float ay, float az, float s) {
  const float lo = fminf(ax, ay), hi = fmaxf(ax, ay);
  const float a1 = fminf(lo, az), mid = fmaxf(lo, az);
  const float a2 = fminf(hi, mid), a3 = fmaxf(hi, mid);
  const float u1 = a1 + s;
  if (u1 <= a2) return u1;  // also covers a1 = +inf (returns +inf)
  const float s2 = s * s;
  const float b = a2 - a1;
  const float u2 = a1 + 0.5f * (b + sqrt_fast(fmaxf(2.0f * s2 - b * b, 0.0f)));
  if (u2 <= a3) return u2;
  const float b3 = a3 - a1, e = b3 - b;
  float d3 = 3.0f * s2 - (b * b + b3 * b3 + e * e);
  if (d3 < 0.0029296875f * s2) {  // 2^-10 * 3 s^2
    const double bd = (double)a2 - (double)a1, b3d = (double)a3 - (double)a1;
    const double ed = b3d - bd, sd = (double)s;
    const double dd = 3.0 * sd * sd - (bd * bd + b3d * b3d + ed * ed);
    return a1 + (float)((bd + b3d + sqrt(fmax(dd, 0.0))) / 3.0);
  }
  return a1 + (b + b3 + sqrt_fast(d3)) * (1.0f / 3.0f);
}

// Values are stored relative to the smallest exit value, so every value is
// >= 0 or +inf and two doubles order like their bit patterns: the FP64
// min / max / compare run on the integer pipes, leaving the (narrow) FP64
// pipe to the arithmetic.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ double dmin_nn(double a, double b) {
  const long long ia = dbits(a), ib = dbits(b);
  return __longlong_as_double(ia < ib ? ia : ib);
}
__device__ __forceinline__ double dmax_nn(double a, double b) {
  const long long ia = dbits(a), ib = dbits(b);
  return __longlong_as_double(ia < ib ? ib : ia);
}
__device__ __forceinline__ bool dle_nn(double a, double b) { return dbits(a) <= dbits(b); }

// Direct FP64 evaluation of the same root, with sqrt(double): the reference
// eik_selftest_local_solve checks the sweeps' solve against.
__device__ __forceinline__ double local_solve_direct(double ax, double ay, double az, double s) {
  const double lo = dmin_nn(ax, ay), hi = dmax_nn(ax, ay);
  const double a1 = dmin_nn(lo, az), mid = dmax_nn(lo, az);
  const double a2 = dmin_nn(hi, mid), a3 = dmax_nn(hi, mid);
  const double u1 = a1 + s;
  if (dle_nn(u1, a2)) return u1;  // also covers a1 = +inf (returns +inf)
  const double s2 = s * s;
  const double b = a2 - a1;
  const double u2 = a1 + 0.5 * (b + sqrt(fmax(2.0 * s2 - b * b, 0.0)));
  if (dle_nn(u2, a3)) return u2;
  const double b3 = a3 - a1, e = b3 - b;
  const double d3 = 3.0 * s2 - (b * b + b3 * b3 + e * e);
  return a1 + (b + b3 + sqrt(fmax(d3, 0.0))) * 0.33333333333333331;
}

// double <-> float conversions on the integer pipe for values >= 0: the
// conversion instructions take the FP64 path, whose latency (about 64 cycles
// per dependent operation on this GPU) dominates the FP64 sweeps.  The
// narrowing truncates the mantissa (relative error < 2^-23), which is all
// the FP32 estimate below needs; values below the float range become 0,
// above it +inf.
__device__ __forceinline__ float f32_of_f64_nn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) - 896;
  const unsigned r = ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull);
  return __uint_as_float(e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : r));
}
__device__ __forceinline__ double f64_of_f32_nn(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long e = u >> 23;
  const unsigned long long r = ((e + 896ull) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double(
      (long long)(e == 0 ? 0ull : (e == 255 ? 0x7ff0000000000000ull : r)));
}
__device__ __forceinline__ bool dlt_nn(double a, double b) { return dbits(a) < dbits(b); }
// Round-to-nearest narrowing of a double x >= 0 (or +inf) on the integer
// pipe: the truncation plus one float ulp when the dropped bits are more
// than half an ulp (ties away from zero; values below the float normal
// range become 0).
__device__ __forceinline__ float f32_of_f64_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const float t = f32_of_f64_nn(x);
  const unsigned up = ((b >> 28) & 1ull) && (b >> 52) > 896 && (b >> 52) < 1151 ? 1u : 0u;
  return __uint_as_float(__float_as_uint(t) + up);
}

// A double x >= 0 as hi + lo with hi its leading 24 mantissa bits (the
// truncation f32_of_f64_nn) and lo the remaining 29 bits rounded to a float:
// x = hi + lo to about 2^-48 relative.  Integer pipe and one int -> float
// conversion; no FP64 instruction.  Values below 2^-74 give lo = 0.
__device__ __forceinline__ void split_nn(double x, float& hi, float& lo) {
  hi = f32_of_f64_nn(x);
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52);
  const unsigned low = (unsigned)(b & 0x1fffffffull);  // bits below the float mantissa
  // low * 2^(e - 1075), the scale built as a float power of two
  const int pe = e - 1075 + 127;
  lo = (pe >= 1 && pe <= 254 && e < 2047) ? __uint2float_rn(low) * __int_as_float(pe << 23)
                                           : 0.0f;
}

// a + b = s + t exactly (Knuth's two-sum), FP32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// a double from a float of either sign, on the integer pipe (0 for float
// subnormals, which only arise as negligible corrections here).
__device__ __forceinline__ double f64_of_f32(float x) {
  const double m = f64_of_f32_nn(fabsf(x));
  return __longlong_as_double(__double_as_longlong(m) |
                              ((long long)(__float_as_uint(x) & 0x80000000u) << 32));
}

// FP64 local solve used by the sweeps: the shifted root w = U - a1 of
//   f(w) = sum_{d<=m} (w - b_d)^2 - s^2 = 0,   b_1 = 0, b_d = a_d - a1,
// is first found in FP32 (term count m, and w32 to ~1e-7 relative), then
// refined by one step:  U = (a1 + w32) + delta with delta from f(w32) and
// f'(w) = 2 sum_{d<=m} (w - b_d) >= 2w >= 2s/sqrt(3) (newton_step: Newton
// plus the second-order term, since f is quadratic; a plain Newton step
// would leave m e0^2 / f' ~ 2^-41 s).  The one-term root is exact
// (U = a1 + s).  Near a branch boundary the m-term
// roots of both branches agree to O(e0^2 / s), so the FP32 choice of m
// costs nothing.
//
// f(w32) is a small difference of O(s^2) terms, so it is evaluated with
// error-free FP32 transformations instead of FP64 arithmetic: with b_d and
// s split into float pairs (hi + lo), w32 - hi(b_d) and every square are
// formed exactly (two-sum, FMA), the large terms are summed exactly, and
// the lo parts enter through their first- and second-order terms.  f then
// carries an error of ~2^-48 s^2, below what the FP64 result can resolve.
// On this GPU an FP64 warp instruction occupies a scheduler's FP64 unit
// for ~80 cycles (measured) against ~1 for FP32, so the step uses four FP64
// instructions (b2, b3, a1 + w32, + correction) instead of ten.
template <int M>
__device__ __forceinline__ float newton_residual(float w, float B2, float L2, float B3, float L3,
                                                 float S, float LS) {
  // d = 1: (w - 0)^2 exactly
  const float q = w * w, qe = fmaf(w, w, -q);
  // d = 2: w - b2 = r2 + (er2 - L2)
  float r2, er2;
  two_sum(w, -B2, r2, er2);
  const float e2 = er2 - L2;
  const float p2 = r2 * r2, p2e = fmaf(r2, r2, -p2);
  // s^2 = S^2 + 2 S LS + LS^2, S^2 exactly
  const float ss = S * S, sse = fmaf(S, S, -ss);
  float t1, c1, t2, c2;
  two_sum(q, p2, t1, c1);
  float small = c1 + qe + p2e - sse + fmaf(2.0f * r2, e2, e2 * e2) - fmaf(2.0f * S, LS, LS * LS);
  if constexpr (M == 3) {
    float r3, er3;
    two_sum(w, -B3, r3, er3);
    const float e3 = er3 - L3;
    const float p3 = r3 * r3, p3e = fmaf(r3, r3, -p3);
    float t0, c0;
    two_sum(t1, p3, t0, c0);
    t1 = t0;
    small += c0 + p3e + fmaf(2.0f * r3, e3, e3 * e3);
  }
  two_sum(t1, -ss, t2, c2);
  return t2 + (c2 + small);
}

// The correction delta solving f(w0) + f'(w0) delta + M delta^2 = 0 (f is a
// quadratic with f'' = 2M) to second order: delta1 = -f / f', then
// delta = delta1 (1 - M delta1 / f'), leaving an error O(delta1^3 / s^2).
template <int M>
__device__ __forceinline__ float newton_step(float f, float rinv) {
  const float d1 = -f * rinv;
  return d1 * fmaf(-(float)M * d1, rinv, 1.0f);
}

__device__ __forceinline__ double local_solve(double ax, double ay, double az, double s) {
  const double lo = dmin_nn(ax, ay), hi = dmax_nn(ax, ay);
  const double a1 = dmin_nn(lo, az), mid = dmax_nn(lo, az);
  const double a2 = dmin_nn(hi, mid), a3 = dmax_nn(hi, mid);
  const double b2 = a2 - a1, b3 = a3 - a1;
  // One term when a1 + s <= a2, tested as s <= b2 so that the sum stays off
  // the two- and three-term paths; a1 = +inf (no information) also returns
  // a1 + s = +inf.  Both tests run on the integer pipe.
  if (dle_nn(s, b2) || dbits(a1) >= dbits(CUDART_INF)) return a1 + s;
  float S, LS, B2, L2, B3, L3;
  split_nn(s, S, LS);
  split_nn(b2, B2, L2);
  split_nn(b3, B3, L3);  // b3 = +inf: B3 = +inf, L3 = 0
  const float S2 = S * S;
  const float w2 = 0.5f * (B2 + sqrt_fast(fmaxf(2.0f * S2 - B2 * B2, 0.0f)));
  if (w2 <= B3) {
    const double a1w = a1 + f64_of_f32_nn(w2);
    const float f = newton_residual<2>(w2, B2, L2, 0.0f, 0.0f, S, LS);
    return a1w + f64_of_f32(newton_step<2>(f, __fdividef(0.5f, 2.0f * w2 - B2)));
  }
  const float e = B3 - B2;
  const float d3 = 3.0f * S2 - (B2 * B2 + B3 * B3 + e * e);
  const float w3 = (B2 + B3 + sqrt_fast(fmaxf(d3, 0.0f))) * (1.0f / 3.0f);
  const double a1w = a1 + f64_of_f32_nn(w3);
  const float f = newton_residual<3>(w3, B2, L2, B3, L3, S, LS);
  return a1w + f64_of_f32(newton_step<3>(f, __fdividef(0.5f, 3.0f * w3 - B2 - B3)));
}

// Whether v - nv > kappa for stored values (>= 0), without an FP64
// instruction: the drop in units of the last place of v (the bit-pattern
// difference; exact within a binade, an over-count by at most 2x across
// one, which only makes the test conservative) against kappa / ulp(v) in
// FP32.  kf = kappa as a float.
__device__ __forceinline__ bool drop_exceeds(double nv, double v, float kf) {
  const long long iv = dbits(v), in = dbits(nv);
  if (in >= iv) return false;
  if (kf == 0.0f || iv >= dbits(CUDART_INF)) return true;
  const unsigned long long D = (unsigned long long)(iv - in);
  const int pe = 1075 - (int)(iv >> 52) + 127;  // 2^(1075 - e_v) = 1 / ulp(v), as a float
  if (pe < 1 || pe > 254) return (v - nv) > (double)kf;
  const float T = kf * __int_as_float(pe << 23);
  const float Df = (D >> 32) ? __uint2float_rn((unsigned)(D >> 20)) * 1048576.0f
                             : __uint2float_rn((unsigned)D);
  return Df > T;
}

// Axis minimum of two neighbour values.
__device__ __forceinline__ float nmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double nmin(double a, double b) { return dmin_nn(a, b); }

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
// b mod kNumBuckets as kSubStacks lock-free stacks (Treiber stacks with a
// 32-bit ABA tag in the head word) and a count of the cells in it.  A push
// picks a sub-stack by a hash of the cell id and a popping warp reads all
// sub-stack heads at once (a lane each), starting its choice at a
// worker-specific one, so the compare-and-swaps of several hundred workers
// spread over 32 words instead of queueing on one.  `cur` is the bucket
// being processed.  Workers take cells only from bucket `cur`, and `cur`
// moves on only when its count is zero AND no cell taken from it is still
// being swept (run[slot] == 0): the buckets are processed in order, like the
// heap of Alg. 1 processes cells in order of their values, while all cells
// of one bucket run in parallel.  A push into a lower bucket lowers `cur`
// (atomicMin).  The count rises before the cell is linked in and falls after
// it is unlinked, so a zero count means an empty bucket; a worker that moves
// `cur` forward re-checks the buckets it skipped, so a push that raced the
// move is not stranded.  Within a bucket the order is arbitrary; the final
// values do not depend on the processing order (Sec. 4).

__device__ __forceinline__ unsigned long long* sub_head(const CellArrays& c, unsigned slot,
                                                        unsigned sub) {
  return c.heads + (size_t)slot * kSubStacks + sub;
}

__device__ __forceinline__ void stack_push(unsigned long long* head, const CellArrays& c,
                                           unsigned cell) {
  unsigned long long old = ld_relaxed_u64(head);
  for (;;) {
    c.next[cell] = (unsigned)(old & 0xffffffffull);
    // release: the link above is visible before the new head
    const unsigned long long nw = (((old >> 32) + 1ull) << 32) | (unsigned long long)(cell + 1u);
    const unsigned long long prev = cas_release_u64(head, old, nw);
    if (prev == old) return;
    old = prev;
  }
}

// Returns the popped cell or -1 when the sub-stack is empty; `old` is a
// recent value of its head.
__device__ __forceinline__ int stack_pop(unsigned long long* head, const CellArrays& c,
                                         unsigned long long old) {
  for (;;) {
    const unsigned top = (unsigned)(old & 0xffffffffull);
    if (top == 0) return -1;
    const unsigned cell = top - 1u;
    const unsigned nxt = ld_relaxed_u32(c.next + cell);
    const unsigned long long nw = (((old >> 32) + 1ull) << 32) | (unsigned long long)nxt;
    // acquire: what the pusher wrote before its release is visible after
    const unsigned long long prev = cas_acquire_u64(head, old, nw);
    if (prev == old) return (int)cell;
    old = prev;
  }
}

__device__ __forceinline__ bool bucket_empty(const CellArrays& c, unsigned slot) {
  return ld_acquire_s32(c.cnt + slot) <= 0;
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
  const unsigned slot = b & kBucketMask;
  atomicAdd(&ctl->queued, 1);
  atomicAdd(c.cnt + slot, 1);
  stack_push(sub_head(c, slot, (cell * 0x9E3779B1u) >> (32 - kSubStackBits)), c, cell);
  __threadfence();
  atomicMin(&ctl->cur, b);
  ++*pushes;
}

// First non-empty bucket at offset 1..kNumBuckets-1 after `cur`, or
// kNumBuckets (warp-collective).  Looks 128 buckets ahead, then, if cells
// are queued further on, around the whole ring.
__device__ __forceinline__ int scan_next_bucket(const CellArrays& c, unsigned cur, bool full,
                                                int lane) {
  const int limit = full ? kNumBuckets : 129;
  for (int base = 1; base < limit; base += 128) {
    unsigned m = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int o = base + r * 32 + lane;
      const bool ne = o < kNumBuckets &&
                      ld_relaxed_s32(c.cnt + ((cur + (unsigned)o) & kBucketMask)) > 0;
      const unsigned bal = __ballot_sync(0xffffffffu, ne);
      if (bal && m == 0) m = (unsigned)(base + r * 32 + __ffs(bal) - 1);
    }
    if (m) return (int)m;
  }
  return kNumBuckets;
}

// Warp-collective attempt to take a cell from bucket `b` (absolute index):
// the lanes read the bucket's 32 sub-stack heads at once and pop from the
// first non-empty one at or after the warp's own starting sub-stack.
// Returns the cell, now RUNNING, or -1 if every sub-stack was empty or every
// pop lost its race; *stop is set on a queue inconsistency (status set).
// The bucket's run count is raised before the pop (so a strict-order
// advance waits for it) and stays raised for a taken cell until it retires.
__device__ __forceinline__ int try_pop_bucket(const CellArrays& c, Control* ctl, unsigned b,
                                              unsigned sub, int lane, unsigned* slot_out,
                                              int* stop) {
  const unsigned slot = b & kBucketMask;
  unsigned long long* head = sub_head(c, slot, sub);
  const unsigned long long h = ld_acquire_u64(head);
  unsigned ne = __ballot_sync(0xffffffffu, (h & 0xffffffffull) != 0ull);
  if (!ne) return -1;
  if (lane == 0) atomicAdd(c.run + slot, 1);  // reserve before taking: blocks an advance
  __syncwarp();
  int cell = -1;
  while (ne) {
    const int l = __ffs(ne) - 1;
    int got = -1;
    if (lane == l) got = stack_pop(head, c, h);
    got = __shfl_sync(0xffffffffu, got, l);
    if (got >= 0) {
      cell = got;
      break;
    }
    ne &= ne - 1u;
  }
  int bad = 0;
  if (lane == 0) {
    if (cell < 0) {
      atomicSub(c.run + slot, 1);
    } else {
      atomicSub(c.cnt + slot, 1);
      atomicSub(&ctl->queued, 1);
      // QUEUED -> RUNNING (drops DIRTY: this visit loads the newest data)
      unsigned st = ld_relaxed_u32(c.state + cell);
      for (;;) {
        if (!(st & kStQueued)) {
          set_status(ctl, EIK_EQUEUE);
          bad = 1;
          break;
        }
        const unsigned prev = atomicCAS(c.state + cell, st, kStRunning);
        if (prev == st) break;
        st = prev;
      }
      __threadfence();
      *slot_out = slot;
    }
  }
  bad = __shfl_sync(0xffffffffu, bad, 0);
  if (bad) {
    *stop = 1;
    return -1;
  }
  return __shfl_sync(0xffffffffu, cell, 0);
}

// Move `cur` from `from` to `to` (> from) if no other worker moved it, then
// pull it back to any bucket in between that a racing push filled.
// Lane 0 only.
__device__ __forceinline__ void advance_cur(const CellArrays& c, Control* ctl, unsigned from,
                                            unsigned to) {
  if (atomicCAS(&ctl->cur, from, to) == from) {
    __threadfence();
    for (unsigned o = from; o < to; ++o) {
      if (!bucket_empty(c, o & kBucketMask)) {
        atomicMin(&ctl->cur, o);
        break;
      }
    }
  }
}

// Warp-collective pop (all 32 lanes of the calling warp).  Returns a cell
// whose state is now RUNNING (and the ring slot it came from in *slot_out),
// or -1 when the solve is finished or failed.  `rot` picks the sub-stack the
// warp tries first.
//
// Relaxed order takes a cell from the lowest non-empty bucket: when bucket
// `cur` has nothing to take, the warp looks at once at the bucket counts
// ahead of it and pops from the first non-empty bucket, moving `cur` there
// if bucket `cur` is empty.  (Waiting for `cur` to advance before looking
// further left most workers idle while thousands of cells sat in the next
// few buckets: pushes of revisited cells keep pulling `cur` back.)  Strict
// order takes cells from bucket `cur` only, and moves on once none taken
// from it is still running.
static __device__ int queue_pop_warp(const CellArrays& c, Control* ctl,
                                     unsigned long long spin_cap_ns, int lane,
                                     unsigned* slot_out, bool relaxed, unsigned rot) {
  unsigned last_prog = 0xffffffffu;
  unsigned long long t_idle = 0;
  unsigned backoff = 64;
  unsigned polls = 0;
  const unsigned sub = (lane + rot) & (kSubStacks - 1);
  for (;;) {
    int stop = 0, can_advance = 0;
    unsigned cur = 0;
    // Termination and errors are checked every 4th poll, to keep the
    // traffic of waiting workers on the shared control words low.
    const bool full_check = (polls & 3u) == 0u;
    if (lane == 0) {
      if (full_check)
        stop = (ld_acquire_s32(&ctl->status) != 0) || (ld_acquire_s32(&ctl->active) <= 0);
      if (!stop) cur = ld_acquire_u32(&ctl->cur);
    }
    stop = __shfl_sync(0xffffffffu, stop, 0);
    if (stop) return -1;
    cur = __shfl_sync(0xffffffffu, cur, 0);
    const unsigned slot = cur & kBucketMask;
    int cell = try_pop_bucket(c, ctl, cur, sub, lane, slot_out, &stop);
    if (stop) return -1;
    if (cell >= 0) return cell;
    ++polls;
    if (relaxed) {
      // the lowest non-empty bucket within 128 ahead of `cur`
      const int found = scan_next_bucket(c, cur, false, lane);
      if (found < kNumBuckets) {
        const unsigned b = cur + (unsigned)found;
        if (lane == 0 && bucket_empty(c, slot)) advance_cur(c, ctl, cur, b);
        __syncwarp();
        cell = try_pop_bucket(c, ctl, b, sub, lane, slot_out, &stop);
        if (stop) return -1;
        if (cell >= 0) return cell;
        // lost every race, or caught a push or pop between its count and
        // its link: look again after the shortest wait (which still runs
        // the no-progress watchdog below)
        backoff = 64;
      }
    }
    if (lane == 0 && full_check) {
      // strict order: the bucket is done when no cell taken from it is
      // still running; relaxed order: as soon as it is empty
      can_advance = (relaxed || ld_acquire_s32(c.run + slot) == 0) && bucket_empty(c, slot);
    }
    can_advance = __shfl_sync(0xffffffffu, can_advance, 0);

    if (can_advance) {
      // bucket `cur` is finished: move to the next non-empty bucket
      int queued = 0;
      if (lane == 0) queued = ld_acquire_s32(&ctl->queued);
      queued = __shfl_sync(0xffffffffu, queued, 0);
      if (queued > 0) {
        int found = scan_next_bucket(c, cur, false, lane);
        if (found == kNumBuckets) found = scan_next_bucket(c, cur, true, lane);
        if (found < kNumBuckets) {
          if (lane == 0) advance_cur(c, ctl, cur, cur + (unsigned)found);
          __syncwarp();
          backoff = 64;
          continue;
        }
      }
    }
    // Nothing to take: wait for running cells, with a no-progress limit.
    int timed_out = 0;
    if (lane == 0 && spin_cap_ns == 0) {  // the test hook: no idle wait at all
      set_status(ctl, EIK_ETIMEOUT);
      timed_out = 1;
    } else if (lane == 0 && (polls & 15u) == 1u) {
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
    if (backoff < 2048) backoff *= 2;
  }
}

// Tell cell `nb` that a neighbour changed its inflow border (the neighbour
// flagging steps of Alg. 2 and Alg. 3): lower its cell value (Eq. 3), add preferred
// directions, and queue it unless it is queued or dirty already.  A running
// cell is marked DIRTY and re-queues itself when its visit ends.  The
// caller has made its new border values visible (__threadfence) before.
__device__ __forceinline__ void flag_cell(const CellArrays& c, Control* ctl, unsigned nb,
                                          unsigned key, unsigned dirbits,
                                          unsigned long long* pushes, bool gated = false) {
  atomicMin(c.key + nb, key);
  atomicOr(c.dir + nb, dirbits);
  // Polish schedule: a cell whose upwind neighbours have not all finished a
  // first visit is not queued yet; that first visit comes later and loads
  // this data (the read-modify-write orders it before the release).
  if (gated && atomicAdd(c.deps + nb, 0) > 0) return;
  const unsigned old = atomicOr(c.state + nb, kStDirty);
  if ((old & (kStQueued | kStRunning | kStDirty)) == 0u) {
    atomicAdd(&ctl->active, 1);
    atomicOr(c.state + nb, kStQueued);
    __threadfence();
    queue_push(c, ctl, nb, pushes);
  }
}

// End of a visit: RUNNING -> IDLE, or RUNNING|DIRTY -> QUEUED with a re-push;
// then the bucket the cell came from counts one running cell less.  The
// active count drops only after every flag of this visit (Sec. 5: the
// counter is decremented after processing so no worker quits early).
__device__ __forceinline__ void retire_cell(const CellArrays& c, Control* ctl, unsigned cell,
                                            unsigned slot, unsigned long long* pushes) {
  unsigned st = ld_relaxed_u32(c.state + cell);
  unsigned nw;
  for (;;) {
    nw = (st & kStDirty) ? kStQueued : 0u;
    const unsigned prev = atomicCAS(c.state + cell, st, nw);
    if (prev == st) break;
    st = prev;
  }
  __threadfence();
  if (nw == kStQueued) {
    queue_push(c, ctl, cell, pushes);
    __threadfence();
  }
  atomicSub(c.run + slot, 1);
  if (nw != kStQueued) atomicSub(&ctl->active, 1);
}

}  // namespace eik
