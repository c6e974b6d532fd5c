// eik_selftest.cu -- eik_selftest_local_solve: the sweeps' FP64 local solve
// (FP32 estimate + Newton step with an error-free FP32 residual) against
// the direct FP64 closed forms, on device-generated inputs.
#include <cuda_runtime.h>

#include "eik.h"
#include "eik_device.cuh"

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): a counter-based stream of 64-bit
// words; u01 takes the top 53 bits.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(unsigned long long key, int k) {
  return (double)(mix64(key + 0x632be59bd9b4e019ull * (unsigned long long)(k + 1)) >> 11) *
         (1.0 / 9007199254740992.0);
}

__global__ void selftest_kernel(long long count, unsigned long long seed,
                                unsigned long long* out) {
  unsigned long long worst_ulp = 0, worst_rel = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = mix64(seed ^ (unsigned long long)t);
    const double h = exp2(-10.0 + 6.0 * u01(key, 0));
    const double F = 0.05 + 1.95 * u01(key, 1);
    const double s = h / F;
    const double base = 2.0 * u01(key, 2);
    double a[3];
    for (int d = 0; d < 3; ++d) a[d] = base + 2.0 * s * u01(key, 3 + d);
    if (u01(key, 6) < 0.125) a[(int)(3.0 * u01(key, 7)) % 3] = CUDART_INF;
    const double u1 = eik::local_solve(a[0], a[1], a[2], s);
    const double u0 = eik::local_solve_direct(a[0], a[1], a[2], s);
    const long long d = eik::dbits(u1) - eik::dbits(u0);
    const unsigned long long du = (unsigned long long)(d < 0 ? -d : d);
    worst_ulp = du > worst_ulp ? du : worst_ulp;
    // difference over (one ulp of the direct result + 2^-44 s): the sweeps'
    // solve carries its Newton residual in FP32 pairs, good to ~2^-45 s
    const double ulp0 = fabs(__longlong_as_double(eik::dbits(u0) + 1) - u0);
    const double rel = fabs(u1 - u0) / (ulp0 + 5.684341886080802e-14 * s);
    const unsigned long long rb = (unsigned long long)__double_as_longlong(rel);
    worst_rel = rb > worst_rel ? rb : worst_rel;
  }
  atomicMax(out, worst_ulp);
  atomicMax(out + 1, worst_rel);
}

}  // namespace

extern "C" int eik_selftest_local_solve(int device, int64_t count, uint64_t seed,
                                        double* max_ulps, double* max_rel) {
  if (count < 1 || !max_ulps || !max_rel) return EIK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return EIK_ECUDA;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return EIK_ECUDA;
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) {
    long long blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    selftest_kernel<<<(unsigned)blocks, 256>>>((long long)count, (unsigned long long)seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return EIK_ECUDA;
  *max_ulps = (double)h[0];
  *max_rel = __builtin_bit_cast(double, h[1]);
  return EIK_OK;
}
