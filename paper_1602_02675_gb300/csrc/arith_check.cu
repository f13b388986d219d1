// Accuracy of the FP32 reciprocal and quotient that the FP32 kernels use
// (fp32_arith.cuh), measured against CUDA's correctly rounded division.
// Declared in include/lbm.h (lbm_check_fp32_arith).
#include <cuda_runtime.h>

#include <cstdint>

#include "fp32_arith.cuh"
#include "lbm.h"

namespace {

// Largest ulp distances found (reciprocal, quotient).  A file-scope device
// pair: the check allocates nothing.
__device__ unsigned g_worst[2];

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the i-th value of stream `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Distance in units in the last place between two positive normal floats.
__device__ __forceinline__ unsigned ulp_dist(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  return (unsigned)(ia > ib ? ia - ib : ib - ia);
}

__global__ void __launch_bounds__(256) arith_check(long long n, uint64_t seed) {
  unsigned w0 = 0, w1 = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed ^ (uint64_t)i * 0x2545F4914F6CDD1Dull);
    // x = m 2^e: mantissa bits random, exponent in [-30, 30]
    const float m = __int_as_float(0x3f800000 | (unsigned)(r & 0x7fffff));
    const int e = (int)((r >> 23) % 61) - 30;
    const float x = ldexpf(m, e);
    w0 = max(w0, ulp_dist(lbm::rcp_nr(x), __frcp_rn(x)));
    // quotient by the level denominators 4 (2 c1 + 1), c1 = 0 .. 15
    const float den = 4.0f * (float)(2 * (int)((r >> 40) & 15) + 1);
    const float num = ldexpf(m, (int)((r >> 44) % 41) - 20);
    w1 = max(w1, ulp_dist(lbm::div_markstein(num, den, lbm::rcp_nr(den)),
                          __fdiv_rn(num, den)));
  }
  w0 = __reduce_max_sync(0xffffffffu, w0);
  w1 = __reduce_max_sync(0xffffffffu, w1);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&g_worst[0], w0);
    atomicMax(&g_worst[1], w1);
  }
}

}  // namespace

extern "C" lbm_status lbm_check_fp32_arith(int64_t n, uint64_t seed,
                                           double worst_ulp[2], void* stream) {
  if (n < 0 || !worst_ulp) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned zero[2] = {0u, 0u};
  cudaError_t e = cudaMemcpyToSymbolAsync(g_worst, zero, sizeof(zero), 0,
                                          cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 0) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    arith_check<<<(unsigned)blocks, 256, 0, s>>>(n, seed);
    e = cudaGetLastError();
  }
  unsigned got[2] = {0u, 0u};
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(got, g_worst, sizeof(got), 0,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  worst_ulp[0] = (double)got[0];
  worst_ulp[1] = (double)got[1];
  return LBM_OK;
}
