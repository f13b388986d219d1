// Fused multiply-add throughput of the device, FP32 and FP64: the ALU
// roof against which the step kernels' arithmetic is reported.  Declared in
// include/lbm.h (lbm_measure_fma_peak).
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// Sink for the chains' results: written only if their sum equals a value it
// never takes, so the loop is kept without storing anything.
__device__ double g_fma_sink;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == (T)-1.0) g_fma_sink = (double)s;
}

template <typename T>
cudaError_t time_chains(int iters, int blocks, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = -1.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    fma_chains<T><<<blocks, 256, 0, s>>>(iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best < 0.0f || t < best)) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return e;
}

}  // namespace

extern "C" lbm_status lbm_measure_fma_peak(int32_t precision,
                                           double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != LBM_F32 && precision != LBM_F64))
    return LBM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess)
    return LBM_ECUDA;
  const int blocks = sms * 8;
  const int iters = precision == LBM_F32 ? 8192 : 256;
  float ms = 0.0f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = precision == LBM_F32
                            ? time_chains<float>(iters, blocks, s, &ms)
                            : time_chains<double>(iters, blocks, s, &ms);
  if (e != cudaSuccess || !(ms > 0.0f)) return LBM_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * 256.0;
  *flops_per_s = flops / (ms * 1e-3);
  return LBM_OK;
}
