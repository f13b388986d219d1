// FP32 step kernels (compensated or plain summation of the row-pair sums).
#include "step_fast_f32.cuh"
#include "step_kernel.cuh"

namespace lbm {

namespace {

// Blocks of the register kernel resident on the whole device at once
// (occupancy x multiprocessors), per device, or 0 if the query fails.
int fast_resident_blocks() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cached[dev] == 0) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, fast::step2d_f32, fast::NTHR, fast::smem_bytes()) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cached[dev] = per_sm * sms > 0 ? per_sm * sms : -1;
  }
  return cached[dev] > 0 ? cached[dev] : 0;
}

}  // namespace

cudaError_t launch_step_f32(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s) {
  if (dim == 1) {
    dim3 grid((a.nx + TileShape<1>::TX - 1) / TileShape<1>::TX, 1);
    if (a.kahan)
      step_kernel<float, 1, true><<<grid, 256, smem, s>>>(a);
    else
      step_kernel<float, 1, false><<<grid, 256, smem, s>>>(a);
  } else if (a.kahan || a.r_cap > fast::RMAX || !a.rin_a || !a.rout_a) {
    // exact-order kernel: compensated sums, large reach, or a caller
    // without equilibrium records
    dim3 grid((a.nx + TileShape<2>::TX - 1) / TileShape<2>::TX,
              (a.ny + TileShape<2>::TY - 1) / TileShape<2>::TY);
    if (a.kahan)
      step_kernel<float, 2, true><<<grid, 256, smem, s>>>(a);
    else
      step_kernel<float, 2, false><<<grid, 256, smem, s>>>(a);
  } else {
    dim3 grid((a.nx + fast::TX - 1) / fast::TX, (a.ny + fast::TY - 1) / fast::TY);
    StepArgs b = a;  // the last-block ticket counts this kernel's tiles
    b.nblocks = (int)(grid.x * grid.y);
    b.prefetch_ahead = fast_resident_blocks();
    // its own fixed layout: no more shared memory than that (occupancy)
    fast::step2d_f32<<<grid, fast::NTHR, fast::smem_bytes(), s>>>(b);
    fast::finalize2d_f32<<<1, fast::NTHR, 0, s>>>(b.scr, b.part, b.nblocks,
                                                  b.do_cons);
  }
  return cudaGetLastError();
}

bool step_uses_records(int dim, bool f64, int kahan, int r_cap) {
  return dim == 2 && !f64 && !kahan && r_cap <= fast::RMAX;
}

cudaError_t launch_records_f32(const void* const f[4], void* rec_a,
                               void* rec_b, int64_t n, const EqConst& k,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  fast::records2d_f32<<<(unsigned)blocks, 256, 0, s>>>(
      static_cast<const float*>(f[0]), static_cast<const float*>(f[1]),
      static_cast<const float*>(f[2]), static_cast<const float*>(f[3]),
      static_cast<float4*>(rec_a), static_cast<float2*>(rec_b), (long long)n,
      (float)k.kq);
  return cudaGetLastError();
}

size_t step_smem_f32(int dim, int r_cap) {
  if (dim == 1) return step_smem_bytes_t<float, 1>(r_cap);
  size_t g = step_smem_bytes_t<float, 2>(r_cap), f = fast::smem_bytes();
  return g > f ? g : f;
}

cudaError_t step_prepare_f32(int dim, size_t smem) {
  cudaError_t e;
  if (dim == 1) {
    e = cudaFuncSetAttribute(step_kernel<float, 1, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(step_kernel<float, 1, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  e = cudaFuncSetAttribute(step_kernel<float, 2, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<float, 2, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fast::step2d_f32,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace lbm

namespace lbm {

// Raise (never lower) the dynamic shared-memory limit of the FP32 step
// kernels so a launch needing smem bytes is allowed.
cudaError_t step_raise_smem_f32(int dim, size_t smem) {
  const void* fns[3] = {
      dim == 1 ? (const void*)step_kernel<float, 1, true>
               : (const void*)step_kernel<float, 2, true>,
      dim == 1 ? (const void*)step_kernel<float, 1, false>
               : (const void*)step_kernel<float, 2, false>,
      dim == 1 ? (const void*)step_kernel<float, 1, false>
               : (const void*)fast::step2d_f32};
  for (const void* fn : fns) {
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)at.maxDynamicSharedSizeBytes >= smem) continue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lbm
