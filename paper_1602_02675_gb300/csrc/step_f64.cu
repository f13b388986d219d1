// FP64 step kernels.  This unit is compiled with -fmad=false: every product
// and sum rounds on its own, in the same order the arithmetic is written, so
// the FP64 step reproduces a plain evaluation of the same formulas.
#include "step_rec.cuh"

namespace lbm {

cudaError_t launch_step_f64(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s) {
  if (dim == 1) {
    const int tw = step_tile_1d(a.nx, device_sm_count());
    dim3 grid((a.nx + tw - 1) / tw, 1);
    if (tw == 16)
      step_kernel<double, 1, false, 32, 16><<<grid, 32,
          step_smem_bytes_t<double, 1, 16>(a.r_cap), s>>>(a);
    else if (tw == 32)
      step_kernel<double, 1, false, 32><<<grid, 32,
          step_smem_bytes_t<double, 1, 32>(a.r_cap), s>>>(a);
    else
      step_kernel<double, 1, false><<<grid, 256, smem, s>>>(a);
  } else {
    dim3 grid((a.nx + TileShape<2>::TX - 1) / TileShape<2>::TX,
              (a.ny + TileShape<2>::TY - 1) / TileShape<2>::TY);
    if (a.src) {
      const long long PX = (long long)a.nx + 2 * a.r_cap;
      const long long PY = (long long)a.ny + 2 * a.r_cap;
      dim3 rgrid((unsigned)((PX + 255) / 256),
                 (unsigned)(PY < 65535 ? PY : 65535));
      records2d<double><<<rgrid, 256, 0, s>>>(a);
      step2d_rec<double, false><<<grid, 256, 0, s>>>(a);
    } else {
      step_kernel<double, 2, false><<<grid, 256, smem, s>>>(a);
    }
  }
  return cudaGetLastError();
}

size_t step_smem_f64(int dim, int r_cap) {
  return dim == 1 ? step_smem_bytes_t<double, 1>(r_cap)
                  : step_smem_bytes_t<double, 2>(r_cap);
}

cudaError_t step_prepare_f64(int dim, size_t smem) {
  if (dim == 1) {
    const void* fns[3] = {(const void*)step_kernel<double, 1, false, 32, 16>,
                          (const void*)step_kernel<double, 1, false, 32>,
                          (const void*)step_kernel<double, 1, false>};
    for (const void* fn : fns) {
      cudaError_t e = cudaFuncSetAttribute(
          fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return cudaFuncSetAttribute(step_kernel<double, 2, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

}  // namespace lbm

namespace lbm {

// Raise (never lower) the dynamic shared-memory limit of the FP64 step
// kernel so a launch needing smem bytes is allowed.
cudaError_t step_raise_smem_f64(int dim, size_t smem) {
  const void* fns[3] = {
      dim == 1 ? (const void*)step_kernel<double, 1, false>
               : (const void*)step_kernel<double, 2, false>,
      dim == 1 ? (const void*)step_kernel<double, 1, false, 32>
               : (const void*)step_kernel<double, 2, false>,
      dim == 1 ? (const void*)step_kernel<double, 1, false, 32, 16>
               : (const void*)step_kernel<double, 2, false>};
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
