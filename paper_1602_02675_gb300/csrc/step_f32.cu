// FP32 step kernels (compensated or plain summation of the row-pair sums).
#include "step_ds.cuh"
#include "step_kernel.cuh"

namespace lbm {
namespace ds {
// One grid's finalize launch: FIN_BLOCKS blocks (ds_finalize_part).
__global__ void __launch_bounds__(NTHR)
    finalize2d(Scratch* scr, double* __restrict__ part, int nblk,
               int do_cons) {
  ds_finalize_part(scr, part, nblk, do_cons, blockIdx.x);
}
}  // namespace ds

cudaError_t launch_step_f32(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s) {
  if (dim == 1) {
    const int tw = step_tile_1d(a.nx, device_sm_count());
    dim3 grid((a.nx + tw - 1) / tw, 1);
    const size_t sm32 = step_smem_bytes_t<float, 1, 32>(a.r_cap);
    const size_t sm16 = step_smem_bytes_t<float, 1, 16>(a.r_cap);
    if (tw == 16 && a.kahan)
      step_kernel<float, 1, true, 32, 16><<<grid, 32, sm16, s>>>(a);
    else if (tw == 16)
      step_kernel<float, 1, false, 32, 16><<<grid, 32, sm16, s>>>(a);
    else if (tw == 32 && a.kahan)
      step_kernel<float, 1, true, 32><<<grid, 32, sm32, s>>>(a);
    else if (tw == 32)
      step_kernel<float, 1, false, 32><<<grid, 32, sm32, s>>>(a);
    else if (a.kahan)
      step_kernel<float, 1, true><<<grid, 256, smem, s>>>(a);
    else
      step_kernel<float, 1, false><<<grid, 256, smem, s>>>(a);
  } else if (a.r_cap > ds::RMAX || a.exact_order) {
    // exact-order kernel: a reach limit beyond the deposit kernel's window,
    // or asked for (the allocation-free step, whose scratch holds this
    // kernel's per-tile partials)
    dim3 grid((a.nx + TileShape<2>::TX - 1) / TileShape<2>::TX,
              (a.ny + TileShape<2>::TY - 1) / TileShape<2>::TY);
    if (a.kahan)
      step_kernel<float, 2, true><<<grid, 256, smem, s>>>(a);
    else
      step_kernel<float, 2, false><<<grid, 256, smem, s>>>(a);
  } else {
    // deposit-and-shift kernel, plain or compensated gather: the grid holds
    // the tiles of the largest reach the handle allows; blocks beyond the
    // step's tile count exit
    StepArgs b = a;
    b.nblocks = ds::tiles_for(a.nx, a.ny, a.r_cap);
    if (!b.hint) return cudaErrorInvalidValue;
    // one persistent kernel, two blocks per multiprocessor
    int nb = 2 * device_sm_count();
    if (nb > b.nblocks) nb = b.nblocks;
    if (a.kahan)
      ds::step2d_ds_fused<true><<<(unsigned)nb, ds::NTHR, ds::smem_bytes(), s>>>(b);
    else
      ds::step2d_ds_fused<false><<<(unsigned)nb, ds::NTHR, ds::smem_bytes(), s>>>(b);
    ds::finalize2d<<<ds::FIN_BLOCKS, ds::NTHR, 0, s>>>(b.scr, b.part, b.nblocks,
                                                       b.do_cons);
  }
  return cudaGetLastError();
}

int ds_finalize_blocks() { return ds::FIN_BLOCKS; }

int ds_rmax() { return ds::RMAX; }

int ds_tiles(int nx, int ny, int r_cap) {
  return r_cap > ds::RMAX ? 0 : ds::tiles_for(nx, ny, r_cap);
}

size_t step_smem_f32(int dim, int r_cap) {
  if (dim == 1) return step_smem_bytes_t<float, 1>(r_cap);
  size_t g = step_smem_bytes_t<float, 2>(r_cap), f = ds::smem_bytes();
  return g > f ? g : f;
}

cudaError_t step_prepare_f32(int dim, size_t smem) {
  cudaError_t e;
  if (dim == 1) {
    const void* fns[6] = {(const void*)step_kernel<float, 1, true>,
                          (const void*)step_kernel<float, 1, false>,
                          (const void*)step_kernel<float, 1, true, 32>,
                          (const void*)step_kernel<float, 1, false, 32>,
                          (const void*)step_kernel<float, 1, true, 32, 16>,
                          (const void*)step_kernel<float, 1, false, 32, 16>};
    for (const void* fn : fns) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(step_kernel<float, 2, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_kernel<float, 2, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // two blocks per multiprocessor need the largest shared-memory carveout
  for (const void* fn : {(const void*)ds::step2d_ds_fused<false>,
                         (const void*)ds::step2d_ds_fused<true>}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ds::smem_bytes());
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lbm

namespace lbm {

// Raise (never lower) the dynamic shared-memory limit of the FP32 step
// kernels so a launch needing smem bytes is allowed.
cudaError_t step_raise_smem_f32(int dim, size_t smem) {
  const void* fns[6] = {
      dim == 1 ? (const void*)step_kernel<float, 1, true>
               : (const void*)step_kernel<float, 2, true>,
      dim == 1 ? (const void*)step_kernel<float, 1, false>
               : (const void*)step_kernel<float, 2, false>,
      dim == 1 ? (const void*)step_kernel<float, 1, true, 32>
               : (const void*)ds::step2d_ds_fused<true>,
      dim == 1 ? (const void*)step_kernel<float, 1, false, 32>
               : (const void*)ds::step2d_ds_fused<false>,
      dim == 1 ? (const void*)step_kernel<float, 1, true, 32, 16>
               : (const void*)ds::step2d_ds_fused<false>,
      dim == 1 ? (const void*)step_kernel<float, 1, false, 32, 16>
               : (const void*)ds::step2d_ds_fused<false>};
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
