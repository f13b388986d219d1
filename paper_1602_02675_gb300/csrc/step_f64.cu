// FP64 step kernels.  This unit is compiled with -fmad=false: every product
// and sum rounds on its own, in the same order the arithmetic is written, so
// the FP64 step reproduces a plain evaluation of the same formulas.
#include "step_kernel.cuh"

namespace lbm {

// FP64 square lattice: the source records of the input state (one thread
// per node), written before each step; energy clamps and bad states are
// counted here, once per node.
__global__ void __launch_bounds__(256) records2d_f64(const StepArgs a) {
  const long long n = (long long)a.nx * a.ny;
  double* Sr = a.src64;
  unsigned long long clamps = 0;
  bool bad = false;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x) {
    const Equil<double> q =
        equilibrium<double, 2>(ld<double>(a.in[0], g), ld<double>(a.in[1], g),
                               ld<double>(a.in[2], g), ld<double>(a.in[3], g),
                               a.k);
    clamps += q.clamp ? 1 : 0;
    bad |= q.bad;
    long long w = s64_word(-1, 0, 0);
    if (q.emits) {
#pragma unroll
      for (int p = 0; p < TileShape<2>::NP; ++p) {
        double px, py, pe;
        packet_fields<double, 2>(q, p, &px, &py, &pe);
        Sr[(kS64Px + p) * n + g] = px;
        Sr[(kS64Py + p) * n + g] = py;
        Sr[(kS64PE + p) * n + g] = pe;
      }
      Sr[kS64Mass * n + g] = q.d1;
      Sr[(kS64Mass + 1) * n + g] = q.d2;
      double w4[4];
      corner_weights(q, w4);
#pragma unroll
      for (int k = 0; k < 4; ++k) Sr[(kS64W + k) * n + g] = w4[k];
      Sr[kS64V * n + g] = q.V0;
      Sr[(kS64V + 1) * n + g] = q.V1;
      Sr[kS64Phi * n + g] = q.phi;
      w = s64_word(q.c1, q.n0, q.n1);
    }
    reinterpret_cast<long long*>(Sr + kS64Word * n)[g] = w;
  }
  const unsigned long long wc = __reduce_add_sync(0xffffffffu, (unsigned)clamps);
  const bool wb = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (wc) atomicAdd(&a.scr->eclamps, wc);
    if (wb) atomicOr(&a.scr->flags, kFlagState);
  }
}

cudaError_t launch_step_f64(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s) {
  if (dim == 1) {
    const int tw = step_tile_1d(a.nx);
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
    if (a.src64) {
      const long long n = (long long)a.nx * a.ny;
      const long long nb = (n + 255) / 256;
      records2d_f64<<<(unsigned)(nb < 152 * 16 ? nb : 152 * 16), 256, 0, s>>>(a);
    }
    dim3 grid((a.nx + TileShape<2>::TX - 1) / TileShape<2>::TX,
              (a.ny + TileShape<2>::TY - 1) / TileShape<2>::TY);
    step_kernel<double, 2, false><<<grid, 256, smem, s>>>(a);
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
