// FP32 step kernels (compensated or plain summation of the row-pair sums).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

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
    const int tw = step_tile_1d(a.nx);
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
  } else if (a.kahan || a.r_cap > fast::RMAX || !a.rin_a || !a.rout_a ||
             !a.map_a || !a.map_b) {
    // exact-order kernel: compensated sums, large reach, or a caller
    // without equilibrium records
    dim3 grid((a.nx + TileShape<2>::TX - 1) / TileShape<2>::TX,
              (a.ny + TileShape<2>::TY - 1) / TileShape<2>::TY);
    if (a.kahan)
      step_kernel<float, 2, true><<<grid, 256, smem, s>>>(a);
    else
      step_kernel<float, 2, false><<<grid, 256, smem, s>>>(a);
  } else {
    // one block per tile (one partial-totals row each); blocks prefetch the
    // tile one resident wave ahead
    const long long tiles = (long long)((a.nx + fast::TX - 1) / fast::TX) *
                            ((a.ny + fast::TY - 1) / fast::TY);
    StepArgs b = a;
    b.nblocks = (int)tiles;
    b.prefetch_ahead = fast_resident_blocks();
    dim3 grid((unsigned)tiles, 1);
    // its own fixed layout: no more shared memory than that (occupancy)
    fast::step2d_f32<<<grid, fast::NTHR, fast::smem_bytes(), s>>>(b, *a.map_a,
                                                                  *a.map_b);
    fast::finalize2d_f32<<<1, fast::NTHR, 0, s>>>(b.scr, b.part, b.nblocks,
                                                  b.do_cons);
  }
  return cudaGetLastError();
}

bool step_uses_records(int dim, bool f64, int kahan, int r_cap) {
  return dim == 2 && !f64 && !kahan && r_cap <= fast::RMAX;
}

cudaError_t launch_records_f32(const void* const f[4], void* rec_a,
                               void* rec_b, int nx, int ny, int pitch,
                               const EqConst& k, cudaStream_t s) {
  const long long n = (long long)nx * ny;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  fast::records2d_f32<<<(unsigned)blocks, 256, 0, s>>>(
      static_cast<const float*>(f[0]), static_cast<const float*>(f[1]),
      static_cast<const float*>(f[2]), static_cast<const float*>(f[3]),
      static_cast<float4*>(rec_a), static_cast<float2*>(rec_b), nx, ny, pitch,
      (float)k.kq);
  return cudaGetLastError();
}

cudaError_t make_record_maps(void* rec_a, void* rec_b, int nx, int ny,
                             int pitch, TmaMap* map_a, TmaMap* map_b) {
  static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "tensor map size");
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion(
        "cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if ((pitch & 1) || pitch < nx) return cudaErrorInvalidValue;
  // rec_a: FP32 tensor 4 nx wide, rows of 16 pitch bytes; rec_b: 2 nx wide,
  // rows of 8 pitch bytes (a multiple of 16: pitch is even).  Boxes: the
  // window of reach RMAX around a 32 x 32 tile.
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)4 * nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)16 * pitch};
    const cuuint32_t box[2] = {(cuuint32_t)fast::BOX_A_W, (cuuint32_t)fast::HMAX};
    if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rec_a, dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    std::memcpy(map_a->bytes, &m, sizeof(m));
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)2 * nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)8 * pitch};
    const cuuint32_t box[2] = {(cuuint32_t)fast::BOX_B_W, (cuuint32_t)fast::HMAX};
    if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rec_b, dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    std::memcpy(map_b->bytes, &m, sizeof(m));
  }
  return cudaSuccess;
}

size_t step_smem_f32(int dim, int r_cap) {
  if (dim == 1) return step_smem_bytes_t<float, 1>(r_cap);
  size_t g = step_smem_bytes_t<float, 2>(r_cap), f = fast::smem_bytes();
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
  e = cudaFuncSetAttribute(fast::step2d_f32,
                           cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fast::step2d_f32,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
               : (const void*)fast::step2d_f32,
      dim == 1 ? (const void*)step_kernel<float, 1, false, 32>
               : (const void*)fast::step2d_f32,
      dim == 1 ? (const void*)step_kernel<float, 1, true, 32, 16>
               : (const void*)fast::step2d_f32,
      dim == 1 ? (const void*)step_kernel<float, 1, false, 32, 16>
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
