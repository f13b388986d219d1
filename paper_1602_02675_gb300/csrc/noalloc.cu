// lbm_step_noalloc: one step between caller-owned device arrays that
// allocates nothing.  Contract: include/lbm.h.
//
// Some callers cannot call cudaMalloc at all: code running under an
// allocator they do not own, memory-budgeted services that pre-reserve
// everything up front, or real-time loops where an allocation can stall.
// This entry point serves them: its scratch words (the migration reach, the
// error flags, the last-block ticket and the FP64 partial sums of the step
// kernel) live in one file-scope device array that every GPU loading the
// library holds until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
cudaError_t step_raise_smem_f64(int dim, size_t smem);
cudaError_t step_raise_smem_f32(int dim, size_t smem);
}  // namespace lbm

using namespace lbm;

namespace {

// Header (Scratch words) padded to 256 bytes, then FP64 partial sums, four
// per tile of the step kernel.
constexpr size_t kHeader = 256;
constexpr size_t kScratchBytes = (size_t)LBM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxTiles = (int)((kScratchBytes - kHeader) / (4 * sizeof(double)));
static_assert(sizeof(Scratch) <= kHeader, "scratch header too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {nullptr};
// Context the cached address belongs to: a context torn down and created
// again (cudaDeviceReset) loads the module anew, so the address is looked
// up again when the current context changes.
CUcontext g_ctx[kMaxDevices] = {nullptr};

void set_err(char* err, size_t len, const char* msg) {
  if (err && len > 0) {
    std::snprintf(err, len, "%s", msg);
  }
}

void set_cuda_err(char* err, size_t len, const char* what, cudaError_t e) {
  if (err && len > 0)
    std::snprintf(err, len, "lbm_step_noalloc: %s: %s", what,
                  cudaGetErrorString(e));
}

// Current driver context (through the runtime's driver entry point, so the
// library needs no link against the driver library); nullptr if unknown.
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 get = nullptr;
  static bool tried = false;
  if (!tried) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000,
                                         cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    else
      cudaGetLastError();
    tried = true;
  }
  CUcontext c = nullptr;
  if (get && get(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch array on the current device.  The symbol's
// name in host code is only a host-side stand-in, so the address is taken
// with cudaGetSymbolAddress, once per device (and again if that device's
// context was replaced), with that device current.
cudaError_t scratch_on(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  const CUcontext ctx = current_context();
  if (g_ptr[dev] == nullptr || ctx == nullptr || ctx != g_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<unsigned char*>(p);
    g_ctx[dev] = ctx;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_noalloc_desc* d,
                                       const void* const in[4],
                                       void* const out[4], double* totals,
                                       int32_t* reach, uint32_t* flags,
                                       void* stream, char* err,
                                       size_t err_len) {
  set_err(err, err_len, "");
  if (!d || !in || !out) {
    set_err(err, err_len, "lbm_step_noalloc: NULL descriptor or array list");
    return LBM_EINVAL;
  }
  if ((d->dim != 1 && d->dim != 2) ||
      (d->precision != LBM_F32 && d->precision != LBM_F64) || d->nx < 1 ||
      d->ny < 1 || (d->dim == 1 && d->ny != 1) || d->nx > INT32_MAX ||
      d->ny > INT32_MAX || d->bc_x < 0 || d->bc_x > 2 ||
      (d->dim == 2 && (d->bc_y < 0 || d->bc_y > 2)) || !(d->gamma > 1.0) ||
      !std::isfinite(d->gamma) ||
      (d->dim == 1 && !(d->theta >= 0.0 && d->theta < 1.0)) ||
      (d->dim == 2 && d->theta != 0.0)) {
    set_err(err, err_len, "lbm_step_noalloc: invalid descriptor");
    return LBM_EINVAL;
  }
  if (!in[0] || !in[1] || !in[3] || !out[0] || !out[1] || !out[3] ||
      (d->dim == 2 && (!in[2] || !out[2]))) {
    set_err(err, err_len, "lbm_step_noalloc: NULL field array");
    return LBM_EINVAL;
  }
  const int nx = (int)d->nx, ny = (int)(d->dim == 2 ? d->ny : 1);
  // tile count in 64 bits, checked before anything is launched
  const long long tiles64 = step_blocks(d->dim, nx, ny);
  if (tiles64 > kMaxTiles) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "lbm_step_noalloc: %lld x %lld nodes need %lld tiles; the "
                  "static scratch holds at most %d (use lbm_create/lbm_step)",
                  (long long)d->nx, (long long)d->ny, tiles64, kMaxTiles);
    set_err(err, err_len, msg);
    return LBM_EINVAL;
  }
  const int tiles = (int)tiles64;
  const bool f64 = d->precision == LBM_F64;
  const int r_cap = d->dim == 1 ? 64 : 6;
  const size_t smem = step_smem_bytes(d->dim, f64, r_cap);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_err(err, err_len, "cudaGetDevice", e);
    return LBM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "lbm_step_noalloc: device ordinal out of range");
    return LBM_EINVAL;
  }
  unsigned char* base = nullptr;
  e = scratch_on(dev, &base);
  if (e != cudaSuccess) {
    set_cuda_err(err, err_len, "cudaGetSymbolAddress", e);
    return LBM_ECUDA;
  }
  e = f64 ? step_raise_smem_f64(d->dim, smem) : step_raise_smem_f32(d->dim, smem);
  if (e != cudaSuccess) {
    set_cuda_err(err, err_len, "kernel attribute", e);
    return LBM_ECUDA;
  }

  cudaStream_t s = (cudaStream_t)stream;
  Scratch* scr = reinterpret_cast<Scratch*>(base);
  double* part = reinterpret_cast<double*>(base + kHeader);

  EqConst k;
  const double D = (double)d->dim;
  k.theta = d->dim == 1 ? d->theta : 0.0;
  k.kq = D * (d->gamma - 1.0);
  k.kphi = 1.0 - 0.5 * D * (d->gamma - 1.0);
  k.b1 = d->dim == 1 ? 2.0 : 4.0;
  k.kreach = k.kq / (1.0 - k.theta);
  k.set_fp32_copies();

  // the array keeps the previous call's contents: start from zero
  e = cudaMemsetAsync(scr, 0, kHeader, s);
  void* fin[4] = {const_cast<void*>(in[0]), const_cast<void*>(in[1]),
                  const_cast<void*>(in[2]), const_cast<void*>(in[3])};
  if (e == cudaSuccess)
    e = launch_reach(f64, d->dim, fin, (int64_t)nx * ny, k, scr, s);
  if (e != cudaSuccess) {
    set_cuda_err(err, err_len, "reach kernel", e);
    return LBM_ECUDA;
  }
  StepArgs a;
  for (int f = 0; f < 4; ++f) {
    a.in[f] = in[f];
    a.out[f] = out[f];
  }
  a.nx = nx;
  a.ny = ny;
  a.bc_x = d->bc_x;
  a.bc_y = d->dim == 2 ? d->bc_y : 0;
  a.r_cap = r_cap;
  a.kahan = 1;
  a.exact_order = 1;
  a.do_cons = totals ? 1 : 0;
  a.nblocks = tiles;
  a.k = k;
  a.scr = scr;
  a.part = part;
  e = launch_step(d->dim, f64, a, smem, s);
  if (e == cudaSuccess && totals)
    e = cudaMemcpyAsync(totals, base + offsetof(Scratch, cons),
                        sizeof(double) * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && reach)
    e = cudaMemcpyAsync(reach, base + offsetof(Scratch, reach),
                        sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && flags)
    e = cudaMemcpyAsync(flags, base + offsetof(Scratch, flags),
                        sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    set_cuda_err(err, err_len, "step", e);
    return LBM_ECUDA;
  }
  return LBM_OK;
}
