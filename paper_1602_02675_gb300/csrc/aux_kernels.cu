// Initial states, unit conversion at the host boundary, reach seeding and
// FP64 totals.  Compiled with -fmad=false like the FP64 step, so the unit
// conversions round exactly as their formulas are written.
#include <atomic>

#include "step_kernel.cuh"

namespace lbm {

size_t step_smem_f64(int dim, int r_cap);
size_t step_smem_f32(int dim, int r_cap);
cudaError_t step_prepare_f64(int dim, size_t smem);
cudaError_t step_prepare_f32(int dim, size_t smem);
cudaError_t launch_step_f64(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s);
cudaError_t launch_step_f32(int dim, const StepArgs& a, size_t smem,
                            cudaStream_t s);

int device_sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess ||
      v < 1) {
    cudaGetLastError();
    return 1;
  }
  cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

size_t step_smem_bytes(int dim, bool f64, int r_cap) {
  return f64 ? step_smem_f64(dim, r_cap) : step_smem_f32(dim, r_cap);
}

cudaError_t step_prepare(int dim, bool f64, size_t smem) {
  return f64 ? step_prepare_f64(dim, smem) : step_prepare_f32(dim, smem);
}

long long step_blocks(int dim, int nx, int ny) {
  const long long X = nx, Y = ny;
  if (dim == 1) {
    const long long tw = step_tile_1d(nx, device_sm_count());
    return (X + tw - 1) / tw;
  }
  return ((X + TileShape<2>::TX - 1) / TileShape<2>::TX) *
         ((Y + TileShape<2>::TY - 1) / TileShape<2>::TY);
}

cudaError_t launch_step(int dim, bool f64, const StepArgs& a, size_t smem,
                        cudaStream_t s) {
  return f64 ? launch_step_f64(dim, a, smem, s) : launch_step_f32(dim, a, smem, s);
}

// Lattice moments of a primitive state: V = u lambda, m = rho V,
// rhoE = p lambda^2/(gamma - 1) + rho |V|^2 / 2.
template <typename T>
__device__ __forceinline__ void prim_to_lattice(int dim, double rho, double u,
                                                double v, double p, double lam,
                                                double gamma, T* out) {
  double Vx = u * lam;
  double Vy = v * lam;
  double kin = (dim == 2) ? Vx * Vx + Vy * Vy : Vx * Vx;
  double rhoE = p * lam * lam / (gamma - 1.0) + 0.5 * rho * kin;
  out[0] = (T)rho;
  out[1] = (T)(rho * Vx);
  out[2] = (T)(rho * Vy);
  out[3] = (T)rhoE;
}

template <typename T>
__global__ void init_kernel(const InitArgs a) {
  long long n = (long long)a.nx * a.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int ix = (int)(i % a.nx);
    int iy = (int)(i / a.nx);
    double x = a.x0 + ((double)ix + 0.5) * a.dx;
    double y = a.y0 + ((double)iy + 0.5) * a.dx;
    bool inside;
    if (a.geom == 0) {
      inside = x < a.a0;
    } else {
      double r2 = (x - a.a0) * (x - a.a0) + (y - a.a1) * (y - a.a1);
      inside = r2 < a.radius * a.radius;
    }
    const double* s = inside ? a.in_ : a.out_;
    T o[4];
    prim_to_lattice<T>(a.dim, s[0], s[1], s[2], s[3], a.lambda, a.gamma, o);
    reinterpret_cast<T*>(a.f[0])[i] = o[0];
    reinterpret_cast<T*>(a.f[1])[i] = o[1];
    if (a.dim == 2) reinterpret_cast<T*>(a.f[2])[i] = o[2];
    reinterpret_cast<T*>(a.f[3])[i] = o[3];
  }
}

cudaError_t launch_init(bool f64, const InitArgs& a, cudaStream_t s) {
  long long n = (long long)a.nx * a.ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 32) blocks = device_sm_count() * 32;
  if (f64)
    init_kernel<double><<<blocks, 256, 0, s>>>(a);
  else
    init_kernel<float><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
__global__ void from_host_kernel(int kind, int dim, const double* st,
                                 T* f0, T* f1, T* f2, T* f3, long long n,
                                 double lam, double gamma) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double a = st[i], b = st[n + i], c = (dim == 2) ? st[2 * n + i] : 0.0,
           d = st[3 * n + i];
    T o[4];
    if (kind == 0) {
      prim_to_lattice<T>(dim, a, b, c, d, lam, gamma, o);
    } else {  // physical conserved -> lattice: m lambda, rhoE lambda^2
      o[0] = (T)a;
      o[1] = (T)(b * lam);
      o[2] = (T)(c * lam);
      o[3] = (T)(d * lam * lam);
    }
    f0[i] = o[0];
    f1[i] = o[1];
    if (dim == 2) f2[i] = o[2];
    f3[i] = o[3];
  }
}

cudaError_t launch_from_host_layout(bool f64, int kind, int dim,
                                    const double* staging, void* const f[4],
                                    int64_t n, double lambda, double gamma,
                                    cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 32) blocks = device_sm_count() * 32;
  if (f64)
    from_host_kernel<double><<<blocks, 256, 0, s>>>(
        kind, dim, staging, (double*)f[0], (double*)f[1], (double*)f[2],
        (double*)f[3], n, lambda, gamma);
  else
    from_host_kernel<float><<<blocks, 256, 0, s>>>(
        kind, dim, staging, (float*)f[0], (float*)f[1], (float*)f[2],
        (float*)f[3], n, lambda, gamma);
  return cudaGetLastError();
}

// Lattice moments -> physical rho, m/lambda, rhoE/lambda^2 and the pressure
// P = (gamma - 1)(rhoE - |m|^2/(2 rho)) (eq 27), all in FP64.
template <typename T>
__global__ void to_host_kernel(int dim, const T* f0, const T* f1, const T* f2,
                               const T* f3, double* st, long long n,
                               double lam, double gamma) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double rho = (double)f0[i];
    double mx = (double)f1[i] / lam;
    double my = (dim == 2) ? (double)f2[i] / lam : 0.0;
    double rhoE = (double)f3[i] / (lam * lam);
    double kin = (dim == 2) ? mx * mx + my * my : mx * mx;
    double p = (gamma - 1.0) * (rhoE - 0.5 * kin / rho);
    st[i] = rho;
    st[n + i] = mx;
    st[2 * n + i] = my;
    st[3 * n + i] = rhoE;
    st[4 * n + i] = p;
  }
}

cudaError_t launch_to_host_layout(bool f64, int dim, const void* const f[4],
                                  double* staging, int64_t n, double lambda,
                                  double gamma, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 32) blocks = device_sm_count() * 32;
  if (f64)
    to_host_kernel<double><<<blocks, 256, 0, s>>>(
        dim, (const double*)f[0], (const double*)f[1], (const double*)f[2],
        (const double*)f[3], staging, n, lambda, gamma);
  else
    to_host_kernel<float><<<blocks, 256, 0, s>>>(
        dim, (const float*)f[0], (const float*)f[1], (const float*)f[2],
        (const float*)f[3], staging, n, lambda, gamma);
  return cudaGetLastError();
}

template <typename T>
__global__ void reach_kernel(int dim, const T* f0, const T* f1, const T* f2,
                             const T* f3, long long n, float kreach,
                             Scratch* scr) {
  int r = 0;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double rho = (double)f0[i], mx = (double)f1[i];
    double my = (dim == 2) ? (double)f2[i] : 0.0, rE = (double)f3[i];
    if (!isfinite(rho) || !isfinite(mx) || !isfinite(my) || !isfinite(rE) ||
        rho < 0.0)
      bad = true;
    r = max(r, reach_bound(rho, mx, my, rE, kreach));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    r = max(r, __shfl_xor_sync(0xffffffffu, r, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&scr->reach, r);
  if (bad) atomicOr(&scr->flags, kFlagState);
}

cudaError_t launch_reach(bool f64, int dim, const void* const f[4], int64_t n,
                         const EqConst& k, Scratch* scr, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&scr->reach, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int blocks = (int)((n + 255) / 256);
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  if (f64)
    reach_kernel<double><<<blocks, 256, 0, s>>>(
        dim, (const double*)f[0], (const double*)f[1], (const double*)f[2],
        (const double*)f[3], n, (float)k.kreach, scr);
  else
    reach_kernel<float><<<blocks, 256, 0, s>>>(
        dim, (const float*)f[0], (const float*)f[1], (const float*)f[2],
        (const float*)f[3], n, (float)k.kreach, scr);
  return cudaGetLastError();
}

// FP64 totals: each block sums a fixed slice (grid-stride, fixed tree), the
// partials are then summed by one block in block order.
constexpr int kTotThreads = 256;

int totals_blocks(int64_t n) {
  long long b = (n + kTotThreads - 1) / kTotThreads;
  const long long cap = 8LL * device_sm_count();
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T>
__global__ void totals_partial(int dim, const T* f0, const T* f1, const T* f2,
                               const T* f3, long long n, double* part) {
  __shared__ double red[4][kTotThreads / 32];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    s[0] += (double)f0[i];
    s[1] += (double)f1[i];
    if (dim == 2) s[2] += (double)f2[i];
    s[3] += (double)f3[i];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      s[f] += __shfl_down_sync(0xffffffffu, s[f], off);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
    for (int f = 0; f < 4; ++f) red[f][w] = s[f];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int f = 0; f < 4; ++f) {
      double t = red[f][0];
      for (int k = 1; k < kTotThreads / 32; ++k) t += red[f][k];
      part[blockIdx.x * 4 + f] = t;
    }
  }
}

__global__ void totals_final(const double* part, int nb, Scratch* scr) {
  if (threadIdx.x != 0) return;
  for (int f = 0; f < 4; ++f) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b * 4 + f];
    scr->cons[f] = t;
  }
}

cudaError_t launch_totals(bool f64, int dim, const void* const f[4], int64_t n,
                          double* part, int nblocks_cap, Scratch* scr,
                          cudaStream_t s) {
  int nb = totals_blocks(n);
  if (nb > nblocks_cap) nb = nblocks_cap;
  if (f64)
    totals_partial<double><<<nb, kTotThreads, 0, s>>>(
        dim, (const double*)f[0], (const double*)f[1], (const double*)f[2],
        (const double*)f[3], n, part);
  else
    totals_partial<float><<<nb, kTotThreads, 0, s>>>(
        dim, (const float*)f[0], (const float*)f[1], (const float*)f[2],
        (const float*)f[3], n, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  totals_final<<<1, 32, 0, s>>>(part, nb, scr);
  return cudaGetLastError();
}

}  // namespace lbm
