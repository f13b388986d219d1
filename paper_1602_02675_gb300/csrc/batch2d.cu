// Batched small 2-D grids: many independent square-lattice grids advanced
// together by the deposit kernel (step_ds.cuh), two launches per lattice
// step for the whole batch instead of two per grid.  Contract:
// include/lbm.h.
//
// Each grid is an ordinary FP32 square-lattice handle (its own buffers,
// per-tile records, partial totals and scratch); the batch adds a table of
// the grids' step arguments for both state parities and the first tile of
// each grid in one batch-wide tile numbering.  The persistent deposit
// kernel's blocks take batch tiles by ticket and find each tile's grid from
// its number; the finalize kernel runs FIN_BLOCKS blocks per grid.
// A grid that has taken its steps is left as it is.  Every grid's tiles do
// exactly what lbm_step does on that grid's handle, so its results are the
// same bit for bit.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "step_ds.cuh"

using namespace lbm;

namespace {

struct B2Args {
  const StepArgs* args;     // grid g from state parity p at [2 g + p]
  const int* tile_base;     // [ngrids + 1]: first batch tile of each grid
  const long long* nsteps;  // [ngrids]
  const int* cons_every;    // [ngrids]
  int ngrids;
  long long step;           // the batch step this launch takes
  unsigned* q;              // [2]: unused, tiles taken
};

// Largest g with tile_base[g] <= item.
__device__ __forceinline__ int grid_of(const int* base, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Whether grid g still takes this batch step.
__device__ __forceinline__ bool grid_active(const B2Args& B, int g) {
  return B.step < __ldg(B.nsteps + g);
}
// Step arguments of grid g at this batch step, copied by the whole block
// into the block's shared copy (the tile code reads them from there rather
// than holding them in registers).  All threads call it.
__device__ __forceinline__ const StepArgs& grid_args(const B2Args& B, int g,
                                                     unsigned* raw) {
  constexpr int W = (int)(sizeof(StepArgs) / sizeof(unsigned));
  static_assert(sizeof(StepArgs) % sizeof(unsigned) == 0, "word copy");
  __syncthreads();  // the previous tile is done with the copy
  const unsigned* src = reinterpret_cast<const unsigned*>(
      B.args + 2 * g + (int)(B.step & 1));
  for (int i = threadIdx.x; i < W; i += blockDim.x) raw[i] = src[i];
  __syncthreads();
  StepArgs& a = *reinterpret_cast<StepArgs*>(raw);
  if (threadIdx.x == 0) {
    const int every = __ldg(B.cons_every + g);
    a.do_cons = (every > 0 && ((B.step + 1) % every) == 0) ? 1 : 0;
  }
  __syncthreads();
  return a;
}

// The whole batch step in one persistent kernel: blocks take batch tiles by
// ticket (the next one taken ahead) and finish each in the same block, the
// one-type walk first and the group walks when the window is mixed.
template <bool KAHAN>
__global__ void __launch_bounds__(ds::NTHR, 2) b2_fused(const B2Args B,
                                                        int total) {
  extern __shared__ __align__(16) float4 dsm[];
  __shared__ int red[ds::NGSTAT * ds::NWARP];
  __shared__ ds::TileRed tred;
  __shared__ int s_k[2];
  __shared__ __align__(16) unsigned raw[sizeof(StepArgs) / sizeof(unsigned)];
  const ds::DsSmem sm{dsm, dsm + ds::PLANE,
                      reinterpret_cast<float*>(dsm + 2 * ds::PLANE), red,
                      &tred};
  if (threadIdx.x == 0) s_k[0] = (int)atomicAdd(&B.q[1], 1u);
  for (int it = 0;; ++it) {
    __syncthreads();  // the ticket is visible; the last tile is done
    const int item = s_k[it & 1];
    if (item >= total) break;
    if (threadIdx.x == 0) s_k[(it + 1) & 1] = (int)atomicAdd(&B.q[1], 1u);
    const int g = grid_of(B.tile_base, B.ngrids, item);
    if (!grid_active(B, g)) continue;
    const StepArgs& a = grid_args(B, g, raw);
    const int b = item - __ldg(B.tile_base + g);
    if (ds::ds_first_tile<KAHAN>(a, b, sm)) {
      __syncthreads();  // the walk's deposits and record are settled
      ds::ds_mixed_tile<KAHAN>(a, b, sm);
    }
  }
}

__global__ void __launch_bounds__(ds::NTHR) b2_finalize(const B2Args B) {
  // the queue is empty again for the next step (the mixed-window kernel
  // has finished)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.q[0] = 0u;
    B.q[1] = 0u;
  }
  __shared__ __align__(16) unsigned raw[sizeof(StepArgs) / sizeof(unsigned)];
  const int g = blockIdx.x / ds::FIN_BLOCKS, j = blockIdx.x % ds::FIN_BLOCKS;
  if (!grid_active(B, g)) return;
  const StepArgs& a = grid_args(B, g, raw);
  ds::ds_finalize_part(a.scr, a.part, a.nblocks, a.do_cons, j);
}

}  // namespace

struct lbm_batch2d {
  cudaStream_t stream = nullptr;
  std::vector<lbm_handle*> h;
  std::vector<long long> nsteps;
  int kahan = 0;
  int total_tiles = 0;
  long long step = 0, last = 0;
  StepArgs* d_args = nullptr;
  int* d_base = nullptr;
  long long* d_nsteps = nullptr;
  int* d_every = nullptr;
  unsigned* d_q = nullptr;
  bool broken = false;
  std::string err;
};

namespace {

lbm_status b2fail(lbm_batch2d* b, lbm_status st, const std::string& m) {
  if (b) {
    b->err = m;
    if (st != LBM_EINVAL) b->broken = true;
  }
  return st;
}

lbm_status b2cuda(lbm_batch2d* b, cudaError_t e, const char* what) {
  return b2fail(b, LBM_ECUDA,
                std::string("lbm_batch2d: ") + what + ": " +
                    cudaGetErrorString(e));
}

void b2free(lbm_batch2d* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  cudaFree(b->d_args);
  cudaFree(b->d_base);
  cudaFree(b->d_nsteps);
  cudaFree(b->d_every);
  cudaFree(b->d_q);
  for (lbm_handle* h : b->h) lbm_destroy(h);
  b->h.clear();
}

}  // namespace

lbm_status lbm_batch2d_create(const lbm_grid2d* grids, int32_t count,
                              void* stream, lbm_batch2d** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!grids || count < 1) return LBM_EINVAL;
  for (int g = 0; g < count; ++g) {
    const lbm_config& c = grids[g].cfg;
    if (c.dim != 2 || c.precision != LBM_F32 || c.max_reach < 0 ||
        c.max_reach > ds_rmax() || grids[g].nsteps < 0 ||
        (c.kahan ? 1 : 0) != (grids[0].cfg.kahan ? 1 : 0))
      return LBM_EINVAL;
  }
  lbm_batch2d* b = new (std::nothrow) lbm_batch2d;
  if (!b) return LBM_ENOMEM;
  b->stream = static_cast<cudaStream_t>(stream);
  b->kahan = grids[0].cfg.kahan ? 1 : 0;
  std::vector<StepArgs> args(2 * (size_t)count);
  std::vector<int> base(count + 1, 0), every(count);
  for (int g = 0; g < count; ++g) {
    lbm_config c = grids[g].cfg;
    c.stream = stream;
    lbm_handle* h = nullptr;
    lbm_status st = lbm_create(&c, &h);
    if (st != LBM_OK) {
      b2free(b);
      delete b;
      return st;
    }
    b->h.push_back(h);
    st = lbm_init_riemann(h, &grids[g].inner, &grids[g].outer, grids[g].geom,
                          grids[g].a0, grids[g].a1, grids[g].radius);
    if (st != LBM_OK || !handle_ds_args(h, 0, &args[2 * g]) ||
        !handle_ds_args(h, 1, &args[2 * g + 1])) {
      b2free(b);
      delete b;
      return st != LBM_OK ? st : LBM_EINVAL;
    }
    b->nsteps.push_back(grids[g].nsteps);
    b->last = std::max(b->last, (long long)grids[g].nsteps);
    every[g] = handle_cons_every(h);
    base[g + 1] = base[g] + args[2 * g].nblocks;
  }
  b->total_tiles = base[count];
  cudaError_t e = cudaSuccess;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(reinterpret_cast<void**>(&b->d_args), args.data(),
     sizeof(StepArgs) * args.size());
  up(reinterpret_cast<void**>(&b->d_base), base.data(), sizeof(int) * base.size());
  up(reinterpret_cast<void**>(&b->d_nsteps), b->nsteps.data(),
     sizeof(long long) * b->nsteps.size());
  up(reinterpret_cast<void**>(&b->d_every), every.data(), sizeof(int) * every.size());
  const unsigned zero[2] = {0u, 0u};
  up(reinterpret_cast<void**>(&b->d_q), zero, sizeof(zero));
  const int smem = (int)ds::smem_bytes();
  const void* fns[2] = {(const void*)b2_fused<false>, (const void*)b2_fused<true>};
  for (const void* fn : fns)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem);
  if (e != cudaSuccess) {
    const lbm_status st = b2cuda(b, e, "create");
    b2free(b);
    delete b;
    return st;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch2d_run(lbm_batch2d* b, int64_t max_steps) {
  if (!b) return LBM_EINVAL;
  if (b->broken) return b2fail(b, LBM_ECUDA, "lbm_batch2d: in an error state: " + b->err);
  long long todo = b->last - b->step;
  if (max_steps >= 0 && max_steps < todo) todo = max_steps;
  if (todo <= 0) return LBM_OK;
  B2Args B{b->d_args, b->d_base, b->d_nsteps, b->d_every, (int)b->h.size(),
           0, b->d_q};
  const size_t smem = ds::smem_bytes();
  int nb = 2 * device_sm_count();
  if (nb > b->total_tiles) nb = b->total_tiles;
  const unsigned nfin = (unsigned)(ds::FIN_BLOCKS * b->h.size());
  const long long s0 = b->step;
  for (long long s = 0; s < todo; ++s) {
    B.step = s0 + s;
    if (b->kahan)
      b2_fused<true><<<(unsigned)nb, ds::NTHR, smem, b->stream>>>(B, b->total_tiles);
    else
      b2_fused<false><<<(unsigned)nb, ds::NTHR, smem, b->stream>>>(B, b->total_tiles);
    b2_finalize<<<nfin, ds::NTHR, 0, b->stream>>>(B);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return b2cuda(b, e, "step launches");
  b->step = s0 + todo;
  for (size_t g = 0; g < b->h.size(); ++g) {
    const long long done = std::min(b->step, b->nsteps[g]) - std::min(s0, b->nsteps[g]);
    if (done > 0) handle_took_steps(b->h[g], done);
  }
  return LBM_OK;
}

lbm_status lbm_batch2d_steps(const lbm_batch2d* b, int64_t* steps) {
  if (!b || !steps) return LBM_EINVAL;
  *steps = b->step;
  return LBM_OK;
}

lbm_status lbm_batch2d_moments(lbm_batch2d* b, int32_t grid, double* rho,
                               double* mx, double* my, double* rhoE,
                               double* p, int64_t n) {
  if (!b || grid < 0 || grid >= (int32_t)b->h.size()) return LBM_EINVAL;
  const lbm_status st = lbm_moments(b->h[grid], rho, mx, my, rhoE, p, n);
  if (st != LBM_OK) {
    const char* m = lbm_last_error(b->h[grid]);
    b2fail(b, st, std::string("grid ") + std::to_string(grid) + ": " + (m ? m : ""));
  }
  return st;
}

const char* lbm_batch2d_last_error(const lbm_batch2d* b) {
  return b ? b->err.c_str() : "lbm_batch2d: NULL handle";
}

void lbm_batch2d_destroy(lbm_batch2d* b) {
  if (!b) return;
  b2free(b);
  delete b;
}
