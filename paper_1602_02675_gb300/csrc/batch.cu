// Batched 1-D tubes: many independent shock tubes of different lengths and
// step counts advanced together, one persistent kernel launch per step,
// launches replayed from captured CUDA graphs.  Contract: include/lbm.h.
//
// Layout: every tube's nodes are concatenated (tube after tube) in one SoA
// buffer of three fields (rho, m, rhoE), two ping-pong copies.  Tubes are
// ordered by decreasing step count, so at global step s the tubes still
// running are a prefix, and so are their work items (tube, tile of TW nodes):
// the kernel reads how many items are active from a table indexed by the
// device step counter.  Each item runs the 1-D tau = 1 step of its tile with
// the same arithmetic and summation order as the single-tube step kernel
// (Section III.B eqs 13-15, 24-26; Section IV.A; eqs 6, 10, 22, 28; Section
// V.B boundaries).  A tube that has taken its steps keeps its last state.
//
// Tile width: lbm_batch_create times a few real steps of the batch with each
// candidate width (kTileChoices) and keeps the fastest (an autotuner over
// the tile shape of this batch); the state is then reset to the initial
// one.  The result does not depend on the width: every destination sums its
// arrivals in the same order.  The shared-memory halo is sized for the
// maximum reach (64) rather than tuned: a halo tuned below the reach a later
// step meets would end the run with LBM_EREACH.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "step_kernel.cuh"
#include "tile1d.cuh"

namespace lbm {
namespace batch {

constexpr int TILE = kTile1d;              // block size of the helper kernels
constexpr int kTileChoices[3] = {128, 256, 512};

struct Tube {
  long long off;     // first node in the concatenated buffers
  int n;             // nodes
  int nsteps;        // steps this tube takes
  int bc;            // boundary rule at both ends
  int pad_;
};

struct Args {
  const void* cur[3];  // fields of the state before the step (per parity)
  void* nxt[3];
  void* f0[3];         // buffers of parity 0 / 1
  void* f1[3];
  const Tube* tubes;
  const int2* items;   // (tube, tile) in tube order
  const int* active;   // active item count per step
  int* reach;          // [3][ntubes] triple-buffered per-tube reach
  int ntubes;
  int max_steps;
  int r_cap;
  int kahan;
  EqConst k;
  int* step;           // device step counter
  unsigned* ticket;
  unsigned* flags;
  unsigned long long* eclamps;
};

template <typename T, bool KAHAN, int TW>
__global__ void __launch_bounds__(TW) batch_step(const Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int is_last;
  const int s = *a.step;
  if (s >= a.max_steps) return;  // every tube has finished
  const int nact = a.active[s];
  const int par = s & 1;
  const T* in0 = (const T*)(par ? a.f1[0] : a.f0[0]);
  const T* in1 = (const T*)(par ? a.f1[1] : a.f0[1]);
  const T* in2 = (const T*)(par ? a.f1[2] : a.f0[2]);
  T* o0 = (T*)(par ? a.f0[0] : a.f1[0]);
  T* o1 = (T*)(par ? a.f0[1] : a.f1[1]);
  T* o2 = (T*)(par ? a.f0[2] : a.f1[2]);
  int* rcur = a.reach + (s % 3) * a.ntubes;
  int* rnext = a.reach + ((s + 1) % 3) * a.ntubes;
  int* rclear = a.reach + ((s + 2) % 3) * a.ntubes;
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < a.ntubes; t += TW) rclear[t] = 0;
  for (int it = blockIdx.x; it < nact; it += gridDim.x) {
    const int2 w = a.items[it];
    const Tube tb = a.tubes[w.x];
    const int R = rcur[w.x];
    if (R > a.r_cap) {
      if (threadIdx.x == 0) atomicOr(a.flags, kFlagReach);
      continue;
    }
    tile1d_step<T, KAHAN, TW>(in0, in1, in2, o0, o1, o2, tb.off, tb.n, tb.bc,
                          w.y, R, a.r_cap, a.k, rnext + w.x, a.flags,
                          a.eclamps, smem);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(a.ticket, 1u);
    is_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    *a.step = s + 1;
    *a.ticket = 0u;
    __threadfence();
  }
}

// The state of tube j after its last step lives in the buffers of parity
// nsteps_j % 2; later launches do not touch it.

template <typename T>
__global__ void batch_reach_seed(const Args a, const T* f0, const T* f1,
                                 const T* f2, long long total) {
  // per-tube reach of the initial state (slot 0)
  for (int j = blockIdx.x; j < a.ntubes; j += gridDim.x) {
    const Tube tb = a.tubes[j];
    int r = 0;
    for (int i = threadIdx.x; i < tb.n; i += blockDim.x) {
      const long long g = tb.off + i;
      r = max(r, reach_bound((double)f0[g], (double)f1[g], 0.0, (double)f2[g],
                             (float)a.k.kreach));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      r = max(r, __shfl_xor_sync(0xffffffffu, r, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&a.reach[j], r);
  }
  (void)total;
}

template <typename T>
__global__ void batch_init(const Args a, T* f0, T* f1, T* f2,
                           const double* st /* per tube: x_d, lam, gamma, rhoL,uL,pL,rhoR,uR,pR */) {
  for (int j = blockIdx.x; j < a.ntubes; j += gridDim.x) {
    const Tube tb = a.tubes[j];
    const double* q = st + 9 * (long long)j;
    const double dx = 1.0 / (double)tb.n;
    for (int i = threadIdx.x; i < tb.n; i += blockDim.x) {
      const double x = ((double)i + 0.5) * dx;
      const bool left = x < q[0];
      const double rho = left ? q[3] : q[6];
      const double u = left ? q[4] : q[7];
      const double p = left ? q[5] : q[8];
      const double lam = q[1];
      const double V = u * lam;
      const double rhoE = p * lam * lam / (q[2] - 1.0) + 0.5 * rho * (V * V);
      const long long g = tb.off + i;
      f0[g] = (T)rho;
      f1[g] = (T)(rho * V);
      f2[g] = (T)rhoE;
    }
  }
}

// FP64 totals of one tube's nodes (fixed order: strided partial sums per
// thread, then a fixed tree), physical units applied on the host.
template <typename T>
__global__ void batch_totals(const Args a, const T* f0, const T* f1,
                             const T* f2, double* out) {
  __shared__ double red[3][TILE / 32];
  for (int j = blockIdx.x; j < a.ntubes; j += gridDim.x) {
    const Tube tb = a.tubes[j];
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < tb.n; i += blockDim.x) {
      const long long g = tb.off + i;
      s[0] += (double)f0[g];
      s[1] += (double)f1[g];
      s[2] += (double)f2[g];
    }
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        s[f] += __shfl_down_sync(0xffffffffu, s[f], off);
    if ((threadIdx.x & 31) == 0)
      for (int f = 0; f < 3; ++f) red[f][threadIdx.x >> 5] = s[f];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int f = 0; f < 3; ++f) {
        double t = red[f][0];
        for (int w = 1; w < TILE / 32; ++w) t += red[f][w];
        out[3 * (long long)j + f] = t;
      }
    __syncthreads();
  }
}

}  // namespace batch
}  // namespace lbm

using namespace lbm;
using namespace lbm::batch;

struct lbm_batch {
  bool f64 = false;
  cudaStream_t stream = nullptr;
  int ntubes = 0;
  long long total = 0;
  int max_steps = 0;
  int r_cap = 64;
  int kahan = 1;
  size_t smem = 0;
  int grid = 0;
  int tile = 256;                // nodes per work item (chosen by tuning)
  double tune_ms[3] = {-1.0, -1.0, -1.0};  // ms per step of kTileChoices
  int nsm = 0;
  double* d_st = nullptr;        // initial states (for resets)
  int runs = 0;                  // lbm_batch_run calls so far
  EqConst k{};
  std::vector<int> order;        // sorted position -> caller's tube index
  std::vector<int> pos;          // caller's tube index -> sorted position
  std::vector<Tube> tubes;       // sorted
  std::vector<double> lambda;    // per sorted tube
  void* buf[2][3] = {{nullptr}};
  Tube* d_tubes = nullptr;
  int2* d_items = nullptr;
  int* d_active = nullptr;
  int* d_reach = nullptr;
  int* d_step = nullptr;
  unsigned* d_ticket = nullptr;
  unsigned* d_flags = nullptr;
  unsigned long long* d_eclamps = nullptr;
  double* d_totals = nullptr;
  int steps_done = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  bool broken = false;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& m) {
  if (b) {
    b->err = m;
    if (st != LBM_EINVAL) b->broken = true;
  }
  return st;
}

#define BCUDA(b, call, what)                                              \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess)                                                \
      return bfail((b), LBM_ECUDA,                                        \
                   std::string("lbm_batch: ") + (what) + ": " +           \
                       cudaGetErrorString(e_));                           \
  } while (0)

Args make_args(lbm_batch* b) {
  Args a{};
  for (int f = 0; f < 3; ++f) {
    a.f0[f] = b->buf[0][f];
    a.f1[f] = b->buf[1][f];
  }
  a.tubes = b->d_tubes;
  a.items = b->d_items;
  a.active = b->d_active;
  a.reach = b->d_reach;
  a.ntubes = b->ntubes;
  a.max_steps = b->max_steps;
  a.r_cap = b->r_cap;
  a.kahan = b->kahan;
  a.k = b->k;
  a.step = b->d_step;
  a.ticket = b->d_ticket;
  a.flags = b->d_flags;
  a.eclamps = b->d_eclamps;
  return a;
}

template <int TW>
const void* step_fn_tw(bool f64, int kahan) {
  if (f64) return (const void*)batch_step<double, false, TW>;
  return kahan ? (const void*)batch_step<float, true, TW>
               : (const void*)batch_step<float, false, TW>;
}

const void* step_fn(bool f64, int kahan, int tile) {
  return tile == 128 ? step_fn_tw<128>(f64, kahan)
                     : (tile == 512 ? step_fn_tw<512>(f64, kahan)
                                    : step_fn_tw<256>(f64, kahan));
}

template <int TW>
void launch_tw(lbm_batch* b, const Args& a) {
  if (b->f64)
    batch_step<double, false, TW><<<b->grid, TW, b->smem, b->stream>>>(a);
  else if (b->kahan)
    batch_step<float, true, TW><<<b->grid, TW, b->smem, b->stream>>>(a);
  else
    batch_step<float, false, TW><<<b->grid, TW, b->smem, b->stream>>>(a);
}

cudaError_t launch_one(lbm_batch* b) {
  Args a = make_args(b);
  if (b->tile == 128)
    launch_tw<128>(b, a);
  else if (b->tile == 512)
    launch_tw<512>(b, a);
  else
    launch_tw<256>(b, a);
  return cudaGetLastError();
}

size_t step_smem(bool f64, int tile, int r_cap) {
  if (f64)
    return tile == 128 ? step_smem_bytes_t<double, 1, 128>(r_cap)
           : tile == 512 ? step_smem_bytes_t<double, 1, 512>(r_cap)
                         : step_smem_bytes_t<double, 1, 256>(r_cap);
  return tile == 128 ? step_smem_bytes_t<float, 1, 128>(r_cap)
         : tile == 512 ? step_smem_bytes_t<float, 1, 512>(r_cap)
                       : step_smem_bytes_t<float, 1, 256>(r_cap);
}

// Work items, active-item table, shared memory and persistent grid for
// tiles of `tile` nodes; uploads the tables (stream-ordered).
cudaError_t configure(lbm_batch* b, int tile) {
  std::vector<int2> items;
  std::vector<int> items_upto(b->ntubes + 1, 0);
  for (int i = 0; i < b->ntubes; ++i) {
    const int nt = (int)((b->tubes[i].n + tile - 1) / tile);
    for (int q = 0; q < nt; ++q) items.push_back(make_int2(i, q));
    items_upto[i + 1] = items_upto[i] + nt;
  }
  // the tubes with nsteps > s form a prefix of the sorted order, and so do
  // their items
  std::vector<int> active(std::max(b->max_steps, 1), 0);
  int p = b->ntubes;
  for (int st = 0; st < b->max_steps; ++st) {
    while (p > 0 && b->tubes[p - 1].nsteps <= st) --p;
    active[st] = items_upto[p];
  }
  b->tile = tile;
  b->smem = step_smem(b->f64, tile, b->r_cap);
  const void* fn = step_fn(b->f64, b->kahan, tile);
  cudaError_t e = cudaFuncSetAttribute(
      fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tile, b->smem);
  if (e != cudaSuccess) return e;
  b->grid = std::max(1, per_sm) * b->nsm;
  e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(),
                      cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * active.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

// Initial state of every tube, step counter, reach, flags: as after
// creation.
cudaError_t reset_state(lbm_batch* b) {
  cudaStream_t s = b->stream;
  const int count = b->ntubes;
  cudaError_t e = cudaMemsetAsync(b->d_reach, 0, sizeof(int) * 3 * count, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_step, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flags, 0, sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_eclamps, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  Args a = make_args(b);
  const int g = std::min(b->ntubes, 65535);
  if (b->f64) {
    batch_init<double><<<g, TILE, 0, s>>>(a, (double*)b->buf[0][0],
                                          (double*)b->buf[0][1],
                                          (double*)b->buf[0][2], b->d_st);
    batch_reach_seed<double><<<g, TILE, 0, s>>>(
        a, (double*)b->buf[0][0], (double*)b->buf[0][1],
        (double*)b->buf[0][2], b->total);
  } else {
    batch_init<float><<<g, TILE, 0, s>>>(a, (float*)b->buf[0][0],
                                         (float*)b->buf[0][1],
                                         (float*)b->buf[0][2], b->d_st);
    batch_reach_seed<float><<<g, TILE, 0, s>>>(
        a, (float*)b->buf[0][0], (float*)b->buf[0][1], (float*)b->buf[0][2],
        b->total);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Times up to 6 steps (after one untimed) with each candidate width from
// the initial state, keeps the fastest, and resets.
cudaError_t tune(lbm_batch* b) {
  const int K = std::min(6, b->max_steps - 1);
  if (K < 2) return configure(b, 256);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  int best = 256;
  double best_ms = -1.0;
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    const int tw = kTileChoices[c];
    e = configure(b, tw);
    if (e == cudaSuccess) e = reset_state(b);
    if (e == cudaSuccess) e = launch_one(b);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    for (int k = 0; k < K && e == cudaSuccess; ++k) e = launch_one(b);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
      b->tune_ms[c] = ms / K;
      if (best_ms < 0.0 || b->tune_ms[c] < best_ms) {
        best_ms = b->tune_ms[c];
        best = tw;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  e = configure(b, best);
  if (e == cudaSuccess) e = reset_state(b);
  return e;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int32_t precision, double gamma, double theta,
                            int32_t kahan, const lbm_tube* tubes, int64_t count,
                            void* stream, lbm_batch** out) {
  if (!out || !tubes || count < 1 || count > (1 << 24)) return LBM_EINVAL;
  *out = nullptr;
  if (precision != LBM_F32 && precision != LBM_F64) return LBM_EINVAL;
  if (!(gamma > 1.0) || !(theta >= 0.0 && theta < 1.0)) return LBM_EINVAL;
  long long total = 0;
  int maxs = 0;
  for (int64_t j = 0; j < count; ++j) {
    const lbm_tube& t = tubes[j];
    if (t.n < 1 || t.n > (1 << 30) || t.nsteps < 0 || t.nsteps > (1 << 30) ||
        !(t.dt > 0.0) || t.bc < 0 || t.bc > 2 || !(t.left.rho >= 0.0) ||
        !(t.right.rho >= 0.0) || !(t.left.p >= 0.0) || !(t.right.p >= 0.0))
      return LBM_EINVAL;
    total += t.n;
    maxs = std::max(maxs, (int)t.nsteps);
  }
  if (total > (long long)1 << 34) return LBM_EINVAL;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->f64 = precision == LBM_F64;
  b->stream = (cudaStream_t)stream;
  b->ntubes = (int)count;
  b->total = total;
  b->max_steps = maxs;
  b->kahan = kahan ? 1 : 0;
  b->k.theta = theta;
  b->k.kq = 1.0 * (gamma - 1.0);
  b->k.kphi = 1.0 - 0.5 * 1.0 * (gamma - 1.0);
  b->k.b1 = 2.0;
  b->k.kreach = b->k.kq / (1.0 - theta);
  b->k.set_fp32_copies();
  b->smem = step_smem_bytes(1, b->f64, b->r_cap);

  // sort by decreasing step count (stable: ties keep the caller's order)
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return tubes[x].nsteps > tubes[y].nsteps;
  });
  b->pos.resize(count);
  std::vector<double> st(9 * (size_t)count);
  long long off = 0, max_items = 0;
  for (int i = 0; i < (int)count; ++i) {
    const lbm_tube& t = tubes[b->order[i]];
    b->pos[b->order[i]] = i;
    Tube tb{off, (int)t.n, (int)t.nsteps, t.bc, 0};
    b->tubes.push_back(tb);
    const double lam = t.dt * (double)t.n;  // dx = 1/n on [0, 1]
    b->lambda.push_back(lam);
    max_items += (t.n + kTileChoices[0] - 1) / kTileChoices[0];
    double* q = &st[9 * (size_t)i];
    q[0] = t.x_d;
    q[1] = lam;
    q[2] = gamma;
    q[3] = t.left.rho;
    q[4] = t.left.u;
    q[5] = t.left.p;
    q[6] = t.right.rho;
    q[7] = t.right.u;
    q[8] = t.right.p;
    off += t.n;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete b;
    return LBM_ECUDA;
  }
  const size_t es = b->f64 ? 8 : 4;
  bool ok = true;
  for (int p = 0; p < 2 && ok; ++p)
    for (int f = 0; f < 3 && ok; ++f)
      ok = cudaMalloc(&b->buf[p][f], es * (size_t)total) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_tubes, sizeof(Tube) * count) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_items, sizeof(int2) * (size_t)max_items) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_active, sizeof(int) * (size_t)std::max(maxs, 1)) ==
                 cudaSuccess;
  ok = ok && cudaMalloc(&b->d_reach, sizeof(int) * 3 * count) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_step, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_ticket, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_flags, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_eclamps, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_totals, sizeof(double) * 3 * count) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_st, sizeof(double) * st.size()) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ENOMEM;
  }
  e = cudaMemcpyAsync(b->d_tubes, b->tubes.data(), sizeof(Tube) * count,
                      cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_st, st.data(), sizeof(double) * st.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = step_prepare(1, b->f64, b->smem);
  if (e == cudaSuccess) e = tune(b);  // leaves the initial state
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch* b, int64_t max_launches) {
  if (!b) return LBM_EINVAL;
  if (b->broken) return bfail(b, LBM_ECUDA, "lbm_batch: in an error state: " + b->err);
  b->runs += 1;
  int64_t want = b->max_steps - b->steps_done;
  if (max_launches >= 0 && max_launches < want) want = max_launches;
  if (want <= 0) return LBM_OK;
  // one captured graph of G launches, replayed; the rest launched directly
  const int G = 32;
  if (!b->graph && want >= G) {
    cudaGraph_t g;
    cudaStream_t cs;
    BCUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    cudaStream_t keep = b->stream;
    b->stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; i < G && e == cudaSuccess; ++i) e = launch_one(b);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    b->stream = keep;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) BCUDA(b, e, "capture");
    BCUDA(b, e2, "end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    BCUDA(b, e, "graph instantiate");
    b->graph_len = G;
  }
  int64_t left = want;
  while (b->graph && left >= b->graph_len) {
    BCUDA(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
    left -= b->graph_len;
  }
  while (left > 0) {
    BCUDA(b, launch_one(b), "step launch");
    --left;
  }
  b->steps_done += (int)want;
  return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b, int64_t* steps_done, uint32_t* flags) {
  if (!b) return LBM_EINVAL;
  BCUDA(b, cudaStreamSynchronize(b->stream), "synchronize");
  unsigned f = 0;
  int sd = 0;
  BCUDA(b, cudaMemcpy(&f, b->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost), "flags");
  BCUDA(b, cudaMemcpy(&sd, b->d_step, sizeof(int), cudaMemcpyDeviceToHost), "step");
  if (steps_done) *steps_done = sd;
  if (flags) *flags = f;
  if (f & kFlagState) return bfail(b, LBM_ESTATE, "lbm_batch: rho < 0 or non-finite moment");
  if (f & kFlagReach) return bfail(b, LBM_EREACH, "lbm_batch: reach exceeded 64");
  return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch* b, int64_t tube, double* rho,
                             double* mx, double* rhoE, double* p, int64_t n) {
  if (!b || tube < 0 || tube >= b->ntubes || !rho || !mx || !rhoE) return LBM_EINVAL;
  const int i = b->pos[tube];
  const Tube& tb = b->tubes[i];
  if (n != tb.n) return bfail(b, LBM_EINVAL, "lbm_batch_moments: size");
  lbm_status st = lbm_batch_sync(b, nullptr, nullptr);
  if (st != LBM_OK) return st;
  // the tube's state after its own last step sits in parity nsteps % 2
  const int par = tb.nsteps & 1;
  const size_t es = b->f64 ? 8 : 4;
  std::vector<unsigned char> raw(es * (size_t)tb.n);
  double* outs[3] = {rho, mx, rhoE};
  std::vector<double> f[3];
  for (int k = 0; k < 3; ++k) {
    const unsigned char* src = (const unsigned char*)b->buf[par][k] + es * tb.off;
    BCUDA(b, cudaMemcpy(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost), "copy");
    f[k].resize(tb.n);
    for (int i2 = 0; i2 < tb.n; ++i2)
      f[k][i2] = b->f64 ? ((const double*)raw.data())[i2]
                        : (double)((const float*)raw.data())[i2];
  }
  const double lam = b->lambda[i];
  const double gm1 = b->k.kq;  // D (gamma - 1) with D = 1
  for (int i2 = 0; i2 < tb.n; ++i2) {
    const double r = f[0][i2];
    const double m = f[1][i2] / lam;
    const double E = f[2][i2] / (lam * lam);
    outs[0][i2] = r;
    outs[1][i2] = m;
    outs[2][i2] = E;
    if (p) p[i2] = gm1 * (E - 0.5 * (m * m) / r);
  }
  return LBM_OK;
}

lbm_status lbm_batch_totals(lbm_batch* b, double* out, int64_t count) {
  if (!b || !out || count != b->ntubes) return LBM_EINVAL;
  // each tube's totals from the parity holding its final state: launch
  // once per parity and pick per tube
  std::vector<double> t[2];
  for (int par = 0; par < 2; ++par) {
    Args a = make_args(b);
    const int g = std::min(b->ntubes, 65535);
    if (b->f64)
      batch_totals<double><<<g, TILE, 0, b->stream>>>(
          a, (const double*)b->buf[par][0], (const double*)b->buf[par][1],
          (const double*)b->buf[par][2], b->d_totals);
    else
      batch_totals<float><<<g, TILE, 0, b->stream>>>(
          a, (const float*)b->buf[par][0], (const float*)b->buf[par][1],
          (const float*)b->buf[par][2], b->d_totals);
    BCUDA(b, cudaGetLastError(), "totals");
    t[par].resize(3 * (size_t)b->ntubes);
    BCUDA(b, cudaMemcpyAsync(t[par].data(), b->d_totals,
                             sizeof(double) * t[par].size(),
                             cudaMemcpyDeviceToHost, b->stream), "copy");
    BCUDA(b, cudaStreamSynchronize(b->stream), "synchronize");
  }
  for (int j = 0; j < b->ntubes; ++j) {
    const int i = b->pos[j];
    const int par = b->tubes[i].nsteps & 1;
    const double lam = b->lambda[i];
    out[3 * j + 0] = t[par][3 * i + 0];
    out[3 * j + 1] = t[par][3 * i + 1] / lam;
    out[3 * j + 2] = t[par][3 * i + 2] / (lam * lam);
  }
  return LBM_OK;
}

lbm_status lbm_batch_tuning(const lbm_batch* b, int32_t* tile,
                            double* ms_per_step) {
  if (!b) return LBM_EINVAL;
  if (tile) *tile = b->tile;
  if (ms_per_step)
    for (int c = 0; c < 3; ++c) ms_per_step[c] = b->tune_ms[c];
  return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch* b, int32_t tile) {
  if (!b || (tile != 128 && tile != 256 && tile != 512)) return LBM_EINVAL;
  if (b->runs > 0)
    return bfail(b, LBM_EINVAL, "lbm_batch_set_tile: the batch has run");
  if (b->broken) return bfail(b, LBM_ECUDA, "lbm_batch: in an error state: " + b->err);
  BCUDA(b, configure(b, tile), "configure");
  BCUDA(b, reset_state(b), "reset");
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
  return b ? b->err.c_str() : "lbm_batch: NULL handle";
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (int p = 0; p < 2; ++p)
    for (int f = 0; f < 3; ++f)
      if (b->buf[p][f]) cudaFree(b->buf[p][f]);
  void* ptrs[] = {b->d_tubes, b->d_items, b->d_active, b->d_reach, b->d_step,
                  b->d_ticket, b->d_flags, b->d_eclamps, b->d_totals, b->d_st};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
