// Tube pool for continuous batching: 1-D tubes (Section V.C shock tubes)
// join and leave between steps while one launch per step advances every
// tube that still has steps to take.  Contract: include/lbm.h.
//
// Each slot owns a node range of one SoA buffer (rho, m, rhoE; two parities)
// and its own step counter on the device: a tube that joined later reads the
// parity and reach slot of its own step.  The work items (slot, 256-node
// tile) of the stepping slots are rebuilt on the host only when that set
// changes.  The step of a tile is the shared 1-D tile step (tile1d.cuh), so a
// tube's result does not depend on what else is in the pool.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "tile1d.cuh"

namespace lbm {
namespace pool {

struct Slot {
  long long off;
  int n, bc, nsteps, k;  // k: steps taken (device copy advanced by the kernel)
  int live, pad_;
};

struct Args {
  void* f0[3];
  void* f1[3];
  Slot* slots;
  const int2* items;      // (slot, tile)
  const int* stepping;    // slots that step in this launch
  int nitems, nstepping;
  int* reach;             // [3][max_slots]
  int max_slots;
  int r_cap;
  EqConst k;
  unsigned* ticket;
  unsigned* flags;
  unsigned long long* eclamps;
};

template <typename T, bool KAHAN>
__global__ void __launch_bounds__(kTile1d) pool_step(const Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int is_last;
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const int2 w = a.items[it];
    const Slot sl = a.slots[w.x];
    const int par = sl.k & 1;
    const T* in0 = (const T*)(par ? a.f1[0] : a.f0[0]);
    const T* in1 = (const T*)(par ? a.f1[1] : a.f0[1]);
    const T* in2 = (const T*)(par ? a.f1[2] : a.f0[2]);
    T* o0 = (T*)(par ? a.f0[0] : a.f1[0]);
    T* o1 = (T*)(par ? a.f0[1] : a.f1[1]);
    T* o2 = (T*)(par ? a.f0[2] : a.f1[2]);
    const int R = a.reach[(sl.k % 3) * a.max_slots + w.x];
    if (R > a.r_cap) {
      if (threadIdx.x == 0) atomicOr(a.flags, kFlagReach);
      continue;
    }
    tile1d_step<T, KAHAN>(in0, in1, in2, o0, o1, o2, sl.off, sl.n, sl.bc, w.y,
                          R, a.r_cap, a.k,
                          a.reach + ((sl.k + 1) % 3) * a.max_slots + w.x,
                          a.flags, a.eclamps, smem);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // every stepping slot: clear the reach slot its next step writes into,
  // then count the step
  for (int i = threadIdx.x; i < a.nstepping; i += kTile1d) {
    const int s = a.stepping[i];
    const int k = a.slots[s].k;
    a.reach[((k + 2) % 3) * a.max_slots + s] = 0;
    a.slots[s].k = k + 1;
  }
  if (threadIdx.x == 0) *a.ticket = 0u;
}

template <typename T>
__global__ void pool_init(Slot* slots, int s, T* f0, T* f1, T* f2, int* reach,
                          int max_slots, double x_d, double lam, double gamma,
                          double rl, double ul, double pl, double rr,
                          double ur, double pr, float kreach) {
  __shared__ int red[kTile1d / 32];
  const Slot sl = slots[s];
  const double dx = 1.0 / (double)sl.n;
  int r = 0;
  for (int i = threadIdx.x; i < sl.n; i += blockDim.x) {
    const double x = ((double)i + 0.5) * dx;
    const bool left = x < x_d;
    const double rho = left ? rl : rr, u = left ? ul : ur, p = left ? pl : pr;
    const double V = u * lam;
    const double rhoE = p * lam * lam / (gamma - 1.0) + 0.5 * rho * (V * V);
    const long long g = sl.off + i;
    f0[g] = (T)rho;
    f1[g] = (T)(rho * V);
    f2[g] = (T)rhoE;
    r = max(r, reach_bound((double)(T)rho, (double)(T)(rho * V), 0.0,
                           (double)(T)rhoE, kreach));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < kTile1d / 32; ++w) m = max(m, red[w]);
    reach[0 * max_slots + s] = m;
    reach[1 * max_slots + s] = 0;
    reach[2 * max_slots + s] = 0;
  }
}

}  // namespace pool
}  // namespace lbm

using namespace lbm;
using namespace lbm::pool;

struct lbm_pool {
  bool f64 = false;
  int kahan = 1;
  cudaStream_t stream = nullptr;
  double gamma = 1.4;
  EqConst k{};
  long long capacity = 0;
  int max_slots = 0;
  int r_cap = 64;
  size_t smem = 0;
  int grid = 0;
  void* buf[2][3] = {{nullptr}};
  Slot* d_slots = nullptr;
  int2* d_items = nullptr;
  int* d_stepping = nullptr;
  int* d_reach = nullptr;
  unsigned* d_ticket = nullptr;
  unsigned* d_flags = nullptr;
  unsigned long long* d_eclamps = nullptr;
  int max_items = 0;
  std::vector<Slot> slots;         // host mirror (k counted on the host too)
  std::vector<double> lambda;
  std::map<long long, long long> free_ranges;  // offset -> length
  std::vector<int> stepping;
  int nitems = 0;
  bool dirty = true;
  std::string err;
  bool broken = false;
};

namespace {

lbm_status pfail(lbm_pool* p, lbm_status st, const std::string& m) {
  if (p) {
    p->err = m;
    if (st != LBM_EINVAL && st != LBM_EBUDGET) p->broken = true;
  }
  return st;
}

#define PCUDA(p, call, what)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return pfail((p), LBM_ECUDA, std::string("lbm_pool: ") + (what) + ": " + \
                                       cudaGetErrorString(e_));               \
  } while (0)

bool take_range(lbm_pool* p, long long n, long long* off) {
  for (auto it = p->free_ranges.begin(); it != p->free_ranges.end(); ++it) {
    if (it->second >= n) {
      *off = it->first;
      const long long rest = it->second - n;
      const long long at = it->first + n;
      p->free_ranges.erase(it);
      if (rest > 0) p->free_ranges[at] = rest;
      return true;
    }
  }
  return false;
}

void give_range(lbm_pool* p, long long off, long long n) {
  auto it = p->free_ranges.emplace(off, n).first;
  auto nx = std::next(it);
  if (nx != p->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    p->free_ranges.erase(nx);
  }
  if (it != p->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      p->free_ranges.erase(it);
    }
  }
}

}  // namespace

extern "C" {

lbm_status lbm_pool_create(int32_t precision, double gamma, double theta,
                           int32_t kahan, int64_t capacity_nodes,
                           int32_t max_slots, void* stream, lbm_pool** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if ((precision != LBM_F32 && precision != LBM_F64) || !(gamma > 1.0) ||
      !(theta >= 0.0 && theta < 1.0) || capacity_nodes < 1 ||
      capacity_nodes > ((long long)1 << 36) || max_slots < 1 ||
      max_slots > (1 << 20))
    return LBM_EINVAL;
  lbm_pool* p = new (std::nothrow) lbm_pool();
  if (!p) return LBM_ENOMEM;
  p->f64 = precision == LBM_F64;
  p->kahan = kahan ? 1 : 0;
  p->stream = (cudaStream_t)stream;
  p->gamma = gamma;
  p->k.theta = theta;
  p->k.kq = gamma - 1.0;
  p->k.kphi = 1.0 - 0.5 * (gamma - 1.0);
  p->k.b1 = 2.0;
  p->k.kreach = p->k.kq / (1.0 - theta);
  p->k.set_fp32_copies();
  p->capacity = capacity_nodes;
  p->max_slots = max_slots;
  p->smem = step_smem_bytes(1, p->f64, p->r_cap);
  p->max_items = (int)std::min<long long>(
      (capacity_nodes + kTile1d - 1) / kTile1d + max_slots, 1 << 30);
  p->slots.assign(max_slots, Slot{0, 0, 0, 0, 0, 0, 0});
  p->lambda.assign(max_slots, 0.0);
  p->free_ranges[0] = capacity_nodes;
  const void* fn = p->f64 ? (const void*)pool_step<double, false>
                          : (p->kahan ? (const void*)pool_step<float, true>
                                      : (const void*)pool_step<float, false>);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p->smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTile1d,
                                                      p->smem);
  if (e != cudaSuccess) {
    delete p;
    return LBM_ECUDA;
  }
  p->grid = std::max(1, per_sm) * nsm;
  const size_t es = p->f64 ? 8 : 4;
  bool ok = true;
  for (int q = 0; q < 2 && ok; ++q)
    for (int f = 0; f < 3 && ok; ++f)
      ok = cudaMalloc(&p->buf[q][f], es * (size_t)capacity_nodes) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_slots, sizeof(Slot) * max_slots) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_items, sizeof(int2) * p->max_items) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_stepping, sizeof(int) * max_slots) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_reach, sizeof(int) * 3 * max_slots) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_ticket, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_flags, sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMalloc(&p->d_eclamps, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_pool_destroy(p);
    return LBM_ENOMEM;
  }
  e = cudaMemsetAsync(p->d_slots, 0, sizeof(Slot) * max_slots, p->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(p->d_reach, 0, sizeof(int) * 3 * max_slots, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_ticket, 0, sizeof(unsigned), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_flags, 0, sizeof(unsigned), p->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(p->d_eclamps, 0, sizeof(unsigned long long), p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    lbm_pool_destroy(p);
    return LBM_ECUDA;
  }
  *out = p;
  return LBM_OK;
}

lbm_status lbm_pool_add(lbm_pool* p, const lbm_tube* t, int32_t* slot) {
  if (!p || !t || !slot) return LBM_EINVAL;
  if (p->broken) return pfail(p, LBM_ECUDA, "lbm_pool: in an error state");
  if (t->n < 1 || t->n > (1 << 30) || t->nsteps < 0 || t->nsteps > (1 << 30) ||
      !(t->dt > 0.0) || t->bc < 0 || t->bc > 2 || !(t->left.rho >= 0.0) ||
      !(t->right.rho >= 0.0) || !(t->left.p >= 0.0) || !(t->right.p >= 0.0))
    return pfail(p, LBM_EINVAL, "lbm_pool_add: bad tube");
  int s = -1;
  for (int i = 0; i < p->max_slots; ++i)
    if (!p->slots[i].live) {
      s = i;
      break;
    }
  long long off = 0;
  if (s < 0 || !take_range(p, t->n, &off))
    return pfail(p, LBM_EBUDGET, "lbm_pool_add: no free slot or node range");
  Slot sl{off, (int)t->n, t->bc, (int)t->nsteps, 0, 1, 0};
  p->slots[s] = sl;
  const double lam = t->dt * (double)t->n;
  p->lambda[s] = lam;
  PCUDA(p, cudaMemcpyAsync(p->d_slots + s, &p->slots[s], sizeof(Slot),
                           cudaMemcpyHostToDevice, p->stream), "slot upload");
  if (p->f64)
    pool_init<double><<<1, kTile1d, 0, p->stream>>>(
        p->d_slots, s, (double*)p->buf[0][0], (double*)p->buf[0][1],
        (double*)p->buf[0][2], p->d_reach, p->max_slots, t->x_d, lam, p->gamma,
        t->left.rho, t->left.u, t->left.p, t->right.rho, t->right.u,
        t->right.p, (float)p->k.kreach);
  else
    pool_init<float><<<1, kTile1d, 0, p->stream>>>(
        p->d_slots, s, (float*)p->buf[0][0], (float*)p->buf[0][1],
        (float*)p->buf[0][2], p->d_reach, p->max_slots, t->x_d, lam, p->gamma,
        t->left.rho, t->left.u, t->left.p, t->right.rho, t->right.u,
        t->right.p, (float)p->k.kreach);
  PCUDA(p, cudaGetLastError(), "init kernel");
  p->dirty = true;
  *slot = s;
  return LBM_OK;
}

lbm_status lbm_pool_step(lbm_pool* p) {
  if (!p) return LBM_EINVAL;
  if (p->broken) return pfail(p, LBM_ECUDA, "lbm_pool: in an error state");
  if (p->dirty) {
    std::vector<int2> items;
    p->stepping.clear();
    for (int s = 0; s < p->max_slots; ++s) {
      const Slot& sl = p->slots[s];
      if (!sl.live || sl.k >= sl.nsteps) continue;
      p->stepping.push_back(s);
      for (int q = 0; q < (sl.n + kTile1d - 1) / kTile1d; ++q)
        items.push_back(make_int2(s, q));
    }
    p->nitems = (int)items.size();
    if (!items.empty())
      PCUDA(p, cudaMemcpyAsync(p->d_items, items.data(), sizeof(int2) * items.size(),
                               cudaMemcpyHostToDevice, p->stream), "items");
    if (!p->stepping.empty())
      PCUDA(p, cudaMemcpyAsync(p->d_stepping, p->stepping.data(),
                               sizeof(int) * p->stepping.size(),
                               cudaMemcpyHostToDevice, p->stream), "stepping");
    p->dirty = false;
  }
  if (p->stepping.empty()) return LBM_OK;
  Args a{};
  for (int f = 0; f < 3; ++f) {
    a.f0[f] = p->buf[0][f];
    a.f1[f] = p->buf[1][f];
  }
  a.slots = p->d_slots;
  a.items = p->d_items;
  a.stepping = p->d_stepping;
  a.nitems = p->nitems;
  a.nstepping = (int)p->stepping.size();
  a.reach = p->d_reach;
  a.max_slots = p->max_slots;
  a.r_cap = p->r_cap;
  a.k = p->k;
  a.ticket = p->d_ticket;
  a.flags = p->d_flags;
  a.eclamps = p->d_eclamps;
  const int grid = std::max(1, std::min(p->grid, p->nitems));
  if (p->f64)
    pool_step<double, false><<<grid, kTile1d, p->smem, p->stream>>>(a);
  else if (p->kahan)
    pool_step<float, true><<<grid, kTile1d, p->smem, p->stream>>>(a);
  else
    pool_step<float, false><<<grid, kTile1d, p->smem, p->stream>>>(a);
  PCUDA(p, cudaGetLastError(), "step kernel");
  bool finished = false;
  for (int s : p->stepping) {
    p->slots[s].k += 1;
    if (p->slots[s].k >= p->slots[s].nsteps) finished = true;
  }
  if (finished) p->dirty = true;
  return LBM_OK;
}

lbm_status lbm_pool_run(lbm_pool* p, int64_t nsteps) {
  if (!p || nsteps < 0) return LBM_EINVAL;
  for (int64_t i = 0; i < nsteps; ++i) {
    const lbm_status st = lbm_pool_step(p);
    if (st != LBM_OK) return st;
    if (p->stepping.empty() && !p->dirty) break;  // nothing left to step
  }
  return LBM_OK;
}

lbm_status lbm_pool_progress(lbm_pool* p, int32_t slot, int64_t* taken,
                             int64_t* nsteps) {
  if (!p || slot < 0 || slot >= p->max_slots || !p->slots[slot].live)
    return LBM_EINVAL;
  if (taken) *taken = p->slots[slot].k;
  if (nsteps) *nsteps = p->slots[slot].nsteps;
  return LBM_OK;
}

lbm_status lbm_pool_read(lbm_pool* p, int32_t slot, double* rho, double* mx,
                         double* rhoE, double* pr, int64_t n) {
  if (!p || slot < 0 || slot >= p->max_slots || !p->slots[slot].live || !rho ||
      !mx || !rhoE || n != p->slots[slot].n)
    return LBM_EINVAL;
  const Slot& sl = p->slots[slot];
  PCUDA(p, cudaStreamSynchronize(p->stream), "synchronize");
  unsigned f = 0;
  PCUDA(p, cudaMemcpy(&f, p->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost),
        "flags");
  if (f & kFlagState) return pfail(p, LBM_ESTATE, "lbm_pool: bad state");
  if (f & kFlagReach) return pfail(p, LBM_EREACH, "lbm_pool: reach above 64");
  const int par = sl.k & 1;
  const size_t es = p->f64 ? 8 : 4;
  std::vector<unsigned char> raw(es * (size_t)sl.n);
  std::vector<double> v[3];
  for (int q = 0; q < 3; ++q) {
    PCUDA(p, cudaMemcpy(raw.data(), (const unsigned char*)p->buf[par][q] + es * sl.off,
                        raw.size(), cudaMemcpyDeviceToHost), "copy");
    v[q].resize(sl.n);
    for (int i = 0; i < sl.n; ++i)
      v[q][i] = p->f64 ? ((const double*)raw.data())[i]
                       : (double)((const float*)raw.data())[i];
  }
  const double lam = p->lambda[slot];
  for (int i = 0; i < sl.n; ++i) {
    const double r = v[0][i], m = v[1][i] / lam, E = v[2][i] / (lam * lam);
    rho[i] = r;
    mx[i] = m;
    rhoE[i] = E;
    if (pr) pr[i] = (p->gamma - 1.0) * (E - 0.5 * (m * m) / r);
  }
  return LBM_OK;
}

lbm_status lbm_pool_remove(lbm_pool* p, int32_t slot) {
  if (!p || slot < 0 || slot >= p->max_slots || !p->slots[slot].live)
    return LBM_EINVAL;
  Slot& sl = p->slots[slot];
  give_range(p, sl.off, sl.n);
  sl.live = 0;
  // the device copy keeps its values; the slot is no longer in any item
  p->dirty = true;
  return LBM_OK;
}

const char* lbm_pool_last_error(const lbm_pool* p) {
  return p ? p->err.c_str() : "lbm_pool: NULL handle";
}

void lbm_pool_destroy(lbm_pool* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  for (int q = 0; q < 2; ++q)
    for (int f = 0; f < 3; ++f)
      if (p->buf[q][f]) cudaFree(p->buf[q][f]);
  void* ptrs[] = {p->d_slots, p->d_items, p->d_stepping, p->d_reach,
                  p->d_ticket, p->d_flags, p->d_eclamps};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  cudaGetLastError();
  delete p;
}

}  // extern "C"
