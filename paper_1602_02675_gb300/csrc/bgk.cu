// Relaxation-time step (general tau, eqs 4-5) on a per-packet state.
//
// With tau != 1 the collision keeps part of the distribution that arrived,
// so a node's state is the set of packets it holds rather than its moments:
// one slot j per entry of the velocity set (Section IV; 1-D: 5 slots, 2-D:
// 8 slots in the table order of packet<DIM>), each slot carrying mass,
// momentum and energy (the integrand of eq 6 for one migrating velocity).
// One step, per node:
//   Y = sum_j f_j (eq 6), slots in table order;
//   f_eq_j of Y (Section III.B, eqs 11-26), as in the tau = 1 step;
//   collision (eqs 4-5): f*_j = (1 - 1/tau) f_j + (1/tau) f_eq_j, which is
//     f_eq_j exactly at tau = 1 (eq 10);
//   migration: slot j moves with the node's V + c'_j and splits over
//     s + n + c'_j + k with the weights of eqs 23, 28-29;
//   the destination's slot j is the sum of its slot-j arrivals, sources in
//   ascending order (y-major, x fastest), then corners.
// Additional points (Section V.B) hold the supplying node's packets: copied
// (transmissive, periodic) or mirrored across a reflecting wall (the slot
// whose c' points the other way along the normal, normal momentum negated,
// moments the node's with that component negated).
//
// Square lattice with a reach limit up to 4: one kernel per step
// (step2d), each block colliding its tile's window into shared memory and
// gathering the tile from it.  Otherwise two kernels per step:
//  * collide: one thread per source of the grid padded by the reach limit
//    r_cap (additional points included): moments, equilibrium, post-collision
//    packets, corner weights and a word (c1, n) into the source records;
//    clamps, bad states and the step's reach of the grid's nodes are
//    reduced on the device;
//  * gather: one thread per destination of a 32 x 8 tile.
// In either gather a tile whose source window holds one type (c1, n) reads
// each slot's four arriving corners directly; otherwise every source of the
// (2R + 1)^D window is tested once, all slots' sums in registers.  Either
// way in the order above, so both paths give the same bits.
// This unit is built without floating-point contraction, so the FP64
// instance reproduces a plain evaluation of the same formulas bit for bit;
// FP32 multiply-adds are explicit fused multiply-adds (mad).
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"
#include "step_kernel.cuh"

namespace lbm {
namespace bgk {

template <int DIM>
struct Shape {
  static constexpr int NP = DIM == 1 ? 5 : 8;  // slots
  static constexpr int NF = DIM + 2;           // mass, momentum, energy
};

struct Args {
  const void* f;   // packets in: element (j * NF + c) * n + i
  void* fo;        // packets out, same layout
  void* rec;       // source records (layout: rec_layout)
  void* mom[4];    // moments buffer: rho, m_x, m_y (2-D), rhoE
  int nx, ny, bc_x, bc_y, rc;
  long long n;
  double omega, keep;     // 1/tau, 1 - 1/tau
  float omega_f, keep_f;  // the same rounded to FP32 on the host
  EqConst k;
  Scratch* scr;
  int rs;      // reach slot of this step (see reach_slot / step2d)
  int* rslot;  // one-launch step: three reach slots
};

// The two reach slots alternate between steps: the collision of a step
// max-reduces into its slot, the gather reads it and clears the other one
// for the next step (no gather of the previous step still reads it).
__device__ __forceinline__ int* reach_slot(Scratch* scr, int rs) {
  return rs ? &scr->reach_next : &scr->reach;
}

// Source records over the padded grid (PX = nx + 2 rc, PY = ny + 2 rc in
// 2-D, 1 in 1-D; cap = PX PY sources, source (x, y) at (y + rc) PX + x + rc
// in 2-D, x + rc in 1-D): first one 64-bit word per source (c1, n_x, n_y as
// 16-bit fields; c1 = -1: the source emits nothing; rounded up to an even
// count), then per slot j an array of cap groups of NF post-collision
// fields (source i's at (j cap + i) NF), then the corner weights of eqs
// 28-29 (arrays NP * NF + k of cap elements: 1-D k = 0, 1 for (1 - f, f);
// 2-D k = kx + 2 ky for (1 - f_x or f_x) (1 - f_y or f_y)).
template <typename T, int DIM>
struct RecView {
  static constexpr int NF = Shape<DIM>::NF;
  long long cap;
  long long* word;
  T* v;
  // slot j's fields of source i are contiguous (one 16-byte access per
  // slot in 2-D FP32, two in FP64)
  __device__ __forceinline__ T* slot(int j, long long i) const {
    return v + ((long long)j * cap + i) * NF;
  }
  __device__ __forceinline__ void ld(int j, long long i, T (&o)[NF]) const {
    const T* p = slot(j, i);
    if constexpr (NF == 4 && sizeof(T) == 4) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      o[0] = q.x;
      o[1] = q.y;
      o[2] = q.z;
      o[3] = q.w;
    } else if constexpr (NF == 4 && sizeof(T) == 8) {
      const double2 q0 = reinterpret_cast<const double2*>(p)[0];
      const double2 q1 = reinterpret_cast<const double2*>(p)[1];
      o[0] = q0.x;
      o[1] = q0.y;
      o[2] = q1.x;
      o[3] = q1.y;
    } else {
#pragma unroll
      for (int c = 0; c < NF; ++c) o[c] = p[c];
    }
  }
  __device__ __forceinline__ void st(int j, long long i,
                                     const T (&o)[NF]) const {
    T* p = slot(j, i);
    if constexpr (NF == 4 && sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (NF == 4 && sizeof(T) == 8) {
      reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
      reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
    } else {
#pragma unroll
      for (int c = 0; c < NF; ++c) p[c] = o[c];
    }
  }
  __device__ __forceinline__ T& wt(int k, long long i) const {
    return v[(long long)(Shape<DIM>::NP * NF + k) * cap + i];
  }
};
// Words of a record view, rounded up to an even count so that the fields
// after them start on a 16-byte boundary.
__host__ __device__ inline long long rec_words(long long cap) {
  return (cap + 1) & ~1LL;
}
template <typename T, int DIM>
__device__ __forceinline__ RecView<T, DIM> rec_view(const Args& a) {
  const long long PX = (long long)a.nx + 2 * a.rc;
  const long long PY = DIM == 2 ? (long long)a.ny + 2 * a.rc : 1;
  RecView<T, DIM> r;
  r.cap = PX * PY;
  r.word = static_cast<long long*>(a.rec);
  r.v = reinterpret_cast<T*>(r.word + rec_words(r.cap));
  return r;
}

// Bytes of the records of an nx x ny grid with reach limit rc.
inline size_t rec_bytes(int dim, int nx, int ny, int rc, size_t es) {
  const size_t PX = (size_t)nx + 2 * (size_t)rc;
  const size_t PY = dim == 2 ? (size_t)ny + 2 * (size_t)rc : 1;
  const int arrays = dim == 1 ? 5 * 3 + 2 : 8 * 4 + 4;
  return (size_t)rec_words((long long)(PX * PY)) * 8 + PX * PY * arrays * es;
}

// Slot of the packet mirrored across a wall normal to `axis`.
template <int DIM>
__device__ __forceinline__ int mirror_slot(int axis, int j) {
  if (DIM == 1) return j == 0 ? 0 : ((j & 1) ? j + 1 : j - 1);
  const int dir = j & 3;  // 0: +x, 1: -x, 2: +y, 3: -y
  if (axis == 0 && dir < 2) return j ^ 1;
  if (axis == 1 && dir >= 2) return j ^ 1;
  return j;
}

template <typename T>
__device__ __forceinline__ T rel_const(double d, float f);
template <>
__device__ __forceinline__ double rel_const<double>(double d, float) {
  return d;
}
template <>
__device__ __forceinline__ float rel_const<float>(double, float f) {
  return f;
}

// a * b + c: FP64 with two roundings, as the oracle evaluates it (this unit
// is built without contraction); FP32 as one fused multiply-add.
__device__ __forceinline__ double mad(double a, double b, double c) {
  return a * b + c;
}
__device__ __forceinline__ float mad(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}

// Equilibrium packet j of q as (mass, m_x, [m_y,] energy).
template <typename T, int DIM>
__device__ __forceinline__ void eq_packet(const Equil<T>& q, int j,
                                          T (&out)[Shape<DIM>::NF]) {
  int cx, cy, lev;
  packet<DIM>(j, q.c1, &cx, &cy, &lev);
  const T d = DIM == 1 ? (lev == 0 ? q.d0 : (lev == 1 ? q.d1 : q.d2))
                       : (lev == 0 ? q.d1 : q.d2);
  T px, py, pe;
  packet_fields<T, DIM>(q, j, &px, &py, &pe);
  out[0] = d;
  out[1] = px;
  if (DIM == 2) out[2] = py;
  out[Shape<DIM>::NF - 1] = pe;
}

// Migration reach floor(|V_a|) + 1 + c2 of a node (0 if it emits nothing).
template <typename T>
__device__ __forceinline__ int node_reach(const Equil<T>& q) {
  if (!q.emits) return 0;
  const T a0 = q.V0 < T(0) ? -q.V0 : q.V0;
  const T a1 = q.V1 < T(0) ? -q.V1 : q.V1;
  const T v = dev_floor(a0 > a1 ? a0 : a1);
  if (!(v < T(1.0e8))) return 100000000;
  return (int)v + 2 + q.c1;
}

template <typename T, int DIM>
__device__ __forceinline__ void node_moments(const T* f, long long n,
                                             long long g, T (&Y)[4]) {
  constexpr int NP = Shape<DIM>::NP, NF = Shape<DIM>::NF;
  Y[0] = Y[1] = Y[2] = Y[3] = T(0);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    Y[0] = Y[0] + f[(long long)(j * NF) * n + g];
    Y[1] = Y[1] + f[(long long)(j * NF + 1) * n + g];
    if (DIM == 2) Y[2] = Y[2] + f[(long long)(j * NF + 2) * n + g];
    Y[3] = Y[3] + f[(long long)(j * NF + NF - 1) * n + g];
  }
}

__device__ __forceinline__ void flag_warp(Scratch* scr, int rs,
                                          unsigned long long c, bool bad,
                                          int rmax) {
  const unsigned wc = __reduce_add_sync(0xffffffffu, (unsigned)c);
  const bool wb = __any_sync(0xffffffffu, bad);
  const int wr = __reduce_max_sync(0xffffffffu, rmax);
  if ((threadIdx.x & 31) == 0) {
    if (wc) atomicAdd(&scr->eclamps, (unsigned long long)wc);
    if (wb) atomicOr(&scr->flags, kFlagState);
    if (wr) atomicMax(reach_slot(scr, rs), wr);
  }
}

// Collision of one source (sx, sy) into entry i of a record view (the
// padded grid's records, or a window in shared memory): the supplying
// node's moments (eq 6; across a reflecting wall its normal momentum
// negated), its equilibrium, the blend per slot, the corner weights and the
// word.  `owned`: the source is a node of the grid counted by this thread
// (clamps, bad state, reach).
// REGS: the node's slots stay in registers from the moments to the blend
// (one round of loads; the one-launch step, whose window sources miss L1);
// otherwise each slot is read again at its blend (fewer registers; the
// collision kernel, whose re-reads hit L1).
template <typename T, int DIM, bool REGS>
__device__ __forceinline__ void collide_one(const Args& a, const T* f,
                                            long long sx, long long sy,
                                            bool owned,
                                            const RecView<T, DIM>& r,
                                            long long i,
                                            unsigned long long& clamps,
                                            bool& bad, int& rmax) {
  constexpr int NP = Shape<DIM>::NP, NF = Shape<DIM>::NF;
  const T omega = rel_const<T>(a.omega, a.omega_f);
  const T keep = rel_const<T>(a.keep, a.keep_f);
  bool flx = false, fly = false;
  const int gx = virtual_axis(a.bc_x, a.nx, sx, &flx);
  const int gy = DIM == 2 ? virtual_axis(a.bc_y, a.ny, sy, &fly) : 0;
  const long long g = (long long)gy * a.nx + gx;
  // the node's moments, slots summed in table order
  T fa[NP][NF];
  T Y[4] = {T(0), T(0), T(0), T(0)};
  if (REGS) {
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
      for (int c = 0; c < NF; ++c)
        fa[j][c] = f[(long long)(j * NF + c) * a.n + g];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      Y[0] = Y[0] + fa[j][0];
      Y[1] = Y[1] + fa[j][1];
      if (DIM == 2) Y[2] = Y[2] + fa[j][2];
      Y[3] = Y[3] + fa[j][NF - 1];
    }
  } else {
    node_moments<T, DIM>(f, a.n, g, Y);
  }
  if (flx) Y[1] = -Y[1];
  if (fly) Y[2] = -Y[2];
  const Equil<T> q = equilibrium<T, DIM>(Y[0], Y[1], Y[2], Y[3], a.k);
  if (owned) {
    clamps += q.clamp ? 1 : 0;
    bad |= q.bad;
    rmax = max(rmax, node_reach(q));
  }
  long long w = s64_word(-1, 0, 0);
  if (q.emits && REGS) {
    // the mirror image's slots: the node's, swapped across each reflecting
    // wall (the two mirrors act on different slots and commute), normal
    // momentum negated
    if (flx) {
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int m = mirror_slot<DIM>(0, j);
        if (m > j) {
#pragma unroll
          for (int c = 0; c < NF; ++c) {
            const T t = fa[j][c];
            fa[j][c] = fa[m][c];
            fa[m][c] = t;
          }
        }
        fa[j][1] = -fa[j][1];
      }
    }
    if (DIM == 2 && fly) {
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int m = mirror_slot<DIM>(1, j);
        if (m > j) {
#pragma unroll
          for (int c = 0; c < NF; ++c) {
            const T t = fa[j][c];
            fa[j][c] = fa[m][c];
            fa[m][c] = t;
          }
        }
        fa[j][2] = -fa[j][2];
      }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      T fj[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) fj[c] = fa[j][c];
      T feq[NF];
      eq_packet<T, DIM>(q, j, feq);
      // eqs 4-5 as the blend (1 - 1/tau) f + (1/tau) f_eq
      T o[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) o[c] = mad(keep, fj[c], omega * feq[c]);
      r.st(j, i, o);
    }
  } else if (q.emits) {
#pragma unroll 1
    for (int j = 0; j < NP; ++j) {
      int jg = j;
      if (flx) jg = mirror_slot<DIM>(0, jg);
      if (fly) jg = mirror_slot<DIM>(1, jg);
      T fj[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c)
        fj[c] = f[(long long)(jg * NF + c) * a.n + g];
      if (flx) fj[1] = -fj[1];
      if (DIM == 2 && fly) fj[2] = -fj[2];
      T feq[NF];
      eq_packet<T, DIM>(q, j, feq);
      // eqs 4-5 as the blend (1 - 1/tau) f + (1/tau) f_eq
      T o[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) o[c] = mad(keep, fj[c], omega * feq[c]);
      r.st(j, i, o);
    }
  }
  if (q.emits) {
    // corner weights as products of (1 - f, f) per axis (eqs 28-29)
    const T g0 = T(1) - q.f0;
    if (DIM == 1) {
      r.wt(0, i) = g0;
      r.wt(1, i) = q.f0;
    } else {
      const T g1 = T(1) - q.f1;
      r.wt(0, i) = g0 * g1;
      r.wt(1, i) = q.f0 * g1;
      r.wt(2, i) = g0 * q.f1;
      r.wt(3, i) = q.f0 * q.f1;
    }
    w = s64_word(q.c1, q.n0, q.n1);
  }
  r.word[i] = w;
}

// Collision of every source of the padded grid into the records.
template <typename T, int DIM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    collide(const Args a) {
  const RecView<T, DIM> r = rec_view<T, DIM>(a);
  const T* f = static_cast<const T*>(a.f);
  const long long PX = (long long)a.nx + 2 * a.rc;
  const long long PY = DIM == 2 ? (long long)a.ny + 2 * a.rc : 1;
  unsigned long long clamps = 0;
  bool bad = false;
  int rmax = 0;
  const long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long py = blockIdx.y; py < PY && px < PX; py += gridDim.y) {
    const long long sx = px - a.rc, sy = DIM == 2 ? py - a.rc : 0;
    const bool owned = sx >= 0 && sx < a.nx && sy >= 0 && sy < a.ny;
    collide_one<T, DIM, false>(a, f, sx, sy, owned, r, py * PX + px, clamps,
                               bad, rmax);
  }
  flag_warp(a.scr, a.rs, clamps, bad, rmax);
}

// Type of a source word as one comparable key: c1, n_x, n_y (c1 = 0xffff:
// the source emits nothing).
__device__ __forceinline__ unsigned long long word_key(long long w) {
  return (unsigned long long)w & 0xffffffffffffull;
}
__device__ __forceinline__ void decode(long long w, int* c1, int* n0,
                                       int* n1) {
  *c1 = (short)(w & 0xffff);
  *n0 = (short)((w >> 16) & 0xffff);
  *n1 = (short)((w >> 32) & 0xffff);
}

// Slots of destination (dx, dy) from a record view; idx(sx, sy) gives a
// source's entry.  one: every source the destination can receive from
// has type (c1, n0, n1) and emits; then slot j's arrivals come from the
// four sources d - n - c'_j - k, in ascending source order corners (1,1),
// (0,1), (1,0), (0,0) (1-D: 1, 0).  Otherwise every source of the (2R +
// 1)^D window is tested once, all slots' sums in registers.  emit(j, v)
// receives the slots in table order.
template <typename T, int DIM, class Idx, class Emit>
__device__ __forceinline__ void gather_one(const RecView<T, DIM>& r, Idx idx,
                                           int dx, int dy, int R, bool one,
                                           int c1, int n0, int n1,
                                           Emit emit) {
  constexpr int NP = Shape<DIM>::NP, NF = Shape<DIM>::NF;
  constexpr int NK = DIM == 1 ? 2 : 4;
  if (one) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      int cx, cy, lev;
      packet<DIM>(j, c1, &cx, &cy, &lev);
      T acc[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) acc[c] = T(0);
#pragma unroll
      for (int kk = 0; kk < NK; ++kk) {
        const int k = NK - 1 - kk;
        const long long i = idx(dx - n0 - cx - (k & 1),
                                DIM == 2 ? dy - n1 - cy - (k >> 1) : 0);
        const T al = r.wt(k, i);
        T fv[NF];
        r.ld(j, i, fv);
#pragma unroll
        for (int c = 0; c < NF; ++c) acc[c] = mad(al, fv[c], acc[c]);
      }
      emit(j, acc);
    }
    return;
  }
  const int Ry = DIM == 2 ? R : 0;
  T acc[NP][NF];
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int c = 0; c < NF; ++c) acc[j][c] = T(0);
  for (int oyo = -Ry; oyo <= Ry; ++oyo) {
    for (int oxo = -R; oxo <= R; ++oxo) {
      const long long i = idx(dx + oxo, dy + oyo);
      int sc1, sn0, sn1;
      decode(r.word[i], &sc1, &sn0, &sn1);
      if (sc1 < 0) continue;
      // destination relative to the source's lattice shift: an arrival
      // needs offset 0 or 1 across the packet's axis
      const int ox = -oxo - sn0;
      const int oy = DIM == 2 ? -oyo - sn1 : 0;
      const int c2 = sc1 + 1;
      const bool xarm = (oy == 0 || oy == 1) && ox >= -c2 && ox <= c2 + 1;
      const bool yarm = DIM == 2 && (ox == 0 || ox == 1) && oy >= -c2 &&
                        oy <= c2 + 1;
      if (!xarm && !yarm) continue;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        int cx, cy, lev;
        packet<DIM>(j, sc1, &cx, &cy, &lev);
        const int kx = ox - cx, ky = oy - cy;
        if (kx < 0 || kx > 1) continue;
        if (DIM == 2 && (ky < 0 || ky > 1)) continue;
        const T al = r.wt(kx + 2 * ky, i);
        T fv[NF];
        r.ld(j, i, fv);
#pragma unroll
        for (int c = 0; c < NF; ++c) acc[j][c] = mad(al, fv[c], acc[j][c]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) emit(j, acc[j]);
}

// Smallest and largest word key over a block of NW warps (every thread
// gets them; one barrier; red holds 2 NW words).
template <int NW = 8>
__device__ __forceinline__ void block_key_range(unsigned long long& lo,
                                                unsigned long long& hi,
                                                unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = lo;
    red[NW + (threadIdx.x >> 5)] = hi;
  }
  __syncthreads();
  lo = red[0];
  hi = red[NW];
#pragma unroll
  for (int w = 1; w < NW; ++w) {
    lo = red[w] < lo ? red[w] : lo;
    hi = red[NW + w] > hi ? red[NW + w] : hi;
  }
}

// Gather of every destination's slots from the records (a 256-node row
// segment in 1-D, a 32 x 8 tile in 2-D per block).  A reach beyond the
// records' padding leaves the state as it was (copied through) and flags
// LBM_EREACH.
template <typename T, int DIM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    gather(const Args a) {
  constexpr int NP = Shape<DIM>::NP, NF = Shape<DIM>::NF;
  constexpr int TXB = DIM == 1 ? 256 : 32, TYB = DIM == 1 ? 1 : 8;
  __shared__ unsigned long long red[16];
  const RecView<T, DIM> r = rec_view<T, DIM>(a);
  const T* fin = static_cast<const T*>(a.f);
  T* fo = static_cast<T*>(a.fo);
  const int R = *reach_slot(a.scr, a.rs);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    *reach_slot(a.scr, a.rs ^ 1) = 0;
  const int x0 = blockIdx.x * TXB, y0 = DIM == 2 ? blockIdx.y * TYB : 0;
  const int dx = x0 + (DIM == 1 ? threadIdx.x : (threadIdx.x & 31));
  const int dy = DIM == 2 ? y0 + (threadIdx.x >> 5) : 0;
  const bool valid = dx < a.nx && dy < a.ny;
  const long long d = (long long)dy * a.nx + dx;
  if (R > a.rc) {  // the same for every thread of the launch
    if (!valid) return;
    if (d == 0) atomicOr(&a.scr->flags, kFlagReach);
    for (int q = 0; q < NP * NF; ++q) fo[q * a.n + d] = fin[q * a.n + d];
    return;
  }
  const long long PX = (long long)a.nx + 2 * a.rc;
  const int rc = a.rc;
  auto idx = [PX, rc](int sx, int sy) -> long long {
    return DIM == 2 ? (long long)(sy + rc) * PX + (sx + rc)
                    : (long long)(sx + rc);
  };
  // does the window of the block's destinations hold one type only?
  const int W = min(TXB, a.nx - x0) + 2 * R;
  const int H = DIM == 2 ? min(TYB, a.ny - y0) + 2 * R : 1;
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int t = threadIdx.x; t < W * H; t += 256) {
    const int ly = t / W, lx = t - ly * W;
    const unsigned long long k =
        word_key(r.word[idx(x0 - R + lx, y0 - (DIM == 2 ? R : 0) + ly)]);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  block_key_range(lo, hi, red);
  if (!valid) return;
  int c1, n0, n1;
  decode((long long)lo, &c1, &n0, &n1);
  gather_one<T, DIM>(r, idx, dx, dy, R, lo == hi && c1 >= 0, c1, n0, n1,
                     [&](int j, const T (&v)[NF]) {
#pragma unroll
                       for (int c = 0; c < NF; ++c)
                         fo[(long long)(j * NF + c) * a.n + d] = v[c];
                     });
}

// Shared memory of the one-launch step (step2d): the collided window of a
// 32 x 8 tile at reach limit rc, (32 + 2 rc) x (8 + 2 rc) sources, each a
// word, 32 packet fields and 4 corner weights.
// Rows of the one-launch step's tile: 16 in FP32 (one 512-thread block per
// multiprocessor: the window of 40 x 24 sources at R = 4 holds 1.9 sources
// per destination), 8 in FP64 (its window's 296-byte sources).
template <typename T>
__host__ __device__ constexpr int step2d_rows() {
  return sizeof(T) == 4 ? 16 : 8;
}
inline size_t step2d_smem(int rc, size_t es) {
  const int ty = es == 4 ? step2d_rows<float>() : step2d_rows<double>();
  return (size_t)(32 + 2 * rc) * (size_t)(ty + 2 * rc) * (8 + 36 * es);
}
// Largest reach limit the one-launch step takes (two blocks per
// multiprocessor in FP32).
constexpr int kStep2dRmax = 4;

// Reach of every node of the state (the first step of the one-launch path
// reads it): into slot rs of the three a step rotates through.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) reach_pass(const Args a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int rm = 0;
  if (i < a.n) {
    T Y[4];
    node_moments<T, DIM>(static_cast<const T*>(a.f), a.n, i, Y);
    rm = node_reach(equilibrium<T, DIM>(Y[0], Y[1], Y[2], Y[3], a.k));
  }
  rm = __reduce_max_sync(0xffffffffu, rm);
  if ((threadIdx.x & 31) == 0 && rm) atomicMax(&a.rslot[a.rs], rm);
}

// One-launch square-lattice step: each block (a 32 x step2d_rows tile)
// collides the sources of its tile's window into shared memory (the same
// values collide() writes), then
// gathers its destinations (the same sums, in the same order, as gather()),
// and forms the new nodes' reach for the next step.  The reach rotates
// through three slots: step s reads slot s % 3, max-reduces the next
// state's reach into slot (s + 1) % 3 and clears slot (s + 2) % 3, which
// the previous step read.
template <typename T>
__global__ void __launch_bounds__(32 * step2d_rows<T>(), 1)
    step2d(const Args a) {
  constexpr int NP = 8, NF = 4;
  constexpr int TY = step2d_rows<T>(), NT = 32 * TY;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[2 * TY];
  const int rc = a.rc;
  const int WM = (32 + 2 * rc) * (TY + 2 * rc);
  RecView<T, 2> r;
  r.cap = WM;
  r.word = reinterpret_cast<long long*>(smem);
  r.v = reinterpret_cast<T*>(r.word + WM);
  const T* fin = static_cast<const T*>(a.f);
  T* fo = static_cast<T*>(a.fo);
  const int rs = a.rs;
  const int R = a.rslot[rs];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    a.rslot[(rs + 2) % 3] = 0;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int dx = x0 + (threadIdx.x & 31), dy = y0 + (threadIdx.x >> 5);
  const bool valid = dx < a.nx && dy < a.ny;
  const long long d = (long long)dy * a.nx + dx;
  if (R > rc) {  // the same for every thread of the launch
    if (!valid) return;
    if (d == 0) atomicOr(&a.scr->flags, kFlagReach);
    for (int q = 0; q < NP * NF; ++q) fo[q * a.n + d] = fin[q * a.n + d];
    return;
  }
  // the window, collided into shared memory
  const int W = 32 + 2 * R, H = TY + 2 * R;
  unsigned long long clamps = 0, lo = ~0ull, hi = 0ull;
  bool bad = false;
  int rdummy = 0;
  for (int t = threadIdx.x; t < W * H; t += NT) {
    const int ly = t / W, lx = t - ly * W;
    const int sx = x0 - R + lx, sy = y0 - R + ly;
    const bool owned = lx >= R && lx < R + 32 && ly >= R && ly < R + TY &&
                       sx < a.nx && sy < a.ny;
    collide_one<T, 2, true>(a, fin, sx, sy, owned, r, t, clamps, bad,
                            rdummy);
    const unsigned long long k = word_key(r.word[t]);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  block_key_range<TY>(lo, hi, red);  // its barrier also publishes the window
  int rm = 0;
  if (valid) {
    int c1, n0, n1;
    decode((long long)lo, &c1, &n0, &n1);
    auto idx = [W, x0, y0, R](int sx, int sy) -> long long {
      return (long long)(sy - y0 + R) * W + (sx - x0 + R);
    };
    // the new node's moments (slots in table order) for its reach
    T Y[4] = {T(0), T(0), T(0), T(0)};
    gather_one<T, 2>(r, idx, dx, dy, R, lo == hi && c1 >= 0, c1, n0, n1,
                     [&](int j, const T (&v)[NF]) {
#pragma unroll
                       for (int c = 0; c < NF; ++c)
                         fo[(long long)(j * NF + c) * a.n + d] = v[c];
                       Y[0] = Y[0] + v[0];
                       Y[1] = Y[1] + v[1];
                       Y[2] = Y[2] + v[2];
                       Y[3] = Y[3] + v[3];
                     });
    rm = node_reach(equilibrium<T, 2>(Y[0], Y[1], Y[2], Y[3], a.k));
  }
  const unsigned wc = __reduce_add_sync(0xffffffffu, (unsigned)clamps);
  const bool wb = __any_sync(0xffffffffu, bad);
  const int wr = __reduce_max_sync(0xffffffffu, rm);
  if ((threadIdx.x & 31) == 0) {
    if (wc) atomicAdd(&a.scr->eclamps, (unsigned long long)wc);
    if (wb) atomicOr(&a.scr->flags, kFlagState);
    if (wr) atomicMax(&a.rslot[(rs + 1) % 3], wr);
  }
}

// Moments of every node (eq 6) into the moments buffer.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) moments(const Args a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  T Y[4];
  node_moments<T, DIM>(static_cast<const T*>(a.f), a.n, i, Y);
  static_cast<T*>(a.mom[0])[i] = Y[0];
  static_cast<T*>(a.mom[1])[i] = Y[1];
  if (DIM == 2) static_cast<T*>(a.mom[2])[i] = Y[2];
  static_cast<T*>(a.mom[3])[i] = Y[3];
}

// Equilibrium packets of the moments buffer into the packets (fo).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) from_moments(const Args a) {
  constexpr int NP = Shape<DIM>::NP, NF = Shape<DIM>::NF;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < a.n) {
    const T rho = static_cast<const T*>(a.mom[0])[i];
    const T mx = static_cast<const T*>(a.mom[1])[i];
    const T my = DIM == 2 ? static_cast<const T*>(a.mom[2])[i] : T(0);
    const T rE = static_cast<const T*>(a.mom[3])[i];
    const Equil<T> q = equilibrium<T, DIM>(rho, mx, my, rE, a.k);
    bad = q.bad;
    T* fo = static_cast<T*>(a.fo);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      T p[NF];
#pragma unroll
      for (int c = 0; c < NF; ++c) p[c] = T(0);
      if (q.emits) eq_packet<T, DIM>(q, j, p);
#pragma unroll
      for (int c = 0; c < NF; ++c) fo[(long long)(j * NF + c) * a.n + i] = p[c];
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicOr(&a.scr->flags, kFlagState);
}

// One packet array between host doubles (physical units) and the state
// (lattice units): x_lattice = x_physical * scale.
template <typename T>
__global__ void __launch_bounds__(256) to_lattice(const double* src, T* dst,
                                                  long long n, double scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)(src[i] * scale);
}
template <typename T>
__global__ void __launch_bounds__(256) to_physical(const T* src, double* dst,
                                                   long long n, double inv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i] * inv;
}

}  // namespace bgk
}  // namespace lbm

// ---------------------------------------------------------------------------
// C ABI (include/lbm.h: lbm_bgk_*)
// ---------------------------------------------------------------------------

using namespace lbm;

struct lbm_bgk {
  lbm_config cfg;
  cudaStream_t stream = nullptr;
  bool f64 = true;
  int dim = 1, np = 5, nf = 3;
  int nx = 1, ny = 1;
  int64_t n = 0;
  double dx = 0.0, lambda = 0.0, tau = 1.0;
  EqConst k{};
  int r_cap = 0;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  void* mom[4] = {nullptr, nullptr, nullptr, nullptr};
  void* rec = nullptr;      // two-kernel step: source records
  bool one_launch = false;  // 2-D with max_reach <= 4: step2d
  size_t smem = 0;          // step2d's dynamic shared memory
  int* rslot = nullptr;     // step2d's three reach slots
  Scratch* scr = nullptr;
  double* part = nullptr;
  int part_cap = 0;
  double* staging = nullptr;  // 5 n doubles
  int64_t steps = 0;
  bool broken = false;
  std::string err;
};

namespace {

lbm_status bfail(lbm_bgk* h, lbm_status st, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (st != LBM_EINVAL) h->broken = true;
  }
  return st;
}

lbm_status bcuda(lbm_bgk* h, cudaError_t e, const char* what) {
  return bfail(h, LBM_ECUDA,
               std::string("lbm_bgk: ") + what + ": " + cudaGetErrorString(e));
}

#define BGK_CUDA(h, call, what)                              \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return bcuda((h), e_, (what));    \
  } while (0)

lbm_status busable(lbm_bgk* h) {
  if (!h) return LBM_EINVAL;
  if (h->broken)
    return bfail(h, LBM_ECUDA, "lbm_bgk: handle is in an error state: " + h->err);
  return LBM_OK;
}

size_t bes(const lbm_bgk* h) { return h->f64 ? 8 : 4; }

bgk::Args args_of(const lbm_bgk* h) {
  bgk::Args a;
  a.f = h->f[h->cur];
  a.fo = h->f[h->cur ^ 1];
  a.rec = h->rec;
  for (int i = 0; i < 4; ++i) a.mom[i] = h->mom[i];
  a.nx = h->nx;
  a.ny = h->ny;
  a.bc_x = h->cfg.bc_x;
  a.bc_y = h->dim == 2 ? h->cfg.bc_y : 0;
  a.rc = h->r_cap;
  a.n = h->n;
  a.omega = 1.0 / h->tau;
  a.keep = 1.0 - a.omega;
  a.omega_f = (float)a.omega;
  a.keep_f = (float)a.keep;
  a.k = h->k;
  a.scr = h->scr;
  a.rs = 0;
  a.rslot = h->rslot;
  return a;
}

unsigned blocks_1d(long long n) { return (unsigned)((n + 255) / 256); }

template <typename T, int DIM>
cudaError_t launch_step_t(const bgk::Args& a, cudaStream_t s) {
  const long long PX = (long long)a.nx + 2 * a.rc;
  const long long PY = DIM == 2 ? (long long)a.ny + 2 * a.rc : 1;
  dim3 cg((unsigned)((PX + 255) / 256), (unsigned)(PY < 65535 ? PY : 65535));
  bgk::collide<T, DIM><<<cg, 256, 0, s>>>(a);
  if (DIM == 1) {
    bgk::gather<T, 1><<<blocks_1d(a.nx), 256, 0, s>>>(a);
  } else {
    dim3 gg((unsigned)((a.nx + 31) / 32), (unsigned)((a.ny + 7) / 8));
    bgk::gather<T, 2><<<gg, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t bgk_launch_step(const lbm_bgk* h, const bgk::Args& a) {
  if (h->one_launch) {
    constexpr int t32 = bgk::step2d_rows<float>(), t64 = bgk::step2d_rows<double>();
    if (h->f64)
      bgk::step2d<double><<<dim3((unsigned)((a.nx + 31) / 32),
                                 (unsigned)((a.ny + t64 - 1) / t64)),
                            32 * t64, h->smem, h->stream>>>(a);
    else
      bgk::step2d<float><<<dim3((unsigned)((a.nx + 31) / 32),
                                (unsigned)((a.ny + t32 - 1) / t32)),
                           32 * t32, h->smem, h->stream>>>(a);
    return cudaGetLastError();
  }
  if (h->f64)
    return h->dim == 1 ? launch_step_t<double, 1>(a, h->stream)
                       : launch_step_t<double, 2>(a, h->stream);
  return h->dim == 1 ? launch_step_t<float, 1>(a, h->stream)
                     : launch_step_t<float, 2>(a, h->stream);
}

// Moments of the current packets into the moments buffer.
cudaError_t launch_moments(const lbm_bgk* h) {
  const bgk::Args a = args_of(h);
  const unsigned g = blocks_1d(h->n);
  if (h->f64) {
    if (h->dim == 1) bgk::moments<double, 1><<<g, 256, 0, h->stream>>>(a);
    else bgk::moments<double, 2><<<g, 256, 0, h->stream>>>(a);
  } else {
    if (h->dim == 1) bgk::moments<float, 1><<<g, 256, 0, h->stream>>>(a);
    else bgk::moments<float, 2><<<g, 256, 0, h->stream>>>(a);
  }
  return cudaGetLastError();
}

// Equilibrium packets of the moments buffer into the current packets.
cudaError_t launch_from_moments(const lbm_bgk* h) {
  bgk::Args a = args_of(h);
  a.fo = h->f[h->cur];
  const unsigned g = blocks_1d(h->n);
  if (h->f64) {
    if (h->dim == 1) bgk::from_moments<double, 1><<<g, 256, 0, h->stream>>>(a);
    else bgk::from_moments<double, 2><<<g, 256, 0, h->stream>>>(a);
  } else {
    if (h->dim == 1) bgk::from_moments<float, 1><<<g, 256, 0, h->stream>>>(a);
    else bgk::from_moments<float, 2><<<g, 256, 0, h->stream>>>(a);
  }
  return cudaGetLastError();
}

lbm_status bcheck_flags(lbm_bgk* h) {
  Scratch s;
  cudaError_t e = cudaMemcpyAsync(&s, h->scr, sizeof(Scratch),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bcuda(h, e, "synchronize");
  if (s.flags & kFlagState)
    return bfail(h, LBM_ESTATE,
                 "lbm_bgk: a node reached rho < 0 or a non-finite moment");
  if (s.flags & kFlagReach)
    return bfail(h, LBM_EREACH,
                 "lbm_bgk: migration reach exceeded max_reach (raise "
                 "lbm_config.max_reach)");
  return LBM_OK;
}

// A new state was set: scratch and step count cleared; the one-launch step
// needs the state's reach before its first step.
lbm_status state_was_set(lbm_bgk* h) {
  BGK_CUDA(h, cudaMemsetAsync(h->scr, 0, sizeof(Scratch), h->stream),
           "scratch clear");
  h->steps = 0;
  if (h->one_launch) {
    BGK_CUDA(h, cudaMemsetAsync(h->rslot, 0, 3 * sizeof(int), h->stream),
             "reach clear");
    const bgk::Args a = args_of(h);
    if (h->f64)
      bgk::reach_pass<double, 2><<<blocks_1d(h->n), 256, 0, h->stream>>>(a);
    else
      bgk::reach_pass<float, 2><<<blocks_1d(h->n), 256, 0, h->stream>>>(a);
    BGK_CUDA(h, cudaGetLastError(), "reach kernel");
  }
  return LBM_OK;
}

// Moments were written into the moments buffer: the packets at equilibrium.
lbm_status seed_from_moments(lbm_bgk* h) {
  BGK_CUDA(h, launch_from_moments(h), "equilibrium kernel");
  return state_was_set(h);
}

}  // namespace

extern "C" {

lbm_status lbm_bgk_create(const lbm_config* cfg, double tau, lbm_bgk** out) {
  if (!cfg || !out) return LBM_EINVAL;
  *out = nullptr;
  const lbm_config& c = *cfg;
  if (!config_ok(c) || c.max_reach > 1024) return LBM_EINVAL;
  // the 2-D gather launch takes 8 rows per block along grid y
  if (c.dim == 2 && (c.ny + 7) / 8 > 65535) return LBM_EINVAL;
  if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;

  lbm_bgk* h = new (std::nothrow) lbm_bgk();
  if (!h) return LBM_ENOMEM;
  h->cfg = c;
  h->stream = (cudaStream_t)c.stream;
  h->f64 = c.precision == LBM_F64;
  h->dim = c.dim;
  h->np = c.dim == 1 ? 5 : 8;
  h->nf = c.dim + 2;
  h->nx = (int)c.nx;
  h->ny = (int)(c.dim == 2 ? c.ny : 1);
  h->n = (int64_t)h->nx * h->ny;
  h->dx = (c.x1 - c.x0) / (double)c.nx;
  h->lambda = c.dt / h->dx;
  h->tau = tau;
  const double D = (double)c.dim;
  h->k.theta = c.dim == 1 ? c.theta : 0.0;
  h->k.kq = D * (c.gamma - 1.0);
  h->k.kphi = 1.0 - 0.5 * D * (c.gamma - 1.0);
  h->k.b1 = c.dim == 1 ? 2.0 : 4.0;
  h->k.kreach = h->k.kq / (1.0 - h->k.theta);
  h->k.set_fp32_copies();
  h->r_cap = c.max_reach > 0 ? c.max_reach : (c.dim == 1 ? 64 : 6);
  h->part_cap = totals_blocks(h->n);
  const size_t fb = bes(h) * (size_t)h->n * (size_t)(h->np * h->nf);
  bool ok = true;
  for (int b = 0; b < 2 && ok; ++b) ok = cudaMalloc(&h->f[b], fb) == cudaSuccess;
  for (int i = 0; i < 4 && ok; ++i) {
    if (i == 2 && c.dim == 1) continue;
    ok = cudaMalloc(&h->mom[i], bes(h) * (size_t)h->n) == cudaSuccess;
  }
  // 2-D with a reach limit the one-launch step's window takes: no records
  h->one_launch = c.dim == 2 && h->r_cap <= bgk::kStep2dRmax;
  if (h->one_launch) {
    h->smem = bgk::step2d_smem(h->r_cap, bes(h));
    const cudaError_t ea =
        h->f64 ? cudaFuncSetAttribute(bgk::step2d<double>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)h->smem)
               : cudaFuncSetAttribute(bgk::step2d<float>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)h->smem);
    if (ea != cudaSuccess) {
      const lbm_status st = bcuda(h, ea, "kernel attribute");
      lbm_bgk_destroy(h);
      return st;
    }
    ok = ok && cudaMalloc(&h->rslot, 3 * sizeof(int)) == cudaSuccess;
  } else {
    ok = ok && cudaMalloc(&h->rec, bgk::rec_bytes(h->dim, h->nx, h->ny,
                                                  h->r_cap, bes(h))) ==
                   cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->scr, sizeof(Scratch)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->part, sizeof(double) * 4 * (size_t)h->part_cap) ==
                 cudaSuccess;
  ok = ok && cudaMalloc(&h->staging, sizeof(double) * 5 * (size_t)h->n) ==
                 cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_bgk_destroy(h);
    return LBM_ENOMEM;
  }
  for (int b = 0; b < 2; ++b) cudaMemsetAsync(h->f[b], 0, fb, h->stream);
  cudaMemsetAsync(h->scr, 0, sizeof(Scratch), h->stream);
  if (h->rslot) cudaMemsetAsync(h->rslot, 0, 3 * sizeof(int), h->stream);
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    const lbm_status st = bcuda(h, e, "initial clear");
    lbm_bgk_destroy(h);
    return st;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_bgk_init_riemann(lbm_bgk* h, const lbm_prim* inner,
                                const lbm_prim* outer, int32_t geom, double a0,
                                double a1, double radius) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!inner || !outer || (geom != LBM_PLANAR_X && geom != LBM_CIRCLE))
    return bfail(h, LBM_EINVAL, "lbm_bgk_init_riemann: bad argument");
  if (!(inner->rho >= 0.0) || !(outer->rho >= 0.0) || !(inner->p >= 0.0) ||
      !(outer->p >= 0.0))
    return bfail(h, LBM_EINVAL, "lbm_bgk_init_riemann: negative rho or p");
  InitArgs a;
  for (int i = 0; i < 4; ++i) a.f[i] = h->mom[i];
  a.nx = h->nx;
  a.ny = h->ny;
  a.dim = h->dim;
  a.x0 = h->cfg.x0;
  a.y0 = h->cfg.y0;
  a.dx = h->dx;
  a.lambda = h->lambda;
  a.gamma = h->cfg.gamma;
  a.geom = geom;
  a.a0 = a0;
  a.a1 = a1;
  a.radius = radius;
  const lbm_prim* s[2] = {inner, outer};
  for (int j = 0; j < 2; ++j) {
    double* d = j == 0 ? a.in_ : a.out_;
    d[0] = s[j]->rho;
    d[1] = s[j]->u;
    d[2] = h->dim == 2 ? s[j]->v : 0.0;
    d[3] = s[j]->p;
  }
  BGK_CUDA(h, launch_init(h->f64, a, h->stream), "init kernel");
  return seed_from_moments(h);
}

lbm_status lbm_bgk_set_moments(lbm_bgk* h, const double* rho, const double* mx,
                               const double* my, const double* rhoE,
                               int64_t n) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!rho || !mx || !rhoE || (h->dim == 2 && !my) || n != h->n)
    return bfail(h, LBM_EINVAL, "lbm_bgk_set_moments: bad arrays or size");
  const size_t nb = sizeof(double) * (size_t)n;
  const double* src[4] = {rho, mx, h->dim == 2 ? my : nullptr, rhoE};
  for (int i = 0; i < 4; ++i)
    if (src[i])
      BGK_CUDA(h, cudaMemcpyAsync(h->staging + (size_t)i * n, src[i], nb,
                                  cudaMemcpyHostToDevice, h->stream),
               "copy to device");
  BGK_CUDA(h, launch_from_host_layout(h->f64, 1, h->dim, h->staging, h->mom, n,
                                      h->lambda, h->cfg.gamma, h->stream),
           "convert kernel");
  st = seed_from_moments(h);
  if (st != LBM_OK) return st;
  BGK_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

// Unit scale of packet field c (lattice = physical * scale): mass 1,
// momentum lambda, energy lambda^2.
static double field_scale(const lbm_bgk* h, int c) {
  if (c == 0) return 1.0;
  if (c == h->nf - 1) return h->lambda * h->lambda;
  return h->lambda;
}

lbm_status lbm_bgk_set_packets(lbm_bgk* h, const double* f, int64_t n) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!f || n != h->n)
    return bfail(h, LBM_EINVAL, "lbm_bgk_set_packets: bad array or size");
  const size_t nb = sizeof(double) * (size_t)n;
  for (int q = 0; q < h->np * h->nf; ++q) {
    BGK_CUDA(h, cudaMemcpyAsync(h->staging, f + (size_t)q * n, nb,
                                cudaMemcpyHostToDevice, h->stream),
             "copy to device");
    const double sc = field_scale(h, q % h->nf);
    if (h->f64)
      bgk::to_lattice<double><<<blocks_1d(n), 256, 0, h->stream>>>(
          h->staging, static_cast<double*>(h->f[h->cur]) + (size_t)q * n, n, sc);
    else
      bgk::to_lattice<float><<<blocks_1d(n), 256, 0, h->stream>>>(
          h->staging, static_cast<float*>(h->f[h->cur]) + (size_t)q * n, n, sc);
    BGK_CUDA(h, cudaGetLastError(), "convert kernel");
  }
  st = state_was_set(h);
  if (st != LBM_OK) return st;
  BGK_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

lbm_status lbm_bgk_packets(lbm_bgk* h, double* f, int64_t n) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!f || n != h->n)
    return bfail(h, LBM_EINVAL, "lbm_bgk_packets: bad array or size");
  const size_t nb = sizeof(double) * (size_t)n;
  for (int q = 0; q < h->np * h->nf; ++q) {
    const double inv = 1.0 / field_scale(h, q % h->nf);
    if (h->f64)
      bgk::to_physical<double><<<blocks_1d(n), 256, 0, h->stream>>>(
          static_cast<const double*>(h->f[h->cur]) + (size_t)q * n, h->staging,
          n, inv);
    else
      bgk::to_physical<float><<<blocks_1d(n), 256, 0, h->stream>>>(
          static_cast<const float*>(h->f[h->cur]) + (size_t)q * n, h->staging,
          n, inv);
    BGK_CUDA(h, cudaGetLastError(), "convert kernel");
    BGK_CUDA(h, cudaMemcpyAsync(f + (size_t)q * n, h->staging, nb,
                                cudaMemcpyDeviceToHost, h->stream),
             "copy to host");
    // the staging buffer is reused by the next array
    BGK_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  }
  return bcheck_flags(h);
}

lbm_status lbm_bgk_step(lbm_bgk* h, int64_t nsteps) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (nsteps < 0) return bfail(h, LBM_EINVAL, "lbm_bgk_step: nsteps < 0");
  for (int64_t s = 0; s < nsteps; ++s) {
    bgk::Args a = args_of(h);
    a.rs = h->one_launch ? (int)(h->steps % 3) : (int)(h->steps & 1);
    BGK_CUDA(h, bgk_launch_step(h, a), "step kernels");
    h->cur ^= 1;
    h->steps += 1;
  }
  return LBM_OK;
}

lbm_status lbm_bgk_moments(lbm_bgk* h, double* rho, double* mx, double* my,
                           double* rhoE, double* p, int64_t n) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!rho || !mx || !rhoE || n != h->n)
    return bfail(h, LBM_EINVAL, "lbm_bgk_moments: bad arrays or size");
  BGK_CUDA(h, launch_moments(h), "moments kernel");
  BGK_CUDA(h, launch_to_host_layout(h->f64, h->dim, h->mom, h->staging, n,
                                    h->lambda, h->cfg.gamma, h->stream),
           "readback kernel");
  const size_t nb = sizeof(double) * (size_t)n;
  double* dst[5] = {rho, mx, h->dim == 2 ? my : nullptr, rhoE, p};
  for (int i = 0; i < 5; ++i)
    if (dst[i])
      BGK_CUDA(h, cudaMemcpyAsync(dst[i], h->staging + (size_t)i * n, nb,
                                  cudaMemcpyDeviceToHost, h->stream),
               "copy to host");
  return bcheck_flags(h);
}

lbm_status lbm_bgk_conservation(lbm_bgk* h, double out[4]) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  if (!out) return bfail(h, LBM_EINVAL, "lbm_bgk_conservation: NULL out");
  BGK_CUDA(h, launch_moments(h), "moments kernel");
  BGK_CUDA(h, launch_totals(h->f64, h->dim, h->mom, h->n, h->part, h->part_cap,
                            h->scr, h->stream),
           "totals kernel");
  st = bcheck_flags(h);
  if (st != LBM_OK) return st;
  Scratch sc;
  BGK_CUDA(h, cudaMemcpyAsync(&sc, h->scr, sizeof(Scratch),
                              cudaMemcpyDeviceToHost, h->stream),
           "copy totals");
  BGK_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  out[0] = sc.cons[0];
  out[1] = sc.cons[1] / h->lambda;
  out[2] = sc.cons[2] / h->lambda;
  out[3] = sc.cons[3] / (h->lambda * h->lambda);
  return LBM_OK;
}

lbm_status lbm_bgk_diagnostics(lbm_bgk* h, int64_t* steps, int64_t* eclamps,
                               int32_t* reach, uint32_t* flags) {
  if (!h) return LBM_EINVAL;
  Scratch s;
  int rs[3] = {0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(&s, h->scr, sizeof(Scratch),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && h->one_launch)
    e = cudaMemcpyAsync(rs, h->rslot, sizeof(rs), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bcuda(h, e, "diagnostics");
  if (steps) *steps = h->steps;
  if (eclamps) *eclamps = (int64_t)s.eclamps;
  // the slot of the last step (0 before the first)
  if (reach) {
    if (h->one_launch)
      *reach = h->steps > 0 ? rs[(h->steps - 1) % 3] : 0;
    else
      *reach = (h->steps & 1) ? s.reach : s.reach_next;
  }
  if (flags) *flags = s.flags;
  return LBM_OK;
}

lbm_status lbm_bgk_synchronize(lbm_bgk* h) {
  lbm_status st = busable(h);
  if (st != LBM_OK) return st;
  return bcheck_flags(h);
}

const char* lbm_bgk_last_error(const lbm_bgk* h) {
  return h ? h->err.c_str() : "lbm_bgk: NULL handle";
}

void lbm_bgk_destroy(lbm_bgk* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b)
    if (h->f[b]) cudaFree(h->f[b]);
  for (int i = 0; i < 4; ++i)
    if (h->mom[i]) cudaFree(h->mom[i]);
  if (h->rec) cudaFree(h->rec);
  if (h->rslot) cudaFree(h->rslot);
  if (h->scr) cudaFree(h->scr);
  if (h->part) cudaFree(h->part);
  if (h->staging) cudaFree(h->staging);
  cudaGetLastError();
  delete h;
}

}  // extern "C"
