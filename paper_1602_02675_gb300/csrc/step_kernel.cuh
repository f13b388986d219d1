// Fused tau = 1 step: equilibrium + migration + summation + reach, one launch.
//
// One block owns a tile of destination nodes (1-D: 16, 32 or 256 x 1 by the
// tube's length, 2-D: 32 x 8; one destination per thread).  It
//  1. computes the equilibrium packets of every source node within the
//     migration reach R of the tile once (Section III.B eqs 13-15, 24-26;
//     packets eqs 11-14, 21; split weights eq 23, 28, 29) and keeps them in
//     shared memory; sources beyond the domain edge are the additional points
//     of Section V.B (zero-gradient, periodic image or mirror image);
//  2. lets each thread gather the arrivals at its destination (eqs 6, 10,
//     22): source rows at distance j below and above the destination are
//     summed row by row (ascending x, packet table order, corner order) and
//     added as pairs, j = 0..R.  The order is the same relative to every
//     destination and symmetric under y -> -y.  A square-lattice window
//     whose sources share one type visits its 32 landings from a
//     compile-time list in that order; other windows test every candidate;
//  3. writes the new moments, reduces a conservative reach for the next step
//     and, when asked, FP64 totals; the last block to finish publishes them.
// No floating-point atomics anywhere; every sum has a fixed order.
//
// FP64 square-lattice handles step with step2d_rec (step_rec.cuh) instead:
// the same gather and sums, reading packets that a records pass formed once
// per source; this kernel serves that case for lbm_step_noalloc, which has
// no room for the records.
#pragma once

#include <cstdint>

#include "fp32_arith.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int DIM>
struct TileShape;
template <>
struct TileShape<1> {
  static constexpr int TX = 256, TY = 1, NP = 5, NK = 2, NLEV = 3;
};
template <>
struct TileShape<2> {
  static constexpr int TX = 32, TY = 8, NP = 8, NK = 4, NLEV = 2;
};

// 1-D tile width of the exact-order kernel for a tube of nx nodes on a
// device with `sms` multiprocessors: 256 once such tiles give two blocks per
// multiprocessor; below that 32-thread blocks with narrow tiles, so that
// short tubes spread over many multiprocessors (the FP64 rate per
// multiprocessor is low) and the window of a tile (its width + 2 R sources)
// is formed in one pass of the block's 32 threads.  Each destination's sum
// order does not depend on the tile.
__host__ __device__ inline int step_tile_1d(int nx, int sms) {
  const long long n = nx;
  return n < 2LL * sms * 256 ? (n <= 16LL * sms ? 16 : 32) : 256;
}

// Shared-memory layout of the source records, structure of arrays, sized
// for r_cap and a tile TXW destinations wide.  Per source: packet fields Px,
// Py (2-D), PE per packet, the mass per level, the split fraction f (1-D)
// or the four corner weights (2-D, eq 29: (1-f_x)(1-f_y), f_x(1-f_y),
// (1-f_x)f_y, f_x f_y), and packed integers (c1, n_x, n_y).
template <typename T, int DIM, int TXW = TileShape<DIM>::TX>
struct SrcLayout {
  using S = TileShape<DIM>;
  int cap;  // sources the buffers hold
  T* Px;
  T* Py;
  T* PE;
  T* mass;
  T* f0;  // 1-D
  T* wt;  // 2-D, corner k at wt[k * cap + source]
  short* c1;
  short* n0;
  short* n1;

  __host__ __device__ static int capacity(int r_cap) {
    return (TXW + 2 * r_cap) * (DIM == 2 ? (S::TY + 2 * r_cap) : 1);
  }
  __host__ __device__ static size_t bytes(int r_cap) {
    size_t c = (size_t)capacity(r_cap);
    size_t nt = (size_t)S::NP * (DIM == 2 ? 3 : 2) + S::NLEV + (DIM == 2 ? 4 : 1);
    size_t b = c * nt * sizeof(T) + c * 3 * sizeof(short);
    return (b + 15) & ~size_t(15);
  }
  __device__ void bind(unsigned char* base, int r_cap) {
    cap = capacity(r_cap);
    T* p = reinterpret_cast<T*>(base);
    Px = p;
    p += S::NP * cap;
    if (DIM == 2) {
      Py = p;
      p += S::NP * cap;
    } else {
      Py = nullptr;
    }
    PE = p;
    p += S::NP * cap;
    mass = p;
    p += S::NLEV * cap;
    if (DIM == 2) {
      f0 = nullptr;
      wt = p;
      p += 4 * cap;
    } else {
      f0 = p;
      wt = nullptr;
      p += cap;
    }
    short* q = reinterpret_cast<short*>(p);
    c1 = q;
    n0 = q + cap;
    n1 = q + 2 * cap;
  }
};

// Interior node supplying the state of source coordinate L on one axis, and
// the sign of the momentum component along that axis there (Section V.B).
__device__ __forceinline__ int virtual_axis(int bc, int n, long long L,
                                            bool* flip) {
  *flip = false;
  if (L >= 0 && L < n) return (int)L;
  if (bc == 0) return L < 0 ? 0 : n - 1;  // transmissive: zero gradient
  if (bc == 2) {                          // periodic
    long long w = L % n;
    return (int)(w < 0 ? w + n : w);
  }
  long long p2 = 2LL * n;                 // reflecting: mirror, period 2n
  long long w = L % p2;
  if (w < 0) w += p2;
  if (w >= n) {
    *flip = true;
    return (int)(p2 - 1 - w);
  }
  return (int)w;
}

template <typename T>
struct Equil {
  bool emits, bad, clamp;
  T V0, V1, e, d0, d1, d2, phi, f0, f1;
  int c1, n0, n1;
};

__device__ __forceinline__ float dev_floor(float x) { return floorf(x); }
__device__ __forceinline__ double dev_floor(double x) { return floor(x); }

// A constant of the equilibrium in the step's type: FP64 kernels take the
// double, FP32 kernels the copy rounded to FP32 on the host (the same value
// a conversion on the GPU gives).
template <typename T>
__device__ __forceinline__ T eq_const(double d, float f);
template <>
__device__ __forceinline__ double eq_const<double>(double d, float) {
  return d;
}
template <>
__device__ __forceinline__ float eq_const<float>(double, float f) {
  return f;
}

// Estimate of floor(sqrt(X)) for 0 <= X <= 2^40, within one of the exact
// value: X rounded to FP32 and its correctly rounded FP32 square root are
// within 1.5 * 2^-24 sqrt(X) of sqrt(X), less than 0.1 for X <= 2^40.  (The
// FP64 square root would take a long chain of FP64 operations for the same
// integer.)
__device__ __forceinline__ int isqrt_estimate(double X) {
  return (int)floorf(sqrtf((float)X));
}
__device__ __forceinline__ int isqrt_estimate(float X) {
  return (int)floorf(sqrtf(X));
}

// Lattice shift n = floor(V) and split fraction f = V - n per axis (eqs
// 23, 28, 29).
template <typename T>
__device__ __forceinline__ void equil_split(Equil<T>& q) {
  T fl0 = dev_floor(q.V0);
  q.n0 = (int)fl0;
  q.f0 = q.V0 - fl0;
  T fl1 = dev_floor(q.V1);
  q.n1 = (int)fl1;
  q.f1 = q.V1 - fl1;
}

// Equilibrium of one node (Section III.B): V and e (eq 13, eq 15 text),
// c1 = int(sqrt(D (gamma-1) e rho / (rho - b0 d0))), c2 = c1 + 1 (eq 26),
// d1, d2 (eqs 24-25), phi (eq 15), floor/fraction of V (eqs 23, 28, 29).
template <typename T, int DIM>
__device__ __forceinline__ Equil<T> equilibrium(T rho, T mx, T my, T rhoE,
                                                const EqConst& k) {
  Equil<T> q;
  q.emits = false;
  q.bad = false;
  q.clamp = false;
  if (!isfinite(rho) || !isfinite(mx) || !isfinite(my) || !isfinite(rhoE) ||
      rho < T(0)) {
    q.bad = true;
    return q;
  }
  if (rho == T(0)) return q;
  q.V0 = mx / rho;
  q.V1 = (DIM == 2) ? my / rho : T(0);
  T E = rhoE / rho;
  T e = E - T(0.5) * (q.V0 * q.V0 + q.V1 * q.V1);
  if (e < T(0)) {
    e = T(0);
    q.clamp = true;
  }
  q.e = e;
  T d0 = (DIM == 1) ? eq_const<T>(k.theta, k.theta_f) * rho : T(0);
  T rho_p = rho - T(1) * d0;
  T Q = eq_const<T>(k.kq, k.kq_f) * rho * e;
  T X = Q / rho_p;
  // X beyond 2^40 would mean c1 > 2^20: far past any supported reach
  if (!isfinite(X) || !(X >= T(0)) || X > T(1099511627776.0)) {
    q.bad = true;
    return q;
  }
  // c1 is the integer floor(sqrt(X)), fixed by c1^2 <= X < (c1+1)^2: an
  // estimate within one of it and one exact fix-up each way give it
  int c1 = isqrt_estimate(X);
  if ((T)((long long)(c1 + 1) * (c1 + 1)) <= X) ++c1;
  if (c1 > 0 && (T)((long long)c1 * c1) > X) --c1;
  q.c1 = c1;
  T c1sq = (T)(c1 * c1);
  T c2sq = (T)((c1 + 1) * (c1 + 1));
  T den = eq_const<T>(k.b1, k.b1_f) * (c2sq - c1sq);
  q.d0 = d0;
  q.d1 = (c2sq * rho_p - Q) / den;
  q.d2 = (Q - c1sq * rho_p) / den;
  if (sizeof(T) == sizeof(float)) {
    // eq 15 as e - (D/2)(gamma-1) e: the packets then carry exactly
    // rho e = rho phi + Q/2 up to unbiased rounding; with the FP32-rounded
    // constants kphi + kq/2 != 1 and every step would add a fixed bias
    q.phi = e - T(0.5) * (eq_const<T>(k.kq, k.kq_f) * e);
  } else {
    q.phi = eq_const<T>(k.kphi, k.kphi_f) * e;
  }
  equil_split(q);
  q.emits = true;
  return q;
}

// Packet p of the velocity set (Section IV): lattice offset and level.
//   1-D: (0; d0), (+c1; d1), (-c1; d1), (+c2; d2), (-c2; d2)
//   2-D: (+c1 ex), (-c1 ex), (+c1 ey), (-c1 ey) with d1, then the same with
//        c2 and d2.
template <int DIM>
__device__ __forceinline__ void packet(int p, int c1, int* cx, int* cy,
                                       int* lev) {
  if (DIM == 1) {
    int c = (p == 0) ? 0 : (p <= 2 ? c1 : c1 + 1);
    *cx = (p == 2 || p == 4) ? -c : c;
    *cy = 0;
    *lev = (p == 0) ? 0 : (p <= 2 ? 1 : 2);
  } else {
    int lv = p >> 2;  // 0 -> level 1, 1 -> level 2
    int c = c1 + lv;
    int j = p & 3;
    *cx = (j == 0) ? c : (j == 1 ? -c : 0);
    *cy = (j == 2) ? c : (j == 3 ? -c : 0);
    *lev = lv;  // index into the 2-D mass slots (d1, d2)
  }
}

// Fields of packet p of an emitting node (eqs 11-14, 21): momentum d (V +
// c') per axis and energy d (|V + c'|^2 / 2 + phi).
template <typename T, int DIM>
__device__ __forceinline__ void packet_fields(const Equil<T>& q, int p,
                                              T* px, T* py, T* pe) {
  int cx, cy, lev;
  packet<DIM>(p, q.c1, &cx, &cy, &lev);
  const T d = DIM == 1 ? (lev == 0 ? q.d0 : (lev == 1 ? q.d1 : q.d2))
                       : (lev == 0 ? q.d1 : q.d2);
  T cbx = q.V0 + (T)cx;  // eq 12: V + c'
  if (DIM == 1) {
    *px = d * cbx;
    *py = T(0);
    *pe = d * (T(0.5) * (cbx * cbx) + q.phi);
  } else {
    T cby = q.V1 + (T)cy;
    *px = d * cbx;
    *py = d * cby;
    *pe = d * (T(0.5) * (cbx * cbx + cby * cby) + q.phi);
  }
}

// Square-lattice source records (step_rec.cuh), written for every node and
// every additional point before each step by a records pass and read by the
// step's gather instead of forming each window source's equilibrium again.
// Structure of arrays over the grid padded by r_cap on every side (source
// (x, y) at (y + r_cap) * (nx + 2 r_cap) + x + r_cap), one element of the
// step's type per source each: P_x of packets 0-7, P_y of 0-7, P_E of 0-7,
// d1, d2, the four corner weights, then one array of 64-bit words holding
// c1, n_x, n_y as 16-bit fields (c1 = -1: the source emits nothing).
enum : int {
  kRecPx = 0,
  kRecPy = 8,
  kRecPE = 16,
  kRecMass = 24,
  kRecW = 26,
  kRecWord = 30,
  kRecArrays = 31
};

// Corner weights of a square-lattice source (eq 29), in corner order
// (0,0), (1,0), (0,1), (1,1): products of (1 - f, f) per axis.
template <typename T>
__device__ __forceinline__ void corner_weights(const Equil<T>& q, T (&w)[4]) {
  const T wx0 = T(1) - q.f0, wy0 = T(1) - q.f1;
  w[0] = wx0 * wy0;
  w[1] = q.f0 * wy0;
  w[2] = wx0 * q.f1;
  w[3] = q.f0 * q.f1;
}

__device__ __forceinline__ long long s64_word(int c1, int n0, int n1) {
  return (long long)(unsigned short)(short)c1 |
         ((long long)(unsigned short)(short)n0 << 16) |
         ((long long)(unsigned short)(short)n1 << 32);
}

// Conservative migration reach of one node: >= floor(|V_a|) + 1 + c2 as the
// step computes them, evaluated in FP32 with margins that cover its rounding
// (an over-estimate only widens the source window).
__device__ __forceinline__ int reach_bound(double rho, double mx, double my,
                                           double rhoE, float kreach) {
  if (!(rho > 0.0)) return 0;
  float inv = 1.0f / (float)rho;
  float v0 = fabsf((float)mx) * inv;
  float v1 = fabsf((float)my) * inv;
  float E = (float)rhoE * inv;
  float kin = 0.5f * (v0 * v0 + v1 * v1);
  float e = E - kin + 1e-5f * (fabsf(E) + kin);
  e = fmaxf(e, 0.0f);
  float X = kreach * e * 1.0001f;
  float c1 = floorf(sqrtf(X));
  float v = floorf(fmaxf(v0, v1) * 1.00001f);
  float r = v + 1.0f + c1 + 1.0f;
  return r > 1.0e8f ? 100000000 : (int)r;
}

// Adds a row pair's sums to a destination's totals (plain, or compensated
// when KAHAN).
template <typename T, bool KAHAN>
__device__ __forceinline__ void add_pair(T (&tot)[4], T (&comp)[4],
                                         const T (&pair)[4]) {
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (KAHAN) {
      T yk = pair[f] - comp[f];
      T t = tot[f] + yk;
      comp[f] = (t - tot[f]) - yk;
      tot[f] = t;
    } else {
      tot[f] = tot[f] + pair[f];
    }
  }
}

// ---- square lattice, uniform window ----
// When every source of the block's window emits with the same level c1 and
// the same lattice shift (n_x, n_y) = floor(V) (eqs 23, 29), packet p and
// corner k of the source at offset a from a destination land on it exactly
// when a = -(n + c'_p + k), so each of the 32 landings comes from a source
// at a compile-time offset.  RowLandingList holds them in the order of the
// scan in step 2: rows by j = |a_y| (a_y = -j first), then a_x, packet,
// corner.  Visiting them with the same row, pair and total sums gives the
// scan's result bit for bit: the scan's other candidates contribute no
// term.
__host__ __device__ constexpr int sq_cx(int p, int c1) {
  return (p & 3) == 0 ? c1 + (p >> 2) : ((p & 3) == 1 ? -(c1 + (p >> 2)) : 0);
}
__host__ __device__ constexpr int sq_cy(int p, int c1) {
  return (p & 3) == 2 ? c1 + (p >> 2) : ((p & 3) == 3 ? -(c1 + (p >> 2)) : 0);
}

struct RowLanding {
  int j, side, ax, p, k;
};

template <int C1, int NX, int NY>
struct RowLandingList {
  static constexpr int N = 32;
  RowLanding v[N];
  __host__ __device__ constexpr RowLandingList() : v{} {
    int n = 0;
    for (int p = 0; p < 8; ++p)
      for (int k = 0; k < 4; ++k) {
        const int ax = -(NX + sq_cx(p, C1) + (k & 1));
        const int ay = -(NY + sq_cy(p, C1) + (k >> 1));
        v[n] = RowLanding{ay < 0 ? -ay : ay, ay > 0 ? 1 : 0, ax, p, k};
        ++n;
      }
    for (int a = 1; a < N; ++a) {
      RowLanding x = v[a];
      int b = a - 1;
      while (b >= 0 && before(x, v[b])) {
        v[b + 1] = v[b];
        --b;
      }
      v[b + 1] = x;
    }
  }
  __host__ __device__ static constexpr bool before(const RowLanding& x,
                                                   const RowLanding& y) {
    if (x.j != y.j) return x.j < y.j;
    if (x.side != y.side) return x.side < y.side;
    if (x.ax != y.ax) return x.ax < y.ax;
    if (x.p != y.p) return x.p < y.p;
    return x.k < y.k;
  }
  // first landing of row (j, side) and one past its last
  __host__ __device__ constexpr int begin(int j, int side) const {
    int i = 0;
    while (i < N && (v[i].j < j || (v[i].j == j && v[i].side < side))) ++i;
    return i;
  }
  __host__ __device__ constexpr int end(int j, int side) const {
    int i = begin(j, side);
    while (i < N && v[i].j == j && v[i].side == side) ++i;
    return i;
  }
  __host__ __device__ constexpr int jmax() const { return v[N - 1].j; }
};

// Landings I .. E-1 of one row into the row sums r (the scan's expressions:
// corner weight (eq 29) times the packet's mass, momentum and energy).
// srow: the slot of the row's source at a_x = 0.  ASSIGN: the first landing
// of the row sets r instead of adding to a zero.
template <typename T, class LL, int I, int E, bool ASSIGN, typename Lay,
          typename Idx>
__device__ __forceinline__ void row_range(const Lay& L, Idx srow, T (&r)[4]) {
  if constexpr (I < E) {
    constexpr LL ll{};
    constexpr RowLanding q = ll.v[I];
    constexpr bool first = I == 0 || ll.v[I - 1].j != q.j ||
                           ll.v[I - 1].side != q.side;
    const Idx s = srow + q.ax;
    const T al = L.wt[q.k * L.cap + s];
    const T m = L.mass[(q.p >> 2) * L.cap + s];
    const T px = L.Px[q.p * L.cap + s];
    const T py = L.Py[q.p * L.cap + s];
    const T pe = L.PE[q.p * L.cap + s];
    if constexpr (ASSIGN && first) {
      r[0] = al * m;
      r[1] = al * px;
      r[2] = al * py;
      r[3] = al * pe;
    } else {
      r[0] = r[0] + al * m;
      r[1] = r[1] + al * px;
      r[2] = r[2] + al * py;
      r[3] = r[3] + al * pe;
    }
    row_range<T, LL, I + 1, E, ASSIGN>(L, srow, r);
  }
}

// Rows J .. jmax of a uniform window; s0: the destination's slot, W: the
// distance between the slots of vertically adjacent sources.
//
// Compensated (KAHAN): the scan's sums operation for operation.  Plain: a
// row sum starts from its first term instead of zero, a row without
// landings adds nothing, and rows beyond jmax are not visited.  That can
// only change the sign of a zero row or pair sum, and the destination's
// total, which starts at +0 and is never -0 under round-to-nearest,
// absorbs it: total + (+0) and total + (-0) are the same number.  So the
// totals stay bit-identical with the scan's.
template <typename T, bool KAHAN, class LL, int J, typename Lay, typename Idx>
__device__ __forceinline__ void uniform_rows(const Lay& L, Idx s0, Idx W,
                                             T (&tot)[4], T (&comp)[4]) {
  constexpr LL ll{};
  if constexpr (J <= ll.jmax()) {
    constexpr int b0 = ll.begin(J, 0), e0 = ll.end(J, 0);
    constexpr int b1 = J > 0 ? ll.begin(J, 1) : 0, e1 = J > 0 ? ll.end(J, 1) : 0;
    if constexpr (KAHAN) {
      T pair[4];
      {
        T r[4] = {T(0), T(0), T(0), T(0)};
        row_range<T, LL, b0, e0, false>(L, s0 - J * W, r);
#pragma unroll
        for (int f = 0; f < 4; ++f) pair[f] = r[f];
      }
      if constexpr (J > 0) {
        T r[4] = {T(0), T(0), T(0), T(0)};
        row_range<T, LL, b1, e1, false>(L, s0 + J * W, r);
#pragma unroll
        for (int f = 0; f < 4; ++f) pair[f] = pair[f] + r[f];
      }
      add_pair<T, KAHAN>(tot, comp, pair);
    } else {
      constexpr bool has0 = b0 < e0, has1 = b1 < e1;
      if constexpr (has0 || has1) {
        T pair[4];
        if constexpr (has0) row_range<T, LL, b0, e0, true>(L, s0 - J * W, pair);
        if constexpr (has1) {
          T r[4];
          row_range<T, LL, b1, e1, true>(L, s0 + J * W, r);
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            if constexpr (has0)
              pair[f] = pair[f] + r[f];
            else
              pair[f] = r[f];
          }
        }
        add_pair<T, KAHAN>(tot, comp, pair);
      }
    }
    uniform_rows<T, KAHAN, LL, J + 1>(L, s0, W, tot, comp);
  }
}

// A uniform window's gather: the compile-time rows, then (compensated sums
// only) rows jmax+1 .. R, which hold no landing: their pair sums are zero,
// added as the scan adds them, because the compensation term makes such an
// addition change the total.
template <typename T, bool KAHAN, int C1, int NX, int NY, typename Lay,
          typename Idx>
__device__ __forceinline__ void uniform_gather(const Lay& L, Idx s0, Idx W,
                                               int R, T (&tot)[4],
                                               T (&comp)[4]) {
  using LL = RowLandingList<C1, NX, NY>;
  uniform_rows<T, KAHAN, LL, 0>(L, s0, W, tot, comp);
  if constexpr (KAHAN) {
    for (int j = LL{}.jmax() + 1; j <= R; ++j) {
      T pair[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int f = 0; f < 4; ++f) pair[f] = pair[f] + T(0);
      add_pair<T, KAHAN>(tot, comp, pair);
    }
  }
}

// Type word of a source for the uniformity test: 0 if it does not emit,
// else bit 31, c1 (bits 16..23) and n_x, n_y + 128 (bits 8..15, 0..7),
// each clamped so that no other value aliases the fast path's.
__device__ __forceinline__ unsigned window_type(bool emits, int c1, int n0,
                                                int n1) {
  if (!emits) return 0u;
  const unsigned c = (unsigned)min(c1, 255);
  const unsigned ux = (unsigned)(min(max(n0, -128), 127) + 128);
  const unsigned uy = (unsigned)(min(max(n1, -128), 127) + 128);
  return 0x80000000u | (c << 16) | (ux << 8) | uy;
}

template <typename T>
__device__ __forceinline__ T ld(const void* p, long long i) {
  return reinterpret_cast<const T*>(p)[i];
}

// Warp 0 of a block: lane 8 f + w takes warp w's compensated partial of
// field f (NW <= 8 warps, the rest zero) and the xor 4, 2, 1 exchanges
// combine them in a fixed pairing; lanes 8 f return field f.
template <int NW>
__device__ __forceinline__ Sum2 combine_warps_f2(const float2 (&red)[4][NW],
                                                 int lane) {
  static_assert(NW <= 8, "one lane per (field, warp)");
  const int w = lane & 7;
  const float2 h = w < NW ? red[lane >> 3][w] : make_float2(0.f, 0.f);
  Sum2 b{h.x, h.y};
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) b = sum2_add(b, sum2_shfl_xor(b, off));
  return b;
}

// Step 3 of a step launch (all NT threads of the block call it): write the
// destination's new moments (tot; valid: the thread has a destination at
// (dx, dy)), reduce a conservative reach for the next step and, when asked,
// the block's FP64 partial totals; the last block to finish combines the
// partials in a fixed order and publishes reach and totals.
template <typename T, int DIM, int NT>
__device__ __forceinline__ void step_finish(const StepArgs& a, bool valid,
                                            int dx, int dy,
                                            const T (&tot)[4]) {
  __shared__ double red_sum[4][NT / 32];
  __shared__ float2 red_f2[4][NT / 32];
  __shared__ int red_reach[NT / 32];
  __shared__ int is_last;
  const int tid = threadIdx.x;
  int my_reach = 0;
  if (valid) {
    const long long o = (long long)dy * a.nx + dx;
    reinterpret_cast<T*>(a.out[0])[o] = tot[0];
    reinterpret_cast<T*>(a.out[1])[o] = tot[1];
    if (DIM == 2) reinterpret_cast<T*>(a.out[2])[o] = tot[2];
    reinterpret_cast<T*>(a.out[3])[o] = tot[3];
    if constexpr (sizeof(T) == sizeof(float))
      my_reach = reach_bound_f32(tot[0], tot[1], DIM == 2 ? tot[2] : 0.0f,
                                 tot[3], a.k.kreach_f);
    else
      my_reach = reach_bound((double)tot[0], (double)tot[1],
                             DIM == 2 ? (double)tot[2] : 0.0, (double)tot[3],
                             (float)a.k.kreach);
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    my_reach = max(my_reach, __shfl_xor_sync(0xffffffffu, my_reach, off));
  if (a.do_cons) {
    if constexpr (sizeof(T) == sizeof(float)) {
      // FP32: compensated FP32 sums (the FP64 pipe is 1/64 of FP32 on this
      // GPU), per warp here and over the warps below
      Sum2 p4[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) p4[f] = Sum2{valid ? (float)tot[f] : 0.0f, 0.0f};
      const Sum2 k = warp_sum2_fields(p4, lane);
      if ((lane & 7) == 0) red_f2[lane >> 3][warp] = make_float2(k.hi, k.lo);
    } else {
      double ps[4] = {0.0, 0.0, 0.0, 0.0};
      if (valid) {
#pragma unroll
        for (int f = 0; f < 4; ++f) ps[f] = (double)tot[f];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
          ps[f] += __shfl_down_sync(0xffffffffu, ps[f], off);
      if (lane == 0) {
#pragma unroll
        for (int f = 0; f < 4; ++f) red_sum[f][warp] = ps[f];
      }
    }
  }
  if (lane == 0) red_reach[warp] = my_reach;
  __syncthreads();
  const int nblk = a.nblocks;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  double bs[4] = {0.0, 0.0, 0.0, 0.0};
  float2 bf[4];  // FP32: the block's compensated partials (hi, lo)
  if constexpr (sizeof(T) == sizeof(float)) {
    if (warp == 0 && a.do_cons) {
      const Sum2 b = combine_warps_f2<NT / 32>(red_f2, lane);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        bf[f] = make_float2(__shfl_sync(0xffffffffu, b.hi, 8 * f),
                            __shfl_sync(0xffffffffu, b.lo, 8 * f));
    }
  }
  if (tid == 0) {
    int rb = red_reach[0];
    if constexpr (sizeof(T) != sizeof(float)) {
#pragma unroll
      for (int f = 0; f < 4; ++f) bs[f] = red_sum[f][0];
    }
    for (int w = 1; w < NT / 32; ++w) {
      rb = max(rb, red_reach[w]);
      if constexpr (sizeof(T) != sizeof(float)) {
#pragma unroll
        for (int f = 0; f < 4; ++f) bs[f] += red_sum[f][w];
      }
    }
    atomicMax(&a.scr->reach_next, rb);
    if (a.do_cons) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if constexpr (sizeof(T) == sizeof(float))
          reinterpret_cast<float2*>(a.part)[(long long)bid * 4 + f] = bf[f];
        else
          a.part[(long long)bid * 4 + f] = bs[f];
      }
    }
    __threadfence();
    unsigned done = atomicAdd(&a.scr->ticket, 1u);
    is_last = (done == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!is_last) return;

  // ---- last block: publish reach and totals (fixed order) ----
  __threadfence();
  if constexpr (sizeof(T) == sizeof(float)) {
    if (a.do_cons) {
      // the blocks' (hi, lo) partials in compensated FP32 sums, each
      // thread a fixed strided set, then the warps and the block as above
      Sum2 s4[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      for (int b = tid; b < nblk; b += NT) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float2 v =
              __ldcg(&reinterpret_cast<const float2*>(a.part)[(long long)b * 4 + f]);
          s4[f] = sum2_add(s4[f], Sum2{v.x, v.y});
        }
      }
      const Sum2 k = warp_sum2_fields(s4, lane);
      if ((lane & 7) == 0) red_f2[lane >> 3][warp] = make_float2(k.hi, k.lo);
      __syncthreads();
      if (warp == 0) {
        const Sum2 b = combine_warps_f2<NT / 32>(red_f2, lane);
        if ((lane & 7) == 0) a.scr->cons[lane >> 3] = (double)b.hi + (double)b.lo;
      }
    }
  } else if (a.do_cons) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < nblk; b += NT) {
#pragma unroll
      for (int f = 0; f < 4; ++f) s[f] += __ldcg(&a.part[(long long)b * 4 + f]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        s[f] += __shfl_down_sync(0xffffffffu, s[f], off);
    if (lane == 0) {
#pragma unroll
      for (int f = 0; f < 4; ++f) red_sum[f][warp] = s[f];
    }
    __syncthreads();
    if (tid == 0) {
      for (int f = 0; f < 4; ++f) {
        double t = red_sum[f][0];
        for (int w = 1; w < NT / 32; ++w) t += red_sum[f][w];
        a.scr->cons[f] = t;
      }
    }
  }
  if (tid == 0) {
    int rn = atomicAdd(&a.scr->reach_next, 0);
    a.scr->reach = rn;
    a.scr->reach_next = 0;
    a.scr->ticket = 0u;
    __threadfence();
  }
}

// Blocks per multiprocessor the register budget is sized for: the FP64
// square-lattice window fills the shared memory of a multiprocessor, so one
// block may use up to 255 registers a thread.
template <typename T, int DIM>
constexpr int step_min_blocks() {
  return (DIM == 2 && sizeof(T) == 8) ? 1 : 4;
}

template <typename T, int DIM, bool KAHAN, int NT = 256, int TW1 = NT>
__global__ void __launch_bounds__(NT, (step_min_blocks<T, DIM>()))
    step_kernel(const StepArgs a) {
  using S = TileShape<DIM>;
  // tile width: TW1 <= NT destinations in 1-D (one per thread; the other
  // threads only help form the window's sources), TXW = 32 in 2-D
  constexpr int TXW = DIM == 1 ? TW1 : S::TX;
  static_assert(DIM == 2 ? NT == S::TX * S::TY
                         : (NT % 32 == 0 && TW1 <= NT && NT % TW1 == 0),
                "tile");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned red_tmin[NT / 32], red_tmax[NT / 32];

  const int tid = threadIdx.x;
  const int R = a.scr->reach;
  if (R > a.r_cap) {
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0)
      atomicOr(&a.scr->flags, kFlagReach);
    return;
  }
  const int Ry = (DIM == 2) ? R : 0;
  const int x0 = blockIdx.x * TXW;
  const int y0 = blockIdx.y * S::TY;
  const int W = TXW + 2 * R;
  const int H = (DIM == 2) ? S::TY + 2 * R : 1;
  const int NS = W * H;

  SrcLayout<T, DIM, TXW> L;
  L.bind(smem_raw, a.r_cap);

  // ---- 1. equilibrium packets of every source in reach of the tile ----
  unsigned long long my_clamps = 0;
  bool my_bad = false;
  unsigned my_tmin = 0xffffffffu, my_tmax = 0u;  // window types (2-D)
  for (int i = tid; i < NS; i += NT) {
    int ly = i / W;
    int lx = i - ly * W;
    long long sx = (long long)x0 - R + lx;
    long long sy = (DIM == 2) ? (long long)y0 - R + ly : 0;
    bool fx, fy = false;
    int gx = virtual_axis(a.bc_x, a.nx, sx, &fx);
    int gy = (DIM == 2) ? virtual_axis(a.bc_y, a.ny, sy, &fy) : 0;
    long long g = (long long)gy * a.nx + gx;
    Equil<T> q;
    {
      T rho = ld<T>(a.in[0], g);
      T mx = ld<T>(a.in[1], g);
      T my = (DIM == 2) ? ld<T>(a.in[2], g) : T(0);
      T rE = ld<T>(a.in[3], g);
      if (fx) mx = -mx;
      if (fy) my = -my;
      q = equilibrium<T, DIM>(rho, mx, my, rE, a.k);
      bool own = sx >= x0 && sx < x0 + TXW && sx < a.nx &&
                 (DIM == 1 || (sy >= y0 && sy < y0 + S::TY && sy < a.ny));
      if (own) {
        my_clamps += q.clamp ? 1 : 0;
        my_bad |= q.bad;
      }
    }
    if (DIM == 2) {
      const unsigned wt = window_type(q.emits, q.c1, q.n0, q.n1);
      my_tmin = min(my_tmin, wt);
      my_tmax = max(my_tmax, wt);
    }
    if (!q.emits) {
      L.c1[i] = -1;
      continue;
    }
    L.c1[i] = (short)q.c1;
    L.n0[i] = (short)q.n0;
    L.n1[i] = (short)q.n1;
    if (DIM == 1) {
      L.f0[i] = q.f0;
    } else {
      T w4[4];
      corner_weights(q, w4);
#pragma unroll
      for (int k = 0; k < 4; ++k) L.wt[k * L.cap + i] = w4[k];
    }
    if (DIM == 1) {
      L.mass[0 * L.cap + i] = q.d0;
      L.mass[1 * L.cap + i] = q.d1;
      L.mass[2 * L.cap + i] = q.d2;
    } else {
      L.mass[0 * L.cap + i] = q.d1;
      L.mass[1 * L.cap + i] = q.d2;
    }
#pragma unroll
    for (int p = 0; p < S::NP; ++p) {
      T px, py, pe;
      packet_fields<T, DIM>(q, p, &px, &py, &pe);
      L.Px[p * L.cap + i] = px;
      if (DIM == 2) L.Py[p * L.cap + i] = py;
      L.PE[p * L.cap + i] = pe;
    }
  }
  if (my_clamps) atomicAdd(&a.scr->eclamps, my_clamps);
  if (my_bad) atomicOr(&a.scr->flags, kFlagState);
  if (DIM == 2) {
    const unsigned wmin = __reduce_min_sync(0xffffffffu, my_tmin);
    const unsigned wmax = __reduce_max_sync(0xffffffffu, my_tmax);
    if ((tid & 31) == 0) {
      red_tmin[tid >> 5] = wmin;
      red_tmax[tid >> 5] = wmax;
    }
  }
  __syncthreads();
  // One (c1, n) for the whole window?  Then step 2 takes the compile-time
  // landings (c1 <= 2, n_x, n_y in {-1, 0}; their offsets are within c1 + 2
  // <= R of the destination).
  int uni_sel = -1;
  if (DIM == 2) {
    unsigned tmin = red_tmin[0], tmax = red_tmax[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      tmin = min(tmin, red_tmin[w]);
      tmax = max(tmax, red_tmax[w]);
    }
    const int c1 = (int)((tmin >> 16) & 0xff);
    const int nx = (int)((tmin >> 8) & 0xff) - 128;
    const int ny = (int)(tmin & 0xff) - 128;
    if (tmin == tmax && tmin != 0u && c1 <= 2 && c1 + 2 <= R && nx >= -1 &&
        nx <= 0 && ny >= -1 && ny <= 0)
      uni_sel = c1 * 4 + (nx + 1) * 2 + (ny + 1);
  }

  // ---- 2. gather the arrivals at this thread's destination ----
  const int tx = tid % TXW;
  const int ty = tid / TXW;
  const int dx = x0 + tx;
  const int dy = y0 + ty;
  const bool valid = dx < a.nx && dy < a.ny;
  T tot[4] = {T(0), T(0), T(0), T(0)};
  T comp[4] = {T(0), T(0), T(0), T(0)};
  bool gathered = false;
  if constexpr (DIM == 2) {
   if (valid && uni_sel >= 0) {
    gathered = true;
    const int s0 = (ty + R) * W + (tx + R);
    switch (uni_sel) {
      case 0: uniform_gather<T, KAHAN, 0, -1, -1>(L, s0, W, R, tot, comp); break;
      case 1: uniform_gather<T, KAHAN, 0, -1, 0>(L, s0, W, R, tot, comp); break;
      case 2: uniform_gather<T, KAHAN, 0, 0, -1>(L, s0, W, R, tot, comp); break;
      case 3: uniform_gather<T, KAHAN, 0, 0, 0>(L, s0, W, R, tot, comp); break;
      case 4: uniform_gather<T, KAHAN, 1, -1, -1>(L, s0, W, R, tot, comp); break;
      case 5: uniform_gather<T, KAHAN, 1, -1, 0>(L, s0, W, R, tot, comp); break;
      case 6: uniform_gather<T, KAHAN, 1, 0, -1>(L, s0, W, R, tot, comp); break;
      case 7: uniform_gather<T, KAHAN, 1, 0, 0>(L, s0, W, R, tot, comp); break;
      case 8: uniform_gather<T, KAHAN, 2, -1, -1>(L, s0, W, R, tot, comp); break;
      case 9: uniform_gather<T, KAHAN, 2, -1, 0>(L, s0, W, R, tot, comp); break;
      case 10: uniform_gather<T, KAHAN, 2, 0, -1>(L, s0, W, R, tot, comp); break;
      default: uniform_gather<T, KAHAN, 2, 0, 0>(L, s0, W, R, tot, comp); break;
    }
   }
  }
  if (valid && !gathered) {
    for (int j = 0; j <= Ry; ++j) {
      T pair[4];
#pragma unroll 1
      for (int side = 0; side < (j == 0 ? 1 : 2); ++side) {
        const int sy = (side == 0) ? dy - j : dy + j;
        const int ly = (DIM == 2) ? sy - (y0 - R) : 0;  // 1-D: one row
        const int base = ly * W + tx;  // source dx - R sits at lx = tx
        T r = T(0), x = T(0), y = T(0), e = T(0);
        for (int i = 0; i <= 2 * R; ++i) {
          const int s = base + i;
          const int c1 = L.c1[s];
          if (c1 < 0) continue;
          const int c2 = c1 + 1;
          const int ox = R - i - L.n0[s];
          const int oy = (DIM == 2) ? (dy - sy) - L.n1[s] : 0;
          bool near_x = ox >= -c2 && ox <= c2 + 1;
          if (DIM == 1) {
            if (!near_x) continue;
          } else {
            bool near_y = oy >= -c2 && oy <= c2 + 1;
            bool xarm = (oy == 0 || oy == 1) && near_x;
            bool yarm = (ox == 0 || ox == 1) && near_y;
            if (!xarm && !yarm) continue;
          }
          T wx[2] = {T(1), T(0)};
          if (DIM == 1) {
            const T fx0 = L.f0[s];
            wx[0] = T(1) - fx0;
            wx[1] = fx0;
          }
#pragma unroll
          for (int p = 0; p < S::NP; ++p) {
            int cx, cy, lev;
            packet<DIM>(p, c1, &cx, &cy, &lev);
#pragma unroll
            for (int kk = 0; kk < S::NK; ++kk) {
              const int kx = kk & 1, ky = kk >> 1;
              if (cx + kx != ox) continue;
              if (DIM == 2 && cy + ky != oy) continue;
              const T al = (DIM == 1) ? wx[kx] : L.wt[kk * L.cap + s];
              r = r + al * L.mass[lev * L.cap + s];
              x = x + al * L.Px[p * L.cap + s];
              if (DIM == 2) y = y + al * L.Py[p * L.cap + s];
              e = e + al * L.PE[p * L.cap + s];
            }
          }
        }
        if (side == 0) {
          pair[0] = r;
          pair[1] = x;
          pair[2] = y;
          pair[3] = e;
        } else {
          pair[0] = pair[0] + r;
          pair[1] = pair[1] + x;
          pair[2] = pair[2] + y;
          pair[3] = pair[3] + e;
        }
      }
      add_pair<T, KAHAN>(tot, comp, pair);  // compensated when KAHAN
    }
  }

  // ---- 3. write, reach of the new state, FP64 totals ----
  step_finish<T, DIM, NT>(a, valid, dx, dy, tot);
}

template <typename T, int DIM, int TXW = TileShape<DIM>::TX>
size_t step_smem_bytes_t(int r_cap) {
  return SrcLayout<T, DIM, TXW>::bytes(r_cap);
}

}  // namespace lbm
