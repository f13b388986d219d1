// One tile (TW nodes, one per thread; 256 by default) of the 1-D tau = 1
// step, for kernels that process many tubes (batched tubes, the serving
// pool).  Same arithmetic and summation
// order as the single-tube step kernel: equilibrium packets of the tile's
// sources within reach R in shared memory (Section III.B eqs 13-15, 24-26;
// Section IV.A), then each thread sums the arrivals at its node over the
// sources in ascending order, packets in table order, corners in order (eqs
// 6, 10, 22, 28); additional points beyond the ends per Section V.B.
// FP64 instantiations must be compiled without contraction to round as the
// oracle does.
#pragma once

#include <utility>

#include "fp32_arith.cuh"
#include "step_kernel.cuh"

namespace lbm {

constexpr int kTile1d = 256;

// Equilibrium of one node on the 1-D lattice in FP32 (Section III.B: d0 =
// theta rho, b0 = 1, b1 = b2 = 2; eqs 13-15, 24-26), branch-free: the
// quantities of the general equilibrium, with X = D (gamma - 1) e /
// (1 - theta), c1 from c1_of, d1 by the corrected quotient and d2 from the
// mass constraint d0 + 2 (d1 + d2) = rho, phi = e - (D/2)(gamma - 1) e.  V a
// hair below an integer (f = V - floor(V) rounds to 1) is taken as
// (n + 1, f = 0): the same landings up to a zero-weight term.
__device__ __forceinline__ Equil<float> equilibrium_1d_f32(float rho, float mx,
                                                          float rhoE,
                                                          const EqConst& k) {
  Equil<float> q;
  const float inv = rcp_nr(rho);
  q.V0 = mx * inv;
  q.V1 = 0.0f;
  const float e_raw = rhoE * inv - 0.5f * (q.V0 * q.V0);
  const float e = fmaxf(e_raw, 0.0f);
  q.e = e;
  const float X = k.kreach_f * e;
  const bool finite_in = fabsf(rho + mx + rhoE) <= 3.0e38f;
  q.bad = !finite_in || rho < 0.0f || (rho > 0.0f && rho < 1.17549435e-38f) ||
          !(X <= 1099511627776.0f);
  q.emits = !q.bad && rho > 0.0f;
  q.clamp = q.emits && e_raw < 0.0f;
  const float c1f = c1_of(X);
  q.c1 = (int)c1f;
  const float c2f = c1f + 1.0f;
  const float c1sq = c1f * c1f, c2sq = c2f * c2f;
  const float den = 2.0f * (c2sq - c1sq);
  q.d0 = k.theta_f * rho;
  const float rho_p = rho - q.d0;
  q.d1 = div_markstein(rho_p * (c2sq - X), den, rcp_nr(den));
  q.d2 = 0.5f * rho_p - q.d1;
  q.phi = e - 0.5f * (k.kq_f * e);
  const float fl = floorf(q.V0);
  q.n0 = (int)fl;
  q.f0 = q.V0 - fl;
  if (q.f0 == 1.0f) {
    q.n0 += 1;
    q.f0 = 0.0f;
  }
  q.n1 = 0;
  q.f1 = 0.0f;
  return q;
}

// Fast path of the gather for a warp whose sources all share the lattice
// shift n = floor(V) (N) and the level c1 (C1): packet p, corner k of the
// source at window slot tid + R + delta lands on the thread's destination,
// delta = -(N + c_p + k) (eq 28).  The ten landings, sorted as the general
// loop visits them (source ascending, then packet, then corner), with the
// same arithmetic, so results are identical to it.
struct Landing1 {
  int delta, p, k;
};

__host__ __device__ constexpr int pk1_cx(int p, int c1) {
  return p == 0 ? 0 : (p == 1 ? c1 : (p == 2 ? -c1 : (p == 3 ? c1 + 1 : -(c1 + 1))));
}

template <int N, int C1>
struct Landings1 {
  Landing1 v[10];
  __host__ __device__ constexpr Landings1() : v{} {
    int m = 0;
    for (int p = 0; p < 5; ++p)
      for (int k = 0; k < 2; ++k) v[m++] = Landing1{-N - pk1_cx(p, C1) - k, p, k};
    for (int a = 1; a < 10; ++a) {
      Landing1 x = v[a];
      int b = a - 1;
      while (b >= 0 && (v[b].delta > x.delta ||
                        (v[b].delta == x.delta &&
                         (v[b].p > x.p || (v[b].p == x.p && v[b].k > x.k))))) {
        v[b + 1] = v[b];
        --b;
      }
      v[b + 1] = x;
    }
  }
};

template <typename T, bool KAHAN, int N, int C1, int I, typename Lay>
__device__ __forceinline__ void land1(const Lay& L, int base, T& r, T& x,
                                      T& e, T& cr, T& cx_, T& ce) {
  constexpr Landings1<N, C1> list{};
  constexpr Landing1 q = list.v[I];
  constexpr int lev = q.p == 0 ? 0 : (q.p <= 2 ? 1 : 2);
  const int s = base + q.delta;
  const T fx0 = L.f0[s];
  const T al = q.k == 0 ? T(1) - fx0 : fx0;
  if (KAHAN) {
    T y = al * L.mass[lev * L.cap + s] - cr;
    T t = r + y;
    cr = (t - r) - y;
    r = t;
    y = al * L.Px[q.p * L.cap + s] - cx_;
    t = x + y;
    cx_ = (t - x) - y;
    x = t;
    y = al * L.PE[q.p * L.cap + s] - ce;
    t = e + y;
    ce = (t - e) - y;
    e = t;
  } else {
    r = r + al * L.mass[lev * L.cap + s];
    x = x + al * L.Px[q.p * L.cap + s];
    e = e + al * L.PE[q.p * L.cap + s];
  }
}

// The same landing for FP32 with compensated sums, mass and momentum as one
// pair in the packed FP32 instructions, each half rounding exactly as the
// scalar form of the units that use it (built without contraction): y =
// al m - c, t = s + y, c = (t - s) - y.
template <int N, int C1, int I, typename Lay>
__device__ __forceinline__ void land1_k2(const Lay& L, int base, float2& rx,
                                         float& e, float2& crx, float& ce) {
  constexpr Landings1<N, C1> list{};
  constexpr Landing1 q = list.v[I];
  constexpr int lev = q.p == 0 ? 0 : (q.p <= 2 ? 1 : 2);
  const int s = base + q.delta;
  const float fx0 = L.f0[s];
  const float al = q.k == 0 ? 1.0f - fx0 : fx0;
  const float2 a2 = make_float2(al, al);
  const float2 v2 = make_float2(L.mass[lev * L.cap + s], L.Px[q.p * L.cap + s]);
  const float2 y = __fadd2_rn(__fmul2_rn(a2, v2), make_float2(-crx.x, -crx.y));
  const float2 t = __fadd2_rn(rx, y);
  const float2 d = __fadd2_rn(t, make_float2(-rx.x, -rx.y));
  crx = __fadd2_rn(d, make_float2(-y.x, -y.y));
  rx = t;
  const float ye = al * L.PE[q.p * L.cap + s] - ce;
  const float te = e + ye;
  ce = (te - e) - ye;
  e = te;
}

template <int N, int C1, typename Lay, int... I>
__device__ __forceinline__ void land1_k2_all(const Lay& L, int base,
                                             float2& rx, float& e, float2& crx,
                                             float& ce,
                                             std::integer_sequence<int, I...>) {
  (land1_k2<N, C1, I>(L, base, rx, e, crx, ce), ...);
}

template <typename T, bool KAHAN, int N, int C1, typename Lay, int... I>
__device__ __forceinline__ void land1_all(const Lay& L, int base, T& r, T& x,
                                          T& e, T& cr, T& cx_, T& ce,
                                          std::integer_sequence<int, I...>) {
  (land1<T, KAHAN, N, C1, I>(L, base, r, x, e, cr, cx_, ce), ...);
}

template <typename T, bool KAHAN, int N, int C1, typename Lay>
__device__ __forceinline__ void fast_gather1(const Lay& L, int base, T& r,
                                             T& x, T& e, T& cr, T& cx_,
                                             T& ce) {
  if constexpr (KAHAN && sizeof(T) == sizeof(float)) {
    float2 rx = make_float2(r, x), crx = make_float2(cr, cx_);
    land1_k2_all<N, C1>(L, base, rx, e, crx, ce,
                        std::make_integer_sequence<int, 10>{});
    r = rx.x;
    x = rx.y;
    cr = crx.x;
    cx_ = crx.y;
  } else {
    land1_all<T, KAHAN, N, C1>(L, base, r, x, e, cr, cx_, ce,
                               std::make_integer_sequence<int, 10>{});
  }
}

template <typename T, bool KAHAN, int TW = kTile1d>
__device__ void tile1d_step(const T* __restrict__ in0,
                            const T* __restrict__ in1,
                            const T* __restrict__ in2, T* __restrict__ o0,
                            T* __restrict__ o1, T* __restrict__ o2,
                            long long off, int n, int bc, int tile, int R,
                            int r_cap, const EqConst& k, int* reach_next,
                            unsigned* flags, unsigned long long* eclamps,
                            unsigned char* smem) {
  using S = TileShape<1>;
  const int tid = threadIdx.x;
  SrcLayout<T, 1, TW> L;
  L.bind(smem, r_cap);
  const int x0 = tile * TW;
  const int W = TW + 2 * R;
  unsigned long long clamps = 0;
  bool bad = false;
  for (int i = tid; i < W; i += TW) {
    const long long sx = (long long)x0 - R + i;
    bool fx;
    const int gx = virtual_axis(bc, n, sx, &fx);
    const long long g = off + gx;
    T rho = in0[g], mx = in1[g], rE = in2[g];
    if (fx) mx = -mx;
    Equil<T> q;
    if constexpr (sizeof(T) == sizeof(float))
      q = equilibrium_1d_f32(rho, mx, rE, k);
    else
      q = equilibrium<T, 1>(rho, mx, T(0), rE, k);
    if (sx >= x0 && sx < x0 + TW && sx < n) {
      clamps += q.clamp ? 1 : 0;
      bad |= q.bad;
    }
    if (!q.emits) {
      L.c1[i] = -1;
      continue;
    }
    L.c1[i] = (short)q.c1;
    L.n0[i] = (short)q.n0;
    L.f0[i] = q.f0;
    L.mass[0 * L.cap + i] = q.d0;
    L.mass[1 * L.cap + i] = q.d1;
    L.mass[2 * L.cap + i] = q.d2;
#pragma unroll
    for (int p = 0; p < S::NP; ++p) {
      int cx, cy, lev;
      packet<1>(p, q.c1, &cx, &cy, &lev);
      const T d = L.mass[lev * L.cap + i];
      const T cbx = q.V0 + (T)cx;
      L.Px[p * L.cap + i] = d * cbx;
      L.PE[p * L.cap + i] = d * (T(0.5) * (cbx * cbx) + q.phi);
    }
  }
  if (clamps) atomicAdd(eclamps, clamps);
  if (bad) atomicOr(flags, kFlagState);
  __syncthreads();

  const int dx = x0 + tid;
  int my_reach = 0;
  // Does every source of this warp's destinations (window slots wb ..
  // wb + 31 + 2R) share one type with n in {-1, 0} and c1 <= 3?
  int sel = -1;
  if (R <= 16) {
    const int lane = tid & 31, wb = tid & ~31;
    const int c1r = L.c1[wb], n0r = L.n0[wb];
    // (R >= c1 + 2 keeps every landing's source inside the window)
    bool same = c1r >= 0 && c1r <= 3 && n0r >= -1 && n0r <= 0 && R >= c1r + 2 &&
                L.c1[wb + lane] == c1r && L.n0[wb + lane] == n0r;
    if (lane < 2 * R)
      same = same && L.c1[wb + lane + 32] == c1r && L.n0[wb + lane + 32] == n0r;
    if (__all_sync(0xffffffffu, same)) sel = c1r * 2 + (n0r + 1);
  }
  if (dx < n && sel >= 0) {
    T r = T(0), x = T(0), e = T(0);
    T cr = T(0), cx_ = T(0), ce = T(0);
    const int base = tid + R;
    switch (sel) {
      case 0: fast_gather1<T, KAHAN, -1, 0>(L, base, r, x, e, cr, cx_, ce); break;
      case 1: fast_gather1<T, KAHAN, 0, 0>(L, base, r, x, e, cr, cx_, ce); break;
      case 2: fast_gather1<T, KAHAN, -1, 1>(L, base, r, x, e, cr, cx_, ce); break;
      case 3: fast_gather1<T, KAHAN, 0, 1>(L, base, r, x, e, cr, cx_, ce); break;
      case 4: fast_gather1<T, KAHAN, -1, 2>(L, base, r, x, e, cr, cx_, ce); break;
      case 5: fast_gather1<T, KAHAN, 0, 2>(L, base, r, x, e, cr, cx_, ce); break;
      case 6: fast_gather1<T, KAHAN, -1, 3>(L, base, r, x, e, cr, cx_, ce); break;
      default: fast_gather1<T, KAHAN, 0, 3>(L, base, r, x, e, cr, cx_, ce); break;
    }
    // the single-tube kernel adds the row sum to a zero total: 0 + s = s
    const long long o = off + dx;
    o0[o] = T(0) + r;
    o1[o] = T(0) + x;
    o2[o] = T(0) + e;
    if constexpr (sizeof(T) == sizeof(float))
      my_reach = reach_bound_f32(r, x, 0.0f, e, k.kreach_f);
    else
      my_reach = reach_bound((double)r, (double)x, 0.0, (double)e,
                             (float)k.kreach);
  } else if (dx < n) {
    // one source row; ascending x, packet order, corner order (as the
    // single-tube kernel and the oracle)
    T r = T(0), x = T(0), e = T(0);
    T cr = T(0), cx_ = T(0), ce = T(0);
    for (int i = 0; i <= 2 * R; ++i) {
      const int s = tid + i;
      const int c1 = L.c1[s];
      if (c1 < 0) continue;
      const int c2 = c1 + 1;
      const int ox = R - i - L.n0[s];
      if (ox < -c2 || ox > c2 + 1) continue;
      const T fx0 = L.f0[s];
      const T wx[2] = {T(1) - fx0, fx0};
#pragma unroll
      for (int p = 0; p < S::NP; ++p) {
        int px, py, lev;
        packet<1>(p, c1, &px, &py, &lev);
#pragma unroll
        for (int kk = 0; kk < S::NK; ++kk) {
          if (px + kk != ox) continue;
          const T al = wx[kk];
          if (KAHAN) {
            T y = al * L.mass[lev * L.cap + s] - cr;
            T t = r + y;
            cr = (t - r) - y;
            r = t;
            y = al * L.Px[p * L.cap + s] - cx_;
            t = x + y;
            cx_ = (t - x) - y;
            x = t;
            y = al * L.PE[p * L.cap + s] - ce;
            t = e + y;
            ce = (t - e) - y;
            e = t;
          } else {
            r = r + al * L.mass[lev * L.cap + s];
            x = x + al * L.Px[p * L.cap + s];
            e = e + al * L.PE[p * L.cap + s];
          }
        }
      }
    }
    // the single-tube kernel adds the row sum to a zero total: 0 + s = s
    const long long o = off + dx;
    o0[o] = T(0) + r;
    o1[o] = T(0) + x;
    o2[o] = T(0) + e;
    if constexpr (sizeof(T) == sizeof(float))
      my_reach = reach_bound_f32(r, x, 0.0f, e, k.kreach_f);
    else
      my_reach = reach_bound((double)r, (double)x, 0.0, (double)e,
                             (float)k.kreach);
  }
  // the item's reach: one atomic per item rather than one per warp (all
  // items of a tube update the same word)
  __shared__ int red_r[TW / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    my_reach = max(my_reach, __shfl_xor_sync(0xffffffffu, my_reach, off));
  if ((tid & 31) == 0) red_r[tid >> 5] = my_reach;
  __syncthreads();  // shared records are reused by the next item
  if (tid == 0) {
    int m = red_r[0];
    for (int w = 1; w < TW / 32; ++w) m = max(m, red_r[w]);
    if (m > 0) atomicMax(reach_next, m);
  }
}


}  // namespace lbm
