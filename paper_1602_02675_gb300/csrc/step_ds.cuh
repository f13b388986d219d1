// FP32 fused step for the square lattice (2-D): deposit, then shift.
//
// The method (Section III.B, eqs 11-15, 21-26, 29; Section V.A-B) moves,
// from every source s, eight packets: packet p of level v carries mass d_v,
// momentum d_v (V + c'_p) and energy d_v (E_b + V.c'_p + |c'_p|^2/2), with
// E_b = |V|^2/2 + phi (eqs 12-15), and lands bilinearly (eq 29) on the four
// nodes around s + V + c'_p: corner k = (k_x, k_y) at s + n + c'_p + k,
// n = floor(V), with weight w_k(s) = ((1-f_x) or f_x) ((1-f_y) or f_y).
// Every packet field is a fixed linear map of the level record
//   L_v(s) = d_v (1, V_x, V_y, E_b)
// that depends only on c'_p.  So, among sources that share n and c1 (one
// "type"), the arrivals at a destination x are
//   Y(x) = sum_v sum_{p in v} M(c'_p) D_v(x - n - c'_p),
//   D_v(q) = sum_k w_k(q - k) L_v(q - k)                       (deposit)
// i.e. the records are deposited bilinearly once (32 multiply-adds per
// position) and each destination then reads eight shifted deposits, instead
// of visiting 32 packet landings.  The arithmetic differs from the landing
// by landing sum only in rounding; the sum of every destination has the same
// form and order relative to the destination, so uniform states stay uniform
// and data that vary along x only stay so bit for bit (their y-momentum
// arrivals from rows +-c cancel exactly).
//
// Layout: persistent blocks take tiles by ticket, one at a time.  A block's
// window is 59 x 48 sources (WCOLS x WROWS); with the step's reach R the
// tile is the window minus R on every side, (59 - 2R) x (48 - 2R)
// destinations.
//  * Phase 1 (window).  Thread (lane, wx, g) owns window column
//    lane + 28 wx (the two warps of a row overlap by four columns; column 59
//    holds deposits only) and walks the rows of group g (12 deposit rows,
//    the groups' walks overlap; row 48 holds deposits only).  Walking down
//    its column it loads each source's moments (coalesced: a warp reads 32
//    consecutive nodes of a row), forms the equilibrium and deposits: the
//    parts that land in its own column it sums itself over the rows, the
//    parts that land one or more columns to the right come from the lanes to
//    the left by shuffles, and the deposit goes to shared memory.  Sources
//    outside the grid are the additional points of Section V.B (nearest
//    node, periodic image, or mirror image with the normal momentum negated).
//  * Phase 2 (tile).  Each thread gathers destinations of the tile in
//    row-major order, 256 apart, from the deposits: per level four reads
//    (+x, -x, +y, -y packets), and writes the new moments; then the new
//    node's reach and the block's compensated partial totals.
// The window's sources are all of one type in most tiles early in a flow:
// the one-type walk deposits for the type of the tile's central node and
// checks that every source had that type.  Otherwise the tile goes on to
// the group walks, which group the sources by c1 and by blocks of SX x SY
// lattice shifts (SX, SY up to 4, from the spread of n over the window):
// n in {a .. a+SX-1} x {b .. b+SY-1}.  Relative to the base (a, b) such a
// source lands at s + dn + k, dn in {0 .. SX-1} x {0 .. SY-1}, so the
// deposit weights become hat functions over SX + 1 and SY + 1 offsets (one
// walk per group), and the gather is the one-type gather at shift (a, b).
// Groups are done in ascending order, each adding its arrivals to the
// destinations.  The smallest c1 and shift of a window and its block are
// taken from the tile's previous step and checked during its first walk
// (redone when the block does not hold the window).
#pragma once

#include <cstdint>

#include "fp32_arith.cuh"
#include "step_kernel.cuh"

namespace lbm {
namespace ds {

constexpr int NWX = 2;                    // warps across a window row
constexpr int CW = 32 * NWX;              // threads across
constexpr int SPMAX = 4;                  // largest shift block of a group
constexpr int WSTEP = 32 - SPMAX;         // column offset of the second warp
constexpr int DCOLS = WSTEP + 32;         // deposit columns 1 .. 59
constexpr int WCOLS = DCOLS - 1;          // source columns 0 .. 58
constexpr int NG = 4;                     // row groups
constexpr int SH = 12;                    // rows a group deposits
constexpr int WROWS = NG * SH;            // source rows 0 .. 47
constexpr int NTHR = CW * NG;             // 256
constexpr int NWARP = NTHR / 32;
constexpr int RMAX = 6;                   // largest reach of this layout
constexpr int PF = 3;                     // rows loaded ahead of the walk
constexpr int DP = DCOLS;                 // deposit row pitch (positions)
constexpr int PLANE = DP * (WROWS + 1);   // deposit rows 1 .. 48
// Each walking thread's ring of source moments in flight: PF rows of its
// column, 4 fields, copied asynchronously (cp.async) so that the loads are
// issued PF rows before they are needed and hold no registers meanwhile.
constexpr int RING = PF * 4 * NTHR;       // floats
// Type ids: c1 * 65536 + (n_x + 128) * 256 + (n_y + 128), held exactly in
// a float; sources that emit nothing have no type.
constexpr float kNoType = 16777216.0f;

__host__ __device__ constexpr size_t smem_bytes() {
  return (size_t)2 * PLANE * sizeof(float4) + (size_t)RING * sizeof(float);
}
__host__ __device__ inline int tile_w(int R) { return WCOLS - 2 * R; }
__host__ __device__ inline int tile_h(int R) { return WROWS - 2 * R; }
// Tiles of an nx x ny grid at reach R (at least 1).
__host__ __device__ inline int tiles_for(int nx, int ny, int R) {
  const int r = R < 1 ? 1 : R;
  return ((nx + tile_w(r) - 1) / tile_w(r)) * ((ny + tile_h(r) - 1) / tile_h(r));
}

// The part of a node's equilibrium that both the window phase and the
// producing step's reach need, in explicitly rounded operations so that the
// two agree bit for bit: V = m / rho (one refined reciprocal), |V|^2,
// e = E - |V|^2/2 (eq 13, eq 15 text) before and after the clamp at 0, and
// X = D (gamma - 1) e (eq 26 with d0 = 0 on the square lattice).
struct EqCore {
  float Vx, Vy, kin2, eraw, X;
};
__device__ __forceinline__ EqCore eq_core(float rho, float mx, float my,
                                          float rhoE, float kq) {
  EqCore c;
  const float inv = rcp_nr(rho);
  c.Vx = __fmul_rn(mx, inv);
  c.Vy = __fmul_rn(my, inv);
  c.kin2 = __fmaf_rn(c.Vy, c.Vy, __fmul_rn(c.Vx, c.Vx));
  c.eraw = __fmaf_rn(-0.5f, c.kin2, __fmul_rn(rhoE, inv));
  c.X = __fmul_rn(kq, fmaxf(c.eraw, 0.0f));
  return c;
}

// c1 = int(sqrt(X)) (eq 26), exactly: below 16 by counting the squares
// X reaches, above by the estimate with the integer test (c1_of).  Every
// lane of the warp must call it.
__device__ __forceinline__ float c1_exact(float X) {
  float c = (X >= 1.0f ? 1.0f : 0.0f) + (X >= 4.0f ? 1.0f : 0.0f) +
            (X >= 9.0f ? 1.0f : 0.0f);
  if (__any_sync(0xffffffffu, !(X < 16.0f))) c = X < 16.0f ? c : c1_of(X);
  return c;
}

// n = floor(V), f = V - n (eq 23); f rounded to 1 is taken as (n + 1, 0).
__device__ __forceinline__ void split_f(float V, float& n, float& f) {
  const float fl = floorf(V);
  const float fr = __fsub_rn(V, fl);
  const bool one = fr == 1.0f;
  n = one ? __fadd_rn(fl, 1.0f) : fl;
  f = one ? 0.0f : fr;
}

// Migration reach floor(max |V_a|) + 1 + c2 (eq 26) of a node whose core
// and c1 are given; 0 for a node that emits nothing.
__device__ __forceinline__ int reach_of(bool emits, const EqCore& c,
                                        float c1) {
  const float v = floorf(fmaxf(fabsf(c.Vx), fabsf(c.Vy)));
  const float r = v + 2.0f + c1;
  return !emits ? 0 : (r > 1.0e8f ? 100000000 : (int)r);
}

// Interior node supplying source coordinate L on one axis (Section V.B).
__device__ __forceinline__ int axis_src(int bc, int n, int L, bool* flip) {
  *flip = false;
  if ((unsigned)L < (unsigned)n) return L;
  return virtual_axis(bc, n, (long long)L, flip);
}

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) {
  return make_float4(a, b, c, d);
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return f4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 mul4(float s, float4 a) {
  const float2 ss = make_float2(s, s);
  const float2 lo = __fmul2_rn(ss, make_float2(a.x, a.y));
  const float2 hi = __fmul2_rn(ss, make_float2(a.z, a.w));
  return f4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 fma4(float s, float4 a, float4 b) {
  const float2 ss = make_float2(s, s);
  const float2 lo = __ffma2_rn(ss, make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 hi = __ffma2_rn(ss, make_float2(a.z, a.w), make_float2(b.z, b.w));
  return f4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 shfl_up4n(float4 v, int d) {
  return f4(__shfl_up_sync(0xffffffffu, v.x, d),
            __shfl_up_sync(0xffffffffu, v.y, d),
            __shfl_up_sync(0xffffffffu, v.z, d),
            __shfl_up_sync(0xffffffffu, v.w, d));
}
__device__ __forceinline__ float4 shfl_up4(float4 v) {
  return f4(__shfl_up_sync(0xffffffffu, v.x, 1),
            __shfl_up_sync(0xffffffffu, v.y, 1),
            __shfl_up_sync(0xffffffffu, v.z, 1),
            __shfl_up_sync(0xffffffffu, v.w, 1));
}

// Decoded type: lattice shift n and level speeds c1, c2.
struct Type {
  int nx, ny, c1;
};
__device__ __forceinline__ Type decode_type(float t) {
  const float c1 = floorf(t * (1.0f / 65536.0f));
  const float r = __fmaf_rn(-65536.0f, c1, t);
  const float hx = floorf(r * (1.0f / 256.0f));
  const float hy = __fmaf_rn(-256.0f, hx, r);
  return Type{(int)hx - 128, (int)hy - 128, (int)c1};
}

// Constants of one level pair (c1, c2 = c1 + 1) for the level densities
// (eqs 24-25 with d0 = 0 and b1 = 4 on the square lattice): c1^2, c2^2, the
// denominator 4 (c2^2 - c1^2) = 4 (2 c1 + 1) and its correctly rounded
// reciprocal (from a table for c1 <= 3, no estimate on the dependency chain).
struct LevelK {
  float c1sq, c2sq, den, rden;
};
__device__ __forceinline__ LevelK level_k(float c1) {
  LevelK k;
  const float c2 = __fadd_rn(c1, 1.0f);
  k.c1sq = __fmul_rn(c1, c1);
  k.c2sq = __fmul_rn(c2, c2);
  k.den = __fmul_rn(4.0f, __fmaf_rn(2.0f, c1, 1.0f));
  k.rden = c1 < 1.0f ? 0.25f
                     : (c1 < 2.0f ? 1.0f / 12.0f
                                  : (c1 < 3.0f ? 1.0f / 20.0f
                                               : (c1 < 4.0f ? 1.0f / 28.0f
                                                            : rcp_nr(k.den))));
  return k;
}
// d1 = (c2^2 rho - X rho) / (4 (c2^2 - c1^2)), d2 = rho / 4 - d1 of a source
// whose c1 is k's; the quotient rounded as one division would round it
// (Markstein's correction): a shared rounding of 1 / den would bias the
// packets' energy of every node alike.  Zero for a source that emits
// nothing.
__device__ __forceinline__ void level_dens(float rho, float X, bool emits,
                                           const LevelK& k, float& d1,
                                           float& d2) {
  const float num = __fmaf_rn(k.c2sq, rho, -__fmul_rn(X, rho));
  const float q = div_markstein(num, k.den, k.rden);
  d1 = emits ? q : 0.0f;
  d2 = emits ? __fmaf_rn(0.25f, rho, -q) : 0.0f;
}

// Equilibrium of one window source (Section III.B with d0 = 0 and b1 = 4
// on the square lattice): c1 (eq 26), the level records' shared part
// (1, V_x, V_y, E_b) with E_b = |V|^2/2 + phi (eqs 13-15), the split of V
// (eq 23), and the level densities (eqs 24-25).  A source that emits
// nothing (rho <= 0) has zero densities, V and E_b.
struct SrcEq {
  bool emits, clamp;
  float c1, nxf, nyf, fx, fy, d1, d2, Vx, Vy, Eb;
};
// kg: the level constants of the walk's group when every member shares
// them (the densities of sources outside the group are never used), else
// null: each source's own.
__device__ __forceinline__ SrcEq source_eq(float4 m, float kq,
                                           const LevelK* kg = nullptr) {
  SrcEq q;
  const float rho = m.x;
  const EqCore c = eq_core(rho, m.y, m.z, m.w, kq);
  q.emits = rho > 0.0f;
  q.clamp = q.emits && c.eraw < 0.0f;
  // c1 below 4 for the whole warp (X < 16): counted squares; otherwise
  // c1_of
  const bool wide = __any_sync(0xffffffffu, !(c.X < 16.0f));
  q.c1 = (c.X >= 1.0f ? 1.0f : 0.0f) + (c.X >= 4.0f ? 1.0f : 0.0f) +
         (c.X >= 9.0f ? 1.0f : 0.0f);
  if (wide) q.c1 = c.X < 16.0f ? q.c1 : c1_of(c.X);
  level_dens(rho, c.X, q.emits, kg ? *kg : level_k(q.c1), q.d1, q.d2);
  // phi = e - X / 2 (eq 15 with D/2 (gamma - 1) e = X / 2)
  const float phi = __fmaf_rn(-0.5f, c.X, fmaxf(c.eraw, 0.0f));
  q.Eb = q.emits ? __fmaf_rn(0.5f, c.kin2, phi) : 0.0f;
  q.Vx = q.emits ? c.Vx : 0.0f;
  q.Vy = q.emits ? c.Vy : 0.0f;
  split_f(q.Vx, q.nxf, q.fx);
  split_f(q.Vy, q.nyf, q.fy);
  return q;
}
// The same for a source of the tile's guessed type: whether it has that
// type (c1^2 <= X < c2^2 with k's c1, the same shift n) replaces c1.
struct SrcEqT {
  bool emits, clamp, mine;
  float fx, fy, d1, d2, Vx, Vy, Eb;
};
__device__ __forceinline__ SrcEqT source_eq_typed(float4 m, float kq,
                                                  const LevelK& k, float nxT,
                                                  float nyT) {
  SrcEqT q;
  const float rho = m.x;
  const EqCore c = eq_core(rho, m.y, m.z, m.w, kq);
  q.emits = rho > 0.0f;
  q.clamp = q.emits && c.eraw < 0.0f;
  level_dens(rho, c.X, q.emits, k, q.d1, q.d2);
  const float phi = __fmaf_rn(-0.5f, c.X, fmaxf(c.eraw, 0.0f));
  q.Eb = q.emits ? __fmaf_rn(0.5f, c.kin2, phi) : 0.0f;
  q.Vx = q.emits ? c.Vx : 0.0f;
  q.Vy = q.emits ? c.Vy : 0.0f;
  float nxf, nyf;
  split_f(q.Vx, nxf, q.fx);
  split_f(q.Vy, nyf, q.fy);
  q.mine = q.emits && c.X >= k.c1sq && c.X < k.c2sq && nxf == nxT &&
           nyf == nyT;
  return q;
}

__device__ __forceinline__ float type_of(float c1, float nxf, float nyf) {
  return __fmaf_rn(65536.0f, c1,
                   __fmaf_rn(256.0f, __fadd_rn(nxf, 128.0f),
                             __fadd_rn(nyf, 128.0f)));
}
__device__ __forceinline__ float type_id(const SrcEq& q) {
  return q.emits ? type_of(q.c1, q.nxf, q.nyf) : kNoType;
}

// Statistics of a window walk, per thread until reduce_gstats combines them
// over the block: smallest and largest c1 and shift over the emitting
// sources, the next group above the walk's, whether a source of the walk's
// group was deposited, and the clamped energies of owned nodes.
struct GStats {
  float c1min, nxmin, nymin, tnext, c1max, nxmax, nymax;
  unsigned clamps;
  bool any;
};
__device__ __forceinline__ GStats gstats_init() {
  return GStats{kNoType, kNoType, kNoType, kNoType, -kNoType, -kNoType,
                -kNoType, 0u, false};
}
__device__ __forceinline__ void gstats_add(GStats& st, bool emits, float c1,
                                           float nxf, float nyf) {
  if (emits) {
    st.c1min = fminf(st.c1min, c1);
    st.c1max = fmaxf(st.c1max, c1);
    st.nxmin = fminf(st.nxmin, nxf);
    st.nxmax = fmaxf(st.nxmax, nxf);
    st.nymin = fminf(st.nymin, nyf);
    st.nymax = fmaxf(st.nymax, nyf);
  }
}

// Block reduction of GStats (all threads call it and get the result; it
// holds the barrier that makes a walk's deposits visible).  The values are
// small integers, reduced as ints.
constexpr int NGSTAT = 8;
__device__ __forceinline__ void reduce_gstats(GStats& st, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr unsigned F = 0xffffffffu;
  int v[NGSTAT];
  v[0] = __reduce_min_sync(F, (int)st.c1min);
  v[1] = __reduce_min_sync(F, (int)st.nxmin);
  v[2] = __reduce_min_sync(F, (int)st.nymin);
  v[3] = __reduce_min_sync(F, (int)st.tnext);
  v[4] = __reduce_max_sync(F, (int)st.c1max);
  v[5] = __reduce_max_sync(F, (int)st.nxmax);
  v[6] = __reduce_max_sync(F, (int)st.nymax);
  v[7] = __any_sync(F, st.any) ? 1 : 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NGSTAT; ++k) red[k * NWARP + warp] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NGSTAT; ++k) v[k] = red[k * NWARP];
#pragma unroll
  for (int w = 1; w < NWARP; ++w) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = min(v[k], red[k * NWARP + w]);
#pragma unroll
    for (int k = 4; k < NGSTAT; ++k) v[k] = max(v[k], red[k * NWARP + w]);
  }
  st.c1min = (float)v[0];
  st.nxmin = (float)v[1];
  st.nymin = (float)v[2];
  st.tnext = (float)v[3];
  st.c1max = (float)v[4];
  st.nxmax = (float)v[5];
  st.nymax = (float)v[6];
  st.any = v[7] != 0;
}

// Where a thread's column sits and how it reads its sources.
struct Column {
  int lane, wx, g, lx, sx, gx;
  bool flipx, col_valid, col_own, store_col;
};
__device__ __forceinline__ Column column_of(const StepArgs& a, int x0, int R,
                                            int TX, bool interior) {
  Column c;
  const int tid = threadIdx.x;
  c.lane = tid & 31;
  c.wx = (tid >> 5) & (NWX - 1);
  c.g = tid / CW;
  c.lx = c.lane + WSTEP * c.wx;
  c.sx = x0 - R + c.lx;
  c.col_valid = c.lx < WCOLS;
  c.flipx = false;
  c.gx = (interior || !c.col_valid) ? c.sx
                                    : axis_src(a.bc_x, a.nx, c.sx, &c.flipx);
  // deposits of column 0 are never read; the second warp's first SPMAX
  // lanes repeat the first warp's last SPMAX columns (and lack the parts
  // that shuffles from farther left would bring)
  c.store_col = c.wx == 0 ? c.lane >= 1 : c.lane >= SPMAX;
  c.col_own = c.store_col && c.lx >= R && c.lx < R + TX && c.sx < a.nx;
  return c;
}

// 4-byte asynchronous global -> shared copy; src_bytes 0 fills zero.
__device__ __forceinline__ void cp_async4(float* dst, const float* src,
                                          bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The walking thread's ring: slot k holds the 4 fields of one source row
// of its column, field f at ring[(k * 4 + f) * NTHR + tid] (consecutive
// threads at consecutive words).  Sources outside the window arrive as
// zeros; mirrored momentum components are negated when read.
struct SrcRing {
  float* base;
  const float* f[4];
  int stride_rows;
  template <bool INT>
  __device__ __forceinline__ void issue(const StepArgs& a, const Column& c,
                                        int y0, int R, int ly, int slot) {
    const bool valid = c.col_valid && ly >= 0 && ly < WROWS;
    long long i = 0;
    if (valid) {
      const int sy = y0 - R + ly;
      bool flipy = false;
      const int gy = INT ? sy : axis_src(a.bc_y, a.ny, sy, &flipy);
      i = (long long)gy * a.nx + c.gx;
    }
    float* d = base + slot * 4 * NTHR + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async4(d + k * NTHR, f[k] + i, valid);
    cp_async_commit();
  }
  template <bool INT>
  __device__ __forceinline__ float4 take(const StepArgs& a, const Column& c,
                                         int y0, int R, int ly,
                                         int slot) const {
    const float* d = base + slot * 4 * NTHR + threadIdx.x;
    float4 m = f4(d[0], d[NTHR], d[2 * NTHR], d[3 * NTHR]);
    if (c.flipx) m.y = -m.y;
    if (!INT && ly >= 0 && ly < WROWS) {
      bool flipy = false;
      axis_src(a.bc_y, a.ny, y0 - R + ly, &flipy);
      if (flipy) m.z = -m.z;
    }
    return m;
  }
};
__device__ __forceinline__ SrcRing ring_of(const StepArgs& a, float* base) {
  SrcRing r;
  r.base = base;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.f[k] = static_cast<const float*>(a.in[k]);
  r.stride_rows = 0;
  return r;
}

// Type of one window source without its level densities: emits, c1, the
// shift n = floor(V) (eq 23) and whether its energy was clamped.
__device__ __forceinline__ void source_type(float4 m, float kq, bool& emits,
                                            bool& clamp, float& id,
                                            float& c1, float& nxf,
                                            float& nyf) {
  const EqCore c = eq_core(m.x, m.y, m.z, m.w, kq);
  emits = m.x > 0.0f;
  clamp = emits && c.eraw < 0.0f;
  c1 = c1_exact(c.X);
  float f;
  split_f(emits ? c.Vx : 0.0f, nxf, f);
  split_f(emits ? c.Vy : 0.0f, nyf, f);
  id = emits ? __fmaf_rn(65536.0f, c1,
                         __fmaf_rn(256.0f, __fadd_rn(nxf, 128.0f),
                                   __fadd_rn(nyf, 128.0f)))
             : kNoType;
}

// Result of a one-type walk, per thread: whether an emitting source has
// another type than the walk's, and the clamped energies of owned nodes.
struct OneTypeFlags {
  unsigned clamps;
  bool other;
};

// One-type walk for the tile's guessed type T, the type of its central node
// m (every thread forms it): deposits the sources of type T (the corner
// weights of eq 29 on offsets {0, 1}^2) and notes whether any emitting
// source has another type.
template <bool INT>
__device__ __forceinline__ void walk_one_type(
    const StepArgs& a, float4* __restrict__ D1, float4* __restrict__ D2,
    float* rbase, int x0, int y0, int R, int TX, int TY, float4 m,
    float& T, OneTypeFlags& fl) {
  const Column col = column_of(a, x0, R, TX, INT);
  const int ly0 = SH * col.g;
  const float kq = a.k.kq_f;
  // rows r of this walk whose node the tile owns (its energy clamps are
  // counted here); none if the column is not owned
  const int own_lo = max(1, R - ly0);
  const int own_hi = col.col_own
                         ? min(min(SH, R + TY - 1 - ly0), a.ny - 1 - (y0 - R) - ly0)
                         : -1;
  float4 pw01a1 = f4(0.f, 0.f, 0.f, 0.f), pw01a2 = pw01a1;
  float4 pw11a1 = pw01a1, pw11a2 = pw01a1;
  // rows PF ahead are in flight (asynchronous copies into the thread's
  // ring) while a row is formed: global-load latency is the walk's main
  // stall
  SrcRing ring = ring_of(a, rbase);
#pragma unroll
  for (int k = 0; k < PF; ++k) ring.template issue<INT>(a, col, y0, R, ly0 + k, k);
  float c1T, nxT, nyT;
  {
    bool emits, clamp;
    source_type(m, kq, emits, clamp, T, c1T, nxT, nyT);
    if (!emits) c1T = 1.0e6f;   // no source has this type
  }
  const LevelK lk = level_k(c1T);
  // Software pipeline: the equilibrium of row r + 1 is formed while row r
  // is deposited (two independent dependency chains per thread).
  // (a rolled loop: the walk's code stays small in the instruction cache)
  auto row_eq = [&](int r, int slot) {
    if (r + PF - 1 <= SH)
      cp_async_wait<PF - 1>();
    else
      cp_async_wait<0>();
    const float4 mm = ring.template take<INT>(a, col, y0, R, ly0 + r, slot);
    if (r + PF <= SH) ring.template issue<INT>(a, col, y0, R, ly0 + r + PF, slot);
    return source_eq_typed(mm, kq, lk, nxT, nyT);
  };
  SrcEqT qn = row_eq(0, 0);
  int slot = 1;
#pragma unroll 1
  for (int r = 0; r <= SH; ++r) {
    const int ly = ly0 + r;
    const SrcEqT q = qn;
    if (r < SH) {
      qn = row_eq(r + 1, slot);
      slot = slot + 1 == PF ? 0 : slot + 1;
    }
    fl.other |= q.emits && !q.mine;
    if (q.clamp && r >= own_lo && r <= own_hi) fl.clamps += 1;
    // level records L_v = d_v (1, V_x, V_y, E_b) of the sources of type T
    const float4 v4 = f4(1.0f, q.Vx, q.Vy, q.Eb);
    const float4 a1 = mul4(q.mine ? q.d1 : 0.0f, v4);
    const float4 a2 = mul4(q.mine ? q.d2 : 0.0f, v4);
    // corner weights (eq 29)
    const float gx1 = __fsub_rn(1.0f, q.fx), gy1 = __fsub_rn(1.0f, q.fy);
    const float w00 = __fmul_rn(gx1, gy1), w10 = __fmul_rn(q.fx, gy1);
    const float w01 = __fmul_rn(gx1, q.fy), w11 = __fmul_rn(q.fx, q.fy);
    // own-column part (this row's (0,0) corner and the row above's (0,1))
    // and the part for the column to the right ((1,0) and (1,1))
    const float4 t01 = fma4(w00, a1, pw01a1), t02 = fma4(w00, a2, pw01a2);
    const float4 t11 = fma4(w10, a1, pw11a1), t12 = fma4(w10, a2, pw11a2);
    pw01a1 = mul4(w01, a1);
    pw01a2 = mul4(w01, a2);
    pw11a1 = mul4(w11, a1);
    pw11a2 = mul4(w11, a2);
    const float4 u1 = shfl_up4(t11), u2 = shfl_up4(t12);
    if (r >= 1 && col.store_col) {
      D1[ly * DP + col.lx] = add4(t01, u1);
      D2[ly * DP + col.lx] = add4(t02, u2);
    }
  }
}


// Shift block of a window's groups: per axis the spread of n over the
// window's emitting sources, at most SPMAX, raised to the next block the
// group walk is built for (1x1, 2x2, 2x3, 3x2, 3x3, 3x4, 4x3, 4x4).  A
// block that holds a window's shifts deposits what the tightest one
// deposits, so raising it changes no result; a window wider than SPMAX on
// an axis keeps exactly SPMAX there (its groups are then split on that
// axis, and the split must not change).
struct Blk {
  int sx, sy;
};
__device__ __forceinline__ Blk blk_pick(int sx, int sy) {
  if (sx <= 1 && sy <= 1) return Blk{1, 1};
  if (sx <= 2 && sy <= 2) return Blk{2, 2};
  if (sx <= 2 && sy <= 3) return Blk{2, 3};
  if (sx <= 3 && sy <= 2) return Blk{3, 2};
  if (sx <= 3 && sy <= 3) return Blk{3, 3};
  if (sx <= 3) return Blk{3, 4};
  if (sy <= 3) return Blk{4, 3};
  return Blk{4, 4};
}
__device__ __forceinline__ int spread_axis(float lo, float hi) {
  const float s = hi - lo + 1.0f;
  return s <= 1.0f ? 1 : (s >= (float)SPMAX ? SPMAX : (int)s);
}
__device__ __forceinline__ Blk block_of(const GStats& st) {
  return blk_pick(spread_axis(st.nxmin, st.nxmax),
                  spread_axis(st.nymin, st.nymax));
}

// Per-tile record a step leaves for the next: 0 when the window held one
// type (or nothing), else bit 31 with the window's smallest c1 and shift and
// its block, or bit 31 and bit 30 when those do not fit the record; bit 28
// marks a tile whose carried-over block had to be redone.
constexpr unsigned kRecUnknown = 0xc0000000u;
constexpr unsigned kRecRedone = 0x10000000u;  // block redone at that step
__device__ __forceinline__ unsigned rec_encode(float c1min, float nxmin,
                                               float nymin, Blk B) {
  if (!(c1min <= 63.0f && nxmin >= -128.0f && nxmin <= 127.0f &&
        nymin >= -128.0f && nymin <= 127.0f))
    return kRecUnknown;
  return 0x80000000u | ((unsigned)(B.sy - 1) << 26) |
         ((unsigned)(B.sx - 1) << 24) | ((unsigned)c1min << 16) |
         ((unsigned)((int)nxmin + 128) << 8) | (unsigned)((int)nymin + 128);
}
__device__ __forceinline__ unsigned rec_of(const GStats& st) {
  if (st.c1max < 0.0f) return 0u;   // nothing emits
  if (st.c1min == st.c1max && st.nxmin == st.nxmax && st.nymin == st.nymax)
    return 0u;
  return rec_encode(st.c1min, st.nxmin, st.nymin, block_of(st));
}

// Statistics walk of a mixed tile without a usable record: c1 and shifts
// of every window source and the clamped energies of the owned nodes,
// without deposits.
template <bool INT>
__device__ __forceinline__ void walk_stats(const StepArgs& a, float* rbase,
                                           int x0, int y0, int R, int TX,
                                           int TY, GStats& st) {
  const Column col = column_of(a, x0, R, TX, INT);
  const int ly0 = SH * col.g;
  const float kq = a.k.kq_f;
  const int own_lo = max(1, R - ly0);
  const int own_hi = col.col_own
                         ? min(min(SH, R + TY - 1 - ly0), a.ny - 1 - (y0 - R) - ly0)
                         : -1;
  SrcRing ring = ring_of(a, rbase);
#pragma unroll
  for (int k = 0; k < PF; ++k) ring.template issue<INT>(a, col, y0, R, ly0 + k, k);
  int slot = 0;
#pragma unroll 1
  for (int r = 0; r <= SH; ++r) {
    if (r + PF - 1 <= SH)
      cp_async_wait<PF - 1>();
    else
      cp_async_wait<0>();
    const float4 m = ring.template take<INT>(a, col, y0, R, ly0 + r, slot);
    if (r + PF <= SH) ring.template issue<INT>(a, col, y0, R, ly0 + r + PF, slot);
    slot = slot + 1 == PF ? 0 : slot + 1;
    bool emits, clamp;
    float id, c1, nxf, nyf;
    source_type(m, kq, emits, clamp, id, c1, nxf, nyf);
    gstats_add(st, emits, c1, nxf, nyf);
    if (clamp && r >= own_lo && r <= own_hi) st.clamps += 1;
  }
}

// A group walk's view of one source: its level records (zero unless the
// source is in the group) and its hat weights over offsets 0 .. SX and
// 0 .. SY.
template <int SX, int SY>
struct GSrc {
  float4 l1, l2;
  float ax[SX + 1], ay[SY + 1];
};

// Group walk (block SX x SY): deposits the sources of group G, i.e. c1 =
// c1m + Gc and n in {a .. a+SX-1} x {b .. b+SY-1} with a = nxm + SX GX,
// b = nym + SY GY (G = Gc 65536 + GX 256 + GY):
//   D(q) = sum over the group's sources s and offsets o of
//          h_x(o_x) h_y(o_y) L(s),  q = s + o,
// h the hat weights of eq 29 at dn = n - (a, b): (1 - f) at dn, f at dn + 1.
// Deposit row t takes the sources of rows t - SY .. t of this column (kept
// from the rows walked before), oldest first, and, for o_x > 0, those of the
// columns to the left (shuffles by o_x).  Also gathers the window
// statistics and the next group above G.
template <int SX, int SY, bool INT>
__device__ __forceinline__ void walk_group(
    const StepArgs& a, float4* __restrict__ D1, float4* __restrict__ D2,
    float* rbase, int x0, int y0, int R, int TX, int TY,
    float G, float c1m, float nxm, float nym, bool count_clamps,
    GStats& st) {
  const Column col = column_of(a, x0, R, TX, INT);
  const int ly0 = SH * col.g - (SY - 1);
  constexpr int LAST = SH + SY - 1;
  const float kq = a.k.kq_f;
  // rows of this walk whose node the tile owns and that lie in the group's
  // deposit rows (each owned node counted by one walk)
  const int own_lo = max(SY, R - ly0);
  const int own_hi = col.col_own && count_clamps
                         ? min(min(LAST, R + TY - 1 - ly0), a.ny - 1 - (y0 - R) - ly0)
                         : -1;
  const float Gc = floorf(G * (1.0f / 65536.0f));
  const float Gr = __fmaf_rn(-65536.0f, Gc, G);
  const float GX = floorf(Gr * (1.0f / 256.0f));
  const float GY = __fmaf_rn(-256.0f, GX, Gr);
  // 1/SX, 1/SY rounded up (1/3 rounds up in FP32): exact floors of the
  // small integers they divide
  constexpr float rX = 1.0f / (float)SX, rY = 1.0f / (float)SY;
  // the group's level constants (its members' densities), where the
  // registers allow; larger blocks form them per source
  constexpr bool kGroupK = SX * SY <= 9;
  const LevelK lk = level_k(__fadd_rn(c1m, Gc));
  // h[k]: the source k + 1 rows above the current one
  GSrc<SX, SY> h[SY];
#pragma unroll
  for (int k = 0; k < SY; ++k) {
    h[k].l1 = h[k].l2 = f4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int o = 0; o <= SX; ++o) h[k].ax[o] = 0.0f;
#pragma unroll
    for (int o = 0; o <= SY; ++o) h[k].ay[o] = 0.0f;
  }
  SrcRing ring = ring_of(a, rbase);
#pragma unroll
  for (int k = 0; k < PF; ++k) ring.template issue<INT>(a, col, y0, R, ly0 + k, k);
  auto row_eq = [&](int r, int slot) {
    if (r + PF - 1 <= LAST)
      cp_async_wait<PF - 1>();
    else
      cp_async_wait<0>();
    const float4 m = ring.template take<INT>(a, col, y0, R, ly0 + r, slot);
    if (r + PF <= LAST) ring.template issue<INT>(a, col, y0, R, ly0 + r + PF, slot);
    return source_eq(m, kq, kGroupK ? &lk : nullptr);
  };
  SrcEq qn = row_eq(0, 0);
  int slot = 1;
#pragma unroll 1
  for (int r = 0; r <= LAST; ++r) {
    const int ly = ly0 + r;
    const SrcEq q = qn;
    if (r < LAST) {
      qn = row_eq(r + 1, slot);
      slot = slot + 1 == PF ? 0 : slot + 1;
    }
    // the source's group, relative to the assumed minima
    const float dc = __fsub_rn(q.c1, c1m);
    const float dx = __fsub_rn(q.nxf, nxm), dy = __fsub_rn(q.nyf, nym);
    const float gx = floorf(dx * rX), gy = floorf(dy * rY);
    const float gid = q.emits ? __fmaf_rn(65536.0f, dc, __fmaf_rn(256.0f, gx, gy))
                              : kNoType;
    const bool mine = gid == G;
    st.any |= mine;
    st.tnext = fminf(st.tnext, gid > G ? gid : kNoType);
    gstats_add(st, q.emits, q.c1, q.nxf, q.nyf);
    if (q.clamp && r >= own_lo && r <= own_hi) st.clamps += 1;
    GSrc<SX, SY> cur;
    const float4 v4 = f4(1.0f, q.Vx, q.Vy, q.Eb);
    cur.l1 = mul4(mine ? q.d1 : 0.0f, v4);
    cur.l2 = mul4(mine ? q.d2 : 0.0f, v4);
    const float dnx = __fmaf_rn(-(float)SX, gx, dx);
    const float dny = __fmaf_rn(-(float)SY, gy, dy);
    const float gx1 = __fsub_rn(1.0f, q.fx), gy1 = __fsub_rn(1.0f, q.fy);
    // hat weights: (1 - f) at dn, f at dn + 1 (one comparison per offset)
    bool px[SX], py[SY];
#pragma unroll
    for (int o = 0; o < SX; ++o) px[o] = dnx == (float)o;
#pragma unroll
    for (int o = 0; o < SY; ++o) py[o] = dny == (float)o;
    cur.ax[0] = px[0] ? gx1 : 0.0f;
#pragma unroll
    for (int o = 1; o < SX; ++o) cur.ax[o] = px[o] ? gx1 : (px[o - 1] ? q.fx : 0.0f);
    cur.ax[SX] = px[SX - 1] ? q.fx : 0.0f;
    cur.ay[0] = py[0] ? gy1 : 0.0f;
#pragma unroll
    for (int o = 1; o < SY; ++o) cur.ay[o] = py[o] ? gy1 : (py[o - 1] ? q.fy : 0.0f);
    cur.ay[SY] = py[SY - 1] ? q.fy : 0.0f;
    // deposit row ly: the part of this column's sources landing o_x columns
    // to the right, summed over their rows, then moved right by shuffles
    float4 D1r = f4(0.f, 0.f, 0.f, 0.f), D2r = D1r;
#pragma unroll
    for (int ox = 0; ox <= SX; ++ox) {
      // oldest source first, the current one last: with a 1 x 1 block the
      // one-type walk's operations in its order, so both give the same bits
      const float wl = __fmul_rn(h[SY - 1].ax[ox], h[SY - 1].ay[SY]);
      float4 t1 = mul4(wl, h[SY - 1].l1), t2 = mul4(wl, h[SY - 1].l2);
#pragma unroll
      for (int k = SY - 2; k >= 0; --k) {
        const float w = __fmul_rn(h[k].ax[ox], h[k].ay[k + 1]);
        t1 = fma4(w, h[k].l1, t1);
        t2 = fma4(w, h[k].l2, t2);
      }
      const float w0 = __fmul_rn(cur.ax[ox], cur.ay[0]);
      t1 = fma4(w0, cur.l1, t1);
      t2 = fma4(w0, cur.l2, t2);
      if (ox == 0) {
        D1r = t1;
        D2r = t2;
      } else {
        const float4 z = f4(0.f, 0.f, 0.f, 0.f);
        const bool ok = col.lane >= ox;
        const float4 s1 = shfl_up4n(t1, ox), s2 = shfl_up4n(t2, ox);
        D1r = add4(D1r, ok ? s1 : z);
        D2r = add4(D2r, ok ? s2 : z);
      }
    }
#pragma unroll
    for (int k = SY - 1; k > 0; --k) h[k] = h[k - 1];
    h[0] = cur;
    if (r >= SY && col.store_col) {
      D1[ly * DP + col.lx] = D1r;
      D2[ly * DP + col.lx] = D2r;
    }
  }
}

// The group walk for block B (the blocks blk_pick returns).
template <bool INT>
__device__ __forceinline__ void walk_group_blk(
    Blk B, const StepArgs& a, float4* __restrict__ D1,
    float4* __restrict__ D2, float* rbase, int x0, int y0, int R, int TX,
    int TY, float G, float c1m, float nxm, float nym, bool cc, GStats& st) {
  if (B.sx == 1)
    walk_group<1, 1, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sx == 2 && B.sy == 2)
    walk_group<2, 2, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sx == 2)
    walk_group<2, 3, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sx == 3 && B.sy == 2)
    walk_group<3, 2, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sx == 3 && B.sy == 3)
    walk_group<3, 3, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sx == 3)
    walk_group<3, 4, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else if (B.sy == 3)
    walk_group<4, 3, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
  else
    walk_group<4, 4, INT>(a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m, nxm,
                                  nym, cc, st);
}

// Arrivals of the four packets of one level with speed c (template C >= 0;
// C < 0: runtime c) at base position q of the deposits: +x, -x, +y, -y
// packets read D at q - c, q + c, q - c DP, q + c DP.
template <int C>
__device__ __forceinline__ float4 level_arrivals(const float4* __restrict__ P,
                                                 int q, int crt) {
  const int c = C >= 0 ? C : crt;
  const float cf = (float)c;
  const float4 A = P[q - c], B = P[q + c];
  const float4 Cu = P[q - c * DP], E = P[q + c * DP];
  const float4 s = add4(add4(A, B), add4(Cu, E));
  // mass; momentum + c (A - B) along x, + c (C - E) along y; energy
  // + c (A.mx - B.mx) + c (C.my - E.my) + c^2/2 mass (eq 14 with the cross
  // term 2 c'.V)
  const float mx = __fmaf_rn(cf, __fsub_rn(A.x, B.x), s.y);
  const float my = __fmaf_rn(cf, __fsub_rn(Cu.x, E.x), s.z);
  float en = __fmaf_rn(cf, __fsub_rn(A.y, B.y), s.w);
  en = __fmaf_rn(cf, __fsub_rn(Cu.z, E.z), en);
  en = __fmaf_rn(0.5f * cf * cf, s.x, en);
  return f4(s.x, mx, my, en);
}

// a - b in one packed instruction (exact: a fused multiply by -1).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
// Two compensated partial sums at once (Knuth's TwoSum on float pairs, as
// sum2_add does for one).
struct Sum2x2 {
  float2 hi, lo;
};
__device__ __forceinline__ void sum2x2_add(Sum2x2& a, float2 v) {
  const float2 s = __fadd2_rn(a.hi, v);
  const float2 bb = sub2(s, a.hi);
  const float2 e = __fadd2_rn(sub2(a.hi, sub2(s, bb)), sub2(v, bb));
  a.hi = s;
  a.lo = __fadd2_rn(a.lo, e);
}

// Compensated arrivals of one level: the four packets' fields (eqs 12-14
// from the deposited level record, the cross term 2 c'.V included), each
// added into the destination's (hi, lo) sums by TwoSum.
template <int C>
__device__ __forceinline__ void level_arrivals_comp(
    const float4* __restrict__ P, int q, int crt, Sum2x2& s01, Sum2x2& s23) {
  const int c = C >= 0 ? C : crt;
  const float cf = (float)c, k2 = 0.5f * cf * cf;
  const float4 A = P[q - c], B = P[q + c];
  const float4 Cu = P[q - c * DP], E = P[q + c * DP];
  // +x and -x packets: momentum +-c d along x, energy +-c (d V_x) + c^2/2 d
  sum2x2_add(s01, make_float2(A.x, __fmaf_rn(cf, A.x, A.y)));
  sum2x2_add(s23, make_float2(A.z, __fmaf_rn(cf, A.y, __fmaf_rn(k2, A.x, A.w))));
  sum2x2_add(s01, make_float2(B.x, __fmaf_rn(-cf, B.x, B.y)));
  sum2x2_add(s23, make_float2(B.z, __fmaf_rn(-cf, B.y, __fmaf_rn(k2, B.x, B.w))));
  // +y and -y packets
  sum2x2_add(s01, make_float2(Cu.x, Cu.y));
  sum2x2_add(s23, make_float2(__fmaf_rn(cf, Cu.x, Cu.z),
                              __fmaf_rn(cf, Cu.z, __fmaf_rn(k2, Cu.x, Cu.w))));
  sum2x2_add(s01, make_float2(E.x, E.y));
  sum2x2_add(s23, make_float2(__fmaf_rn(-cf, E.x, E.z),
                              __fmaf_rn(-cf, E.z, __fmaf_rn(k2, E.x, E.w))));
}

template <int C1, bool KAHAN>
__device__ __forceinline__ float4 gather_one(const float4* __restrict__ D1,
                                             const float4* __restrict__ D2,
                                             int q, int c1) {
  if constexpr (KAHAN) {
    Sum2x2 s01{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, s23 = s01;
    level_arrivals_comp<C1>(D1, q, c1, s01, s23);
    level_arrivals_comp<(C1 >= 0 ? C1 + 1 : -1)>(D2, q, c1 + 1, s01, s23);
    const float2 a = __fadd2_rn(s01.hi, s01.lo), b = __fadd2_rn(s23.hi, s23.lo);
    return f4(a.x, a.y, b.x, b.y);
  } else {
    const float4 y1 = level_arrivals<C1>(D1, q, c1);
    const float4 y2 = level_arrivals<(C1 >= 0 ? C1 + 1 : -1)>(D2, q, c1 + 1);
    return add4(y1, y2);
  }
}

// Per-destination end of the step: write, reach and state check of the new
// node, compensated partial totals: s01 for (rho, m_x), s23 for (m_y, rhoE).
struct TileOut {
  int reach;
  bool bad;
  Sum2x2 s01, s23;
};

__device__ __forceinline__ void finish_node(const StepArgs& a, bool valid,
                                            long long o, float4 v,
                                            TileOut& t) {
  if (valid) {
    static_cast<float*>(a.out[0])[o] = v.x;
    static_cast<float*>(a.out[1])[o] = v.y;
    static_cast<float*>(a.out[2])[o] = v.z;
    static_cast<float*>(a.out[3])[o] = v.w;
  } else {
    v = f4(0.f, 0.f, 0.f, 0.f);
  }
  const EqCore c = eq_core(v.x, v.y, v.z, v.w, a.k.kq_f);
  const float c1 = c1_exact(c.X);
  const bool emits = v.x > 0.0f;
  t.reach = max(t.reach, reach_of(emits, c, c1));
  const bool finite_in = fabsf(v.x + v.y + v.z + v.w) <= 3.0e38f;
  t.bad |= !finite_in || v.x < 0.0f ||
           (v.x > 0.0f && v.x < 1.17549435e-38f) || !(c.X <= 1099511627776.0f);
  if (a.do_cons) {
    sum2x2_add(t.s01, make_float2(v.x, v.y));
    sum2x2_add(t.s23, make_float2(v.z, v.w));
  }
}

// Destinations of this thread: tile positions tid, tid + NTHR, ... in
// row-major order over the TX x TY tile.
struct DestWalk {
  int dx, dy, sx, sy, TX;
  __device__ __forceinline__ void init(int k, int tx) {
    TX = tx;
    dy = k / TX;
    dx = k - dy * TX;
    sy = NTHR / TX;
    sx = NTHR - sy * TX;
  }
  __device__ __forceinline__ void next() {
    dy += sy;
    dx += sx;
    if (dx >= TX) {
      dx -= TX;
      ++dy;
    }
  }
};

// Gather pass for type T over the tile: first pass writes, later passes
// add to what the earlier passes wrote; the last pass finishes the nodes.
template <int C1, bool KAHAN>
__device__ __forceinline__ void gather_pass(const StepArgs& a,
                                           const float4* __restrict__ D1,
                                           const float4* __restrict__ D2,
                                           int x0, int y0, int R, int TX,
                                           int TY, Type ty, bool first,
                                           bool last, TileOut& t) {
  DestWalk w;
  w.init(threadIdx.x, TX);
  const int n = TX * TY;
  const int iters = (n + NTHR - 1) / NTHR;
  // one destination's arrivals, the RMW of earlier passes, its end
  auto dest = [&](const DestWalk& d, float4 v, bool in_tile) {
    const int x = x0 + d.dx, y = y0 + d.dy;
    const bool valid = in_tile && x < a.nx && y < a.ny;
    const long long o = (long long)y * a.nx + x;
    if (!first && valid) {
      const float4 p = f4(static_cast<const float*>(a.out[0])[o],
                          static_cast<const float*>(a.out[1])[o],
                          static_cast<const float*>(a.out[2])[o],
                          static_cast<const float*>(a.out[3])[o]);
      v = add4(p, v);
    }
    if (last) {
      finish_node(a, valid, o, v, t);
    } else if (valid) {
      static_cast<float*>(a.out[0])[o] = v.x;
      static_cast<float*>(a.out[1])[o] = v.y;
      static_cast<float*>(a.out[2])[o] = v.z;
      static_cast<float*>(a.out[3])[o] = v.w;
    }
  };
  auto arrivals = [&](const DestWalk& d, bool in_tile) {
    float4 v = f4(0.f, 0.f, 0.f, 0.f);
    if (in_tile) {
      const int q = (R + d.dy - ty.ny) * DP + (R + d.dx - ty.nx);
      v = gather_one<C1, KAHAN>(D1, D2, q, ty.c1);
    }
    return v;
  };
  // two destinations per round: their reads and sums interleave
  for (int it = 0; it < iters; it += 2) {
    DestWalk w2 = w;
    w2.next();
    const bool two = it + 1 < iters;   // uniform over the block
    const bool in1 = w.dy < TY, in2 = two && w2.dy < TY;
    const float4 v1 = arrivals(w, in1);
    const float4 v2 = arrivals(w2, in2);
    dest(w, v1, in1);
    if (two) dest(w2, v2, in2);
    w = w2;
    w.next();
  }
}

template <bool KAHAN>
__device__ __forceinline__ void gather_dispatch(const StepArgs& a,
                                                const float4* D1,
                                                const float4* D2, int x0,
                                                int y0, int R, int TX, int TY,
                                                Type ty, bool first, bool last,
                                                TileOut& t) {
  // one instantiation with the level speeds at run time (a few address
  // additions more than compile-time offsets, far less code)
  gather_pass<-1, KAHAN>(a, D1, D2, x0, y0, R, TX, TY, ty, first, last, t);
}

// Finishes every destination of the tile without a gather: with zeros
// (nothing landed) when first, else with what earlier passes wrote.  All
// threads run the same number of iterations (c1_exact is warp-collective).
__device__ __forceinline__ void finish_tile(const StepArgs& a, int x0, int y0,
                                            int TX, int TY, bool first,
                                            TileOut& t) {
  const int n = TX * TY;
  const int iters = (n + NTHR - 1) / NTHR;
  for (int it = 0; it < iters; ++it) {
    const int k = threadIdx.x + it * NTHR;
    const int dy = k / TX, dx = k - dy * TX;
    const int x = x0 + dx, y = y0 + dy;
    const bool valid = k < n && x < a.nx && y < a.ny;
    const long long o = (long long)y * a.nx + x;
    float4 v = f4(0.f, 0.f, 0.f, 0.f);
    if (valid && !first)
      v = f4(static_cast<const float*>(a.out[0])[o],
             static_cast<const float*>(a.out[1])[o],
             static_cast<const float*>(a.out[2])[o],
             static_cast<const float*>(a.out[3])[o]);
    finish_node(a, valid, o, v, t);
  }
}

// Every packet of a one-type walk (slack 0) or of a group walk (slack 1:
// its base may lie below its sources' shift) within reach R reads deposits
// that lie in rows 1 .. 48 and columns 1 .. 59.
__device__ __forceinline__ bool type_fits(Type ty, int R, int slack) {
  const int c2 = ty.c1 + 1;
  return ty.nx <= R - 1 - c2 && -ty.nx <= R - c2 + slack &&
         ty.ny <= R - 1 - c2 && -ty.ny <= R - c2 + slack;
}

// Tile geometry of a step: reach R (at least 1), tile size, tile count.
struct TileGeo {
  int R, TX, TY, tiles_x, ntiles;
  bool over;  // the reach exceeds the layout or the handle's limit
};
__device__ __forceinline__ TileGeo geo_of(const StepArgs& a) {
  TileGeo g;
  const int R0 = a.scr->reach;
  g.R = R0 < 1 ? 1 : R0;
  g.TX = tile_w(g.R);
  g.TY = tile_h(g.R);
  g.tiles_x = (a.nx + g.TX - 1) / g.TX;
  g.ntiles = g.tiles_x * ((a.ny + g.TY - 1) / g.TY);
  g.over = R0 > a.r_cap || R0 > RMAX;
  return g;
}

// Block-wide end of a tile: its reach, bad-state flag and compensated
// partial totals (part[b], the finalize kernel sums them).
struct TileRed {
  float2 sum[4][NWARP];
  int reach[NWARP];
  int bad[NWARP];
};
__device__ __forceinline__ void tile_publish(const StepArgs& a, int b,
                                             const TileOut& to, TileRed& red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = __reduce_max_sync(0xffffffffu, to.reach);
  const int bad = __any_sync(0xffffffffu, to.bad) ? 1 : 0;
  if (a.do_cons) {
    const Sum2 ps[4] = {{to.s01.hi.x, to.s01.lo.x}, {to.s01.hi.y, to.s01.lo.y},
                        {to.s23.hi.x, to.s23.lo.x}, {to.s23.hi.y, to.s23.lo.y}};
    const Sum2 k = warp_sum2_fields(ps, lane);
    if ((lane & 7) == 0) red.sum[lane >> 3][warp] = make_float2(k.hi, k.lo);
  }
  if (lane == 0) {
    red.reach[warp] = r;
    red.bad[warp] = bad;
  }
  __syncthreads();
  if (warp == 0) {
    int rb = lane < NWARP ? red.reach[lane] : 0;
    rb = __reduce_max_sync(0xffffffffu, rb);
    const int bb = __any_sync(0xffffffffu, lane < NWARP && red.bad[lane] != 0);
    if (lane == 0) {
      atomicMax(&a.scr->reach_next, rb);
      if (bb) atomicOr(&a.scr->flags, kFlagState);
    }
    if (a.do_cons) {
      static_assert(NWARP == 8, "one lane per (field, warp)");
      const Sum2 s = combine_warps_f2<NWARP>(red.sum, lane);
      if ((lane & 7) == 0)
        reinterpret_cast<float2*>(a.part)[(long long)b * 4 + (lane >> 3)] =
            make_float2(s.hi, s.lo);
    }
  }
}

__device__ __forceinline__ TileOut tile_out_init() {
  TileOut to;
  to.reach = 0;
  to.bad = false;
  to.s01 = to.s23 = Sum2x2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  return to;
}

// Commits the block's clamped-energy count (one atomic per warp).
__device__ __forceinline__ void commit_clamps(const StepArgs& a, unsigned c) {
  const unsigned cl = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && cl)
    atomicAdd(&a.scr->eclamps, (unsigned long long)cl);
}

// Shared memory of a deposit block: the two deposit planes and the source
// ring (dynamic), the statistics and totals scratch (static).
struct DsSmem {
  float4* D1;
  float4* D2;
  float* rbase;
  int* red;
  TileRed* tred;
};
// Tile b of the grid a describes (the tiles of the largest reach are
// numbered; those beyond the step's count only clear their partial totals),
// if its window holds one type; returns true when the tile is left for the
// group walks (ds_mixed_tile): its window held several types at the last
// step, or turns out to hold several now.
template <bool KAHAN>
__device__ __forceinline__ bool ds_first_tile(const StepArgs& a, int b,
                                              const DsSmem& sm) {
  float4* D1 = sm.D1;
  float4* D2 = sm.D2;
  float* rbase = sm.rbase;
  const int tid = threadIdx.x;
  const TileGeo g = geo_of(a);
  if (g.over || b >= g.ntiles) {
    if (g.over && tid == 0 && b == 0) atomicOr(&a.scr->flags, kFlagReach);
    if (a.do_cons && tid < 4)
      reinterpret_cast<float2*>(a.part)[(long long)b * 4 + tid] =
          make_float2(0.f, 0.f);
    return false;
  }
  if (a.hint[b]) return true;
  const int R = g.R, TX = g.TX, TY = g.TY;
  const int ty_i = b / g.tiles_x, tx_i = b - ty_i * g.tiles_x;
  const int x0 = tx_i * TX, y0 = ty_i * TY;
  const bool interior = x0 - R >= 0 && x0 - R + WCOLS <= a.nx &&
                        y0 - R >= 0 && y0 - R + WROWS <= a.ny;

  // guess: the type of the tile's central node (every thread forms it; its
  // load overlaps the walk's first loads)
  float T0;
  OneTypeFlags fl{0u, false};
  {
    const int cx = min(x0 + TX / 2, a.nx - 1), cy = min(y0 + TY / 2, a.ny - 1);
    const long long i = (long long)cy * a.nx + cx;
    const float4 m = f4(__ldg(static_cast<const float*>(a.in[0]) + i),
                        __ldg(static_cast<const float*>(a.in[1]) + i),
                        __ldg(static_cast<const float*>(a.in[2]) + i),
                        __ldg(static_cast<const float*>(a.in[3]) + i));
    // interior windows need no boundary handling: their own, smaller walk
    if (interior)
      walk_one_type<true>(a, D1, D2, rbase, x0, y0, R, TX, TY, m, T0, fl);
    else
      walk_one_type<false>(a, D1, D2, rbase, x0, y0, R, TX, TY, m, T0, fl);
  }
  // the barrier after the deposits, with the block's flag; without another
  // type in the window, nothing emits exactly when the central node does
  // not (every emitting source would have another type than its kNoType)
  const bool other = __syncthreads_or(fl.other) != 0;
  const bool none = T0 == kNoType;
  if (other) {
    // the group walks find the window's minima and count its clamps
    if (tid == 0) a.hint[b] = kRecUnknown;
    return true;
  }
  commit_clamps(a, fl.clamps);
  TileOut to = tile_out_init();
  if (none) {
    finish_tile(a, x0, y0, TX, TY, true, to);  // nothing lands
  } else {
    const Type ty = decode_type(T0);
    if (type_fits(ty, R, 0)) {
      gather_dispatch<KAHAN>(a, D1, D2, x0, y0, R, TX, TY, ty, true, true, to);
    } else {
      if (tid == 0) atomicOr(&a.scr->flags, kFlagReach);
      finish_tile(a, x0, y0, TX, TY, true, to);
    }
  }
  tile_publish(a, b, to, *sm.tred);
  return false;
}

// Tile b whose window holds several types: its sources are grouped by c1
// and by shift blocks (c1 relative to the window's smallest, n relative to
// the smallest shift in blocks of SX x SY); one group walk per group, in
// ascending group order, each gather adding its arrivals.  The minima and
// block come from the tile's record of the previous step; when the first
// walk finds that the block does not hold the window, the walks restart
// from the window's own minima and block.  What a tile computes depends
// only on the state.
template <bool KAHAN>
__device__ __forceinline__ void ds_mixed_tile(const StepArgs& a, int b,
                                              const DsSmem& sm) {
  float4* D1 = sm.D1;
  float4* D2 = sm.D2;
  float* rbase = sm.rbase;
  int* red = sm.red;
  const int tid = threadIdx.x;
  const TileGeo g = geo_of(a);
  if (g.over) return;
  const int R = g.R, TX = g.TX, TY = g.TY;
  {
    const int ty_i = b / g.tiles_x, tx_i = b - ty_i * g.tiles_x;
    const int x0 = tx_i * TX, y0 = ty_i * TY;
    const bool interior = x0 - R >= 0 && x0 - R + WCOLS <= a.nx &&
                          y0 - R >= 0 && y0 - R + WROWS <= a.ny;
    const unsigned rec = a.hint[b];
    float c1m, nxm, nym;
    Blk B;
    bool counted = false, checked = false, redone = false;
    // a tile whose carried-over block failed at the last step starts with
    // the statistics walk (cheaper than a group walk redone)
    if ((rec & 0xd0000000u) == 0x80000000u) {
      B = blk_pick((int)((rec >> 24) & 3u) + 1, (int)((rec >> 26) & 3u) + 1);
      c1m = (float)((rec >> 16) & 0xffu);
      nxm = (float)((int)((rec >> 8) & 0xffu) - 128);
      nym = (float)((int)(rec & 0xffu) - 128);
    } else {
      GStats s0 = gstats_init();
      if (interior)
        walk_stats<true>(a, rbase, x0, y0, R, TX, TY, s0);
      else
        walk_stats<false>(a, rbase, x0, y0, R, TX, TY, s0);
      commit_clamps(a, s0.clamps);
      counted = true;
      reduce_gstats(s0, red);
      c1m = s0.c1min;
      nxm = s0.nxmin;
      nym = s0.nymin;
      B = block_of(s0);
      checked = true;
    }
    float G = 0.0f;  // (c1m, blocks (0, 0)); possibly empty
    bool first = true;
    while (true) {
      __syncthreads();  // the previous gather and statistics are done
      GStats s2 = gstats_init();
      const bool cc = !counted;
      if (interior)
        walk_group_blk<true>(B, a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m,
                             nxm, nym, cc, s2);
      else
        walk_group_blk<false>(B, a, D1, D2, rbase, x0, y0, R, TX, TY, G, c1m,
                              nxm, nym, cc, s2);
      if (!counted) commit_clamps(a, s2.clamps);
      counted = true;
      reduce_gstats(s2, red);
      if (!checked) {
        // the result must follow from this step's state alone.  Groups go
        // in ascending c1, and on an axis where the window's shifts span
        // at most SPMAX any block that holds them all deposits the same
        // values (offsets outside the sources' range add exact zeros in
        // the same order), so minima and block taken from an earlier step
        // stand when the c1 minimum is not above the state's and each axis
        // holds its shifts; a wider axis needs blocks of SPMAX from the
        // state's minimum.  (And the packets of the largest level speed
        // must stay within the deposits, which a block based below the
        // state's minima can miss.)
        checked = true;
        const bool wx = s2.nxmax - s2.nxmin >= (float)SPMAX;
        const bool wy = s2.nymax - s2.nymin >= (float)SPMAX;
        const bool okx = wx ? (nxm == s2.nxmin && B.sx == SPMAX)
                            : (nxm <= s2.nxmin &&
                               s2.nxmax <= nxm + (float)(B.sx - 1));
        const bool oky = wy ? (nym == s2.nymin && B.sy == SPMAX)
                            : (nym <= s2.nymin &&
                               s2.nymax <= nym + (float)(B.sy - 1));
        const bool holds =
            c1m <= s2.c1min && okx && oky &&
            type_fits(Type{(int)nxm, (int)nym, (int)s2.c1max}, R, 1);
        if (s2.c1max >= 0.0f && !holds) {
          redone = true;
          c1m = s2.c1min;
          nxm = s2.nxmin;
          nym = s2.nymin;
          B = block_of(s2);
          G = 0.0f;
          continue;
        }
      }
      const bool last = !(s2.tnext < kNoType);
      // the node ends and totals of the last pass (nothing held across
      // the walks)
      TileOut to = tile_out_init();
      const float Gc = floorf(G * (1.0f / 65536.0f));
      const float Gr = __fmaf_rn(-65536.0f, Gc, G);
      const float GX = floorf(Gr * (1.0f / 256.0f));
      const float GY = __fmaf_rn(-256.0f, GX, Gr);
      const Type ty{(int)__fmaf_rn((float)B.sx, GX, nxm),
                    (int)__fmaf_rn((float)B.sy, GY, nym), (int)(c1m + Gc)};
      if (s2.any && type_fits(ty, R, 1)) {
        gather_dispatch<KAHAN>(a, D1, D2, x0, y0, R, TX, TY, ty, first, last,
                               to);
        first = false;
      } else {
        if (s2.any && tid == 0) atomicOr(&a.scr->flags, kFlagReach);
        if (last) finish_tile(a, x0, y0, TX, TY, first, to);
      }
      if (last) {
        if (tid == 0) {
          const unsigned r = rec_of(s2);
          a.hint[b] = r != 0u && redone ? (r | kRecRedone) : r;
        }
        tile_publish(a, b, to, *sm.tred);
        break;
      }
      G = s2.tnext;
    }
  }
}

// The step in one persistent kernel: blocks take tiles by ticket (all the
// tiles of the largest reach); a tile whose window held several types at
// the last step, or turns out to hold several now, goes on to the group
// walks in the same block.  No queue, no second launch, and no idle tail
// between the one-type and the mixed tiles.  Same tile code, so the same
// results as the two kernels.
template <bool KAHAN>
__global__ void __launch_bounds__(NTHR, 2) step2d_ds_fused(const StepArgs a) {
  extern __shared__ __align__(16) float4 dsm[];
  __shared__ int red[NGSTAT * NWARP];
  __shared__ TileRed tred;
  __shared__ int s_k[2];
  const DsSmem sm{dsm, dsm + PLANE, reinterpret_cast<float*>(dsm + 2 * PLANE),
                  red, &tred};
  if (threadIdx.x == 0) s_k[0] = (int)atomicAdd(&a.scr->mixed_ticket, 1u);
  for (int it = 0;; ++it) {
    __syncthreads();  // the ticket is visible; the last tile is done
    const int k = s_k[it & 1];
    if (k >= a.nblocks) break;
    // the next ticket, taken now into the other slot: its latency hides
    // behind this tile
    if (threadIdx.x == 0)
      s_k[(it + 1) & 1] = (int)atomicAdd(&a.scr->mixed_ticket, 1u);
    if (ds_first_tile<KAHAN>(a, k, sm)) {
      __syncthreads();  // the walk's deposits and record are settled
      ds_mixed_tile<KAHAN>(a, k, sm);
    }
  }
}

// After each step (FIN_BLOCKS blocks): the tiles' compensated (hi, lo)
// partial totals summed in compensated FP32 in a fixed order -- block j
// takes the j-th of FIN_BLOCKS equal runs of tiles, the last block to finish
// sums the blocks' results in block order and converts them to FP64 once per
// field -- and the reach hand-off to the next step.  A step that met a reach
// beyond its layout leaves the reach as it was, so later steps report the
// same error.  The blocks' results follow the tiles' partials in part.
constexpr int FIN_BLOCKS = 32;
// Block j of a grid's FIN_BLOCKS finalize blocks (all threads call it).
__device__ __forceinline__ void ds_finalize_part(Scratch* scr,
                                                 double* __restrict__ part,
                                                 int nblk, int do_cons,
                                                 int j) {
  __shared__ float2 red[4][NWARP];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* fin = reinterpret_cast<float2*>(part) + (long long)nblk * 4;
  if (do_cons) {
    const int chunk = (nblk + FIN_BLOCKS - 1) / FIN_BLOCKS;
    const int lo = j * chunk;
    const int hi = min(nblk, lo + chunk);
    // each thread a fixed strided set of tiles, four at a time (their loads
    // in flight together), then a fixed combine
    const float4* p4 = reinterpret_cast<const float4*>(part);
    constexpr int U = 4;
    Sum2 s4[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int f = 0; f < 4; ++f) s4[u][f] = Sum2{0.f, 0.f};
    for (int b0 = lo + tid; b0 < hi; b0 += U * NTHR) {
      float4 v[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int b = b0 + u * NTHR;
        const bool ok = b < hi;
        v[u][0] = ok ? p4[(long long)b * 2] : f4(0.f, 0.f, 0.f, 0.f);
        v[u][1] = ok ? p4[(long long)b * 2 + 1] : f4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        s4[u][0] = sum2_add(s4[u][0], Sum2{v[u][0].x, v[u][0].y});
        s4[u][1] = sum2_add(s4[u][1], Sum2{v[u][0].z, v[u][0].w});
        s4[u][2] = sum2_add(s4[u][2], Sum2{v[u][1].x, v[u][1].y});
        s4[u][3] = sum2_add(s4[u][3], Sum2{v[u][1].z, v[u][1].w});
      }
    }
#pragma unroll
    for (int u = 1; u < U; ++u)
#pragma unroll
      for (int f = 0; f < 4; ++f) s4[0][f] = sum2_add(s4[0][f], s4[u][f]);
    const Sum2 k = warp_sum2_fields(s4[0], lane);
    if ((lane & 7) == 0) red[lane >> 3][warp] = make_float2(k.hi, k.lo);
    __syncthreads();
    if (warp == 0) {
      const Sum2 t = combine_warps_f2<NWARP>(red, lane);
      if ((lane & 7) == 0)
        fin[(long long)j * 4 + (lane >> 3)] = make_float2(t.hi, t.lo);
      __threadfence();
    }
  }
  __syncthreads();
  if (tid == 0) last = atomicAdd(&scr->ticket, 1u) == FIN_BLOCKS - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (do_cons && warp == 0) {
    static_assert(FIN_BLOCKS == 32, "one lane per block result");
    Sum2 ps[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float2 v = __ldcg(&fin[(long long)lane * 4 + f]);
      ps[f] = Sum2{v.x, v.y};
    }
    const Sum2 t = warp_sum2_fields(ps, lane);
    if ((lane & 7) == 0) scr->cons[lane >> 3] = (double)t.hi + (double)t.lo;
  }
  if (tid == 0) {
    if (!(scr->flags & kFlagReach)) scr->reach = scr->reach_next;
    scr->reach_next = 0;
    scr->ticket = 0u;
    scr->mixed_ticket = 0u;
  }
}

}  // namespace ds
}  // namespace lbm
