// Square-lattice step from source records: a records pass forms every
// source's packets, level densities and corner weights once per step (over
// the grid padded by the reach limit, additional points of Section V.B
// included), and the gather reads them instead of forming the equilibrium
// of every window source in every tile.  The arithmetic and the sum order
// are those of step_kernel.cuh, so the FP64 instance (built with
// -fmad=false) is bit-identical with the oracle.  Used by FP64 handles; in
// FP32 the records' traffic (30 fields per source written and read) costs
// more than forming the equilibria in every tile (measured 11 % slower on
// the 4096 x 512 tube with compensated sums).
#pragma once

#include "step_kernel.cuh"

namespace lbm {

// The word array follows the kRecWord field arrays of T.
template <typename T>
__device__ __forceinline__ long long* rec_words(T* Sr, long long n) {
  return reinterpret_cast<long long*>(Sr + kRecWord * n);
}
template <typename T>
__device__ __forceinline__ const long long* rec_words(const T* Sr,
                                                      long long n) {
  return reinterpret_cast<const long long*>(Sr + kRecWord * n);
}

// Square lattice: the source records of the input state, one thread per
// source of the padded grid (rows of nx + 2 r_cap, r_cap rows above and
// below), written before each step.  A source outside the grid is the
// additional point of Section V.B: its equilibrium is formed from the
// supplying node's moments with the mirrored momentum component negated,
// exactly as a step forms it.  Energy clamps and bad states are counted
// here, once per node of the grid.
template <typename T>
__global__ void __launch_bounds__(256) records2d(const StepArgs a) {
  const int rc = a.r_cap;
  const long long PX = (long long)a.nx + 2 * rc, PY = (long long)a.ny + 2 * rc;
  const long long n = PX * PY;
  T* Sr = static_cast<T*>(a.src);
  unsigned long long clamps = 0;
  bool bad = false;
  const long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long py = blockIdx.y; py < PY && px < PX; py += gridDim.y) {
    const long long sx = px - rc, sy = py - rc;
    bool fx, fy;
    const int gx = virtual_axis(a.bc_x, a.nx, sx, &fx);
    const int gy = virtual_axis(a.bc_y, a.ny, sy, &fy);
    const long long g = (long long)gy * a.nx + gx;
    T mx = ld<T>(a.in[1], g), my = ld<T>(a.in[2], g);
    if (fx) mx = -mx;
    if (fy) my = -my;
    const Equil<T> q = equilibrium<T, 2>(ld<T>(a.in[0], g), mx, my,
                                         ld<T>(a.in[3], g), a.k);
    if (sx >= 0 && sx < a.nx && sy >= 0 && sy < a.ny) {
      clamps += q.clamp ? 1 : 0;
      bad |= q.bad;
    }
    const long long i = py * PX + px;
    long long w = s64_word(-1, 0, 0);
    if (q.emits) {
#pragma unroll
      for (int p = 0; p < TileShape<2>::NP; ++p) {
        T ppx, ppy, ppe;
        packet_fields<T, 2>(q, p, &ppx, &ppy, &ppe);
        Sr[(kRecPx + p) * n + i] = ppx;
        Sr[(kRecPy + p) * n + i] = ppy;
        Sr[(kRecPE + p) * n + i] = ppe;
      }
      Sr[kRecMass * n + i] = q.d1;
      Sr[(kRecMass + 1) * n + i] = q.d2;
      T w4[4];
      corner_weights(q, w4);
#pragma unroll
      for (int k = 0; k < 4; ++k) Sr[(kRecW + k) * n + i] = w4[k];
      w = s64_word(q.c1, q.n0, q.n1);
    }
    rec_words(Sr, n)[i] = w;
  }
  const unsigned wc = __reduce_add_sync(0xffffffffu, (unsigned)clamps);
  const bool wb = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (wc) atomicAdd(&a.scr->eclamps, (unsigned long long)wc);
    if (wb) atomicOr(&a.scr->flags, kFlagState);
  }
}

// The source records as the gather reads them: one base pointer per field
// group, cap = sources per array.
template <typename T>
struct RecLayout {
  long long cap;
  const T* Px;
  const T* Py;
  const T* PE;
  const T* mass;
  const T* wt;
  const long long* word;
};

__device__ __forceinline__ void decode_word(long long w, int* c1, int* n0,
                                            int* n1) {
  *c1 = (short)(w & 0xffff);
  *n0 = (short)((w >> 16) & 0xffff);
  *n1 = (short)((w >> 32) & 0xffff);
}

// Gather of one destination from the records by testing every candidate
// source within reach R, in the order of step_kernel's scan (rows at
// distance j above then below, sources left to right, packet, corner; row
// sums added as pairs).  s0: the destination's index, PX: the padded row
// length.
template <typename T, bool KAHAN>
__device__ __noinline__ void scan_gather_rec(const RecLayout<T>& L,
                                             long long s0, long long PX, int R,
                                             T (&tot)[4], T (&comp)[4]) {
  for (int j = 0; j <= R; ++j) {
    T pair[4];
    for (int side = 0; side < (j == 0 ? 1 : 2); ++side) {
      const int dyo = side == 0 ? j : -j;  // destination row - source row
      const long long base = s0 - (long long)dyo * PX - R;
      T r = T(0), x = T(0), y = T(0), e = T(0);
      for (int i = 0; i <= 2 * R; ++i) {
        const long long s = base + i;
        int c1, n0, n1;
        decode_word(L.word[s], &c1, &n0, &n1);
        if (c1 < 0) continue;
        const int c2 = c1 + 1;
        const int ox = R - i - n0;
        const int oy = dyo - n1;
        const bool near_x = ox >= -c2 && ox <= c2 + 1;
        const bool near_y = oy >= -c2 && oy <= c2 + 1;
        const bool xarm = (oy == 0 || oy == 1) && near_x;
        const bool yarm = (ox == 0 || ox == 1) && near_y;
        if (!xarm && !yarm) continue;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          int cx, cy, lev;
          packet<2>(p, c1, &cx, &cy, &lev);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (cx + (kk & 1) != ox || cy + (kk >> 1) != oy) continue;
            const T al = L.wt[kk * L.cap + s];
            r = r + al * L.mass[lev * L.cap + s];
            x = x + al * L.Px[p * L.cap + s];
            y = y + al * L.Py[p * L.cap + s];
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
    add_pair<T, KAHAN>(tot, comp, pair);
  }
}

// Square-lattice step from the source records: one destination per thread,
// 32 x 8 tiles, no shared-memory window (the gather reads the records
// through the cache), so that several blocks share a multiprocessor.  Same
// sums, in the same order, as step_kernel<T, 2, KAHAN>.
template <typename T, bool KAHAN>
__global__ void __launch_bounds__(256, 2) step2d_rec(const StepArgs a) {
  using S = TileShape<2>;
  constexpr int NT = S::TX * S::TY;
  __shared__ unsigned red_tmin[NT / 32], red_tmax[NT / 32];
  const int tid = threadIdx.x;
  const int R = a.scr->reach;
  if (R > a.r_cap) {
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0)
      atomicOr(&a.scr->flags, kFlagReach);
    return;
  }
  const int rc = a.r_cap;
  const long long PX = (long long)a.nx + 2 * rc;
  const long long cap = PX * ((long long)a.ny + 2 * rc);
  const T* Sr = static_cast<const T*>(a.src);
  const RecLayout<T> L{cap,
                       Sr + kRecPx * cap,
                       Sr + kRecPy * cap,
                       Sr + kRecPE * cap,
                       Sr + kRecMass * cap,
                       Sr + kRecW * cap,
                       rec_words(Sr, cap)};
  const int x0 = blockIdx.x * S::TX, y0 = blockIdx.y * S::TY;
  // the window of the tile's destinations inside the grid (a tile at the
  // far edge may be partial; the padded records end r_cap past the grid)
  const int W = min(S::TX, a.nx - x0) + 2 * R;
  const int H = min(S::TY, a.ny - y0) + 2 * R;

  // one type for the whole window?
  unsigned tmin = 0xffffffffu, tmax = 0u;
  for (int i = tid; i < W * H; i += NT) {
    const int ly = i / W, lx = i - ly * W;
    const long long s = (long long)(y0 - R + ly + rc) * PX + (x0 - R + lx + rc);
    int c1, n0, n1;
    decode_word(L.word[s], &c1, &n0, &n1);
    const unsigned t = window_type(c1 >= 0, c1, n0, n1);
    tmin = min(tmin, t);
    tmax = max(tmax, t);
  }
  tmin = __reduce_min_sync(0xffffffffu, tmin);
  tmax = __reduce_max_sync(0xffffffffu, tmax);
  if ((tid & 31) == 0) {
    red_tmin[tid >> 5] = tmin;
    red_tmax[tid >> 5] = tmax;
  }
  __syncthreads();
  tmin = red_tmin[0];
  tmax = red_tmax[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) {
    tmin = min(tmin, red_tmin[w]);
    tmax = max(tmax, red_tmax[w]);
  }
  int uni_sel = -1;
  {
    const int c1 = (int)((tmin >> 16) & 0xff);
    const int nx = (int)((tmin >> 8) & 0xff) - 128;
    const int ny = (int)(tmin & 0xff) - 128;
    if (tmin == tmax && tmin != 0u && c1 <= 2 && c1 + 2 <= R && nx >= -1 &&
        nx <= 0 && ny >= -1 && ny <= 0)
      uni_sel = c1 * 4 + (nx + 1) * 2 + (ny + 1);
  }

  const int dx = x0 + (tid % S::TX), dy = y0 + tid / S::TX;
  const bool valid = dx < a.nx && dy < a.ny;
  T tot[4] = {T(0), T(0), T(0), T(0)};
  T comp[4] = {T(0), T(0), T(0), T(0)};
  if (valid) {
    const long long s0 = (long long)(dy + rc) * PX + (dx + rc);
    switch (uni_sel) {
      case 0: uniform_gather<T, KAHAN, 0, -1, -1>(L, s0, PX, R, tot, comp); break;
      case 1: uniform_gather<T, KAHAN, 0, -1, 0>(L, s0, PX, R, tot, comp); break;
      case 2: uniform_gather<T, KAHAN, 0, 0, -1>(L, s0, PX, R, tot, comp); break;
      case 3: uniform_gather<T, KAHAN, 0, 0, 0>(L, s0, PX, R, tot, comp); break;
      case 4: uniform_gather<T, KAHAN, 1, -1, -1>(L, s0, PX, R, tot, comp); break;
      case 5: uniform_gather<T, KAHAN, 1, -1, 0>(L, s0, PX, R, tot, comp); break;
      case 6: uniform_gather<T, KAHAN, 1, 0, -1>(L, s0, PX, R, tot, comp); break;
      case 7: uniform_gather<T, KAHAN, 1, 0, 0>(L, s0, PX, R, tot, comp); break;
      case 8: uniform_gather<T, KAHAN, 2, -1, -1>(L, s0, PX, R, tot, comp); break;
      case 9: uniform_gather<T, KAHAN, 2, -1, 0>(L, s0, PX, R, tot, comp); break;
      case 10: uniform_gather<T, KAHAN, 2, 0, -1>(L, s0, PX, R, tot, comp); break;
      case 11: uniform_gather<T, KAHAN, 2, 0, 0>(L, s0, PX, R, tot, comp); break;
      default: scan_gather_rec<T, KAHAN>(L, s0, PX, R, tot, comp); break;
    }
  }
  step_finish<T, 2, NT>(a, valid, dx, dy, tot);
}

}  // namespace lbm
