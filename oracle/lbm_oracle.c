/*
 * Plain FP64 CPU oracle of the tau = 1 semi-discrete lattice Boltzmann step
 * (Komeili, Mirzaei, Shabouei, "Performance of 1-D and 2-D Lattice Boltzmann
 * (LB) in Solution of the Shock Tube Problem"), and, at the end of the file,
 * of the step with a general relaxation time tau (eqs 4-5) on a per-packet
 * state.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, constant or helper with the CUDA library.
 *
 * Everything is in lattice units: dx = dt = 1 in the lattice, so the flow
 * velocity of a node is V = u*lambda (lambda = dt/dx) and energies per unit
 * mass scale with lambda^2.  Conversion from/to physical units lives in
 * oracle.py.
 *
 * The step follows Section V.A: every node turns its moments into packets,
 * the packets migrate, and each node's new moments are the sum over all
 * packets that land on it.  Written out per destination node d (ascending
 * linear index, y-major, x fastest):
 *   for every source node s within the migration reach R of d, in ascending
 *   coordinate order (y-major, x fastest), including the "additional points"
 *   beyond the domain edge that Section V.B adds:
 *     equilibrium of s (Section III.B):
 *       V = m/rho, E = rhoE/rho, e = E - |V|^2/2            (eq 13, eq 15 text)
 *       rho' = rho - b0*d0,  Q = D*(gamma-1)*rho*e
 *       c1 = int(sqrt(Q/rho')), c2 = c1 + 1                   (eq 26)
 *       d1 = (c2^2 rho' - Q) / (b1 (c2^2 - c1^2))            (eq 24)
 *       d2 = (Q - c1^2 rho') / (b1 (c2^2 - c1^2))            (eq 25)
 *       phi = (1 - D/2 (gamma-1)) e                           (eq 15)
 *     packets (eqs 11-14, 21, 31-33): packet j of level v carries
 *       mass d_v, momentum d_v (V + c'_jv), energy d_v (|V + c'_jv|^2/2 + phi)
 *     split (eq 23, eq 28 for 1-D, eq 29 for 2-D): the end point s + V + c'
 *       lies between lattice nodes s + n + c' + k, n = floor(V); node k gets
 *       the linear (1-D) / bilinear (2-D) weight alpha_k;
 *     for every packet in table order, every corner k in order (0,0), (1,0),
 *     (0,1), (1,1): if s + n + c' + k == d, the arrival is alpha_k * packet
 *                                                       (eqs 6, 10, 22).
 * Summation order (the paper does not fix one): arrivals from one source row
 * are summed left to right (ascending x, then packet, then corner) into a row
 * sum; the two row sums at distance j below and above d are added to each
 * other, and these pair sums are added to d's total for j = 0, 1, ..., R.
 * The order is the same relative to every destination and symmetric under
 * y -> -y, so a uniform state stays uniform bit for bit, and data that vary
 * along x only stay so (their y-momentum arrivals cancel exactly) even
 * between reflecting walls.  This matters because the square-lattice step
 * amplifies some perturbations of a uniform state.
 *
 * Velocity sets (Section IV):
 *   1-D: c' in {0, +c1, -c1, +c2, -c2} with masses d0, d1, d1, d2, d2;
 *        b0 = 1, b1 = b2 = 2, d0 = theta*rho.
 *   2-D square lattice: c' in {+c1 ex, -c1 ex, +c1 ey, -c1 ey,
 *                              +c2 ex, -c2 ex, +c2 ey, -c2 ey}
 *        with masses d1 (first four) and d2; d0 = 0, b1 = b2 = 4.
 *
 * Boundaries (Section V.B): every source coordinate outside the domain is an
 * additional point whose state is taken, per axis, from
 *   transmissive : the nearest interior node (zero gradient);
 *   periodic     : the node at the coordinate modulo the axis length;
 *   reflecting   : the node at the mirror image about the wall half a cell
 *                  beyond the last node (repeated mirroring, period 2n), with
 *                  the momentum component normal to that wall negated.
 * Packets landing outside the domain are not gathered; what re-enters through
 * a periodic or reflecting edge is carried by the additional points.  For a
 * reflecting wall this equals mirroring each escaping packet back with its
 * normal momentum negated (the exact tracer in the tests does it that way).
 *
 * Readings where the text is silent or garbled are listed in the design
 * notes; the ones that shape this file: d0 = theta*rho; zeta uses the cross
 * term 2 c'.V; e < 0 from round-off is clamped to 0; nodes with rho <= 0 emit
 * nothing; additional points extend as far as the migration reach R.
 *
 * Build with -ffp-contract=off so that every product and sum rounds on its
 * own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORA_TRANSMISSIVE = 0, ORA_REFLECTING = 1, ORA_PERIODIC = 2 };

enum {
  ORA_OK = 0,
  ORA_EINVAL = 1,
  ORA_ESTATE = 4   /* rho < 0 or non-finite moment met */
};

typedef struct {
  int32_t dim;      /* 1 or 2 */
  int32_t bc_x, bc_y;
  int32_t pad_;
  int64_t nx, ny;   /* ny == 1 in 1-D */
  double gamma;
  double theta;     /* d0 = theta*rho in 1-D; unused in 2-D (d0 = 0) */
} ora_params;

/* One node's equilibrium (Section III.B). */
typedef struct {
  int emits;        /* 0 when rho <= 0 */
  int eclamp;       /* 1 when e < 0 was clamped to 0 */
  double V[2];      /* lattice flow velocity */
  double e;         /* internal energy per unit mass */
  int64_t c1, c2;   /* eq 26 */
  double dlev[3];   /* d0, d1, d2 */
  double phi;       /* eq 15 */
  int64_t n[2];     /* floor(V): lattice part of the flow displacement */
  double f[2];      /* V - n: fractional part, drives the split */
} ora_eq;

static int ora_equilibrium(const ora_params* P, double rho, double mx,
                           double my, double rhoE, ora_eq* q) {
  const double D = (double)P->dim;
  const double b0 = 1.0;
  const double b1 = (P->dim == 1) ? 2.0 : 4.0;
  memset(q, 0, sizeof(*q));
  if (!isfinite(rho) || !isfinite(mx) || !isfinite(my) || !isfinite(rhoE))
    return ORA_ESTATE;
  if (rho < 0.0) return ORA_ESTATE;
  if (rho == 0.0) return ORA_OK;  /* empty node: emits nothing */
  q->emits = 1;

  /* flow velocity and internal energy (eq 13; e = E - v^2/2 below eq 15) */
  q->V[0] = mx / rho;
  q->V[1] = (P->dim == 2) ? my / rho : 0.0;
  double E = rhoE / rho;
  double e = E - 0.5 * (q->V[0] * q->V[0] + q->V[1] * q->V[1]);
  if (e < 0.0) {
    e = 0.0;
    q->eclamp = 1;
  }
  q->e = e;

  /* level densities: d0 is a fixed share of rho in 1-D, zero on the square
     lattice (Section IV.B) */
  double d0 = (P->dim == 1) ? P->theta * rho : 0.0;
  double rho_p = rho - b0 * d0;
  double kq = D * (P->gamma - 1.0);
  double Q = kq * rho * e;            /* D (gamma-1) rho e */

  /* eq 26: c1 = int(sqrt(D (gamma-1) e rho / (rho - b0 d0))), fixed up so that
     c1^2 <= X < (c1+1)^2 holds exactly for the rounded X */
  double X = Q / rho_p;
  if (!isfinite(X) || X < 0.0) return ORA_ESTATE;
  int64_t c1 = (int64_t)floor(sqrt(X));
  while ((double)((c1 + 1) * (c1 + 1)) <= X) c1++;
  while (c1 > 0 && (double)(c1 * c1) > X) c1--;
  int64_t c2 = c1 + 1;
  q->c1 = c1;
  q->c2 = c2;

  double c1sq = (double)(c1 * c1);
  double c2sq = (double)(c2 * c2);
  double den = b1 * (c2sq - c1sq);
  q->dlev[0] = d0;
  q->dlev[1] = (c2sq * rho_p - Q) / den;   /* eq 24 */
  q->dlev[2] = (Q - c1sq * rho_p) / den;   /* eq 25 */

  double kphi = 1.0 - 0.5 * D * (P->gamma - 1.0);
  q->phi = kphi * e;                        /* eq 15 */

  for (int a = 0; a < 2; ++a) {
    double fl = floor(q->V[a]);
    q->n[a] = (int64_t)fl;
    q->f[a] = q->V[a] - fl;
  }
  return ORA_OK;
}

/* Migration reach of one node: the largest |lattice offset| any of its
   landings can have along one axis: floor(|V_a|) + 1 + c2. */
static int64_t ora_node_reach(const ora_params* P, const ora_eq* q) {
  if (!q->emits) return 0;
  int64_t r = 0;
  for (int a = 0; a < P->dim; ++a) {
    int64_t ra = (int64_t)floor(fabs(q->V[a])) + 1 + q->c2;
    if (ra > r) r = ra;
  }
  return r;
}

/* Packet table of one node: lattice offset c' and level v. */
typedef struct {
  int64_t cx, cy;
  int lev;
} ora_packet;

static int ora_packets(const ora_params* P, const ora_eq* q, ora_packet* pk) {
  if (P->dim == 1) {
    ora_packet t[5] = {{0, 0, 0},
                       {q->c1, 0, 1},
                       {-q->c1, 0, 1},
                       {q->c2, 0, 2},
                       {-q->c2, 0, 2}};
    memcpy(pk, t, sizeof(t));
    return 5;
  }
  ora_packet t[8] = {{q->c1, 0, 1},  {-q->c1, 0, 1}, {0, q->c1, 1},
                     {0, -q->c1, 1}, {q->c2, 0, 2},  {-q->c2, 0, 2},
                     {0, q->c2, 2},  {0, -q->c2, 2}};
  memcpy(pk, t, sizeof(t));
  return 8;
}

/* Interior node that supplies the state of source coordinate L on one axis,
   and the sign its momentum component along that axis takes there. */
static int64_t ora_virtual_axis(int bc, int64_t n, int64_t L, double* flip) {
  *flip = 1.0;
  if (L >= 0 && L < n) return L;
  if (bc == ORA_TRANSMISSIVE) return L < 0 ? 0 : n - 1;
  if (bc == ORA_PERIODIC) {
    int64_t w = L % n;
    return w < 0 ? w + n : w;
  }
  /* reflecting: mirror images about -1/2 and n - 1/2, period 2n */
  int64_t w = L % (2 * n);
  if (w < 0) w += 2 * n;
  if (w >= n) {
    *flip = -1.0;
    return 2 * n - 1 - w;
  }
  return w;
}

/* Current migration reach: max over interior nodes. */
int ora_reach(const ora_params* P, const double* rho, const double* mx,
              const double* my, const double* rhoE, int64_t* reach_out) {
  int64_t R = 0;
  int64_t N = P->nx * P->ny;
  for (int64_t i = 0; i < N; ++i) {
    ora_eq q;
    int st = ora_equilibrium(P, rho[i], mx[i], P->dim == 2 ? my[i] : 0.0,
                             rhoE[i], &q);
    if (st != ORA_OK) return st;
    int64_t r = ora_node_reach(P, &q);
    if (r > R) R = r;
  }
  *reach_out = R;
  return ORA_OK;
}

static int ora_check_params(const ora_params* P) {
  if (P->dim != 1 && P->dim != 2) return ORA_EINVAL;
  if (P->nx < 1 || P->ny < 1) return ORA_EINVAL;
  if (P->dim == 1 && P->ny != 1) return ORA_EINVAL;
  if (!(P->gamma > 1.0)) return ORA_EINVAL;
  return ORA_OK;
}

/* Sum of the arrivals at destination (dx, dy) from the sources of row sy
   within reach, ascending x, packets in table order, corners in order.
   out = {rho, m_x, m_y, rhoE}. */
static void ora_row_arrivals(const ora_params* P, const ora_eq* eq, int64_t wx,
                             int64_t R, int64_t Ry, int64_t dx, int64_t dy,
                             int64_t sy, double out[4]) {
  const int dim = P->dim;
  double r = 0.0, x = 0.0, y = 0.0, e = 0.0;
  ora_packet pk[8];
  for (int64_t sx = dx - R; sx <= dx + R; ++sx) {
    const ora_eq* q = &eq[(sy + Ry) * wx + (sx + R)];
    if (!q->emits) continue;
    /* split weights alpha_k (eq 28 / eq 29) */
    double wxk[2] = {1.0 - q->f[0], q->f[0]};
    double wyk[2] = {1.0 - q->f[1], q->f[1]};
    int nk = (dim == 1) ? 2 : 4;
    int np = ora_packets(P, q, pk);
    for (int p = 0; p < np; ++p) {
      double d = q->dlev[pk[p].lev];
      double cbx = q->V[0] + (double)pk[p].cx; /* eq 12: V + c' */
      double cby = q->V[1] + (double)pk[p].cy;
      double Pm = d;                                            /* eq 31 */
      double Px = d * cbx;                                      /* eq 32 */
      double Py = d * cby;
      double PE = d * (0.5 * (cbx * cbx + cby * cby) + q->phi); /* eq 33 */
      for (int k = 0; k < nk; ++k) {
        int64_t kx = k & 1, ky = k >> 1;
        if (sx + q->n[0] + pk[p].cx + kx != dx) continue;
        if (dim == 2 && sy + q->n[1] + pk[p].cy + ky != dy) continue;
        double a = (dim == 1) ? wxk[kx] : wxk[kx] * wyk[ky];
        r = r + a * Pm;
        x = x + a * Px;
        y = y + a * Py;
        e = e + a * PE;
      }
    }
  }
  out[0] = r;
  out[1] = x;
  out[2] = y;
  out[3] = e;
}

/*
 * One tau = 1 step (eq 10): each destination's new moments are the sum of
 * the migrated equilibrium packets that land on it.  Arrays hold nx*ny
 * nodes, x fastest; my may be NULL in 1-D.  eclamp_out (nullable) receives
 * the number of interior nodes whose e < 0 was clamped, reach_out (nullable)
 * the reach R that bounds the source window.
 */
int ora_step(const ora_params* P, const double* rho, const double* mx,
             const double* my, const double* rhoE, double* rho_o,
             double* mx_o, double* my_o, double* rhoE_o, int64_t* eclamp_out,
             int64_t* reach_out) {
  int st = ora_check_params(P);
  if (st != ORA_OK) return st;
  const int dim = P->dim;
  const int64_t nx = P->nx, ny = P->ny, N = nx * ny;
  int64_t R = 0;
  st = ora_reach(P, rho, mx, my, rhoE, &R);
  if (st != ORA_OK) return st;
  if (reach_out) *reach_out = R;

  /* equilibrium of every source coordinate within R of the domain, once */
  const int64_t Ry = (dim == 2) ? R : 0;
  const int64_t wx = nx + 2 * R, wy = ny + 2 * Ry;
  ora_eq* eq = (ora_eq*)malloc(sizeof(ora_eq) * (size_t)(wx * wy));
  if (!eq) return ORA_EINVAL;
  int64_t eclamps = 0;
  for (int64_t sy = -Ry; sy < ny + Ry; ++sy) {
    for (int64_t sx = -R; sx < nx + R; ++sx) {
      double fx, fy = 1.0;
      int64_t gx = ora_virtual_axis(P->bc_x, nx, sx, &fx);
      int64_t gy = (dim == 2) ? ora_virtual_axis(P->bc_y, ny, sy, &fy) : 0;
      int64_t g = gy * nx + gx;
      ora_eq* q = &eq[(sy + Ry) * wx + (sx + R)];
      st = ora_equilibrium(P, rho[g], fx * mx[g], dim == 2 ? fy * my[g] : 0.0,
                           rhoE[g], q);
      if (st != ORA_OK) {
        free(eq);
        return st;
      }
      if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) eclamps += q->eclamp;
    }
  }

  for (int64_t dy = 0; dy < ny; ++dy) {
    for (int64_t dx = 0; dx < nx; ++dx) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int64_t j = 0; j <= Ry; ++j) {
        double lo[4], hi[4];
        ora_row_arrivals(P, eq, wx, R, Ry, dx, dy, dy - j, lo);
        double pair[4];
        if (j == 0) {
          for (int f = 0; f < 4; ++f) pair[f] = lo[f];
        } else {
          ora_row_arrivals(P, eq, wx, R, Ry, dx, dy, dy + j, hi);
          for (int f = 0; f < 4; ++f) pair[f] = lo[f] + hi[f];
        }
        for (int f = 0; f < 4; ++f) acc[f] = acc[f] + pair[f];
      }
      int64_t t = dy * nx + dx;
      rho_o[t] = acc[0];
      mx_o[t] = acc[1];
      if (dim == 2) my_o[t] = acc[2];
      rhoE_o[t] = acc[3];
    }
  }
  free(eq);
  if (eclamp_out) *eclamp_out = eclamps;
  (void)N;
  return ORA_OK;
}

/* nsteps steps in place (ping-pong through scratch the oracle allocates). */
int ora_run(const ora_params* P, double* rho, double* mx, double* my,
            double* rhoE, int64_t nsteps, int64_t* eclamp_total) {
  int64_t N = P->nx * P->ny;
  double* buf = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  if (!buf) return ORA_EINVAL;
  double *r2 = buf, *x2 = buf + N, *y2 = buf + 2 * N, *e2 = buf + 3 * N;
  int64_t total = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t ec = 0;
    int st = ora_step(P, rho, mx, my, rhoE, r2, x2, P->dim == 2 ? y2 : NULL,
                      e2, &ec, NULL);
    if (st != ORA_OK) {
      free(buf);
      return st;
    }
    total += ec;
    memcpy(rho, r2, sizeof(double) * (size_t)N);
    memcpy(mx, x2, sizeof(double) * (size_t)N);
    if (P->dim == 2) memcpy(my, y2, sizeof(double) * (size_t)N);
    memcpy(rhoE, e2, sizeof(double) * (size_t)N);
  }
  free(buf);
  if (eclamp_total) *eclamp_total = total;
  return ORA_OK;
}

/* Equilibrium of one state, exposed for the closed-form tests:
   out = {c1, c2, d0, d1, d2, phi, e, n_x, f_x, n_y, f_y}. */
int ora_equilibrium_probe(const ora_params* P, double rho, double mx,
                          double my, double rhoE, double* out) {
  ora_eq q;
  int st = ora_equilibrium(P, rho, mx, my, rhoE, &q);
  if (st != ORA_OK) return st;
  out[0] = (double)q.c1;
  out[1] = (double)q.c2;
  out[2] = q.dlev[0];
  out[3] = q.dlev[1];
  out[4] = q.dlev[2];
  out[5] = q.phi;
  out[6] = q.e;
  out[7] = (double)q.n[0];
  out[8] = q.f[0];
  out[9] = (double)q.n[1];
  out[10] = q.f[1];
  return ORA_OK;
}

/* The packets of one state, for the moment and symmetry tests:
   rows of {c'_x, c'_y, mass, mom_x, mom_y, energy}; returns the count. */
int ora_packets_probe(const ora_params* P, double rho, double mx, double my,
                      double rhoE, double* out) {
  ora_eq q;
  if (ora_equilibrium(P, rho, mx, my, rhoE, &q) != ORA_OK || !q.emits)
    return 0;
  ora_packet pk[8];
  int np = ora_packets(P, &q, pk);
  for (int p = 0; p < np; ++p) {
    double d = q.dlev[pk[p].lev];
    double cbx = q.V[0] + (double)pk[p].cx;
    double cby = q.V[1] + (double)pk[p].cy;
    out[6 * p + 0] = (double)pk[p].cx;
    out[6 * p + 1] = (double)pk[p].cy;
    out[6 * p + 2] = d;
    out[6 * p + 3] = d * cbx;
    out[6 * p + 4] = d * cby;
    out[6 * p + 5] = d * (0.5 * (cbx * cbx + cby * cby) + q.phi);
  }
  return np;
}

/* ==========================================================================
 * General relaxation time tau (eqs 4-5) with per-packet storage.
 *
 * With tau != 1 the distribution no longer collapses to its equilibrium, so
 * a node's state is the set of packets it holds: one slot j per entry of
 * the velocity set (1-D: 5 slots, 2-D: 8 slots, in the table order of
 * ora_packets), each slot carrying mass, momentum and energy (the integrand
 * eta f of eq 6 summed over one migrating velocity).  Fields per slot:
 * NF = dim + 2, i.e. (mass, m_x, energy) in 1-D and (mass, m_x, m_y, energy)
 * in 2-D.  Array layout: f[(j * NF + c) * N + i], node i x fastest.
 *
 * One step, per node:
 *   Y = sum_j f_j (eq 6), slots in table order;
 *   f_eq_j from Y exactly as in the tau = 1 step (Section III.B);
 *   collision (eqs 4-5): f*_j = f_j - (f_j - f_eq_j)/tau, evaluated as the
 *     blend (1 - 1/tau) f_j + (1/tau) f_eq_j, which at tau = 1 is f_eq_j
 *     exactly (eq 10);
 *   migration: slot j moves with the node's migrating velocity V + c'_j of
 *     the same table entry (c' from the node's own c1, eq 26) and splits over
 *     the nodes s + n + c'_j + k with the weights of eqs 28-29;
 *   every destination's slot j is the sum of the slot-j arrivals.
 * Per destination and slot the arrivals are added in ascending source order
 * (y-major, x fastest), then corner order.  New slot contents are a
 * function of the arrivals alone, so conservation of sum_j f_j over the
 * domain follows from sum_j f*_j = Y.
 *
 * Additional points (Section V.B) hold the supplying node's packets:
 * transmissive and periodic copy them; a reflecting wall mirrors them: the
 * slot whose c' points the other way along the wall normal, with the normal
 * momentum negated.  The additional point's moments are the supplying
 * node's with that component negated (not re-summed in mirrored order), so
 * its packets and equilibrium are the exact mirror images.
 * ========================================================================== */

static int ora_slots(const ora_params* P) { return P->dim == 1 ? 5 : 8; }

/* Slot of the mirrored packet across a wall normal to `axis`. */
static int ora_mirror_slot(int dim, int axis, int j) {
  if (dim == 1) {
    if (j == 0) return 0;
    return (j % 2 == 1) ? j + 1 : j - 1; /* +c1 <-> -c1, +c2 <-> -c2 */
  }
  const int dir = j & 3; /* 0: +x, 1: -x, 2: +y, 3: -y */
  if (axis == 0 && dir < 2) return j ^ 1;
  if (axis == 1 && dir >= 2) return j ^ 1;
  return j;
}

/* Moments of node i from its slots (eq 6), slots in table order. */
static void ora_bgk_node_moments(const ora_params* P, const double* f,
                                 int64_t N, int64_t i, double Y[4]) {
  const int NF = P->dim + 2, NP = ora_slots(P);
  double r = 0.0, x = 0.0, y = 0.0, e = 0.0;
  for (int j = 0; j < NP; ++j) {
    const double* s = f + (int64_t)j * NF * N;
    r = r + s[0 * N + i];
    x = x + s[1 * N + i];
    if (P->dim == 2) y = y + s[2 * N + i];
    e = e + s[(NF - 1) * N + i];
  }
  Y[0] = r;
  Y[1] = x;
  Y[2] = y;
  Y[3] = e;
}

/* Equilibrium packet j of q as (mass, m_x, m_y, energy); zero if q emits
   nothing. */
static void ora_eq_packet(const ora_params* P, const ora_eq* q, int j,
                          double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  if (!q->emits) return;
  ora_packet pk[8];
  ora_packets(P, q, pk);
  const double d = q->dlev[pk[j].lev];
  const double cbx = q->V[0] + (double)pk[j].cx; /* eq 12 */
  const double cby = q->V[1] + (double)pk[j].cy;
  out[0] = d;                                            /* eq 31 */
  out[1] = d * cbx;                                      /* eq 32 */
  out[2] = (P->dim == 2) ? d * cby : 0.0;
  out[3] = d * (0.5 * (cbx * cbx + cby * cby) + q->phi); /* eq 33 */
}

/* f = f_eq of the given moments at every node (the state a tau = 1 step
   would migrate).  my may be NULL in 1-D. */
int ora_bgk_equilibrium(const ora_params* P, const double* rho,
                        const double* mx, const double* my,
                        const double* rhoE, double* f) {
  int st = ora_check_params(P);
  if (st != ORA_OK) return st;
  const int NF = P->dim + 2, NP = ora_slots(P);
  const int64_t N = P->nx * P->ny;
  for (int64_t i = 0; i < N; ++i) {
    ora_eq q;
    st = ora_equilibrium(P, rho[i], mx[i], P->dim == 2 ? my[i] : 0.0,
                         rhoE[i], &q);
    if (st != ORA_OK) return st;
    for (int j = 0; j < NP; ++j) {
      double pj[4];
      ora_eq_packet(P, &q, j, pj);
      double* s = f + (int64_t)j * NF * N;
      s[0 * N + i] = pj[0];
      s[1 * N + i] = pj[1];
      if (P->dim == 2) s[2 * N + i] = pj[2];
      s[(NF - 1) * N + i] = pj[3];
    }
  }
  return ORA_OK;
}

/* Moments of every node from its slots (eq 6).  my may be NULL in 1-D. */
int ora_bgk_moments(const ora_params* P, const double* f, double* rho,
                    double* mx, double* my, double* rhoE) {
  int st = ora_check_params(P);
  if (st != ORA_OK) return st;
  const int64_t N = P->nx * P->ny;
  for (int64_t i = 0; i < N; ++i) {
    double Y[4];
    ora_bgk_node_moments(P, f, N, i, Y);
    rho[i] = Y[0];
    mx[i] = Y[1];
    if (P->dim == 2) my[i] = Y[2];
    rhoE[i] = Y[3];
  }
  return ORA_OK;
}

/* One source of the tau != 1 step: its equilibrium and its post-collision
   packets (mass, m_x, m_y, energy per slot). */
typedef struct {
  ora_eq q;
  double fs[8][4];
} ora_bgk_src;

/*
 * One step with relaxation time tau (eqs 4-5) of the per-packet state f
 * (layout above) into f_out.  eclamp_out (nullable): interior nodes whose
 * e < 0 was clamped; reach_out (nullable): the reach R of the source window.
 */
int ora_bgk_step(const ora_params* P, double tau, const double* f,
                 double* f_out, int64_t* eclamp_out, int64_t* reach_out) {
  int st = ora_check_params(P);
  if (st != ORA_OK) return st;
  if (!(tau > 0.5) || !isfinite(tau)) return ORA_EINVAL;
  const int dim = P->dim, NF = dim + 2, NP = ora_slots(P);
  const int64_t nx = P->nx, ny = P->ny, N = nx * ny;
  const double omega = 1.0 / tau;
  const double keep = 1.0 - omega;

  /* moments and equilibrium of every node, and the reach */
  double* Y = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  ora_eq* nq = (ora_eq*)malloc(sizeof(ora_eq) * (size_t)N);
  if (!Y || !nq) {
    free(Y);
    free(nq);
    return ORA_EINVAL;
  }
  int64_t R = 0, eclamps = 0;
  for (int64_t i = 0; i < N; ++i) {
    ora_bgk_node_moments(P, f, N, i, Y + 4 * i);
    st = ora_equilibrium(P, Y[4 * i], Y[4 * i + 1], Y[4 * i + 2],
                         Y[4 * i + 3], &nq[i]);
    if (st != ORA_OK) {
      free(Y);
      free(nq);
      return st;
    }
    eclamps += nq[i].eclamp;
    const int64_t r = ora_node_reach(P, &nq[i]);
    if (r > R) R = r;
  }
  if (reach_out) *reach_out = R;

  /* every source coordinate within R of the domain: collision (eqs 4-5) */
  const int64_t Ry = (dim == 2) ? R : 0;
  const int64_t wx = nx + 2 * R, wy = ny + 2 * Ry;
  ora_bgk_src* src =
      (ora_bgk_src*)malloc(sizeof(ora_bgk_src) * (size_t)(wx * wy));
  if (!src) {
    free(Y);
    free(nq);
    return ORA_EINVAL;
  }
  for (int64_t sy = -Ry; sy < ny + Ry; ++sy) {
    for (int64_t sx = -R; sx < nx + R; ++sx) {
      double flx, fly = 1.0;
      const int64_t gx = ora_virtual_axis(P->bc_x, nx, sx, &flx);
      const int64_t gy = (dim == 2) ? ora_virtual_axis(P->bc_y, ny, sy, &fly)
                                    : 0;
      const int64_t g = gy * nx + gx;
      ora_bgk_src* S = &src[(sy + Ry) * wx + (sx + R)];
      /* the additional point's moments: the node's, normal momentum
         negated across a reflecting wall */
      const double* Yg = Y + 4 * g;
      if (flx == 1.0 && fly == 1.0) {
        S->q = nq[g];
      } else {
        st = ora_equilibrium(P, Yg[0], flx * Yg[1], fly * Yg[2], Yg[3],
                             &S->q);
        if (st != ORA_OK) {
          free(Y);
          free(nq);
          free(src);
          return st;
        }
      }
      for (int j = 0; j < NP; ++j) {
        /* the node's slot that this source's slot j mirrors */
        int jg = j;
        if (flx < 0.0) jg = ora_mirror_slot(dim, 0, jg);
        if (fly < 0.0) jg = ora_mirror_slot(dim, 1, jg);
        const double* s = f + (int64_t)jg * NF * N;
        double fj[4];
        fj[0] = s[0 * N + g];
        fj[1] = flx * s[1 * N + g];
        fj[2] = (dim == 2) ? fly * s[2 * N + g] : 0.0;
        fj[3] = s[(NF - 1) * N + g];
        double feq[4];
        ora_eq_packet(P, &S->q, j, feq);
        for (int c = 0; c < 4; ++c)
          S->fs[j][c] = keep * fj[c] + omega * feq[c];
      }
    }
  }

  /* migration: each destination's slot j sums its slot-j arrivals,
     sources ascending (y-major, x fastest), then corners */
  const int nk = (dim == 1) ? 2 : 4;
  for (int64_t dy = 0; dy < ny; ++dy) {
    for (int64_t dx = 0; dx < nx; ++dx) {
      const int64_t t = dy * nx + dx;
      for (int j = 0; j < NP; ++j) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t sy = dy - Ry; sy <= dy + Ry; ++sy) {
          for (int64_t sx = dx - R; sx <= dx + R; ++sx) {
            const ora_bgk_src* S = &src[(sy + Ry) * wx + (sx + R)];
            const ora_eq* q = &S->q;
            if (!q->emits) continue;
            ora_packet pk[8];
            ora_packets(P, q, pk);
            const double wxk[2] = {1.0 - q->f[0], q->f[0]};
            const double wyk[2] = {1.0 - q->f[1], q->f[1]};
            for (int k = 0; k < nk; ++k) {
              const int64_t kx = k & 1, ky = k >> 1;
              if (sx + q->n[0] + pk[j].cx + kx != dx) continue;
              if (dim == 2 && sy + q->n[1] + pk[j].cy + ky != dy) continue;
              const double a = (dim == 1) ? wxk[kx] : wxk[kx] * wyk[ky];
              for (int c = 0; c < 4; ++c) acc[c] = acc[c] + a * S->fs[j][c];
            }
          }
        }
        double* o = f_out + (int64_t)j * NF * N;
        o[0 * N + t] = acc[0];
        o[1 * N + t] = acc[1];
        if (dim == 2) o[2 * N + t] = acc[2];
        o[(NF - 1) * N + t] = acc[3];
      }
    }
  }
  free(src);
  free(Y);
  free(nq);
  if (eclamp_out) *eclamp_out = eclamps;
  return ORA_OK;
}

/* nsteps tau != 1 steps of f in place. */
int ora_bgk_run(const ora_params* P, double tau, double* f, int64_t nsteps,
                int64_t* eclamp_total) {
  const int64_t N = P->nx * P->ny;
  const size_t bytes = sizeof(double) * (size_t)((P->dim + 2) *
                                                 ora_slots(P)) * (size_t)N;
  double* buf = (double*)malloc(bytes);
  if (!buf) return ORA_EINVAL;
  int64_t total = 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t ec = 0;
    const int st = ora_bgk_step(P, tau, f, buf, &ec, NULL);
    if (st != ORA_OK) {
      free(buf);
      return st;
    }
    total += ec;
    memcpy(f, buf, bytes);
  }
  free(buf);
  if (eclamp_total) *eclamp_total = total;
  return ORA_OK;
}
