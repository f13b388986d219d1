/*
 * lbm.h - C ABI of the GB300 tau = 1 semi-discrete lattice Boltzmann solver.
 *
 * The method (Komeili, Mirzaei, Shabouei, "Performance of 1-D and 2-D Lattice
 * Boltzmann (LB) in Solution of the Shock Tube Problem"): with relaxation time
 * tau = 1 the BGK update reduces to f(x + r dt, t + dt) = f_eq(x, t)
 * (Section III.A, eqs 9-10), so a node's state is its moments
 * Y = (rho, rho V, rho E) alone (eq 7).  One step expands every node's moments
 * into its equilibrium packets over the triple-level (1-D) or dual-level
 * square (2-D) velocity set (Section III.B, eqs 11-26; Section IV), migrates
 * each packet to x + (V + c') dt with linear (eq 28) or bilinear (eq 29)
 * splitting, and sums the arrivals into the new moments (eqs 6, 22; Section
 * V.A).  The shock-tube problem of Section V.C is the initial state.
 *
 * Conventions shared by every entry point:
 *  - Plain C types only.  Host arrays are caller-owned, hold n = nx*ny
 *    doubles with x fastest, and are not retained after the call returns.
 *  - All device memory is owned by the handle and allocated in lbm_create:
 *    two moment buffers (4 fields x n x 4 or 8 bytes each), a few scratch
 *    words and per-block partial totals; an F32 square-lattice handle with
 *    max_reach <= 6 adds 8 bytes per tile of its deposit kernel (a record
 *    of the tile's window at the last step, a starting guess only, and a
 *    queue slot; a tile holds about 2000 nodes); an F64 square-lattice
 *    handle holds one set of source records (248 bytes per node of the
 *    grid padded by max_reach on every side: each source's packets, level
 *    densities and corner weights), rewritten from the moments at the start
 *    of every step.
 *  - Work is issued on the stream given in lbm_config.stream (a
 *    cudaStream_t, or NULL for the default stream), in call order.
 *    lbm_step returns before the GPU finishes; lbm_moments, lbm_conservation,
 *    lbm_reach, lbm_diagnostics and lbm_synchronize wait for it.
 *  - Every call returns an lbm_status; nothing throws across the ABI.
 *    lbm_last_error gives a message for the last failure on a handle.
 *    LBM_EINVAL leaves the handle usable; after any other error the handle
 *    may only be destroyed.
 *  - A handle is not thread-safe; separate handles are independent.
 *  - Physical units at the ABI: positions in [x0, x1] along x, square cells
 *    dx = (x1 - x0)/nx, time step dt.  Internally the lattice velocity is
 *    V = u*lambda with lambda = dt/dx and energies per unit mass scale with
 *    lambda^2.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,   /* bad argument or configuration */
  LBM_ENOMEM = 2,   /* device or host allocation failed */
  LBM_ECUDA = 3,    /* a CUDA call failed (message in lbm_last_error) */
  LBM_ESTATE = 4,   /* a node reached rho < 0 or a non-finite moment */
  LBM_EREACH = 5,   /* migration reach exceeded the configured max_reach */
  LBM_ETIMEOUT = 6, /* a bounded device-side wait gave up */
  LBM_EBUDGET = 7   /* request does not fit the memory budget */
} lbm_status;

typedef enum { LBM_F32 = 0, LBM_F64 = 1 } lbm_precision;

/* Boundary rule per axis (Section V.B).  Beyond the edge a source node
   ("additional point") holds the state of: the nearest edge node
   (TRANSMISSIVE, zero gradient); the mirror image about the wall half a cell
   beyond the edge node, normal momentum negated (REFLECTING); the node one
   period away (PERIODIC).  Packets landing outside the domain are dropped. */
typedef enum {
  LBM_TRANSMISSIVE = 0,
  LBM_REFLECTING = 1,
  LBM_PERIODIC = 2
} lbm_bc;

typedef enum { LBM_PLANAR_X = 0, LBM_CIRCLE = 1 } lbm_geom;

typedef struct {
  int32_t dim;        /* 1 or 2 (Section IV.A / IV.B) */
  int32_t precision;  /* lbm_precision of the stored moments and the step */
  int32_t bc_x, bc_y; /* lbm_bc; bc_y ignored in 1-D */
  int64_t nx, ny;     /* nodes; ny must be 1 in 1-D */
  double x0, x1;      /* physical extent along x; dx = (x1 - x0)/nx */
  double y0;          /* lower edge along y (2-D); cells are square */
  double gamma;       /* ratio of specific heats, > 1 (eqs 15, 24-27) */
  double theta;       /* 1-D rest share d0 = theta*rho (Section III.B,
                         0.4..0.55); must be 0 in 2-D where d0 = 0 */
  double dt;          /* physical time step; lambda = dt/dx */
  int32_t max_reach;  /* largest migration reach R (lattice cells) a step
                         may meet; 0 picks the default (1-D 64, 2-D 6).
                         Shared memory per block grows with it (F64 2-D:
                         the padding of the source records instead).  A step
                         that meets a larger R leaves the state untouched
                         and reports LBM_EREACH at the next waiting call. */
  int32_t kahan;      /* F32 only: 1 = compensated (Kahan) summation of
                         the gathered arrivals, 0 = plain summation */
  int32_t cons_every; /* also sum total mass/momentum/energy in FP64 every
                         this many steps inside the step kernel (0 = never;
                         lbm_conservation computes them on request) */
  int32_t reserved_;
  void* stream;       /* cudaStream_t; NULL = legacy default stream */
} lbm_config;

/* Primitive state (physical units): density, velocity, pressure. */
typedef struct {
  double rho, u, v, p;
} lbm_prim;

/* ABI revision of this header. */
int32_t lbm_abi_version(void);

/* Validate cfg, allocate the handle and its device buffers.  *out is set
   only on LBM_OK.  Errors: LBM_EINVAL (cfg), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out);

/* Riemann initial state of Section V.C (Sod: left (1, 0, 1), right
   (0.125, 0, 0.1)).  Nodes sit at cell centres x_i = x0 + (i + 1/2) dx.
   geom = LBM_PLANAR_X: nodes with x < a0 take *inner, the rest *outer.
   geom = LBM_CIRCLE: nodes with (x - a0)^2 + (y - a1)^2 < radius^2 take
   *inner, the rest *outer.  Moments: m = rho u lambda,
   rhoE = p lambda^2/(gamma - 1) + rho |u lambda|^2 / 2.  Also sets the
   migration reach for the first step.  Stream-ordered, does not wait. */
lbm_status lbm_init_riemann(lbm_handle* h, const lbm_prim* inner,
                            const lbm_prim* outer, int32_t geom, double a0,
                            double a1, double radius);

/* Set every node from host primitive arrays (rho, u, v, p; v may be NULL in
   1-D), converted to moments on the device as in lbm_init_riemann.  Waits
   for the copy to finish before returning. */
lbm_status lbm_set_primitives(lbm_handle* h, const double* rho,
                              const double* u, const double* v,
                              const double* p, int64_t n);

/* Set every node from host conserved arrays in physical units (rho,
   rho*u, rho*v, rho*E with E = e + |u|^2/2); my may be NULL in 1-D.  With
   lbm_moments this is checkpoint / restart: the tau = 1 state is the moments
   alone (eq 10).  Waits for the copy to finish before returning. */
lbm_status lbm_set_moments(lbm_handle* h, const double* rho, const double* mx,
                           const double* my, const double* rhoE, int64_t n);

/* Advance nsteps tau = 1 steps (eq 10), one fused kernel launch each:
   equilibrium (eqs 13-15, 24-26), packets (eqs 11-14, 21), split (eqs 23,
   28, 29), migration and summation (eqs 6, 22), boundaries (Section V.B);
   the same launch reduces the next step's migration reach.  Returns after
   queueing the work (stream-ordered, does not wait).  Errors found on the
   device (LBM_ESTATE, LBM_EREACH) are reported by the next waiting call. */
lbm_status lbm_step(lbm_handle* h, int64_t nsteps);

/* Copy the current state to host arrays in physical units: rho, rho*u,
   rho*v (NULL allowed; ignored in 1-D), rho*E and, if p is not NULL, the
   pressure P = (gamma - 1) rho e (eq 27), recovered in FP64 on the device.
   Waits for all queued work. */
lbm_status lbm_moments(lbm_handle* h, double* rho, double* mx, double* my,
                       double* rhoE, double* p, int64_t n);

/* FP64 totals over all nodes, physical units, in a fixed reduction order:
   out[0] = sum rho, out[1] = sum rho*u, out[2] = sum rho*v, out[3] =
   sum rho*E.  Conserved exactly by the step on periodic and closed domains
   (eq 22 with eqs 16-18).  Waits for all queued work. */
lbm_status lbm_conservation(lbm_handle* h, double out[4]);

/* The totals the step kernel itself formed (cons_every > 0) at the last
   step that summed them, physical units, same order as lbm_conservation
   (or what a later lbm_conservation computed); zeros if nothing has summed
   them since the state was set.  The FP32
   kernels sum in compensated FP32 (pairs of floats carried through every
   partial) and convert to FP64 once per field; the FP64 kernels sum in
   FP64.  Waits for all queued work.  (The paper has no counterpart: this
   reads what a10 of the step produced, without another pass over the
   state.) */
lbm_status lbm_last_totals(lbm_handle* h, double out[4]);

/* Migration reach R the next step will use (lattice cells): the maximum over
   nodes of floor(|V_a|) + 1 + c2 (eq 26), computed conservatively.  Waits. */
lbm_status lbm_reach(lbm_handle* h, int32_t* reach);

/* Counters: steps taken since the last state set, number of nodes whose
   internal energy came out below zero from round-off and was clamped to 0,
   and the device error flags (bit 0: LBM_ESTATE, bit 1: LBM_EREACH).
   Any pointer may be NULL.  Waits. */
lbm_status lbm_diagnostics(lbm_handle* h, int64_t* steps, int64_t* eclamps,
                           uint32_t* flags);

/* Wait for queued work and report device-side errors. */
lbm_status lbm_synchronize(lbm_handle* h);

/* Lattice velocity scale lambda = dt/dx of a handle (0 for NULL). */
double lbm_lambda(const lbm_handle* h);

/* Message for the last failure on h (empty string if none; static text for
   h == NULL).  Owned by the handle. */
const char* lbm_last_error(const lbm_handle* h);

/* Free the handle and its device memory.  NULL-safe.  Waits for queued
   work first. */
void lbm_destroy(lbm_handle* h);

/* ---- batched 1-D tubes --------------------------------------------------
 *
 * Many independent 1-D shock tubes (Section V.C, each on [0, 1] with its own
 * node count, Riemann state, time step and step count) advanced together:
 * one persistent kernel launch per step covers every tube that still has
 * steps to take, and the launches are replayed from a captured CUDA graph.
 * Each tube's step is the same tau = 1 step as lbm_step on a 1-D handle
 * (eq 10; Section III.B; Section IV.A; Section V.B), so in FP64 a tube's
 * result is the result of running it alone.
 */
typedef struct lbm_batch lbm_batch;

typedef struct {
  int64_t n;       /* nodes; dx = 1/n */
  int64_t nsteps;  /* steps this tube takes */
  double dt;       /* time step; lambda = dt*n */
  double x_d;      /* diaphragm position in (0, 1) */
  lbm_prim left, right;  /* states for x < x_d and x >= x_d (v ignored) */
  int32_t bc;      /* lbm_bc at both ends */
  int32_t pad_;
} lbm_tube;

/* Create a batch: device buffers for all tubes, their initial states and
   first reach.  precision: lbm_precision; theta as lbm_config.theta; kahan
   (F32): compensated summation of each destination's arrivals.  Tubes keep
   the caller's indices in every other call.  Synchronous.  Creation also
   picks the tile width (nodes per work item: 128, 256 or 512) by timing a
   few steps of this batch with each and keeping the fastest, then resets
   every tube to its initial state; the width does not change any result. */
lbm_status lbm_batch_create(int32_t precision, double gamma, double theta,
                            int32_t kahan, const lbm_tube* tubes, int64_t count,
                            void* stream, lbm_batch** out);

/* Queue up to max_launches steps (negative: until every tube has taken its
   steps).  One persistent launch per step; stream-ordered, does not wait. */
lbm_status lbm_batch_run(lbm_batch* b, int64_t max_launches);

/* Wait; report launches executed and device flags (bit 0 LBM_ESTATE, bit 1
   LBM_EREACH).  Either pointer may be NULL. */
lbm_status lbm_batch_sync(lbm_batch* b, int64_t* steps_done, uint32_t* flags);

/* Physical rho, rho*u, rho*E and (if p != NULL) pressure of one tube after
   its last step (or its latest step if the batch has not finished).  n must
   be the tube's node count.  Waits. */
lbm_status lbm_batch_moments(lbm_batch* b, int64_t tube, double* rho,
                             double* mx, double* rhoE, double* p, int64_t n);

/* FP64 totals (rho, rho*u, rho*E; physical units) of every tube, 3 per tube
   in the caller's order; count = number of tubes.  Waits. */
lbm_status lbm_batch_totals(lbm_batch* b, double* out, int64_t count);

/* The tile width in use and the measured ms per step of the candidates
   128, 256, 512 (ms_per_step[3], -1 where not timed; either pointer may be
   NULL). */
lbm_status lbm_batch_tuning(const lbm_batch* b, int32_t* tile,
                            double* ms_per_step);

/* Use tile width `tile` (128, 256 or 512) instead of the tuned one.  Only
   before the first lbm_batch_run (LBM_EINVAL after); resets every tube to
   its initial state.  Synchronous. */
lbm_status lbm_batch_set_tile(lbm_batch* b, int32_t tile);

const char* lbm_batch_last_error(const lbm_batch* b);

/* Free a batch; NULL-safe; waits for queued work. */
void lbm_batch_destroy(lbm_batch* b);

/* ---- batched small 2-D grids -------------------------------------------
 *
 * Many independent square-lattice grids (Section IV.B; each with its own
 * size, boundaries, time step, initial state and step count) advanced
 * together in FP32: a lattice step is two launches for the whole batch --
 * the persistent deposit kernel over the tiles of every grid that still has
 * steps to take, and the finalize kernel (each grid's totals and reach) --
 * instead of two per grid.  Each grid's step is the step lbm_step takes on a handle of the
 * grid's configuration (same kernels and arithmetic), so every grid's
 * result equals that handle's bit for bit.
 */
typedef struct lbm_batch2d lbm_batch2d;

typedef struct {
  lbm_config cfg;        /* dim 2, precision LBM_F32, max_reach 0 (6) or
                            at most 6; cfg.stream is ignored */
  lbm_prim inner, outer; /* initial state, as lbm_init_riemann */
  int32_t geom;          /* lbm_geom */
  int32_t pad_;
  double a0, a1, radius; /* as lbm_init_riemann */
  int64_t nsteps;        /* steps this grid takes */
} lbm_grid2d;

/* Create a batch of count grids (device memory for each, initial states,
   first reach), all on `stream`.  LBM_EINVAL for a grid the deposit kernel
   does not take (1-D, FP64, a reach limit above 6), a negative step count,
   or grids that differ in cfg.kahan (one summation form per batch).  Grids
   keep the caller's indices.  Synchronous. */
lbm_status lbm_batch2d_create(const lbm_grid2d* grids, int32_t count,
                              void* stream, lbm_batch2d** out);

/* Queue up to max_steps lattice steps (negative: until every grid has
   taken its steps); grids past their step count are left as they are.
   Stream-ordered, does not wait. */
lbm_status lbm_batch2d_run(lbm_batch2d* b, int64_t max_steps);

/* Lattice steps queued so far (the batch's step counter). */
lbm_status lbm_batch2d_steps(const lbm_batch2d* b, int64_t* steps);

/* Physical moments of one grid after its last step (or its latest, if the
   batch has not reached it), as lbm_moments; errors the grid's steps met
   (LBM_ESTATE, LBM_EREACH) are reported here.  Waits. */
lbm_status lbm_batch2d_moments(lbm_batch2d* b, int32_t grid, double* rho,
                               double* mx, double* my, double* rhoE,
                               double* p, int64_t n);

const char* lbm_batch2d_last_error(const lbm_batch2d* b);

/* Free a batch; NULL-safe; waits for queued work. */
void lbm_batch2d_destroy(lbm_batch2d* b);

/* ---- tube pool for continuous batching ---------------------------------
 *
 * 1-D tubes (lbm_tube) join and leave between steps; each lbm_pool_step is
 * one launch that advances every tube still short of its step count by one
 * step.  Each tube keeps its own step counter, so a tube's result does not
 * depend on when it joined or what else is in the pool (same step as
 * lbm_step on a 1-D handle).  Node ranges come from one buffer of
 * capacity_nodes nodes per field and parity, allocated at creation.
 */
typedef struct lbm_pool lbm_pool;

lbm_status lbm_pool_create(int32_t precision, double gamma, double theta,
                           int32_t kahan, int64_t capacity_nodes,
                           int32_t max_slots, void* stream, lbm_pool** out);

/* Take a slot and a node range for the tube and initialise it (stream-
   ordered).  LBM_EBUDGET when no slot or contiguous range is free. */
lbm_status lbm_pool_add(lbm_pool* p, const lbm_tube* t, int32_t* slot);

/* One step of every tube that still has steps to take (one launch). */
lbm_status lbm_pool_step(lbm_pool* p);

/* nsteps successive lbm_pool_step calls in one call (stops early once no
   tube has steps left); stream-ordered, does not wait. */
lbm_status lbm_pool_run(lbm_pool* p, int64_t nsteps);

/* Steps taken and step count of a slot (host-side, does not wait). */
lbm_status lbm_pool_progress(lbm_pool* p, int32_t slot, int64_t* taken,
                             int64_t* nsteps);

/* Physical rho, rho*u, rho*E and pressure (nullable) of a slot's current
   state; n = the tube's node count.  Waits for the pool's stream. */
lbm_status lbm_pool_read(lbm_pool* p, int32_t slot, double* rho, double* mx,
                         double* rhoE, double* pr, int64_t n);

/* Release a slot and its node range. */
lbm_status lbm_pool_remove(lbm_pool* p, int32_t slot);

const char* lbm_pool_last_error(const lbm_pool* p);

void lbm_pool_destroy(lbm_pool* p);

/* ---- general relaxation time tau (eqs 4-5) ------------------------------
 *
 * With tau != 1 the collision f*_j = f_j - (f_j - f_eq_j)/tau (eqs 4-5)
 * keeps part of what arrived, so the state is per packet: every node holds
 * one slot per entry of its velocity set (Section IV; 1-D: 5 slots in the
 * order 0, +c1, -c1, +c2, -c2; 2-D: 8 slots +c1 x, -c1 x, +c1 y, -c1 y,
 * then the same with c2), each slot carrying NF = dim + 2 fields: mass,
 * momentum per axis, energy.  Per step and node: Y = sum_j f_j (eq 6), the
 * equilibrium of Y as in the tau = 1 step (Section III.B), the collision,
 * evaluated as (1 - 1/tau) f_j + (1/tau) f_eq_j (exactly eq 10 at tau = 1);
 * slot j then migrates with the node's V + c'_j (the same landings and
 * weights as at tau = 1, eqs 23, 28-29) into the same slot of the nodes it
 * lands on, whose slot j is the sum of its arrivals (sources in ascending
 * order, y-major, then corners).  Additional points (Section V.B) copy the
 * supplying node's slots, or mirror them across a reflecting wall (slot of
 * the opposite c' along the normal, normal momentum negated).  A node whose
 * slot masses sum to 0 emits nothing.
 *
 * Packet arrays at the ABI: NP * NF arrays of n doubles, array j * NF + c
 * for slot j and field c, nodes x fastest (NP * NF * n doubles in all),
 * physical units (momentum = lattice momentum / lambda, energy = lattice
 * energy / lambda^2).
 *
 * Step paths: on the square lattice with max_reach <= 4 one kernel launch
 * per step (each tile's window collided in shared memory, then gathered);
 * otherwise (1-D, or a larger reach limit) a collision pass into source
 * records and a gather pass, two launches.  Both give the same bits.
 * Device memory per handle: two packet sets (NP * NF * n elements each), a
 * moments buffer (4 fields), 5 n doubles of staging, scratch; the
 * two-launch path adds source records over the grid padded by max_reach
 * (8 bytes plus NP * NF + 4 (2-D) or NP * NF + 2 (1-D) elements per padded
 * node, rewritten every step).  Both precisions; kahan and cons_every are
 * ignored (the configuration is checked as by lbm_create; max_reach at
 * most 1024).  Conventions of lbm_create otherwise (stream order, errors,
 * not thread-safe). */
typedef struct lbm_bgk lbm_bgk;

/* Validate cfg and tau (tau > 0.5, finite) and allocate.  tau < 1
   over-relaxes: packets may then carry negative mass, and a state far from
   equilibrium next to a reflecting wall need not stay positive (reported as
   LBM_ESTATE).  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_bgk_create(const lbm_config* cfg, double tau, lbm_bgk** out);

/* Riemann initial state as lbm_init_riemann; the packets start at the
   equilibrium of the moments.  Stream-ordered, does not wait. */
lbm_status lbm_bgk_init_riemann(lbm_bgk* h, const lbm_prim* inner,
                                const lbm_prim* outer, int32_t geom, double a0,
                                double a1, double radius);

/* Packets at the equilibrium of host conserved arrays (physical units, as
   lbm_set_moments; my may be NULL in 1-D).  Waits for the copies. */
lbm_status lbm_bgk_set_moments(lbm_bgk* h, const double* rho, const double* mx,
                               const double* my, const double* rhoE,
                               int64_t n);

/* Set / read every node's packets (layout above, NP * NF * n doubles; n must
   be nx * ny).  lbm_bgk_packets waits and reports device errors; with
   lbm_bgk_set_packets it is checkpoint / restart of the tau != 1 state. */
lbm_status lbm_bgk_set_packets(lbm_bgk* h, const double* f, int64_t n);
lbm_status lbm_bgk_packets(lbm_bgk* h, double* f, int64_t n);

/* Advance nsteps steps: per step a collision pass over the padded grid and
   a gather pass over the nodes.  Stream-ordered, does not wait; LBM_ESTATE
   and LBM_EREACH (the state is then left as it was) arrive at the next
   waiting call. */
lbm_status lbm_bgk_step(lbm_bgk* h, int64_t nsteps);

/* Moments Y = sum_j f_j of every node, physical units, as lbm_moments
   (p nullable).  Waits. */
lbm_status lbm_bgk_moments(lbm_bgk* h, double* rho, double* mx, double* my,
                           double* rhoE, double* p, int64_t n);

/* FP64 totals of the moments, as lbm_conservation.  Waits. */
lbm_status lbm_bgk_conservation(lbm_bgk* h, double out[4]);

/* Steps since the state was set, clamped energies (e < 0 set to 0), the
   reach R of the last step, device flags (bit 0 LBM_ESTATE, bit 1
   LBM_EREACH).  Any pointer may be NULL.  Waits. */
lbm_status lbm_bgk_diagnostics(lbm_bgk* h, int64_t* steps, int64_t* eclamps,
                               int32_t* reach, uint32_t* flags);

/* Wait for queued work and report device-side errors. */
lbm_status lbm_bgk_synchronize(lbm_bgk* h);

const char* lbm_bgk_last_error(const lbm_bgk* h);

/* Free the handle and its device memory.  NULL-safe.  Waits first. */
void lbm_bgk_destroy(lbm_bgk* h);

/* ---- allocation-free single step --------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code running under an allocator it does not
 * own, services that must reserve all their memory up front, or real-time
 * loops where an allocation could stall.  It performs one tau = 1 step, the
 * same fused kernel as lbm_step, from caller-owned device arrays to
 * caller-owned device arrays, and allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine).
 *
 * Its scratch (migration reach, error flags, a block ticket and the FP64
 * partial sums for the totals) is one static device array of
 * LBM_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits.  It bounds the grid: at most 32,760 tiles of the
 * step kernel (1-D tiles are 256 nodes, 2-D tiles 32 x 8 nodes: about 8.3
 * million nodes).  Larger grids are rejected with LBM_EINVAL and a message
 * naming the limit; use lbm_create / lbm_step for them.
 *
 * Arrays are in lattice units (m = rho u lambda, rhoE scaled by lambda^2),
 * element type float (LBM_F32) or double (LBM_F64), nx*ny nodes, x fastest,
 * order {rho, m_x, m_y, rhoE}; m_y may be NULL in 1-D.  in and out must not
 * overlap.  totals (4 doubles), reach (1 int32) and flags (1 uint32) are
 * optional device pointers that receive the new state's FP64 totals, the
 * reach of the new state and the device error flags.  The maximum reach
 * is the lbm_create default (1-D 64, 2-D 6).  Work is queued on stream
 * (cudaStream_t, NULL = default stream); the call returns without waiting,
 * so device-side errors arrive only through flags: a caller that passes
 * flags = NULL cannot tell a failed step from a good one.  Per bit:
 *   bit 1 (2, LBM_EREACH): the input's reach exceeds the maximum; the step
 *     did not run: out is left as it was, totals are 0 and reach is the
 *     input's;
 *   bit 0 (1, LBM_ESTATE): a node of the input or of the new state has
 *     rho < 0 or a non-finite moment; the step ran, but out and totals
 *     hold whatever that state produced and must not be used.
 * With flags == 0, out, totals and reach are valid.  err (nullable, err_len
 * bytes) receives a message on a host-side failure.
 *
 * Every call shares the one scratch array, which keeps the last call's
 * contents; each call clears the part that must start at zero.  Calls that
 * overlap on the GPU (different streams or threads at the same time) race
 * on it and must be serialized by the caller.  The first call on a device
 * looks up the array's device address (once per device, with that device
 * current; again after the device's context was destroyed and created
 * anew, e.g. by cudaDeviceReset); make that first call, and the first call
 * after such a reset, before any stream capture.
 */
#define LBM_NOALLOC_SCRATCH_BYTES (1u << 20)

typedef struct {
  int32_t dim, precision, bc_x, bc_y;
  int64_t nx, ny;
  double gamma, theta;
} lbm_noalloc_desc;

lbm_status lbm_step_noalloc(const lbm_noalloc_desc* d, const void* const in[4],
                            void* const out[4], double* totals, int32_t* reach,
                            uint32_t* flags, void* stream, char* err,
                            size_t err_len);

/* ---- measurement: arithmetic roof of the device ------------------------
 * The paper has no counterpart: this reports the device's fused
 * multiply-add throughput so that the step kernels' arithmetic can be stated
 * as a fraction of what the current GPU sustains.
 *
 * Runs, on the current device and the given stream (cudaStream_t, NULL =
 * default), a kernel of independent FMA chains in precision (lbm_precision:
 * FP32 or FP64), several times, and writes the best rate to *flops_per_s
 * (2 flops per FMA).  Synchronizes the stream; allocates nothing.  Returns
 * LBM_EINVAL for a NULL pointer or unknown precision, LBM_ECUDA if a launch
 * or timing call fails.
 */
lbm_status lbm_measure_fma_peak(int32_t precision, double* flops_per_s,
                                void* stream);

/* ---- diagnostics: FP32 reciprocal and quotient of the FP32 kernels -----
 * The paper has no counterpart: the FP32 kernels form 1/rho from the
 * hardware reciprocal estimate with one Newton-Raphson step and the level
 * densities' quotient by 4 (2 c1 + 1) (eqs 24-25) with Markstein's
 * correction.  This measures both against CUDA's correctly rounded division
 * on n inputs from a counter-based generator (SplitMix64, stream `seed`):
 * x = m 2^e with e in [-30, 30] for the reciprocal, numerators m 2^e with e
 * in [-20, 20] over the denominators 4 (2 c + 1), c = 0 .. 15, for the
 * quotient.  worst_ulp[0] and worst_ulp[1] receive the largest distances in
 * units in the last place.  Runs on the current device and the given
 * stream (NULL = default) and synchronizes it; allocates nothing (its two
 * result words are a file-scope device array).  LBM_EINVAL for n < 0 or a
 * NULL pointer, LBM_ECUDA if a launch or copy fails.
 */
lbm_status lbm_check_fp32_arith(int64_t n, uint64_t seed, double worst_ulp[2],
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
