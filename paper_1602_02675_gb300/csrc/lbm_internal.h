// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

struct lbm_handle;
#include "lbm.h"

namespace lbm {

// Device error flags (Scratch::flags).
enum : unsigned { kFlagState = 1u, kFlagReach = 2u, kFlagTimeout = 4u };

// Small device-resident block of per-handle scratch words.
struct Scratch {
  int reach;               // migration reach the next step uses
  int reach_next;          // max-reduced by the running step
  unsigned flags;          // kFlag*
  unsigned ticket;         // blocks finished in the running launch
  unsigned long long eclamps;  // nodes whose e < 0 was clamped to 0
  double cons[4];          // FP64 totals (lattice units) of the last sum
  unsigned spare_;
  unsigned mixed_ticket;   // FP32 square lattice: tiles taken this step
};

// Constants of the equilibrium (Section III.B) for one lattice and gas.
struct EqConst {
  double theta;  // 1-D: d0 = theta*rho; 2-D: 0
  double kq;     // D (gamma - 1)
  double kphi;   // 1 - D/2 (gamma - 1)     (eq 15)
  double b1;     // directions per level: 2 (1-D), 4 (square lattice)
  double kreach; // D (gamma - 1) / (1 - b0 theta): X = kreach * e
  // the same constants rounded to FP32 once on the host (set_fp32_copies),
  // so that FP32 kernels convert nothing on the GPU's slow FP64 pipe
  float theta_f, kq_f, kphi_f, b1_f, kreach_f;

  void set_fp32_copies() {
    theta_f = (float)theta;
    kq_f = (float)kq;
    kphi_f = (float)kphi;
    b1_f = (float)b1;
    kreach_f = (float)kreach;
  }
};

struct StepArgs {
  const void* in[4];  // rho, m_x, m_y, rhoE (m_y unused in 1-D)
  void* out[4];
  int nx, ny;
  int bc_x, bc_y;
  int r_cap;          // largest reach the launch's shared memory holds
  int kahan;          // F32: compensated summation of the arrivals
  int exact_order = 0;  // F32 2-D: step with the exact-order kernel
  int do_cons;        // this launch also sums FP64 totals
  int nblocks;
  EqConst k;
  Scratch* scr;
  double* part;       // [nblocks * 4] FP64 partial sums
  // FP32 square lattice (deposit kernel): per tile, the record of its
  // window at the last step (0: one type; else the window's smallest c1 and
  // shift and its group block, a starting guess only), sized for the tiles
  // of the largest reach.
  unsigned* hint = nullptr;
  // FP64 square lattice: source records of the input state over the grid
  // padded by r_cap (layout in step_kernel.cuh), written by the launcher's
  // records pass before each step, or null.
  void* src = nullptr;
};

// Bytes of the square-lattice source records of an nx x ny grid with reach
// limit r_cap and elements of esize bytes: 30 fields of esize bytes and one
// 8-byte word per padded node.
inline size_t src_bytes(int nx, int ny, int r_cap, size_t esize) {
  return (size_t)(nx + 2 * r_cap) * (size_t)(ny + 2 * r_cap) * (30 * esize + 8);
}

// Checks of an lbm_config shared by the handle constructors (sizes,
// boundary kinds, gas, extent, time step, rest share, reach limit); no CUDA
// call.  True if the configuration is valid.
bool config_ok(const lbm_config& c);

// Multiprocessors of the current device (cached per device; 1 if the
// query fails, which only makes grids smaller).
int device_sm_count();

// Tiles of the FP32 square-lattice deposit kernel at the largest reach
// r_cap (0 if r_cap is beyond its layout): the size of the per-tile hint
// and queue arrays a handle holds for it.
int ds_tiles(int nx, int ny, int r_cap);
// Largest reach limit the deposit kernel's window takes.
int ds_rmax();

// For the batched 2-D grids (batch2d.cu): the deposit kernel's arguments of
// handle h's step from state parity `parity` (in = buffers parity, out = the
// other set; do_cons 0), or false if h does not step with the deposit kernel
// or is broken; the handle's cons_every and step count; and the bookkeeping
// after the batch took n steps of h's grid.
bool handle_ds_args(lbm_handle* h, int parity, StepArgs* a);
int handle_cons_every(const lbm_handle* h);
int64_t handle_steps(const lbm_handle* h);
void handle_took_steps(lbm_handle* h, int64_t n);

// Blocks of the deposit kernel's finalize launch// Blocks of the deposit kernel's finalize launch (each leaves one set of
// partial totals after the tiles' partials).
int ds_finalize_blocks();

// Launch helpers (step kernels).
size_t step_smem_bytes(int dim, bool f64, int r_cap);
cudaError_t step_prepare(int dim, bool f64, size_t smem);
// Blocks of the exact-order step kernel for an nx x ny grid (64-bit: no
// overflow for any int sizes).
long long step_blocks(int dim, int nx, int ny);
cudaError_t launch_step(int dim, bool f64, const StepArgs& a, size_t smem,
                        cudaStream_t s);

// Auxiliary kernels (init, conversion, reductions).
struct InitArgs {
  void* f[4];
  int nx, ny, dim;
  double x0, y0, dx, lambda, gamma;
  int geom;                 // 0 planar (x < a0 -> inner), 1 circle
  double a0, a1, radius;
  double in_[4], out_[4];   // rho, u, v, p of the inner / outer state
};
cudaError_t launch_init(bool f64, const InitArgs& a, cudaStream_t s);

// staging holds n doubles per field; kind 0 = primitives (rho, u, v, p),
// kind 1 = physical conserved (rho, rho u, rho v, rho E).
cudaError_t launch_from_host_layout(bool f64, int kind, int dim,
                                    const double* staging, void* const f[4],
                                    int64_t n, double lambda, double gamma,
                                    cudaStream_t s);

// Lattice state -> physical (rho, m_x, m_y, rhoE, p) in staging.
cudaError_t launch_to_host_layout(bool f64, int dim, const void* const f[4],
                                  double* staging, int64_t n, double lambda,
                                  double gamma, cudaStream_t s);

// Reach of the current state into scr->reach (conservative, see kernels).
cudaError_t launch_reach(bool f64, int dim, const void* const f[4], int64_t n,
                         const EqConst& k, Scratch* scr, cudaStream_t s);

// FP64 totals of the current state into scr->cons (fixed order).
cudaError_t launch_totals(bool f64, int dim, const void* const f[4], int64_t n,
                          double* part, int nblocks_cap, Scratch* scr,
                          cudaStream_t s);
int totals_blocks(int64_t n);

}  // namespace lbm
