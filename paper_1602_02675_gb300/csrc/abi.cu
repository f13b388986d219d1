// C ABI of the solver: handle lifetime, configuration checks, launches and
// host transfers.  Declarations and contracts: include/lbm.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_handle {
  lbm_config cfg;
  cudaStream_t stream = nullptr;
  bool f64 = true;
  int dim = 1;
  int nx = 1, ny = 1;
  int64_t n = 0;
  double dx = 0.0, lambda = 0.0;
  EqConst k{};
  int r_cap = 0;
  size_t smem = 0;
  int nblocks = 0;
  void* buf[2][4] = {{nullptr}};
  int cur = 0;
  // FP64 square lattice: source records of the state being stepped,
  // rewritten before every step.
  void* src = nullptr;
  // FP32 square lattice: per-tile window records of the deposit kernel.
  unsigned* hint = nullptr;
  Scratch* scr = nullptr;
  double* part = nullptr;
  int part_cap = 0;
  double* staging = nullptr;
  int64_t steps = 0;
  bool broken = false;
  std::string err;
};

namespace {

const char* kNoHandle = "lbm: NULL handle";

lbm_status fail(lbm_handle* h, lbm_status st, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (st != LBM_EINVAL) h->broken = true;
  }
  return st;
}

lbm_status cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
  return fail(h, LBM_ECUDA,
              std::string("lbm: ") + what + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, call, what)                 \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, (what)); \
  } while (0)

lbm_status check_usable(lbm_handle* h) {
  if (!h) return LBM_EINVAL;
  if (h->broken)
    return fail(h, LBM_ECUDA, "lbm: handle is in an error state: " + h->err);
  return LBM_OK;
}

size_t esize(const lbm_handle* h) { return h->f64 ? 8 : 4; }

// Device pointers of the current state.
void cur_fields(lbm_handle* h, void* f[4]) {
  for (int i = 0; i < 4; ++i) f[i] = h->buf[h->cur][i];
}

lbm_status ensure_staging(lbm_handle* h) {
  if (h->staging) return LBM_OK;
  cudaError_t e = cudaMalloc(&h->staging, sizeof(double) * 5 * (size_t)h->n);
  if (e != cudaSuccess) {
    h->staging = nullptr;
    return fail(h, LBM_ENOMEM, "lbm: staging allocation failed");
  }
  return LBM_OK;
}

// Read device flags; map them to a status.
lbm_status check_flags(lbm_handle* h) {
  Scratch s;
  cudaError_t e = cudaMemcpyAsync(&s, h->scr, sizeof(Scratch),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  if (s.flags & kFlagState)
    return fail(h, LBM_ESTATE,
                "lbm: a node reached rho < 0 or a non-finite moment");
  if (s.flags & kFlagTimeout)
    return fail(h, LBM_ETIMEOUT,
                "lbm: a bounded wait for a shared-memory copy gave up");
  if (s.flags & kFlagReach)
    return fail(h, LBM_EREACH,
                "lbm: migration reach exceeded max_reach (raise "
                "lbm_config.max_reach)");
  return LBM_OK;
}

lbm_status seed_reach(lbm_handle* h) {
  void* f[4];
  cur_fields(h, f);
  LBM_CUDA(h, launch_reach(h->f64, h->dim, f, h->n, h->k, h->scr, h->stream),
           "reach kernel");
  return LBM_OK;
}

}  // namespace

namespace lbm {

bool handle_ds_args(lbm_handle* h, int parity, StepArgs* a) {
  if (!h || h->broken || h->dim != 2 || h->f64 || h->r_cap > ds_rmax() ||
      !h->hint)
    return false;
  a->nx = h->nx;
  a->ny = h->ny;
  a->bc_x = h->cfg.bc_x;
  a->bc_y = h->cfg.bc_y;
  a->r_cap = h->r_cap;
  a->kahan = h->cfg.kahan ? 1 : 0;
  a->exact_order = 0;
  a->do_cons = 0;
  a->nblocks = ds_tiles(h->nx, h->ny, h->r_cap);
  a->k = h->k;
  a->scr = h->scr;
  a->part = h->part;
  a->src = nullptr;
  a->hint = h->hint;
  for (int f = 0; f < 4; ++f) {
    a->in[f] = h->buf[parity][f];
    a->out[f] = h->buf[parity ^ 1][f];
  }
  return true;
}

int handle_cons_every(const lbm_handle* h) { return h->cfg.cons_every; }

int64_t handle_steps(const lbm_handle* h) { return h->steps; }

void handle_took_steps(lbm_handle* h, int64_t n) {
  h->cur ^= (int)(n & 1);
  h->steps += n;
}

}  // namespace lbm

extern "C" {

int32_t lbm_abi_version(void) { return 1; }

}  // extern "C"

namespace lbm {

bool config_ok(const lbm_config& c) {
  if (c.dim != 1 && c.dim != 2) return false;
  if (c.precision != LBM_F32 && c.precision != LBM_F64) return false;
  if (c.nx < 1 || c.ny < 1 || (c.dim == 1 && c.ny != 1)) return false;
  if (c.nx > INT32_MAX || c.ny > INT32_MAX ||
      c.nx * c.ny > (int64_t)INT32_MAX)
    return false;
  if (c.bc_x < 0 || c.bc_x > 2 || (c.dim == 2 && (c.bc_y < 0 || c.bc_y > 2)))
    return false;
  if (!(c.x1 > c.x0) || !(c.gamma > 1.0) || !(c.dt > 0.0)) return false;
  if (!std::isfinite(c.x0) || !std::isfinite(c.x1) || !std::isfinite(c.y0) ||
      !std::isfinite(c.dt) || !std::isfinite(c.gamma))
    return false;
  if (c.dim == 1 && !(c.theta >= 0.0 && c.theta < 1.0)) return false;
  if (c.dim == 2 && c.theta != 0.0) return false;
  if (c.max_reach < 0 || c.cons_every < 0) return false;
  return true;
}

}  // namespace lbm

extern "C" {

lbm_status lbm_create(const lbm_config* cfg, lbm_handle** out) {
  if (!cfg || !out) return LBM_EINVAL;
  *out = nullptr;
  const lbm_config& c = *cfg;
  if (!config_ok(c)) return LBM_EINVAL;

  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return LBM_ENOMEM;
  h->cfg = c;
  h->stream = (cudaStream_t)c.stream;
  h->f64 = (c.precision == LBM_F64);
  h->dim = c.dim;
  h->nx = (int)c.nx;
  h->ny = (int)(c.dim == 2 ? c.ny : 1);
  h->n = (int64_t)h->nx * h->ny;
  h->dx = (c.x1 - c.x0) / (double)c.nx;
  h->lambda = c.dt / h->dx;
  const double D = (double)c.dim;
  h->k.theta = (c.dim == 1) ? c.theta : 0.0;
  h->k.kq = D * (c.gamma - 1.0);
  h->k.kphi = 1.0 - 0.5 * D * (c.gamma - 1.0);
  h->k.b1 = (c.dim == 1) ? 2.0 : 4.0;
  h->k.kreach = h->k.kq / (1.0 - h->k.theta);
  h->k.set_fp32_copies();
  h->r_cap = c.max_reach > 0 ? c.max_reach : (c.dim == 1 ? 64 : 6);
  // the FP64 square-lattice step gathers from source records and needs no
  // shared-memory window; every other step holds its window there
  h->smem = (h->f64 && c.dim == 2) ? 0 : step_smem_bytes(c.dim, h->f64, h->r_cap);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int optin = 0;
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               dev);
  if (e != cudaSuccess) {
    lbm_status st = cuda_fail(h, e, "device query");
    delete h;
    return st;
  }
  if (h->smem + 1024 > (size_t)optin) {
    delete h;
    return LBM_EINVAL;  // max_reach too large for shared memory
  }
  e = step_prepare(c.dim, h->f64, h->smem);
  if (e != cudaSuccess) {
    lbm_status st = cuda_fail(h, e, "kernel attribute");
    delete h;
    return st;
  }
  h->nblocks = (int)step_blocks(c.dim, h->nx, h->ny);  // nx ny <= INT32_MAX
  h->part_cap = h->nblocks > totals_blocks(h->n) ? h->nblocks
                                                 : totals_blocks(h->n);
  if (c.dim == 2 && !h->f64) {
    // the deposit kernel's tiles and its finalize blocks' partials
    const int dt = ds_tiles(h->nx, h->ny, h->r_cap) + ds_finalize_blocks();
    if (dt > h->part_cap) h->part_cap = dt;
  }
  const size_t fb = esize(h) * (size_t)h->n;
  bool ok = true;
  for (int b = 0; b < 2 && ok; ++b)
    for (int f = 0; f < 4 && ok; ++f) {
      if (f == 2 && c.dim == 1) continue;
      ok = cudaMalloc(&h->buf[b][f], fb) == cudaSuccess;
    }
  if (ok && c.dim == 2 && h->f64)
    ok = cudaMalloc(&h->src, src_bytes(h->nx, h->ny, h->r_cap, esize(h))) ==
         cudaSuccess;
  const int dst = (c.dim == 2 && !h->f64) ? ds_tiles(h->nx, h->ny, h->r_cap) : 0;
  if (ok && dst > 0) {
    ok = cudaMalloc(&h->hint, sizeof(unsigned) * (size_t)dst) == cudaSuccess;
    if (ok)
      ok = cudaMemsetAsync(h->hint, 0, sizeof(unsigned) * (size_t)dst,
                           h->stream) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&h->scr, sizeof(Scratch)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->part, sizeof(double) * 4 * (size_t)h->part_cap) ==
                 cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_destroy(h);
    return LBM_ENOMEM;
  }
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 4; ++f)
      if (h->buf[b][f]) cudaMemsetAsync(h->buf[b][f], 0, fb, h->stream);
  cudaMemsetAsync(h->scr, 0, sizeof(Scratch), h->stream);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    lbm_status st = cuda_fail(h, e, "initial clear");
    lbm_destroy(h);
    return st;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_init_riemann(lbm_handle* h, const lbm_prim* inner,
                            const lbm_prim* outer, int32_t geom, double a0,
                            double a1, double radius) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!inner || !outer || (geom != LBM_PLANAR_X && geom != LBM_CIRCLE))
    return fail(h, LBM_EINVAL, "lbm_init_riemann: bad argument");
  if (!(inner->rho >= 0.0) || !(outer->rho >= 0.0) || !(inner->p >= 0.0) ||
      !(outer->p >= 0.0))
    return fail(h, LBM_EINVAL, "lbm_init_riemann: negative rho or p");
  InitArgs a;
  cur_fields(h, a.f);
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
  LBM_CUDA(h, launch_init(h->f64, a, h->stream), "init kernel");
  LBM_CUDA(h, cudaMemsetAsync(h->scr, 0, sizeof(Scratch), h->stream),
           "scratch clear");
  h->steps = 0;
  return seed_reach(h);
}

static lbm_status set_from_host(lbm_handle* h, int kind, const double* a,
                                const double* b, const double* c,
                                const double* d, int64_t n) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!a || !b || !d || (h->dim == 2 && !c) || n != h->n)
    return fail(h, LBM_EINVAL, "lbm_set: bad arrays or size");
  st = ensure_staging(h);
  if (st != LBM_OK) return st;
  const size_t nb = sizeof(double) * (size_t)n;
  LBM_CUDA(h, cudaMemcpyAsync(h->staging, a, nb, cudaMemcpyHostToDevice,
                              h->stream), "copy to device");
  LBM_CUDA(h, cudaMemcpyAsync(h->staging + n, b, nb, cudaMemcpyHostToDevice,
                              h->stream), "copy to device");
  if (h->dim == 2)
    LBM_CUDA(h, cudaMemcpyAsync(h->staging + 2 * n, c, nb,
                                cudaMemcpyHostToDevice, h->stream),
             "copy to device");
  LBM_CUDA(h, cudaMemcpyAsync(h->staging + 3 * n, d, nb,
                              cudaMemcpyHostToDevice, h->stream),
           "copy to device");
  void* f[4];
  cur_fields(h, f);
  LBM_CUDA(h, launch_from_host_layout(h->f64, kind, h->dim, h->staging, f, n,
                                      h->lambda, h->cfg.gamma, h->stream),
           "convert kernel");
  LBM_CUDA(h, cudaMemsetAsync(h->scr, 0, sizeof(Scratch), h->stream),
           "scratch clear");
  h->steps = 0;
  st = seed_reach(h);
  if (st != LBM_OK) return st;
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LBM_OK;
}

lbm_status lbm_set_primitives(lbm_handle* h, const double* rho,
                              const double* u, const double* v,
                              const double* p, int64_t n) {
  return set_from_host(h, 0, rho, u, v, p, n);
}

lbm_status lbm_set_moments(lbm_handle* h, const double* rho, const double* mx,
                           const double* my, const double* rhoE, int64_t n) {
  return set_from_host(h, 1, rho, mx, my, rhoE, n);
}

lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (nsteps < 0) return fail(h, LBM_EINVAL, "lbm_step: nsteps < 0");
  StepArgs a;
  a.nx = h->nx;
  a.ny = h->ny;
  a.bc_x = h->cfg.bc_x;
  a.bc_y = h->dim == 2 ? h->cfg.bc_y : 0;
  a.r_cap = h->r_cap;
  a.kahan = h->cfg.kahan ? 1 : 0;
  a.nblocks = h->nblocks;
  a.k = h->k;
  a.scr = h->scr;
  a.part = h->part;
  a.src = h->src;
  a.hint = h->hint;
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int f = 0; f < 4; ++f) {
      a.in[f] = h->buf[h->cur][f];
      a.out[f] = h->buf[h->cur ^ 1][f];
    }
    const int every = h->cfg.cons_every;
    a.do_cons = (every > 0 && ((h->steps + 1) % every) == 0) ? 1 : 0;
    LBM_CUDA(h, launch_step(h->dim, h->f64, a, h->smem, h->stream),
             "step kernel");
    h->cur ^= 1;
    h->steps += 1;
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_handle* h, double* rho, double* mx, double* my,
                       double* rhoE, double* p, int64_t n) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!rho || !mx || !rhoE || n != h->n)
    return fail(h, LBM_EINVAL, "lbm_moments: bad arrays or size");
  st = ensure_staging(h);
  if (st != LBM_OK) return st;
  void* f[4];
  cur_fields(h, f);
  LBM_CUDA(h, launch_to_host_layout(h->f64, h->dim, f, h->staging, n,
                                    h->lambda, h->cfg.gamma, h->stream),
           "readback kernel");
  const size_t nb = sizeof(double) * (size_t)n;
  double* dst[5] = {rho, mx, (h->dim == 2) ? my : nullptr, rhoE, p};
  for (int i = 0; i < 5; ++i)
    if (dst[i])
      LBM_CUDA(h, cudaMemcpyAsync(dst[i], h->staging + (size_t)i * n, nb,
                                  cudaMemcpyDeviceToHost, h->stream),
               "copy to host");
  return check_flags(h);
}

lbm_status lbm_conservation(lbm_handle* h, double out[4]) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!out) return fail(h, LBM_EINVAL, "lbm_conservation: NULL out");
  void* f[4];
  cur_fields(h, f);
  LBM_CUDA(h, launch_totals(h->f64, h->dim, f, h->n, h->part, h->part_cap,
                            h->scr, h->stream), "totals kernel");
  st = check_flags(h);
  if (st != LBM_OK) return st;
  Scratch sc;
  LBM_CUDA(h, cudaMemcpyAsync(&sc, h->scr, sizeof(Scratch),
                              cudaMemcpyDeviceToHost, h->stream),
           "copy totals");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  const double* c = sc.cons;
  out[0] = c[0];
  out[1] = c[1] / h->lambda;
  out[2] = c[2] / h->lambda;
  out[3] = c[3] / (h->lambda * h->lambda);
  return LBM_OK;
}

lbm_status lbm_last_totals(lbm_handle* h, double out[4]) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!out) return fail(h, LBM_EINVAL, "lbm_last_totals: NULL out");
  st = check_flags(h);
  if (st != LBM_OK) return st;
  Scratch sc;
  LBM_CUDA(h, cudaMemcpyAsync(&sc, h->scr, sizeof(Scratch),
                              cudaMemcpyDeviceToHost, h->stream),
           "copy totals");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  out[0] = sc.cons[0];
  out[1] = sc.cons[1] / h->lambda;
  out[2] = sc.cons[2] / h->lambda;
  out[3] = sc.cons[3] / (h->lambda * h->lambda);
  return LBM_OK;
}

lbm_status lbm_reach(lbm_handle* h, int32_t* reach) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  if (!reach) return fail(h, LBM_EINVAL, "lbm_reach: NULL out");
  st = check_flags(h);
  if (st != LBM_OK) return st;
  Scratch sc;
  LBM_CUDA(h, cudaMemcpyAsync(&sc, h->scr, sizeof(Scratch),
                              cudaMemcpyDeviceToHost, h->stream),
           "copy reach");
  LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
  *reach = sc.reach;
  return LBM_OK;
}

lbm_status lbm_diagnostics(lbm_handle* h, int64_t* steps, int64_t* eclamps,
                           uint32_t* flags) {
  if (!h) return LBM_EINVAL;
  Scratch s;
  cudaError_t e = cudaMemcpyAsync(&s, h->scr, sizeof(Scratch),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
  if (steps) *steps = h->steps;
  if (eclamps) *eclamps = (int64_t)s.eclamps;
  if (flags) *flags = s.flags;
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_handle* h) {
  lbm_status st = check_usable(h);
  if (st != LBM_OK) return st;
  return check_flags(h);
}

double lbm_lambda(const lbm_handle* h) { return h ? h->lambda : 0.0; }

const char* lbm_last_error(const lbm_handle* h) {
  return h ? h->err.c_str() : kNoHandle;
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 4; ++f)
      if (h->buf[b][f]) cudaFree(h->buf[b][f]);
  if (h->src) cudaFree(h->src);
  if (h->hint) cudaFree(h->hint);
  if (h->scr) cudaFree(h->scr);
  if (h->part) cudaFree(h->part);
  if (h->staging) cudaFree(h->staging);
  cudaGetLastError();
  delete h;
}

}  // extern "C"
