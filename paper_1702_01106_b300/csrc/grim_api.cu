// C ABI of the grim library (declarations and documentation: include/grim.h).
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <vector>

#include "grim_dev.cuh"
#include "../../include/grim.h"

namespace grim {
cudaError_t launch_explicit(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                            double* K, double* P0, cudaStream_t st);
cudaError_t launch_newton(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                          Counters* cnt, cudaStream_t st);
cudaError_t launch_residual(const Params& p, const double* K, const double* Pk, int scaled, double dts, double* R,
                            cudaStream_t st);
cudaError_t launch_rcp_check(int n, unsigned long long seed, double* worst, cudaStream_t st);
long long face_scratch_doubles(int n1, int n2);
cudaError_t launch_faces(const Params& p, const double* PE, double* faces, cudaStream_t st);
cudaError_t launch_zone_const(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                              double* K, double* P0, double* faces, double* cache, int mode, cudaStream_t st);
long long pn_cache_doubles(long long N);
cudaError_t launch_newton_fb(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                             Counters* cnt, const double* Pfb, double accept, cudaStream_t st);
cudaError_t launch_mlp_features(const Params& p, const double* K, const double* Pn, const double* Pc, float* X,
                                float* Y, cudaStream_t st);
cudaError_t launch_mlp_guess(const Params& p, const double* K, const double* Pn, const double* Un, const grim_mlp* m,
                             double* P0, cudaStream_t st);
}  // namespace grim

using grim::Params;

struct grim_ctx {
  Params p;
  int precision;
  cudaStream_t stream;
  double* K = nullptr;        // NK x N stage constants
  double* faces = nullptr;    // face fluxes of one stage
  double* pncache = nullptr;  // P_n quantities shared by the two stages of a step
  double* Ph = nullptr;       // half-step state
  uint8_t* iters = nullptr;   // per-zone Newton updates of the last stage
  uint8_t* status = nullptr;  // per-zone status bits of the last stage
  grim::Counters* cnt = nullptr;
  double* dev_in = nullptr;   // device copies for grim_step_host
  double* dev_out = nullptr;
  unsigned long long launches = 0;
  grim_mlp* mlp = nullptr;    // learned initial guess (grim_set_guess)
  double accept = 0.0;
  // per-kernel timing: (class, start, stop) event triples
  bool profile = false;
  struct Mark { int cls; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double ms_acc[GRIM_K_COUNT] = {0};
  unsigned long long n_acc[GRIM_K_COUNT] = {0};
  char err[256];

  cudaEvent_t event() {
    cudaEvent_t e;
    if (!pool.empty()) { e = pool.back(); pool.pop_back(); return e; }
    cudaEventCreate(&e);
    return e;
  }
};

// Record an event pair around one launch when profiling.
struct KernelMark {
  grim_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  KernelMark(grim_ctx* ctx, int k) : c(ctx), cls(k) {
    c->launches++;
    if (c->profile) { a = c->event(); cudaEventRecord(a, c->stream); }
  }
  ~KernelMark() {
    if (c->profile) {
      cudaEvent_t b = c->event();
      cudaEventRecord(b, c->stream);
      c->marks.push_back({cls, a, b});
    }
  }
};

static int fail(grim_ctx* c, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (c) {
    if (e != cudaSuccess)
      snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
    else
      snprintf(c->err, sizeof(c->err), "%s", what);
  }
  return code;
}

#define GRIM_CUDA(call, what)                                  \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fail(ctx, GRIM_ECUDA, what, e_); \
  } while (0)

extern "C" {

const char* grim_strerror(int code) {
  switch (code) {
    case GRIM_OK: return "ok";
    case GRIM_EINVAL: return "invalid argument or unsupported configuration";
    case GRIM_ECUDA: return "CUDA runtime error";
    case GRIM_ENOMEM: return "device allocation failed";
    case GRIM_ESIZE: return "size outside the limit of this entry point";
    default: return "unknown error";
  }
}

const char* grim_last_error(grim_ctx* ctx) { return ctx ? ctx->err : "no context"; }

void grim_destroy(grim_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->K);
  cudaFree(ctx->faces);
  cudaFree(ctx->pncache);
  cudaFree(ctx->Ph);
  cudaFree(ctx->iters);
  cudaFree(ctx->status);
  cudaFree(ctx->cnt);
  cudaFree(ctx->dev_in);
  cudaFree(ctx->dev_out);
  for (auto& m : ctx->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

int grim_init(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys, const grim_solver* solver,
              void* stream, grim_ctx** out) {
  if (!out) return GRIM_EINVAL;
  *out = nullptr;
  if (!grid || !metric || !phys || !solver) return GRIM_EINVAL;
  if (grid->dim != 2 || grid->n3 != 1 || grid->n1 < 1 || grid->n2 < 1) return GRIM_EINVAL;
  if (metric->kind != GRIM_METRIC_MINKOWSKI) return GRIM_EINVAL;
  if (phys->recon != GRIM_RECON_MC && phys->recon != GRIM_RECON_WENO5) return GRIM_EINVAL;
  if (solver->precision != GRIM_FP64 && solver->precision != GRIM_MIXED) return GRIM_EINVAL;
  if (!(phys->gamma > 1.0) || !(phys->tau_R > 0.0) || !(solver->tol > 0.0) || solver->k_max < 0 ||
      solver->k_max > 250 || solver->ls_max < 0)
    return GRIM_EINVAL;
  for (int d = 0; d < 3; d++)
    for (int s = 0; s < 2; s++)
      if (grid->bc[d][s] < 0 || grid->bc[d][s] > 2) return GRIM_EINVAL;
  grim_ctx* ctx = new grim_ctx();
  ctx->err[0] = 0;
  Params& p = ctx->p;
  std::memset(&p, 0, sizeof(p));
  p.dim = grid->dim; p.n1 = grid->n1; p.n2 = grid->n2; p.n3 = grid->n3;
  for (int d = 0; d < 3; d++) {
    p.bc[d][0] = grid->bc[d][0]; p.bc[d][1] = grid->bc[d][1];
    int n = (d == 0) ? grid->n1 : (d == 1) ? grid->n2 : grid->n3;
    p.dx[d] = (grid->x_end[d] - grid->x_start[d]) / n;
    p.idx[d] = 1.0 / p.dx[d];
  }
  p.gamma = phys->gamma; p.phi = phys->phi; p.psi = phys->psi; p.tauR = phys->tau_R; p.theta = phys->theta;
  p.cond = phys->conduction; p.visc = phys->viscosity; p.ho = phys->higher_order; p.recon = phys->recon;
  p.tol = solver->tol; p.eps64 = solver->eps_fd; p.eps32 = (float)solver->eps_fd32;
  p.kmax = solver->k_max; p.lsmax = solver->ls_max; p.fd32c = solver->fd32_central != 0;
  p.N = (long long)grid->n1 * grid->n2 * grid->n3;
  ctx->precision = solver->precision;
  ctx->stream = (cudaStream_t)stream;
  const size_t N = (size_t)p.N;
  cudaError_t e;
  if ((e = cudaMalloc(&ctx->K, sizeof(double) * grim::NK * N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->Ph, sizeof(double) * grim::NV * N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->faces, sizeof(double) * grim::face_scratch_doubles(p.n1, p.n2))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->pncache, sizeof(double) * grim::pn_cache_doubles(p.N))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->iters, N)) != cudaSuccess || (e = cudaMalloc(&ctx->status, N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->cnt, sizeof(grim::Counters))) != cudaSuccess) {
    grim_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
  }
  if ((e = cudaMemsetAsync(ctx->cnt, 0, sizeof(grim::Counters), ctx->stream)) != cudaSuccess) {
    grim_destroy(ctx);
    return GRIM_ECUDA;
  }
  *out = ctx;
  return GRIM_OK;
}

// The explicit part of a stage: face fluxes, then flux-CT and the constants.
static int run_explicit(grim_ctx* ctx, const double* Pn, const double* PE, double dts, const double* guess,
                        double* Pout, int mode) {
  {
    KernelMark m(ctx, GRIM_K_FACES);
    GRIM_CUDA(grim::launch_faces(ctx->p, PE, ctx->faces, ctx->stream), "face kernel");
  }
  {
    KernelMark m(ctx, GRIM_K_ZONECONST);
    GRIM_CUDA(grim::launch_zone_const(ctx->p, Pn, PE, guess, dts, ctx->K, Pout, ctx->faces, ctx->pncache, mode,
                                      ctx->stream),
              "zone-constant kernel");
  }
  return GRIM_OK;
}

static int run_stage(grim_ctx* ctx, const double* Pn, const double* PE, double dts, const double* guess,
                     double* Pout, uint8_t* iters, uint8_t* status, int mode = 0) {
  int rc = run_explicit(ctx, Pn, PE, dts, guess, Pout, mode);
  if (rc) return rc;
  const bool learned = ctx->mlp && !guess;
  if (learned) {
    KernelMark m(ctx, GRIM_K_MLP);
    GRIM_CUDA(grim::launch_mlp_guess(ctx->p, ctx->K, Pn, mode ? ctx->pncache : nullptr, ctx->mlp, Pout, ctx->stream),
              "mlp kernel");
  }
  {
    KernelMark m(ctx, ctx->precision ? GRIM_K_NEWTON32 : GRIM_K_NEWTON64);
    GRIM_CUDA(grim::launch_newton_fb(ctx->p, ctx->precision, ctx->K, Pout, iters ? iters : ctx->iters,
                                     status ? status : ctx->status, ctx->cnt, learned ? Pn : nullptr, ctx->accept,
                                     ctx->stream),
              "newton kernel");
  }
  return GRIM_OK;
}

int grim_stage(grim_ctx* ctx, const double* P_n, const double* P_E, double dts, const double* guess, double* P_out,
               unsigned char* iters, unsigned char* status) {
  if (!ctx || !P_n || !P_E || !P_out || !(dts > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_stage: bad argument");
  // other CTAs read P_E around their tiles while P_out is written
  if (P_out == P_E) return fail(ctx, GRIM_EINVAL, "grim_stage: P_out must not alias P_E");
  return run_stage(ctx, P_n, P_E, dts, guess, P_out, iters, status);
}

int grim_step(grim_ctx* ctx, const double* P_in, double* P_out, double dt) {
  if (!ctx || !P_in || !P_out || !(dt > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_step: bad argument");
  // The half step (P^E = P_n) caches the P_n quantities the full step reuses.
  int rc = run_stage(ctx, P_in, P_in, 0.5 * dt, nullptr, ctx->Ph, nullptr, nullptr, 1);
  if (rc) return rc;
  // The full stage reads P_n only at each zone itself, so P_out may alias P_in.
  return run_stage(ctx, P_in, ctx->Ph, dt, nullptr, P_out, nullptr, nullptr, 2);
}

int grim_step_host(grim_ctx* ctx, const double* P_in_host, double* P_out_host, double dt) {
  if (!ctx || !P_in_host || !P_out_host) return fail(ctx, GRIM_EINVAL, "grim_step_host: bad argument");
  const size_t bytes = sizeof(double) * grim::NV * (size_t)ctx->p.N;
  if (!ctx->dev_in) {
    cudaError_t e;
    if ((e = cudaMalloc(&ctx->dev_in, bytes)) != cudaSuccess || (e = cudaMalloc(&ctx->dev_out, bytes)) != cudaSuccess)
      return fail(ctx, GRIM_ENOMEM, "grim_step_host: device buffers", e);
  }
  GRIM_CUDA(cudaMemcpyAsync(ctx->dev_in, P_in_host, bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D copy");
  int rc = grim_step(ctx, ctx->dev_in, ctx->dev_out, dt);
  if (rc) return rc;
  GRIM_CUDA(cudaMemcpyAsync(P_out_host, ctx->dev_out, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H copy");
  GRIM_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return GRIM_OK;
}

int grim_residual(grim_ctx* ctx, const double* P_n, const double* P_E, double dts, const double* P_k, int scaled,
                  double* R_out) {
  if (!ctx || !P_n || !P_E || !P_k || !R_out || !(dts > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_residual: bad argument");
  // the explicit kernel also writes an initial guess; send it to the half-step scratch
  int rc = run_explicit(ctx, P_n, P_E, dts, nullptr, ctx->Ph, 0);
  if (rc) return rc;
  {
    KernelMark m(ctx, GRIM_K_RESIDUAL);
    GRIM_CUDA(grim::launch_residual(ctx->p, ctx->K, P_k, scaled, dts, R_out, ctx->stream), "residual kernel");
  }
  return GRIM_OK;
}

int grim_get_stats(grim_ctx* ctx, grim_stats* out) {
  if (!ctx || !out) return GRIM_EINVAL;
  grim::Counters c;
  GRIM_CUDA(cudaMemcpyAsync(&c, ctx->cnt, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream), "stats copy");
  GRIM_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  std::memset(out, 0, sizeof(*out));
  out->zones = c.zones; out->failed = c.failed; out->iters = c.iters;
  out->evals64 = c.evals64; out->evals32 = c.evals32; out->lu64 = c.lu64; out->lu32 = c.lu32;
  for (int i = 0; i < 32; i++) out->hist[i] = c.hist[i];
  long long bits = (long long)c.maxres_bits;
  double mr;
  std::memcpy(&mr, &bits, sizeof(mr));
  out->max_res = mr;
  out->launches = ctx->launches;
  out->fallbacks = c.fallbacks;
  return GRIM_OK;
}

int grim_set_guess(grim_ctx* ctx, grim_mlp* mlp, double accept) {
  if (!ctx || !(accept >= 0.0)) return GRIM_EINVAL;
  ctx->mlp = mlp;
  ctx->accept = accept;
  return GRIM_OK;
}

int grim_mlp_sample(grim_ctx* ctx, const double* P_n, const double* P_conv, float* X, float* Y) {
  if (!ctx || !P_n || !X || (Y && !P_conv)) return GRIM_EINVAL;
  {
    KernelMark m(ctx, GRIM_K_MLP);
    GRIM_CUDA(grim::launch_mlp_features(ctx->p, ctx->K, P_n, P_conv, X, Y, ctx->stream), "feature kernel");
  }
  return GRIM_OK;
}

int grim_profile(grim_ctx* ctx, int enable) {
  if (!ctx) return GRIM_EINVAL;
  ctx->profile = enable != 0;
  return GRIM_OK;
}

int grim_kernel_times(grim_ctx* ctx, double* ms, unsigned long long* launches) {
  if (!ctx) return GRIM_EINVAL;
  GRIM_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  for (auto& m : ctx->marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
      ctx->ms_acc[m.cls] += t;
      ctx->n_acc[m.cls] += 1;
    }
    ctx->pool.push_back(m.a);
    ctx->pool.push_back(m.b);
  }
  ctx->marks.clear();
  for (int k = 0; k < GRIM_K_COUNT; k++) {
    if (ms) ms[k] = ctx->ms_acc[k];
    if (launches) launches[k] = ctx->n_acc[k];
    ctx->ms_acc[k] = 0.0;
    ctx->n_acc[k] = 0;
  }
  return GRIM_OK;
}

int grim_reset_stats(grim_ctx* ctx) {
  if (!ctx) return GRIM_EINVAL;
  GRIM_CUDA(cudaMemsetAsync(ctx->cnt, 0, sizeof(grim::Counters), ctx->stream), "stats reset");
  return GRIM_OK;
}

int grim_math_selftest(int n, double* max_rel_err) {
  if (n < 1 || !max_rel_err) return GRIM_EINVAL;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return GRIM_ENOMEM;
  cudaError_t e = cudaMemset(d, 0, sizeof(double));
  if (e == cudaSuccess) e = grim::launch_rcp_check(n, 12345ull, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(max_rel_err, d, sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? GRIM_OK : GRIM_ECUDA;
}

}  // extern "C"
