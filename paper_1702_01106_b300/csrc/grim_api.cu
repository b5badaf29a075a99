// C ABI of the grim library (declarations and documentation: include/grim.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <string>
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
cudaError_t launch_faces(const Params& p, const double* PE, double* faces, int bs, int ffstates, cudaStream_t st);
cudaError_t launch_zone_const(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                              double* K, double* P0, double* faces, double* cache, int mode, int bs, float* feat,
                              int ffslopes, cudaStream_t st);
long long pn_cache_doubles(long long N);
cudaError_t launch_newton_fb(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                             Counters* cnt, const double* Pfb, double accept, const NewtonCfg& cfg, int* queue,
                             int* qcount, double* rq, const Rescue& rs, const float* rn, cudaStream_t st);
cudaError_t launch_mlp_features(const Params& p, const double* K, const double* Pn, const double* Pc, float* X,
                                float* Y, cudaStream_t st);
cudaError_t launch_mlp_guess(const Params& p, const float* feat, const double* Pn, const grim_mlp* m, double* P0,
                             const float* gf, unsigned long long* stalls, cudaStream_t st);
cudaError_t launch_mlp_metric_table(const Params& p, const double* gc, float* gf, cudaStream_t st);
cudaError_t launch_features_gr(const Params& p, const double* K, const double* gc, const double* Pn, const double* Pc,
                               float* X, float* Y, float* feat, cudaStream_t st);
long long gr_geometry_doubles(const Params& p);
long long gr_face_doubles(const Params& p);
cudaError_t launch_gr_geometry(const Params& p, int metric, double spin, double h, const double x0[3],
                               double* geo, cudaStream_t st);
cudaError_t launch_gr_faces(const Params& p, const double* PE, const double* geo, double* faces, int ffstates,
                            cudaStream_t st);
cudaError_t launch_gr_zone_const(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                                 const double* geo, double* faces, double* K, double* P0, double* cache, int mode,
                                 float* feat, int ffslopes, cudaStream_t st);
long long gr_cache_doubles(long long N);
cudaError_t launch_gr_floors(const Params& p, const double* geo, const double* K, const double* Pn,
                             const uint8_t* status, double* P, cudaStream_t st);
cudaError_t launch_newton_gr(const Params& p, int mixed, const double* K, const double* gc, double* P,
                             uint8_t* iters, uint8_t* status, Counters* cnt, const NewtonCfg& cfg, int* queue,
                             int* qcount, double* rq, const double* Pfb, double accept, const Rescue& rs,
                             const float* rn, cudaStream_t st);
cudaError_t launch_residual_gr(const Params& p, const double* K, const double* gc, const double* Pk, int scaled,
                               double dts, double* R, cudaStream_t st);
}  // namespace grim

using grim::Params;

struct grim_ctx {
  Params p;
  int precision;
  cudaStream_t stream;        // the caller's stream
  cudaStream_t cur;           // where launches go: stream, or cap while capturing
  cudaStream_t cap = nullptr; // private stream for graph capture
  grim_tuning tune{64, 2, 128, 128, 0};
  int* queue = nullptr;       // zones left for the queue kernel
  int* qcount = nullptr;      // their number, then the rescue queue's length
  int* rqueue = nullptr;      // mixed-solver zones handed to the float64 rescue
  bool graphs = false, warmed = false;
  grim_tuning warm_tune{};    // launch shape and guess of the last eager step: every
  bool warm_mlp = false;      // kernel a capture records has been configured
  struct Graph {
    const double* in; double* out; double dt; grim_mlp* mlp; double accept; grim_tuning tune;
    cudaGraphExec_t exec; unsigned long long kernels, last;
  };
  std::vector<Graph> gcache;
  unsigned long long gclock = 0;
  bool gr = false;            // general-metric kernels (3-D or Kerr)
  double* geo = nullptr;      // geometry tables of the general-metric path
  double* K = nullptr;        // NK x N stage constants
  double* faces = nullptr;    // face fluxes of one stage; during the Newton solve,
                              // the residuals of the zones handed to the queue kernel
  double* pncache = nullptr;  // P_n quantities shared by the two stages of a step
  double* Ph = nullptr;       // half-step state
  double* Pcopy = nullptr;    // copy of P_n for a stage written over P_n (allocated on first use)
  uint8_t* iters = nullptr;   // per-zone Newton updates of the last stage
  uint8_t* status = nullptr;  // per-zone status bits of the last stage
  grim::Counters* cnt = nullptr;
  double* dev_in = nullptr;   // device copies for grim_step_host
  double* dev_out = nullptr;
  unsigned long long launches = 0;
  grim_mlp* mlp = nullptr;    // learned initial guess (grim_set_guess)
  float* feat = nullptr;      // its increment features [10][N], written by the zone kernel
  float* gfeat = nullptr;     // its metric features: float copy of g_{mu nu} at zone centres (general metric)
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
  KernelMark(grim_ctx* ctx, int k, int n = 1) : c(ctx), cls(k) {
    c->launches += n;
    if (c->profile) { a = c->event(); cudaEventRecord(a, c->cur); }
  }
  ~KernelMark() {
    if (c->profile) {
      cudaEvent_t b = c->event();
      cudaEventRecord(b, c->cur);
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
  cudaFree(ctx->geo);
  cudaFree(ctx->faces);
  cudaFree(ctx->pncache);
  cudaFree(ctx->Ph);
  cudaFree(ctx->Pcopy);
  cudaFree(ctx->iters);
  cudaFree(ctx->status);
  cudaFree(ctx->cnt);
  cudaFree(ctx->dev_in);
  cudaFree(ctx->dev_out);
  cudaFree(ctx->queue);
  cudaFree(ctx->qcount);
  cudaFree(ctx->rqueue);
  cudaFree(ctx->feat);
  cudaFree(ctx->gfeat);
  for (auto& g : ctx->gcache) cudaGraphExecDestroy(g.exec);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  for (auto& m : ctx->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

int grim_init(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys, const grim_solver* solver,
              void* stream, grim_ctx** out) {
  if (!out) return GRIM_EINVAL;
  *out = nullptr;
  if (!grid || !metric || !phys || !solver) return GRIM_EINVAL;
  if (grid->dim < 2 || grid->dim > 3 || grid->n1 < 1 || grid->n2 < 1 || grid->n3 < 1) return GRIM_EINVAL;
  if (grid->dim == 2 && grid->n3 != 1) return GRIM_EINVAL;
  if (metric->kind != GRIM_METRIC_MINKOWSKI && metric->kind != GRIM_METRIC_MKS_KERR) return GRIM_EINVAL;
  if (metric->kind == GRIM_METRIC_MKS_KERR && !(std::fabs(metric->spin) < 1.0)) return GRIM_EINVAL;
  if (phys->recon != GRIM_RECON_MC && phys->recon != GRIM_RECON_WENO5 && phys->recon != GRIM_RECON_PPM)
    return GRIM_EINVAL;
  if (phys->riemann != GRIM_FLUX_LLF && phys->riemann != GRIM_FLUX_HLLE) return GRIM_EINVAL;
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
  p.metric = metric->kind; p.floors = phys->floors; p.riemann = phys->riemann;
  p.N = (long long)grid->n1 * grid->n2 * grid->n3;
  ctx->precision = solver->precision;
  ctx->gr = grid->dim == 3 || metric->kind != GRIM_METRIC_MINKOWSKI;
  ctx->stream = (cudaStream_t)stream;
  ctx->cur = ctx->stream;
  const size_t N = (size_t)p.N;
  cudaError_t e;
  if ((e = cudaMalloc(&ctx->K, sizeof(double) * grim::NK * N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->Ph, sizeof(double) * grim::NV * N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->faces, sizeof(double) * (ctx->gr ? grim::gr_face_doubles(p)
                                                              : grim::face_scratch_doubles(p.n1, p.n2)))) !=
          cudaSuccess ||
      (ctx->gr && (e = cudaMalloc(&ctx->geo, sizeof(double) * grim::gr_geometry_doubles(p))) != cudaSuccess) ||
      (e = cudaMalloc(&ctx->pncache, sizeof(double) * (ctx->gr ? grim::gr_cache_doubles(p.N)
                                                              : grim::pn_cache_doubles(p.N)))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->iters, N)) != cudaSuccess || (e = cudaMalloc(&ctx->status, N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->cnt, sizeof(grim::Counters))) != cudaSuccess ||
      (e = cudaMalloc(&ctx->queue, sizeof(int) * N)) != cudaSuccess ||
      (e = cudaMalloc(&ctx->qcount, 2 * sizeof(int))) != cudaSuccess ||
      (solver->precision == GRIM_MIXED && (e = cudaMalloc(&ctx->rqueue, sizeof(int) * N)) != cudaSuccess) ||
      (e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking)) != cudaSuccess) {
    grim_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? GRIM_ENOMEM : GRIM_ECUDA;
  }
  if ((e = cudaMemsetAsync(ctx->cnt, 0, sizeof(grim::Counters), ctx->stream)) != cudaSuccess ||
      (ctx->gr && (e = grim::launch_gr_geometry(p, metric->kind, metric->spin, metric->h, grid->x_start, ctx->geo,
                                                ctx->stream)) != cudaSuccess)) {
    grim_destroy(ctx);
    return GRIM_ECUDA;
  }
  *out = ctx;
  return GRIM_OK;
}

// The explicit part of a stage: face fluxes, then flux-CT and the constants.
static int run_explicit(grim_ctx* ctx, const double* Pn, const double* PE, double dts, const double* guess,
                        double* Pout, int mode, float* feat = nullptr) {
  if (ctx->gr) {
    {
      KernelMark m(ctx, GRIM_K_FACES, ctx->p.dim);
      GRIM_CUDA(grim::launch_gr_faces(ctx->p, PE, ctx->geo, ctx->faces, ctx->precision == GRIM_MIXED, ctx->cur), "face kernel");
    }
    KernelMark m(ctx, GRIM_K_ZONECONST, 3);
    GRIM_CUDA(grim::launch_gr_zone_const(ctx->p, Pn, PE, guess, dts, ctx->geo, ctx->faces, ctx->K, Pout,
                                         ctx->pncache, mode, feat, ctx->precision == GRIM_MIXED, ctx->cur),
              "zone-constant kernel");
    return GRIM_OK;
  }
  {
    KernelMark m(ctx, GRIM_K_FACES);
    GRIM_CUDA(grim::launch_faces(ctx->p, PE, ctx->faces, ctx->tune.faces_bs, ctx->precision == GRIM_MIXED, ctx->cur),
              "face kernel");
  }
  {
    KernelMark m(ctx, GRIM_K_ZONECONST, ctx->precision == GRIM_MIXED ? 1 : 2);
    GRIM_CUDA(grim::launch_zone_const(ctx->p, Pn, PE, guess, dts, ctx->K, Pout, ctx->faces, ctx->pncache, mode,
                                      ctx->tune.zone_bs, feat, ctx->precision == GRIM_MIXED, ctx->cur),
              "zone-constant kernel");
  }
  return GRIM_OK;
}

// The mixed solver hands the zones its float32-Jacobian iteration cannot
// solve to the float64 kernel, which starts from P_n; when the stage writes
// over P_n (an in-place full step), from P^E instead.
static grim::Rescue rescue(grim_ctx* ctx, const double* Pn, const double* PE, const double* Pout) {
  if (ctx->precision != GRIM_MIXED || !ctx->rqueue || ctx->p.kmax < 1) return grim::Rescue{nullptr, nullptr, nullptr};
  return grim::Rescue{ctx->rqueue, ctx->qcount + 1, Pout == Pn ? PE : Pn};
}

// A stage whose output is its own P_n: the start written into P_out would
// replace P_n while the learned start's fallback and the revert of failed
// zones still read it, so the stage reads a copy of P_n instead.  The copy's
// buffer is allocated here, before any capture (grim_step, grim_stage and
// grim_batch_step call this ahead of their launches).
static int ensure_copy(grim_ctx* ctx, const double* Pn, const double* Pout) {
  if (Pn != Pout || ctx->Pcopy) return GRIM_OK;
  if (cudaMalloc(&ctx->Pcopy, sizeof(double) * grim::NV * (size_t)ctx->p.N) != cudaSuccess) {
    ctx->Pcopy = nullptr;
    return fail(ctx, GRIM_ENOMEM, "copy of P_n for an in-place stage");
  }
  return GRIM_OK;
}
static int pn_of_stage(grim_ctx* ctx, const double* Pn, const double* Pout, const double** out) {
  *out = Pn;
  if (Pn != Pout) return GRIM_OK;
  GRIM_CUDA(cudaMemcpyAsync(ctx->Pcopy, Pn, sizeof(double) * grim::NV * (size_t)ctx->p.N, cudaMemcpyDeviceToDevice,
                            ctx->cur),
            "in-place copy of P_n");
  *out = ctx->Pcopy;
  return GRIM_OK;
}

static int run_stage(grim_ctx* ctx, const double* Pn, const double* PE, double dts, const double* guess,
                     double* Pout, uint8_t* iters, uint8_t* status, int mode = 0) {
  const bool learned = ctx->mlp && !guess;
  int rc = run_explicit(ctx, Pn, PE, dts, guess, Pout, mode, learned ? ctx->feat : nullptr);
  if (rc) return rc;
  if (learned) {
    // the zone-constant kernel wrote the increment features beside the constants
    KernelMark m(ctx, GRIM_K_MLP, 1);
    GRIM_CUDA(grim::launch_mlp_guess(ctx->p, ctx->feat, Pn, ctx->mlp, Pout, ctx->gfeat,
                                     &ctx->cnt->mlp_stalls, ctx->cur),
              "mlp kernel");
  }
  if (ctx->gr) {
    const grim::NewtonCfg cfg{ctx->tune.newton_bs, ctx->tune.newton_kcut, ctx->tune.newton_rounds != 0};
    {
      KernelMark m(ctx, ctx->precision ? GRIM_K_NEWTON32 : GRIM_K_NEWTON64,
                   (cfg.kcut < ctx->p.kmax ? 2 : 1) + (rescue(ctx, Pn, PE, Pout).queue ? 1 : 0));
      GRIM_CUDA(grim::launch_newton_gr(ctx->p, ctx->precision, ctx->K, ctx->geo, Pout, iters ? iters : ctx->iters,
                                       status ? status : ctx->status, ctx->cnt, cfg, ctx->queue, ctx->qcount,
                                       ctx->faces, learned ? Pn : nullptr, ctx->accept, rescue(ctx, Pn, PE, Pout),
                                       learned ? ctx->feat : nullptr, ctx->cur),
                "newton kernel");
    }
    if (ctx->p.floors) {
      KernelMark m(ctx, GRIM_K_ZONECONST);
      GRIM_CUDA(grim::launch_gr_floors(ctx->p, ctx->geo, ctx->K, Pn, status ? status : ctx->status, Pout, ctx->cur),
                "floor kernel");
    }
    return GRIM_OK;
  }
  {
    const grim::NewtonCfg cfg{ctx->tune.newton_bs, ctx->tune.newton_kcut, ctx->tune.newton_rounds != 0};
    KernelMark m(ctx, ctx->precision ? GRIM_K_NEWTON32 : GRIM_K_NEWTON64,
                 (cfg.kcut < ctx->p.kmax ? 2 : 1) + (rescue(ctx, Pn, PE, Pout).queue ? 1 : 0));
    GRIM_CUDA(grim::launch_newton_fb(ctx->p, ctx->precision, ctx->K, Pout, iters ? iters : ctx->iters,
                                     status ? status : ctx->status, ctx->cnt, learned ? Pn : nullptr, ctx->accept,
                                     cfg, ctx->queue, ctx->qcount, ctx->faces, rescue(ctx, Pn, PE, Pout),
                                     learned ? ctx->feat : nullptr, ctx->cur),
              "newton kernel");
  }
  return GRIM_OK;
}

int grim_stage(grim_ctx* ctx, const double* P_n, const double* P_E, double dts, const double* guess, double* P_out,
               unsigned char* iters, unsigned char* status) {
  if (!ctx || !P_n || !P_E || !P_out || !(dts > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_stage: bad argument");
  // other CTAs read P_E around their tiles while P_out is written
  if (P_out == P_E) return fail(ctx, GRIM_EINVAL, "grim_stage: P_out must not alias P_E");
  const double* Pn = nullptr;
  int rc = ensure_copy(ctx, P_n, P_out);
  if (!rc) rc = pn_of_stage(ctx, P_n, P_out, &Pn);
  return rc ? rc : run_stage(ctx, Pn, P_E, dts, guess, P_out, iters, status);
}

static int step_launches(grim_ctx* ctx, const double* P_in, double* P_out, double dt) {
  // The half step (P^E = P_n) caches the P_n quantities the full step reuses.
  int rc = run_stage(ctx, P_in, P_in, 0.5 * dt, nullptr, ctx->Ph, nullptr, nullptr, 1);
  if (rc) return rc;
  const double* Pn = nullptr;
  if ((rc = pn_of_stage(ctx, P_in, P_out, &Pn))) return rc;
  return run_stage(ctx, Pn, ctx->Ph, dt, nullptr, P_out, nullptr, nullptr, 2);
}

static bool same_tuning(const grim_tuning& a, const grim_tuning& b) {
  return a.newton_bs == b.newton_bs && a.newton_kcut == b.newton_kcut && a.newton_rounds == b.newton_rounds &&
         a.faces_bs == b.faces_bs &&
         a.zone_bs == b.zone_bs;
}

// Capture the step's launches on the private stream into an executable graph.
static int capture_step(grim_ctx* ctx, const double* P_in, double* P_out, double dt, grim_ctx::Graph& g) {
  GRIM_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  const unsigned long long before = ctx->launches;
  ctx->cur = ctx->cap;
  const int rc = step_launches(ctx, P_in, P_out, dt);
  ctx->cur = ctx->stream;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap, &graph);
  g.kernels = ctx->launches - before;
  ctx->launches = before;
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e != cudaSuccess) return fail(ctx, GRIM_ECUDA, "end capture", e);
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(ctx, GRIM_ECUDA, "graph instantiate", ei);
  g.in = P_in; g.out = P_out; g.dt = dt; g.mlp = ctx->mlp; g.accept = ctx->accept; g.tune = ctx->tune;
  return GRIM_OK;
}

int grim_step(grim_ctx* ctx, const double* P_in, double* P_out, double dt) {
  if (!ctx || !P_in || !P_out || !(dt > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_step: bad argument");
  if (const int rc = ensure_copy(ctx, P_in, P_out)) return rc;
  if (!ctx->graphs || ctx->profile || !ctx->warmed || !same_tuning(ctx->warm_tune, ctx->tune) ||
      ctx->warm_mlp != (ctx->mlp != nullptr)) {
    const int rc = step_launches(ctx, P_in, P_out, dt);
    if (!rc) { ctx->warmed = true; ctx->warm_tune = ctx->tune; ctx->warm_mlp = ctx->mlp != nullptr; }
    return rc;
  }
  grim_ctx::Graph* hit = nullptr;
  for (auto& g : ctx->gcache)
    if (g.in == P_in && g.out == P_out && g.dt == dt && g.mlp == ctx->mlp && g.accept == ctx->accept &&
        same_tuning(g.tune, ctx->tune))
      hit = &g;
  if (!hit) {
    grim_ctx::Graph g{};
    const int rc = capture_step(ctx, P_in, P_out, dt, g);
    if (rc) return rc;
    if (ctx->gcache.size() >= 4) {  // drop the least recently used
      auto lru = std::min_element(ctx->gcache.begin(), ctx->gcache.end(),
                                  [](const grim_ctx::Graph& a, const grim_ctx::Graph& b) { return a.last < b.last; });
      cudaGraphExecDestroy(lru->exec);
      ctx->gcache.erase(lru);
    }
    ctx->gcache.push_back(g);
    hit = &ctx->gcache.back();
  }
  hit->last = ++ctx->gclock;
  GRIM_CUDA(cudaGraphLaunch(hit->exec, ctx->stream), "graph launch");
  ctx->launches += hit->kernels;
  return GRIM_OK;
}

int grim_use_graphs(grim_ctx* ctx, int enable) {
  if (!ctx) return GRIM_EINVAL;
  ctx->graphs = enable != 0;
  return GRIM_OK;
}

static bool valid_tuning(const grim_tuning& t) {
  auto in = [](int v, std::initializer_list<int> s) { return std::find(s.begin(), s.end(), v) != s.end(); };
  return in(t.newton_bs, {32, 64, 128}) && t.newton_kcut >= 1 && in(t.newton_rounds, {0, 1}) &&
         in(t.faces_bs, {64, 128, 256}) &&
         in(t.zone_bs, {64, 128, 256});
}

int grim_get_tuning(grim_ctx* ctx, grim_tuning* out) {
  if (!ctx || !out) return GRIM_EINVAL;
  *out = ctx->tune;
  return GRIM_OK;
}

int grim_set_tuning(grim_ctx* ctx, const grim_tuning* t) {
  if (!ctx || !t || !valid_tuning(*t)) return fail(ctx, GRIM_EINVAL, "grim_set_tuning: value outside the allowed set");
  ctx->tune = *t;
  return GRIM_OK;
}

// Key of a tuning-cache line: what the launch shapes depend on.
static std::string tuning_key(grim_ctx* ctx) {
  int dev = 0;
  cudaDeviceProp prop;
  cudaGetDevice(&dev);
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) prop.name[0] = 0;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|%dx%dx%d|prec%d|recon%d|cond%d|visc%d|ho%d|mlp%d|kmax%d", prop.name, ctx->p.n1,
           ctx->p.n2, ctx->p.n3, ctx->precision, ctx->p.recon, ctx->p.cond, ctx->p.visc, ctx->p.ho,
           ctx->mlp ? 1 : 0, ctx->p.kmax);
  for (char* c = buf; *c; c++)
    if (*c == '"' || *c == '\\') *c = '_';
  return buf;
}

static bool read_cached_tuning(const char* path, const std::string& key, grim_tuning& t, double& ms) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  const std::string tag = "\"key\": \"" + key + "\"";
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    if (!std::strstr(line, tag.c_str())) continue;
    const char* q = std::strstr(line, "\"newton_bs\":");
    grim_tuning c;
    double m = 0.0;
    if (q && std::sscanf(q, "\"newton_bs\": %d, \"newton_kcut\": %d, \"newton_rounds\": %d, \"faces_bs\": %d, \"zone_bs\": %d, \"step_ms\": %lf",
                         &c.newton_bs, &c.newton_kcut, &c.newton_rounds, &c.faces_bs, &c.zone_bs, &m) == 6 &&
        valid_tuning(c)) {
      t = c; ms = m; found = true;
    }
  }
  std::fclose(f);
  return found;
}

static void write_cached_tuning(const char* path, const std::string& key, const grim_tuning& t, double ms) {
  std::vector<std::string> keep;
  const std::string tag = "\"key\": \"" + key + "\"";
  if (FILE* f = std::fopen(path, "r")) {
    char line[1024];
    while (std::fgets(line, sizeof(line), f))
      if (!std::strstr(line, tag.c_str()) && line[0] == '{') keep.push_back(line);
    std::fclose(f);
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (auto& l : keep) std::fputs(l.c_str(), f);
  std::fprintf(f, "{%s, \"newton_bs\": %d, \"newton_kcut\": %d, \"newton_rounds\": %d, \"faces_bs\": %d, \"zone_bs\": %d, \"step_ms\": %.6f}\n",
               tag.c_str(), t.newton_bs, t.newton_kcut, t.newton_rounds, t.faces_bs, t.zone_bs, ms);
  std::fclose(f);
}

// Median of 3 timed steps after one warm-up step, eagerly launched.
static int time_steps(grim_ctx* ctx, const double* P, double* out, double dt, double& ms) {
  cudaEvent_t a = ctx->event(), b = ctx->event();
  float t[5];
  int rc = step_launches(ctx, P, out, dt);
  for (int i = 0; i < 5 && !rc; i++) {
    cudaEventRecord(a, ctx->stream);
    rc = step_launches(ctx, P, out, dt);
    cudaEventRecord(b, ctx->stream);
    if (!rc && cudaEventSynchronize(b) != cudaSuccess) rc = fail(ctx, GRIM_ECUDA, "autotune timing");
    if (!rc) cudaEventElapsedTime(&t[i], a, b);
  }
  ctx->pool.push_back(a);
  ctx->pool.push_back(b);
  if (rc) return rc;
  std::sort(t, t + 5);
  ms = t[2];
  return GRIM_OK;
}

int grim_autotune(grim_ctx* ctx, const double* P, double dt, const char* cache_path, grim_tuning* out,
                  double* step_ms) {
  if (!ctx || !P || !(dt > 0.0)) return fail(ctx, GRIM_EINVAL, "grim_autotune: bad argument");
  const std::string key = tuning_key(ctx);
  grim_tuning best = ctx->tune;
  double best_ms = 0.0;
  if (!(cache_path && read_cached_tuning(cache_path, key, best, best_ms))) {
    double* out_state = nullptr;
    cudaError_t e = cudaMalloc(&out_state, sizeof(double) * grim::NV * (size_t)ctx->p.N);
    if (e != cudaSuccess) return fail(ctx, GRIM_ENOMEM, "grim_autotune: scratch state", e);
    const bool prof = ctx->profile;
    ctx->profile = false;
    int rc = time_steps(ctx, P, out_state, dt, best_ms);
    const int kmax = ctx->p.kmax;
    const std::vector<int> sets[5] = {{32, 64, 128}, {0, 1}, {1, 2, 3, 4, kmax > 4 ? kmax : 5}, {64, 128, 256},
                                      {64, 128, 256}};
    // two passes of coordinate descent: the second revisits each field
    // after the others have moved
    for (int f = 0; f < 10 && !rc; f++) {
      for (int v : sets[f % 5]) {
        grim_tuning c = best;
        const int fi = f % 5;
        int* field = fi == 0 ? &c.newton_bs : fi == 1 ? &c.newton_rounds : fi == 2 ? &c.newton_kcut
                   : fi == 3 ? &c.faces_bs : &c.zone_bs;
        if (*field == v) continue;
        *field = v;
        ctx->tune = c;
        double ms = 0.0;
        rc = time_steps(ctx, P, out_state, dt, ms);
        if (rc) break;
        if (ms < best_ms) { best_ms = ms; best = c; }
      }
    }
    ctx->profile = prof;
    cudaFree(out_state);
    if (rc) { ctx->tune = best; return rc; }
    if (cache_path) write_cached_tuning(cache_path, key, best, best_ms);
  }
  ctx->tune = best;
  if (out) *out = best;
  if (step_ms) *step_ms = best_ms;
  GRIM_CUDA(cudaMemsetAsync(ctx->cnt, 0, sizeof(grim::Counters), ctx->stream), "stats reset");
  GRIM_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return GRIM_OK;
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
    if (ctx->gr)
      GRIM_CUDA(grim::launch_residual_gr(ctx->p, ctx->K, ctx->geo, P_k, scaled, dts, R_out, ctx->stream),
                "residual kernel");
    else
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
  out->rescued = c.rescued;
  out->mlp_stalls = c.mlp_stalls;
  return GRIM_OK;
}

int grim_set_guess(grim_ctx* ctx, grim_mlp* mlp, double accept) {
  if (!ctx || !(accept >= 0.0)) return GRIM_EINVAL;
  if (mlp && !ctx->feat) {
    const cudaError_t e = cudaMalloc(&ctx->feat, sizeof(float) * grim::NV * (size_t)ctx->p.N);
    if (e != cudaSuccess) return fail(ctx, GRIM_ENOMEM, "grim_set_guess: feature buffer", e);
  }
  if (mlp && ctx->gr && !ctx->gfeat) {
    cudaError_t e = cudaMalloc(&ctx->gfeat, sizeof(float) * 10 * (size_t)(ctx->p.n1 + 2) * (ctx->p.n2 + 2));
    if (e != cudaSuccess) {
      ctx->gfeat = nullptr;
      return fail(ctx, GRIM_ENOMEM, "grim_set_guess: metric features", e);
    }
    if ((e = grim::launch_mlp_metric_table(ctx->p, ctx->geo, ctx->gfeat, ctx->stream)) != cudaSuccess)
      return fail(ctx, GRIM_ECUDA, "grim_set_guess: metric features", e);
  }
  ctx->mlp = mlp;
  ctx->accept = accept;
  return GRIM_OK;
}

int grim_mlp_sample(grim_ctx* ctx, const double* P_n, const double* P_conv, float* X, float* Y) {
  if (!ctx || !P_n || !X || (Y && !P_conv)) return GRIM_EINVAL;
  {
    KernelMark m(ctx, GRIM_K_MLP);
    if (ctx->gr)
      GRIM_CUDA(grim::launch_features_gr(ctx->p, ctx->K, ctx->geo, P_n, P_conv, X, Y, nullptr, ctx->stream),
                "feature kernel");
    else
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

// ---------------------------------------------------------------- batched boxes
// Independent boxes of any sizes stepped together: one context per box, the
// boxes' launch sequences spread round-robin over side streams forked from
// the caller's stream (so small boxes run concurrently), the whole step
// replayed as one CUDA graph once captured.
struct grim_batch {
  std::vector<grim_ctx*> box;
  cudaStream_t stream = nullptr;           // the caller's stream
  cudaStream_t cap = nullptr;              // capture origin
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;             // fork event + one join event per side stream
  bool graphs = true, warmed = false;
  struct Graph {
    std::vector<const double*> in; std::vector<double*> out; std::vector<double> dt;
    cudaGraphExec_t exec = nullptr; unsigned long long kernels = 0, last = 0;
  };
  std::vector<Graph> gcache;
  unsigned long long clock = 0, launches = 0;
  char err[256] = {0};
};

static int batch_fail(grim_batch* b, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (b) snprintf(b->err, sizeof(b->err), "%s%s%s", what, e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
  return code;
}

void grim_batch_destroy(grim_batch* b) {
  if (!b) return;
  for (auto c : b->box) grim_destroy(c);
  for (auto& g : b->gcache) cudaGraphExecDestroy(g.exec);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->ev) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

int grim_batch_init(int nbox, const grim_grid* grids, const grim_metric* metric, const grim_physics* phys,
                    const grim_solver* solver, void* stream, grim_batch** out) {
  if (!out) return GRIM_EINVAL;
  *out = nullptr;
  if (nbox < 1 || !grids) return GRIM_EINVAL;
  grim_batch* b = new grim_batch();
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < nbox; i++) {
    grim_ctx* c = nullptr;
    const int rc = grim_init(&grids[i], metric, phys, solver, stream, &c);
    if (rc) { grim_batch_destroy(b); return rc; }
    b->box.push_back(c);
  }
  const int ns = nbox < 16 ? nbox : 16;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int i = 0; i < ns && e == cudaSuccess; i++) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->side.push_back(s);
  }
  for (int i = 0; i <= ns && e == cudaSuccess; i++) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev.push_back(ev);
  }
  if (e != cudaSuccess) { grim_batch_destroy(b); return GRIM_ECUDA; }
  *out = b;
  return GRIM_OK;
}

int grim_batch_context(grim_batch* b, int i, grim_ctx** out) {
  if (!b || !out || i < 0 || i >= (int)b->box.size()) return GRIM_EINVAL;
  *out = b->box[i];
  return GRIM_OK;
}

int grim_batch_use_graphs(grim_batch* b, int enable) {
  if (!b) return GRIM_EINVAL;
  b->graphs = enable != 0;
  return GRIM_OK;
}

// Fork from `origin` onto the side streams, launch every box, join back.
static int batch_launches(grim_batch* b, cudaStream_t origin, const double* const* P_in, double* const* P_out,
                          const double* dt, unsigned long long& kernels) {
  const int ns = (int)b->side.size();
  cudaError_t e = cudaEventRecord(b->ev[0], origin);
  for (int s = 0; s < ns && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->side[s], b->ev[0], 0);
  if (e != cudaSuccess) return batch_fail(b, GRIM_ECUDA, "batch fork", e);
  int rc = GRIM_OK;
  kernels = 0;
  for (size_t i = 0; i < b->box.size() && !rc; i++) {
    grim_ctx* c = b->box[i];
    c->cur = b->side[i % ns];
    const unsigned long long before = c->launches;
    rc = step_launches(c, P_in[i], P_out[i], dt[i]);
    kernels += c->launches - before;
    c->cur = c->stream;
    if (rc) batch_fail(b, rc, c->err);
  }
  for (int s = 0; s < ns; s++) {
    cudaError_t e1 = cudaEventRecord(b->ev[1 + s], b->side[s]);
    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(origin, b->ev[1 + s], 0);
    if (e1 != cudaSuccess && !rc) rc = batch_fail(b, GRIM_ECUDA, "batch join", e1);
  }
  return rc;
}

int grim_batch_step(grim_batch* b, const double* const* P_in, double* const* P_out, const double* dt) {
  if (!b || !P_in || !P_out || !dt) return GRIM_EINVAL;
  const size_t n = b->box.size();
  for (size_t i = 0; i < n; i++)
    if (!P_in[i] || !P_out[i] || !(dt[i] > 0.0)) return batch_fail(b, GRIM_EINVAL, "grim_batch_step: bad argument");
  for (size_t i = 0; i < n; i++)
    if (const int rc = ensure_copy(b->box[i], P_in[i], P_out[i])) return batch_fail(b, rc, b->box[i]->err);
  bool profiling = false;
  for (auto c : b->box) profiling = profiling || c->profile;
  if (!b->graphs || !b->warmed || profiling) {
    unsigned long long k = 0;
    const int rc = batch_launches(b, b->stream, P_in, P_out, dt, k);
    b->launches += k;
    if (!rc) b->warmed = true;
    return rc;
  }
  grim_batch::Graph* hit = nullptr;
  for (auto& g : b->gcache) {
    bool same = true;
    for (size_t i = 0; i < n && same; i++) same = g.in[i] == P_in[i] && g.out[i] == P_out[i] && g.dt[i] == dt[i];
    if (same) hit = &g;
  }
  if (!hit) {
    grim_batch::Graph g;
    g.in.assign(P_in, P_in + n);
    g.out.assign(P_out, P_out + n);
    g.dt.assign(dt, dt + n);
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, GRIM_ECUDA, "begin capture", e);
    const int rc = batch_launches(b, b->cap, P_in, P_out, dt, g.kernels);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return batch_fail(b, GRIM_ECUDA, "end capture", e);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return batch_fail(b, GRIM_ECUDA, "graph instantiate", e);
    if (b->gcache.size() >= 2) {
      auto lru = std::min_element(b->gcache.begin(), b->gcache.end(),
                                  [](const grim_batch::Graph& x, const grim_batch::Graph& y) { return x.last < y.last; });
      cudaGraphExecDestroy(lru->exec);
      b->gcache.erase(lru);
    }
    b->gcache.push_back(g);
    hit = &b->gcache.back();
  }
  hit->last = ++b->clock;
  cudaError_t e = cudaGraphLaunch(hit->exec, b->stream);
  if (e != cudaSuccess) return batch_fail(b, GRIM_ECUDA, "graph launch", e);
  b->launches += hit->kernels;
  return GRIM_OK;
}

int grim_batch_get_stats(grim_batch* b, grim_stats* out) {
  if (!b || !out) return GRIM_EINVAL;
  grim_stats t;
  std::memset(&t, 0, sizeof(t));
  for (auto c : b->box) {
    grim_stats s;
    const int rc = grim_get_stats(c, &s);
    if (rc) return rc;
    t.zones += s.zones; t.failed += s.failed; t.iters += s.iters;
    t.evals64 += s.evals64; t.evals32 += s.evals32; t.lu64 += s.lu64; t.lu32 += s.lu32;
    for (int i = 0; i < 32; i++) t.hist[i] += s.hist[i];
    t.max_res = std::max(t.max_res, s.max_res);
    t.fallbacks += s.fallbacks;
    t.rescued += s.rescued;
    t.mlp_stalls += s.mlp_stalls;
  }
  t.launches = b->launches;
  *out = t;
  return GRIM_OK;
}

int grim_batch_reset_stats(grim_batch* b) {
  if (!b) return GRIM_EINVAL;
  for (auto c : b->box) {
    const int rc = grim_reset_stats(c);
    if (rc) return rc;
  }
  return GRIM_OK;
}

const char* grim_batch_last_error(grim_batch* b) { return b ? b->err : "no batch"; }

}  // extern "C"
