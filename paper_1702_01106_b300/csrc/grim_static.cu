// grim_step_static: one time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: host applications that own every byte
// of device memory through their own pool allocator, and loops that must not
// allocate after start-up because cudaMalloc can synchronise the device.
// This entry point serves them: its scratch (the per-zone stage constants,
// the half-step state, the per-zone status bytes and the counters) lives in
// one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.  The caller still passes the
// input and output states.
#include <cstring>
#include <mutex>

#include "grim_dev.cuh"
#include "../../include/grim.h"

namespace grim {
cudaError_t launch_explicit(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                            double* K, double* P0, cudaStream_t st);
cudaError_t launch_newton(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                          Counters* cnt, cudaStream_t st);
}  // namespace grim

namespace {

constexpr long long kMaxZones = GRIM_STATIC_MAX_ZONES;
constexpr long long kOffPh = (long long)grim::NK * kMaxZones;                   // half-step state
constexpr long long kOffCnt = kOffPh + (long long)grim::NV * kMaxZones;         // counters
constexpr long long kCntDoubles = (sizeof(grim::Counters) + 255) / 256 * 32;  // 256-byte rounded
constexpr long long kOffBytes = kOffCnt + kCntDoubles;                          // iters, status bytes
constexpr long long kTotal = kOffBytes + (2 * kMaxZones + 7) / 8;

// The scratch.  In host code this name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_scratch[kTotal];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up on the first
// call for that device (with that device current).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

int make_params(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys,
                const grim_solver* solver, grim::Params& p) {
  if (!grid || !metric || !phys || !solver) return GRIM_EINVAL;
  if (grid->dim != 2 || grid->n3 != 1 || grid->n1 < 1 || grid->n2 < 1) return GRIM_EINVAL;
  if (metric->kind != GRIM_METRIC_MINKOWSKI) return GRIM_EINVAL;
  if (phys->recon != GRIM_RECON_MC && phys->recon != GRIM_RECON_WENO5) return GRIM_EINVAL;
  if (phys->riemann != GRIM_FLUX_LLF) return GRIM_EINVAL;  // the tile kernel has the LLF flux only
  if (solver->precision != GRIM_FP64 && solver->precision != GRIM_MIXED) return GRIM_EINVAL;
  if (!(phys->gamma > 1.0) || !(phys->tau_R > 0.0) || !(solver->tol > 0.0) || solver->k_max < 0 ||
      solver->k_max > 250 || solver->ls_max < 0)
    return GRIM_EINVAL;
  for (int d = 0; d < 3; d++)
    for (int s = 0; s < 2; s++)
      if (grid->bc[d][s] < 0 || grid->bc[d][s] > 2) return GRIM_EINVAL;
  if ((long long)grid->n1 * grid->n2 > kMaxZones) return GRIM_ESIZE;
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
  return GRIM_OK;
}

}  // namespace

extern "C" int grim_step_static(const grim_grid* grid, const grim_metric* metric, const grim_physics* phys,
                                const grim_solver* solver, void* stream, const double* P_in, double* P_out,
                                double dt) {
  grim::Params p;
  int rc = make_params(grid, metric, phys, solver, p);
  if (rc) return rc;
  if (!P_in || !P_out || !(dt > 0.0)) return GRIM_EINVAL;
  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return GRIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  double* K = base;
  double* Ph = base + kOffPh;
  grim::Counters* cnt = (grim::Counters*)(base + kOffCnt);
  uint8_t* iters = (uint8_t*)(base + kOffBytes);
  uint8_t* status = iters + kMaxZones;
  // the counters accumulate atomically: start each call from zero
  if (cudaMemsetAsync(cnt, 0, sizeof(grim::Counters), st) != cudaSuccess) return GRIM_ECUDA;
  const int mixed = solver->precision;
  if (grim::launch_explicit(p, P_in, P_in, nullptr, 0.5 * dt, K, Ph, st) != cudaSuccess) return GRIM_ECUDA;
  if (grim::launch_newton(p, mixed, K, Ph, iters, status, cnt, st) != cudaSuccess) return GRIM_ECUDA;
  if (grim::launch_explicit(p, P_in, Ph, nullptr, dt, K, P_out, st) != cudaSuccess) return GRIM_ECUDA;
  if (grim::launch_newton(p, mixed, K, P_out, iters, status, cnt, st) != cudaSuccess) return GRIM_ECUDA;
  return GRIM_OK;
}

extern "C" int grim_step_static_stats(void* stream, grim_stats* out) {
  if (!out) return GRIM_EINVAL;
  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return GRIM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  grim::Counters c;
  if (cudaMemcpyAsync(&c, base + kOffCnt, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GRIM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GRIM_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->zones = c.zones; out->failed = c.failed; out->iters = c.iters;
  out->evals64 = c.evals64; out->evals32 = c.evals32; out->lu64 = c.lu64; out->lu32 = c.lu32;
  for (int i = 0; i < 32; i++) out->hist[i] = c.hist[i];
  const long long bits = (long long)c.maxres_bits;
  std::memcpy(&out->max_res, &bits, sizeof(bits));
  out->launches = 4;
  return GRIM_OK;
}
