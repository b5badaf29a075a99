// Per-zone Newton solve of the stage residual (Section 3): FD Jacobian
// (Section 3.1), 10x10 partial-pivot LU, quadratic backtracking line search
// (Section 3.2), convergence test max_a |r_a| <= tol before each Jacobian.
//
// One thread owns one zone.  The Jacobian and right-hand side live in shared
// memory (stride = block size, so a warp's accesses are conflict-free); the
// state, the residual and the zone constants live in registers.
//
// Precision variants:
//   FP64  -- everything in double.
//   MIXED -- the Jacobian (its 11 residual evaluations) and the LU in float;
//            the residual of the iterate, the update, the line search and the
//            convergence test in double (inexact Newton).
#include "grim_dev.cuh"

namespace grim {

// Scaled residual r(P) of one zone from its constants kk (see grim_dev.cuh).
template <typename T>
__device__ __forceinline__ void zone_residual(const T* P, const T* kk, const Params& p, T* r) {
  Pt<T> s;
  point_state(P, p, s);
  T row[4];
  stress_row(s, 0, row);
  T U[NV];
  U[0] = s.rho * s.ut;
  U[1] = row[0]; U[2] = row[1]; U[3] = row[2]; U[4] = row[3];
  U[5] = P[5]; U[6] = P[6]; U[7] = P[7];
  U[8] = s.qt * s.ut;
  U[9] = s.dpt * s.ut;
#pragma unroll
  for (int a = 0; a < NV; a++) r[a] = kk[K_U + a] * U[a] + kk[K_C + a];
  const T ul[4] = {-s.ut, s.uc[0], s.uc[1], s.uc[2]};
  T e8 = kk[K_Q + 0] * s.qt + kk[K_Q + 1] * s.theta + kk[K_Q + 6] * s.ut;
  T e9 = kk[K_D + 0] * s.dpt + kk[K_D + 5] * s.ut;
#pragma unroll
  for (int m = 0; m < 4; m++) {
    e8 += kk[K_Q + 2 + m] * ul[m];
    e9 += kk[K_D + 1 + m] * ul[m];
  }
  r[8] += e8;
  r[9] += e9;
}

// Perturbed component of the FD Jacobian (Section 3.1): (1 + eps) x, or
// x + eps when |x| < 5 eps (small() read as an absolute step, so the divisor
// never approaches zero).
template <typename T> __device__ __forceinline__ T fd_step(T x, T eps) {
  return (fabs(x) < T(5) * eps) ? x + eps : (T(1) + eps) * x;
}

// Partial-pivot LU solve J x = b with J, b in shared memory at stride BS
// (element (i,j) at J[(i*10+j)*BS], b[i] at b[i*BS]); x returned in registers.
// Pivot: largest |a_ik|, lowest row on ties.  Returns false on a zero pivot.
template <typename T, int BS>
__device__ __forceinline__ bool lu_solve_smem(T* J, T* b, T x[NV]) {
#pragma unroll
  for (int k = 0; k < NV; k++) {
    int piv = k;
    T best = fabs(J[(k * NV + k) * BS]);
#pragma unroll
    for (int i = k + 1; i < NV; i++) {
      T a = fabs(J[(i * NV + k) * BS]);
      if (a > best) { best = a; piv = i; }
    }
    if (!(best > T(0))) return false;
    if (piv != k) {
#pragma unroll
      for (int c = k; c < NV; c++) {
        T t = J[(k * NV + c) * BS];
        J[(k * NV + c) * BS] = J[(piv * NV + c) * BS];
        J[(piv * NV + c) * BS] = t;
      }
      T t = b[k * BS];
      b[k * BS] = b[piv * BS];
      b[piv * BS] = t;
    }
    const T inv = T(1) / J[(k * NV + k) * BS];
    const T bk = b[k * BS];
#pragma unroll
    for (int i = k + 1; i < NV; i++) {
      const T l = J[(i * NV + k) * BS] * inv;
#pragma unroll
      for (int c = k + 1; c < NV; c++) J[(i * NV + c) * BS] -= l * J[(k * NV + c) * BS];
      b[i * BS] -= l * bk;
    }
  }
#pragma unroll
  for (int i = NV - 1; i >= 0; i--) {
    T acc = b[i * BS];
#pragma unroll
    for (int c = i + 1; c < NV; c++) acc -= J[(i * NV + c) * BS] * x[c];
    x[i] = acc / J[(i * NV + i) * BS];
  }
  return true;
}

__device__ __forceinline__ double max_abs10(const double* r) {
  double m = 0.0;
#pragma unroll
  for (int a = 0; a < NV; a++) m = fmax(m, fabs(r[a]));
  return m;
}
__device__ __forceinline__ double sum_sq10(const double* r) {
  double f = 0.0;
#pragma unroll
  for (int a = 0; a < NV; a++) f += r[a] * r[a];
  return f;
}

struct ZoneResult {
  int iters, status, evals64, evals32, lu64, lu32;
  double res;
};

// Newton on one zone, starting from P (updated in place).
template <bool MIXED, int BS>
__device__ __forceinline__ ZoneResult newton_zone(const Params& p, const double* kk, double P[NV], void* smem_v) {
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0.0};
  double r[NV];
  zone_residual<double>(P, kk, p, r);
  o.evals64++;
  double f = sum_sq10(r);
  float kf[NK];
  if (MIXED) {
#pragma unroll
    for (int a = 0; a < NK; a++) kf[a] = (float)kk[a];
  }
  int k = 0;
  for (;;) {
    if (!isfinite(f)) { o.status |= ST_NONFINITE; break; }
    if (max_abs10(r) <= p.tol) break;
    if (k >= p.kmax) { o.status |= ST_MAXIT; break; }
    double dP[NV];
    bool ok;
    if (!MIXED) {
      double* J = (double*)smem_v + threadIdx.x;
      double* b = J + NV * NV * BS;
#pragma unroll 1
      for (int j = 0; j < NV; j++) {
        double Pe[NV];
#pragma unroll
        for (int a = 0; a < NV; a++) Pe[a] = P[a];
        // select component j without dynamic register indexing
        double pj = 0.0;
#pragma unroll
        for (int a = 0; a < NV; a++) if (a == j) pj = P[a];
        const double pe = fd_step(pj, p.eps64);
#pragma unroll
        for (int a = 0; a < NV; a++) if (a == j) Pe[a] = pe;
        double re[NV];
        zone_residual<double>(Pe, kk, p, re);
        const double ih = 1.0 / (pe - pj);
#pragma unroll
        for (int i = 0; i < NV; i++) J[(i * NV + j) * BS] = (re[i] - r[i]) * ih;
      }
      o.evals64 += NV;
#pragma unroll
      for (int i = 0; i < NV; i++) b[i * BS] = -r[i];
      ok = lu_solve_smem<double, BS>(J, b, dP);
      o.lu64++;
    } else {
      float* J = (float*)smem_v + threadIdx.x;
      float* b = J + NV * NV * BS;
      float Pf[NV], rf[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pf[a] = (float)P[a];
      zone_residual<float>(Pf, kf, p, rf);
#pragma unroll 1
      for (int j = 0; j < NV; j++) {
        float Pe[NV];
#pragma unroll
        for (int a = 0; a < NV; a++) Pe[a] = Pf[a];
        float pj = 0.0f;
#pragma unroll
        for (int a = 0; a < NV; a++) if (a == j) pj = Pf[a];
        const float pe = fd_step(pj, p.eps32);
#pragma unroll
        for (int a = 0; a < NV; a++) if (a == j) Pe[a] = pe;
        float re[NV];
        zone_residual<float>(Pe, kf, p, re);
        const float ih = 1.0f / (pe - pj);
#pragma unroll
        for (int i = 0; i < NV; i++) J[(i * NV + j) * BS] = (re[i] - rf[i]) * ih;
      }
      o.evals32 += NV + 1;
#pragma unroll
      for (int i = 0; i < NV; i++) b[i * BS] = (float)(-r[i]);
      float df[NV];
      ok = lu_solve_smem<float, BS>(J, b, df);
#pragma unroll
      for (int i = 0; i < NV; i++) dP[i] = (double)df[i];
      o.lu32++;
    }
    if (!ok) { o.status |= ST_SINGULAR; break; }
    // quadratic backtracking line search on f = |r|^2
    double lam = 1.0, Pt[NV], rt[NV], ft = 0.0;
    for (int t = 0;; t++) {
#pragma unroll
      for (int a = 0; a < NV; a++) Pt[a] = P[a] + lam * dP[a];
      zone_residual<double>(Pt, kk, p, rt);
      o.evals64++;
      ft = sum_sq10(rt);
      const bool fin = isfinite(ft);
      const double lim = 1.0 - 1e-4 * lam;
      if (fin && ft < f * lim * lim) break;
      if (t >= p.lsmax) { o.status |= ST_LSSTALL; break; }
      lam = fin ? f * lam * lam / (ft + (2.0 * lam - 1.0) * f) : 0.5 * lam;
    }
#pragma unroll
    for (int a = 0; a < NV; a++) { P[a] = Pt[a]; r[a] = rt[a]; }
    f = ft;
    k++;
  }
  o.iters = k;
  o.res = max_abs10(r);
  if (!(P[0] > 0.0) || !(P[1] > 0.0)) o.status |= ST_INADMISSIBLE;
  return o;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void accumulate(Counters* c, const ZoneResult& o, bool active) {
  const int lane = threadIdx.x & 31;
  unsigned long long e64 = active ? o.evals64 : 0, e32 = active ? o.evals32 : 0;
  unsigned long long l64 = active ? o.lu64 : 0, l32 = active ? o.lu32 : 0;
  unsigned long long it = active ? o.iters : 0, fl = (active && o.status) ? 1 : 0, zn = active ? 1 : 0;
  e64 = warp_sum(e64); e32 = warp_sum(e32); l64 = warp_sum(l64); l32 = warp_sum(l32);
  it = warp_sum(it); fl = warp_sum(fl); zn = warp_sum(zn);
  if (lane == 0 && zn) {
    atomicAdd(&c->evals64, e64); atomicAdd(&c->evals32, e32);
    atomicAdd(&c->lu64, l64); atomicAdd(&c->lu32, l32);
    atomicAdd(&c->iters, it); atomicAdd(&c->failed, fl); atomicAdd(&c->zones, zn);
  }
  if (active) {
    atomicAdd(&c->hist[o.iters < 31 ? o.iters : 31], 1ull);
    if (isfinite(o.res)) atomicMax(&c->maxres_bits, (unsigned long long)__double_as_longlong(o.res));
  }
}

template <bool MIXED, int BS>
__global__ void __launch_bounds__(BS) newton_dense(const __grid_constant__ Params p, const double* __restrict__ K,
                                                   double* __restrict__ P, uint8_t* __restrict__ iters,
                                                   uint8_t* __restrict__ status, Counters* __restrict__ cnt) {
  extern __shared__ double smem[];
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * BS + threadIdx.x;
  const bool active = z < N;
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0.0};
  if (active) {
    double kk[NK], Pz[NV];
#pragma unroll
    for (int a = 0; a < NK; a++) kk[a] = __ldg(K + a * N + z);
#pragma unroll
    for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z];
    o = newton_zone<MIXED, BS>(p, kk, Pz, smem);
#pragma unroll
    for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
    iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
    status[z] = (uint8_t)o.status;
  }
  accumulate(cnt, o, active);
}

// Evaluate the scaled (or raw) residual at Pk once per zone.
__global__ void residual_once(const __grid_constant__ Params p, const double* __restrict__ K,
                              const double* __restrict__ Pk, int scaled, double dts, double* __restrict__ R) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  double kk[NK], Pz[NV], r[NV];
#pragma unroll
  for (int a = 0; a < NK; a++) kk[a] = __ldg(K + a * N + z);
#pragma unroll
  for (int a = 0; a < NV; a++) Pz[a] = Pk[a * N + z];
  zone_residual<double>(Pz, kk, p, r);
#pragma unroll
  for (int a = 0; a < NV; a++) {
    // the row scale is kU * dt_s; divide it out for the raw residual
    R[a * N + z] = scaled ? r[a] : r[a] / (kk[K_U + a] * dts);
  }
}

template <bool MIXED, int BS>
static cudaError_t launch_newton_t(const Params& p, const double* K, double* P, uint8_t* iters, uint8_t* status,
                                   Counters* cnt, cudaStream_t st) {
  const size_t elem = MIXED ? sizeof(float) : sizeof(double);
  const size_t bytes = elem * (NV * NV + NV) * BS;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(newton_dense<MIXED, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long nb = (p.N + BS - 1) / BS;
  newton_dense<MIXED, BS><<<(unsigned)nb, BS, bytes, st>>>(p, K, P, iters, status, cnt);
  return cudaGetLastError();
}

cudaError_t launch_newton(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                          Counters* cnt, cudaStream_t st) {
  if (mixed) return launch_newton_t<true, 128>(p, K, P, iters, status, cnt, st);
  return launch_newton_t<false, 64>(p, K, P, iters, status, cnt, st);
}

cudaError_t launch_residual(const Params& p, const double* K, const double* Pk, int scaled, double dts, double* R,
                            cudaStream_t st) {
  const int bs = 128;
  const long long nb = (p.N + bs - 1) / bs;
  residual_once<<<(unsigned)nb, bs, 0, st>>>(p, K, Pk, scaled, dts, R);
  return cudaGetLastError();
}

}  // namespace grim
