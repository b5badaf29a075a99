// Device-side definitions shared by the grim CUDA kernels (sm_103a).
//
// The implicit zone step of Chandra, Foucart & Gammie (2017) for the
// 10-field extended GRMHD system (Minkowski space here; the general-metric
// definitions are in grim_gr.cuh).  Fields, in order:
// rho, u, u^1, u^2, u^3, B^1, B^2, B^3, q~, dP~ (q~, dP~ are the rescaled
// heat flux and pressure anisotropy of Section 4, Eqs. q and dP).
// State arrays are structure-of-arrays float64 [10][n3][n2][n1], X1 fastest.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace grim {

// One-time set-up per device, safe between host threads.  Kernel attributes
// (the dynamic shared-memory limit) and occupancy-derived grid sizes belong
// to a device, so each is set up once for every device that launches the
// kernel: the first call with a device current runs f(&value) under a lock
// and keeps value; a failing f is tried again on the next call.
struct PerDevice {
  static constexpr int kMaxDevices = 64;
  std::mutex m;
  bool done[kMaxDevices] = {};
  int value[kMaxDevices] = {};
  template <class F> cudaError_t get(F f, int* out = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(m);
    if (!done[dev]) {
      int v = 0;
      if ((e = f(&v)) != cudaSuccess) return e;
      value[dev] = v;
      done[dev] = true;
    }
    if (out) *out = value[dev];
    return cudaSuccess;
  }
};

constexpr int NV = 10;

// Per-zone stage constants written by the explicit kernel and read by the
// Newton kernels (structure of arrays, NK planes of N doubles).  With the row
// scale s_a = dt_s / (|U_a(P_n)| + |U_0(P_n)|) folded in, the scaled residual
// of a zone is
//   r_a(P) = kU[a] * U_a(P) + kC[a]                                (a = 0..9)
//   r_8   += kQ[0] q~ + kQ[1] Theta + kQ[2..5] . u_mu + kQ[6] u^t
//   r_9   += kD[0] dP~ + kD[1..4] . u_mu + kD[5] u^t
// where U(P) are the conserved variables and Theta, u_mu, u^t are functions of
// the unknown P; the q~ and dP~ lines carry the implicit relaxation source and
// the time-derivative parts of q~_0, dP~_0 and nabla_mu u^mu (Section 2.3).
enum {
  K_U = 0,        // 10 planes
  K_C = 10,       // 10 planes
  K_Q = 20,       // 7 planes
  K_D = 27,       // 6 planes
  NK = 33
};

struct Params {
  int dim, n1, n2, n3;
  int bc[3][2];
  double dx[3], idx[3];
  double gamma, phi, psi, tauR, theta;
  int cond, visc, ho, recon;
  double tol, eps64;
  float eps32;
  int kmax, lsmax;
  int fd32c;  // centred differences for the float32 Jacobian
  int metric, floors;
  int riemann;  // 0 LLF, 1 HLLE
  long long N;
};

// Launch shape of the Newton solves: threads per block (32, 64 or 128) and
// the update count after which unconverged zones move to the queue kernel
// (>= k_max: no queue).
struct NewtonCfg {
  int bs;
  int kcut;
  bool rounds;  // one update per round, unconverged zones packed between rounds
};

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2 };
enum { RECON_MC = 0, RECON_WENO5 = 1, RECON_PPM = 2 };

// Status bits per zone.
enum { ST_MAXIT = 1, ST_LSSTALL = 2, ST_SINGULAR = 4, ST_NONFINITE = 8, ST_INADMISSIBLE = 16 };

// Global counters of one stage (device memory, atomically accumulated).
struct Counters {
  unsigned long long evals64;   // FP64 residual evaluations
  unsigned long long evals32;   // FP32 residual evaluations
  unsigned long long lu64;      // FP64 LU factor-and-solve
  unsigned long long lu32;      // FP32 LU factor-and-solve
  unsigned long long iters;     // Newton updates
  unsigned long long failed;    // zones with a non-zero status
  unsigned long long zones;     // zones solved
  unsigned long long hist[32];  // Newton updates per zone
  unsigned long long maxres_bits;  // max over zones of max_a |r_a|, as ordered bits
  unsigned long long fallbacks;    // zones whose learned start lost to the plain start
  unsigned long long rescued;      // mixed-solver zones re-solved by the float64 kernel
  unsigned long long mlp_stalls;   // learned-start launches that gave up waiting on the tensor cores
};

// The learned start's variables, in the units the scaled residual measures
// each field in (its rows divide by the conserved magnitudes, which carry the
// rest-mass density): rho and u enter as logarithms and their stage change
// is predicted relative to P_n, (P_conv - P_n)/P_n; q~ and dP~ enter and are
// predicted in units of |X_n| + rho_n; the velocities as they are.  Across
// the orders of magnitude between a torus and its atmosphere this keeps
// features and targets of one size.
__device__ __forceinline__ float mlp_pn_feature(int a, double x, double rho) {
  if (a <= 1) return logf(fmaxf((float)x, 1e-37f));
  if (a >= 8) return (float)(x / (fabs(x) + rho));
  return (float)x;
}
// mlp_pn_feature in float, from the float values of x and rho.
__device__ __forceinline__ float mlp_pn_feature_f(int a, float x, float rho) {
  if (a <= 1) return logf(fmaxf(x, 1e-37f));
  if (a >= 8) return x / (fabsf(x) + rho);
  return x;
}
__device__ __forceinline__ double mlp_unit(int a, double pn, double rho) {
  return a <= 1 ? pn : (a >= 8 ? fabs(pn) + rho : 1.0);
}
__device__ __forceinline__ float mlp_target(int a, double pc, double pn, double rho) {
  return (float)((pc - pn) / mlp_unit(a, pn, rho));
}
__device__ __forceinline__ double mlp_apply(int a, double pn, double d, double rho) {
  return pn + d * mlp_unit(a, pn, rho);
}

// Zones whose mixed-precision Newton iteration ended with a non-zero status
// are handed to the float64 Newton kernel, which solves them again from the
// stage's start (queue of zone indices, its length, and P_n).  All NULL:
// no rescue (the zone keeps its status).
struct Rescue {
  int* queue;
  int* count;
  const double* Pn;
};

// ----------------------------------------------------------------------------
// Math helpers: exact roundings for double, fast approximations for the FP32
// Jacobian (whose error is far below its finite-difference error).
__device__ __forceinline__ double gsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float gsqrt(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double grcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float grcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double grsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float grsqrt(float x) { return rsqrtf(x); }

// ----------------------------------------------------------------------------
// Point physics in Minkowski space for the fused tile kernel of the
// no-allocation step.  Primitive velocity components are u^i;
// u^t = sqrt(1 + u^i u^i), u_t = -u^t, u_i = u^i.
template <typename T> struct Pt {
  T rho, u, ut, uc[3];      // u^t and u^i
  T bt, bc[3], bsq;         // b^t, b^i (b_t = -b^t, b_i = b^i)
  T pg, theta, cs2;
  T q, dp;                  // physical heat flux and anisotropy
  T bht, bh[3];             // bhat^t, bhat^i
  T qt, dpt;                // rescaled primitives
};

// Derived quantities of Section 4: b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t,
// P_g = (gamma-1)u, Theta = P_g/rho, c_s^2 = gamma P_g/(rho + gamma u),
// chi = phi c_s^2 tau_R and nu = psi c_s^2 tau_R, so that
// q = q~ (chi rho Theta^2/tau_R)^(1/2) = q~ Theta (phi c_s^2 rho)^(1/2) and
// dP = dP~ (nu rho Theta/tau_R)^(1/2) = dP~ (psi c_s^2 P_g)^(1/2).
template <typename T>
__device__ __forceinline__ void point_state(const T* P, const Params& p, Pt<T>& s) {
  s.rho = P[0];
  s.u = P[1];
  s.uc[0] = P[2]; s.uc[1] = P[3]; s.uc[2] = P[4];
  T v2 = s.uc[0] * s.uc[0] + s.uc[1] * s.uc[1] + s.uc[2] * s.uc[2];
  s.ut = gsqrt(T(1) + v2);
  T iut = grcp(s.ut);
  s.bt = P[5] * s.uc[0] + P[6] * s.uc[1] + P[7] * s.uc[2];
  s.bc[0] = (P[5] + s.bt * s.uc[0]) * iut;
  s.bc[1] = (P[6] + s.bt * s.uc[1]) * iut;
  s.bc[2] = (P[7] + s.bt * s.uc[2]) * iut;
  s.bsq = s.bc[0] * s.bc[0] + s.bc[1] * s.bc[1] + s.bc[2] * s.bc[2] - s.bt * s.bt;
  const T gam = T(p.gamma);
  s.pg = (gam - T(1)) * s.u;
  T irho = grcp(s.rho);
  s.theta = s.pg * irho;
  s.cs2 = gam * s.pg * grcp(s.rho + gam * s.u);
  s.qt = P[8];
  s.dpt = P[9];
  s.q = p.cond ? s.qt * s.theta * gsqrt(T(p.phi) * s.cs2 * s.rho) : T(0);
  s.dp = p.visc ? s.dpt * gsqrt(T(p.psi) * s.cs2 * s.pg) : T(0);
  if (s.bsq > T(0)) {
    T ib = grsqrt(s.bsq);
    s.bht = s.bt * ib;
    s.bh[0] = s.bc[0] * ib; s.bh[1] = s.bc[1] * ib; s.bh[2] = s.bc[2] * ib;
  } else {
    s.bht = T(0); s.bh[0] = s.bh[1] = s.bh[2] = T(0);
  }
}

// Row m (0 = t, 1..3 = x^j) of T^m_nu (Eq. fullSEtens), nu = t, x, y, z:
//   w u^m u_nu + p_t delta^m_nu - b^m b_nu + q (bhat^m u_nu + u^m bhat_nu)
//   - dP (bhat^m bhat_nu - (delta^m_nu + u^m u_nu)/3),
// w = rho + u + P_g + b^2, p_t = P_g + b^2/2; lowering flips the t component.
template <typename T>
__device__ __forceinline__ void stress_row(const Pt<T>& s, int m, T out[4]) {
  const T w = s.rho + s.u + s.pg + s.bsq;
  const T pt = s.pg + T(0.5) * s.bsq;
  const T um = (m == 0) ? s.ut : s.uc[m - 1];
  const T bm = (m == 0) ? s.bt : s.bc[m - 1];
  const T bhm = (m == 0) ? s.bht : s.bh[m - 1];
  const T third = T(1.0 / 3.0);
  // lowered vectors
  T ul[4] = {-s.ut, s.uc[0], s.uc[1], s.uc[2]};
  T bl[4] = {-s.bt, s.bc[0], s.bc[1], s.bc[2]};
  T bhl[4] = {-s.bht, s.bh[0], s.bh[1], s.bh[2]};
  const T wum = w * um;
  const T dpum = s.dp * um * third;
#pragma unroll
  for (int n = 0; n < 4; n++) {
    T v = wum * ul[n] - bm * bl[n] + s.q * (bhm * ul[n] + um * bhl[n]) - s.dp * bhm * bhl[n] + dpum * ul[n];
    if (n == m) v += pt + s.dp * third;
    out[n] = v;
  }
}

}  // namespace grim
