// Per-zone Newton solve of the stage residual (Section 3): FD Jacobian
// (Section 3.1), partial-pivot LU of the non-magnetic 7x7 block (5x5 in ideal
// MHD), quadratic backtracking line search
// (Section 3.2), convergence test max_a |r_a| <= tol before each Jacobian.
//
// One thread owns one zone.  The zone constants, the Jacobian and the
// right-hand side live in shared memory (stride = block size, so a warp's
// accesses are conflict-free); the state, the residual and the cached
// intermediates of the residual live in registers.
//
// The FP64 pipe bounds these kernels (B300: 1/58 of the FP32 rate), so the
// residual is organised to spend as few float64 instructions as possible
// without changing what it computes:
//  * its intermediates are grouped by the primitives they depend on
//    (thermodynamic: rho, u; kinematic: u^i; magnetic: B^i, u^i), so a
//    finite-difference column recomputes only the groups its perturbed
//    component touches, and only the residual rows that component can change
//    (the others are exact zeros of the FD Jacobian);
//  * five root operations per full evaluation (1/rho = rsqrt(rho)^2, ...);
//  * divisors of the FD columns and the LU pivots use a Newton-Raphson
//    reciprocal, comparisons of magnitudes use the integer order of the
//    IEEE bit patterns, and eliminations with an exactly zero multiplier are
//    skipped (a - 0*x = a).
//
// Precision variants:
//   FP64  -- everything in double.
//   MIXED -- the Jacobian (its residual evaluations) and the LU in float;
//            the residual of the iterate, the update, the line search and the
//            convergence test in double (inexact Newton).
#include "grim_zone.cuh"

namespace grim {

// Zone-constant accessors: shared memory at stride BS, or global at stride N.
template <typename T, int BS> struct KSm {
  const T* p;
  __device__ __forceinline__ T operator()(int a) const { return p[a * BS]; }
};
struct KGl {
  const double* p;
  long long N;
  __device__ __forceinline__ double operator()(int a) const { return __ldg(p + a * N); }
};

// Rows of the scaled residual (see grim_dev.cuh for the constants).
// T^t_nu of Eq. fullSEtens: A u_nu - b^t b_nu + q (bhat^t u_nu + u^t bhat_nu)
// - dP bhat^t bhat_nu + (p_t + dP/3) delta^t_nu with A = (w + dP/3) u^t,
// w = rho + u + P_g + b^2, p_t = P_g + b^2/2; lowering flips the t component.
template <typename T, class KA>
__device__ __forceinline__ void r_T(const Z<T>& z, const KA& k, T out[4]) {
  const T q = z.qt * z.qs, dp = z.dpt * z.ds;
  const T third = dp * T(1.0 / 3.0);
  const T A = (z.w0 + z.bsq + third) * z.ut;
  const T qb = q * z.bht, dpb = dp * z.bht, qut = q * z.ut;
  // nu = t: u_t = -u^t, b_t = -b^t, bhat_t = -bhat^t
  const T Ttt = -A * z.ut + z.bt * z.bt - T(2) * qb * z.ut + dpb * z.bht + z.pg + T(0.5) * z.bsq + third;
  out[0] = k(K_U + 1) * Ttt + k(K_C + 1);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const T Tti = A * z.v[i] - z.bt * z.bc[i] + qb * z.v[i] + qut * z.bh[i] - dpb * z.bh[i];
    out[1 + i] = k(K_U + 2 + i) * Tti + k(K_C + 2 + i);
  }
}
template <typename T, class KA> __device__ __forceinline__ T r_mass(const Z<T>& z, const KA& k) {
  return k(K_U + 0) * (z.rho * z.ut) + k(K_C + 0);
}
template <typename T, class KA> __device__ __forceinline__ T r_field(const Z<T>& z, const KA& k, int i) {
  return k(K_U + 5 + i) * z.B[i] + k(K_C + 5 + i);
}
template <typename T, class KA> __device__ __forceinline__ T r_heat(const Z<T>& z, const KA& k) {
  T r = k(K_U + 8) * (z.qt * z.ut) + k(K_C + 8);
  r += k(K_Q + 0) * z.qt + k(K_Q + 1) * z.theta + k(K_Q + 6) * z.ut;
  r += -k(K_Q + 2) * z.ut + k(K_Q + 3) * z.v[0] + k(K_Q + 4) * z.v[1] + k(K_Q + 5) * z.v[2];
  return r;
}
template <typename T, class KA> __device__ __forceinline__ T r_aniso(const Z<T>& z, const KA& k) {
  T r = k(K_U + 9) * (z.dpt * z.ut) + k(K_C + 9);
  r += k(K_D + 0) * z.dpt + k(K_D + 5) * z.ut;
  r += -k(K_D + 1) * z.ut + k(K_D + 2) * z.v[0] + k(K_D + 3) * z.v[1] + k(K_D + 4) * z.v[2];
  return r;
}
template <typename T, class KA> __device__ __forceinline__ void r_all(const Z<T>& z, const KA& k, T r[NV]) {
  r[0] = r_mass(z, k);
  r_T(z, k, r + 1);
  r[5] = r_field(z, k, 0);
  r[6] = r_field(z, k, 1);
  r[7] = r_field(z, k, 2);
  r[8] = r_heat(z, k);
  r[9] = r_aniso(z, k);
}

// The non-magnetic block of the Jacobian: its m-th component is nb7(m)
// (rho, u, u^1..3, q~, dP~), and component i sits in slot jslot(i) (-1 for
// B).  Shared memory holds only this NJ x NJ block and its right-hand side.
constexpr int NJ = 7;
__host__ __device__ constexpr int nb7(int m) { return m < 5 ? m : m + 3; }
__host__ __device__ constexpr int jslot(int i) { return i < 5 ? i : (i >= 8 ? i - 3 : -1); }

// Perturbed component of the FD Jacobian (Section 3.1): (1 + eps) x, or
// x + eps when |x| < 5 eps (small() read as an absolute step, so the divisor
// never approaches zero).  The absolute floor is for components that pass
// through zero: the positive rho and u (positive = true) keep the relative
// step at every magnitude.
template <typename T> __device__ __forceinline__ T fd_step(T x, T eps, bool positive) {
  return (fabs(x) < T(5) * eps && !(positive && x > T(0))) ? x + eps : (T(1) + eps) * x;
}

// Residual rows of the state z after its component C changed to x (groups
// that depend on C recomputed); rows that cannot depend on C keep r.
template <int C, typename T, class KA>
__device__ __forceinline__ void perturbed_rows(const Z<T>& z0, T x, const T r[NV], const KA& k, const RC<T>& c,
                                               T re[NV]) {
  Z<T> z = z0;
  if constexpr (C == 0) { z.rho = x; z_thermo(z, c); }
  else if constexpr (C == 1) { z.u = x; z_thermo(z, c); }
  else if constexpr (C <= 4) { z.v[C - 2] = x; z_kin(z); z_mag(z); }
  else if constexpr (C <= 7) { z.B[C - 5] = x; z_mag(z); }
  else if constexpr (C == 8) z.qt = x;
  else z.dpt = x;
  constexpr bool kin = (C >= 2 && C <= 4);
#pragma unroll
  for (int i = 0; i < NV; i++) re[i] = r[i];
  if constexpr (C == 0 || kin) re[0] = r_mass(z, k);
  r_T(z, k, re + 1);
  if constexpr (C >= 5 && C <= 7) re[C] = r_field(z, k, C - 5);
  if constexpr (C <= 4 || C == 8) re[8] = r_heat(z, k);
  if constexpr (kin || C == 9) re[9] = r_aniso(z, k);
}

// Whether residual row i can depend on component C (the other entries of the
// FD Jacobian are exact zeros).
template <int C> __device__ __forceinline__ constexpr bool row_depends(int i) {
  constexpr bool kin = (C >= 2 && C <= 4);
  return (i >= 1 && i <= 4) || (i == 0 && (C == 0 || kin)) || (i == C && C >= 5 && C <= 7) ||
         (i == 8 && (C <= 4 || C == 8)) || (i == 9 && (kin || C == 9));
}

template <int C, typename T> __device__ __forceinline__ T component(const Z<T>& z) {
  if constexpr (C == 0) return z.rho;
  else if constexpr (C == 1) return z.u;
  else if constexpr (C <= 4) return z.v[C - 2];
  else if constexpr (C <= 7) return z.B[C - 5];
  else if constexpr (C == 8) return z.qt;
  else return z.dpt;
}

// Column C of the FD Jacobian, written to shared memory in the compact 7x7
// layout of the non-magnetic block (element (i, C) at
// Jc[(jslot(i)*NJ + jslot(C))*BS]; the B rows are not stored).  One-sided (Section 3.1):
// J_iC = (r_i(P_eps) - r_i(P)) / (P_eps,C - P_C).  Centred (float32 option):
// J_iC = (r_i(P + h e_C) - r_i(P - h e_C)) / (2h) with h = P_eps,C - P_C.
template <int C, bool CENTRAL, typename T, int BS, class KA>
__device__ __forceinline__ void fd_column(const Z<T>& z, const T r[NV], const KA& k, const RC<T>& c, T eps,
                                          T* Jc) {
  const T pj = component<C>(z);
  const T pe = fd_step(pj, eps, C <= 1);
  const T h = pe - pj;
  T rp[NV];
  perturbed_rows<C>(z, pe, r, k, c, rp);
  if constexpr (!CENTRAL) {
    const T ih = nr_rcp(h);
#pragma unroll
    for (int i = 0; i < NV; i++)
      if (jslot(i) >= 0) Jc[(jslot(i) * NJ + jslot(C)) * BS] = row_depends<C>(i) ? (rp[i] - r[i]) * ih : T(0);
  } else {
    T rm[NV];
    perturbed_rows<C>(z, pj - h, r, k, c, rm);
    const T ih = T(0.5) * nr_rcp(h);
#pragma unroll
    for (int i = 0; i < NV; i++)
      if (jslot(i) >= 0) Jc[(jslot(i) * NJ + jslot(C)) * BS] = row_depends<C>(i) ? (rp[i] - rm[i]) * ih : T(0);
  }
}

// The Jacobian columns of rho, u, u^i, q~, dP~.  The B columns are not
// formed: the B rows are linear in B alone (r_B = kU_B B + kC_B) and the
// start already holds their root, the flux-CT field, so the Newton update of
// B is zero to round-off and the system reduces to the 7x7 block of the
// other components (the paper's EMHD solve, Section 8.2).  five: ideal MHD
// (see ideal_zone), where the q~ and dP~ columns are not formed either and
// the block is 5x5.
template <typename T, bool CENTRAL, int BS, class KA>
__device__ __forceinline__ void fd_jacobian(const Z<T>& z, const T r[NV], const KA& k, const RC<T>& c, T eps,
                                            T* J, bool five = false) {
  fd_column<0, CENTRAL, T, BS>(z, r, k, c, eps, J);
  fd_column<1, CENTRAL, T, BS>(z, r, k, c, eps, J);
  fd_column<2, CENTRAL, T, BS>(z, r, k, c, eps, J);
  fd_column<3, CENTRAL, T, BS>(z, r, k, c, eps, J);
  fd_column<4, CENTRAL, T, BS>(z, r, k, c, eps, J);
  if (!five) {
    fd_column<8, CENTRAL, T, BS>(z, r, k, c, eps, J);
    fd_column<9, CENTRAL, T, BS>(z, r, k, c, eps, J);
  }
}

// Ideal MHD (conduction and viscosity off, Section 8.2's 5x5 solve): in a
// zone whose q~ and dP~ and their residual rows are zero, those rows stay
// exactly zero for any rho, u, u^i (every term of them carries q~, dP~ or a
// closure coefficient), so their Newton update is zero and the system
// reduces to the 5x5 block of rho, u, u^i.  Other zones keep the 7x7 block.
__device__ __forceinline__ bool ideal_zone(const Params& p, const double P[NV], const double r[NV]) {
  return !p.cond && !p.visc && P[8] == 0.0 && P[9] == 0.0 && r[8] == 0.0 && r[9] == 0.0;
}


// Partial-pivot LU solve of the leading NB x NB block of the compact
// Jacobian (NB = 7: the non-magnetic components nb7(0..6); NB = 5: rho, u,
// u^i) in shared memory at stride BS, with the right-hand side b in slots
// 0..NB-1; the other components of x are 0.  Pivot: largest |a_ik|, lowest
// row on ties.  Returns false on a zero pivot.
template <typename T, int BS, int NB = 7>
__device__ __forceinline__ bool lu_solve_block_smem(T* J, T* b, T x[NV]) {
  static_assert(NB == 7 || NB == 5, "7x7 or 5x5 block");
  T inv[NB];
#pragma unroll
  for (int k = 0; k < NB; k++) {
    int piv = k;
    auto best = abits(J[(k * NJ + k) * BS]);
#pragma unroll
    for (int i = k + 1; i < NB; i++) {
      const auto a = abits(J[(i * NJ + k) * BS]);
      if (a > best) { best = a; piv = i; }
    }
    if (best == 0) return false;
    if (piv != k) {
#pragma unroll
      for (int c = k; c < NB; c++) {
        const T t = J[(k * NJ + c) * BS];
        J[(k * NJ + c) * BS] = J[(piv * NJ + c) * BS];
        J[(piv * NJ + c) * BS] = t;
      }
      const T t = b[k * BS];
      b[k * BS] = b[piv * BS];
      b[piv * BS] = t;
    }
    inv[k] = nr_rcp(J[(k * NJ + k) * BS]);
    const T bk = b[k * BS];
#pragma unroll
    for (int i = k + 1; i < NB; i++) {
      const T a = J[(i * NJ + k) * BS];
      if (abits(a) == 0) continue;  // zero multiplier: row i is unchanged
      const T l = a * inv[k];
#pragma unroll
      for (int c = k + 1; c < NB; c++) J[(i * NJ + c) * BS] -= l * J[(k * NJ + c) * BS];
      b[i * BS] -= l * bk;
    }
  }
  x[5] = x[6] = x[7] = T(0);
  if (NB == 5) x[8] = x[9] = T(0);
#pragma unroll
  for (int i = NB - 1; i >= 0; i--) {
    T acc = b[i * BS];
#pragma unroll
    for (int c = i + 1; c < NB; c++) acc -= J[(i * NJ + c) * BS] * x[nb7(c)];
    x[nb7(i)] = acc * inv[i];
  }
  return true;
}

__device__ __forceinline__ unsigned long long max_abits10(const double* r) {
  unsigned long long m = 0;
#pragma unroll
  for (int a = 0; a < NV; a++) m = max(m, abits(r[a]));
  return m;
}
__device__ __forceinline__ double sum_sq10(const double* r) {
  double f = 0.0;
#pragma unroll
  for (int a = 0; a < NV; a++) f = fma(r[a], r[a], f);
  return f;
}

// The learned start's fallback test without a float64 evaluation of the
// plain start: rn (stride `stride`, may be NULL) holds the increment
// features -r_a(P_n), the plain start's scaled residual in float (its
// magnetic rows are those of P_n's field, which the plain start replaces
// by the flux-CT update, so they are left out).  The learned start is kept
// when its |r|^2 does not exceed theirs; otherwise the plain start is
// evaluated and the two compared as before (it is needed in float64 then
// anyway, as the solve's first residual).
__device__ __forceinline__ bool learned_wins(double f, const float* rn, long long stride) {
  if (!rn) return false;
  double fp = 0.0;
#pragma unroll
  for (int a = 0; a < NV; a++)
    if (a < 5 || a > 7) {
      const double x = (double)__ldg(rn + a * stride);
      fp = fma(x, x, fp);
    }
  return f <= fp;
}

struct ZoneResult {
  int iters, status, evals64, evals32, lu64, lu32;
  int done;       // Newton updates made by this call (iters counts from the zone's first)
  bool pending;   // stopped at kstop, unconverged: the zone continues in the queue kernel
  double res;
  double bsq, ds; // general metric with floors and viscosity: b^2 and dP / dP~ of the final state
};

// Newton on one zone, starting from P (updated in place) after k0 updates
// made by an earlier call; stops unconverged (o.pending) once the zone has
// made kstop updates, kstop < k_max.  kd: the zone's float64 constants in
// shared memory (stride BS); kf: their float copies.  Pfb (non-NULL with a
// learned start): the plain start P_n, whose magnetic components are those
// of P; if the learned start's max|r| exceeds accept_bits the plain start is
// evaluated too and the smaller |r|^2 wins.  rq (stride rs, may be NULL):
// the zone's residual slot for the queue: a call that stops pending stores
// r(P) there, and a resumed call (k0 > 0) reads it instead of evaluating it
// again.
template <bool MIXED, int BS, bool IDEAL>
__device__ __forceinline__ ZoneResult newton_zone(const Params& p, const double* kd, const float* kf, double P[NV],
                                                  void* jac, const double* Pfb, long long fb_stride,
                                                  unsigned long long accept_bits, bool& fellback, int k0,
                                                  int kstop, double* rq, long long rs, const float* rn = nullptr) {
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
  const RC<double> c64 = make_rc<double>(p);
  const KSm<double, BS> k64{kd};
  const unsigned long long tol_bits = abits(p.tol);
  Z<double> z;
  double r[NV];
  if (rq && k0 > 0) {
    if (!MIXED) z_load(z, P, c64);  // the float64 Jacobian differentiates from z
#pragma unroll
    for (int a = 0; a < NV; a++) r[a] = rq[a * rs];
  } else {
    z_load(z, P, c64);
    r_all(z, k64, r);
    o.evals64++;
  }
  double f = sum_sq10(r);
  fellback = false;
  if (Pfb && !(max_abits10(r) <= accept_bits) && !learned_wins(f, rn, fb_stride)) {
    double Pp[NV], rp[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) Pp[a] = (a >= 5 && a <= 7) ? P[a] : Pfb[a * fb_stride];
    Z<double> zp;
    z_load(zp, Pp, c64);
    r_all(zp, k64, rp);
    o.evals64++;
    const double fp = sum_sq10(rp);
    if (!(f <= fp)) {
      fellback = true;
#pragma unroll
      for (int a = 0; a < NV; a++) { P[a] = Pp[a]; r[a] = rp[a]; }
      z = zp;
      f = fp;
    }
  }
  const bool five = IDEAL && ideal_zone(p, P, r);
  int k = k0;
  for (;;) {
    if (!finite_bits(f)) { o.status |= ST_NONFINITE; break; }
    if (max_abits10(r) <= tol_bits) break;
    if (k >= p.kmax) { o.status |= ST_MAXIT; break; }
    if (k >= kstop) { o.pending = true; break; }
    double dP[NV];
    bool ok;
    if (!MIXED) {
      double* J = (double*)jac + threadIdx.x;
      double* b = J + NJ * NJ * BS;
      fd_jacobian<double, false, BS>(z, r, k64, c64, p.eps64, J, five);
      o.evals64 += five ? 5 : 7;
#pragma unroll
      for (int m = 0; m < NJ; m++) b[m * BS] = -r[nb7(m)];
      ok = five ? lu_solve_block_smem<double, BS, 5>(J, b, dP) : lu_solve_block_smem<double, BS, 7>(J, b, dP);
      o.lu64++;
    } else {
      const RC<float> c32 = make_rc<float>(p);
      const KSm<float, BS> k32{kf};
      float* J = (float*)jac + threadIdx.x;
      float* b = J + NJ * NJ * BS;
      float Pf[NV], rf[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pf[a] = d2f_jac(P[a]);
      Z<float> zf;
      z_load(zf, Pf, c32);
      r_all(zf, k32, rf);
      const int ncol = five ? 5 : 7;
      if (p.fd32c) {
        fd_jacobian<float, true, BS>(zf, rf, k32, c32, p.eps32, J, five);
        o.evals32 += 2 * ncol + 1;
      } else {
        fd_jacobian<float, false, BS>(zf, rf, k32, c32, p.eps32, J, five);
        o.evals32 += ncol + 1;
      }
#pragma unroll
      for (int m = 0; m < NJ; m++) b[m * BS] = d2f_jac(-r[nb7(m)]);
      float df[NV];
      ok = five ? lu_solve_block_smem<float, BS, 5>(J, b, df) : lu_solve_block_smem<float, BS, 7>(J, b, df);
      // a float32 solve that overflowed or met a NaN pivot has no direction:
      // the zone is reported singular, not moved by a huge step
#pragma unroll
      for (int i = 0; i < NV; i++) ok = ok && isfinite(df[i]);
#pragma unroll
      for (int i = 0; i < NV; i++) dP[i] = f2d_jac(df[i]);
      o.lu32++;
    }
    if (!ok) { o.status |= ST_SINGULAR; break; }
    // quadratic backtracking line search on f = |r|^2
    double lam = 1.0, Pt[NV], rt[NV], ft = 0.0;
    Z<double> zt;
    for (int t = 0;; t++) {
#pragma unroll
      for (int a = 0; a < NV; a++) Pt[a] = fma(lam, dP[a], P[a]);
      z_load(zt, Pt, c64);
      r_all(zt, k64, rt);
      o.evals64++;
      ft = sum_sq10(rt);
      const bool fin = finite_bits(ft);
      const double lim = 1.0 - 1e-4 * lam;
      if (fin && ft < f * lim * lim) break;
      if (t >= p.lsmax) { o.status |= ST_LSSTALL; break; }
      // the quadratic model's minimiser when it is a positive finite number,
      // else half the step (a non-finite trial, or an overflowed denominator
      // that would leave lambda = 0 and then 0/0)
      const double ln = fin ? f * lam * lam / (ft + (2.0 * lam - 1.0) * f) : 0.0;
      lam = (ln > 0.0 && finite_bits(ln)) ? ln : 0.5 * lam;
    }
#pragma unroll
    for (int a = 0; a < NV; a++) { P[a] = Pt[a]; r[a] = rt[a]; }
    z = zt;
    f = ft;
    k++;
  }
  o.iters = k;
  o.done = k - k0;
  unsigned long long mb = max_abits10(r);
  o.res = __longlong_as_double((long long)mb);
  if (!(P[0] > 0.0) || !(P[1] > 0.0)) o.status |= ST_INADMISSIBLE;
  if (o.pending && rq) {
#pragma unroll
    for (int a = 0; a < NV; a++) rq[a * rs] = r[a];
  }
  return o;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Add one warp's zones to the counters.  Work counts (evaluations, LU
// solves, updates, fallbacks) are added by every call; a zone's totals
// (zones, failures, the update histogram, the residual maximum) only by the
// call that finishes it.
__device__ __forceinline__ void accumulate(Counters* c, const ZoneResult& o, bool active, bool fellback) {
  const int lane = threadIdx.x & 31;
  const bool fin = active && !o.pending;
  unsigned long long e64 = active ? o.evals64 : 0, e32 = active ? o.evals32 : 0;
  unsigned long long l64 = active ? o.lu64 : 0, l32 = active ? o.lu32 : 0;
  unsigned long long it = active ? o.done : 0, fl = (fin && o.status) ? 1 : 0, zn = fin ? 1 : 0;
  const unsigned any = __ballot_sync(0xffffffffu, active);
  e64 = warp_sum(e64); e32 = warp_sum(e32); l64 = warp_sum(l64); l32 = warp_sum(l32);
  it = warp_sum(it); fl = warp_sum(fl); zn = warp_sum(zn);
  if (lane == 0 && any) {
    atomicAdd(&c->evals64, e64); atomicAdd(&c->evals32, e32);
    atomicAdd(&c->lu64, l64); atomicAdd(&c->lu32, l32);
    atomicAdd(&c->iters, it);
    if (zn) { atomicAdd(&c->failed, fl); atomicAdd(&c->zones, zn); }
  }
  const unsigned fb = __ballot_sync(0xffffffffu, active && fellback);
  if (lane == 0 && fb) atomicAdd(&c->fallbacks, (unsigned long long)__popc(fb));
  if (fin) {
    atomicAdd(&c->hist[o.iters < 31 ? o.iters : 31], 1ull);
    if (finite_bits(o.res)) atomicMax(&c->maxres_bits, (unsigned long long)__double_as_longlong(o.res));
  }
}

// Append the warp's pending zones to the queue (one atomic per warp).
__device__ __forceinline__ void enqueue(int* queue, int* qcount, bool pending, long long z) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, pending);
  if (!m) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(qcount, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pending) queue[base + __popc(m & ((1u << lane) - 1u))] = (int)z;
}

// A mixed-precision zone solve that ended with a non-zero status (no
// convergence, a stalled line search, a singular or non-finite float32
// solve) goes to the rescue queue, and counts as unfinished here: the
// float64 kernel solves it again and finishes it.
__device__ __forceinline__ void to_rescue(int* rqueue, int* rcount, ZoneResult& o, bool active, long long z) {
  const bool resc = active && !o.pending && o.status != 0;
  enqueue(rqueue, rcount, resc, z);
  o.pending = o.pending || resc;
}

// Per-thread tallies of a block's zone solves, added to the counters once,
// at the end of the kernel (warp sums, one atomic per warp and counter); a
// zone's histogram bin and residual maximum go in when it finishes.  Work
// counts belong to whichever thread did the work, zone counts to the thread
// that finished the zone.
struct Tally {
  unsigned e64 = 0, e32 = 0, l64 = 0, l32 = 0, it = 0, zn = 0, fl = 0, fb = 0;  // one thread's share: small
  __device__ __forceinline__ void work(const ZoneResult& o) {
    e64 += o.evals64; e32 += o.evals32; l64 += o.lu64; l32 += o.lu32; it += o.done;
  }
  __device__ __forceinline__ void finish(Counters* c, const ZoneResult& o) {
    zn++;
    fl += o.status != 0;
    atomicAdd(&c->hist[o.iters < 31 ? o.iters : 31], 1ull);
    if (finite_bits(o.res)) atomicMax(&c->maxres_bits, (unsigned long long)__double_as_longlong(o.res));
  }
  // every lane of the warp calls it
  __device__ __forceinline__ void flush(Counters* c) {
    using u64 = unsigned long long;
    const u64 s64 = warp_sum(e64), s32 = warp_sum(e32), sl64 = warp_sum(l64), sl32 = warp_sum(l32);
    const u64 sit = warp_sum(it), szn = warp_sum(zn), sfl = warp_sum(fl), sfb = warp_sum(fb);
    if ((threadIdx.x & 31) == 0 && (s64 | s32 | szn | sit)) {
      atomicAdd(&c->evals64, s64); atomicAdd(&c->evals32, s32);
      atomicAdd(&c->lu64, sl64); atomicAdd(&c->lu32, sl32);
      atomicAdd(&c->iters, sit);
      if (szn) { atomicAdd(&c->failed, sfl); atomicAdd(&c->zones, szn); }
      if (sfb) atomicAdd(&c->fallbacks, sfb);
    }
  }
};

// Rank of this thread among the threads of the block whose flag is set (in
// thread order), and in `total` their number.  wsum: BS/32 ints of shared
// memory.  Every thread of the block calls it; it holds a barrier, after
// which every thread has passed its call.
template <int BS>
__device__ __forceinline__ int block_rank(bool flag, int* wsum, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < BS / 32; i++) {
    const int c = wsum[i];
    base += i < w ? c : 0;
    tot += c;
  }
  total = tot;
  return base + __popc(m & ((1u << lane) - 1u));
}

// Compaction between updates.  Between two rounds of one update each, a
// zone that goes on moves to the thread of its rank among the block's
// unconverged zones, through the Jacobian area of shared memory (free
// between updates): its state P, its residual r (the resumed solve reads r
// instead of evaluating it again), the slot of its constants (they stay in
// their column) and its update count.  The Jacobian area holds 20 doubles
// and an int per thread at least (MIXED: 56 floats).
struct Staging {
  double* P;
  double* r;
  int* meta;
  template <int BS> __device__ __forceinline__ static Staging at(void* jac) {
    double* d = (double*)jac;
    return Staging{d, d + NV * BS, (int*)(d + 2 * NV * BS)};
  }
  template <int BS> __device__ __forceinline__ void put(int i, const double P_[NV], const double r_[NV], int slot, int k) const {
#pragma unroll
    for (int a = 0; a < NV; a++) { P[a * BS + i] = P_[a]; r[a * BS + i] = r_[a]; }
    meta[i] = slot | (k << 16);
  }
  template <int BS> __device__ __forceinline__ void get(int i, double P_[NV], double r_[NV], int& slot, int& k) const {
#pragma unroll
    for (int a = 0; a < NV; a++) { P_[a] = P[a * BS + i]; r_[a] = r[a * BS + i]; }
    slot = meta[i] & 0xffff;
    k = meta[i] >> 16;
  }
};
static_assert(sizeof(float) * (NJ * NJ + NJ) >= 2 * NV * sizeof(double) + sizeof(int), "staging fits the Jacobian area");

// Shared memory per thread: zone constants (NK doubles, plus NK floats for
// MIXED), the Jacobian and the right-hand side (110 elements of the Jacobian
// precision).
template <bool MIXED, int BS> struct NewtonSmem {
  static constexpr size_t kd = sizeof(double) * NK * BS;
  static constexpr size_t kf = MIXED ? sizeof(float) * NK * BS : 0;
  static constexpr size_t jac = (MIXED ? sizeof(float) : sizeof(double)) * (NJ * NJ + NJ) * BS;
  static constexpr size_t bytes = kd + kf + jac;
};

// One thread per zone, zones in order; each zone runs to convergence or to
// kstop updates, after which it is appended to the queue (kstop >= k_max:
// no queue).
template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS, 1) newton_dense(const __grid_constant__ Params p, const double* __restrict__ K,
                                                   double* __restrict__ P, uint8_t* __restrict__ iters,
                                                   uint8_t* __restrict__ status, Counters* __restrict__ cnt,
                                                   const double* __restrict__ Pfb, double accept, int kstop,
                                                   int* __restrict__ queue, int* __restrict__ qcount,
                                                   double* __restrict__ rq, int* __restrict__ rqueue,
                                                   int* __restrict__ rcount,
                                                   const float* __restrict__ rn) {
  using S = NewtonSmem<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  float* kf = (float*)(smem_raw + S::kd) + threadIdx.x;
  void* jac = smem_raw + S::kd + S::kf;
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * BS + threadIdx.x;
  const bool active = z < N;
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
  bool fellback = false;
  if (active) {
#pragma unroll
    for (int a = 0; a < NK; a++) {
      const double x = __ldg(K + a * N + z);
      kd[a * BS] = x;
      if (MIXED) kf[a * BS] = d2f_jac(x);
    }
    double Pz[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z];
    o = newton_zone<MIXED, BS, IDEAL>(p, kd, kf, Pz, jac, Pfb ? Pfb + z : nullptr, N, abits(accept), fellback, 0,
                               kstop < p.kmax ? kstop : p.kmax, queue && rq ? rq + z : nullptr, N,
                               Pfb && rn ? rn + z : nullptr);
#pragma unroll
    for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
    iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
    status[z] = (uint8_t)o.status;
  }
  if (queue) enqueue(queue, qcount, active && o.pending, z);
  if (MIXED && rqueue) to_rescue(rqueue, rcount, o, active, z);
  accumulate(cnt, o, active, fellback);
}

// newton_dense in rounds of one update, with the block's unconverged zones
// packed into its lowest threads between rounds (see Staging): a converged
// zone stops costing its warp issue slots (a float64 warp instruction costs
// the pipe the same whatever lanes are live).  A zone makes at most kstop
// updates here, then goes on in the queue kernel (kstop >= k_max: no queue).
// The zone solves are those of newton_dense, bit for bit.
template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_rounds(const __grid_constant__ Params p, const double* __restrict__ K,
                                                    double* __restrict__ P, uint8_t* __restrict__ iters,
                                                    uint8_t* __restrict__ status, Counters* __restrict__ cnt,
                                                    const double* __restrict__ Pfb, double accept, int kstop,
                                                    int* __restrict__ queue, int* __restrict__ qcount,
                                                    double* __restrict__ rq, int* __restrict__ rqueue,
                                                    int* __restrict__ rcount,
                                                    const float* __restrict__ rn) {
  using S = NewtonSmem<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int wsum[BS / 32];
  double* kd = (double*)smem_raw;
  float* kf = (float*)(smem_raw + S::kd);
  void* jac = smem_raw + S::kd + S::kf;
  const Staging stg = Staging::at<BS>(jac);
  const long long N = p.N;
  const long long z0 = (long long)blockIdx.x * BS;
  const int t = threadIdx.x;
  const int ks = kstop < p.kmax ? kstop : p.kmax;
  const unsigned long long acc = abits(accept);
  bool own = z0 + t < N;
  int sl = t, k = 0;
  double Pz[NV], rz[NV];
  if (own) {
#pragma unroll
    for (int a = 0; a < NK; a++) {
      const double x = __ldg(K + a * N + z0 + t);
      kd[a * BS + t] = x;
      if (MIXED) kf[a * BS + t] = d2f_jac(x);
    }
#pragma unroll
    for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z0 + t];
  }
  Tally tl;
  for (int round = 0;; round++) {
    const long long z = z0 + sl;
    bool go = false, resc = false;
    if (own) {
      bool fb = false;
      const ZoneResult o = newton_zone<MIXED, BS, IDEAL>(p, kd + sl, kf + sl, Pz, jac,
                                                         round == 0 && Pfb ? Pfb + z : nullptr, N, acc, fb, k,
                                                         k + 1, rz, 1, round == 0 && Pfb && rn ? rn + z : nullptr);
      tl.work(o);
      tl.fb += fb;
      k = o.iters;
      go = o.pending;
      if (!go) {
#pragma unroll
        for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
        iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
        status[z] = (uint8_t)o.status;
        if (MIXED && rqueue && o.status != 0) resc = true;  // finished by the rescue kernel
        else tl.finish(cnt, o);
      }
    }
    if (MIXED && rqueue) enqueue(rqueue, rcount, resc, z);
    int n = 0;
    const int rank = block_rank<BS>(go, wsum, n);
    if (n == 0) break;
    if (round + 1 >= ks) {
      // unconverged after ks updates: on to the queue kernel
      if (go) {
#pragma unroll
        for (int a = 0; a < NV; a++) {
          P[a * N + z] = Pz[a];
          if (rq) rq[a * N + z] = rz[a];
        }
        iters[z] = (uint8_t)k;
      }
      enqueue(queue, qcount, go, z);
      break;
    }
    if (n > BS - 32) {
      // packing would free no warp: every zone stays with its thread
      own = go;
      continue;
    }
    if (go) stg.put<BS>(rank, Pz, rz, sl, k);
    __syncthreads();
    own = t < n;
    if (own) stg.get<BS>(t, Pz, rz, sl, k);
    __syncthreads();
  }
  tl.flush(cnt);
}

// The zones queued by newton_dense, packed densely into warps: a persistent
// grid strides over the queue and continues each zone from its state and
// update count to convergence or k_max.
template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_queue(const __grid_constant__ Params p, const double* __restrict__ K,
                                                   double* __restrict__ P, uint8_t* __restrict__ iters,
                                                   uint8_t* __restrict__ status, Counters* __restrict__ cnt,
                                                   const int* __restrict__ queue, const int* __restrict__ qcount,
                                                   double* __restrict__ rq, int* __restrict__ rqueue,
                                                   int* __restrict__ rcount) {
  using S = NewtonSmem<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  float* kf = (float*)(smem_raw + S::kd) + threadIdx.x;
  void* jac = smem_raw + S::kd + S::kf;
  const long long N = p.N;
  const int count = *qcount;
  for (int base = blockIdx.x * BS; base < count; base += gridDim.x * BS) {
    const int q = base + (int)threadIdx.x;
    const bool active = q < count;
    ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
    bool fellback = false;
    if (active) {
      const long long z = queue[q];
#pragma unroll
      for (int a = 0; a < NK; a++) {
        const double x = __ldg(K + a * N + z);
        kd[a * BS] = x;
        if (MIXED) kf[a * BS] = d2f_jac(x);
      }
      double Pz[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z];
      o = newton_zone<MIXED, BS, IDEAL>(p, kd, kf, Pz, jac, nullptr, N, 0ull, fellback, iters[z], p.kmax,
                                 rq ? rq + z : nullptr, N);
#pragma unroll
      for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
      iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
      status[z] = (uint8_t)o.status;
    }
    if (MIXED && rqueue) to_rescue(rqueue, rcount, o, active, active ? queue[q] : 0);
    accumulate(cnt, o, active, fellback);
  }
}

// The mixed solver's rescue: the zones of the rescue queue solved again with
// the float64 Jacobian, from the stage's start (P_n; the magnetic components
// are still the start's, since no update changes them), to convergence or
// k_max.  Persistent grid over the queue; the zone's counters are finished
// here.
template <int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_rescue(const __grid_constant__ Params p, const double* __restrict__ K,
                                                    const double* __restrict__ Pn, double* __restrict__ P,
                                                    uint8_t* __restrict__ iters, uint8_t* __restrict__ status,
                                                    Counters* __restrict__ cnt, const int* __restrict__ rqueue,
                                                    const int* __restrict__ rcount) {
  using S = NewtonSmem<false, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  void* jac = smem_raw + S::kd;
  const long long N = p.N;
  const int count = *rcount;
  for (int base = blockIdx.x * BS; base < count; base += gridDim.x * BS) {
    const int q = base + (int)threadIdx.x;
    const bool active = q < count;
    ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
    bool fb = false;
    if (active) {
      const long long z = rqueue[q];
#pragma unroll
      for (int a = 0; a < NK; a++) kd[a * BS] = __ldg(K + a * N + z);
      double Pz[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pz[a] = (a >= 5 && a <= 7) ? P[a * N + z] : __ldg(Pn + a * N + z);
      o = newton_zone<false, BS, IDEAL>(p, kd, nullptr, Pz, jac, nullptr, N, 0ull, fb, 0, p.kmax, nullptr, N);
#pragma unroll
      for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
      iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
      status[z] = (uint8_t)o.status;
    }
    accumulate(cnt, o, active, false);
    const unsigned m = __ballot_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&cnt->rescued, (unsigned long long)__popc(m));
  }
}

// Launch the rescue kernel over the queue filled by the mixed kernels.
template <int BS, bool IDEAL> struct RescueKernels {
  using S = NewtonSmem<false, BS>;
  static cudaError_t launch(const Params& p, const double* K, double* P, uint8_t* iters, uint8_t* status,
                            Counters* cnt, const Rescue& rs, cudaStream_t st) {
    static PerDevice once;
    int grid = 0;
    cudaError_t e = once.get(
        [](int* g) {
          cudaError_t r = cudaFuncSetAttribute(newton_rescue<BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)S::bytes);
          int dev = 0, sms = 0;
          if (r == cudaSuccess) r = cudaGetDevice(&dev);
          if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          // rescued zones are rare: one block per SM keeps the launch of an
          // empty queue cheap
          if (r == cudaSuccess) *g = sms;
          return r;
        },
        &grid);
    if (e != cudaSuccess) return e;
    newton_rescue<BS, IDEAL><<<(unsigned)grid, BS, S::bytes, st>>>(p, K, rs.Pn, P, iters, status, cnt, rs.queue,
                                                                    rs.count);
    return cudaGetLastError();
  }
};

// Evaluate the scaled (or raw) residual at Pk once per zone.
__global__ void residual_once(const __grid_constant__ Params p, const double* __restrict__ K,
                              const double* __restrict__ Pk, int scaled, double dts, double* __restrict__ R) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const KGl kg{K + z, N};
  const RC<double> c = make_rc<double>(p);
  double Pz[NV], r[NV];
#pragma unroll
  for (int a = 0; a < NV; a++) Pz[a] = Pk[a * N + z];
  Z<double> zz;
  z_load(zz, Pz, c);
  r_all(zz, kg, r);
#pragma unroll
  for (int a = 0; a < NV; a++) {
    // the row scale is kU * dt_s; divide it out for the raw residual
    R[a * N + z] = scaled ? r[a] : r[a] / (kg(K_U + a) * dts);
  }
}

// Reciprocal self-check: max |nr_rcp(x) - 1/x| / |1/x| over x = m * 2^e for
// seeded mantissas m in [1, 2) and exponents e in [-300, 300], both signs.
__global__ void rcp_check(int n, unsigned long long seed, double* worst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  unsigned long long s = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(t + 1);
  s ^= s >> 33; s *= 0xff51afd7ed558ccdull; s ^= s >> 33;
  const double m = 1.0 + (double)(s >> 11) * (1.0 / 9007199254740992.0);
  const int e = (int)((s >> 3) % 601) - 300;
  const double x = ((s & 1) ? -1.0 : 1.0) * ldexp(m, e);
  const double a = nr_rcp(x), b = 1.0 / x;
  const double rel = fabs(a - b) / fabs(b);
  atomicMax((unsigned long long*)worst, (unsigned long long)__double_as_longlong(rel));
}

template <bool MIXED, int BS, bool IDEAL> struct NewtonKernels {
  using S = NewtonSmem<MIXED, BS>;
  // the kernels' shared-memory limit and the queue kernel's persistent grid
  // (SMs x resident blocks), once per device
  static cudaError_t configure(int& qgrid) {
    static PerDevice once;
    return once.get(
        [](int* grid) {
          cudaError_t e = cudaFuncSetAttribute(newton_dense<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_rounds<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_queue<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          int dev = 0, sms = 0, per_sm = 0;
          if (e == cudaSuccess) e = cudaGetDevice(&dev);
          if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_queue<MIXED, BS, IDEAL>, BS, S::bytes);
          if (e == cudaSuccess) *grid = sms * (per_sm > 0 ? per_sm : 1);
          return e;
        },
        &qgrid);
  }
  static cudaError_t launch(const Params& p, const double* K, double* P, uint8_t* iters, uint8_t* status,
                            Counters* cnt, const double* Pfb, double accept, int kcut, bool rounds, int* queue,
                            int* qcount, double* rq, const Rescue& rs, const float* rn, cudaStream_t st) {
    int qgrid = 0;
    cudaError_t e = configure(qgrid);
    if (e != cudaSuccess) return e;
    const bool compact = queue && qcount && kcut < p.kmax;
    const bool rescue = MIXED && rs.queue && rs.count && rs.Pn;
    if (compact && (e = cudaMemsetAsync(qcount, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (rescue && (e = cudaMemsetAsync(rs.count, 0, sizeof(int), st)) != cudaSuccess) return e;
    int* rqueue = rescue ? rs.queue : nullptr;
    const long long nb = (p.N + BS - 1) / BS;
    if (rounds)
      newton_rounds<MIXED, BS, IDEAL><<<(unsigned)nb, BS, S::bytes, st>>>(p, K, P, iters, status, cnt, Pfb, accept,
                                                                    compact ? kcut : p.kmax,
                                                                    compact ? queue : nullptr, qcount, rq, rqueue,
                                                                    rs.count, rn);
    else
      newton_dense<MIXED, BS, IDEAL><<<(unsigned)nb, BS, S::bytes, st>>>(p, K, P, iters, status, cnt, Pfb, accept,
                                                                   compact ? kcut : p.kmax,
                                                                   compact ? queue : nullptr, qcount, rq, rqueue,
                                                                   rs.count, rn);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (compact) {
      newton_queue<MIXED, BS, IDEAL><<<(unsigned)qgrid, BS, S::bytes, st>>>(p, K, P, iters, status, cnt, queue,
                                                                          qcount, rq, rqueue, rs.count);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (rescue) return RescueKernels<BS, IDEAL>::launch(p, K, P, iters, status, cnt, rs, st);
    return cudaSuccess;
  }
};

template <bool MIXED, bool IDEAL>
static cudaError_t launch_newton_bs(const Params& p, const double* K, double* P, uint8_t* iters, uint8_t* status,
                                   Counters* cnt, const double* Pfb, double accept, const NewtonCfg& cfg, int* queue,
                                   int* qcount, double* rq, const Rescue& rs, const float* rn, cudaStream_t st) {
  switch (cfg.bs) {
    case 32:
      return NewtonKernels<MIXED, 32, IDEAL>::launch(p, K, P, iters, status, cnt, Pfb, accept, cfg.kcut, cfg.rounds, queue,
                                                     qcount, rq, rs, rn, st);
    case 64:
      return NewtonKernels<MIXED, 64, IDEAL>::launch(p, K, P, iters, status, cnt, Pfb, accept, cfg.kcut, cfg.rounds, queue,
                                                     qcount, rq, rs, rn, st);
    case 128:
      return NewtonKernels<MIXED, 128, IDEAL>::launch(p, K, P, iters, status, cnt, Pfb, accept, cfg.kcut, cfg.rounds, queue,
                                                      qcount, rq, rs, rn, st);
    default: return cudaErrorInvalidValue;
  }
}

// Newton solves of one stage: the in-order kernel, then (cfg.kcut < k_max)
// the queue kernel over the zones still unconverged after kcut updates.
// rq: scratch of NV x N doubles for the residuals of the zones handed to the
// queue kernel (may be NULL: the queue kernel then re-evaluates them).
// rs: the mixed solver's rescue (Rescue{} for none).  rn: with a learned
// start (Pfb), the increment features -r_a(P_n) ([NV][N] floats, may be
// NULL), which let the fallback test skip a float64 evaluation of the plain
// start (learned_wins).
cudaError_t launch_newton_fb(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                             Counters* cnt, const double* Pfb, double accept, const NewtonCfg& cfg, int* queue,
                             int* qcount, double* rq, const Rescue& rs, const float* rn, cudaStream_t st) {
  // ideal MHD: the kernels that may take the 5x5 block (ideal_zone)
  if (!p.cond && !p.visc) {
    if (mixed)
      return launch_newton_bs<true, true>(p, K, P, iters, status, cnt, Pfb, accept, cfg, queue, qcount, rq, rs, rn, st);
    return launch_newton_bs<false, true>(p, K, P, iters, status, cnt, Pfb, accept, cfg, queue, qcount, rq, rs, rn, st);
  }
  if (mixed)
    return launch_newton_bs<true, false>(p, K, P, iters, status, cnt, Pfb, accept, cfg, queue, qcount, rq, rs, rn, st);
  return launch_newton_bs<false, false>(p, K, P, iters, status, cnt, Pfb, accept, cfg, queue, qcount, rq, rs, rn, st);
}

cudaError_t launch_newton(const Params& p, int mixed, const double* K, double* P, uint8_t* iters, uint8_t* status,
                          Counters* cnt, cudaStream_t st) {
  const NewtonCfg cfg{64, 1 << 30, false};
  return launch_newton_fb(p, mixed, K, P, iters, status, cnt, nullptr, 0.0, cfg, nullptr, nullptr, nullptr, Rescue{}, nullptr,
                          st);
}

cudaError_t launch_residual(const Params& p, const double* K, const double* Pk, int scaled, double dts, double* R,
                            cudaStream_t st) {
  const int bs = 128;
  const long long nb = (p.N + bs - 1) / bs;
  residual_once<<<(unsigned)nb, bs, 0, st>>>(p, K, Pk, scaled, dts, R);
  return cudaGetLastError();
}

cudaError_t launch_rcp_check(int n, unsigned long long seed, double* worst, cudaStream_t st) {
  rcp_check<<<(n + 255) / 256, 256, 0, st>>>(n, seed, worst);
  return cudaGetLastError();
}

}  // namespace grim

// ============================================================================
// General metric (3-D grids and modified Kerr-Schild): the same Newton
// iteration on the residual in a general metric.  The zone's metric (g_{mu
// nu}, alpha, g^{ti}) comes from the centre table and sits in shared memory
// beside the zone constants.  The FD Jacobian recomputes the whole state per
// column (no structural specialisation), with the same step rule.
#include "grim_gr.cuh"

namespace grim {

constexpr int NMET = 14;  // g_{mu nu} (10), alpha, g^{ti} (3)

template <typename T, int BS> __device__ __forceinline__ Met<T> met_smem(const double* md) {
  Met<T> m;
#pragma unroll
  for (int a = 0; a < 10; a++) m.gcov[a] = from_double<T>(md[a * BS]);
  m.alpha = from_double<T>(md[10 * BS]);
#pragma unroll
  for (int i = 0; i < 3; i++) m.gti[i] = from_double<T>(md[(11 + i) * BS]);
  return m;
}

// Scaled residual of the stage in a general metric: r_a = kU_a U~_a(P) + kC_a
// with U~ = U/sqrt(-g), plus the implicit relaxation terms of the q~ and dP~
// rows in Theta, u_mu and u^t.
template <typename T, class KA> __device__ __forceinline__ void r_all_gr(const ZG<T>& z, const KA& k, T r[NV]) {
  T U[NV];
  zg_conserved(z, U);
#pragma unroll
  for (int a = 0; a < NV; a++) r[a] = k(K_U + a) * U[a] + k(K_C + a);
  T h = k(K_Q + 0) * z.qt + k(K_Q + 1) * z.theta + k(K_Q + 6) * z.ucon[0];
  T d = k(K_D + 0) * z.dpt + k(K_D + 5) * z.ucon[0];
#pragma unroll
  for (int m = 0; m < 4; m++) {
    h += k(K_Q + 2 + m) * z.ucov[m];
    d += k(K_D + 1 + m) * z.ucov[m];
  }
  r[8] += h;
  r[9] += d;
}

// Column steps: the FP64 Jacobian uses the step rule of Section 3.1
// (fd_step; relative for rho and u).  The float32 Jacobian (SCALED) takes h_j = eps (|P_j| + s_j)
// with the natural scale of each component: s = 0 for rho and u (their step
// is relative; the torus atmosphere holds rho ~ 1e-7, u ~ 1e-10, where an
// absolute float32 step would jump by orders of magnitude), 1/sqrt(g_jj)
// for the velocity u~^j (unit proper speed), sqrt(rho) for B^i, q~ and dP~
// (field-like: they enter the stress as squares over rho).
template <typename T, bool CENTRAL, bool SCALED, int BS, class KA>
__device__ __forceinline__ void fd_jacobian_gr(const T P[NV], const T r[NV], const KA& k, const Met<T>& m,
                                               const RC<T>& c, T eps, T* J, bool five = false) {
  T sfield = T(0);
  if (SCALED) sfield = sqr_root(fabs(P[0]));
#pragma unroll 1
  for (int mc = 0; mc < (five ? 5 : 7); mc++) {  // the non-magnetic columns (see fd_jacobian)
    const int col = nb7(mc);
    T Pe[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) Pe[a] = P[a];
    const T pj = P[col];
    T pe;
    if (SCALED) {
      T s = sfield;
      if (col <= 1) s = T(0);
      else if (col <= 4) s = rsq(m.gcov[sym(col - 1, col - 1)]);
      pe = pj + eps * (fabs(pj) + s);
    } else {
      pe = fd_step(pj, eps, col <= 1);
    }
    const T hstep = pe - pj;
    Pe[col] = pe;
    ZG<T> z;
    zg_load(z, Pe, m, c);
    T rp[NV];
    r_all_gr(z, k, rp);
    if (!CENTRAL) {
      const T ih = nr_rcp(hstep);
#pragma unroll
      for (int i = 0; i < NV; i++)
        if (jslot(i) >= 0) J[(jslot(i) * NJ + mc) * BS] = (rp[i] - r[i]) * ih;
    } else {
      Pe[col] = pj - hstep;
      zg_load(z, Pe, m, c);
      T rm[NV];
      r_all_gr(z, k, rm);
      const T ih = T(0.5) * nr_rcp(hstep);
#pragma unroll
      for (int i = 0; i < NV; i++)
        if (jslot(i) >= 0) J[(jslot(i) * NJ + mc) * BS] = (rp[i] - rm[i]) * ih;
    }
  }
}

// rq, rs: the zone's residual slot for the queue; Pfb, accept_bits,
// fellback: the plain start of a learned start; both as in newton_zone.
template <bool MIXED, int BS, bool IDEAL>
__device__ ZoneResult newton_zone_gr(const Params& p, const double* kd, const float* kf, const double* md,
                                     double P[NV], void* jac, int k0, int kstop, double* rq, long long rs,
                                     const double* Pfb, long long fb_stride, unsigned long long accept_bits,
                                     bool& fellback, const float* rn = nullptr) {
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
  const RC<double> c64 = make_rc<double>(p);
  const KSm<double, BS> k64{kd};
  const Met<double> m64 = met_smem<double, BS>(md);
  const unsigned long long tol_bits = abits(p.tol);
  ZG<double> z;
  double r[NV];
  bool zvalid = false;  // z holds the state of P
  if (rq && k0 > 0) {
#pragma unroll
    for (int a = 0; a < NV; a++) r[a] = rq[a * rs];
  } else {
    zg_load(z, P, m64, c64);
    zvalid = true;
    r_all_gr(z, k64, r);
    o.evals64++;
  }
  double f = sum_sq10(r);
  fellback = false;
  if (Pfb && !(max_abits10(r) <= accept_bits) && !learned_wins(f, rn, fb_stride)) {
    double Pp[NV], rp[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) Pp[a] = (a >= 5 && a <= 7) ? P[a] : Pfb[a * fb_stride];
    ZG<double> zp;
    zg_load(zp, Pp, m64, c64);
    r_all_gr(zp, k64, rp);
    o.evals64++;
    const double fp = sum_sq10(rp);
    if (!(f <= fp)) {
      fellback = true;
      zvalid = false;
#pragma unroll
      for (int a = 0; a < NV; a++) { P[a] = Pp[a]; r[a] = rp[a]; }
      f = fp;
    }
  }
  const bool five = IDEAL && ideal_zone(p, P, r);
  int k = k0;
  for (;;) {
    if (!finite_bits(f)) { o.status |= ST_NONFINITE; break; }
    if (max_abits10(r) <= tol_bits) break;
    if (k >= p.kmax) { o.status |= ST_MAXIT; break; }
    if (k >= kstop) { o.pending = true; break; }
    double dP[NV];
    bool ok;
    if (!MIXED) {
      double* J = (double*)jac + threadIdx.x;
      double* b = J + NJ * NJ * BS;
      fd_jacobian_gr<double, false, false, BS>(P, r, k64, m64, c64, p.eps64, J, five);
      o.evals64 += five ? 5 : 7;
#pragma unroll
      for (int m = 0; m < NJ; m++) b[m * BS] = -r[nb7(m)];
      ok = five ? lu_solve_block_smem<double, BS, 5>(J, b, dP) : lu_solve_block_smem<double, BS, 7>(J, b, dP);
      o.lu64++;
    } else {
      const RC<float> c32 = make_rc<float>(p);
      const KSm<float, BS> k32{kf};
      const Met<float> m32 = met_smem<float, BS>(md);
      float* J = (float*)jac + threadIdx.x;
      float* b = J + NJ * NJ * BS;
      float Pf[NV], rf[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pf[a] = d2f_jac(P[a]);
      ZG<float> zf;
      zg_load(zf, Pf, m32, c32);
      r_all_gr(zf, k32, rf);
      const int ncol = five ? 5 : 7;
      if (p.fd32c) {
        fd_jacobian_gr<float, true, true, BS>(Pf, rf, k32, m32, c32, p.eps32, J, five);
        o.evals32 += 2 * ncol + 1;
      } else {
        fd_jacobian_gr<float, false, true, BS>(Pf, rf, k32, m32, c32, p.eps32, J, five);
        o.evals32 += ncol + 1;
      }
#pragma unroll
      for (int m = 0; m < NJ; m++) b[m * BS] = d2f_jac(-r[nb7(m)]);
      float df[NV];
      ok = five ? lu_solve_block_smem<float, BS, 5>(J, b, df) : lu_solve_block_smem<float, BS, 7>(J, b, df);
      // a float32 solve that overflowed or met a NaN pivot has no direction:
      // the zone is reported singular, not moved by a huge step
#pragma unroll
      for (int i = 0; i < NV; i++) ok = ok && isfinite(df[i]);
#pragma unroll
      for (int i = 0; i < NV; i++) dP[i] = f2d_jac(df[i]);
      o.lu32++;
    }
    if (!ok) { o.status |= ST_SINGULAR; break; }
    double lam = 1.0, Pt[NV], rt[NV], ft = 0.0;
    for (int t = 0;; t++) {
#pragma unroll
      for (int a = 0; a < NV; a++) Pt[a] = fma(lam, dP[a], P[a]);
      zg_load(z, Pt, m64, c64);
      r_all_gr(z, k64, rt);
      o.evals64++;
      ft = sum_sq10(rt);
      const bool fin = finite_bits(ft);
      const double lim = 1.0 - 1e-4 * lam;
      if (fin && ft < f * lim * lim) break;
      if (t >= p.lsmax) { o.status |= ST_LSSTALL; break; }
      // the quadratic model's minimiser when it is a positive finite number,
      // else half the step (a non-finite trial, or an overflowed denominator
      // that would leave lambda = 0 and then 0/0)
      const double ln = fin ? f * lam * lam / (ft + (2.0 * lam - 1.0) * f) : 0.0;
      lam = (ln > 0.0 && finite_bits(ln)) ? ln : 0.5 * lam;
    }
#pragma unroll
    for (int a = 0; a < NV; a++) { P[a] = Pt[a]; r[a] = rt[a]; }
    f = ft;
    zvalid = true;
    k++;
  }
  o.iters = k;
  o.done = k - k0;
  o.res = __longlong_as_double((long long)max_abits10(r));
  if (!(P[0] > 0.0) || !(P[1] > 0.0)) o.status |= ST_INADMISSIBLE;
  if (p.floors && p.visc && !o.pending && o.status == 0) {
    // what the anisotropy clamp of the floors needs of the final state
    if (!zvalid) zg_load(z, P, m64, c64);
    o.bsq = z.bsq;
    o.ds = z.ds;
  }
  if (o.pending && rq) {
#pragma unroll
    for (int a = 0; a < NV; a++) rq[a * rs] = r[a];
  }
  return o;
}

// The floors of a converged zone, in the kernel that finishes it (a failed
// zone keeps its status and is reverted and floored by floors_gr): rho >=
// 1e-5 r^{-3/2}, u >= 1e-7 r^{-5/2}, then -b^2 <= dP <= b^2/2 on the physical
// anisotropy dP = dP~ ds, with b^2 and ds of the final state.  b^2 depends
// on B and u^i only, so the floors of rho and u leave it; ds = (psi gamma)^(1/2)
// P_g (rho + gamma u)^(-1/2) is recomputed where they moved rho or u.
__device__ __forceinline__ void floors_converged(const Params& p, const double* gc, long long z, const ZoneResult& o,
                                                 double P[NV]) {
  const int i = (int)(z % p.n1), j = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
  const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
  const double r = __ldg(gc + G_R * nc + (long long)(j + 1) * (p.n1 + 2) + (i + 1));
  const double rho = fmax(P[0], 1e-5 / (r * sqrt(r)));
  const double u = fmax(P[1], 1e-7 / (r * r * sqrt(r)));
  const bool moved = rho != P[0] || u != P[1];
  P[0] = rho;
  P[1] = u;
  if (!p.visc) return;
  double f = o.ds;
  if (moved) {
    const RC<double> c = make_rc<double>(p);
    f = c.spsig * (c.gm1 * u) * rsq(rho + c.gam * u);
  }
  if (f > 0.0) {
    const double dP = P[9] * f, hi = 0.5 * o.bsq, lo = -o.bsq;
    if (dP > hi) P[9] = hi / f;
    else if (dP < lo) P[9] = lo / f;
  }
}

template <bool MIXED, int BS> struct NewtonSmemGr {
  static constexpr size_t kd = sizeof(double) * NK * BS;
  static constexpr size_t md = sizeof(double) * NMET * BS;
  static constexpr size_t kf = MIXED ? sizeof(float) * NK * BS : 0;
  static constexpr size_t jac = (MIXED ? sizeof(float) : sizeof(double)) * (NJ * NJ + NJ) * BS;
  static constexpr size_t bytes = kd + md + kf + jac;
};

// Zone z's constants and metric into shared memory (this thread's column).
template <bool MIXED, int BS>
__device__ __forceinline__ void load_zone_gr(const Params& p, const double* K, const double* gc, long long z,
                                             double* kd, float* kf, double* md) {
  const long long N = p.N;
#pragma unroll
  for (int a = 0; a < NK; a++) {
    const double x = __ldg(K + a * N + z);
    kd[a * BS] = x;
    if (MIXED) kf[a * BS] = d2f_jac(x);
  }
  const int i = (int)(z % p.n1), j = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
  const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
  const double* g = gc + (long long)(j + 1) * (p.n1 + 2) + (i + 1);
#pragma unroll
  for (int a = 0; a < 10; a++) md[a * BS] = __ldg(g + (G_COV + a) * nc);
  md[10 * BS] = __ldg(g + G_ALPHA * nc);
#pragma unroll
  for (int q = 0; q < 3; q++) md[(11 + q) * BS] = __ldg(g + (G_CON + sym(0, q + 1)) * nc);
}

template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_dense_gr(const __grid_constant__ Params p, const double* __restrict__ K,
                                                      const double* __restrict__ gc, double* __restrict__ P,
                                                      uint8_t* __restrict__ iters, uint8_t* __restrict__ status,
                                                      Counters* __restrict__ cnt, int kstop, int* __restrict__ queue,
                                                      int* __restrict__ qcount, double* __restrict__ rq,
                                                      const double* __restrict__ Pfb, double accept,
                                                      int* __restrict__ rqueue, int* __restrict__ rcount,
                                                      const float* __restrict__ rn) {
  using S = NewtonSmemGr<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  double* md = (double*)(smem_raw + S::kd) + threadIdx.x;
  float* kf = (float*)(smem_raw + S::kd + S::md) + threadIdx.x;
  void* jac = smem_raw + S::kd + S::md + S::kf;
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * BS + threadIdx.x;
  const bool active = z < N;
  ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
  bool fellback = false;
  if (active) {
    load_zone_gr<MIXED, BS>(p, K, gc, z, kd, kf, md);
    double Pz[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z];
    o = newton_zone_gr<MIXED, BS, IDEAL>(p, kd, kf, md, Pz, jac, 0, kstop < p.kmax ? kstop : p.kmax,
                                  queue && rq ? rq + z : nullptr, N, Pfb ? Pfb + z : nullptr, N, abits(accept),
                                  fellback, Pfb && rn ? rn + z : nullptr);
    if (p.floors && !o.pending && o.status == 0) floors_converged(p, gc, z, o, Pz);
#pragma unroll
    for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
    iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
    status[z] = (uint8_t)o.status;
  }
  if (queue) enqueue(queue, qcount, active && o.pending, z);
  if (MIXED && rqueue) to_rescue(rqueue, rcount, o, active, z);
  accumulate(cnt, o, active, fellback);
}

// newton_dense_gr in rounds of one update with the block's unconverged
// zones packed between rounds (see newton_rounds); the metric of a zone
// stays in its column of shared memory like its constants.
template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_rounds_gr(const __grid_constant__ Params p, const double* __restrict__ K,
                                                       const double* __restrict__ gc, double* __restrict__ P,
                                                       uint8_t* __restrict__ iters, uint8_t* __restrict__ status,
                                                       Counters* __restrict__ cnt, int kstop, int* __restrict__ queue,
                                                       int* __restrict__ qcount, double* __restrict__ rq,
                                                       const double* __restrict__ Pfb, double accept,
                                                       int* __restrict__ rqueue, int* __restrict__ rcount,
                                                       const float* __restrict__ rn) {
  using S = NewtonSmemGr<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int wsum[BS / 32];
  double* kd = (double*)smem_raw;
  double* md = (double*)(smem_raw + S::kd);
  float* kf = (float*)(smem_raw + S::kd + S::md);
  void* jac = smem_raw + S::kd + S::md + S::kf;
  const Staging stg = Staging::at<BS>(jac);
  const long long N = p.N;
  const long long z0 = (long long)blockIdx.x * BS;
  const int t = threadIdx.x;
  const int ks = kstop < p.kmax ? kstop : p.kmax;
  const unsigned long long acc = abits(accept);
  bool own = z0 + t < N;
  int sl = t, k = 0;
  double Pz[NV], rz[NV];
  if (own) {
    load_zone_gr<MIXED, BS>(p, K, gc, z0 + t, kd + t, kf + t, md + t);
#pragma unroll
    for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z0 + t];
  }
  Tally tl;
  for (int round = 0;; round++) {
    const long long z = z0 + sl;
    bool go = false, resc = false;
    if (own) {
      bool fb = false;
      ZoneResult o = newton_zone_gr<MIXED, BS, IDEAL>(p, kd + sl, kf + sl, md + sl, Pz, jac, k, k + 1, rz, 1,
                                                      round == 0 && Pfb ? Pfb + z : nullptr, N, acc, fb,
                                                      round == 0 && Pfb && rn ? rn + z : nullptr);
      tl.work(o);
      tl.fb += fb;
      k = o.iters;
      go = o.pending;
      if (!go) {
        if (p.floors && o.status == 0) floors_converged(p, gc, z, o, Pz);
#pragma unroll
        for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
        iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
        status[z] = (uint8_t)o.status;
        if (MIXED && rqueue && o.status != 0) resc = true;  // finished by the rescue kernel
        else tl.finish(cnt, o);
      }
    }
    if (MIXED && rqueue) enqueue(rqueue, rcount, resc, z);
    int n = 0;
    const int rank = block_rank<BS>(go, wsum, n);
    if (n == 0) break;
    if (round + 1 >= ks) {
      // unconverged after ks updates: on to the queue kernel
      if (go) {
#pragma unroll
        for (int a = 0; a < NV; a++) {
          P[a * N + z] = Pz[a];
          if (rq) rq[a * N + z] = rz[a];
        }
        iters[z] = (uint8_t)k;
      }
      enqueue(queue, qcount, go, z);
      break;
    }
    if (n > BS - 32) {
      // packing would free no warp: every zone stays with its thread
      own = go;
      continue;
    }
    if (go) stg.put<BS>(rank, Pz, rz, sl, k);
    __syncthreads();
    own = t < n;
    if (own) stg.get<BS>(t, Pz, rz, sl, k);
    __syncthreads();
  }
  tl.flush(cnt);
}

template <bool MIXED, int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_queue_gr(const __grid_constant__ Params p, const double* __restrict__ K,
                                                      const double* __restrict__ gc, double* __restrict__ P,
                                                      uint8_t* __restrict__ iters, uint8_t* __restrict__ status,
                                                      Counters* __restrict__ cnt, const int* __restrict__ queue,
                                                      const int* __restrict__ qcount, double* __restrict__ rq,
                                                      int* __restrict__ rqueue, int* __restrict__ rcount) {
  using S = NewtonSmemGr<MIXED, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  double* md = (double*)(smem_raw + S::kd) + threadIdx.x;
  float* kf = (float*)(smem_raw + S::kd + S::md) + threadIdx.x;
  void* jac = smem_raw + S::kd + S::md + S::kf;
  const long long N = p.N;
  const int count = *qcount;
  for (int base = blockIdx.x * BS; base < count; base += gridDim.x * BS) {
    const int q = base + (int)threadIdx.x;
    const bool active = q < count;
    ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
    if (active) {
      const long long z = queue[q];
      load_zone_gr<MIXED, BS>(p, K, gc, z, kd, kf, md);
      double Pz[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pz[a] = P[a * N + z];
      bool fb = false;
      o = newton_zone_gr<MIXED, BS, IDEAL>(p, kd, kf, md, Pz, jac, iters[z], p.kmax, rq ? rq + z : nullptr, N, nullptr,
                                           N, 0ull, fb);
      if (p.floors && o.status == 0) floors_converged(p, gc, z, o, Pz);
#pragma unroll
      for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
      iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
      status[z] = (uint8_t)o.status;
    }
    if (MIXED && rqueue) to_rescue(rqueue, rcount, o, active, active ? queue[q] : 0);
    accumulate(cnt, o, active, false);
  }
}

// The rescue of the general-metric mixed solver (see newton_rescue).
template <int BS, bool IDEAL>
__global__ void __launch_bounds__(BS) newton_rescue_gr(const __grid_constant__ Params p,
                                                       const double* __restrict__ K, const double* __restrict__ gc,
                                                       const double* __restrict__ Pn, double* __restrict__ P,
                                                       uint8_t* __restrict__ iters, uint8_t* __restrict__ status,
                                                       Counters* __restrict__ cnt, const int* __restrict__ rqueue,
                                                       const int* __restrict__ rcount) {
  using S = NewtonSmemGr<false, BS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* kd = (double*)smem_raw + threadIdx.x;
  double* md = (double*)(smem_raw + S::kd) + threadIdx.x;
  void* jac = smem_raw + S::kd + S::md;
  const long long N = p.N;
  const int count = *rcount;
  for (int base = blockIdx.x * BS; base < count; base += gridDim.x * BS) {
    const int q = base + (int)threadIdx.x;
    const bool active = q < count;
    ZoneResult o = {0, 0, 0, 0, 0, 0, 0, false, 0.0};
    if (active) {
      const long long z = rqueue[q];
      load_zone_gr<false, BS>(p, K, gc, z, kd, nullptr, md);
      double Pz[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) Pz[a] = (a >= 5 && a <= 7) ? P[a * N + z] : __ldg(Pn + a * N + z);
      bool fb = false;
      o = newton_zone_gr<false, BS, IDEAL>(p, kd, nullptr, md, Pz, jac, 0, p.kmax, nullptr, N, nullptr, N, 0ull, fb);
      if (p.floors && o.status == 0) floors_converged(p, gc, z, o, Pz);
#pragma unroll
      for (int a = 0; a < NV; a++) P[a * N + z] = Pz[a];
      iters[z] = (uint8_t)(o.iters < 255 ? o.iters : 255);
      status[z] = (uint8_t)o.status;
    }
    accumulate(cnt, o, active, false);
    const unsigned m = __ballot_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&cnt->rescued, (unsigned long long)__popc(m));
  }
}

template <int BS, bool IDEAL> struct RescueKernelsGr {
  using S = NewtonSmemGr<false, BS>;
  static cudaError_t launch(const Params& p, const double* K, const double* gc, double* P, uint8_t* iters,
                            uint8_t* status, Counters* cnt, const Rescue& rs, cudaStream_t st) {
    static PerDevice once;
    int grid = 0;
    cudaError_t e = once.get(
        [](int* g) {
          cudaError_t r = cudaFuncSetAttribute(newton_rescue_gr<BS, IDEAL>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          int dev = 0, sms = 0;
          if (r == cudaSuccess) r = cudaGetDevice(&dev);
          if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          // rescued zones are rare: one block per SM keeps the launch of an
          // empty queue cheap
          if (r == cudaSuccess) *g = sms;
          return r;
        },
        &grid);
    if (e != cudaSuccess) return e;
    newton_rescue_gr<BS, IDEAL><<<(unsigned)grid, BS, S::bytes, st>>>(p, K, gc, rs.Pn, P, iters, status, cnt,
                                                                       rs.queue, rs.count);
    return cudaGetLastError();
  }
};

// Scaled (or raw) residual at Pk, general metric.
__global__ void residual_once_gr(const __grid_constant__ Params p, const double* __restrict__ K,
                                 const double* __restrict__ gc, const double* __restrict__ Pk, int scaled,
                                 double dts, double* __restrict__ R) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const KGl kg{K + z, N};
  const RC<double> c = make_rc<double>(p);
  const int i = (int)(z % p.n1), j = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
  const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
  const double* g = gc + (long long)(j + 1) * (p.n1 + 2) + (i + 1);
  Met<double> m;
#pragma unroll
  for (int a = 0; a < 10; a++) m.gcov[a] = __ldg(g + (G_COV + a) * nc);
  m.alpha = __ldg(g + G_ALPHA * nc);
#pragma unroll
  for (int q = 0; q < 3; q++) m.gti[q] = __ldg(g + (G_CON + sym(0, q + 1)) * nc);
  const double sg = __ldg(g + G_SQRTG * nc);
  double Pz[NV], r[NV];
#pragma unroll
  for (int a = 0; a < NV; a++) Pz[a] = Pk[a * N + z];
  ZG<double> zz;
  zg_load(zz, Pz, m, c);
  r_all_gr(zz, kg, r);
#pragma unroll
  for (int a = 0; a < NV; a++) {
    // the row weight is sqrt(-g) s_a / dt_s; divide out s_a / dt_s for the raw residual
    R[a * N + z] = scaled ? r[a] : r[a] * sg / (kg(K_U + a) * dts);
  }
}

template <bool MIXED, int BS, bool IDEAL> struct NewtonKernelsGr {
  using S = NewtonSmemGr<MIXED, BS>;
  // the kernels' shared-memory limit and the queue kernel's persistent grid
  // (SMs x resident blocks), once per device
  static cudaError_t configure(int& qgrid) {
    static PerDevice once;
    return once.get(
        [](int* grid) {
          cudaError_t e = cudaFuncSetAttribute(newton_dense_gr<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_rounds_gr<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(newton_queue_gr<MIXED, BS, IDEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
          int dev = 0, sms = 0, per_sm = 0;
          if (e == cudaSuccess) e = cudaGetDevice(&dev);
          if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_queue_gr<MIXED, BS, IDEAL>, BS, S::bytes);
          if (e == cudaSuccess) *grid = sms * (per_sm > 0 ? per_sm : 1);
          return e;
        },
        &qgrid);
  }
  static cudaError_t launch(const Params& p, const double* K, const double* gc, double* P, uint8_t* iters,
                            uint8_t* status, Counters* cnt, int kcut, bool rounds, int* queue, int* qcount,
                            double* rq, const double* Pfb, double accept, const Rescue& rs, const float* rn,
                            cudaStream_t st) {
    int qgrid = 0;
    cudaError_t e = configure(qgrid);
    if (e != cudaSuccess) return e;
    const bool compact = queue && qcount && kcut < p.kmax;
    const bool rescue = MIXED && rs.queue && rs.count && rs.Pn;
    if (compact && (e = cudaMemsetAsync(qcount, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (rescue && (e = cudaMemsetAsync(rs.count, 0, sizeof(int), st)) != cudaSuccess) return e;
    int* rqueue = rescue ? rs.queue : nullptr;
    const long long nb = (p.N + BS - 1) / BS;
    if (rounds)
      newton_rounds_gr<MIXED, BS, IDEAL><<<(unsigned)nb, BS, S::bytes, st>>>(p, K, gc, P, iters, status, cnt,
                                                                       compact ? kcut : p.kmax,
                                                                       compact ? queue : nullptr, qcount, rq, Pfb,
                                                                       accept, rqueue, rs.count, rn);
    else
      newton_dense_gr<MIXED, BS, IDEAL><<<(unsigned)nb, BS, S::bytes, st>>>(p, K, gc, P, iters, status, cnt,
                                                                      compact ? kcut : p.kmax,
                                                                      compact ? queue : nullptr, qcount, rq, Pfb,
                                                                      accept, rqueue, rs.count, rn);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (compact) {
      newton_queue_gr<MIXED, BS, IDEAL><<<(unsigned)qgrid, BS, S::bytes, st>>>(p, K, gc, P, iters, status, cnt,
                                                                               queue, qcount, rq, rqueue, rs.count);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (rescue) return RescueKernelsGr<BS, IDEAL>::launch(p, K, gc, P, iters, status, cnt, rs, st);
    return cudaSuccess;
  }
};

// Newton solves of one stage in a general metric (block size 32 or 64).
// rq, Pfb, accept: as in launch_newton_fb.
template <bool IDEAL>
static cudaError_t launch_newton_gr_i(const Params& p, int mixed, const double* K, const double* gc, double* P,
                                     uint8_t* iters, uint8_t* status, Counters* cnt, const NewtonCfg& cfg,
                                     int* queue, int* qcount, double* rq, const double* Pfb, double accept,
                                     const Rescue& rs, const float* rn, cudaStream_t st) {
  const bool b32 = cfg.bs == 32;
  if (mixed) {
    if (b32)
      return NewtonKernelsGr<true, 32, IDEAL>::launch(p, K, gc, P, iters, status, cnt, cfg.kcut, cfg.rounds, queue, qcount, rq,
                                                      Pfb, accept, rs, rn, st);
    return NewtonKernelsGr<true, 64, IDEAL>::launch(p, K, gc, P, iters, status, cnt, cfg.kcut, cfg.rounds, queue, qcount, rq,
                                                    Pfb, accept, rs, rn, st);
  }
  if (b32)
    return NewtonKernelsGr<false, 32, IDEAL>::launch(p, K, gc, P, iters, status, cnt, cfg.kcut, cfg.rounds, queue, qcount, rq,
                                                     Pfb, accept, rs, rn, st);
  return NewtonKernelsGr<false, 64, IDEAL>::launch(p, K, gc, P, iters, status, cnt, cfg.kcut, cfg.rounds, queue, qcount, rq,
                                                   Pfb, accept, rs, rn, st);
}

cudaError_t launch_newton_gr(const Params& p, int mixed, const double* K, const double* gc, double* P,
                             uint8_t* iters, uint8_t* status, Counters* cnt, const NewtonCfg& cfg, int* queue,
                             int* qcount, double* rq, const double* Pfb, double accept, const Rescue& rs,
                             const float* rn, cudaStream_t st) {
  // ideal MHD: the kernels that may take the 5x5 block (ideal_zone)
  if (!p.cond && !p.visc)
    return launch_newton_gr_i<true>(p, mixed, K, gc, P, iters, status, cnt, cfg, queue, qcount, rq, Pfb, accept, rs, rn,
                                    st);
  return launch_newton_gr_i<false>(p, mixed, K, gc, P, iters, status, cnt, cfg, queue, qcount, rq, Pfb, accept, rs, rn,
                                   st);
}

// Learned-start features in a general metric, in the flat path's layout:
// x_a = -r_a(P_n) (the scaled residual of the stage at its start, from the
// stage constants K), the zone's g_{mu nu} (10, packed), P_n (10, in the
// learned start's units: log rho, log u, q~ and dP~ over |X| + rho), two
// zeros.  X (row-major [N][32]) and, with Y, the targets P_conv - P_n of
// the predicted fields ([N][16]) for training; or the ten x_a alone into
// feat ([10][N]) for inference.
__global__ void features_gr(const __grid_constant__ Params p, const double* __restrict__ K,
                            const double* __restrict__ gc, const double* __restrict__ Pn,
                            const double* __restrict__ Pc, float* __restrict__ X, float* __restrict__ Y,
                            float* __restrict__ feat) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const KGl kg{K + z, N};
  const RC<double> c = make_rc<double>(p);
  const int i = (int)(z % p.n1), j = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
  const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
  const double* g = gc + (long long)(j + 1) * (p.n1 + 2) + (i + 1);
  Met<double> m;
#pragma unroll
  for (int a = 0; a < 10; a++) m.gcov[a] = __ldg(g + (G_COV + a) * nc);
  m.alpha = __ldg(g + G_ALPHA * nc);
#pragma unroll
  for (int q = 0; q < 3; q++) m.gti[q] = __ldg(g + (G_CON + sym(0, q + 1)) * nc);
  double P[NV], r[NV];
#pragma unroll
  for (int a = 0; a < NV; a++) P[a] = __ldg(Pn + a * N + z);
  ZG<double> zz;
  zg_load(zz, P, m, c);
  r_all_gr(zz, kg, r);
  if (feat) {
#pragma unroll
    for (int a = 0; a < NV; a++) feat[a * N + z] = (float)(-r[a]);
  }
  if (X) {
    float* x = X + z * 32;
#pragma unroll
    for (int a = 0; a < NV; a++) {
      x[a] = (float)(-r[a]);
      x[NV + a] = (float)m.gcov[a];
      x[2 * NV + a] = mlp_pn_feature(a, P[a], P[0]);
    }
    x[30] = 0.f;
    x[31] = 0.f;
    if (Y) {
      float* y = Y + z * 16;
#pragma unroll
      for (int o = 0; o < 16; o++)
        y[o] = (o < NV && !(o >= 5 && o <= 7)) ? mlp_target(o, __ldg(Pc + o * N + z), P[o], P[0]) : 0.f;
    }
  }
}

cudaError_t launch_features_gr(const Params& p, const double* K, const double* gc, const double* Pn, const double* Pc,
                               float* X, float* Y, float* feat, cudaStream_t st) {
  features_gr<<<(unsigned)((p.N + 127) / 128), 128, 0, st>>>(p, K, gc, Pn, Pc, X, Y, feat);
  return cudaGetLastError();
}

cudaError_t launch_residual_gr(const Params& p, const double* K, const double* gc, const double* Pk, int scaled,
                               double dts, double* R, cudaStream_t st) {
  residual_once_gr<<<(unsigned)((p.N + 127) / 128), 128, 0, st>>>(p, K, gc, Pk, scaled, dts, R);
  return cudaGetLastError();
}

}  // namespace grim
