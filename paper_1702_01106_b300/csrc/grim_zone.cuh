// Zone-level physics shared by the explicit and Newton kernels: math helpers
// and the intermediates of a primitive state grouped by dependence
// (thermodynamic: rho, u; kinematic: u^i; magnetic: B^i with u^i).
#pragma once
#include "grim_dev.cuh"
#include "grim_ff.cuh"

namespace grim {

// ---------------------------------------------------------------- math helpers
// Reciprocal by the Newton-Raphson iteration r <- r + r (1 - x r), started
// from the hardware approximation and applied twice (quadratic convergence
// takes its ~2^-20 relative error below 2^-53).  Checked against IEEE division
// by grim_math_selftest.
__device__ __forceinline__ double nr_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float nr_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqr_root(double x) { return sqrt(x); }
__device__ __forceinline__ float sqr_root(float x) { return sqrtf(x); }
// |x| as an unsigned integer: ordered like |x| for every non-NaN value.
__device__ __forceinline__ unsigned long long abits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned int abits(float x) { return __float_as_uint(x) & 0x7fffffffu; }
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// ---------------------------------------------------------------- reconstruction
// Generalized minmod slope (Section 2.4.1) of vm, v0, vp: sign-agreement and
// magnitude tests run on the integer bit patterns.
__device__ __forceinline__ double gm_slope(double theta, double vm, double v0, double vp) {
  const double a = v0 - vm, c = vp - v0;
  const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
  const unsigned long long bc = (unsigned long long)__double_as_longlong(c);
  const unsigned long long ma = ba & 0x7fffffffffffffffull, mc = bc & 0x7fffffffffffffffull;
  if (ma == 0 || mc == 0 || ((ba ^ bc) >> 63)) return 0.0;  // differences of opposite sign or zero
  const double m1 = theta * __longlong_as_double((long long)(ma < mc ? ma : mc));
  const double m2 = 0.5 * fabs(a + c);
  const double m = abits(m1) < abits(m2) ? m1 : m2;
  return (ba >> 63) ? -m : m;
}

// WENO5 of Jiang & Shu (1996): value at the right face of v2 from v0..v4.
__device__ __forceinline__ double weno5v(double v0, double v1, double v2, double v3, double v4) {
  const double eps = 1e-6;
  const double q0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) * (1.0 / 6.0);
  const double q1 = (-v1 + 5.0 * v2 + 2.0 * v3) * (1.0 / 6.0);
  const double q2 = (2.0 * v2 + 5.0 * v3 - v4) * (1.0 / 6.0);
  const double d0 = v0 - 2.0 * v1 + v2, e0 = v0 - 4.0 * v1 + 3.0 * v2;
  const double d1 = v1 - 2.0 * v2 + v3, e1 = v1 - v3;
  const double d2 = v2 - 2.0 * v3 + v4, e2 = 3.0 * v2 - 4.0 * v3 + v4;
  const double b0 = (13.0 / 12.0) * d0 * d0 + 0.25 * e0 * e0;
  const double b1 = (13.0 / 12.0) * d1 * d1 + 0.25 * e1 * e1;
  const double b2 = (13.0 / 12.0) * d2 * d2 + 0.25 * e2 * e2;
  const double a0 = 0.1 / ((eps + b0) * (eps + b0));
  const double a1 = 0.6 / ((eps + b1) * (eps + b1));
  const double a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// PPM (Colella & Woodward 1984) face values of the middle zone of v0..v4:
// interface values from limited slopes, a_{i+-1/2} = (a_i + a_{i+-1})/2 -+
// (da_{i+-1} - da_i)/6, then the monotonicity constraints (both faces take
// the zone value at an extremum; an overshooting parabola has its far face
// moved to 3 a_i - 2 a_near).
__device__ __forceinline__ void ppm_zone(double theta, double v0, double v1, double v2, double v3, double v4,
                                         double& lo, double& hi) {
  const double d1 = gm_slope(theta, v0, v1, v2);
  const double d2 = gm_slope(theta, v1, v2, v3);
  const double d3 = gm_slope(theta, v2, v3, v4);
  double aL = 0.5 * (v1 + v2) - (d2 - d1) * (1.0 / 6.0);
  double aR = 0.5 * (v2 + v3) - (d3 - d2) * (1.0 / 6.0);
  if (!((aR - v2) * (v2 - aL) > 0.0)) {
    aL = v2;
    aR = v2;
  } else {
    const double D = aR - aL;
    const double m6 = 6.0 * (v2 - 0.5 * (aL + aR));
    if (D * m6 > D * D) aL = 3.0 * v2 - 2.0 * aR;
    else if (D * m6 < -(D * D)) aR = 3.0 * v2 - 2.0 * aL;
  }
  lo = aL;
  hi = aR;
}

// ---------------------------------------------------------------- residual
// Constants of the residual in the working precision.
template <typename T> struct RC {
  T gam, gm1, sphig, spsig;  // gamma, gamma - 1, sqrt(phi gamma), sqrt(psi gamma)
  int cond, visc;
};
template <typename T> __device__ __forceinline__ RC<T> make_rc(const Params& p) {
  RC<T> c;
  c.gam = T(p.gamma);
  c.gm1 = T(p.gamma - 1.0);
  c.sphig = T(sqrt(p.phi * p.gamma));
  c.spsig = T(sqrt(p.psi * p.gamma));
  c.cond = p.cond;
  c.visc = p.visc;
  return c;
}

// Intermediates of the residual at one state, grouped by dependence.
template <typename T> struct Z {
  T rho, u, pg, theta, qs, ds, w0;   // thermodynamic group (rho, u)
  T iden;                            // 1/(rho + gamma u)
  T v[3], ut;                        // kinematic group (u^i): u^t = sqrt(1 + u.u)
  T iut;
  T B[3], bt, bc[3], bsq, bht, bh[3];  // magnetic group (B^i, u^i)
  T qt, dpt;
};

// P_g = (gamma-1)u, Theta = P_g/rho, and the factors that turn q~, dP~ into
// q = q~ Theta (phi c_s^2 rho)^(1/2) and dP = dP~ (psi c_s^2 P_g)^(1/2)
// (Eqs. q, dP with chi = phi c_s^2 tau_R, nu = psi c_s^2 tau_R, and
// c_s^2 = gamma P_g/(rho + gamma u)); w0 = rho + u + P_g.
template <typename T> __device__ __forceinline__ void z_thermo(Z<T>& z, const RC<T>& c) {
  const T pg = c.gm1 * z.u;
  const T ra = rsq(z.rho);               // rho^(-1/2)
  const T rb = rsq(z.rho + c.gam * z.u); // (rho + gamma u)^(-1/2)
  z.pg = pg;
  z.iden = rb * rb;
  z.theta = pg * ra * ra;
  z.qs = c.cond ? c.sphig * z.theta * sqr_root(pg) * (z.rho * ra) * rb : T(0);
  z.ds = c.visc ? c.spsig * pg * rb : T(0);
  z.w0 = z.rho + z.u + pg;
}
template <typename T> __device__ __forceinline__ void z_kin(Z<T>& z) {
  const T s = T(1) + z.v[0] * z.v[0] + z.v[1] * z.v[1] + z.v[2] * z.v[2];
  z.iut = rsq(s);
  z.ut = s * z.iut;
}
// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t, b^2, bhat = b/|b| (Section 4).
template <typename T> __device__ __forceinline__ void z_mag(Z<T>& z) {
  z.bt = z.B[0] * z.v[0] + z.B[1] * z.v[1] + z.B[2] * z.v[2];
#pragma unroll
  for (int i = 0; i < 3; i++) z.bc[i] = (z.B[i] + z.bt * z.v[i]) * z.iut;
  if constexpr (std::is_same<T, ff2>::value) {
    // the same as for ff below, with a power of two for each lane
    const float mx = fmaxf(fmaxf(fabsf(z.bt.hi.x), fabsf(z.bc[0].hi.x)), fmaxf(fabsf(z.bc[1].hi.x), fabsf(z.bc[2].hi.x)));
    const float my = fmaxf(fmaxf(fabsf(z.bt.hi.y), fabsf(z.bc[0].hi.y)), fmaxf(fabsf(z.bc[1].hi.y), fabsf(z.bc[2].hi.y)));
    float2 s, r;
    pow2_scale(mx, s.x, r.x);
    pow2_scale(my, s.y, r.y);
    const ff2 t = scale2(z.bt, s), c0 = scale2(z.bc[0], s), c1 = scale2(z.bc[1], s), c2 = scale2(z.bc[2], s);
    const ff2 q = c0 * c0 + c1 * c1 + c2 * c2 - t * t;
    z.bsq = scale2(scale2(q, r), r);
    const bool px = q.hi.x > 0.f, py = q.hi.y > 0.f;
    const ff2 ib = rsq(ff2(make_float2(px ? q.hi.x : 1.f, py ? q.hi.y : 1.f),
                           make_float2(px ? q.lo.x : 0.f, py ? q.lo.y : 0.f)));
    z.bht = keep(t * ib, px, py);
    z.bh[0] = keep(c0 * ib, px, py);
    z.bh[1] = keep(c1 * ib, px, py);
    z.bh[2] = keep(c2 * ib, px, py);
  } else if constexpr (std::is_same<T, ff>::value) {
    // b^2 of a weak field leaves the float range: b^2 and bhat from b scaled
    // by a power of two
    const float m = fmaxf(fmaxf(fabsf(z.bt.hi), fabsf(z.bc[0].hi)), fmaxf(fabsf(z.bc[1].hi), fabsf(z.bc[2].hi)));
    float s, r;
    pow2_scale(m, s, r);
    const ff t = scale2(z.bt, s), c0 = scale2(z.bc[0], s), c1 = scale2(z.bc[1], s), c2 = scale2(z.bc[2], s);
    const ff q = c0 * c0 + c1 * c1 + c2 * c2 - t * t;
    z.bsq = scale2(scale2(q, r), r);
    if (q.hi > 0.f) {
      const ff ib = rsq(q);
      z.bht = t * ib;
      z.bh[0] = c0 * ib; z.bh[1] = c1 * ib; z.bh[2] = c2 * ib;
    } else {
      z.bht = T(0);
      z.bh[0] = z.bh[1] = z.bh[2] = T(0);
    }
  } else {
    z.bsq = z.bc[0] * z.bc[0] + z.bc[1] * z.bc[1] + z.bc[2] * z.bc[2] - z.bt * z.bt;
    if (z.bsq > T(0)) {
      const T ib = rsq(z.bsq);
      z.bht = z.bt * ib;
#pragma unroll
      for (int i = 0; i < 3; i++) z.bh[i] = z.bc[i] * ib;
    } else {
      z.bht = T(0);
      z.bh[0] = z.bh[1] = z.bh[2] = T(0);
    }
  }
}
template <typename T> __device__ __forceinline__ void z_load(Z<T>& z, const T* P, const RC<T>& c) {
  z.rho = P[0]; z.u = P[1];
  z.v[0] = P[2]; z.v[1] = P[3]; z.v[2] = P[4];
  z.B[0] = P[5]; z.B[1] = P[6]; z.B[2] = P[7];
  z.qt = P[8]; z.dpt = P[9];
  z_thermo(z, c);
  z_kin(z);
  z_mag(z);
}

}  // namespace grim
