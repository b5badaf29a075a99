// Point physics in a general metric (Section 4 with the geometry of Section
// 2.1), for the 3-D and curved-space path.  The metric at a point comes from
// precomputed tables (geometry_tables in grim_gr.cu); everything here is
// per point.
//
// Primitive velocity: the normal-observer velocity u~^i, so that u^t =
// gamma/alpha and u^i = u~^i - gamma alpha g^{ti} with gamma = (1 + g_ij u~^i
// u~^j)^(1/2) (equal to u^i in Minkowski space).
#pragma once
#include "grim_zone.cuh"

namespace grim {

// Packed symmetric 4x4 index: (00,01,02,03,11,12,13,22,23,33).
__host__ __device__ constexpr int sym(int m, int n) {
  const int a = m < n ? m : n, b = m < n ? n : m;
  return a == 0 ? b : a == 1 ? 3 + b : a == 2 ? 5 + b : 9;
}

// Geometry-table planes.  Zone centres: [NGC][(n2+2)(n1+2)] (one ring of
// ghost centres); X1 faces: [NGF][(n2+2)(n1+1)]; X2 faces: [NGF][(n2+1)(n1+2)].
// X3 faces share the centre geometry (the metric does not depend on X^3).
enum {
  G_COV = 0,     // g_{mu nu}, 10 packed
  G_CON = 10,    // g^{mu nu}, 10 packed
  G_SQRTG = 20,  // sqrt(-g); exactly 0 on a polar face
  G_ALPHA = 21,  // lapse 1/sqrt(-g^tt)
  NGF = 22,
  G_TAUR = 22,   // relaxation time (centres only)
  G_R = 23,      // Boyer-Lindquist / Kerr-Schild radius (1 in Minkowski space)
  G_GAM = 24,    // Gamma^l_{mu nu}: plane G_GAM + 10 l + sym(mu, nu)
  NGC = 64
};

// Metric of one point in the working precision.
template <typename T> struct Met {
  T gcov[10];
  T alpha, gti[3];   // lapse and g^{ti}
};
template <typename T, class GA> __device__ __forceinline__ void met_load(Met<T>& m, const GA& g) {
#pragma unroll
  for (int a = 0; a < 10; a++) m.gcov[a] = from_double<T>(g(G_COV + a));
  m.alpha = from_double<T>(g(G_ALPHA));
#pragma unroll
  for (int i = 0; i < 3; i++) m.gti[i] = from_double<T>(g(G_CON + sym(0, i + 1)));
}

// Intermediates of a primitive state in a general metric.
template <typename T> struct ZG {
  T rho, u, pg, theta, qs, ds, w0;   // as in Z: w0 = rho + u + P_g
  T ucon[4], ucov[4];
  T B[3], bcon[4], bcov[4], bsq, bhcon[4], bhcov[4];
  T qt, dpt;
};

template <typename T> __device__ __forceinline__ void lower(const Met<T>& m, const T v[4], T out[4]) {
#pragma unroll
  for (int a = 0; a < 4; a++) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < 4; b++) s += m.gcov[sym(a, b)] * v[b];
    out[a] = s;
  }
}

template <typename T>
__device__ __forceinline__ void zg_load(ZG<T>& z, const T* P, const Met<T>& m, const RC<T>& c) {
  z.rho = P[0];
  z.u = P[1];
  z.qt = P[8];
  z.dpt = P[9];
  // thermodynamics, as in the flat path
  const T pg = c.gm1 * z.u;
  const T ra = rsq(z.rho);
  const T rb = rsq(z.rho + c.gam * z.u);
  z.pg = pg;
  z.theta = pg * ra * ra;
  z.qs = c.cond ? c.sphig * z.theta * sqr_root(pg) * (z.rho * ra) * rb : T(0);
  z.ds = c.visc ? c.spsig * pg * rb : T(0);
  z.w0 = z.rho + z.u + pg;
  // four-velocity from the normal-observer velocity
  const T v[3] = {P[2], P[3], P[4]};
  T q = T(0);
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) q += m.gcov[sym(i + 1, j + 1)] * v[i] * v[j];
  const T lor = sqr_root(T(1) + q);
  z.ucon[0] = lor * nr_rcp(m.alpha);
#pragma unroll
  for (int i = 0; i < 3; i++) z.ucon[i + 1] = v[i] - lor * m.alpha * m.gti[i];
  lower(m, z.ucon, z.ucov);
  // b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t
  z.B[0] = P[5]; z.B[1] = P[6]; z.B[2] = P[7];
  const T bt = z.B[0] * z.ucov[1] + z.B[1] * z.ucov[2] + z.B[2] * z.ucov[3];
  const T iut = nr_rcp(z.ucon[0]);
  z.bcon[0] = bt;
#pragma unroll
  for (int i = 0; i < 3; i++) z.bcon[i + 1] = (z.B[i] + bt * z.ucon[i + 1]) * iut;
  lower(m, z.bcon, z.bcov);
  if constexpr (std::is_same<T, ff>::value) {
    // b^2 of a weak field leaves the float range: b^2 and bhat from b scaled
    // by a power of two
    float mx = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++) mx = fmaxf(mx, fmaxf(fabsf(z.bcon[a].hi), fabsf(z.bcov[a].hi)));
    float s, r;
    pow2_scale(mx, s, r);
    ff bc[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; a++) { bc[a] = scale2(z.bcon[a], s); bv[a] = scale2(z.bcov[a], s); }
    const ff q = bc[0] * bv[0] + bc[1] * bv[1] + bc[2] * bv[2] + bc[3] * bv[3];
    z.bsq = scale2(scale2(q, r), r);
    if (q.hi > 0.f) {
      const ff ib = rsq(q);
#pragma unroll
      for (int a = 0; a < 4; a++) { z.bhcon[a] = bc[a] * ib; z.bhcov[a] = bv[a] * ib; }
    } else {
#pragma unroll
      for (int a = 0; a < 4; a++) { z.bhcon[a] = T(0); z.bhcov[a] = T(0); }
    }
    return;
  }
  z.bsq = z.bcon[0] * z.bcov[0] + z.bcon[1] * z.bcov[1] + z.bcon[2] * z.bcov[2] + z.bcon[3] * z.bcov[3];
  if (z.bsq > T(0)) {
    const T ib = rsq(z.bsq);
#pragma unroll
    for (int a = 0; a < 4; a++) { z.bhcon[a] = z.bcon[a] * ib; z.bhcov[a] = z.bcov[a] * ib; }
  } else {
#pragma unroll
    for (int a = 0; a < 4; a++) { z.bhcon[a] = T(0); z.bhcov[a] = T(0); }
  }
}

// Row m of T^m_nu (Eq. fullSEtens): w u^m u_nu + p_t delta^m_nu - b^m b_nu
// + q (bhat^m u_nu + u^m bhat_nu) - dP (bhat^m bhat_nu - (delta^m_nu +
// u^m u_nu)/3), w = rho + u + P_g + b^2, p_t = P_g + b^2/2.
template <typename T> __device__ __forceinline__ void zg_stress_row(const ZG<T>& z, int m, T out[4]) {
  const T q = z.qt * z.qs, dp = z.dpt * z.ds;
  const T third = dp * tconst<T>(1.0 / 3.0);
  const T um = z.ucon[m], bm = z.bcon[m], bhm = z.bhcon[m];
  const T A = (z.w0 + z.bsq + third) * um;
  const T pt = z.pg + tconst<T>(0.5) * z.bsq + third;
#pragma unroll
  for (int n = 0; n < 4; n++) {
    T v = A * z.ucov[n] - bm * z.bcov[n] + q * (bhm * z.ucov[n] + um * z.bhcov[n]) - dp * bhm * z.bhcov[n];
    if (n == m) v += pt;
    out[n] = v;
  }
}

// Conserved variables without the sqrt(-g) factor: (rho u^t, T^t_nu, B^i,
// q~ u^t, dP~ u^t).
template <typename T> __device__ __forceinline__ void zg_conserved(const ZG<T>& z, T U[NV]) {
  U[0] = z.rho * z.ucon[0];
  zg_stress_row(z, 0, U + 1);
  U[5] = z.B[0]; U[6] = z.B[1]; U[7] = z.B[2];
  U[8] = z.qt * z.ucon[0];
  U[9] = z.dpt * z.ucon[0];
}

// Flux along X^j (j = 1..3) without sqrt(-g); induction flux b^i u^j - b^j u^i.
template <typename T> __device__ __forceinline__ void zg_flux(const ZG<T>& z, int j, T F[NV]) {
  F[0] = z.rho * z.ucon[j];
  zg_stress_row(z, j, F + 1);
#pragma unroll
  for (int i = 0; i < 3; i++) F[5 + i] = z.bcon[i + 1] * z.ucon[j] - z.bcon[j] * z.ucon[i + 1];
  F[8] = z.qt * z.ucon[j];
  F[9] = z.dpt * z.ucon[j];
}

// Grid-frame speeds along X^j of waves at +-v_max (v_max^2 = cs~^2 + vA^2 -
// cs~^2 vA^2, Section 4.1): roots c of (k.u)^2 = v^2 (k.k + (k.u)^2),
// k_mu = (-c, e_j), i.e. A c^2 + B c + C = 0 with A = (1-v^2)(u^t)^2 - v^2
// g^tt, B = -2((1-v^2) u^t u^j - v^2 g^tj), C = (1-v^2)(u^j)^2 - v^2 g^jj.
// kappa = cs~^2 / cs^2 (a constant of the closure).  cmin <= cmax.
__device__ __forceinline__ void zg_speeds(const ZG<double>& z, double gtt, double gtj, double gjj, int j,
                                          double gam, double kappa, double& cmin, double& cmax) {
  const double iden = 1.0 / (z.rho + gam * z.u + z.bsq);
  const double cs2 = gam * z.pg / (z.rho + gam * z.u);
  const double cs2t = kappa * cs2;
  const double vA2 = z.bsq * iden;
  const double v2 = cs2t + vA2 - cs2t * vA2;
  const double ut = z.ucon[0], uj = z.ucon[j];
  const double w = 1.0 - v2;
  const double A = w * ut * ut - v2 * gtt;
  const double B = -2.0 * (w * ut * uj - v2 * gtj);
  const double C = w * uj * uj - v2 * gjj;
  double disc = B * B - 4.0 * A * C;
  disc = disc > 0.0 ? disc : 0.0;
  const double sq = sqrt(disc);
  const double i2a = 0.5 / A;
  const double c1 = (-B + sq) * i2a, c2 = (-B - sq) * i2a;
  cmin = fmin(c1, c2);
  cmax = fmax(c1, c2);
}
// The same in float-float (the mixed solver's face states), division-free;
// kg = kappa gamma.
template <typename T>
__device__ __forceinline__ void zg_speeds_kg(const ZG<T>& z, T gtt, T gtj, T gjj, int j, T gam, T kg, T& cmin,
                                             T& cmax) {
  const T den = z.rho + gam * z.u;
  const T cs2t = kg * z.pg * nr_rcp(den);
  const T vA2 = z.bsq * nr_rcp(den + z.bsq);
  const T v2 = cs2t + vA2 - cs2t * vA2;
  const T ut = z.ucon[0], uj = z.ucon[j];
  const T w = tconst<T>(1.0) - v2;
  const T A = w * ut * ut - v2 * gtt;
  const T B = tconst<T>(-2.0) * (w * ut * uj - v2 * gtj);
  const T C = w * uj * uj - v2 * gjj;
  const T disc = fmax(B * B - tconst<T>(4.0) * A * C, tconst<T>(0.0));
  const T sq = sqr_root(disc);
  const T i2a = tconst<T>(0.5) * nr_rcp(A);
  const T c1 = (sq - B) * i2a, c2 = -((sq + B) * i2a);
  cmin = fmin(c1, c2);
  cmax = fmax(c1, c2);
}

}  // namespace grim
