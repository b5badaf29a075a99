// Explicit part of one stage (Section 2.3), 2-D, as two kernels that compute
// every face exactly once:
//
//  face_flux_2d   one thread per face: reconstruction of P^E (generalized
//                 minmod / WENO5, Section 2.4.1) on both sides, conserved
//                 variables, fluxes and the wave-speed bound of Section 4.1 on
//                 each side, the LLF combination (Section 2.4.2).  Faces of
//                 direction X1 cover i = 0..n1, j = -1..n2 and faces of X2 cover
//                 i = -1..n1, j = 0..n2: the transverse ring feeds flux-CT.
//  zone_const_2d  one thread per zone: flux-CT corner values and the B fluxes
//                 (Section 4.2), the flux divergence, the slope-limited
//                 derivatives of Theta and u_mu at P^E, the relaxation targets'
//                 explicit parts (Eqs. q0def, dP0def with Eqs. q, dP), and the
//                 NK residual constants; also the Newton initial guess.
//
// Boundary rules are applied at load time (no ghost arrays).  The face fluxes
// go through HBM (20 doubles per zone): the kernels are bound by the float64
// pipe, not by memory, so computing each face once matters more than keeping
// faces on chip.
#include <type_traits>

#include "grim_zone.cuh"

namespace grim {

__device__ __forceinline__ int map_idx(int i, int n, int lo, int hi, bool& flip) {
  if (i >= 0 && i < n) return i;
  const int bc = (i < 0) ? lo : hi;
  if (bc == BC_PERIODIC) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  if (bc == BC_OUTFLOW) return i < 0 ? 0 : n - 1;
  int m = i % (2 * n);
  if (m < 0) m += 2 * n;
  if (m >= n) {
    flip = !flip;
    return 2 * n - 1 - m;
  }
  return m;
}

// Zone (i, j) of a state with the boundary rules: its flat index and whether
// the X1 / X2 components (u^1, B^1 / u^2, B^2) flip sign.
__device__ __forceinline__ long long zone_at(const Params& p, int i, int j, bool& f1, bool& f2) {
  f1 = f2 = false;
  const int gi = map_idx(i, p.n1, p.bc[0][0], p.bc[0][1], f1);
  const int gj = map_idx(j, p.n2, p.bc[1][0], p.bc[1][1], f2);
  return (long long)gj * p.n1 + gi;
}
__device__ __forceinline__ bool comp_flips(int v, bool f1, bool f2) {
  return (f1 && (v == 2 || v == 5)) || (f2 && (v == 3 || v == 6));
}
__device__ __forceinline__ double load_comp(const double* P, long long N, long long z, int v, bool f1, bool f2) {
  const double x = __ldg(P + v * N + z);
  return comp_flips(v, f1, f2) ? -x : x;
}

// Conserved variables U and flux F^j (j = 1, 2, 3) of a face state (Eqs.
// divN_explicit, divT_explicit, induction_eqn and the q~, dP~ equations), and
// the grid-frame speeds in direction j of waves moving at +-v_max in the
// fluid frame (Section 4.1, Minkowski space): the roots cmin <= cmax of
// (u^j - c u^t)^2 (1 - v^2) = v^2 (1 - c^2).  kappa = cs~^2/c_s^2, a constant
// of the closure chi = phi c_s^2 tau_R, nu = psi c_s^2 tau_R (Eq. modcs).
// gam: gamma; kg: kappa gamma (both in the working precision).
template <int j, typename T>
__device__ __forceinline__ void side_flux(const Z<T>& z, T gam, T kg, T U[NV], T F[NV], T& cmin, T& cmax) {
  const T q = z.qt * z.qs, dp = z.dpt * z.ds;
  const T third = dp * tconst<T>(1.0 / 3.0);
  const T wt = z.w0 + z.bsq + third;
  const T A = wt * z.ut;
  const T qb = q * z.bht, dpb = dp * z.bht, qut = q * z.ut;
  const T pt = z.pg + tconst<T>(0.5) * z.bsq + third;
  U[0] = z.rho * z.ut;
  U[1] = -A * z.ut + z.bt * z.bt - tconst<T>(2.0) * qb * z.ut + dpb * z.bht + pt;
#pragma unroll
  for (int i = 0; i < 3; i++) U[2 + i] = A * z.v[i] - z.bt * z.bc[i] + qb * z.v[i] + qut * z.bh[i] - dpb * z.bh[i];
  U[5] = z.B[0]; U[6] = z.B[1]; U[7] = z.B[2];
  U[8] = z.qt * z.ut;
  U[9] = z.dpt * z.ut;
  // row j of T^mu_nu: (w + dP/3) u^j u_nu - b^j b_nu + q (bhat^j u_nu + u^j bhat_nu)
  // - dP bhat^j bhat_nu + (p_t + dP/3) delta^j_nu
  const T uj = z.v[j - 1], bj = z.bc[j - 1], bhj = z.bh[j - 1];
  const T Aj = wt * uj, qbj = q * bhj, quj = q * uj, dpbj = dp * bhj;
  F[0] = z.rho * uj;
  F[1] = -Aj * z.ut + bj * z.bt - qbj * z.ut - quj * z.bht + dpbj * z.bht;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    T t = Aj * z.v[i] - bj * z.bc[i] + qbj * z.v[i] + quj * z.bh[i] - dpbj * z.bh[i];
    if (i == j - 1) t = t + pt;
    F[2 + i] = t;
  }
#pragma unroll
  for (int i = 0; i < 3; i++) F[5 + i] = z.bc[i] * uj - bj * z.v[i];
  F[8] = z.qt * uj;
  F[9] = z.dpt * uj;
  // speeds
  const T den = z.rho + gam * z.u;
  const T vA2 = z.bsq * nr_rcp(den + z.bsq);
  const T cs2t = kg * z.pg * z.iden;
  const T v2 = cs2t + vA2 - cs2t * vA2;
  const T om = tconst<T>(1.0) - v2;
  const T Aq = om * z.ut * z.ut + v2;
  const T Bq = tconst<T>(-2.0) * om * z.ut * uj;
  const T Cq = om * uj * uj - v2;
  const T disc = fmax(Bq * Bq - tconst<T>(4.0) * Aq * Cq, tconst<T>(0.0));
  const T sq = sqr_root(disc), h = tconst<T>(0.5) * nr_rcp(Aq);  // Aq > 0
  cmax = (sq - Bq) * h;
  cmin = -((sq + Bq) * h);
}

// LLF (F^- + F^+)/2 - c_max (U^+ - U^-)/2 with c_max the largest |c| of both
// sides, or HLLE (c_R F^- + c_L F^+ - c_R c_L (U^+ - U^-))/(c_L + c_R) with
// c_R = max(c, 0), c_L = max(-c, 0) over both sides (Section 2.4.2);
// L: the left state P^-, R: the right state P^+.  Written as float64.
template <typename T>
__device__ __forceinline__ void riemann_flux(int kind, const T FL[NV], const T FR[NV], const T UL[NV], const T UR[NV],
                                             T cminL, T cmaxL, T cminR, T cmaxR, double* out, long long plane) {
  if (kind == 1) {
    const T cR = fmax(fmax(cmaxL, cmaxR), tconst<T>(0.0)), cL = fmax(-fmin(cminL, cminR), tconst<T>(0.0));
    const T iw = nr_rcp(cL + cR);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * plane] = as_double((cR * FL[v] + cL * FR[v] - cR * cL * (UR[v] - UL[v])) * iw);
  } else {
    const T cm = fmax(fmax(cmaxL, -cminL), fmax(cmaxR, -cminR));
#pragma unroll
    for (int v = 0; v < NV; v++)
      out[v * plane] = as_double(tconst<T>(0.5) * (FL[v] + FR[v]) - tconst<T>(0.5) * cm * (UR[v] - UL[v]));
  }
}

struct ExpArgs {
  const double* Pn;
  const double* PE;
  const double* guess;
  double dts;
  double idts, itau;  // 1/dt_s and 1/tau_R, once on the host
  double kappa;
  double* K;
  double* P0;
  double* F1;  // [10][(n2+2)][(n1+1)]
  double* F2;  // [10][(n2+1)][(n1+2)]
  double* Dv;  // [2][N]: Theta and u^t of P^E at every zone (derived_2d)
  // P_n cache shared by the two stages of a step: U(P_n) [10], Theta_n, u^t_n.
  // mode 0: general stage (no cache); 1: half step (P^E = P_n; writes the
  // cache); 2: full step (reads the cache and the row weights K_U the half
  // step wrote, which depend on P_n only).
  double* cache;
  int mode;
  // with a learned start: the ten increment features -r_a(P_n) of each zone
  // (float32 [10][N]), from the constants computed here
  float* feat;
  // float-float copies of gamma, gamma-1, sqrt(phi gamma), sqrt(psi gamma),
  // kappa gamma and the limiter theta (hi, lo pairs), for the float-float
  // face states and slopes
  float ffc[12];
  // float-float copies of 1/dx^1, 1/dx^2, tau_R, phi, psi, 1/tau_R, 1/dt_s,
  // 1/(dt_s tau_R) and dt_s, for the mixed solver's closure constants
  float ffz[18];
};
constexpr int NCACHE = NV + 2;

template <int D, int RECON, typename S>
__device__ __forceinline__ void face_flux_dir(const Params& p, const ExpArgs& a, int i, int j, double* out,
                                              long long plane) {
  constexpr int di = (D == 0), dj = (D == 1);
  const long long N = p.N;
  // zones along the face normal at offsets -3..2 from the zone right of the face
  constexpr bool WIDE = RECON != RECON_MC;
  constexpr int o0 = WIDE ? -3 : -2, o1 = WIDE ? 2 : 1;
  long long zz[6];
  bool fa[6], fb[6];
#pragma unroll
  for (int t = o0; t <= o1; t++) zz[t + 3] = zone_at(p, i + t * di, j + t * dj, fa[t + 3], fb[t + 3]);
  // reconstruction, then the face states in the state precision.  MC runs
  // in the state precision (the limiter is continuous in its arguments, so
  // a decision that differs from float64 at a near-tie moves the face value
  // by no more than the rounding); WENO5 and PPM run in float64.  The paired
  // form (S = ff2) reconstructs in float-float and pairs the two states.
  using SR = typename std::conditional<std::is_same<S, double>::value, double, ff>::type;
  SR Ls[NV], Rs[NV];
  ff2 P2mc[std::is_same<S, ff2>::value && RECON == RECON_MC ? NV : 1];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if constexpr (std::is_same<S, ff2>::value && RECON == RECON_MC) {
      // both zones' limited slopes in paired lanes: P^- = t1 + s_1/2 (lane
      // x), P^+ = t2 - s_2/2 (lane y)
      const ff theta(a.ffc[10], a.ffc[11]);
      ff t[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        t[k] = ff_split(__ldg(a.PE + v * N + zz[k + 1]));
        if (comp_flips(v, fa[k + 1], fb[k + 1])) t[k] = -t[k];
      }
      const ff2 sl = gm_slope2(theta, ff2(t[0], t[1]), ff2(t[1], t[2]), ff2(t[2], t[3]));
      P2mc[v] = ff2(t[1], t[2]) + scale2(sl, make_float2(0.5f, -0.5f));
    } else if constexpr (!std::is_same<S, double>::value && RECON == RECON_MC) {
      const ff theta(a.ffc[10], a.ffc[11]);
      ff t[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        t[k] = ff_split(__ldg(a.PE + v * N + zz[k + 1]));
        if (comp_flips(v, fa[k + 1], fb[k + 1])) t[k] = -t[k];
      }
      Ls[v] = t[1] + scale2(gm_slope(theta, t[0], t[1], t[2]), 0.5f);
      Rs[v] = t[2] - scale2(gm_slope(theta, t[1], t[2], t[3]), 0.5f);
    } else {
      double s[6], L, R;
#pragma unroll
      for (int t = o0; t <= o1; t++) s[t + 3] = load_comp(a.PE, N, zz[t + 3], v, fa[t + 3], fb[t + 3]);
      if (RECON == RECON_WENO5) {
        L = weno5v(s[0], s[1], s[2], s[3], s[4]);
        R = weno5v(s[5], s[4], s[3], s[2], s[1]);
      } else if (RECON == RECON_PPM) {
        double lo, hi;
        ppm_zone(p.theta, s[0], s[1], s[2], s[3], s[4], lo, hi);  // zone left of the face
        L = hi;
        ppm_zone(p.theta, s[1], s[2], s[3], s[4], s[5], lo, hi);  // zone right of the face
        R = lo;
      } else {
        L = fma(0.5, gm_slope(p.theta, s[1], s[2], s[3]), s[2]);
        R = fma(-0.5, gm_slope(p.theta, s[2], s[3], s[4]), s[3]);
      }
      Ls[v] = from_double<SR>(L);
      Rs[v] = from_double<SR>(R);
    }
  }
  if constexpr (std::is_same<S, ff2>::value) {
    // both face states in one paired instruction stream (lane x: left,
    // lane y: right); the Riemann combination takes the lanes apart
    RC<ff2> c;
    c.gam = ff2(ff(a.ffc[0], a.ffc[1]), ff(a.ffc[0], a.ffc[1]));
    c.gm1 = ff2(ff(a.ffc[2], a.ffc[3]), ff(a.ffc[2], a.ffc[3]));
    c.sphig = ff2(ff(a.ffc[4], a.ffc[5]), ff(a.ffc[4], a.ffc[5]));
    c.spsig = ff2(ff(a.ffc[6], a.ffc[7]), ff(a.ffc[6], a.ffc[7]));
    c.cond = p.cond;
    c.visc = p.visc;
    const ff2 kg(ff(a.ffc[8], a.ffc[9]), ff(a.ffc[8], a.ffc[9]));
    ff2 P2[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      if constexpr (RECON == RECON_MC) P2[v] = P2mc[v];
      else P2[v] = ff2(Ls[v], Rs[v]);
    }
    Z<ff2> z2;
    z_load(z2, P2, c);
    ff2 U2[NV], F2[NV], cmin2, cmax2;
    side_flux<D + 1>(z2, c.gam, kg, U2, F2, cmin2, cmax2);
    ff UL[NV], FL[NV], UR[NV], FR[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      UL[v] = U2[v].x(); UR[v] = U2[v].y();
      FL[v] = F2[v].x(); FR[v] = F2[v].y();
    }
    riemann_flux<ff>(p.riemann, FL, FR, UL, UR, cmin2.x(), cmax2.x(), cmin2.y(), cmax2.y(), out, plane);
    return;
  } else {
  // face states and fluxes in the state precision S (float64, or
  // float-float for the mixed solver)
  RC<S> c;
  S gam, kg;
  if constexpr (std::is_same<S, double>::value) {
    c = make_rc<S>(p);
    gam = S(p.gamma);
    kg = S(a.kappa * p.gamma);
  } else {
    c.gam = S(a.ffc[0], a.ffc[1]);
    c.gm1 = S(a.ffc[2], a.ffc[3]);
    c.sphig = S(a.ffc[4], a.ffc[5]);
    c.spsig = S(a.ffc[6], a.ffc[7]);
    c.cond = p.cond;
    c.visc = p.visc;
    gam = c.gam;
    kg = S(a.ffc[8], a.ffc[9]);
  }
  Z<S> zl, zr;
  z_load(zl, Ls, c);
  z_load(zr, Rs, c);
  S UL[NV], FL[NV], UR[NV], FR[NV];
  S cminL, cmaxL, cminR, cmaxR;
  side_flux<D + 1>(zl, gam, kg, UL, FL, cminL, cmaxL);
  side_flux<D + 1>(zr, gam, kg, UR, FR, cminR, cmaxR);
  riemann_flux<S>(p.riemann, FL, FR, UL, UR, cminL, cmaxL, cminR, cmaxR, out, plane);
  }
}

// One kernel per reconstruction, so that each holds only its own registers.
// The float-float form is held to 128 registers a thread (16 warps per SM),
// for the latency of its dependent float chains.
template <int BS, typename S, int RECON>
__global__ void __launch_bounds__(BS, std::is_same<S, double>::value ? 1 : 65536 / (BS * 128)) face_flux_2d(const __grid_constant__ Params p,
                                                  const __grid_constant__ ExpArgs a) {
  const long long nf1 = (long long)(p.n1 + 1) * (p.n2 + 2);
  const long long nf2 = (long long)(p.n1 + 2) * (p.n2 + 1);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf1 + nf2) return;
  if (f < nf1) {
    const int i = (int)(f % (p.n1 + 1)), j = (int)(f / (p.n1 + 1)) - 1;
    double* out = a.F1 + (long long)(j + 1) * (p.n1 + 1) + i;
    face_flux_dir<0, RECON, S>(p, a, i, j, out, nf1);
  } else {
    const long long g = f - nf1;
    const int i = (int)(g % (p.n1 + 2)) - 1, j = (int)(g / (p.n1 + 2));
    double* out = a.F2 + (long long)j * (p.n1 + 2) + (i + 1);
    face_flux_dir<1, RECON, S>(p, a, i, j, out, nf2);
  }
}

// Theta = (gamma-1) u/rho and u^t = (1 + u^i u^i)^(1/2) of P^E at every
// zone, once a stage: the limited slopes of the zone kernel read them for
// four neighbours of each zone.  Both are even under the reflections of the
// boundary rules, so a ghost takes the values of the zone it maps to.
template <int BS>
__global__ void __launch_bounds__(BS) derived_2d(const __grid_constant__ Params p, const __grid_constant__ ExpArgs a) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * BS + threadIdx.x;
  if (z >= N) return;
  const double rho = __ldg(a.PE + z), uu = __ldg(a.PE + N + z);
  const double v1 = __ldg(a.PE + 2 * N + z), v2 = __ldg(a.PE + 3 * N + z), v3 = __ldg(a.PE + 4 * N + z);
  a.Dv[z] = (p.gamma - 1.0) * uu * nr_rcp(rho);
  a.Dv[N + z] = sqrt(1.0 + v1 * v1 + v2 * v2 + v3 * v3);
}

// Theta and u_mu of the state at zone (i, j) of P^E (for the limited slopes).
__device__ __forceinline__ void derived_at(const Params& p, const ExpArgs& a, int i, int j, double& th, double u[4]) {
  bool f1, f2;
  const long long z = zone_at(p, i, j, f1, f2);
  const long long N = p.N;
  th = __ldg(a.Dv + z);
  u[0] = -__ldg(a.Dv + N + z);
  u[1] = load_comp(a.PE, N, z, 2, f1, f2);
  u[2] = load_comp(a.PE, N, z, 3, f1, f2);
  u[3] = __ldg(a.PE + 4 * N + z);
}

// The same computed in float-float from P^E (the mixed solver's slopes;
// there the float pipes make the recomputation cheaper than the pre-pass),
// inputs split without float64 instructions.
__device__ __forceinline__ void derived_at_ff(const Params& p, const ExpArgs& a, int i, int j, ff& th, ff u[4]) {
  bool f1, f2;
  const long long z = zone_at(p, i, j, f1, f2);
  const long long N = p.N;
  const ff rho = ff_split(__ldg(a.PE + z)), uu = ff_split(__ldg(a.PE + N + z));
  const ff v1 = ff_split(load_comp(a.PE, N, z, 2, f1, f2)), v2 = ff_split(load_comp(a.PE, N, z, 3, f1, f2));
  const ff v3 = ff_split(__ldg(a.PE + 4 * N + z));
  th = ff(a.ffc[2], a.ffc[3]) * uu * nr_rcp(rho);
  u[0] = -sqr_root(tconst<ff>(1.0) + v1 * v1 + v2 * v2 + v3 * v3);
  u[1] = v1; u[2] = v2; u[3] = v3;
}

// Flux divergence of zone (i, j) from the face fluxes; flux-CT replaces
// F^1[B^1], F^2[B^2] by 0 and the transverse B fluxes by averages of the
// corner values
// E(i', j') = (F^1[B^2](i',j') + F^1[B^2](i',j'-1) - F^2[B^1](i',j') - F^2[B^1](i'-1,j'))/4
// (Section 4.2).
__device__ __forceinline__ void flux_divergence_ct(const Params& p, const ExpArgs& a, int i, int j, double divF[NV]) {
  const long long w1 = p.n1 + 1, w2 = p.n1 + 2;
  const long long nf1 = w1 * (p.n2 + 2), nf2 = w2 * (p.n2 + 1);
  const double idx1 = p.idx[0], idx2 = p.idx[1];
  const long long f1lo = (long long)(j + 1) * w1 + i, f2lo = (long long)j * w2 + (i + 1);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const double* F1 = a.F1 + v * nf1;
    const double* F2 = a.F2 + v * nf2;
    divF[v] = (__ldg(F1 + f1lo + 1) - __ldg(F1 + f1lo)) * idx1 + (__ldg(F2 + f2lo + w2) - __ldg(F2 + f2lo)) * idx2;
  }
  const double* F1b2 = a.F1 + 6 * nf1;
  const double* F2b1 = a.F2 + 5 * nf2;
  double E[2][2];
#pragma unroll
  for (int dj = 0; dj < 2; dj++)
#pragma unroll
    for (int di = 0; di < 2; di++) {
      const int ii = i + di, jj = j + dj;
      E[dj][di] = 0.25 * (__ldg(F1b2 + (long long)(jj + 1) * w1 + ii) + __ldg(F1b2 + (long long)jj * w1 + ii) -
                          __ldg(F2b1 + (long long)jj * w2 + ii + 1) - __ldg(F2b1 + (long long)jj * w2 + ii));
    }
  divF[6] = (0.5 * (E[0][1] + E[1][1]) - 0.5 * (E[0][0] + E[1][0])) * idx1;
  divF[5] = (-0.5 * (E[1][0] + E[1][1]) + 0.5 * (E[0][0] + E[0][1])) * idx2;
}

// The conserved variables U(P) of a float64 zone state in Minkowski space
// (Section 4, Eqs. fullSEtens, divN_explicit, divT_explicit: rho u^t and
// T^t_mu with the heat-flux and anisotropy terms), with B^i, q~ u^t and
// dP~ u^t for the induction and closure rows.
__device__ __forceinline__ void conserved_of(const Z<double>& zn, const double* P, double U[NV]) {
  const double dp = zn.dpt * zn.ds, q = zn.qt * zn.qs;
  const double third = dp * (1.0 / 3.0);
  const double A = (zn.w0 + zn.bsq + third) * zn.ut;
  const double qb = q * zn.bht, dpb = dp * zn.bht, qut = q * zn.ut;
  U[0] = zn.rho * zn.ut;
  U[1] = -A * zn.ut + zn.bt * zn.bt - 2.0 * qb * zn.ut + dpb * zn.bht + zn.pg + 0.5 * zn.bsq + third;
#pragma unroll
  for (int k = 0; k < 3; k++) U[2 + k] = A * zn.v[k] - zn.bt * zn.bc[k] + qb * zn.v[k] + qut * zn.bh[k] - dpb * zn.bh[k];
  U[5] = P[5]; U[6] = P[6]; U[7] = P[7];
  U[8] = zn.qt * zn.ut;
  U[9] = zn.dpt * zn.ut;
}

// The stage constants of every zone in float64 (the float64 solver): the
// flux divergence with flux-CT, U(P_n), the row scales, the heat-flux and
// anisotropy rows' explicit parts (Eqs. q_evol_eqn_rescaled,
// dP_evol_eqn_rescaled with q0def, dP0def at P^E), and the Newton start.
template <int BS>
__global__ void __launch_bounds__(BS) zone_const_2d(const __grid_constant__ Params p,
                                                   const __grid_constant__ ExpArgs a) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const int i = (int)(z % p.n1), j = (int)(z / p.n1);
  const double idx1 = p.idx[0], idx2 = p.idx[1];
  double divF[NV];
  flux_divergence_ct(p, a, i, j, divF);
  // states at P^E and P_n
  double PEz[NV], Pnz[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    PEz[v] = __ldg(a.PE + v * N + z);
    Pnz[v] = (a.mode == 1) ? PEz[v] : __ldg(a.Pn + v * N + z);
  }
  const RC<double> c = make_rc<double>(p);
  Z<double> ze;
  z_load(ze, PEz, c);
  // P_n quantities: U(P_n), Theta_n, u^t_n (from the cache in the full step)
  double Un[NV], th_n, ut_n;
  if (a.mode == 2) {
#pragma unroll
    for (int v = 0; v < NV; v++) Un[v] = __ldg(a.cache + v * N + z);
    th_n = __ldg(a.cache + NV * N + z);
    ut_n = __ldg(a.cache + (NV + 1) * N + z);
  } else {
    Z<double> zn;
    if (a.mode == 1) zn = ze;
    else z_load(zn, Pnz, c);
    conserved_of(zn, Pnz, Un);
    th_n = zn.theta;
    ut_n = zn.ut;
    if (a.mode == 1) {
#pragma unroll
      for (int v = 0; v < NV; v++) a.cache[v * N + z] = Un[v];
      a.cache[NV * N + z] = th_n;
      a.cache[(NV + 1) * N + z] = ut_n;
    }
  }
  const double qt_n = Pnz[8], dpt_n = Pnz[9];

  // limited slopes at P^E of Theta and u_mu; the spatial part of nabla_mu u^mu
  double dTh[2], du[2][4], divu_sp = 0.0;
  {
    const double th0 = ze.theta, u0[4] = {-ze.ut, ze.v[0], ze.v[1], ze.v[2]};
#pragma unroll
    for (int d = 0; d < 2; d++) {
      double thm, thp, um[4], up[4];
      derived_at(p, a, i - (d == 0), j - (d == 1), thm, um);
      derived_at(p, a, i + (d == 0), j + (d == 1), thp, up);
      const double ih = (d == 0) ? idx1 : idx2;
      dTh[d] = gm_slope(p.theta, thm, th0, thp) * ih;
#pragma unroll
      for (int m = 0; m < 4; m++) du[d][m] = gm_slope(p.theta, um[m], u0[m], up[m]) * ih;
      divu_sp += du[d][1 + d];
    }
  }
  const double tau = p.tauR, dts = a.dts, idts = a.idts, it = a.itau, git = idts * it;
  double* Kz = a.K + z;
  double kU[NV];
  // the learned start's features x_a = -r_a(P_n) (the scaled residual of this
  // stage at its start), written beside the constants when requested
  float* feat = a.feat ? a.feat + z : nullptr;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    // row scale s_v = dt_s/(|U_v(P_n)| + |U_0(P_n)|); kU = s_v/dt_s depends on P_n only
    if (a.mode == 2) {
      kU[v] = Kz[(K_U + v) * N];
    } else {
      kU[v] = nr_rcp(fabs(Un[v]) + fabs(Un[0]));
      Kz[(K_U + v) * N] = kU[v];
    }
    if (v < 8) {
      const double kc = kU[v] * (dts * divF[v] - Un[v]);
      Kz[(K_C + v) * N] = kc;
      if (feat) feat[v * N] = (float)(-(kU[v] * Un[v] + kc));
    }
  }
  const double bhu[4] = {ze.bht, ze.bh[0], ze.bh[1], ze.bh[2]};
  const double ucovn[4] = {-ut_n, Pnz[2], Pnz[3], Pnz[4]};
  const double hoq = p.ho ? 0.5 * ze.qt : 0.0;
  const double hod = p.ho ? 0.5 * ze.dpt : 0.0;
  const double cs2E = p.gamma * ze.pg * ze.iden;
  // heat flux row: q~_0 = Aq + Bq (Theta - Theta_n)/dt_s + Cq^mu (u_mu - u_mu,n)/dt_s
  double Aq = 0.0, Bq = 0.0, Cq[4] = {0.0, 0.0, 0.0, 0.0};
  if (p.cond) {
    const double chi = p.phi * cs2E * tau;
    const double pre = -sqrt(tau * ze.rho * chi) * nr_rcp(ze.theta);  // -rho chi (tau/(chi rho Theta^2))^(1/2)
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 4; m++) acc += bhu[m] * (ze.v[0] * du[0][m] + ze.v[1] * du[1][m]);
    Aq = pre * (bhu[1] * dTh[0] + bhu[2] * dTh[1] + ze.theta * acc);
    Bq = pre * bhu[0];
#pragma unroll
    for (int m = 0; m < 4; m++) Cq[m] = pre * ze.theta * bhu[m] * ze.ut;
  }
  {
    const double s8 = kU[8] * dts;
    double cst = -Un[8] * idts + divF[8] + 0.5 * qt_n * it - Aq * it + Bq * th_n * git;
#pragma unroll
    for (int m = 0; m < 4; m++) cst += Cq[m] * ucovn[m] * git;
    cst -= hoq * (divu_sp - ut_n * idts);
    double kQ[7];
    const double kc = s8 * cst;
    kQ[0] = 0.5 * s8 * it;
    kQ[1] = -s8 * git * Bq;
#pragma unroll
    for (int m = 0; m < 4; m++) kQ[2 + m] = -s8 * git * Cq[m];
    kQ[6] = -s8 * hoq * idts;
    Kz[(K_C + 8) * N] = kc;
#pragma unroll
    for (int q = 0; q < 7; q++) Kz[(K_Q + q) * N] = kQ[q];
    if (feat) {
      const double r8 = kU[8] * Un[8] + kc + kQ[0] * Pnz[8] + kQ[1] * th_n + kQ[6] * ut_n - kQ[2] * ut_n +
                        kQ[3] * Pnz[2] + kQ[4] * Pnz[3] + kQ[5] * Pnz[4];
      feat[8 * N] = (float)(-r8);
    }
  }
  // anisotropy row: dP~_0 = Ad + Dd^nu (u_nu - u_nu,n)/dt_s + Ed (u^t - u^t_n)/dt_s
  double Ad = 0.0, Dd[4] = {0.0, 0.0, 0.0, 0.0}, Ed = 0.0;
  if (p.visc) {
    const double nu = p.psi * cs2E * tau;
    const double pre = 3.0 * sqrt(tau * ze.rho * nu * nr_rcp(ze.theta));  // 3 rho nu (tau/(nu rho Theta))^(1/2)
    double sp = 0.0;
#pragma unroll
    for (int m = 0; m < 4; m++) sp += bhu[m] * (bhu[1] * du[0][m] + bhu[2] * du[1][m]);
    Ad = pre * (sp - divu_sp * (1.0 / 3.0));
#pragma unroll
    for (int m = 0; m < 4; m++) Dd[m] = pre * bhu[0] * bhu[m];
    Ed = -pre * (1.0 / 3.0);
  }
  {
    const double s9 = kU[9] * dts;
    double cst = -Un[9] * idts + divF[9] + 0.5 * dpt_n * it - Ad * it + Ed * ut_n * git;
#pragma unroll
    for (int m = 0; m < 4; m++) cst += Dd[m] * ucovn[m] * git;
    cst -= hod * (divu_sp - ut_n * idts);
    double kD[6];
    const double kc = s9 * cst;
    kD[0] = 0.5 * s9 * it;
#pragma unroll
    for (int m = 0; m < 4; m++) kD[1 + m] = -s9 * git * Dd[m];
    kD[5] = -s9 * (Ed * git + hod * idts);
    Kz[(K_C + 9) * N] = kc;
#pragma unroll
    for (int q = 0; q < 6; q++) Kz[(K_D + q) * N] = kD[q];
    if (feat) {
      const double r9 = kU[9] * Un[9] + kc + kD[0] * Pnz[9] + kD[5] * ut_n - kD[1] * ut_n + kD[2] * Pnz[2] +
                        kD[3] * Pnz[3] + kD[4] * Pnz[4];
      feat[9 * N] = (float)(-r9);
    }
  }
  // initial guess: P_n (or the given guess) with B from the explicit flux-CT update
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double x = a.guess ? __ldg(a.guess + v * N + z) : Pnz[v];
    if (v >= 5 && v <= 7) x = Pnz[v] - dts * divF[v];
    a.P0[v * N + z] = x;
  }
}

// The same constants for the mixed solver.  What sets the conserved update
// stays float64: the flux divergence with flux-CT, U(P_n), the constant
// parts kU (dt_s div F - U(P_n)) and the flux-CT update of B.  The rest is
// explicit source data evaluated at P^E, as the float-float face fluxes
// are: the state at P^E, the limited slopes of Theta and u_mu, and the
// heat-flux and anisotropy rows' coefficients are computed in float-float
// (about 48 bits), and each stored coefficient is joined into a double once.
// The row scales kU are refined in float-float as well.  The learned start's
// features -r_a(P_n) follow from the same terms: for rows 0-7 they are
// -kU dt_s div F, and for the closure rows the P_n parts of the constants
// cancel, leaving -s (div F + (X_n - A)/tau_R - h div_i u^i) with
// s = kU dt_s, X_n = q~_n or dP~_n, A the explicit target and h the
// higher-order coefficient.
template <int BS>
__global__ void __launch_bounds__(BS, 512 / BS) zone_const_2d_mixed(const __grid_constant__ Params p,
                                                         const __grid_constant__ ExpArgs a) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const int i = (int)(z % p.n1), j = (int)(z / p.n1);
  double divF[NV];
  flux_divergence_ct(p, a, i, j, divF);
  double PEz[NV], Pnz[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    PEz[v] = __ldg(a.PE + v * N + z);
    Pnz[v] = (a.mode == 1) ? PEz[v] : __ldg(a.Pn + v * N + z);
  }
  // P_n quantities in float64: U(P_n), Theta_n, u^t_n (from the cache in the full step)
  double Un[NV], th_n, ut_n;
  if (a.mode == 2) {
#pragma unroll
    for (int v = 0; v < NV; v++) Un[v] = __ldg(a.cache + v * N + z);
    th_n = __ldg(a.cache + NV * N + z);
    ut_n = __ldg(a.cache + (NV + 1) * N + z);
  } else {
    Z<double> zn;
    z_load(zn, Pnz, make_rc<double>(p));
    conserved_of(zn, Pnz, Un);
    th_n = zn.theta;
    ut_n = zn.ut;
    if (a.mode == 1) {
#pragma unroll
      for (int v = 0; v < NV; v++) a.cache[v * N + z] = Un[v];
      a.cache[NV * N + z] = th_n;
      a.cache[(NV + 1) * N + z] = ut_n;
    }
  }
  // the state at P^E in float-float
  RC<ff> c;
  c.gam = ff(a.ffc[0], a.ffc[1]);
  c.gm1 = ff(a.ffc[2], a.ffc[3]);
  c.sphig = ff(a.ffc[4], a.ffc[5]);
  c.spsig = ff(a.ffc[6], a.ffc[7]);
  c.cond = p.cond;
  c.visc = p.visc;
  // Of the field, only the direction b-hat enters here, and it does not
  // depend on the field's scale: B^i is split at the power of two that
  // brings its largest component near 1, so that a weak field keeps all its
  // float-float bits (its low parts would otherwise be float denormals).
  // b^2 and b^t of ze are then those of the scaled field and stay unused.
  const int eb = max(max((int)((__double_as_longlong(PEz[5]) >> 52) & 0x7ff),
                         (int)((__double_as_longlong(PEz[6]) >> 52) & 0x7ff)),
                     (int)((__double_as_longlong(PEz[7]) >> 52) & 0x7ff));
  const double sb = (eb > 0 && eb < 0x7ff) ? __longlong_as_double((long long)(2046 - eb) << 52) : 1.0;
  ff PEf[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) PEf[v] = ff_split((v >= 5 && v <= 7) ? PEz[v] * sb : PEz[v]);
  Z<ff> ze;
  z_load(ze, PEf, c);
  const ff idx1(a.ffz[0], a.ffz[1]), idx2(a.ffz[2], a.ffz[3]), tau(a.ffz[4], a.ffz[5]);
  const ff phi(a.ffz[6], a.ffz[7]), psi(a.ffz[8], a.ffz[9]), it(a.ffz[10], a.ffz[11]);
  const ff idts(a.ffz[12], a.ffz[13]), git(a.ffz[14], a.ffz[15]);
  // limited slopes at P^E of Theta and u_mu; the spatial part of nabla_mu u^mu
  ff dTh[2], du[2][4], divu_sp(0.f, 0.f);
  {
    const ff theta(a.ffc[10], a.ffc[11]);
    const ff u0[4] = {-ze.ut, ze.v[0], ze.v[1], ze.v[2]};
#pragma unroll
    for (int d = 0; d < 2; d++) {
      ff thm, thp, um[4], up[4];
      derived_at_ff(p, a, i - (d == 0), j - (d == 1), thm, um);
      derived_at_ff(p, a, i + (d == 0), j + (d == 1), thp, up);
      const ff ih = (d == 0) ? idx1 : idx2;
      dTh[d] = gm_slope(theta, thm, ze.theta, thp) * ih;
#pragma unroll
      for (int m = 0; m < 4; m++) du[d][m] = gm_slope(theta, um[m], u0[m], up[m]) * ih;
      divu_sp += du[d][1 + d];
    }
  }
  const double dts = a.dts, idts_d = a.idts;
  double* Kz = a.K + z;
  float* feat = a.feat ? a.feat + z : nullptr;
  const float fdts = a.ffz[16];
  // row scales (they depend on P_n only) and the conserved rows' constants
  double kU[NV];
  const ff u0abs = fabs(ff_split(Un[0]));
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if (a.mode == 2) {
      kU[v] = Kz[(K_U + v) * N];
    } else {
      kU[v] = ff_join(nr_rcp(fabs(ff_split(Un[v])) + u0abs));
      Kz[(K_U + v) * N] = kU[v];
    }
    if (v < 8) {
      Kz[(K_C + v) * N] = kU[v] * (dts * divF[v] - Un[v]);
      if (feat) feat[v * N] = -(d2f_jac(kU[v]) * fdts) * d2f_jac(divF[v]);
    }
  }
  const ff bhu[4] = {ze.bht, ze.bh[0], ze.bh[1], ze.bh[2]};
  const ff thn = ff_split(th_n), utn = ff_split(ut_n);
  const ff ucovn[4] = {-utn, ff_split(Pnz[2]), ff_split(Pnz[3]), ff_split(Pnz[4])};
  const ff zero(0.f, 0.f);
  const ff hoq = p.ho ? scale2(ze.qt, 0.5f) : zero;
  const ff hod = p.ho ? scale2(ze.dpt, 0.5f) : zero;
  const ff cs2E = c.gam * ze.pg * ze.iden;
  const ff third = tconst<ff>(1.0 / 3.0);
  // heat flux row: q~_0 = Aq + Bq (Theta - Theta_n)/dt_s + Cq^mu (u_mu - u_mu,n)/dt_s
  ff Aq = zero, Bq = zero, Cq[4] = {zero, zero, zero, zero};
  if (p.cond) {
    const ff chi = phi * cs2E * tau;
    const ff pre = -(sqr_root(tau * ze.rho * chi) * nr_rcp(ze.theta));  // -rho chi (tau/(chi rho Theta^2))^(1/2)
    ff acc = zero;
#pragma unroll
    for (int m = 0; m < 4; m++) acc += bhu[m] * (ze.v[0] * du[0][m] + ze.v[1] * du[1][m]);
    Aq = pre * (bhu[1] * dTh[0] + bhu[2] * dTh[1] + ze.theta * acc);
    Bq = pre * bhu[0];
    const ff pt = pre * ze.theta * ze.ut;
#pragma unroll
    for (int m = 0; m < 4; m++) Cq[m] = pt * bhu[m];
  }
  {
    const ff qtn = ff_split(Pnz[8]);
    ff src = scale2(qtn * it, 0.5f) - Aq * it + Bq * thn * git - hoq * (divu_sp - utn * idts);
#pragma unroll
    for (int m = 0; m < 4; m++) src += Cq[m] * ucovn[m] * git;
    const double s8 = kU[8] * dts;
    Kz[(K_C + 8) * N] = s8 * ((divF[8] - Un[8] * idts_d) + ff_join(src));
    const ff s8f = ff_split(s8), sg = s8f * git;
    Kz[(K_Q + 0) * N] = ff_join(scale2(s8f * it, 0.5f));
    Kz[(K_Q + 1) * N] = ff_join(-(sg * Bq));
#pragma unroll
    for (int m = 0; m < 4; m++) Kz[(K_Q + 2 + m) * N] = ff_join(-(sg * Cq[m]));
    Kz[(K_Q + 6) * N] = ff_join(-(s8f * hoq * idts));
    if (feat) feat[8 * N] = -(s8f * (ff_split(divF[8]) + it * (qtn - Aq) - hoq * divu_sp)).hi;
  }
  // anisotropy row: dP~_0 = Ad + Dd^nu (u_nu - u_nu,n)/dt_s + Ed (u^t - u^t_n)/dt_s
  ff Ad = zero, Dd[4] = {zero, zero, zero, zero}, Ed = zero;
  if (p.visc) {
    const ff nu = psi * cs2E * tau;
    const ff pre = tconst<ff>(3.0) * sqr_root(tau * ze.rho * nu * nr_rcp(ze.theta));  // 3 rho nu (tau/(nu rho Theta))^(1/2)
    ff sp = zero;
#pragma unroll
    for (int m = 0; m < 4; m++) sp += bhu[m] * (bhu[1] * du[0][m] + bhu[2] * du[1][m]);
    Ad = pre * (sp - divu_sp * third);
    const ff pb = pre * bhu[0];
#pragma unroll
    for (int m = 0; m < 4; m++) Dd[m] = pb * bhu[m];
    Ed = -(pre * third);
  }
  {
    const ff dptn = ff_split(Pnz[9]);
    ff src = scale2(dptn * it, 0.5f) - Ad * it + Ed * utn * git - hod * (divu_sp - utn * idts);
#pragma unroll
    for (int m = 0; m < 4; m++) src += Dd[m] * ucovn[m] * git;
    const double s9 = kU[9] * dts;
    Kz[(K_C + 9) * N] = s9 * ((divF[9] - Un[9] * idts_d) + ff_join(src));
    const ff s9f = ff_split(s9), sg = s9f * git;
    Kz[(K_D + 0) * N] = ff_join(scale2(s9f * it, 0.5f));
#pragma unroll
    for (int m = 0; m < 4; m++) Kz[(K_D + 1 + m) * N] = ff_join(-(sg * Dd[m]));
    Kz[(K_D + 5) * N] = ff_join(-(s9f * (Ed * git + hod * idts)));
    if (feat) feat[9 * N] = -(s9f * (ff_split(divF[9]) + it * (dptn - Ad) - hod * divu_sp)).hi;
  }
  // initial guess: P_n (or the given guess) with B from the explicit flux-CT update
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double x = a.guess ? __ldg(a.guess + v * N + z) : Pnz[v];
    if (v >= 5 && v <= 7) x = Pnz[v] - dts * divF[v];
    a.P0[v * N + z] = x;
  }
}

// Explicit-stage scratch for an n1 x n2 grid, in doubles: the face arrays,
// then Theta and u^t of every zone.
long long face_scratch_doubles(int n1, int n2) {
  return (long long)NV * ((long long)(n1 + 1) * (n2 + 2) + (long long)(n1 + 2) * (n2 + 1)) +
         2LL * n1 * n2;
}

// cs~^2 / c_s^2 under the closure chi = phi c_s^2 tau_R, nu = psi c_s^2 tau_R
// (Eq. modcs with v_q^2 = (gamma-1) chi/tau_R, v_dP^2 = 4 nu/(3 tau_R)).
static double closure_kappa(const Params& p) {
  const double a = p.cond ? (p.gamma - 1.0) * p.phi : 0.0;
  const double b = p.visc ? 4.0 * p.psi / 3.0 : 0.0;
  return 0.5 * (1.0 + a + sqrt(1.0 + a * a)) + b;
}

void explicit_args(const Params& p, const double* Pn, const double* PE, const double* guess, double dts, double* K,
                   double* P0, double* faces, ExpArgs& a) {
  a.Pn = Pn; a.PE = PE; a.guess = guess; a.dts = dts; a.kappa = closure_kappa(p);
  a.idts = 1.0 / dts;
  a.itau = 1.0 / p.tauR;
  a.cache = nullptr; a.mode = 0; a.feat = nullptr;
  const double cv[6] = {p.gamma, p.gamma - 1.0, sqrt(p.phi * p.gamma), sqrt(p.psi * p.gamma), a.kappa * p.gamma,
                        p.theta};
  for (int k = 0; k < 6; k++) {
    a.ffc[2 * k] = (float)cv[k];
    a.ffc[2 * k + 1] = (float)(cv[k] - (double)(float)cv[k]);
  }
  const double cz[9] = {p.idx[0], p.idx[1], p.tauR, p.phi, p.psi, a.itau, a.idts, a.idts * a.itau, dts};
  for (int k = 0; k < 9; k++) {
    a.ffz[2 * k] = (float)cz[k];
    a.ffz[2 * k + 1] = (float)(cz[k] - (double)(float)cz[k]);
  }
  a.K = K; a.P0 = P0;
  a.F1 = faces;
  a.F2 = faces + (long long)NV * (p.n1 + 1) * (p.n2 + 2);
  a.Dv = a.F2 + (long long)NV * (p.n1 + 2) * (p.n2 + 1);
}

template <typename S, int RECON>
static cudaError_t launch_faces_r(const Params& p, const ExpArgs& a, unsigned nb, int bs, cudaStream_t st) {
  switch (bs) {
    case 64: face_flux_2d<64, S, RECON><<<nb, 64, 0, st>>>(p, a); break;
    case 128: face_flux_2d<128, S, RECON><<<nb, 128, 0, st>>>(p, a); break;
    case 256: face_flux_2d<256, S, RECON><<<nb, 256, 0, st>>>(p, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template <typename S>
static cudaError_t launch_faces_s(const Params& p, const ExpArgs& a, unsigned nb, int bs, cudaStream_t st) {
  if (p.recon == RECON_WENO5) return launch_faces_r<S, RECON_WENO5>(p, a, nb, bs, st);
  if (p.recon == RECON_PPM) return launch_faces_r<S, RECON_PPM>(p, a, nb, bs, st);
  return launch_faces_r<S, RECON_MC>(p, a, nb, bs, st);
}

// bs: threads per block, 64, 128 or 256.  ffstates: face states and fluxes
// in float-float, both states of a face in paired lanes (the mixed solver),
// instead of float64.
cudaError_t launch_faces(const Params& p, const double* PE, double* faces, int bs, int ffstates, cudaStream_t st) {
  ExpArgs a;
  explicit_args(p, nullptr, PE, nullptr, 1.0, nullptr, nullptr, faces, a);
  const long long nf = (long long)(p.n1 + 1) * (p.n2 + 2) + (long long)(p.n1 + 2) * (p.n2 + 1);
  const unsigned nb = (unsigned)((nf + bs - 1) / bs);
  return ffstates ? launch_faces_s<ff2>(p, a, nb, bs, st) : launch_faces_s<double>(p, a, nb, bs, st);
}

long long pn_cache_doubles(long long N) { return (long long)NCACHE * N; }

// mode: 0 general stage, 1 half step (P_E == P_n; fills cache), 2 full step
// of the same step (reads cache and K_U).
// The float64 form first runs derived_2d; the float-float form recomputes
// the neighbours' Theta and u^t itself.
template <bool MIXED>
static cudaError_t launch_zone_const_s(const Params& p, const ExpArgs& a, unsigned nb, int bs, cudaStream_t st) {
  switch (bs) {
    case 64:
      if (MIXED) zone_const_2d_mixed<64><<<nb, 64, 0, st>>>(p, a);
      else { derived_2d<64><<<nb, 64, 0, st>>>(p, a); zone_const_2d<64><<<nb, 64, 0, st>>>(p, a); }
      break;
    case 128:
      if (MIXED) zone_const_2d_mixed<128><<<nb, 128, 0, st>>>(p, a);
      else { derived_2d<128><<<nb, 128, 0, st>>>(p, a); zone_const_2d<128><<<nb, 128, 0, st>>>(p, a); }
      break;
    case 256:
      if (MIXED) zone_const_2d_mixed<256><<<nb, 256, 0, st>>>(p, a);
      else { derived_2d<256><<<nb, 256, 0, st>>>(p, a); zone_const_2d<256><<<nb, 256, 0, st>>>(p, a); }
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ffslopes: the mixed solver's form (zone_const_2d_mixed: the source terms at
// P^E in float-float) instead of the float64 one.
cudaError_t launch_zone_const(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                              double* K, double* P0, double* faces, double* cache, int mode, int bs, float* feat,
                              int ffslopes, cudaStream_t st) {
  ExpArgs a;
  explicit_args(p, Pn, PE, guess, dts, K, P0, faces, a);
  a.cache = cache;
  a.mode = cache ? mode : 0;
  a.feat = feat;
  const unsigned nb = (unsigned)((p.N + bs - 1) / bs);
  return ffslopes ? launch_zone_const_s<true>(p, a, nb, bs, st) : launch_zone_const_s<false>(p, a, nb, bs, st);
}

}  // namespace grim
