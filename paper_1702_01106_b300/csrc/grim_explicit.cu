// Explicit part of one stage of the semi-implicit step (Section 2.3), 2-D:
// reconstruction of P^E (generalized minmod / WENO5, Section 2.4.1), LLF face
// fluxes with the wave-speed bound of Section 4.1, flux-CT (Section 4.2), the
// slope-limited spatial derivatives and the closure terms of q~_0, dP~_0
// (Section 4), folded into the per-zone constants of the Newton residual.
//
// One CTA owns a TX x TY tile of zones.  P^E for the tile and its halo is
// staged in shared memory once (boundary rules applied on load, so there are
// no ghost arrays in HBM); face fluxes, corner EMFs and slopes live only in
// shared memory; each zone writes its NK constants and its initial guess.
#include "grim_dev.cuh"

namespace grim {

__device__ __forceinline__ int map_index(int i, int n, int lo, int hi, bool& flip) {
  if (i >= 0 && i < n) return i;
  int bc = (i < 0) ? lo : hi;
  if (bc == BC_PERIODIC) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  if (bc == BC_OUTFLOW) return i < 0 ? 0 : n - 1;
  // mirror images repeat with period 2n; an odd number of reflections flips
  int m = i % (2 * n);
  if (m < 0) m += 2 * n;
  if (m >= n) {
    flip = !flip;
    return 2 * n - 1 - m;
  }
  return m;
}

// Generalized minmod slope (Section 2.4.1) of three consecutive values.
__device__ __forceinline__ double mc_slope(double theta, double vm, double v0, double vp) {
  double a = theta * (v0 - vm), b = 0.5 * (vp - vm), c = theta * (vp - v0);
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

// WENO5 of Jiang & Shu (1996): value at the right face of v2 from v0..v4.
__device__ __forceinline__ double weno5(double v0, double v1, double v2, double v3, double v4) {
  const double eps = 1e-6;
  double q0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) * (1.0 / 6.0);
  double q1 = (-v1 + 5.0 * v2 + 2.0 * v3) * (1.0 / 6.0);
  double q2 = (2.0 * v2 + 5.0 * v3 - v4) * (1.0 / 6.0);
  double d0 = v0 - 2.0 * v1 + v2, e0 = v0 - 4.0 * v1 + 3.0 * v2;
  double d1 = v1 - 2.0 * v2 + v3, e1 = v1 - v3;
  double d2 = v2 - 2.0 * v3 + v4, e2 = 3.0 * v2 - 4.0 * v3 + v4;
  double b0 = (13.0 / 12.0) * d0 * d0 + 0.25 * e0 * e0;
  double b1 = (13.0 / 12.0) * d1 * d1 + 0.25 * e1 * e1;
  double b2 = (13.0 / 12.0) * d2 * d2 + 0.25 * e2 * e2;
  double a0 = 0.1 / ((eps + b0) * (eps + b0));
  double a1 = 0.6 / ((eps + b1) * (eps + b1));
  double a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Conserved variables U(P) and the flux F^j(P) (Eqs. divN_explicit,
// divT_explicit, induction_eqn, and the q~, dP~ equations); the induction flux
// is b^i u^j - b^j u^i, the divergence of the dual Faraday tensor.
__device__ __forceinline__ void cons_flux(const Pt<double>& s, const double* P, int j, double U[NV], double F[NV]) {
  double row[4];
  stress_row(s, 0, row);
  U[0] = s.rho * s.ut;
  U[1] = row[0]; U[2] = row[1]; U[3] = row[2]; U[4] = row[3];
  U[5] = P[5]; U[6] = P[6]; U[7] = P[7];
  U[8] = s.qt * s.ut;
  U[9] = s.dpt * s.ut;
  stress_row(s, j, row);
  const double uj = s.uc[j - 1], bj = s.bc[j - 1];
  F[0] = s.rho * uj;
  F[1] = row[0]; F[2] = row[1]; F[3] = row[2]; F[4] = row[3];
  F[5] = s.bc[0] * uj - bj * s.uc[0];
  F[6] = s.bc[1] * uj - bj * s.uc[1];
  F[7] = s.bc[2] * uj - bj * s.uc[2];
  F[8] = s.qt * uj;
  F[9] = s.dpt * uj;
}

// Largest |grid-frame speed| in direction j of waves at +-v_max in the fluid
// frame (Section 4.1): roots c of (u^j - c u^t)^2 (1 - v^2) = v^2 (1 - c^2)
// for Minkowski space (g^tt = -1, g^tj = 0, g^jj = 1).
__device__ __forceinline__ double max_speed(const Pt<double>& s, const Params& p, int j) {
  const double gam = p.gamma;
  double vA2 = s.bsq / (s.rho + gam * s.u + s.bsq);
  double chi = p.cond ? p.phi * s.cs2 * p.tauR : 0.0;
  double nu = p.visc ? p.psi * s.cs2 * p.tauR : 0.0;
  double vq2 = (gam - 1.0) * chi / p.tauR;
  double vd2 = 4.0 * nu / (3.0 * p.tauR);
  double cs2t = 0.5 * (s.cs2 + vq2 + sqrt(s.cs2 * s.cs2 + vq2 * vq2)) + vd2;
  double v2 = cs2t + vA2 - cs2t * vA2;
  double ut = s.ut, uj = s.uc[j - 1];
  double A = (1.0 - v2) * ut * ut + v2;
  double B = -2.0 * (1.0 - v2) * ut * uj;
  double C = (1.0 - v2) * uj * uj - v2;
  double disc = fmax(B * B - 4.0 * A * C, 0.0);
  double sq = sqrt(disc);
  double i2a = 0.5 / A;
  double c1 = (-B + sq) * i2a, c2 = (-B - sq) * i2a;
  return fmax(fabs(c1), fabs(c2));
}

template <int TX, int TY, int H>
struct ExpSmem {
  static constexpr int PX = TX + 2 * H, PY = TY + 2 * H;   // staged P^E tile
  static constexpr int F1X = TX + 1, F1Y = TY + 2;         // X1 faces i = 0..TX, rows -1..TY
  static constexpr int F2X = TX + 2, F2Y = TY + 1;         // X2 faces cols -1..TX, j = 0..TY
  static constexpr int DX = TX + 2, DY = TY + 2;           // derived quantities, halo 1
  static constexpr int EX = TX + 1, EY = TY + 1;           // corner EMFs
  static constexpr int nP = NV * PX * PY;
  static constexpr int nF1 = NV * F1X * F1Y;
  static constexpr int nF2 = NV * F2X * F2Y;
  static constexpr int nD = 5 * DX * DY;
  static constexpr int nE = EX * EY;
  static constexpr size_t bytes = sizeof(double) * (nP + nF1 + nF2 + nD + nE);
};

// Reconstructed face states at the face on the low side of tile zone
// (ci, cj) in direction d (0: X1, 1: X2), from the staged tile.
template <int TX, int TY, int H>
__device__ __forceinline__ void face_states(const double* sP, const Params& p, int d, int ci, int cj, double L[NV],
                                            double R[NV]) {
  using S = ExpSmem<TX, TY, H>;
  const int stride = (d == 0) ? 1 : S::PX;
  const int base = (cj + H) * S::PX + (ci + H);  // the zone right of the face
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const double* q = sP + v * S::PX * S::PY + base;
    if (p.recon == RECON_WENO5) {
      double m3 = q[-3 * stride], m2 = q[-2 * stride], m1 = q[-stride], z0 = q[0], p1 = q[stride], p2 = q[2 * stride];
      L[v] = weno5(m3, m2, m1, z0, p1);
      R[v] = weno5(p2, p1, z0, m1, m2);
    } else {
      double m2 = q[-2 * stride], m1 = q[-stride], z0 = q[0], p1 = q[stride];
      L[v] = m1 + 0.5 * mc_slope(p.theta, m2, m1, z0);
      R[v] = z0 - 0.5 * mc_slope(p.theta, m1, z0, p1);
    }
  }
}

template <int TX, int TY, int H>
__global__ void __launch_bounds__(TX* TY) explicit_stage_2d(const __grid_constant__ Params p,
                                                            const double* Pn,
                                                            const double* __restrict__ PE,
                                                            const double* guess, double dts,
                                                            double* __restrict__ K, double* P0) {
  using S = ExpSmem<TX, TY, H>;
  extern __shared__ double smem[];
  double* sP = smem;
  double* sF1 = sP + S::nP;
  double* sF2 = sF1 + S::nF1;
  double* sD = sF2 + S::nF2;
  double* sE = sD + S::nD;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const long long N = p.N;

  // 1. stage P^E (tile + halo H) with the boundary rules
  for (int e = tid; e < S::PX * S::PY; e += TX * TY) {
    int cx = e % S::PX, cy = e / S::PX;
    bool f1 = false, f2 = false;
    int gi = map_index(i0 + cx - H, p.n1, p.bc[0][0], p.bc[0][1], f1);
    int gj = map_index(j0 + cy - H, p.n2, p.bc[1][0], p.bc[1][1], f2);
    long long z = (long long)gj * p.n1 + gi;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double x = __ldg(PE + v * N + z);
      if ((f1 && (v == 2 || v == 5)) || (f2 && (v == 3 || v == 6))) x = -x;
      sP[v * S::PX * S::PY + e] = x;
    }
  }
  __syncthreads();

  // 2. derived quantities for the slope-limited source derivatives (halo 1):
  //    Theta, u_t, u_1, u_2, u_3
  for (int e = tid; e < S::DX * S::DY; e += TX * TY) {
    int cx = e % S::DX, cy = e / S::DX;
    int se = (cy - 1 + H) * S::PX + (cx - 1 + H);
    double rho = sP[0 * S::PX * S::PY + se], u = sP[1 * S::PX * S::PY + se];
    double v1 = sP[2 * S::PX * S::PY + se], v2 = sP[3 * S::PX * S::PY + se], v3 = sP[4 * S::PX * S::PY + se];
    sD[0 * S::DX * S::DY + e] = (p.gamma - 1.0) * u / rho;
    sD[1 * S::DX * S::DY + e] = -sqrt(1.0 + v1 * v1 + v2 * v2 + v3 * v3);
    sD[2 * S::DX * S::DY + e] = v1;
    sD[3 * S::DX * S::DY + e] = v2;
    sD[4 * S::DX * S::DY + e] = v3;
  }

  // 3. LLF face fluxes: X1 faces then X2 faces
  const int nf1 = S::F1X * S::F1Y, nf2 = S::F2X * S::F2Y;
  for (int f = tid; f < nf1 + nf2; f += TX * TY) {
    int d, ci, cj;
    if (f < nf1) { d = 0; ci = f % S::F1X; cj = f / S::F1X - 1; }
    else { int g = f - nf1; d = 1; ci = g % S::F2X - 1; cj = g / S::F2X; }
    double L[NV], R[NV];
    face_states<TX, TY, H>(sP, p, d, ci, cj, L, R);
    Pt<double> sl, sr;
    point_state(L, p, sl);
    point_state(R, p, sr);
    double UL[NV], FL[NV], UR[NV], FR[NV];
    cons_flux(sl, L, d + 1, UL, FL);
    cons_flux(sr, R, d + 1, UR, FR);
    double cm = fmax(max_speed(sl, p, d + 1), max_speed(sr, p, d + 1));
    double* out = (d == 0) ? sF1 + (cj + 1) * S::F1X + ci : sF2 + cj * S::F2X + (ci + 1);
    const int plane = (d == 0) ? S::F1X * S::F1Y : S::F2X * S::F2Y;
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * plane] = 0.5 * (FL[v] + FR[v]) - 0.5 * cm * (UR[v] - UL[v]);
  }
  __syncthreads();

  // 4. flux-CT corner values E(i,j) at (i-1/2, j-1/2), i = 0..TX, j = 0..TY:
  //    the average of the four face estimates of F^1[B^2] = -F^2[B^1]
  for (int e = tid; e < S::EX * S::EY; e += TX * TY) {
    int ci = e % S::EX, cj = e / S::EX;
    const double* f1b2 = sF1 + 6 * S::F1X * S::F1Y;
    const double* f2b1 = sF2 + 5 * S::F2X * S::F2Y;
    double a = f1b2[(cj + 1) * S::F1X + ci] + f1b2[cj * S::F1X + ci];
    double b = f2b1[cj * S::F2X + (ci + 1)] + f2b1[cj * S::F2X + ci];
    sE[e] = 0.25 * (a - b);
  }
  __syncthreads();

  // 5. per-zone constants
  const int ti = tid % TX, tj = tid / TX;
  const int gi = i0 + ti, gj = j0 + tj;
  if (gi >= p.n1 || gj >= p.n2) return;
  const long long z = (long long)gj * p.n1 + gi;
  const double idx1 = p.idx[0], idx2 = p.idx[1];

  double divF[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const double* f1 = sF1 + v * S::F1X * S::F1Y;
    const double* f2 = sF2 + v * S::F2X * S::F2Y;
    double a = (f1[(tj + 1) * S::F1X + ti + 1] - f1[(tj + 1) * S::F1X + ti]) * idx1;
    double b = (f2[(tj + 1) * S::F2X + ti + 1] - f2[tj * S::F2X + ti + 1]) * idx2;
    if (v == 5) a = 0.0;  // F^1[B^1] = 0 under flux-CT
    if (v == 6) b = 0.0;  // F^2[B^2] = 0
    divF[v] = a + b;
  }
  {
    // F^1[B^2](i,j) = (E(i,j) + E(i,j+1))/2, F^2[B^1](i,j) = -(E(i,j) + E(i+1,j))/2
    double e00 = sE[tj * S::EX + ti], e10 = sE[tj * S::EX + ti + 1];
    double e01 = sE[(tj + 1) * S::EX + ti], e11 = sE[(tj + 1) * S::EX + ti + 1];
    divF[6] = (0.5 * (e10 + e11) - 0.5 * (e00 + e01)) * idx1;
    divF[5] = (-0.5 * (e01 + e11) + 0.5 * (e00 + e10)) * idx2;
  }

  // states at P^E and P_n
  double PEz[NV], Pnz[NV];
  const int se = (tj + H) * S::PX + (ti + H);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    PEz[v] = sP[v * S::PX * S::PY + se];
    Pnz[v] = Pn[v * N + z];  // plain load: P0 may be Pn (an in-place step)
  }
  Pt<double> sE_, sn;
  point_state(PEz, p, sE_);
  point_state(Pnz, p, sn);
  double Un[NV], rown[4];
  stress_row(sn, 0, rown);
  Un[0] = sn.rho * sn.ut;
  Un[1] = rown[0]; Un[2] = rown[1]; Un[3] = rown[2]; Un[4] = rown[3];
  Un[5] = Pnz[5]; Un[6] = Pnz[6]; Un[7] = Pnz[7];
  Un[8] = sn.qt * sn.ut; Un[9] = sn.dpt * sn.ut;

  // slope-limited spatial derivatives at P^E: d_i Theta, d_i u_nu, and the
  // spatial part of nabla_mu u^mu (flat: d_i u^i)
  double dTh[2], du[2][4], divu_sp = 0.0;
  const int de = (tj + 1) * S::DX + (ti + 1);
#pragma unroll
  for (int d = 0; d < 2; d++) {
    const int st = (d == 0) ? 1 : S::DX;
    const double ih = (d == 0) ? idx1 : idx2;
    const double* th = sD;
    dTh[d] = mc_slope(p.theta, th[de - st], th[de], th[de + st]) * ih;
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const double* uq = sD + (1 + m) * S::DX * S::DY;
      du[d][m] = mc_slope(p.theta, uq[de - st], uq[de], uq[de + st]) * ih;
    }
    divu_sp += du[d][1 + d];
  }

  const double tau = p.tauR, idts = 1.0 / dts;
  double s[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) s[v] = dts / (fabs(Un[v]) + fabs(Un[0]));

  double* Kz = K + z;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    Kz[(K_U + v) * N] = s[v] * idts;
    Kz[(K_C + v) * N] = s[v] * (divF[v] - Un[v] * idts);
  }
  // coefficients at P^E
  const double rhoE = sE_.rho, thE = sE_.theta, cs2E = sE_.cs2;
  const double bhu[4] = {sE_.bht, sE_.bh[0], sE_.bh[1], sE_.bh[2]};
  const double ucovn[4] = {-sn.ut, sn.uc[0], sn.uc[1], sn.uc[2]};
  // spatial velocities at P^E (u^1, u^2) for the convective parts of a_mu
  const double uEx = sE_.uc[0], uEy = sE_.uc[1];
  const double hoq = p.ho ? 0.5 * sE_.qt : 0.0;
  const double hod = p.ho ? 0.5 * sE_.dpt : 0.0;

  // --- heat flux row: q~_0 = Aq + Bq (Theta - Theta_n)/dts + Cq^mu (u_mu - u_mu,n)/dts
  double Aq = 0.0, Bq = 0.0, Cq[4] = {0.0, 0.0, 0.0, 0.0};
  if (p.cond) {
    const double chi = p.phi * cs2E * tau;
    const double Kq = sqrt(tau / (chi * rhoE * thE * thE));
    const double pre = -Kq * rhoE * chi;
    // spatial parts: bhat^i d_i Theta + Theta bhat^mu u^i d_i u_mu
    double sp = bhu[1] * dTh[0] + bhu[2] * dTh[1];
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 4; m++) acc += bhu[m] * (uEx * du[0][m] + uEy * du[1][m]);
    Aq = pre * (sp + thE * acc);
    Bq = pre * bhu[0];
#pragma unroll
    for (int m = 0; m < 4; m++) Cq[m] = pre * thE * bhu[m] * sE_.ut;
  }
  {
    const double s8 = s[8];
    double cst = -Un[8] * idts + divF[8] + 0.5 * sn.qt / tau - Aq / tau + (Bq * sn.theta) * idts / tau;
#pragma unroll
    for (int m = 0; m < 4; m++) cst += Cq[m] * ucovn[m] * idts / tau;
    cst -= hoq * (divu_sp - sn.ut * idts);
    Kz[(K_C + 8) * N] = s8 * cst;
    Kz[(K_Q + 0) * N] = s8 * 0.5 / tau;
    Kz[(K_Q + 1) * N] = -s8 * Bq * idts / tau;
#pragma unroll
    for (int m = 0; m < 4; m++) Kz[(K_Q + 2 + m) * N] = -s8 * Cq[m] * idts / tau;
    Kz[(K_Q + 6) * N] = -s8 * hoq * idts;
  }
  // --- anisotropy row: dP~_0 = Ad + Dd^nu (u_nu - u_nu,n)/dts + Ed (u^t - u^t_n)/dts
  double Ad = 0.0, Dd[4] = {0.0, 0.0, 0.0, 0.0}, Ed = 0.0;
  if (p.visc) {
    const double nu = p.psi * cs2E * tau;
    const double Kd = sqrt(tau / (nu * rhoE * thE));
    const double pre = Kd * 3.0 * rhoE * nu;
    double sp = 0.0;
#pragma unroll
    for (int m = 0; m < 4; m++) sp += bhu[m] * (bhu[1] * du[0][m] + bhu[2] * du[1][m]);
    Ad = pre * (sp - divu_sp / 3.0);
#pragma unroll
    for (int m = 0; m < 4; m++) Dd[m] = pre * bhu[0] * bhu[m];
    Ed = -pre / 3.0;
  }
  {
    const double s9 = s[9];
    double cst = -Un[9] * idts + divF[9] + 0.5 * sn.dpt / tau - Ad / tau + Ed * sn.ut * idts / tau;
#pragma unroll
    for (int m = 0; m < 4; m++) cst += Dd[m] * ucovn[m] * idts / tau;
    cst -= hod * (divu_sp - sn.ut * idts);
    Kz[(K_C + 9) * N] = s9 * cst;
    Kz[(K_D + 0) * N] = s9 * 0.5 / tau;
#pragma unroll
    for (int m = 0; m < 4; m++) Kz[(K_D + 1 + m) * N] = -s9 * Dd[m] * idts / tau;
    Kz[(K_D + 5) * N] = -s9 * (Ed * idts / tau + hod * idts);
  }

  // initial guess: P_n (or the given guess) with B from the explicit flux-CT update
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double x = guess ? guess[v * N + z] : Pnz[v];
    if (v >= 5 && v <= 7) x = Pnz[v] - dts * divF[v];
    P0[v * N + z] = x;
  }
}

// Host launcher.
template <int TX, int TY, int H>
static cudaError_t launch_explicit_t(const Params& p, const double* Pn, const double* PE, const double* guess,
                                     double dts, double* K, double* P0, cudaStream_t st) {
  using S = ExpSmem<TX, TY, H>;
  static PerDevice once;
  cudaError_t e = once.get([](int*) {
    return cudaFuncSetAttribute(explicit_stage_2d<TX, TY, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)S::bytes);
  });
  if (e != cudaSuccess) return e;
  dim3 grid((p.n1 + TX - 1) / TX, (p.n2 + TY - 1) / TY);
  explicit_stage_2d<TX, TY, H><<<grid, TX * TY, S::bytes, st>>>(p, Pn, PE, guess, dts, K, P0);
  return cudaGetLastError();
}

cudaError_t launch_explicit(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                            double* K, double* P0, cudaStream_t st) {
  if (p.recon == RECON_WENO5) return launch_explicit_t<16, 16, 3>(p, Pn, PE, guess, dts, K, P0, st);
  return launch_explicit_t<16, 16, 2>(p, Pn, PE, guess, dts, K, P0, st);
}

}  // namespace grim
