// grim oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow FP64 CPU restatement of the implicit EMHD zone step of
// Chandra, Foucart & Gammie (2017), "grim: a flexible, conservative scheme for
// relativistic fluid theories".  It exists to check the CUDA library against
// the paper.  Only the test suite, the smoke check and the benchmark's CPU
// baseline may load it; the product library never calls it and shares no code
// with it.
//
// Everything here follows the paper's equations in the paper's order, one zone
// at a time (OpenMP over zones), with no blocking, fusion or reordering beyond
// what the equations state.  The physics is templated on the scalar type so the
// same code also runs on complex numbers (complex-step derivatives), forward
// dual numbers (chain rule for the linearised source) and a flop-counting type.
//
// Readings of the paper (each is also listed in the design notes):
//  * induction flux: the printed flux of Eq. induction_eqn, sqrt(-g)(b^j u^i -
//    b^i u^j), has the opposite sign to the divergence of the dual Faraday
//    tensor *F^{mu nu} = b^mu u^nu - b^nu u^mu with the printed b^mu; with the
//    printed sign Alfven waves grow.  We use sqrt(-g)(b^i u^j - b^j u^i); with
//    it the linearised system reproduces the Table 1 eigenvalue and
//    eigenvector to 1e-10.
//  * primitives: rho, u, three velocity components, B^i, and the rescaled
//    q~, dP~ of Eqs. q, dP.  The velocity is the normal-observer velocity
//    u~^i (u^t = gamma/alpha, u^i = u~^i - gamma*alpha*g^{ti}); in Minkowski
//    space it is exactly the u^i of the paper.
//  * relaxation sources (Eqs. q_evol_eqn_rescaled, dP_evol_eqn_rescaled):
//    implicit part ((X + X_n)/2)/tau_R[P^E] (Section 2.3); q~_0, dP~_0 with
//    coefficients at P^E, spatial derivatives slope limited at P^E, time
//    derivatives as difference quotients (Theta(P)-Theta(P_n))/dt_s,
//    (u_mu(P)-u_mu(P_n))/dt_s, (u^t(P)-u^t(P_n))/dt_s; the higher-order
//    coefficient X/2 taken at P^E.  Eq. dP0def is read with nabla_mu u_nu.
//  * geometric source sqrt(-g) T^k_l Gamma^l_{nu k} explicit at P^E.
//  * residual scale r_i = dt_s R_i / (|U_i(P_n)| + |U_0(P_n)|), frozen per
//    zone per stage; converged when max_i |r_i| <= tol, tested before each
//    Jacobian (Section 3 leaves the norm open).
//  * FD Jacobian (Section 3.1): only component j is perturbed; the divisor is
//    the computed difference P_eps,j - P_j.  small() is there to keep that
//    divisor away from zero, but taken literally (P_eps,j = eps when
//    |P_j| < 5 eps) it makes the divisor vanish at P_j = eps and tiny near
//    it; we perturb small components by +eps (P_eps,j = P_j + eps), which is
//    the printed formula at P_j = 0, the case the text discusses.
//  * line search (Section 3.2): the acceptance test is compared in squared
//    form; a non-finite trial halves lambda; after ls_max backtracks the last
//    trial is taken and a stall flag is set.
//  * magnetic field: solved in the 10x10 system with its guess set to the
//    explicit flux-CT update (its rows are linear and decoupled, so the root
//    is the explicit value and div B is kept to round-off).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------- scalars
// Flop-counting scalar.  A value is either a constant of the zone (dep =
// false: anything that does not depend on the unknown P) or depends on P.
// Only operations with a P-dependent operand are counted (constants are
// hoisted, as the paper precomputes the P_n-only terms, Section 7.1), each
// +,-,*,/ and sqrt as one flop; multiplying by a constant 0 or +-1, adding a
// constant 0 or dividing by a constant 1 is structural and not counted.
struct Cnt {
  double v;
  bool dep;
  Cnt() : v(0), dep(false) {}
  Cnt(double x) : v(x), dep(false) {}
  Cnt(double x, bool d) : v(x), dep(d) {}
};
static thread_local long long g_flops = 0;
inline Cnt operator+(Cnt a, Cnt b) {
  if (!a.dep && !b.dep) return Cnt(a.v + b.v);
  if (!a.dep && a.v == 0.0) return b;
  if (!b.dep && b.v == 0.0) return a;
  g_flops++;
  return Cnt(a.v + b.v, true);
}
inline Cnt operator-(Cnt a) { return Cnt(-a.v, a.dep); }
inline Cnt operator-(Cnt a, Cnt b) {
  if (!a.dep && !b.dep) return Cnt(a.v - b.v);
  if (!a.dep && a.v == 0.0) return -b;
  if (!b.dep && b.v == 0.0) return a;
  g_flops++;
  return Cnt(a.v - b.v, true);
}
inline Cnt operator*(Cnt a, Cnt b) {
  if (!a.dep && !b.dep) return Cnt(a.v * b.v);
  if (!a.dep && a.v == 0.0) return Cnt(0.0);
  if (!b.dep && b.v == 0.0) return Cnt(0.0);
  if (!a.dep && a.v == 1.0) return b;
  if (!b.dep && b.v == 1.0) return a;
  if (!a.dep && a.v == -1.0) return -b;
  if (!b.dep && b.v == -1.0) return -a;
  g_flops++;
  return Cnt(a.v * b.v, true);
}
inline Cnt operator/(Cnt a, Cnt b) {
  if (!a.dep && !b.dep) return Cnt(a.v / b.v);
  if (!b.dep && b.v == 1.0) return a;
  g_flops++;
  return Cnt(a.v / b.v, true);
}
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt& operator/=(Cnt& a, Cnt b) { a = a / b; return a; }
inline Cnt sqrt(Cnt a) {
  if (!a.dep) return Cnt(std::sqrt(a.v));
  g_flops++;
  return Cnt(std::sqrt(a.v), true);
}
inline double re(Cnt a) { return a.v; }
inline bool operator>(Cnt a, double b) { return a.v > b; }
inline bool operator<(Cnt a, double b) { return a.v < b; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline Cnt tabs(Cnt a) { return Cnt(std::fabs(a.v), a.dep); }
inline Cnt tmin(Cnt a, Cnt b) { return a.v < b.v ? a : b; }
inline Cnt tmax(Cnt a, Cnt b) { return a.v > b.v ? a : b; }
inline double tabs(double a) { return std::fabs(a); }
inline double tmin(double a, double b) { return std::min(a, b); }
inline double tmax(double a, double b) { return std::max(a, b); }

// Forward-mode dual number over any scalar T (value + one directional derivative).
template <class T> struct Dual {
  T v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(T x, T y) : v(x), d(y) {}
};
template <class T> Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <class T> Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <class T> Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class T> Dual<T> operator/(Dual<T> a, Dual<T> b) {
  return Dual<T>(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
template <class T> Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <class T> Dual<T> operator+(Dual<T> a, double b) { return a + Dual<T>(b); }
template <class T> Dual<T> operator+(double a, Dual<T> b) { return Dual<T>(a) + b; }
template <class T> Dual<T> operator-(Dual<T> a, double b) { return a - Dual<T>(b); }
template <class T> Dual<T> operator-(double a, Dual<T> b) { return Dual<T>(a) - b; }
template <class T> Dual<T> operator*(Dual<T> a, double b) { return a * Dual<T>(b); }
template <class T> Dual<T> operator*(double a, Dual<T> b) { return Dual<T>(a) * b; }
template <class T> Dual<T> operator/(Dual<T> a, double b) { return a / Dual<T>(b); }
template <class T> Dual<T> operator/(double a, Dual<T> b) { return Dual<T>(a) / b; }
template <class T> Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a = a + b; return a; }
template <class T> Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a = a - b; return a; }
template <class T> Dual<T> sqrt(Dual<T> a) {
  using std::sqrt;
  T s = sqrt(a.v);
  return Dual<T>(s, a.d / (2.0 * s));
}

template <class T> Dual<T> exp(Dual<T> a) {
  T e = std::exp(a.v);
  return Dual<T>(e, e * a.d);
}
template <class T> Dual<T> sin(Dual<T> a) { return Dual<T>(std::sin(a.v), std::cos(a.v) * a.d); }
template <class T> Dual<T> cos(Dual<T> a) { return Dual<T>(std::cos(a.v), -std::sin(a.v) * a.d); }
template <class T> Dual<T> fabs_d(Dual<T> a) { return a.v < 0 ? -a : a; }
inline double fabs_d(double a) { return std::fabs(a); }
using std::exp;
using std::sin;
using std::cos;
inline double re(double a) { return a; }
inline double re(const std::complex<double>& a) { return a.real(); }
template <class T> double re(const Dual<T>& a) { return re(a.v); }
using std::sqrt;
using cplx = std::complex<double>;

// ---------------------------------------------------------------- parameters
// Integer and real parameter vectors, laid out as documented in oracle.py.
enum {
  I_DIM, I_N1, I_N2, I_N3, I_BC1L, I_BC1H, I_BC2L, I_BC2H, I_BC3L, I_BC3H,
  I_METRIC, I_RECON, I_COND, I_VISC, I_HO, I_KMAX, I_LSMAX, I_FLOORS, I_RIEMANN, I_NTHREADS, I_COUNT
};
enum {
  D_X01, D_X02, D_X03, D_DX1, D_DX2, D_DX3, D_GAMMA, D_PHI, D_PSI, D_TAUR,
  D_THETA, D_TOL, D_EPS, D_A, D_H, D_COUNT
};
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2 };
enum { METRIC_MINKOWSKI = 0, METRIC_MKS_KERR = 1 };
enum { RECON_MC = 0, RECON_WENO5 = 1, RECON_PPM = 2 };
enum { ST_MAXIT = 1, ST_LSSTALL = 2, ST_SINGULAR = 4, ST_NONFINITE = 8, ST_INADMISSIBLE = 16 };

struct Params {
  int dim, n[3], bc[3][2], metric, recon, cond, visc, ho, kmax, lsmax, floors, riemann;
  double x0[3], dx[3], gamma, phi, psi, tauR, theta, tol, eps, a, h;
  long long N;
};

static Params read_params(const int* ip, const double* dp) {
  Params p;
  p.dim = ip[I_DIM];
  p.n[0] = ip[I_N1]; p.n[1] = ip[I_N2]; p.n[2] = ip[I_N3];
  p.bc[0][0] = ip[I_BC1L]; p.bc[0][1] = ip[I_BC1H];
  p.bc[1][0] = ip[I_BC2L]; p.bc[1][1] = ip[I_BC2H];
  p.bc[2][0] = ip[I_BC3L]; p.bc[2][1] = ip[I_BC3H];
  p.metric = ip[I_METRIC]; p.recon = ip[I_RECON];
  p.cond = ip[I_COND]; p.visc = ip[I_VISC]; p.ho = ip[I_HO];
  p.kmax = ip[I_KMAX]; p.lsmax = ip[I_LSMAX]; p.floors = ip[I_FLOORS]; p.riemann = ip[I_RIEMANN];
  for (int d = 0; d < 3; d++) { p.x0[d] = dp[D_X01 + d]; p.dx[d] = dp[D_DX1 + d]; }
  p.gamma = dp[D_GAMMA]; p.phi = dp[D_PHI]; p.psi = dp[D_PSI]; p.tauR = dp[D_TAUR];
  p.theta = dp[D_THETA]; p.tol = dp[D_TOL]; p.eps = dp[D_EPS]; p.a = dp[D_A]; p.h = dp[D_H];
  p.N = (long long)p.n[0] * p.n[1] * p.n[2];
  return p;
}

// ---------------------------------------------------------------- geometry
// Metric quantities at one point (Section 2.1): g_{mu nu}, g^{mu nu},
// sqrt(-g), the lapse alpha = 1/sqrt(-g^{tt}), Gamma^l_{mu nu}, and the
// relaxation time there.
struct Geom {
  double gcov[4][4], gcon[4][4], sqrtg, alpha, Gam[4][4][4], tauR;
};

static void geom_minkowski(Geom& g, double tauR) {
  std::memset(&g, 0, sizeof(g));
  for (int m = 0; m < 4; m++) { g.gcov[m][m] = (m == 0) ? -1.0 : 1.0; g.gcon[m][m] = g.gcov[m][m]; }
  g.sqrtg = 1.0; g.alpha = 1.0; g.tauR = tauR;
}

// Modified Kerr-Schild coordinates (Section 2.1 with the Kerr-Schild form of
// the Kerr metric, M = 1): r = exp(X^1), theta = pi X^2 + ((1-h)/2) sin(2 pi
// X^2), phi = X^3.  g_{mu nu}(X) = L^a_mu L^b_nu g^KS_ab with L = diag(1,
// dr/dX^1, dtheta/dX^2, 1).  Kerr-Schild (t, r, theta, phi), Sigma = r^2 +
// a^2 cos^2 theta:
//   g_tt = -(1 - 2r/Sigma), g_tr = 2r/Sigma, g_tphi = -2 a r sin^2/Sigma,
//   g_rr = 1 + 2r/Sigma, g_rphi = -a sin^2 (1 + 2r/Sigma), g_thth = Sigma,
//   g_phiphi = sin^2 (Sigma + a^2 sin^2 (1 + 2r/Sigma)).
// T is double or a dual number (derivative along X^1 or X^2).
template <class T> static void mks_theta(double h, T X2, T& th, T& dth) {
  th = M_PI * X2 + 0.5 * (1.0 - h) * sin(2.0 * M_PI * X2);
  dth = M_PI * (1.0 + (1.0 - h) * cos(2.0 * M_PI * X2));
}
template <class T> static void mks_gcov(double a, double h, T X1, T X2, T g[4][4]) {
  T r = exp(X1);
  T th, dth;
  mks_theta(h, X2, th, dth);
  T sn = sin(th), cs = cos(th);
  T s2 = sn * sn;
  T sig = r * r + a * a * cs * cs;
  T f = 2.0 * r / sig;
  T ks[4][4];
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) ks[m][n] = T(0.0);
  ks[0][0] = -(1.0 - f);
  ks[0][1] = f;
  ks[0][3] = -a * f * s2;
  ks[1][1] = 1.0 + f;
  ks[1][3] = -a * s2 * (1.0 + f);
  ks[2][2] = sig;
  ks[3][3] = s2 * (sig + a * a * s2 * (1.0 + f));
  T L[4] = {T(1.0), r, dth, T(1.0)};
  for (int m = 0; m < 4; m++)
    for (int n = m; n < 4; n++) {
      g[m][n] = ks[m][n] * L[m] * L[n];
      g[n][m] = g[m][n];
    }
}

// Inverse and determinant of a symmetric 4x4 by Gauss-Jordan elimination with
// partial pivoting.
static double invert4(const double A[4][4], double inv[4][4]) {
  double M[4][8];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 8; j++) M[i][j] = (j < 4) ? A[i][j] : (j - 4 == i ? 1.0 : 0.0);
  double det = 1.0;
  for (int c = 0; c < 4; c++) {
    int pv = c;
    for (int i = c + 1; i < 4; i++)
      if (std::fabs(M[i][c]) > std::fabs(M[pv][c])) pv = i;
    if (pv != c) {
      for (int j = 0; j < 8; j++) std::swap(M[c][j], M[pv][j]);
      det = -det;
    }
    const double d = M[c][c];
    det *= d;
    for (int j = 0; j < 8; j++) M[c][j] /= d;
    for (int i = 0; i < 4; i++) {
      if (i == c) continue;
      const double f = M[i][c];
      for (int j = 0; j < 8; j++) M[i][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) inv[i][j] = M[i][j + 4];
  return det;
}

// Geometry of MKS-Kerr at X (X^3 plays no role: the metric is axisymmetric
// and stationary).  Gamma^l_{mu nu} = (1/2) g^{l k} (d_mu g_{k nu} + d_nu
// g_{k mu} - d_k g_{mu nu}) with the derivatives along X^1 and X^2 from
// forward dual numbers.  sqrt(-g) from the determinant.  tau_R = tau_R0
// r^{3/2} (the relaxation time grows with the local dynamical time).
static void geom_mks(const Params& p, const double X[3], Geom& G) {
  std::memset(&G, 0, sizeof(G));
  double g[4][4];
  mks_gcov<double>(p.a, p.h, X[0], X[1], g);
  std::memcpy(G.gcov, g, sizeof(g));
  const double det = invert4(g, G.gcon);
  G.sqrtg = std::sqrt(-det);
  G.alpha = 1.0 / std::sqrt(-G.gcon[0][0]);
  double dg[4][4][4];  // dg[k][m][n] = d_k g_{mn}
  std::memset(dg, 0, sizeof(dg));
  for (int d = 1; d <= 2; d++) {
    Dual<double> x1(X[0], d == 1 ? 1.0 : 0.0), x2(X[1], d == 2 ? 1.0 : 0.0);
    Dual<double> gd[4][4];
    mks_gcov<Dual<double>>(p.a, p.h, x1, x2, gd);
    for (int m = 0; m < 4; m++)
      for (int n = 0; n < 4; n++) dg[d][m][n] = gd[m][n].d;
  }
  for (int l = 0; l < 4; l++)
    for (int m = 0; m < 4; m++)
      for (int n = 0; n < 4; n++) {
        double acc = 0.0;
        for (int k = 0; k < 4; k++) acc += G.gcon[l][k] * (dg[m][k][n] + dg[n][k][m] - dg[k][m][n]);
        G.Gam[l][m][n] = 0.5 * acc;
      }
  const double r = std::exp(X[0]);
  G.tauR = p.tauR * r * std::sqrt(r);
}

// A face of MKS-Kerr on the polar axis (sin theta = 0 there, so sqrt(-g) and
// every flux through it vanish).
static bool polar_face(const Params& p, const double X[3], int d) {
  if (p.metric != METRIC_MKS_KERR || d != 1) return false;
  double th, dth;
  mks_theta<double>(p.h, X[1], th, dth);
  return std::fabs(std::sin(th)) < 1e-10;
}

static void geom_at(const Params& p, const double X[3], Geom& g) {
  if (p.metric == METRIC_MKS_KERR) geom_mks(p, X, g);
  else geom_minkowski(g, p.tauR);
}

// ---------------------------------------------------------------- fluid state
// Derived quantities at a primitive vector P (Section 4): four-velocity,
// magnetic four-vector b^mu = (B^i u_i, (B^i + b^t u^i)/u^t), b^2, unit
// vector bhat, gas pressure P_g = (gamma-1)u, Theta = P_g/rho, sound speed,
// closure chi = phi c_s^2 tau_R, nu = psi c_s^2 tau_R (Section 4), and the
// physical q, dP recovered from the rescaled primitives (Eqs. q, dP).
template <class T> struct State {
  T rho, u, Pg, Theta, cs2, chi, nu, qt, dPt, q, dP, bsq;
  T ucon[4], ucov[4], bcon[4], bcov[4], bhcon[4], bhcov[4], B[3];
  double tauR, sqrtg;
};

template <class T> static void make_state(const T* P, const Geom& g, const Params& p, State<T>& s) {
  s.rho = P[0]; s.u = P[1];
  T vt[3] = {P[2], P[3], P[4]};
  T qsq = T(0.0);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) qsq = qsq + g.gcov[i + 1][j + 1] * vt[i] * vt[j];
  T lor = sqrt(T(1.0) + qsq);
  s.ucon[0] = lor / g.alpha;
  for (int i = 0; i < 3; i++) s.ucon[i + 1] = vt[i] - lor * g.alpha * g.gcon[0][i + 1];
  for (int m = 0; m < 4; m++) {
    s.ucov[m] = T(0.0);
    for (int n = 0; n < 4; n++) s.ucov[m] = s.ucov[m] + g.gcov[m][n] * s.ucon[n];
  }
  for (int i = 0; i < 3; i++) s.B[i] = P[5 + i];
  s.bcon[0] = T(0.0);
  for (int i = 0; i < 3; i++) s.bcon[0] = s.bcon[0] + s.B[i] * s.ucov[i + 1];
  for (int i = 0; i < 3; i++) s.bcon[i + 1] = (s.B[i] + s.bcon[0] * s.ucon[i + 1]) / s.ucon[0];
  s.bsq = T(0.0);
  for (int m = 0; m < 4; m++) {
    s.bcov[m] = T(0.0);
    for (int n = 0; n < 4; n++) s.bcov[m] = s.bcov[m] + g.gcov[m][n] * s.bcon[n];
    s.bsq = s.bsq + s.bcon[m] * s.bcov[m];
  }
  s.Pg = (p.gamma - 1.0) * s.u;
  s.Theta = s.Pg / s.rho;
  s.cs2 = p.gamma * s.Pg / (s.rho + p.gamma * s.u);
  s.tauR = g.tauR;
  s.sqrtg = g.sqrtg;
  s.chi = p.cond ? p.phi * s.cs2 * g.tauR : T(0.0);
  s.nu = p.visc ? p.psi * s.cs2 * g.tauR : T(0.0);
  s.qt = P[8]; s.dPt = P[9];
  s.q = p.cond ? s.qt * sqrt(s.chi * s.rho * s.Theta * s.Theta / g.tauR) : T(0.0);
  s.dP = p.visc ? s.dPt * sqrt(s.nu * s.rho * s.Theta / g.tauR) : T(0.0);
  if (re(s.bsq) > 0.0) {
    T bn = sqrt(s.bsq);
    for (int m = 0; m < 4; m++) { s.bhcon[m] = s.bcon[m] / bn; s.bhcov[m] = s.bcov[m] / bn; }
  } else {
    for (int m = 0; m < 4; m++) { s.bhcon[m] = T(0.0); s.bhcov[m] = T(0.0); }
  }
}

// Row m of the mixed stress tensor T^m_nu of Eq. fullSEtens with
// q^mu = q bhat^mu and Pi^{mu nu} = -dP (bhat^mu bhat^nu - h^{mu nu}/3),
// h^mu_nu = delta^mu_nu + u^mu u_nu.
template <class T> static void stress_row(const State<T>& s, int m, T Trow[4]) {
  T w = s.rho + s.u + s.Pg + s.bsq;
  T pt = s.Pg + 0.5 * s.bsq;
  for (int n = 0; n < 4; n++) {
    double del = (m == n) ? 1.0 : 0.0;
    T h = del + s.ucon[m] * s.ucov[n];
    Trow[n] = w * s.ucon[m] * s.ucov[n] + pt * del - s.bcon[m] * s.bcov[n]
            + s.q * (s.bhcon[m] * s.ucov[n] + s.ucon[m] * s.bhcov[n])
            - s.dP * (s.bhcon[m] * s.bhcov[n] - h / 3.0);
  }
}
template <class T> static void stress(const State<T>& s, T Tmn[4][4]) {
  for (int m = 0; m < 4; m++) stress_row(s, m, Tmn[m]);
}

// Conserved variables (Eqs. divN_explicit, divT_explicit, induction_eqn and the
// left sides of Eqs. q_evol_eqn_rescaled, dP_evol_eqn_rescaled times sqrt(-g)).
template <class T> static void conserved(const State<T>& s, T U[10]) {
  T Trow[4];
  stress_row(s, 0, Trow);
  U[0] = s.sqrtg * s.rho * s.ucon[0];
  for (int n = 0; n < 4; n++) U[1 + n] = s.sqrtg * Trow[n];
  for (int i = 0; i < 3; i++) U[5 + i] = s.sqrtg * s.B[i];
  U[8] = s.sqrtg * s.qt * s.ucon[0];
  U[9] = s.sqrtg * s.dPt * s.ucon[0];
}

// Flux in direction j (1..3).  The induction flux uses the sign derived from
// the dual Faraday tensor (see header).
template <class T> static void flux(const State<T>& s, int j, T F[10]) {
  T Trow[4];
  stress_row(s, j, Trow);
  F[0] = s.sqrtg * s.rho * s.ucon[j];
  for (int n = 0; n < 4; n++) F[1 + n] = s.sqrtg * Trow[n];
  for (int i = 0; i < 3; i++) F[5 + i] = s.sqrtg * (s.bcon[i + 1] * s.ucon[j] - s.bcon[j] * s.ucon[i + 1]);
  F[8] = s.sqrtg * s.qt * s.ucon[j];
  F[9] = s.sqrtg * s.dPt * s.ucon[j];
}

// Relaxation targets q~_0 and dP~_0 (Eqs. q0def, dP0def rescaled by Eqs. q,
// dP).  Coefficients come from state sE; the derivative inputs are
// dTh[mu] = d_mu Theta, du[mu][nu] = d_mu u_nu and divu = nabla_mu u^mu.
// a_mu = u^nu d_nu u_mu - Gamma^l_{nu mu} u^nu u_l, nabla_mu u_nu = d_mu u_nu -
// Gamma^l_{mu nu} u_l.
template <class C, class T>
static void relax_targets(const State<C>& sE, const Geom& g, const Params& p, const T dTh[4],
                          const T du[4][4], const T& divu, T& qt0, T& dPt0) {
  qt0 = T(0.0);
  dPt0 = T(0.0);
  if (p.cond) {
    T acc[4];
    for (int m = 0; m < 4; m++) {
      acc[m] = T(0.0);
      for (int n = 0; n < 4; n++) acc[m] = acc[m] + T(sE.ucon[n]) * du[n][m];
      for (int l = 0; l < 4; l++)
        for (int n = 0; n < 4; n++) acc[m] = acc[m] - T(g.Gam[l][n][m] * sE.ucon[n] * sE.ucov[l]);
    }
    T proj = T(0.0);
    for (int m = 0; m < 4; m++) proj = proj + T(sE.bhcon[m]) * (dTh[m] + T(sE.Theta) * acc[m]);
    T q0 = T(-sE.rho * sE.chi) * proj;
    qt0 = q0 * T(sqrt(sE.tauR / (sE.chi * sE.rho * sE.Theta * sE.Theta)));
  }
  if (p.visc) {
    T proj = T(0.0);
    for (int m = 0; m < 4; m++)
      for (int n = 0; n < 4; n++) {
        T nab = du[m][n];
        for (int l = 0; l < 4; l++) nab = nab - T(g.Gam[l][m][n] * sE.ucov[l]);
        proj = proj + T(sE.bhcon[m] * sE.bhcon[n]) * nab;
      }
    T dP0 = T(3.0 * sE.rho * sE.nu) * (proj - divu / 3.0);
    dPt0 = dP0 * T(sqrt(sE.tauR / (sE.nu * sE.rho * sE.Theta)));
  }
}

// ---------------------------------------------------------------- wave speeds
// Fluid-frame bound v_max^2 = cs~^2 + vA^2 - cs~^2 vA^2 with Eq. modcs and the
// corrections v_q^2 = (gamma-1) chi/tau_R, v_dP^2 = 4 nu/(3 tau_R) (Section 4.1),
// then the grid-frame speeds of waves moving at +-v_max in direction j: the
// roots c of (k.u)^2 = v^2 (k.k + (k.u)^2) with k_mu = (-c, e_j).
template <class T>
static void wave_speeds(const State<T>& s, const Geom& g, const Params& p, int j, T& cmin, T& cmax) {
  T vA2 = s.bsq / (s.rho + p.gamma * s.u + s.bsq);
  T vq2 = (p.gamma - 1.0) * s.chi / s.tauR;
  T vdp2 = 4.0 * s.nu / (3.0 * s.tauR);
  T cs2t = 0.5 * (s.cs2 + vq2 + sqrt(s.cs2 * s.cs2 + vq2 * vq2)) + vdp2;
  T v2 = cs2t + vA2 - cs2t * vA2;
  T ut = s.ucon[0], uj = s.ucon[j];
  T A = (1.0 - v2) * ut * ut - v2 * g.gcon[0][0];
  T B = -2.0 * ((1.0 - v2) * ut * uj - v2 * g.gcon[0][j]);
  T Cc = (1.0 - v2) * uj * uj - v2 * g.gcon[j][j];
  T disc = B * B - 4.0 * A * Cc;
  if (disc < 0.0) disc = T(0.0);
  T sq = sqrt(disc);
  T c1 = (-B + sq) / (2.0 * A), c2 = (-B - sq) / (2.0 * A);
  cmax = tmax(c1, c2);
  cmin = tmin(c1, c2);
}

// ---------------------------------------------------------------- grid access
struct Grid {
  Params p;
  long long idx(int i, int j, int k) const { return ((long long)k * p.n[1] + j) * p.n[0] + i; }
  // Map a possibly out-of-range index to an interior zone by the boundary
  // rule of each direction; 'flip' marks a reflection (component sign flip).
  int map1(int d, int i, bool& flip) const {
    int n = p.n[d];
    if (i >= 0 && i < n) return i;
    int side = (i < 0) ? 0 : 1;
    int bc = p.bc[d][side];
    if (bc == BC_PERIODIC) return ((i % n) + n) % n;
    if (bc == BC_OUTFLOW) return (i < 0) ? 0 : n - 1;
    // reflections: images repeat with period 2n, odd images are mirrored
    int m = ((i % (2 * n)) + 2 * n) % (2 * n);
    if (m >= n) { flip = !flip; return 2 * n - 1 - m; }
    return m;
  }
  // Primitive vector of the (possibly ghost) zone (i,j,k).
  void prim(const double* P, int i, int j, int k, double out[10]) const {
    bool f[3] = {false, false, false};
    int ii = map1(0, i, f[0]);
    int jj = (p.dim >= 2) ? map1(1, j, f[1]) : 0;
    int kk = (p.dim >= 3) ? map1(2, k, f[2]) : 0;
    long long z = idx(ii, jj, kk);
    for (int v = 0; v < 10; v++) out[v] = P[v * p.N + z];
    for (int d = 0; d < 3; d++)
      if (f[d]) { out[2 + d] = -out[2 + d]; out[5 + d] = -out[5 + d]; }
  }
  void center(int i, int j, int k, double X[3]) const {
    int ijk[3] = {i, j, k};
    for (int d = 0; d < 3; d++) X[d] = p.x0[d] + (ijk[d] + 0.5) * p.dx[d];
  }
};

// ---------------------------------------------------------------- reconstruction
// Generalized minmod slope (Section 2.4.1): theta = 1 is minmod, theta = 2 is MC.
template <class T> static T gminmod(double theta, T vm, T v0, T vp) {
  T a = theta * (v0 - vm), b = 0.5 * (vp - vm), c = theta * (vp - v0);
  if (a > 0.0 && b > 0.0 && c > 0.0) return tmin(a, tmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return tmax(a, tmax(b, c));
  return T(0.0);
}

// WENO5 (Jiang & Shu 1996): value at the right face of the middle zone of
// v[0..4] from the three 3-point candidates and their smoothness indicators.
template <class T> static T weno5_right(const T v[5]) {
  const double eps = 1e-6;
  T q0 = (2 * v[0] - 7 * v[1] + 11 * v[2]) / 6.0;
  T q1 = (-v[1] + 5 * v[2] + 2 * v[3]) / 6.0;
  T q2 = (2 * v[2] + 5 * v[3] - v[4]) / 6.0;
  T b0 = 13.0 / 12.0 * (v[0] - 2 * v[1] + v[2]) * (v[0] - 2 * v[1] + v[2]) +
         0.25 * (v[0] - 4 * v[1] + 3 * v[2]) * (v[0] - 4 * v[1] + 3 * v[2]);
  T b1 = 13.0 / 12.0 * (v[1] - 2 * v[2] + v[3]) * (v[1] - 2 * v[2] + v[3]) +
         0.25 * (v[1] - v[3]) * (v[1] - v[3]);
  T b2 = 13.0 / 12.0 * (v[2] - 2 * v[3] + v[4]) * (v[2] - 2 * v[3] + v[4]) +
         0.25 * (3 * v[2] - 4 * v[3] + v[4]) * (3 * v[2] - 4 * v[3] + v[4]);
  T a0 = 0.1 / ((eps + b0) * (eps + b0));
  T a1 = 0.6 / ((eps + b1) * (eps + b1));
  T a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Face states of the zone whose 7-point line (offsets -3..3) is s[]: the value
// at its left face (lo) and right face (hi).
// PPM (Colella & Woodward 1984) face values of the middle zone of v[0..4]:
// interface values a_{i+-1/2} = (a_i + a_{i+-1})/2 -+ (da_{i+-1} - da_i)/6
// from limited slopes da (generalized minmod, theta), then the monotonicity
// constraints: at a local extremum both faces take the zone value; an
// interpolating parabola that would overshoot has the far face moved to
// 3 a_i - 2 a_near.
template <class T> static void ppm_zone(double theta, const T v[5], T& lo, T& hi) {
  T d1 = gminmod(theta, v[0], v[1], v[2]);
  T d2 = gminmod(theta, v[1], v[2], v[3]);
  T d3 = gminmod(theta, v[2], v[3], v[4]);
  T aL = 0.5 * (v[1] + v[2]) - (d2 - d1) / 6.0;
  T aR = 0.5 * (v[2] + v[3]) - (d3 - d2) / 6.0;
  const T a = v[2];
  if (!((aR - a) * (a - aL) > 0.0)) {
    aL = a;
    aR = a;
  } else {
    T D = aR - aL;
    T m6 = 6.0 * (a - 0.5 * (aL + aR));
    if (D * m6 > D * D) aL = 3.0 * a - 2.0 * aR;
    else if (D * m6 < -(D * D)) aR = 3.0 * a - 2.0 * aL;
  }
  lo = aL;
  hi = aR;
}

template <class T> static void recon_zone(const Params& p, const T s[7], T& lo, T& hi) {
  if (p.recon == RECON_PPM) {
    T v[5] = {s[1], s[2], s[3], s[4], s[5]};
    ppm_zone(p.theta, v, lo, hi);
    return;
  }
  if (p.recon == RECON_WENO5) {
    T f[5] = {s[1], s[2], s[3], s[4], s[5]};
    T b[5] = {s[5], s[4], s[3], s[2], s[1]};
    hi = weno5_right(f);
    lo = weno5_right(b);
  } else {
    T sl = gminmod(p.theta, s[2], s[3], s[4]);
    hi = s[3] + 0.5 * sl;
    lo = s[3] - 0.5 * sl;
  }
}

// ---------------------------------------------------------------- the stage
struct Stage {
  Grid G;
  int lo[3], hi[3];       // face index ranges per direction (inclusive lo, exclusive hi)
  int ext[3];             // extended sizes n+2 (offset 1)
  std::vector<double> F[3];  // face fluxes F[d][v*NE + e], e = extended index of the zone right of the face
  long long NE;
  const char* zmask = nullptr;  // zones to solve (nullptr = all); only their stencils are computed
  long long eidx(int i, int j, int k) const {
    return ((long long)(k + 1) * ext[1] + (j + 1)) * ext[0] + (i + 1);
  }
};

// LLF flux at the face on the low side of zone (i,j,k) in direction d
// (Section 2.4.2): F = (F^+ + F^-)/2 - c_max/2 (U^+ - U^-); or HLLE.
static void face_flux(const Grid& G, const double* PE, int d, int i, int j, int k, double Fout[10]) {
  const Params& p = G.p;
  double L[10], R[10];
  int o[3] = {0, 0, 0};
  o[d] = 1;
  // line of primitives around the face: zones at offsets -4..3 along d
  double line[8][10];
  for (int t = -4; t <= 3; t++) G.prim(PE, i + t * o[0], j + t * o[1], k + t * o[2], line[t + 4]);
  for (int v = 0; v < 10; v++) {
    double sL[7], sR[7];
    for (int t = 0; t < 7; t++) { sL[t] = line[t][v]; sR[t] = line[t + 1][v]; }
    double lo, hi;
    recon_zone(p, sL, lo, hi);  // zone on the left of the face: use its right-face value
    L[v] = hi;
    recon_zone(p, sR, lo, hi);  // zone on the right: its left-face value
    R[v] = lo;
  }
  double X[3];
  G.center(i, j, k, X);
  X[d] -= 0.5 * p.dx[d];
  if (polar_face(p, X, d)) {
    for (int v = 0; v < 10; v++) Fout[v] = 0.0;
    return;
  }
  Geom g;
  geom_at(p, X, g);
  State<double> sl, sr;
  make_state(L, g, p, sl);
  make_state(R, g, p, sr);
  double FL[10], FR[10], UL[10], UR[10];
  flux(sl, d + 1, FL);
  flux(sr, d + 1, FR);
  conserved(sl, UL);
  conserved(sr, UR);
  double cminL, cmaxL, cminR, cmaxR;
  wave_speeds(sl, g, p, d + 1, cminL, cmaxL);
  wave_speeds(sr, g, p, d + 1, cminR, cmaxR);
  if (p.riemann == 1) {
    // HLLE (Section 2.4.2): right- and left-going bounds cR = max(c, 0),
    // cL = max(-c, 0) over both sides; L is the left state P^-, R the right P^+
    const double cR = std::max(std::max(cmaxL, cmaxR), 0.0);
    const double cL = std::max(-std::min(cminL, cminR), 0.0);
    for (int v = 0; v < 10; v++) Fout[v] = (cR * FL[v] + cL * FR[v] - cR * cL * (UR[v] - UL[v])) / (cL + cR);
    return;
  }
  double cm = std::max(std::max(std::fabs(cminL), std::fabs(cmaxL)), std::max(std::fabs(cminR), std::fabs(cmaxR)));
  for (int v = 0; v < 10; v++) Fout[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * cm * (UR[v] - UL[v]);
}

static void compute_fluxes(Stage& S, const double* PE) {
  const Params& p = S.G.p;
  for (int d = 0; d < 3; d++) S.ext[d] = p.n[d] + 2;
  S.NE = (long long)S.ext[0] * S.ext[1] * S.ext[2];
  // Faces a zone needs: its own low and high faces in each active direction,
  // and those of its transverse neighbours (the flux-CT corner averages).
  std::vector<char> fm;
  if (S.zmask) {
    fm.assign(S.NE, 0);
    int r[3];
    for (int e = 0; e < 3; e++) r[e] = (e < p.dim) ? 1 : 0;
    for (int k = 0; k < p.n[2]; k++)
      for (int j = 0; j < p.n[1]; j++)
        for (int i = 0; i < p.n[0]; i++) {
          if (!S.zmask[S.G.idx(i, j, k)]) continue;
          // only indices inside the face arrays' extent -1..n (a zone on the
          // high boundary would otherwise mark one past it)
          for (int c = -r[2]; c <= r[2] + (p.dim >= 3); c++)
            for (int b = -r[1]; b <= r[1] + (p.dim >= 2); b++)
              for (int a = -r[0]; a <= r[0] + 1; a++) {
                const int ii = i + a, jj = j + b, kk = k + c;
                if (ii > p.n[0] || (p.dim >= 2 && jj > p.n[1]) || (p.dim >= 3 && kk > p.n[2])) continue;
                fm[S.eidx(ii, jj, kk)] = 1;
              }
        }
  }
  // Faces in direction d: 0..n_d along d; -1..n across it (flux-CT), in active dims.
  for (int d = 0; d < p.dim; d++) {
    S.F[d].assign(10 * S.NE, 0.0);
    int lo[3], hi[3];
    for (int e = 0; e < 3; e++) {
      if (e >= p.dim) { lo[e] = 0; hi[e] = 1; continue; }
      if (e == d) { lo[e] = 0; hi[e] = p.n[e] + 1; }
      else { lo[e] = -1; hi[e] = p.n[e] + 1; }
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = lo[2]; k < hi[2]; k++)
      for (int j = lo[1]; j < hi[1]; j++)
        for (int i = lo[0]; i < hi[0]; i++) {
          long long e = S.eidx(i, j, k);
          if (S.zmask && !fm[e]) continue;
          double Fv[10];
          face_flux(S.G, PE, d, i, j, k, Fv);
          for (int v = 0; v < 10; v++) S.F[d][v * S.NE + e] = Fv[v];
        }
  }
}

// Flux-CT (Section 4.2, Toth 2000): for each pair of active directions
// (a, b), the edge value E_ab is the average of the four face estimates of
// F^a[B^b] = -F^b[B^a]; the face fluxes of B are then replaced by averages of
// two edge values, and F^a[B^a] = 0.
static void flux_ct(Stage& S) {
  const Params& p = S.G.p;
  if (p.dim < 2) {
    for (long long e = 0; e < S.NE; e++) S.F[0][5 * S.NE + e] = 0.0;
    return;
  }
  const long long NE = S.NE;
  std::vector<double> newF[3];
  for (int d = 0; d < p.dim; d++) newF[d] = S.F[d];
  for (int a = 0; a < p.dim; a++)
    for (int b = a + 1; b < p.dim; b++) {
      // Edge values at the (a,b) corner on the low side of zone (i,j,k), for zones -? .. n
      std::vector<double> E(NE, 0.0);
      int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
      for (int e = 0; e < p.dim; e++) { lo[e] = 0; hi[e] = p.n[e] + 1; }
      for (int e = 0; e < p.dim; e++) if (e != a && e != b) { lo[e] = 0; hi[e] = p.n[e]; }
      for (int k = lo[2]; k < hi[2]; k++)
        for (int j = lo[1]; j < hi[1]; j++)
          for (int i = lo[0]; i < hi[0]; i++) {
            int ijk[3] = {i, j, k};
            int m_b[3] = {i, j, k}; m_b[b] -= 1;  // shifted along b
            int m_a[3] = {i, j, k}; m_a[a] -= 1;  // shifted along a
            double fab0 = S.F[a][(5 + b) * NE + S.eidx(ijk[0], ijk[1], ijk[2])];
            double fab1 = S.F[a][(5 + b) * NE + S.eidx(m_b[0], m_b[1], m_b[2])];
            double fba0 = S.F[b][(5 + a) * NE + S.eidx(ijk[0], ijk[1], ijk[2])];
            double fba1 = S.F[b][(5 + a) * NE + S.eidx(m_a[0], m_a[1], m_a[2])];
            E[S.eidx(i, j, k)] = 0.25 * (fab0 + fab1 - fba0 - fba1);
          }
      // replace face fluxes of interior-needed faces
      for (int k = 0; k < (p.dim >= 3 ? p.n[2] + 1 : 1); k++)
        for (int j = 0; j < (p.dim >= 2 ? p.n[1] + 1 : 1); j++)
          for (int i = 0; i < p.n[0] + 1; i++) {
            int ijk[3] = {i, j, k};
            int pb[3] = {i, j, k}; pb[b] += 1;
            int pa[3] = {i, j, k}; pa[a] += 1;
            bool in_a = true, in_b = true;  // face a at (i,j,k) valid if transverse indices < n
            for (int e = 0; e < p.dim; e++) {
              if (e != a && ijk[e] >= p.n[e]) in_a = false;
              if (e != b && ijk[e] >= p.n[e]) in_b = false;
            }
            if (in_a)
              newF[a][(5 + b) * NE + S.eidx(i, j, k)] =
                  0.5 * (E[S.eidx(i, j, k)] + E[S.eidx(pb[0], pb[1], pb[2])]);
            if (in_b)
              newF[b][(5 + a) * NE + S.eidx(i, j, k)] =
                  -0.5 * (E[S.eidx(i, j, k)] + E[S.eidx(pa[0], pa[1], pa[2])]);
          }
    }
  for (int d = 0; d < p.dim; d++) {
    for (long long e = 0; e < NE; e++) newF[d][(5 + d) * NE + e] = 0.0;
    S.F[d].swap(newF[d]);
  }
}

// ---------------------------------------------------------------- per-zone residual
// Everything of the stage residual that does not depend on the unknown P
// (the P_n-only terms the paper precomputes outside the residual assembly, Section 7.1).
struct ZoneConst {
  Geom g;
  State<double> sE;       // state at P^E (coefficients)
  double Un[10];          // U(P_n)
  double divF[10];        // sum_j (F_{j,+} - F_{j,-})/dX^j at P^E
  double Sgeo[10];        // sqrt(-g) T^k_l Gamma^l_{nu k} at P^E (rows 1..4)
  double dTh_sp[4];       // slope-limited d_i Theta at P^E (index 0 unused)
  double du_sp[4][4];     // slope-limited d_i u_nu at P^E (row 0 unused)
  double divu_sp;         // (1/sqrt(-g)) d_i (sqrt(-g) u^i) at P^E
  double Th_n, ut_n, ucov_n[4], qt_n, dPt_n;  // P_n quantities used by the time quotients
  double scale[10];       // dt_s / (|U_i(P_n)| + |U_0(P_n)|)
  double dts;
};

// Stage residual R(P) of Eq. half_step_residual (and its full-step analogue),
// scaled row by row: r_i = scale_i * R_i.
template <class T>
static void residual(const ZoneConst& z, const Params& p, const T* P, T* r) {
  State<T> s;
  make_state(P, z.g, p, s);
  T U[10];
  conserved(s, U);
  T R[10];
  for (int a = 0; a < 10; a++) R[a] = (U[a] - z.Un[a]) / z.dts + z.divF[a] - z.Sgeo[a];
  // time derivatives as difference quotients; spatial ones frozen at P^E
  T dTh[4], du[4][4];
  dTh[0] = (s.Theta - z.Th_n) / z.dts;
  for (int i = 1; i < 4; i++) dTh[i] = T(z.dTh_sp[i]);
  for (int n = 0; n < 4; n++) du[0][n] = (s.ucov[n] - z.ucov_n[n]) / z.dts;
  for (int i = 1; i < 4; i++)
    for (int n = 0; n < 4; n++) du[i][n] = T(z.du_sp[i][n]);
  T divu = (s.ucon[0] - z.ut_n) / z.dts + z.divu_sp;
  T qt0, dPt0;
  relax_targets(z.sE, z.g, p, dTh, du, divu, qt0, dPt0);
  const double tau = z.sE.tauR, sg = z.g.sqrtg;
  T Sq = -((s.qt + z.qt_n) / 2.0 - qt0) / tau;
  T Sd = -((s.dPt + z.dPt_n) / 2.0 - dPt0) / tau;
  if (p.ho) {
    Sq = Sq + (z.sE.qt / 2.0) * divu;
    Sd = Sd + (z.sE.dPt / 2.0) * divu;
  }
  R[8] = R[8] - sg * Sq;
  R[9] = R[9] - sg * Sd;
  for (int a = 0; a < 10; a++) r[a] = R[a] * z.scale[a];
}

// Partial-pivot LU solve of J x = b (10x10, row-major J, overwritten).
// Returns false on an exactly zero pivot.  Pivot: largest |a_ik|, lowest row on ties.
template <int N, class T> static bool lu_solve_n(T J[N][N], T b[N], T x[N]) {
  for (int k = 0; k < N; k++) {
    int piv = k;
    double best = std::fabs(re(J[k][k]));
    for (int i = k + 1; i < N; i++)
      if (std::fabs(re(J[i][k])) > best) { best = std::fabs(re(J[i][k])); piv = i; }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int c = 0; c < N; c++) std::swap(J[k][c], J[piv][c]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < N; i++) {
      T l = J[i][k] / J[k][k];
      for (int c = k + 1; c < N; c++) J[i][c] = J[i][c] - l * J[k][c];
      b[i] = b[i] - l * b[k];
    }
  }
  for (int i = N - 1; i >= 0; i--) {
    T acc = b[i];
    for (int c = i + 1; c < N; c++) acc = acc - J[i][c] * x[c];
    x[i] = acc / J[i][i];
  }
  return true;
}
template <class T> static bool lu_solve(T J[10][10], T b[10], T x[10]) { return lu_solve_n<10>(J, b, x); }

static double maxabs(const double* r) {
  double m = 0;
  for (int a = 0; a < 10; a++) m = std::max(m, std::fabs(r[a]));
  return m;
}
static double sumsq(const double* r) {
  double f = 0;
  for (int a = 0; a < 10; a++) f += r[a] * r[a];
  return f;
}

struct NewtonOut { int iters, status, evals; };

// Perturbed component of the FD Jacobian (Section 3.1): (1 + eps) P_j, or
// P_j + eps where |P_j| < 5 eps (small(), read as an absolute step so that the
// divisor never vanishes).  The absolute floor is for components that pass
// through zero; rho and u are positive, and their step stays relative at
// every magnitude (the internal energy of a cold atmosphere, 1e-11, would
// otherwise move by 1e4 times itself).
static double fd_perturbed(double x, double eps, bool positive) {
  if (positive && x > 0.0) return (1.0 + eps) * x;
  return (std::fabs(x) < 5.0 * eps) ? x + eps : (1.0 + eps) * x;
}

// Newton iteration of Section 3 with the FD Jacobian of Section 3.1 and the
// quadratic backtracking line search of Section 3.2.
static NewtonOut newton(const ZoneConst& z, const Params& p, double P[10]) {
  NewtonOut o = {0, 0, 0};
  double r[10];
  residual(z, p, P, r);
  o.evals++;
  double f = sumsq(r);
  const double eps = p.eps, ebt = 1e-4;
  int k = 0;
  for (;;) {
    if (!std::isfinite(f)) { o.status |= ST_NONFINITE; break; }
    if (maxabs(r) <= p.tol) break;
    if (k >= p.kmax) { o.status |= ST_MAXIT; break; }
    // Jacobian J_ij = (r_i(P_eps) - r_i(P)) / (P_eps,j - P_j)
    double J[10][10];
    for (int j = 0; j < 10; j++) {
      double Pe[10];
      std::memcpy(Pe, P, sizeof(Pe));
      Pe[j] = fd_perturbed(P[j], eps, j <= 1);
      double re_[10];
      residual(z, p, Pe, re_);
      o.evals++;
      double hstep = Pe[j] - P[j];
      for (int i = 0; i < 10; i++) J[i][j] = (re_[i] - r[i]) / hstep;
    }
    double rhs[10], dP[10];
    for (int i = 0; i < 10; i++) rhs[i] = -r[i];
    if (!lu_solve(J, rhs, dP)) { o.status |= ST_SINGULAR; break; }
    // line search
    double lam = 1.0, Pt[10], rt[10], ft = 0;
    for (int t = 0;; t++) {
      for (int a = 0; a < 10; a++) Pt[a] = P[a] + lam * dP[a];
      residual(z, p, Pt, rt);
      o.evals++;
      ft = sumsq(rt);
      bool fin = std::isfinite(ft);
      double lim = 1.0 - ebt * lam;
      if (fin && ft < f * lim * lim) break;
      if (t >= p.lsmax) { o.status |= ST_LSSTALL; break; }
      // the minimiser of the quadratic model; where it is not a positive
      // finite number (a non-finite trial, or a denominator that overflowed
      // to leave 0 and then 0/0), lambda is halved instead
      const double ln = fin ? f * lam * lam / (ft + (2.0 * lam - 1.0) * f) : 0.0;
      lam = (ln > 0.0 && std::isfinite(ln)) ? ln : 0.5 * lam;
    }
    std::memcpy(P, Pt, sizeof(Pt));
    std::memcpy(r, rt, sizeof(rt));
    f = ft;
    k++;
  }
  o.iters = k;
  if (!(P[0] > 0.0) || !(P[1] > 0.0)) o.status |= ST_INADMISSIBLE;
  return o;
}

// Build the per-zone constants of one stage from P_n, P^E and the fluxes.
static void zone_const(const Stage& S, const double* Pn, const double* PE, double dts, int i, int j, int k,
                       ZoneConst& z) {
  const Grid& G = S.G;
  const Params& p = G.p;
  double X[3];
  G.center(i, j, k, X);
  geom_at(p, X, z.g);
  z.dts = dts;
  double PnZ[10], PEZ[10];
  G.prim(Pn, i, j, k, PnZ);
  G.prim(PE, i, j, k, PEZ);
  make_state(PEZ, z.g, p, z.sE);
  State<double> sn;
  make_state(PnZ, z.g, p, sn);
  conserved(sn, z.Un);
  z.Th_n = sn.Theta; z.ut_n = sn.ucon[0];
  for (int n = 0; n < 4; n++) z.ucov_n[n] = sn.ucov[n];
  z.qt_n = sn.qt; z.dPt_n = sn.dPt;
  for (int a = 0; a < 10; a++) z.scale[a] = dts / (std::fabs(z.Un[a]) + std::fabs(z.Un[0]));
  // flux divergence
  for (int a = 0; a < 10; a++) z.divF[a] = 0.0;
  for (int d = 0; d < p.dim; d++) {
    int ip[3] = {i, j, k};
    ip[d] += 1;
    for (int a = 0; a < 10; a++)
      z.divF[a] += (S.F[d][a * S.NE + S.eidx(ip[0], ip[1], ip[2])] - S.F[d][a * S.NE + S.eidx(i, j, k)]) / p.dx[d];
  }
  // geometric source at P^E (Eq. divT_explicit)
  for (int a = 0; a < 10; a++) z.Sgeo[a] = 0.0;
  {
    double Tmn[4][4];
    stress(z.sE, Tmn);
    for (int n = 0; n < 4; n++) {
      double acc = 0;
      for (int kk = 0; kk < 4; kk++)
        for (int l = 0; l < 4; l++) acc += Tmn[kk][l] * z.g.Gam[l][n][kk];
      z.Sgeo[1 + n] = z.g.sqrtg * acc;
    }
  }
  // slope-limited spatial derivatives at P^E (Section 2.3)
  for (int n = 0; n < 4; n++) { z.dTh_sp[n] = 0; for (int m = 0; m < 4; m++) z.du_sp[n][m] = 0; }
  z.divu_sp = 0;
  for (int d = 0; d < p.dim; d++) {
    double th[3], uc[3][4], gu[3];
    for (int t = -1; t <= 1; t++) {
      int q3[3] = {i, j, k};
      q3[d] += t;
      double Pq[10], Xq[3];
      G.prim(PE, q3[0], q3[1], q3[2], Pq);
      G.center(q3[0], q3[1], q3[2], Xq);
      Geom gq;
      geom_at(p, Xq, gq);
      State<double> sq;
      make_state(Pq, gq, p, sq);
      th[t + 1] = sq.Theta;
      for (int m = 0; m < 4; m++) uc[t + 1][m] = sq.ucov[m];
      gu[t + 1] = gq.sqrtg * sq.ucon[d + 1];
    }
    z.dTh_sp[d + 1] = gminmod(p.theta, th[0], th[1], th[2]) / p.dx[d];
    for (int m = 0; m < 4; m++) z.du_sp[d + 1][m] = gminmod(p.theta, uc[0][m], uc[1][m], uc[2][m]) / p.dx[d];
    z.divu_sp += gminmod(p.theta, gu[0], gu[1], gu[2]) / p.dx[d] / z.g.sqrtg;
  }
}

// Post-stage limits for the accreting torus (the paper describes floors and an
// anisotropy limiter without values; a zone whose Newton iteration ended
// with a non-zero status first reverts to its start, see oracle_stage_masked): rho >= 1e-5 r^{-3/2}, u >= 1e-7
// r^{-5/2} (r = 1 in Minkowski space), then the pressure anisotropy clamped
// to the firehose and mirror thresholds, -b^2 <= dP <= b^2/2.
static void apply_floors(const Params& p, const double X[3], const Geom& g, double P[10]) {
  const double r = (p.metric == METRIC_MKS_KERR) ? std::exp(X[0]) : 1.0;
  P[0] = std::max(P[0], 1e-5 / (r * std::sqrt(r)));
  P[1] = std::max(P[1], 1e-7 / (r * r * std::sqrt(r)));
  if (!p.visc) return;
  State<double> s;
  make_state(P, g, p, s);
  const double f = std::sqrt(s.nu * s.rho * s.Theta / g.tauR);  // dP = f dP~
  if (!(f > 0.0)) return;
  const double lo = -s.bsq, hi = 0.5 * s.bsq;
  if (s.dP > hi) P[9] = hi / f;
  else if (s.dP < lo) P[9] = lo / f;
}

static void set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

}  // namespace orc

using namespace orc;

extern "C" {

int oracle_version() { return 1; }

int oracle_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// One stage (Section 2.3): solve R(P) = 0 for every zone, with P^E the explicit
// state and P_n the start of the step.  guess may be NULL (then P_n).  The
// magnetic components of the guess are always the explicit flux-CT update.
// Writes P_out (SoA [10][N]), iters and status per zone.
// One stage solved on the zones with mask[z] != 0 (mask NULL = every zone);
// P_out, iters and status are written only there.
int oracle_stage_masked(const int* ip, const double* dp, const double* Pn, const double* PE, double dts,
                        const double* guess, const char* mask, double* Pout, int* iters, int* status,
                        long long* evals_out) {
  Stage S;
  S.G.p = read_params(ip, dp);
  S.zmask = mask;
  set_threads(ip[I_NTHREADS]);
  const Params& p = S.G.p;
  compute_fluxes(S, PE);
  flux_ct(S);
  long long evals = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 64) reduction(+ : evals)
  for (int k = 0; k < p.n[2]; k++)
    for (int j = 0; j < p.n[1]; j++)
      for (int i = 0; i < p.n[0]; i++) {
        long long zi = S.G.idx(i, j, k);
        if (mask && !mask[zi]) continue;
        ZoneConst z;
        zone_const(S, Pn, PE, dts, i, j, k, z);
        double P[10];
        const double* src = guess ? guess : Pn;
        for (int v = 0; v < 10; v++) P[v] = src[v * p.N + zi];
        for (int c = 0; c < 3; c++)
          P[5 + c] = (z.Un[5 + c] - dts * z.divF[5 + c]) / z.g.sqrtg;
        NewtonOut o = newton(z, p, P);
        if (p.floors) {
          // a zone left without an admissible root keeps its start (P_n with
          // the flux-CT field); then the floors
          if (o.status) {
            for (int v = 0; v < 10; v++) P[v] = Pn[v * p.N + zi];
            for (int c = 0; c < 3; c++) P[5 + c] = (z.Un[5 + c] - dts * z.divF[5 + c]) / z.g.sqrtg;
          }
          double X[3];
          S.G.center(i, j, k, X);
          apply_floors(p, X, z.g, P);
        }
        for (int v = 0; v < 10; v++) Pout[v * p.N + zi] = P[v];
        if (iters) iters[zi] = o.iters;
        if (status) status[zi] = o.status;
        evals += o.evals;
      }
  if (evals_out) *evals_out = evals;
  return 0;
}

// One stage (Section 2.3): solve R(P) = 0 for every zone, with P^E the explicit
// state and P_n the start of the step.  guess may be NULL (then P_n).  The
// magnetic components of the guess are always the explicit flux-CT update.
// Writes P_out (SoA [10][N]), iters and status per zone.
int oracle_stage(const int* ip, const double* dp, const double* Pn, const double* PE, double dts,
                 const double* guess, double* Pout, int* iters, int* status, long long* evals_out) {
  return oracle_stage_masked(ip, dp, Pn, PE, dts, guess, nullptr, Pout, iters, status, evals_out);
}

// One full step evaluated only at the listed zones: the half step is solved on
// the zones within 4 zones of a listed one (all its full-step stencil needs),
// then the full step at the listed zones.  Pout is [10][nz], iters/status [nz].
int oracle_step_sampled(const int* ip, const double* dp, const double* Pn, double dt, const long long* zones,
                        int nz, double* Pout, int* iters, int* status, long long* evals) {
  Params p = read_params(ip, dp);
  Grid G;
  G.p = p;
  std::vector<char> m1(p.N, 0), m2(p.N, 0);
  const int R = 4;
  for (int s = 0; s < nz; s++) {
    long long z = zones[s];
    int i = (int)(z % p.n[0]), j = (int)((z / p.n[0]) % p.n[1]), k = (int)(z / ((long long)p.n[0] * p.n[1]));
    m2[z] = 1;
    int rk = (p.dim >= 3) ? R : 0, rj = (p.dim >= 2) ? R : 0;
    for (int c = -rk; c <= rk; c++)
      for (int b = -rj; b <= rj; b++)
        for (int a = -R; a <= R; a++) {
          bool f = false;
          int ii = G.map1(0, i + a, f);
          int jj = (p.dim >= 2) ? G.map1(1, j + b, f) : 0;
          int kk = (p.dim >= 3) ? G.map1(2, k + c, f) : 0;
          m1[G.idx(ii, jj, kk)] = 1;
        }
  }
  std::vector<double> Ph(10 * p.N, 0.0), Pf(10 * p.N, 0.0);
  std::vector<int> it1(p.N, 0), st1(p.N, 0), it2(p.N, 0), st2(p.N, 0);
  long long e1 = 0, e2 = 0;
  // zones outside the half-step mask keep P_n (they are never read)
  std::memcpy(Ph.data(), Pn, sizeof(double) * 10 * p.N);
  oracle_stage_masked(ip, dp, Pn, Pn, 0.5 * dt, nullptr, m1.data(), Ph.data(), it1.data(), st1.data(), &e1);
  oracle_stage_masked(ip, dp, Pn, Ph.data(), dt, nullptr, m2.data(), Pf.data(), it2.data(), st2.data(), &e2);
  for (int s = 0; s < nz; s++) {
    long long z = zones[s];
    for (int v = 0; v < 10; v++) Pout[v * nz + s] = Pf[v * p.N + z];
    if (iters) iters[s] = it1[z] + it2[z];
    if (status) status[s] = st1[z] | st2[z];
  }
  if (evals) *evals = e1 + e2;
  return 0;
}

// Scaled (scaled != 0) or raw residual of a stage at the state Pk, per zone.
int oracle_residual(const int* ip, const double* dp, const double* Pn, const double* PE, double dts,
                    const double* Pk, int scaled, double* Rout) {
  Stage S;
  S.G.p = read_params(ip, dp);
  set_threads(ip[I_NTHREADS]);
  const Params& p = S.G.p;
  compute_fluxes(S, PE);
  flux_ct(S);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < p.n[2]; k++)
    for (int j = 0; j < p.n[1]; j++)
      for (int i = 0; i < p.n[0]; i++) {
        ZoneConst z;
        zone_const(S, Pn, PE, dts, i, j, k, z);
        long long zi = S.G.idx(i, j, k);
        double P[10], r[10];
        for (int v = 0; v < 10; v++) P[v] = Pk[v * p.N + zi];
        residual(z, p, P, r);
        for (int v = 0; v < 10; v++) Rout[v * p.N + zi] = scaled ? r[v] : r[v] / z.scale[v];
      }
  return 0;
}

// Face fluxes after flux-CT, for the faces on the low side of every zone:
// Fout[d][v][N] for the active directions d.
int oracle_fluxes(const int* ip, const double* dp, const double* PE, double* Fout) {
  Stage S;
  S.G.p = read_params(ip, dp);
  set_threads(ip[I_NTHREADS]);
  const Params& p = S.G.p;
  compute_fluxes(S, PE);
  flux_ct(S);
  for (int d = 0; d < p.dim; d++)
    for (int k = 0; k < p.n[2]; k++)
      for (int j = 0; j < p.n[1]; j++)
        for (int i = 0; i < p.n[0]; i++)
          for (int v = 0; v < 10; v++)
            Fout[((long long)d * 10 + v) * p.N + S.G.idx(i, j, k)] = S.F[d][v * S.NE + S.eidx(i, j, k)];
  return 0;
}

// One full step (Section 2.3): half step P_n -> P_{n+1/2} with P^E = P_n and
// dt/2, then the full step P_n -> P_{n+1} with P^E = P_{n+1/2} and dt.
int oracle_step(const int* ip, const double* dp, const double* Pn, double dt, double* Pout, int* iters,
                int* status, long long* evals) {
  Params p = read_params(ip, dp);
  std::vector<double> Ph(10 * p.N);
  std::vector<int> it1(p.N), st1(p.N);
  long long e1 = 0, e2 = 0;
  oracle_stage(ip, dp, Pn, Pn, 0.5 * dt, nullptr, Ph.data(), it1.data(), st1.data(), &e1);
  oracle_stage(ip, dp, Pn, Ph.data(), dt, nullptr, Pout, iters, status, &e2);
  if (iters)
    for (long long z = 0; z < p.N; z++) iters[z] += it1[z];
  if (status)
    for (long long z = 0; z < p.N; z++) status[z] |= st1[z];
  if (evals) *evals = e1 + e2;
  return 0;
}

// Geometry at the point X (for the tests): g_{mu nu}, g^{mu nu} (row-major
// 4x4), sqrt(-g), alpha, Gamma^l_{mu nu} ([l][mu][nu]) and tau_R.
int oracle_geometry(const int* ip, const double* dp, const double* X, double* gcov, double* gcon, double* sqrtg,
                    double* alpha, double* Gam, double* tauR) {
  Params p = read_params(ip, dp);
  Geom g;
  geom_at(p, X, g);
  std::memcpy(gcov, g.gcov, sizeof(g.gcov));
  std::memcpy(gcon, g.gcon, sizeof(g.gcon));
  *sqrtg = g.sqrtg;
  *alpha = g.alpha;
  std::memcpy(Gam, g.Gam, sizeof(g.Gam));
  *tauR = g.tauR;
  return 0;
}

// Post-stage floors at the zone centre X (for the tests): P updated in place.
int oracle_floors(const int* ip, const double* dp, const double* X, double* P) {
  Params p = read_params(ip, dp);
  Geom g;
  geom_at(p, X, g);
  apply_floors(p, X, g, P);
  return 0;
}

// Pointwise physics for the tests: conserved variables and fluxes at one
// primitive vector in Minkowski space (metric = 0).
int oracle_point(const int* ip, const double* dp, const double* P, double* U, double* F1, double* F2,
                 double* F3, double* cspeeds) {
  Params p = read_params(ip, dp);
  Geom g;
  double X[3] = {0, 0, 0};
  geom_at(p, X, g);
  State<double> s;
  make_state(P, g, p, s);
  conserved(s, U);
  double* Fs[3] = {F1, F2, F3};
  for (int j = 0; j < 3; j++) {
    if (Fs[j]) flux(s, j + 1, Fs[j]);
    if (cspeeds) wave_speeds(s, g, p, j + 1, cspeeds[2 * j], cspeeds[2 * j + 1]);
  }
  return 0;
}

// Continuous source S(P, d_mu P) of the EMHD system at a point (Eqs.
// q_evol_eqn_rescaled, dP_evol_eqn_rescaled and the geometric source of Eq.
// divT_explicit) with all coefficients at P, complex-valued so the tests can
// take complex-step derivatives.  dP is [4][10] (mu, variable).
static void source_cont(const cplx* P, const cplx dPd[4][10], const Geom& g, const Params& p, cplx S[10]) {
  State<cplx> s;
  make_state(P, g, p, s);
  cplx dTh[4], du[4][4], divu(0.0);
  for (int m = 0; m < 4; m++) {
    Dual<cplx> Pd[10];
    for (int a = 0; a < 10; a++) Pd[a] = Dual<cplx>(P[a], dPd[m][a]);
    State<Dual<cplx>> sd;
    make_state(Pd, g, p, sd);
    dTh[m] = sd.Theta.d;
    for (int n = 0; n < 4; n++) du[m][n] = sd.ucov[n].d;
    // nabla_mu u^mu = (1/sqrt(-g)) d_mu (sqrt(-g) u^mu); sqrt(-g) is constant here
    divu += sd.ucon[m].d;
  }
  cplx qt0, dPt0;
  relax_targets(s, g, p, dTh, du, divu, qt0, dPt0);
  for (int a = 0; a < 10; a++) S[a] = 0.0;
  cplx Tmn[4][4];
  stress(s, Tmn);
  for (int n = 0; n < 4; n++) {
    cplx acc = 0;
    for (int kk = 0; kk < 4; kk++)
      for (int l = 0; l < 4; l++) acc += Tmn[kk][l] * g.Gam[l][n][kk];
    S[1 + n] = g.sqrtg * acc;
  }
  cplx Sq = -(s.qt - qt0) / s.tauR, Sd = -(s.dPt - dPt0) / s.tauR;
  if (p.ho) { Sq += s.qt / 2.0 * divu; Sd += s.dPt / 2.0 * divu; }
  S[8] = g.sqrtg * Sq;
  S[9] = g.sqrtg * Sd;
}

// Linearisation about a uniform state P0 (Minkowski) by complex-step
// differentiation of U, F^j and the continuous source: writes MU = dU/dP,
// A[j] = dF^j/dP (j = 1..3), SP = dS/dP, SD[mu] = dS/d(d_mu P), each 10x10
// row-major (row = equation, column = variable).
int oracle_linearize(const int* ip, const double* dp, const double* P0, double* MU, double* A, double* SP,
                     double* SD) {
  Params p = read_params(ip, dp);
  Geom g;
  double X[3] = {0, 0, 0};
  geom_at(p, X, g);
  const double h = 1e-30;
  for (int c = 0; c < 10; c++) {
    cplx P[10];
    for (int a = 0; a < 10; a++) P[a] = P0[a];
    P[c] += cplx(0.0, h);
    State<cplx> s;
    make_state(P, g, p, s);
    cplx U[10];
    conserved(s, U);
    for (int r = 0; r < 10; r++) MU[r * 10 + c] = U[r].imag() / h;
    for (int j = 0; j < 3; j++) {
      cplx F[10];
      flux(s, j + 1, F);
      for (int r = 0; r < 10; r++) A[j * 100 + r * 10 + c] = F[r].imag() / h;
    }
    cplx zero[4][10];
    for (int m = 0; m < 4; m++) for (int a = 0; a < 10; a++) zero[m][a] = 0.0;
    cplx S[10];
    source_cont(P, zero, g, p, S);
    for (int r = 0; r < 10; r++) SP[r * 10 + c] = S[r].imag() / h;
    for (int m = 0; m < 4; m++) {
      cplx Pr[10], dPd[4][10];
      for (int a = 0; a < 10; a++) Pr[a] = P0[a];
      for (int mm = 0; mm < 4; mm++) for (int a = 0; a < 10; a++) dPd[mm][a] = 0.0;
      dPd[m][c] = cplx(0.0, h);
      source_cont(Pr, dPd, g, p, S);
      for (int r = 0; r < 10; r++) SD[m * 100 + r * 10 + c] = S[r].imag() / h;
    }
  }
  return 0;
}

// Single-zone helpers for the Newton tests: a zone with given constants.
// zc layout: Un[10], divF[10], Sgeo[10], dTh_sp[4], du_sp[16], divu_sp, Th_n,
// ut_n, ucov_n[4], qt_n, dPt_n, scale[10], dts, PE[10]  (80 doubles);
// Minkowski geometry.
static void unpack_zone(const Params& p, const double* zc, ZoneConst& z) {
  geom_minkowski(z.g, p.tauR);
  int o = 0;
  for (int a = 0; a < 10; a++) z.Un[a] = zc[o++];
  for (int a = 0; a < 10; a++) z.divF[a] = zc[o++];
  for (int a = 0; a < 10; a++) z.Sgeo[a] = zc[o++];
  for (int a = 0; a < 4; a++) z.dTh_sp[a] = zc[o++];
  for (int a = 0; a < 4; a++) for (int b = 0; b < 4; b++) z.du_sp[a][b] = zc[o++];
  z.divu_sp = zc[o++];
  z.Th_n = zc[o++]; z.ut_n = zc[o++];
  for (int a = 0; a < 4; a++) z.ucov_n[a] = zc[o++];
  z.qt_n = zc[o++]; z.dPt_n = zc[o++];
  for (int a = 0; a < 10; a++) z.scale[a] = zc[o++];
  z.dts = zc[o++];
  double PE[10];
  for (int a = 0; a < 10; a++) PE[a] = zc[o++];
  make_state(PE, z.g, p, z.sE);
}

int oracle_zone_residual(const int* ip, const double* dp, const double* zc, const double* P, double* r) {
  Params p = read_params(ip, dp);
  ZoneConst z;
  unpack_zone(p, zc, z);
  residual(z, p, P, r);
  return 0;
}

// Complex-step Jacobian of the scaled zone residual (exact to rounding).
int oracle_zone_jacobian_cs(const int* ip, const double* dp, const double* zc, const double* P, double* J) {
  Params p = read_params(ip, dp);
  ZoneConst z;
  unpack_zone(p, zc, z);
  const double h = 1e-30;
  for (int c = 0; c < 10; c++) {
    cplx Pc[10], rc[10];
    for (int a = 0; a < 10; a++) Pc[a] = P[a];
    Pc[c] += cplx(0.0, h);
    residual(z, p, Pc, rc);
    for (int r = 0; r < 10; r++) J[r * 10 + c] = rc[r].imag() / h;
  }
  return 0;
}

// FD Jacobian of Section 3.1 for the same zone, as the Newton loop builds it.
int oracle_zone_jacobian_fd(const int* ip, const double* dp, const double* zc, const double* P, double* J) {
  Params p = read_params(ip, dp);
  ZoneConst z;
  unpack_zone(p, zc, z);
  double r[10];
  residual(z, p, P, r);
  for (int j = 0; j < 10; j++) {
    double Pe[10], re_[10];
    std::memcpy(Pe, P, sizeof(Pe));
    Pe[j] = fd_perturbed(P[j], p.eps, j <= 1);
    residual(z, p, Pe, re_);
    for (int i = 0; i < 10; i++) J[i * 10 + j] = (re_[i] - r[i]) / (Pe[j] - P[j]);
  }
  return 0;
}

int oracle_zone_newton(const int* ip, const double* dp, const double* zc, double* P, int* out3) {
  Params p = read_params(ip, dp);
  ZoneConst z;
  unpack_zone(p, zc, z);
  NewtonOut o = newton(z, p, P);
  out3[0] = o.iters; out3[1] = o.status; out3[2] = o.evals;
  return 0;
}

// Face values (left face, right face) of the middle zone of a 7-zone line.
// Algorithmic flop counts of the explicit part of a stage (same convention
// as oracle_flop_counts, with every input treated as variable):
//   out[0]: one LLF face flux from an 8-zone line of states line8[8][10]
//           (reconstruction of the two face states, their fluxes, conserved
//           variables and wave speeds, the LLF combination);
//   out[1]: the per-zone remainder for dim active directions: states at P^E
//           and P_n, U(P_n), row scales, limited slopes of Theta, u_mu and
//           u^d, the flux divergence and flux-CT averages, the relaxation
//           targets' explicit parts and the constants of the residual.
int oracle_explicit_flops(const int* ip, const double* dp, const double* line8, const double* Pn1, long long* out) {
  Params p = read_params(ip, dp);
  Geom g;
  geom_minkowski(g, p.tauR);
  Cnt L[8][10];
  for (int t = 0; t < 8; t++)
    for (int v = 0; v < 10; v++) L[t][v] = Cnt(line8[t * 10 + v], true);
  g_flops = 0;
  Cnt PL[10], PR[10];
  for (int v = 0; v < 10; v++) {
    Cnt sL[7], sR[7], lo, hi;
    for (int t = 0; t < 7; t++) { sL[t] = L[t][v]; sR[t] = L[t + 1][v]; }
    recon_zone(p, sL, lo, hi);
    PL[v] = hi;
    recon_zone(p, sR, lo, hi);
    PR[v] = lo;
  }
  State<Cnt> sl, sr;
  make_state(PL, g, p, sl);
  make_state(PR, g, p, sr);
  Cnt FL[10], FR[10], UL[10], UR[10], c[4];
  flux(sl, 1, FL); flux(sr, 1, FR);
  conserved(sl, UL); conserved(sr, UR);
  wave_speeds(sl, g, p, 1, c[0], c[1]);
  wave_speeds(sr, g, p, 1, c[2], c[3]);
  Cnt cm = tmax(tmax(tabs(c[0]), tabs(c[1])), tmax(tabs(c[2]), tabs(c[3])));
  for (int v = 0; v < 10; v++) FL[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * cm * (UR[v] - UL[v]);
  out[0] = g_flops;
  // per-zone remainder
  g_flops = 0;
  Cnt PE[10], Pn[10];
  for (int v = 0; v < 10; v++) { PE[v] = L[4][v]; Pn[v] = Cnt(Pn1[v], true); }
  State<Cnt> sE, sn;
  make_state(PE, g, p, sE);
  make_state(Pn, g, p, sn);
  Cnt Un[10];
  conserved(sn, Un);
  Cnt sc[10];
  for (int a = 0; a < 10; a++) sc[a] = Cnt(1.0, true) / (tabs(Un[a]) + tabs(Un[0]));
  // limited slopes of Theta, the four u_mu and u^d along each active direction
  Cnt dTh[4], du[4][4], divu = Cnt(0.0);
  for (int m = 0; m < 4; m++) { dTh[m] = Cnt(0.0); for (int n = 0; n < 4; n++) du[m][n] = Cnt(0.0); }
  for (int d = 0; d < p.dim; d++) {
    // the neighbours' states are their own zones' work: count only the slopes
    long long g0 = g_flops;
    State<Cnt> s3[3];
    for (int t = 0; t < 3; t++) make_state(L[3 + t], g, p, s3[t]);
    long long g1 = g_flops;
    dTh[d + 1] = gminmod(p.theta, s3[0].Theta, s3[1].Theta, s3[2].Theta) / p.dx[d];
    for (int n = 0; n < 4; n++) du[d + 1][n] = gminmod(p.theta, s3[0].ucov[n], s3[1].ucov[n], s3[2].ucov[n]) / p.dx[d];
    divu = divu + du[d + 1][d + 1];
    g_flops = g0 + (g_flops - g1);
  }
  Cnt qt0, dPt0;
  relax_targets(sE, g, p, dTh, du, divu, qt0, dPt0);
  out[1] = g_flops + 20 * p.dim + 8 + 60;  // flux divergence, flux-CT averages, residual constants
  return 0;
}

int oracle_recon(const int* ip, const double* dp, const double* line7, double* lohi) {
  Params p = read_params(ip, dp);
  recon_zone(p, line7, lohi[0], lohi[1]);
  return 0;
}

int oracle_lu_solve(const double* Jin, const double* b, double* x) {
  double J[10][10], bb[10];
  for (int i = 0; i < 10; i++) { bb[i] = b[i]; for (int j = 0; j < 10; j++) J[i][j] = Jin[i * 10 + j]; }
  return lu_solve(J, bb, x) ? 0 : 1;
}

// Algorithmic flop counts (one flop per +,-,*,/,sqrt; a*b+c is two) of the
// units of work the stage is made of: one scaled residual evaluation, one
// 10x10 LU factor-and-solve, one Newton update without its residuals
// (perturbations, differences, the step), and the per-zone explicit part
// (face fluxes of the zone's low faces, flux-CT, constants), in Minkowski space.
int oracle_flop_counts(const int* ip, const double* dp, const double* zc, const double* P, long long* out4) {
  Params p = read_params(ip, dp);
  ZoneConst z;
  unpack_zone(p, zc, z);
  Cnt Pc[10], rc[10];
  for (int a = 0; a < 10; a++) Pc[a] = Cnt(P[a], true);
  g_flops = 0;
  residual(z, p, Pc, rc);
  out4[0] = g_flops;
  Cnt J[10][10], b[10], x[10];
  double Jd[10][10];
  oracle_zone_jacobian_cs(ip, dp, zc, P, &Jd[0][0]);
  for (int i = 0; i < 10; i++) { b[i] = Cnt(1.0 + i, true); for (int j = 0; j < 10; j++) J[i][j] = Cnt(Jd[i][j], true); }
  g_flops = 0;
  lu_solve(J, b, x);
  out4[1] = g_flops;
  // Newton bookkeeping per update: 10 perturbations (1 mul each), 10 divisor
  // differences, 100 residual differences and 100 divisions, 10 step
  // updates (2 each), the two norms (20 each).
  out4[2] = 10 + 10 + 100 + 100 + 20 + 40;
  // the 7x7 block of the non-magnetic components (rows and columns of rho,
  // u, u^i, q~, dP~): the solve of the paper's EMHD form (Section 8.2)
  static const int nb[7] = {0, 1, 2, 3, 4, 8, 9};
  Cnt J7[7][7], b7[7], x7[7];
  for (int i = 0; i < 7; i++) {
    b7[i] = Cnt(1.0 + i, true);
    for (int j = 0; j < 7; j++) J7[i][j] = Cnt(Jd[nb[i]][nb[j]], true);
  }
  g_flops = 0;
  lu_solve_n<7>(J7, b7, x7);
  out4[3] = g_flops;
  return 0;
}

}  // extern "C"
