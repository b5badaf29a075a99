// The explicit part of a stage in a general metric and in 3-D (Sections 2.1,
// 2.3, 2.4, 4.2): the geometry tables, the face fluxes along every active
// direction, and per zone the flux-CT on every pair of directions, the flux
// divergence, the geometric source, the limited slopes and the stage
// constants of the residual.  Also the post-stage floors and a residual
// evaluation.  Used for 3-D grids and for the modified Kerr-Schild metric;
// 2-D Minkowski grids take the specialised kernels of grim_faces.cu.
#include <type_traits>

#include "grim_gr.cuh"

namespace grim {

// ---------------------------------------------------------------- geometry
// Value and derivatives along X^1 and X^2 (forward mode).
struct D2 {
  double v, d1, d2;
  __device__ D2(double x = 0.0, double a = 0.0, double b = 0.0) : v(x), d1(a), d2(b) {}
};
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return D2(a.v + b.v, a.d1 + b.d1, a.d2 + b.d2); }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) { return D2(a.v - b.v, a.d1 - b.d1, a.d2 - b.d2); }
__device__ __forceinline__ D2 operator-(D2 a) { return D2(-a.v, -a.d1, -a.d2); }
__device__ __forceinline__ D2 operator*(D2 a, D2 b) {
  return D2(a.v * b.v, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2);
}
__device__ __forceinline__ D2 operator*(double s, D2 a) { return D2(s * a.v, s * a.d1, s * a.d2); }
__device__ __forceinline__ D2 operator/(D2 a, D2 b) {
  const double q = a.v / b.v;
  return D2(q, (a.d1 - q * b.d1) / b.v, (a.d2 - q * b.d2) / b.v);
}
__device__ __forceinline__ D2 dexp(D2 a) { const double e = exp(a.v); return D2(e, e * a.d1, e * a.d2); }
__device__ __forceinline__ D2 dsin(D2 a) { const double c = cos(a.v); return D2(sin(a.v), c * a.d1, c * a.d2); }
__device__ __forceinline__ D2 dcos(D2 a) { const double s = sin(a.v); return D2(cos(a.v), -s * a.d1, -s * a.d2); }

// Modified Kerr-Schild metric at (X^1, X^2): r = exp(X^1), theta = pi X^2 +
// ((1-h)/2) sin(2 pi X^2); g_{mu nu} = L^a_mu L^b_nu g^KS_ab with L =
// diag(1, r, dtheta/dX^2, 1) and the Kerr-Schild form of the Kerr metric
// (M = 1, Sigma = r^2 + a^2 cos^2 theta, f = 2r/Sigma): g_tt = -(1 - f),
// g_tr = f, g_tphi = -a f sin^2, g_rr = 1 + f, g_rphi = -a (1 + f) sin^2,
// g_thth = Sigma, g_phiphi = sin^2 (Sigma + a^2 (1 + f) sin^2).
__device__ void mks_metric(double a, double h, double X1, double X2, D2 g[10]) {
  const D2 x1(X1, 1.0, 0.0), x2(X2, 0.0, 1.0);
  const double tp = 2.0 * M_PI;
  const D2 r = dexp(x1);
  const D2 th = M_PI * x2 + (0.5 * (1.0 - h)) * dsin(tp * x2);
  const D2 dth = M_PI * (D2(1.0) + (1.0 - h) * dcos(tp * x2));
  const D2 sn = dsin(th), cs = dcos(th);
  const D2 s2 = sn * sn;
  const D2 sig = r * r + (a * a) * (cs * cs);
  const D2 f = 2.0 * r / sig;
  const D2 one(1.0);
  for (int q = 0; q < 10; q++) g[q] = D2(0.0);
  g[sym(0, 0)] = f - one;
  g[sym(0, 1)] = f * r;
  g[sym(0, 3)] = -a * (f * s2);
  g[sym(1, 1)] = (one + f) * r * r;
  g[sym(1, 3)] = -a * ((one + f) * s2 * r);
  g[sym(2, 2)] = sig * dth * dth;
  g[sym(3, 3)] = s2 * (sig + (a * a) * ((one + f) * s2));
}

// Inverse of a symmetric 4x4 (Gauss-Jordan, partial pivoting) and its
// determinant.
__device__ double inv4(const double g[10], double gi[10]) {
  double M[4][8];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) { M[i][j] = g[sym(i, j)]; M[i][4 + j] = (i == j) ? 1.0 : 0.0; }
  double det = 1.0;
  for (int c = 0; c < 4; c++) {
    int pv = c;
    for (int i = c + 1; i < 4; i++)
      if (fabs(M[i][c]) > fabs(M[pv][c])) pv = i;
    if (pv != c) {
      for (int j = 0; j < 8; j++) { const double t = M[c][j]; M[c][j] = M[pv][j]; M[pv][j] = t; }
      det = -det;
    }
    const double d = M[c][c];
    det *= d;
    const double id = 1.0 / d;
    for (int j = 0; j < 8; j++) M[c][j] *= id;
    for (int i = 0; i < 4; i++) {
      if (i == c) continue;
      const double m = M[i][c];
      for (int j = 0; j < 8; j++) M[i][j] -= m * M[c][j];
    }
  }
  for (int i = 0; i < 4; i++)
    for (int j = i; j < 4; j++) gi[sym(i, j)] = 0.5 * (M[i][4 + j] + M[j][4 + i]);
  return det;
}

struct GeoArgs {
  int metric;
  double a, h;
  double x0[3], dx[3];
  double tau0;
  int n1, n2;
  double* gc;   // centres, NGC planes
  double* gf1;  // X1 faces, NGF planes
  double* gf2;  // X2 faces, NGF planes
};

// One geometry point at (X1, X2); kind 0: zone centre (all planes), 1: face.
__device__ void geometry_point(const GeoArgs& A, double X1, double X2, bool polar_check, double* out,
                               long long stride, bool centre) {
  double g[10], gi[10], Gam[40], sqrtg, alpha, tau, r;
  if (A.metric == 0) {
    for (int q = 0; q < 10; q++) g[q] = gi[q] = 0.0;
    g[sym(0, 0)] = gi[sym(0, 0)] = -1.0;
    for (int i = 1; i < 4; i++) g[sym(i, i)] = gi[sym(i, i)] = 1.0;
    for (int q = 0; q < 40; q++) Gam[q] = 0.0;
    sqrtg = 1.0; alpha = 1.0; r = 1.0; tau = A.tau0;
  } else {
    D2 gd[10];
    mks_metric(A.a, A.h, X1, X2, gd);
    for (int q = 0; q < 10; q++) g[q] = gd[q].v;
    const double det = inv4(g, gi);
    sqrtg = sqrt(-det);
    alpha = 1.0 / sqrt(-gi[sym(0, 0)]);
    r = exp(X1);
    tau = A.tau0 * r * sqrt(r);
    // Gamma^l_{mn} = (1/2) g^{lk} (d_m g_{kn} + d_n g_{km} - d_k g_{mn}); d_0 = d_3 = 0
    auto dg = [&](int k, int m, int n) -> double {
      return k == 1 ? gd[sym(m, n)].d1 : (k == 2 ? gd[sym(m, n)].d2 : 0.0);
    };
    for (int l = 0; l < 4; l++)
      for (int m = 0; m < 4; m++)
        for (int n = m; n < 4; n++) {
          double s = 0.0;
          for (int k = 0; k < 4; k++) s += gi[sym(l, k)] * (dg(m, k, n) + dg(n, k, m) - dg(k, m, n));
          Gam[10 * l + sym(m, n)] = 0.5 * s;
        }
    if (polar_check) {
      const double th = M_PI * X2 + 0.5 * (1.0 - A.h) * sin(2.0 * M_PI * X2);
      if (fabs(sin(th)) < 1e-10) sqrtg = 0.0;  // polar face: no flux through it
    }
  }
  for (int q = 0; q < 10; q++) { out[(G_COV + q) * stride] = g[q]; out[(G_CON + q) * stride] = gi[q]; }
  out[G_SQRTG * stride] = sqrtg;
  out[G_ALPHA * stride] = alpha;
  if (centre) {
    out[G_TAUR * stride] = tau;
    out[G_R * stride] = r;
    for (int q = 0; q < 40; q++) out[(G_GAM + q) * stride] = Gam[q];
  }
}

__global__ void geometry_tables(const GeoArgs A) {
  const long long nc = (long long)(A.n1 + 2) * (A.n2 + 2);
  const long long nf1 = (long long)(A.n1 + 1) * (A.n2 + 2);
  const long long nf2 = (long long)(A.n1 + 2) * (A.n2 + 1);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nc) {
    const int i = (int)(t % (A.n1 + 2)) - 1, j = (int)(t / (A.n1 + 2)) - 1;
    geometry_point(A, A.x0[0] + (i + 0.5) * A.dx[0], A.x0[1] + (j + 0.5) * A.dx[1], false, A.gc + t, nc, true);
  } else if (t < nc + nf1) {
    const long long u = t - nc;
    const int i = (int)(u % (A.n1 + 1)), j = (int)(u / (A.n1 + 1)) - 1;
    geometry_point(A, A.x0[0] + i * A.dx[0], A.x0[1] + (j + 0.5) * A.dx[1], false, A.gf1 + u, nf1, false);
  } else if (t < nc + nf1 + nf2) {
    const long long u = t - nc - nf1;
    const int i = (int)(u % (A.n1 + 2)) - 1, j = (int)(u / (A.n1 + 2));
    geometry_point(A, A.x0[0] + (i + 0.5) * A.dx[0], A.x0[1] + j * A.dx[1], true, A.gf2 + u, nf2, false);
  }
}

// ---------------------------------------------------------------- grid access
struct GrArgs {
  const double* Pn;
  const double* PE;
  const double* guess;
  double dts, kappa;
  double idts;  // 1/dt_s, once on the host
  double* K;
  double* P0;
  double* F[3];
  double* Dv;   // [ND][ghost-ring grid]: derived P^E quantities of every centre
  double* Src;  // [NSRC][N]: sources at P^E of every zone
  const double* gc;
  const double* gf[2];
  // P_n quantities shared by the two stages of a step (NCACHE_GR planes):
  // sqrt(-g) U(P_n) [10], Theta_n, u_mu,n [4], u^t_n.  mode 0: a general
  // stage (no cache); 1: the half step (the sources kernel, whose P^E is
  // P_n, writes the cache; the zone-constant kernel reads it); 2: the full
  // step (reads the cache and the row weights K_U the half step wrote, which
  // depend on P_n only).
  double* cache;
  int mode;
  // with a learned start: the ten increment features -r_a(P_n) of each zone
  // (float32 [10][N]), from the constants computed here
  float* feat;
  // float-float copies of gamma, gamma-1, sqrt(phi gamma), sqrt(psi gamma)
  // and kappa gamma (hi, lo pairs), for the float-float face states
  float ffc[10];
  // the mixed solver's MC slopes along the face direction being computed
  // ([NV][ghost-ring grid] float pairs, mc_slopes_gr), in the scratch the
  // derived and source quantities take later in the stage
  double* Sl;
};
constexpr int NCACHE_GR = NV + 6;

// Extents and offsets of the face array of direction D: along D the faces
// 0..n_D; across it one ring of ghost faces in every active direction.
struct FaceBox {
  int e[3], o[3];
  long long size;
  __device__ __host__ long long at(int i, int j, int k) const {
    return ((long long)(k + o[2]) * e[1] + (j + o[1])) * e[0] + (i + o[0]);
  }
};
__host__ __device__ inline FaceBox face_box(const Params& p, int D) {
  FaceBox b;
  const int n[3] = {p.n1, p.n2, p.n3};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const bool act = d < p.dim;
    b.e[d] = (d == D) ? n[d] + 1 : (act ? n[d] + 2 : 1);
    b.o[d] = (d == D) ? 0 : (act ? 1 : 0);
  }
  b.size = (long long)b.e[0] * b.e[1] * b.e[2];
  return b;
}

// Map one index by the boundary rule of direction d (periodic, outflow copy,
// or reflection with period 2n and a sign flip of the d-components of u~ and
// B); inactive directions map to 0.
__device__ __forceinline__ int gr_map(const Params& p, int d, int i, bool& flip) {
  const int n = d == 0 ? p.n1 : d == 1 ? p.n2 : p.n3;
  if (d >= p.dim) return 0;
  if (i >= 0 && i < n) return i;
  const int bc = p.bc[d][i < 0 ? 0 : 1];
  if (bc == BC_PERIODIC) return ((i % n) + n) % n;
  if (bc == BC_OUTFLOW) return i < 0 ? 0 : n - 1;
  const int m = ((i % (2 * n)) + 2 * n) % (2 * n);
  if (m >= n) { flip = !flip; return 2 * n - 1 - m; }
  return m;
}
__device__ __forceinline__ long long gr_zone(const Params& p, int i, int j, int k, bool f[3]) {
  f[0] = f[1] = f[2] = false;
  const int a = gr_map(p, 0, i, f[0]), b = gr_map(p, 1, j, f[1]), c = gr_map(p, 2, k, f[2]);
  return ((long long)c * p.n2 + b) * p.n1 + a;
}
__device__ __forceinline__ void gr_prim(const Params& p, const double* P, int i, int j, int k, double out[NV]) {
  bool f[3];
  const long long z = gr_zone(p, i, j, k, f);
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = __ldg(P + v * p.N + z);
#pragma unroll
  for (int d = 0; d < 3; d++)
    if (f[d]) { out[2 + d] = -out[2 + d]; out[5 + d] = -out[5 + d]; }
}

// Table accessor at a 2-D index with a plane stride.
struct GT {
  const double* p;
  long long s;
  __device__ __forceinline__ double operator()(int a) const { return __ldg(p + a * s); }
};
__device__ __forceinline__ GT centre_geo(const Params& p, const double* gc, int i, int j) {
  const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
  if (p.dim < 2) j = 0;
  return GT{gc + (long long)(j + 1) * (p.n1 + 2) + (i + 1), nc};
}

// cs~^2 / c_s^2 of the closure (Eq. modcs with v_q^2 = (gamma-1) chi/tau_R,
// v_dP^2 = 4 nu/(3 tau_R), chi = phi c_s^2 tau_R, nu = psi c_s^2 tau_R).
static double gr_kappa(const Params& p) {
  const double a = p.cond ? (p.gamma - 1.0) * p.phi : 0.0;
  const double b = p.visc ? 4.0 * p.psi / 3.0 : 0.0;
  return 0.5 * (1.0 + a + sqrt(1.0 + a * a)) + b;
}

// ---------------------------------------------------------------- faces
// Physical constants in the working precision: float64 from the parameters,
// float-float from the host-split copies; kk is kappa in float64 and kappa
// gamma in float-float (the argument each form of the speeds takes).
template <typename S> __device__ __forceinline__ void gr_consts(const Params& p, const GrArgs& a, RC<S>& c, S& kk) {
  if constexpr (std::is_same<S, double>::value) {
    c = make_rc<double>(p);
    kk = a.kappa;
  } else {
    c.gam = S(a.ffc[0], a.ffc[1]);
    c.gm1 = S(a.ffc[2], a.ffc[3]);
    c.sphig = S(a.ffc[4], a.ffc[5]);
    c.spsig = S(a.ffc[6], a.ffc[7]);
    c.cond = p.cond;
    c.visc = p.visc;
    kk = S(a.ffc[8], a.ffc[9]);
  }
}
template <typename S>
__device__ __forceinline__ void face_speeds(const ZG<S>& z, S gtt, S gtj, S gjj, int j, const RC<S>& c, S kk, S& cmin,
                                            S& cmax) {
  if constexpr (std::is_same<S, double>::value) zg_speeds(z, gtt, gtj, gjj, j, c.gam, kk, cmin, cmax);
  else zg_speeds_kg(z, gtt, gtj, gjj, j, c.gam, kk, cmin, cmax);
}

// Centres of the grid with one ghost ring in every active direction.
constexpr int ND = 8;  // Theta, u_mu (4), sqrt(-g) u^d (3)
struct GhostBox {
  int e1, e2, e3, o2, o3;
  long long size;
  __device__ __host__ long long at(int i, int j, int k) const {
    return ((long long)(k + o3) * e2 + (j + o2)) * e1 + (i + 1);
  }
};
__host__ __device__ inline GhostBox ghost_box(const Params& p) {
  GhostBox b;
  b.o2 = p.dim >= 2;
  b.o3 = p.dim >= 3;
  b.e1 = p.n1 + 2;
  b.e2 = b.o2 ? p.n2 + 2 : 1;
  b.e3 = b.o3 ? p.n3 + 2 : 1;
  b.size = (long long)b.e1 * b.e2 * b.e3;
  return b;
}

// LLF or HLLE flux (Section 2.4.2) on the face at the low side of zone
// (i,j,k) in direction D, from MC, WENO5 or PPM face states of P^E.  The
// stencil's zone indices and reflection flips are resolved once; the fields
// are then loaded and reconstructed one at a time, in float64.  The face
// states, fluxes and speeds are evaluated in S: float64, or float-float for
// the mixed solver.
template <int D, int RECON, typename S>
__device__ __forceinline__ void face_body(const Params& p, const GrArgs& a, int i, int j, int k, const GT& g,
                                          double* out, long long plane) {
  constexpr bool WIDE = RECON != RECON_MC;
  constexpr int o0 = WIDE ? -3 : -2, o1 = WIDE ? 2 : 1, NS = o1 - o0 + 1;
  long long zz[NS];
  int fl[NS];  // reflection flips of the stencil zone, bit d for direction d
#pragma unroll
  for (int t = 0; t < NS; t++) {
    bool f[3];
    zz[t] = gr_zone(p, i + (D == 0) * (t + o0), j + (D == 1) * (t + o0), k + (D == 2) * (t + o0), f);
    fl[t] = (f[0] ? 1 : 0) | (f[1] ? 2 : 0) | (f[2] ? 4 : 0);
  }
  const long long N = p.N;
  S L[NV], R[NV];
  if constexpr (RECON == RECON_MC && std::is_same<S, ff>::value) {
    // the mixed solver: face values from the two centres beside the face and
    // their float-float slopes (mc_slopes_gr), P -+ slope/2 in float-float
    const GhostBox gb = ghost_box(p);
    const long long c0 = gb.at(i - (D == 0), j - (D == 1), k - (D == 2)), c1 = gb.at(i, j, k);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const int bit = (v >= 2 && v <= 4) ? 1 << (v - 2) : (v >= 5 && v <= 7) ? 1 << (v - 5) : 0;
      const double x0 = __ldg(a.PE + v * N + zz[1]), x1 = __ldg(a.PE + v * N + zz[2]);
      const float2 s0 = __ldg(reinterpret_cast<const float2*>(a.Sl) + v * gb.size + c0);
      const float2 s1 = __ldg(reinterpret_cast<const float2*>(a.Sl) + v * gb.size + c1);
      L[v] = ff_split((fl[1] & bit) ? -x0 : x0) + scale2(ff(s0.x, s0.y), 0.5f);
      R[v] = ff_split((fl[2] & bit) ? -x1 : x1) - scale2(ff(s1.x, s1.y), 0.5f);
    }
  } else {
#pragma unroll
  for (int v = 0; v < NV; v++) {
    // u~^d and B^d change sign in a zone mirrored across a boundary of direction d
    const int bit = (v >= 2 && v <= 4) ? 1 << (v - 2) : (v >= 5 && v <= 7) ? 1 << (v - 5) : 0;
    double s[NS];
#pragma unroll
    for (int t = 0; t < NS; t++) {
      const double x = __ldg(a.PE + v * N + zz[t]);
      s[t] = (fl[t] & bit) ? -x : x;
    }
    double lv, rv;
    if (RECON == RECON_WENO5) {
      lv = weno5v(s[0], s[1], s[2], s[3], s[4]);
      rv = weno5v(s[5], s[4], s[3], s[2], s[1]);
    } else if (RECON == RECON_PPM) {
      double lo, hi;
      ppm_zone(p.theta, s[0], s[1], s[2], s[3], s[4], lo, hi);
      lv = hi;
      ppm_zone(p.theta, s[1], s[2], s[3], s[4], s[5], lo, hi);
      rv = lo;
    } else {
      lv = fma(0.5, gm_slope(p.theta, s[0], s[1], s[2]), s[1]);
      rv = fma(-0.5, gm_slope(p.theta, s[1], s[2], s[3]), s[2]);
    }
    L[v] = from_double<S>(lv);
    R[v] = from_double<S>(rv);
  }
  }
  Met<S> m;
  met_load(m, g);
  RC<S> c;
  S kk;
  gr_consts(p, a, c, kk);
  S FL[NV], FR[NV], UL[NV], UR[NV], cminL, cmaxL, cminR, cmaxR;
  const S gtt = from_double<S>(g(G_CON + sym(0, 0))), gtj = from_double<S>(g(G_CON + sym(0, D + 1)));
  const S gjj = from_double<S>(g(G_CON + sym(D + 1, D + 1)));
  {
    ZG<S> z;
    zg_load(z, L, m, c);
    zg_conserved(z, UL);
    zg_flux(z, D + 1, FL);
    face_speeds(z, gtt, gtj, gjj, D + 1, c, kk, cminL, cmaxL);
  }
  {
    ZG<S> z;
    zg_load(z, R, m, c);
    zg_conserved(z, UR);
    zg_flux(z, D + 1, FR);
    face_speeds(z, gtt, gtj, gjj, D + 1, c, kk, cminR, cmaxR);
  }
  const S sg = from_double<S>(g(G_SQRTG));
  if constexpr (std::is_same<S, double>::value) {
    double Fv[NV];
    if (p.riemann == 1) {  // HLLE (Section 2.4.2)
      const double cR = fmax(fmax(cmaxL, cmaxR), 0.0), cL = fmax(-fmin(cminL, cminR), 0.0);
      const double iw = 1.0 / (cL + cR);
#pragma unroll
      for (int v = 0; v < NV; v++) Fv[v] = (cR * FL[v] + cL * FR[v] - cR * cL * (UR[v] - UL[v])) * iw;
    } else {               // LLF
      const double cm = fmax(fmax(cmaxL, -cminL), fmax(cmaxR, -cminR));
#pragma unroll
      for (int v = 0; v < NV; v++) Fv[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * cm * (UR[v] - UL[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * plane] = sg * Fv[v];
  } else if (p.riemann == 1) {
    const S cR = fmax(fmax(cmaxL, cmaxR), tconst<S>(0.0)), cL = fmax(-fmin(cminL, cminR), tconst<S>(0.0));
    const S iw = sg * nr_rcp(cL + cR);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * plane] = as_double((cR * FL[v] + cL * FR[v] - cR * cL * (UR[v] - UL[v])) * iw);
  } else {               // LLF
    const S cm = fmax(fmax(cmaxL, -cminL), fmax(cmaxR, -cminR));
    const S h = tconst<S>(0.5) * sg;
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * plane] = as_double(h * ((FL[v] + FR[v]) - cm * (UR[v] - UL[v])));
  }
}

// The mixed solver's MC slopes along D, once per centre of the ghost-ring
// grid, in float-float: each face reads the slopes of the two centres beside
// it, which the face kernel formed twice, in float64 (the float64 pipe was
// the face kernel's busiest).  The centres and their reflection flips are
// resolved as in face_body, so every face sees the values it would have
// formed itself; each slope is stored as its float pair (8 bytes, like a
// double, without a rounding to one).
template <int D>
__global__ void __launch_bounds__(128) mc_slopes_gr(const __grid_constant__ Params p,
                                                    const __grid_constant__ GrArgs a) {
  const GhostBox gb = ghost_box(p);
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= gb.size) return;
  const int i = (int)(q % gb.e1) - 1;
  const int j = (int)((q / gb.e1) % gb.e2) - gb.o2;
  const int k = (int)(q / ((long long)gb.e1 * gb.e2)) - gb.o3;
  long long zz[3];
  int fl[3];
#pragma unroll
  for (int t = 0; t < 3; t++) {
    bool f[3];
    zz[t] = gr_zone(p, i + (D == 0) * (t - 1), j + (D == 1) * (t - 1), k + (D == 2) * (t - 1), f);
    fl[t] = (f[0] ? 1 : 0) | (f[1] ? 2 : 0) | (f[2] ? 4 : 0);
  }
  const long long N = p.N;
  const ff theta = ff_split(p.theta);
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const int bit = (v >= 2 && v <= 4) ? 1 << (v - 2) : (v >= 5 && v <= 7) ? 1 << (v - 5) : 0;
    ff t3[3];
#pragma unroll
    for (int t = 0; t < 3; t++) {
      const double x = __ldg(a.PE + v * N + zz[t]);
      t3[t] = ff_split((fl[t] & bit) ? -x : x);
    }
    const ff sl = gm_slope(theta, t3[0], t3[1], t3[2]);
    reinterpret_cast<float2*>(a.Sl)[v * gb.size + q] = make_float2(sl.hi, sl.lo);
  }
}

// One kernel per direction and reconstruction, so that each holds only its
// own registers; the float-float form is held to four blocks of 128 threads
// per SM (128 registers, about 200 bytes spilled), for the latency of its
// dependent float chains: 7 % faster than three blocks at 168 registers.
template <int D, typename S, int RECON>
__global__ void __launch_bounds__(128, std::is_same<S, ff>::value ? 4 : 1) face_flux_gr(const __grid_constant__ Params p,
                                                    const __grid_constant__ GrArgs a) {
  const FaceBox fb = face_box(p, D);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= fb.size) return;
  const int i = (int)(f % fb.e[0]) - fb.o[0];
  const int j = (int)((f / fb.e[0]) % fb.e[1]) - fb.o[1];
  const int k = (int)(f / ((long long)fb.e[0] * fb.e[1])) - fb.o[2];
  double* out = a.F[D] + f;
  // face geometry
  GT g;
  if (D == 0) g = GT{a.gf[0] + (long long)((p.dim >= 2 ? j : 0) + 1) * (p.n1 + 1) + i,
                     (long long)(p.n1 + 1) * (p.n2 + 2)};
  else if (D == 1) g = GT{a.gf[1] + (long long)j * (p.n1 + 2) + (i + 1), (long long)(p.n1 + 2) * (p.n2 + 1)};
  else g = centre_geo(p, a.gc, i, j);
  if (g(G_SQRTG) == 0.0) {
#pragma unroll
    for (int v = 0; v < NV; v++) out[v * fb.size] = 0.0;
    return;
  }
  face_body<D, RECON, S>(p, a, i, j, k, g, out, fb.size);
}

// ---------------------------------------------------------------- zone constants
// Theta, u_mu and sqrt(-g) u^d of the P^E state of zone (i,j,k) (ghosts by the
// boundary rules, geometry of the ghost centre itself).
__device__ __forceinline__ void gr_derived(const Params& p, const GrArgs& a, int i, int j, int k,
                                           const RC<double>& c, double& th, double ucov[4], double sgu[3]) {
  double P[NV];
  gr_prim(p, a.PE, i, j, k, P);
#pragma unroll
  for (int v = 5; v < NV; v++) P[v] = 0.0;  // B, q~, dP~ do not enter
  const GT g = centre_geo(p, a.gc, i, j);
  Met<double> m;
  met_load(m, g);
  ZG<double> z;
  zg_load(z, P, m, c);
  th = z.theta;
  const double sg = g(G_SQRTG);
#pragma unroll
  for (int q = 0; q < 4; q++) ucov[q] = z.ucov[q];
#pragma unroll
  for (int d = 0; d < 3; d++) sgu[d] = sg * z.ucon[d + 1];
}

// The derived quantities of every zone and ghost centre (one ring along each
// active direction), [ND][e1 e2 e3] with e1 = n1+2, e2 = n2+2 or 1, e3 = n3+2
// or 1: computed once a stage here, read by the limited slopes of up to seven
// zones.

__global__ void __launch_bounds__(128) derived_gr(const __grid_constant__ Params p, const __grid_constant__ GrArgs a) {
  const GhostBox gb = ghost_box(p);
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= gb.size) return;
  const int i = (int)(q % gb.e1) - 1;
  const int j = (int)((q / gb.e1) % gb.e2) - gb.o2;
  const int k = (int)(q / ((long long)gb.e1 * gb.e2)) - gb.o3;
  const RC<double> c = make_rc<double>(p);
  double th, u[4], s[3];
  gr_derived(p, a, i, j, k, c, th, u, s);
  double* D = a.Dv + q;
  D[0] = th;
#pragma unroll
  for (int m = 0; m < 4; m++) D[(1 + m) * gb.size] = u[m];
#pragma unroll
  for (int d = 0; d < 3; d++) D[(5 + d) * gb.size] = s[d];
}
__device__ __forceinline__ void derived_load(const GrArgs& a, const GhostBox& gb, int i, int j, int k, double& th,
                                             double u[4], double s[3]) {
  const double* D = a.Dv + gb.at(i, j, k);
  th = __ldg(D);
#pragma unroll
  for (int m = 0; m < 4; m++) u[m] = __ldg(D + (1 + m) * gb.size);
#pragma unroll
  for (int d = 0; d < 3; d++) s[d] = __ldg(D + (5 + d) * gb.size);
}

// Sources at P^E of every zone: the geometric source sqrt(-g) T^k_l
// Gamma^l_{nu k} (rows 1..4), the closure coefficients of q~ and dP~ (with
// the limited slopes of Theta, u_mu and sqrt(-g) u^d from the derived
// quantities) and the spatial part of nabla_mu u^mu; NSRC doubles a zone.
constexpr int NSRC = 17;  // Sg (4), Aq, Bq, Cq (4), Ad, Dd (4), Ed, divu_sp
// Square root in the sources' working precision: the library's in float64
// (as before the float-float form existed), the float-float one otherwise.
__device__ __forceinline__ double src_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ ff src_sqrt(ff x) { return sqr_root(x); }

// FFS: the mixed solver's form.  The sources are explicit terms at P^E, the
// class the mixed solver's float-float face fluxes belong to: the state in
// the metric, the limited slopes, the connection contractions, the geometric
// source and the closure coefficients are evaluated in float-float (T = ff)
// and each stored source is joined into a double once.  The half step's
// P_n cache (sqrt(-g) U(P_n) and the P_n quantities) stays float64.
// Otherwise everything is float64 (T = double).
template <bool FFS>
__global__ void __launch_bounds__(128, FFS ? 4 : 0) sources_gr(const __grid_constant__ Params p, const __grid_constant__ GrArgs a) {
  using T = typename std::conditional<FFS, ff, double>::type;
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const int i = (int)(z % p.n1), j = (int)((z / p.n1) % p.n2), k = (int)(z / ((long long)p.n1 * p.n2));
  const GT g = centre_geo(p, a.gc, i, j);
  const T sg = from_double<T>(g(G_SQRTG)), tau = from_double<T>(g(G_TAUR));
  double PEz[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) PEz[v] = __ldg(a.PE + v * N + z);
  const T zero = T(0), third_c = tconst<T>(1.0 / 3.0);
  // --- limited slopes at P^E of Theta, u_mu and sqrt(-g) u^d
  T dTh[3] = {zero, zero, zero}, du[3][4], divu_sp = zero;
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int q = 0; q < 4; q++) du[d][q] = zero;
  {
    const GhostBox gb = ghost_box(p);
    double th0, u0[4], s0[3];
    derived_load(a, gb, i, j, k, th0, u0, s0);
    const T theta = from_double<T>(p.theta);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      if (d >= p.dim) continue;
      double thm, thp, um[4], up[4], sm[3], sp[3];
      derived_load(a, gb, i - (d == 0), j - (d == 1), k - (d == 2), thm, um, sm);
      derived_load(a, gb, i + (d == 0), j + (d == 1), k + (d == 2), thp, up, sp);
      const T ih = from_double<T>(p.idx[d]);
      dTh[d] = gm_slope(theta, from_double<T>(thm), from_double<T>(th0), from_double<T>(thp)) * ih;
#pragma unroll
      for (int q = 0; q < 4; q++)
        du[d][q] = gm_slope(theta, from_double<T>(um[q]), from_double<T>(u0[q]), from_double<T>(up[q])) * ih;
      divu_sp += gm_slope(theta, from_double<T>(sm[d]), from_double<T>(s0[d]), from_double<T>(sp[d])) * ih;
    }
    divu_sp *= nr_rcp(sg);
  }
  // --- sources at P^E
  RC<T> c;
  T kk;
  gr_consts(p, a, c, kk);
  Met<T> m;
  met_load(m, g);
  T PEt[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) PEt[v] = from_double<T>(PEz[v]);
  ZG<T> ze;
  zg_load(ze, PEt, m, c);
  const T cs2E = c.gam * ze.pg * nr_rcp(ze.rho + c.gam * ze.u);
  const T ith = nr_rcp(ze.theta);
  const T* bh = ze.bhcon;
  // Gl[sym(mu, nu)] = sum_l Gamma^l_{mu nu} u_l and Gb[sym(mu, nu)] = sum_l
  // Gamma^l_{mu nu} bhat_l at P^E (symmetric in mu, nu), and from Gl the sum
  // over nu, l of Gamma^l_{nu mu} u^nu u_l for each mu
  T Gl[10], Gb[10];
#pragma unroll
  for (int a = 0; a < 10; a++) {
    T s = zero, t = zero;
#pragma unroll
    for (int l = 0; l < 4; l++) {
      const T G = from_double<T>(g(G_GAM + 10 * l + a));
      s += G * ze.ucov[l];
      t += G * ze.bhcov[l];
    }
    Gl[a] = s;
    Gb[a] = t;
  }
  T Gu[4];
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    T s = zero;
#pragma unroll
    for (int nu = 0; nu < 4; nu++) s += Gl[sym(nu, mu)] * ze.ucon[nu];
    Gu[mu] = s;
  }
  // --- geometric source at P^E: sqrt(-g) T^k_l Gamma^l_{nu k} (rows 1..4),
  // with T^k_l of Eq. fullSEtens taken apart: (w + b^2 + dP/3) u^k u_l +
  // p_t delta^k_l - b^2 bhat^k bhat_l + q (bhat^k u_l + u^k bhat_l) - dP
  // bhat^k bhat_l, so that each part contracts Gamma with the vectors alone
  T Sg[4];
  {
    const T q = ze.qt * ze.qs, dp = ze.dpt * ze.ds, third = dp * third_c;
    const T A = ze.w0 + ze.bsq + third, pt = ze.pg + tconst<T>(0.5) * ze.bsq + third;
#pragma unroll
    for (int n = 0; n < 4; n++) {
      T bGl = zero, uGb = zero, bGb = zero, tr = zero;
#pragma unroll
      for (int kk2 = 0; kk2 < 4; kk2++) {
        bGl += bh[kk2] * Gl[sym(n, kk2)];
        uGb += ze.ucon[kk2] * Gb[sym(n, kk2)];
        bGb += bh[kk2] * Gb[sym(n, kk2)];
        tr += from_double<T>(g(G_GAM + 10 * kk2 + sym(n, kk2)));  // Gamma^k_{n k}
      }
      Sg[n] = sg * (A * Gu[n] + pt * tr + q * (bGl + uGb) - (ze.bsq + dp) * bGb);
    }
  }
  // heat flux: q~_0 = Aq + Bq (Theta - Theta_n)/dt_s + Cq^mu (u_mu - u_mu,n)/dt_s
  T Aq = zero, Bq = zero, Cq[4] = {zero, zero, zero, zero};
  if (p.cond) {
    const T chi = from_double<T>(p.phi) * cs2E * tau;
    const T pre = -(src_sqrt(tau * ze.rho * chi) * ith);
    T acc = zero;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      T a_sp = -Gu[mu];
#pragma unroll
      for (int d = 0; d < 3; d++) a_sp += ze.ucon[d + 1] * du[d][mu];
      acc += bh[mu] * a_sp;
    }
    Aq = pre * (bh[1] * dTh[0] + bh[2] * dTh[1] + bh[3] * dTh[2] + ze.theta * acc);
    Bq = pre * bh[0];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) Cq[mu] = pre * ze.theta * bh[mu] * ze.ucon[0];
  }
  // anisotropy: dP~_0 = Ad + Dd^nu (u_nu - u_nu,n)/dt_s + Ed (u^t - u^t_n)/dt_s
  T Ad = zero, Dd[4] = {zero, zero, zero, zero}, Ed = zero;
  if (p.visc) {
    const T nu = from_double<T>(p.psi) * cs2E * tau;
    const T pre = tconst<T>(3.0) * src_sqrt(tau * ze.rho * nu * ith);
    T sp = zero;
#pragma unroll
    for (int mu = 0; mu < 4; mu++)
#pragma unroll
      for (int nn = 0; nn < 4; nn++) {
        T nab = zero;
        if (mu >= 1) nab = du[mu - 1][nn];
        nab -= Gl[sym(mu, nn)];
        sp += bh[mu] * bh[nn] * nab;
      }
    Ad = pre * (sp - divu_sp * third_c);
#pragma unroll
    for (int nn = 0; nn < 4; nn++) Dd[nn] = pre * bh[0] * bh[nn];
    Ed = -(pre * third_c);
  }
  double* Sz = a.Src + z;
  const T x[NSRC] = {Sg[0], Sg[1], Sg[2], Sg[3], Aq, Bq, Cq[0], Cq[1], Cq[2], Cq[3],
                     Ad, Dd[0], Dd[1], Dd[2], Dd[3], Ed, divu_sp};
#pragma unroll
  for (int q = 0; q < NSRC; q++) Sz[q * N] = as_double(x[q]);
  if (a.mode == 1) {
    // the half step's P^E is P_n: its quantities go to the step's P_n cache
    // for the zone-constant kernels of both stages, in float64
    ZG<double> zn;
    if constexpr (FFS) {
      Met<double> m64;
      met_load(m64, g);
      zg_load(zn, PEz, m64, make_rc<double>(p));
    } else {
      zn = ze;
    }
    double U[NV];
    zg_conserved(zn, U);
    const double sgd = g(G_SQRTG);
#pragma unroll
    for (int v = 0; v < NV; v++) a.cache[v * N + z] = sgd * U[v];
    a.cache[NV * N + z] = zn.theta;
#pragma unroll
    for (int q = 0; q < 4; q++) a.cache[(NV + 1 + q) * N + z] = zn.ucov[q];
    a.cache[(NV + 5) * N + z] = zn.ucon[0];
  }
}

// The stage constants of every zone (float64): flux divergence with flux-CT,
// U(P_n), the row scales, and the sources from sources_gr.
__global__ void __launch_bounds__(128) zone_const_gr(const __grid_constant__ Params p,
                                                     const __grid_constant__ GrArgs a) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  const int i = (int)(z % p.n1), j = (int)((z / p.n1) % p.n2), k = (int)(z / ((long long)p.n1 * p.n2));
  const int ijk[3] = {i, j, k};
  // --- flux divergence with flux-CT on every pair of active directions
  FaceBox fb[3];
#pragma unroll
  for (int d = 0; d < 3; d++) fb[d] = face_box(p, d);
  double divF[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) divF[v] = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (d >= p.dim) continue;
    const long long lo = fb[d].at(i, j, k);
    const long long hi = fb[d].at(i + (d == 0), j + (d == 1), k + (d == 2));
    const double* F = a.F[d];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      // F^d[B^d] = 0; F^d[B^c] for an active c comes from the corner averages
      // below; for an inactive c (B^3 in 2-D) it is the face flux itself
      if (v >= 5 && v <= 7 && (v - 5 == d || v - 5 < p.dim)) continue;
      divF[v] += (__ldg(F + v * fb[d].size + hi) - __ldg(F + v * fb[d].size + lo)) * p.idx[d];
    }
  }
#pragma unroll
  for (int A = 0; A < 3; A++)
#pragma unroll
    for (int B = A + 1; B < 3; B++) {
      if (B >= p.dim) continue;
      // E_AB at the four (A,B) edges of the zone: E(sa, sb) at zone ijk + sa e_A + sb e_B,
      // E(q) = (F^A[B^B](q) + F^A[B^B](q - e_B) - F^B[B^A](q) - F^B[B^A](q - e_A)) / 4
      double E[2][2];
      const double* FA = a.F[A] + (5 + B) * fb[A].size;
      const double* FB = a.F[B] + (5 + A) * fb[B].size;
#pragma unroll
      for (int sa = 0; sa < 2; sa++)
#pragma unroll
        for (int sb = 0; sb < 2; sb++) {
          int q[3] = {ijk[0], ijk[1], ijk[2]};
          q[A] += sa;
          q[B] += sb;
          int qb[3] = {q[0], q[1], q[2]}; qb[B] -= 1;
          int qa[3] = {q[0], q[1], q[2]}; qa[A] -= 1;
          E[sa][sb] = 0.25 * (__ldg(FA + fb[A].at(q[0], q[1], q[2])) + __ldg(FA + fb[A].at(qb[0], qb[1], qb[2])) -
                              __ldg(FB + fb[B].at(q[0], q[1], q[2])) - __ldg(FB + fb[B].at(qa[0], qa[1], qa[2])));
        }
      // F^A[B^B] = (E(q) + E(q + e_B))/2 on A faces; F^B[B^A] = -(E(q) + E(q + e_A))/2 on B faces
      divF[5 + B] += (0.5 * (E[1][0] + E[1][1]) - 0.5 * (E[0][0] + E[0][1])) * p.idx[A];
      divF[5 + A] += (-0.5 * (E[0][1] + E[1][1]) + 0.5 * (E[0][0] + E[1][0])) * p.idx[B];
    }
  // --- state at P_n and the conserved variables U(P_n) (float64); in a
  // step of grim_step from the cache the half step's sources kernel wrote
  const GT g = centre_geo(p, a.gc, i, j);
  const double sg = g(G_SQRTG), tau = g(G_TAUR);
  double Pnz[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) Pnz[v] = __ldg(a.Pn + v * N + z);
  double Un[NV], th_n, ucn[4], ut_n;
  if (a.mode != 0) {
#pragma unroll
    for (int v = 0; v < NV; v++) Un[v] = __ldg(a.cache + v * N + z);
    th_n = __ldg(a.cache + NV * N + z);
#pragma unroll
    for (int m = 0; m < 4; m++) ucn[m] = __ldg(a.cache + (NV + 1 + m) * N + z);
    ut_n = __ldg(a.cache + (NV + 5) * N + z);
  } else {
    const RC<double> c = make_rc<double>(p);
    Met<double> m;
    met_load(m, g);
    ZG<double> zn;
    zg_load(zn, Pnz, m, c);
    zg_conserved(zn, Un);
#pragma unroll
    for (int v = 0; v < NV; v++) Un[v] *= sg;
    th_n = zn.theta;
#pragma unroll
    for (int q = 0; q < 4; q++) ucn[q] = zn.ucov[q];
    ut_n = zn.ucon[0];
  }
  const double qt_n = Pnz[8], dpt_n = Pnz[9];
  // --- sources at P^E (geometric source, closure coefficients)
  double Sg[4], Aq, Bq, Cq[4], Ad, Dd[4], Ed, divu_sp, hoq, hod;
  {
    const double* Sz = a.Src + z;
    double x[NSRC];
#pragma unroll
    for (int q = 0; q < NSRC; q++) x[q] = __ldg(Sz + q * N);
#pragma unroll
    for (int q = 0; q < 4; q++) { Sg[q] = x[q]; Cq[q] = x[6 + q]; Dd[q] = x[11 + q]; }
    Aq = x[4]; Bq = x[5]; Ad = x[10]; Ed = x[15]; divu_sp = x[16];
    hoq = p.ho ? 0.5 * __ldg(a.PE + 8 * N + z) : 0.0;
    hod = p.ho ? 0.5 * __ldg(a.PE + 9 * N + z) : 0.0;
  }
  // --- stage constants (row scale folded in; sqrt(-g) folded into kU)
  const double dts = a.dts, idts = a.idts, it = nr_rcp(tau), isg = nr_rcp(sg);
  double* Kz = a.K + z;
  double sr[NV];  // 1/(|U_v(P_n)| + |U_0(P_n)|)
  double r[NV];   // the stage's scaled residual at P_n: the learned start's features
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if (a.mode == 2) {
      sr[v] = Kz[(K_U + v) * N] * isg;
    } else {
      sr[v] = nr_rcp(fabs(Un[v]) + fabs(Un[0]));
      Kz[(K_U + v) * N] = sr[v] * sg;
    }
    const double src = (v >= 1 && v <= 4) ? Sg[v - 1] : 0.0;
    const double kc = sr[v] * (dts * (divF[v] - src) - Un[v]);
    Kz[(K_C + v) * N] = kc;
    r[v] = sr[v] * Un[v] + kc;
  }
  {
    const double s8 = sr[8] * dts;
    double cst = -Un[8] * idts + divF[8];
    double src = 0.5 * qt_n * it - Aq * it + Bq * th_n * idts * it;
    #pragma unroll
    for (int mu = 0; mu < 4; mu++) src += Cq[mu] * ucn[mu] * idts * it;
    src -= hoq * (divu_sp - ut_n * idts);
    cst += sg * src;
    const double kq[7] = {sg * 0.5 * s8 * it, -sg * s8 * Bq * idts * it, -sg * s8 * Cq[0] * idts * it,
                          -sg * s8 * Cq[1] * idts * it, -sg * s8 * Cq[2] * idts * it, -sg * s8 * Cq[3] * idts * it,
                          -sg * s8 * hoq * idts};
    const double kc = s8 * cst;
    Kz[(K_C + 8) * N] = kc;
#pragma unroll
    for (int q = 0; q < 7; q++) Kz[(K_Q + q) * N] = kq[q];
    r[8] = sr[8] * Un[8] + kc + kq[0] * qt_n + kq[1] * th_n + kq[6] * ut_n;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) r[8] += kq[2 + mu] * ucn[mu];
  }
  {
    const double s9 = sr[9] * dts;
    double cst = -Un[9] * idts + divF[9];
    double src = 0.5 * dpt_n * it - Ad * it + Ed * ut_n * idts * it;
    #pragma unroll
    for (int nn = 0; nn < 4; nn++) src += Dd[nn] * ucn[nn] * idts * it;
    src -= hod * (divu_sp - ut_n * idts);
    cst += sg * src;
    const double kd[6] = {sg * 0.5 * s9 * it, -sg * s9 * Dd[0] * idts * it, -sg * s9 * Dd[1] * idts * it,
                          -sg * s9 * Dd[2] * idts * it, -sg * s9 * Dd[3] * idts * it,
                          -sg * s9 * (Ed * idts * it + hod * idts)};
    const double kc = s9 * cst;
    Kz[(K_C + 9) * N] = kc;
#pragma unroll
    for (int q = 0; q < 6; q++) Kz[(K_D + q) * N] = kd[q];
    r[9] = sr[9] * Un[9] + kc + kd[0] * dpt_n + kd[5] * ut_n;
#pragma unroll
    for (int nn = 0; nn < 4; nn++) r[9] += kd[1 + nn] * ucn[nn];
  }
  if (a.feat) {
#pragma unroll
    for (int v = 0; v < NV; v++) a.feat[v * N + z] = (float)(-r[v]);
  }
  // --- initial guess: P_n (or the given guess), B from the flux-CT update
#pragma unroll
  for (int v = 0; v < NV; v++) {
    double x = a.guess ? __ldg(a.guess + v * N + z) : Pnz[v];
    if (v >= 5 && v <= 7) x = (Un[v] - dts * divF[v]) * isg;
    a.P0[v * N + z] = x;
  }
}

// ---------------------------------------------------------------- floors
// After the Newton solves of a stage, for the zones whose iteration ended
// with a non-zero status (no admissible root found; the Newton kernels floor
// the converged zones themselves): the zone reverts to its start, P_n with
// the flux-CT field B = -kC/kU of its field rows; then rho >= 1e-5 r^{-3/2},
// u >= 1e-7 r^{-5/2} (r = 1 in Minkowski space), and -b^2 <= dP <= b^2/2 on
// the physical anisotropy dP = dP~ (psi c_s^2 P_g)^(1/2).
__global__ void floors_gr(const __grid_constant__ Params p, const double* __restrict__ gc,
                          const double* __restrict__ K, const double* __restrict__ Pn,
                          const uint8_t* __restrict__ status, double* __restrict__ P) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N || status[z] == 0) return;
  const int i = (int)(z % p.n1), j = (int)((z / p.n1) % p.n2);
  const GT g = centre_geo(p, gc, i, j);
  const double r = g(G_R);
  double Pz[NV];
  const bool failed = true;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    if (failed) Pz[v] = (v >= 5 && v <= 7) ? -__ldg(K + (K_C + v) * N + z) / __ldg(K + (K_U + v) * N + z)
                                           : __ldg(Pn + v * N + z);
    else Pz[v] = P[v * N + z];
  }
  Pz[0] = fmax(Pz[0], 1e-5 / (r * sqrt(r)));
  Pz[1] = fmax(Pz[1], 1e-7 / (r * r * sqrt(r)));
  if (p.visc) {
    Met<double> m;
    met_load(m, g);
    const RC<double> c = make_rc<double>(p);
    ZG<double> zz;
    zg_load(zz, Pz, m, c);
    const double f = zz.ds;
    if (f > 0.0) {
      const double dP = Pz[9] * f, hi = 0.5 * zz.bsq, lo = -zz.bsq;
      if (dP > hi) Pz[9] = hi / f;
      else if (dP < lo) Pz[9] = lo / f;
    }
  }
#pragma unroll
  for (int v = 0; v < NV; v++) P[v * N + z] = Pz[v];
}

// ---------------------------------------------------------------- host side
long long gr_geometry_doubles(const Params& p) {
  return (long long)NGC * (p.n1 + 2) * (p.n2 + 2) + (long long)NGF * (p.n1 + 1) * (p.n2 + 2) +
         (long long)NGF * (p.n1 + 2) * (p.n2 + 1);
}
// The explicit-stage scratch: face fluxes of every active direction, the
// derived quantities of the ghost-ring grid, the sources of every zone.
long long gr_face_doubles(const Params& p) {
  long long s = 0;
  for (int d = 0; d < p.dim; d++) s += (long long)NV * face_box(p, d).size;
  // after the faces: the derived and source planes, which the MC slopes of
  // the mixed solver use before them
  const long long ds = (long long)ND * ghost_box(p).size + (long long)NSRC * p.N;
  const long long sl = (long long)NV * ghost_box(p).size;
  return s + (ds > sl ? ds : sl);
}

static void gr_args(const Params& p, const double* geo, double* faces, GrArgs& a) {
  a.gc = geo;
  a.gf[0] = geo + (long long)NGC * (p.n1 + 2) * (p.n2 + 2);
  a.gf[1] = a.gf[0] + (long long)NGF * (p.n1 + 1) * (p.n2 + 2);
  double* f = faces;
  for (int d = 0; d < 3; d++) {
    a.F[d] = f;
    if (d < p.dim) f += (long long)NV * face_box(p, d).size;
  }
  a.Dv = f;
  a.Src = f + (long long)ND * ghost_box(p).size;
  a.Sl = f;  // the derived and source planes are written after the faces
  a.kappa = gr_kappa(p);
  const double cv[5] = {p.gamma, p.gamma - 1.0, sqrt(p.phi * p.gamma), sqrt(p.psi * p.gamma), a.kappa * p.gamma};
  for (int k = 0; k < 5; k++) {
    a.ffc[2 * k] = (float)cv[k];
    a.ffc[2 * k + 1] = (float)(cv[k] - (double)(float)cv[k]);
  }
}

cudaError_t launch_gr_geometry(const Params& p, int metric, double spin, double h, const double x0[3],
                               double* geo, cudaStream_t st) {
  GeoArgs A;
  A.metric = metric;
  A.a = spin;
  A.h = h;
  for (int d = 0; d < 3; d++) { A.x0[d] = x0[d]; A.dx[d] = p.dx[d]; }
  A.tau0 = p.tauR;
  A.n1 = p.n1;
  A.n2 = p.dim >= 2 ? p.n2 : 1;
  A.gc = geo;
  A.gf1 = geo + (long long)NGC * (A.n1 + 2) * (A.n2 + 2);
  A.gf2 = A.gf1 + (long long)NGF * (A.n1 + 1) * (A.n2 + 2);
  const long long n = (long long)(A.n1 + 2) * (A.n2 + 2) + (long long)(A.n1 + 1) * (A.n2 + 2) +
                      (long long)(A.n1 + 2) * (A.n2 + 1);
  geometry_tables<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A);
  return cudaGetLastError();
}

template <typename S, int RECON>
static cudaError_t launch_gr_faces_r(const Params& p, const GrArgs& a, cudaStream_t st) {
  for (int d = 0; d < p.dim; d++) {
    if (RECON == RECON_MC && std::is_same<S, ff>::value) {
      const unsigned ns = (unsigned)((ghost_box(p).size + 127) / 128);
      if (d == 0) mc_slopes_gr<0><<<ns, 128, 0, st>>>(p, a);
      else if (d == 1) mc_slopes_gr<1><<<ns, 128, 0, st>>>(p, a);
      else mc_slopes_gr<2><<<ns, 128, 0, st>>>(p, a);
    }
    const long long n = face_box(p, d).size;
    const unsigned nb = (unsigned)((n + 127) / 128);
    if (d == 0) face_flux_gr<0, S, RECON><<<nb, 128, 0, st>>>(p, a);
    else if (d == 1) face_flux_gr<1, S, RECON><<<nb, 128, 0, st>>>(p, a);
    else face_flux_gr<2, S, RECON><<<nb, 128, 0, st>>>(p, a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template <typename S>
static cudaError_t launch_gr_faces_s(const Params& p, const GrArgs& a, cudaStream_t st) {
  if (p.recon == RECON_WENO5) return launch_gr_faces_r<S, RECON_WENO5>(p, a, st);
  if (p.recon == RECON_PPM) return launch_gr_faces_r<S, RECON_PPM>(p, a, st);
  return launch_gr_faces_r<S, RECON_MC>(p, a, st);
}

// ffstates: face states and fluxes in float-float (the mixed solver).
cudaError_t launch_gr_faces(const Params& p, const double* PE, const double* geo, double* faces, int ffstates,
                            cudaStream_t st) {
  GrArgs a{};
  gr_args(p, geo, faces, a);
  a.PE = PE;
  return ffstates ? launch_gr_faces_s<ff>(p, a, st) : launch_gr_faces_s<double>(p, a, st);
}

long long gr_cache_doubles(long long N) { return (long long)NCACHE_GR * N; }

// mode, cache: the P_n cache of a step (mode 0: none); feat: the learned
// start's increment features (NULL: not wanted); ffslopes: the limited
// slopes of the sources in float-float (the mixed solver).
cudaError_t launch_gr_zone_const(const Params& p, const double* Pn, const double* PE, const double* guess, double dts,
                                 const double* geo, double* faces, double* K, double* P0, double* cache, int mode,
                                 float* feat, int ffslopes, cudaStream_t st) {
  GrArgs a{};
  gr_args(p, geo, faces, a);
  a.Pn = Pn; a.PE = PE; a.guess = guess; a.dts = dts; a.K = K; a.P0 = P0;
  a.idts = 1.0 / dts;
  a.cache = cache;
  a.mode = cache ? mode : 0;
  a.feat = feat;
  derived_gr<<<(unsigned)((ghost_box(p).size + 127) / 128), 128, 0, st>>>(p, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((p.N + 127) / 128);
  if (ffslopes) sources_gr<true><<<nb, 128, 0, st>>>(p, a);
  else sources_gr<false><<<nb, 128, 0, st>>>(p, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  zone_const_gr<<<nb, 128, 0, st>>>(p, a);
  return cudaGetLastError();
}

cudaError_t launch_gr_floors(const Params& p, const double* geo, const double* K, const double* Pn,
                             const uint8_t* status, double* P, cudaStream_t st) {
  floors_gr<<<(unsigned)((p.N + 127) / 128), 128, 0, st>>>(p, geo, K, Pn, status, P);
  return cudaGetLastError();
}

}  // namespace grim
