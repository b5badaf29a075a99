// Learned initial guess for the Newton solve: a small MLP that maps a zone's
// features to the change of its primitives over a stage, P_conv - P_n.
// (The paper starts Newton from P_n; the learned start and its fallback to
// P_n are this library's additions.)
//
// Network: 30 features -> 128 -> 128 -> 128 -> head, SiLU after each hidden
// layer, bfloat16 weights and activations, float32 accumulation and biases,
// on the tensor cores (mma.sync m16n8k16).  The head (80 outputs, 77 used)
// is a 7x10 matrix M and an offset c: the standardised prediction of the
// seven predicted fields is y = M x_U + c, with x_U the ten standardised
// conserved-increment features.  The prediction is therefore exactly linear
// in the (small) increment, with coefficients the network computes from the
// zone's state; this keeps its relative accuracy independent of the time
// step.  Input padded to 32.
//
// Features (float32, 32 per zone): [0..9] the explicit increment of the
// stage at its start, -r_a(P_n), the scaled residual at P_n: for the
// conserved rows this is U* - U(P_n) in the residual's row scaling (U* =
// U(P_n) - dt_s div F), for the q~ and dP~ rows the explicit part of their
// relaxation equations; it carries the information of U* but stays
// resolvable in bfloat16; [10..19] the ten g_{mu nu} (constant in Minkowski
// space); [20..29] P_n; [30..31] zero.  Targets (16 per zone): P_conv - P_n
// for the non-magnetic fields (the magnetic field comes from the explicit
// flux-CT update and is not predicted); other entries zero.  Both are
// standardised with per-feature means and deviations fitted on the training
// set.
//
// Training (Adam) runs on the device: minibatch gather and standardisation,
// forward GEMMs with bias + SiLU epilogues, an MSE loss on the seven
// predicted fields, backward GEMMs, and the update of float32 master weights
// whose bfloat16 copies feed the GEMMs.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>
#include <cuda_bf16.h>

#include "grim_zone.cuh"
#include "../../include/grim.h"

namespace grim {

constexpr int MLP_IN = 32, MLP_H = 128, MLP_Y = 16, MLP_HEAD = 80;
constexpr int MLP_XU = 10;   // features entering the head linearly
constexpr int MLP_NP = 7;    // predicted fields
__host__ __device__ constexpr int mlp_field(int i) { return i < 5 ? i : i + 3; }  // rho u u1 u2 u3 q~ dP~
constexpr int MLP_NLAYER = 4;
// layer l: W_l [n_out][n_in] row-major (PyTorch Linear layout), b_l [n_out]
__host__ __device__ constexpr int mlp_nin(int l) { return l == 0 ? MLP_IN : MLP_H; }
__host__ __device__ constexpr int mlp_nout(int l) { return l == 3 ? MLP_HEAD : MLP_H; }
__host__ __device__ constexpr int mlp_woff(int l) {
  return l == 0 ? 0 : mlp_woff(l - 1) + mlp_nout(l - 1) * mlp_nin(l - 1) + mlp_nout(l - 1);
}
__host__ __device__ constexpr int mlp_boff(int l) { return mlp_woff(l) + mlp_nout(l) * mlp_nin(l); }
constexpr int MLP_NPARAM = mlp_woff(4);
// fields the network predicts (the magnetic ones come from flux-CT)
__host__ __device__ constexpr bool mlp_predicted(int o) { return o < NV && !(o >= 5 && o <= 7); }

}  // namespace grim

struct grim_mlp {
  float* params = nullptr;        // float32 master weights and biases [MLP_NPARAM]
  float* m = nullptr;             // Adam moments
  float* v = nullptr;
  __nv_bfloat16* wb = nullptr;    // bfloat16 copies of W_l (row-major), contiguous by layer
  __nv_bfloat16* wbt = nullptr;   // bfloat16 transposes W_l^T [n_in][n_out]
  float* norm = nullptr;          // x_mean[32], x_std[32], y_mean[16], y_std[16]
  long long adam_t = 0;
  // training scratch for a batch of B rows
  int cap = 0;
  __nv_bfloat16 *xb = nullptr, *xbt = nullptr;          // standardised inputs [B][32], [32][B]
  float* yb = nullptr;                                   // standardised targets [B][16]
  float* xh = nullptr;                                   // standardised head features, float32 [B][16]
  float* z[4] = {nullptr, nullptr, nullptr, nullptr};    // pre-activations [B][n_out]
  __nv_bfloat16* a[3] = {nullptr, nullptr, nullptr};     // SiLU activations [B][128]
  __nv_bfloat16* at[3] = {nullptr, nullptr, nullptr};    // their transposes [128][B]
  __nv_bfloat16 *g = nullptr, *gt = nullptr;             // output-side gradient of a layer [B][n], [n][B]
  float* dA = nullptr;                                   // input-side gradient [B][128]
  float* grad = nullptr;                                 // parameter gradients [MLP_NPARAM]
  float* loss = nullptr;                                 // [1]
};

namespace grim {

// SiLU(x) = x sigmoid(x), with sigmoid(x) = (1 + tanh(x/2))/2 on the
// hardware tanh approximation (one special-function operation).
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigm(float x) { return fmaf(0.5f, tanh_fast(0.5f * x), 0.5f); }
__device__ __forceinline__ float silu(float x) { return x * sigm(x); }
// SiLU(x) from h = x/2: x sigmoid(x) = h (1 + tanh(h)), one FMA after the
// special-function operation (the inference epilogue forms h = acc/2 + b/2
// in one FMA from halved biases).
__device__ __forceinline__ float silu_of_half(float h) { return fmaf(h, tanh_fast(h), h); }
__device__ __forceinline__ float silu_grad(float x) {
  const float s = sigm(x);
  return s * (1.0f + x * (1.0f - s));
}

// ---------------------------------------------------------------- tensor-core GEMM
// C[M][N] (float32, ldc) = A[M][K] * B[N][K]^T, A and B bfloat16 row-major
// with K contiguous (lda, ldb elements); M, N and K multiples of 16 (rows,
// columns and k-chunks past the ends are read as zeros).
// 64x64 output tile per CTA of 4 warps (2x2), each warp 32x32 = 2x4 mma
// tiles of m16n8k16; operands staged through padded shared memory.
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_nt_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                    int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                    float* __restrict__ C, int ldc, int accumulate) {
  __shared__ __align__(16) __nv_bfloat16 sA[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 sB[GBN][GBK + GPAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) acc[i][j][r] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    // stage: 64 rows x 32 bf16 = 64 x 4 chunks of 16 bytes for each operand
    for (int c = tid; c < GBM * 4; c += 128) {
      const int r = c >> 2, q = (c & 3) * 8;
      uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
      const bool kin = k0 + q + 8 <= K;
      if (kin && m0 + r < M) va = *reinterpret_cast<const uint4*>(A + (long long)(m0 + r) * lda + k0 + q);
      if (kin && n0 + r < N) vb = *reinterpret_cast<const uint4*>(B + (long long)(n0 + r) * ldb + k0 + q);
      *reinterpret_cast<uint4*>(&sA[r][q]) = va;
      *reinterpret_cast<uint4*>(&sB[r][q]) = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      unsigned af[2][4], bf[4][2];
      const int ar = lane >> 2, ac = (lane & 3) * 2;
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int r = wm + i * 16 + ar;
        af[i][0] = *reinterpret_cast<const unsigned*>(&sA[r][kk + ac]);
        af[i][1] = *reinterpret_cast<const unsigned*>(&sA[r + 8][kk + ac]);
        af[i][2] = *reinterpret_cast<const unsigned*>(&sA[r][kk + ac + 8]);
        af[i][3] = *reinterpret_cast<const unsigned*>(&sA[r + 8][kk + ac + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int n = wn + j * 8 + ar;
        bf[j][0] = *reinterpret_cast<const unsigned*>(&sB[n][kk + ac]);
        bf[j][1] = *reinterpret_cast<const unsigned*>(&sB[n][kk + ac + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  // store: c0,c1 at (row lane/4, cols 2*(lane%4)+{0,1}); c2,c3 at row + 8
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = m0 + wm + i * 16 + (lane >> 2);
      const int cidx = n0 + wn + j * 8 + (lane & 3) * 2;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int rr = r + h * 8;
        if (rr < M && cidx < N) {
          float* p = C + (long long)rr * ldc + cidx;
          if (accumulate) { p[0] += acc[i][j][2 * h]; p[1] += acc[i][j][2 * h + 1]; }
          else { p[0] = acc[i][j][2 * h]; p[1] = acc[i][j][2 * h + 1]; }
        }
      }
    }
}

static cudaError_t gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                        float* C, int ldc, cudaStream_t st) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  gemm_nt_bf16<<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise kernels
// Minibatch gather with standardisation: rows idx(i) = (off + i * stride) mod M.
__global__ void mlp_gather(const float* __restrict__ X, const float* __restrict__ Y, long long M, long long off,
                           long long stride, int B, const float* __restrict__ norm, __nv_bfloat16* __restrict__ xb,
                           __nv_bfloat16* __restrict__ xbt, float* __restrict__ yb, float* __restrict__ xh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  const long long r = (off + (long long)t * stride) % M;
  for (int f = 0; f < MLP_IN; f++) {
    const float x = (X[r * MLP_IN + f] - norm[f]) / norm[MLP_IN + f];
    const __nv_bfloat16 h = __float2bfloat16(x);
    xb[(long long)t * MLP_IN + f] = h;
    xbt[(long long)f * B + t] = h;
    if (f < MLP_XU) xh[(long long)t * MLP_Y + f] = x;
  }
  for (int o = 0; o < MLP_Y; o++) {
    const float sd = norm[2 * MLP_IN + MLP_Y + o];  // 0: a constant target, predicted as its mean
    yb[(long long)t * MLP_Y + o] = sd > 0.f ? (Y[r * MLP_Y + o] - norm[2 * MLP_IN + o]) / sd : 0.f;
  }
}

// z += b; a = SiLU(z) in bfloat16, row-major and transposed.
__global__ void mlp_bias_silu(float* __restrict__ z, const float* __restrict__ b, int B, int n,
                              __nv_bfloat16* __restrict__ a, __nv_bfloat16* __restrict__ at) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * n) return;
  const int row = (int)(t / n), col = (int)(t % n);
  const float v = z[t] + b[col];
  z[t] = v;
  const __nv_bfloat16 h = __float2bfloat16(silu(v));
  a[t] = h;
  at[(long long)col * B + row] = h;
}

// Head: out = z + b holds M (7x10, row-major) and c (7); the standardised
// prediction of predicted field i is y_i = sum_j M_ij xh_j + c_i.  Loss:
// mean over rows and the 7 fields of (y_i - t_i)^2; dL/dM_ij = e'_i xh_j,
// dL/dc_i = e'_i with e'_i = 2 (y_i - t_i)/(7 B).
__global__ void mlp_head_loss(float* __restrict__ z, const float* __restrict__ b, const float* __restrict__ yb,
                              const float* __restrict__ xh, int B, __nv_bfloat16* __restrict__ g,
                              __nv_bfloat16* __restrict__ gt, float* __restrict__ gy, float* __restrict__ loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (t < B) {
    float d[MLP_HEAD];
#pragma unroll
    for (int o = 0; o < MLP_HEAD; o++) d[o] = 0.f;
    const float* zt = z + (long long)t * MLP_HEAD;
    const float* x = xh + (long long)t * MLP_Y;
#pragma unroll
    for (int i = 0; i < MLP_NP; i++) {
      float y = zt[MLP_NP * MLP_XU + i] + b[MLP_NP * MLP_XU + i];
#pragma unroll
      for (int j = 0; j < MLP_XU; j++) y += (zt[i * MLP_XU + j] + b[i * MLP_XU + j]) * x[j];
      const float e = y - yb[(long long)t * MLP_Y + mlp_field(i)];
      l += e * e;
      const float de = 2.0f * e / (7.0f * (float)B);
#pragma unroll
      for (int j = 0; j < MLP_XU; j++) d[i * MLP_XU + j] = de * x[j];
      d[MLP_NP * MLP_XU + i] = de;
    }
#pragma unroll
    for (int o = 0; o < MLP_HEAD; o++) {
      gy[(long long)t * MLP_HEAD + o] = d[o];
      const __nv_bfloat16 h = __float2bfloat16(d[o]);
      g[(long long)t * MLP_HEAD + o] = h;
      gt[(long long)o * B + t] = h;
    }
    l /= (7.0f * (float)B);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dZ = dA * SiLU'(z) -> bfloat16 row-major and transposed.
__global__ void mlp_silu_back(const float* __restrict__ dA, const float* __restrict__ z, int B, int n,
                              __nv_bfloat16* __restrict__ g, __nv_bfloat16* __restrict__ gt, float* __restrict__ gz) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * n) return;
  const int row = (int)(t / n), col = (int)(t % n);
  const float d = dA[t] * silu_grad(z[t]);
  if (gz) gz[t] = d;
  const __nv_bfloat16 h = __float2bfloat16(d);
  g[t] = h;
  gt[(long long)col * B + row] = h;
}

// Bias gradient: column sums of a float32 [B][n] matrix.
__global__ void mlp_colsum(const float* __restrict__ g, int B, int n, float* __restrict__ out) {
  const int col = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < B; r += blockDim.x) s += g[(long long)r * n + col];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    out[col] = t;
  }
}

// Adam (Kingma & Ba 2015) on the float32 master parameters, then refresh the
// bfloat16 copies and transposes of the weights.
__global__ void mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                         const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                         float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void mlp_refresh_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb,
                                 __nv_bfloat16* __restrict__ wbt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int off = 0, boff = 0;
  for (int l = 0; l < MLP_NLAYER; l++) {
    const int no = mlp_nout(l), ni = mlp_nin(l), n = no * ni;
    if (i < off + n) {
      const int k = i - off, r = k / ni, c = k % ni;
      const __nv_bfloat16 h = __float2bfloat16(p[mlp_woff(l) + k]);
      wb[boff + k] = h;
      wbt[boff + c * no + r] = h;
      return;
    }
    off += n;
    boff += n;
  }
}

// ---------------------------------------------------------------- features
// x_a = -r_a(P_n) from the zone constants K and the P_n quantities.
__device__ __forceinline__ void increment_features(const double* __restrict__ K, long long N, long long z,
                                                   const double P[NV], const double U[NV], double th_n, double ut_n,
                                                   float x[NV]) {
  auto k = [&](int a) { return __ldg(K + a * N + z); };
#pragma unroll
  for (int a = 0; a < 8; a++) x[a] = (float)(-(k(K_U + a) * U[a] + k(K_C + a)));
  const double r8 = k(K_U + 8) * U[8] + k(K_C + 8) + k(K_Q + 0) * P[8] + k(K_Q + 1) * th_n + k(K_Q + 6) * ut_n -
                    k(K_Q + 2) * ut_n + k(K_Q + 3) * P[2] + k(K_Q + 4) * P[3] + k(K_Q + 5) * P[4];
  const double r9 = k(K_U + 9) * U[9] + k(K_C + 9) + k(K_D + 0) * P[9] + k(K_D + 5) * ut_n - k(K_D + 1) * ut_n +
                    k(K_D + 2) * P[2] + k(K_D + 3) * P[3] + k(K_D + 4) * P[4];
  x[8] = (float)(-r8);
  x[9] = (float)(-r9);
}

// Features and targets of the zones of the last explicit stage.
__global__ void mlp_features(const __grid_constant__ Params p, const double* __restrict__ K,
                             const double* __restrict__ Pn, const double* __restrict__ Pc, float* __restrict__ X,
                             float* __restrict__ Y) {
  const long long N = p.N;
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= N) return;
  double P[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) P[v] = __ldg(Pn + v * N + z);
  const RC<double> c = make_rc<double>(p);
  Z<double> zz;
  z_load(zz, P, c);
  double U[NV];
  {
    const double q = zz.qt * zz.qs, dp = zz.dpt * zz.ds, third = dp * (1.0 / 3.0);
    const double A = (zz.w0 + zz.bsq + third) * zz.ut;
    const double qb = q * zz.bht, dpb = dp * zz.bht, qut = q * zz.ut;
    U[0] = zz.rho * zz.ut;
    U[1] = -A * zz.ut + zz.bt * zz.bt - 2.0 * qb * zz.ut + dpb * zz.bht + zz.pg + 0.5 * zz.bsq + third;
#pragma unroll
    for (int k = 0; k < 3; k++) U[2 + k] = A * zz.v[k] - zz.bt * zz.bc[k] + qb * zz.v[k] + qut * zz.bh[k] - dpb * zz.bh[k];
    U[5] = P[5]; U[6] = P[6]; U[7] = P[7];
    U[8] = zz.qt * zz.ut;
    U[9] = zz.dpt * zz.ut;
  }
  float* x = X + z * MLP_IN;
  float xu[NV];
  increment_features(K, N, z, P, U, zz.theta, zz.ut, xu);
#pragma unroll
  for (int a = 0; a < NV; a++) x[a] = xu[a];
  const float g[10] = {-1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f};  // g_tt, g_tx, ..., g_zz (Minkowski)
#pragma unroll
  for (int a = 0; a < 10; a++) x[NV + a] = g[a];
#pragma unroll
  for (int a = 0; a < NV; a++) x[2 * NV + a] = mlp_pn_feature(a, P[a], P[0]);
  x[30] = 0.f;
  x[31] = 0.f;
  if (Y) {
    float* y = Y + z * MLP_Y;
#pragma unroll
    for (int o = 0; o < MLP_Y; o++) y[o] = (o < NV && mlp_predicted(o)) ? mlp_target(o, __ldg(Pc + o * N + z), P[o], P[0]) : 0.f;
  }
}

// Mean and standard deviation per column of a float32 [M][ncol] matrix
// (two passes in double); deviations below 1e-12 are set to 1 (constant
// columns standardise to zero).
__global__ void mlp_colstats(const float* __restrict__ X, long long M, int ncol, double* __restrict__ acc) {
  const int col = blockIdx.y;
  double s = 0.0, s2 = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (long long)gridDim.x * blockDim.x) {
    const double x = X[r * ncol + col];
    s += x;
    s2 += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[2 * col], s);
    atomicAdd(&acc[2 * col + 1], s2);
  }
}

// ---------------------------------------------------------------- fused inference
// One warp runs 16 zones through the network with the activations kept in
// mma fragments: the float32 accumulator of two adjacent n8 tiles of one
// layer is exactly the bfloat16 A fragment of one k16 step of the next.
// Weights live in shared memory (row stride padded by 8 to keep the
// fragment loads conflict-free).  The result replaces the non-magnetic
// components of the Newton initial guess: P0 = P_n + prediction.
constexpr int IW1 = MLP_IN + 8, IWH = MLP_H + 8;
constexpr int INF_WARPS = 12; // warps per block: one block per SM shares one copy of the weights
struct InferSmem {
  __nv_bfloat16 w0[MLP_H][IW1];
  __nv_bfloat16 w1[MLP_H][IWH];
  __nv_bfloat16 w2[MLP_H][IWH];
  __nv_bfloat16 w3[MLP_HEAD][IWH];
  float b[3 * MLP_H + MLP_HEAD];
  float norm[2 * MLP_IN + 2 * MLP_Y];
  __nv_bfloat16 x[INF_WARPS][16][IW1];   // per-warp input tile
  __align__(16) float xh[INF_WARPS][16][12];  // per-warp head features (float32; 10 used)
  __align__(16) float y[INF_WARPS][16][84];   // per-warp head output tile, bias added (80 used)
};

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&h);
}

// B fragments of n-tiles j and j+1 for one k16 step from the row-major
// [n][k] weights in shared memory with one ldmatrix.x4: matrix q (lanes
// 8q..8q+7 give its row addresses) covers n-tile j + q/2, k half q%2, and the
// m8n8 distribution (row lane/4, columns 2(lane%4), +1) is the mma B layout.
__device__ __forceinline__ void ldsm_b2(const __nv_bfloat16* W, int ldw, int j, int ks, int lane, unsigned b[4]) {
  const int q = lane >> 3, r = lane & 7;
  const __nv_bfloat16* row = W + ((j + (q >> 1)) * 8 + r) * ldw + ks * 16 + (q & 1) * 8;
  const unsigned addr = (unsigned)__cvta_generic_to_shared(row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
               : "r"(addr));
}

template <int NOUT_TILES>
__device__ __forceinline__ void layer_mma(float acc[][4], const unsigned (*afr)[4], int ksteps,
                                          const __nv_bfloat16* W, int ldw, int lane) {
  static_assert(NOUT_TILES % 2 == 0, "n-tiles are loaded in pairs");
#pragma unroll
  for (int j = 0; j < NOUT_TILES; j++) {
    acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  }
  for (int ks = 0; ks < ksteps; ks++) {
#pragma unroll
    for (int j = 0; j < NOUT_TILES; j += 2) {
      unsigned b[4];
      ldsm_b2(W, ldw, j, ks, lane, b);
      mma_bf16(acc[j], afr[ks], b);
      mma_bf16(acc[j + 1], afr[ks], b + 2);
    }
  }
}

// SiLU(acc + b) of 16 n8 tiles -> 8 k16 A fragments; hb: the halved biases.
__device__ __forceinline__ void to_afrag(float acc[16][4], const float* hb, unsigned afr[8][4], int lane) {
  const int ac = (lane & 3) * 2;
  auto act = [](float a, float h) { return silu_of_half(fmaf(a, 0.5f, h)); };
#pragma unroll
  for (int ks = 0; ks < 8; ks++) {
    const int c0 = ks * 16 + ac, c1 = c0 + 8;
    const float* lo = acc[2 * ks];
    const float* hi = acc[2 * ks + 1];
    afr[ks][0] = pack_bf16(act(lo[0], hb[c0]), act(lo[1], hb[c0 + 1]));
    afr[ks][1] = pack_bf16(act(lo[2], hb[c0]), act(lo[3], hb[c0 + 1]));
    afr[ks][2] = pack_bf16(act(hi[0], hb[c1]), act(hi[1], hb[c1 + 1]));
    afr[ks][3] = pack_bf16(act(hi[2], hb[c1]), act(hi[3], hb[c1 + 1]));
  }
}

__global__ void __launch_bounds__(INF_WARPS * 32) mlp_guess(const __grid_constant__ Params p,
                                                             const float* __restrict__ feat,
                                                             const double* __restrict__ Pn,
                                                             const __nv_bfloat16* __restrict__ wb,
                                                             const float* __restrict__ params,
                                                             const float* __restrict__ norm, double* __restrict__ P0,
                                                             const double* __restrict__ gc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // weights to shared memory
  constexpr int NT = INF_WARPS * 32;
  for (int i = tid; i < MLP_H * MLP_IN; i += NT) S.w0[i / MLP_IN][i % MLP_IN] = wb[mlp_woff(0) - 0 + i];
  const int o1 = MLP_H * MLP_IN, o2 = o1 + MLP_H * MLP_H, o3 = o2 + MLP_H * MLP_H;
  for (int i = tid; i < MLP_H * MLP_H; i += NT) {
    S.w1[i / MLP_H][i % MLP_H] = wb[o1 + i];
    S.w2[i / MLP_H][i % MLP_H] = wb[o2 + i];
  }
  for (int i = tid; i < MLP_HEAD * MLP_H; i += NT) S.w3[i / MLP_H][i % MLP_H] = wb[o3 + i];
  for (int i = tid; i < MLP_H; i += NT) {  // hidden biases halved for the SiLU epilogue
    S.b[i] = 0.5f * params[mlp_boff(0) + i];
    S.b[MLP_H + i] = 0.5f * params[mlp_boff(1) + i];
    S.b[2 * MLP_H + i] = 0.5f * params[mlp_boff(2) + i];
  }
  if (tid < MLP_HEAD) S.b[3 * MLP_H + tid] = params[mlp_boff(3) + tid];
  // the feature deviations as reciprocals (one multiply a feature below)
  if (tid < 2 * MLP_IN + 2 * MLP_Y)
    S.norm[tid] = (tid >= MLP_IN && tid < 2 * MLP_IN) ? 1.0f / norm[tid] : norm[tid];
  __syncthreads();
  const long long N = p.N;
  const float g[10] = {-1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f};
  // persistent over tiles of 16 zones per warp
  for (long long base = (long long)blockIdx.x * (16 * INF_WARPS); base < N;
       base += (long long)gridDim.x * (16 * INF_WARPS)) {
    // features: lanes 0..15 of each warp build one zone each (the increment
    // features come from the zone-constant kernel of this stage)
    const long long zw = base + warp * 16;
    double Pkeep[MLP_NP];
    if (lane < 16) {
      const long long z = zw + lane;
      float xf[MLP_IN];
      if (z < N) {
#pragma unroll
        for (int a = 0; a < NV; a++) xf[a] = __ldg(feat + a * N + z);
        if (gc) {  // the zone's g_{mu nu} from the centre table of a general metric
          const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
          const int zi = (int)(z % p.n1), zj = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
          const double* gz = gc + (long long)(zj + 1) * (p.n1 + 2) + (zi + 1);
#pragma unroll
          for (int a = 0; a < 10; a++) xf[NV + a] = (float)__ldg(gz + a * nc);
        } else {
#pragma unroll
          for (int a = 0; a < 10; a++) xf[NV + a] = g[a];
        }
        const double rho_n = __ldg(Pn + z);
#pragma unroll
        for (int a = 0; a < NV; a++) {
          const double x = __ldg(Pn + a * N + z);
          xf[2 * NV + a] = mlp_pn_feature(a, x, rho_n);
          if (a < 5) Pkeep[a] = x;
          else if (a >= 8) Pkeep[a - 3] = x;
        }
        xf[30] = xf[31] = 0.f;
      } else {
#pragma unroll
        for (int a = 0; a < MLP_IN; a++) xf[a] = S.norm[a];
      }
#pragma unroll
      for (int a = 0; a < MLP_IN; a++) {
        const float xs = (xf[a] - S.norm[a]) * S.norm[MLP_IN + a];
        S.x[warp][lane][a] = __float2bfloat16(xs);
        if (a < MLP_XU) S.xh[warp][lane][a] = xs;
      }
    }
    __syncwarp();
    // layer 0: 16 x 32 input, two k16 steps
    unsigned a0[2][4];
    {
      const int ar = lane >> 2, ac = (lane & 3) * 2;
#pragma unroll
      for (int ks = 0; ks < 2; ks++) {
        a0[ks][0] = *reinterpret_cast<const unsigned*>(&S.x[warp][ar][ks * 16 + ac]);
        a0[ks][1] = *reinterpret_cast<const unsigned*>(&S.x[warp][ar + 8][ks * 16 + ac]);
        a0[ks][2] = *reinterpret_cast<const unsigned*>(&S.x[warp][ar][ks * 16 + ac + 8]);
        a0[ks][3] = *reinterpret_cast<const unsigned*>(&S.x[warp][ar + 8][ks * 16 + ac + 8]);
      }
    }
    float acc[16][4];
    unsigned afr[8][4];
    layer_mma<16>(acc, a0, 2, &S.w0[0][0], IW1, lane);
    to_afrag(acc, S.b, afr, lane);
    layer_mma<16>(acc, afr, 8, &S.w1[0][0], IWH, lane);
    to_afrag(acc, S.b + MLP_H, afr, lane);
    layer_mma<16>(acc, afr, 8, &S.w2[0][0], IWH, lane);
    to_afrag(acc, S.b + 2 * MLP_H, afr, lane);
    constexpr int NT = MLP_HEAD / 8;
    float out[NT][4];
    layer_mma<NT>(out, afr, 8, &S.w3[0][0], IWH, lane);
    {
      const int ar = lane >> 2, ac = (lane & 3) * 2;
      const float* hb = S.b + 3 * MLP_H;
#pragma unroll
      for (int j = 0; j < NT; j++) {
        const float b0 = hb[j * 8 + ac], b1 = hb[j * 8 + ac + 1];
        S.y[warp][ar][j * 8 + ac] = out[j][0] + b0;
        S.y[warp][ar][j * 8 + ac + 1] = out[j][1] + b1;
        S.y[warp][ar + 8][j * 8 + ac] = out[j][2] + b0;
        S.y[warp][ar + 8][j * 8 + ac + 1] = out[j][3] + b1;
      }
    }
    __syncwarp();
    // head: y_i = sum_j M_ij x_j + c_i, one zone per lane
    if (lane < 16) {
      const long long z = zw + lane;
      if (z < N) {
        float yo[80], x[12];
        const float4* yv = reinterpret_cast<const float4*>(S.y[warp][lane]);
        const float4* xv = reinterpret_cast<const float4*>(S.xh[warp][lane]);
#pragma unroll
        for (int q = 0; q < 20; q++) {
          const float4 t = yv[q];
          yo[4 * q] = t.x; yo[4 * q + 1] = t.y; yo[4 * q + 2] = t.z; yo[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int q = 0; q < 3; q++) {
          const float4 t = xv[q];
          x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int i = 0; i < MLP_NP; i++) {
          float yi = yo[MLP_NP * MLP_XU + i];
#pragma unroll
          for (int j = 0; j < MLP_XU; j++) yi = fmaf(yo[i * MLP_XU + j], x[j], yi);
          const int f = mlp_field(i);
          const double d = (double)(yi * S.norm[2 * MLP_IN + MLP_Y + f] + S.norm[2 * MLP_IN + f]);
          P0[f * N + z] = mlp_apply(f, Pkeep[i], d, Pkeep[0]);
        }
      }
    }
    __syncwarp();
  }
}

// Kaiming-uniform initialisation with a counter-based hash (splitmix64),
// biases zero.
__global__ void mlp_init_params(float* p, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  for (int l = 0; l < MLP_NLAYER; l++) {
    const int wo = mlp_woff(l), bo = mlp_boff(l), ni = mlp_nin(l), no = mlp_nout(l);
    if (i >= wo && i < bo) {
      unsigned long long s = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
      s = (s ^ (s >> 30)) * 0xbf58476d1ce4e5b9ull;
      s = (s ^ (s >> 27)) * 0x94d049bb133111ebull;
      s ^= s >> 31;
      const float u = (float)((s >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
      const int r = (i - wo) / ni;
      // the padded output rows of the last layer start (and are kept) at zero
      p[i] = (l == 3 && r >= MLP_NP * (MLP_XU + 1)) ? 0.f : u * sqrtf(6.f / (float)ni);
      return;
    }
    if (i >= bo && i < bo + no) { p[i] = 0.f; return; }
  }
}

}  // namespace grim

using namespace grim;

static int mlp_alloc_batch(grim_mlp* m, int B) {
  if (m->cap >= B) return GRIM_OK;
  auto F = [](void* p) { cudaFree(p); };
  F(m->xb); F(m->xbt); F(m->yb); F(m->xh); F(m->g); F(m->gt); F(m->dA);
  for (int l = 0; l < 4; l++) F(m->z[l]);
  for (int l = 0; l < 3; l++) { F(m->a[l]); F(m->at[l]); }
  size_t b = B;
  bool ok = cudaMalloc(&m->xb, 2 * b * MLP_IN) == cudaSuccess && cudaMalloc(&m->xbt, 2 * b * MLP_IN) == cudaSuccess &&
            cudaMalloc(&m->yb, 4 * b * MLP_Y) == cudaSuccess && cudaMalloc(&m->xh, 4 * b * MLP_Y) == cudaSuccess &&
            cudaMalloc(&m->g, 2 * b * MLP_H) == cudaSuccess &&
            cudaMalloc(&m->gt, 2 * b * MLP_H) == cudaSuccess && cudaMalloc(&m->dA, 4 * b * MLP_H) == cudaSuccess;
  for (int l = 0; l < 4 && ok; l++) ok = cudaMalloc(&m->z[l], 4 * b * MLP_H) == cudaSuccess;
  for (int l = 0; l < 3 && ok; l++)
    ok = cudaMalloc(&m->a[l], 2 * b * MLP_H) == cudaSuccess && cudaMalloc(&m->at[l], 2 * b * MLP_H) == cudaSuccess;
  if (!ok) return GRIM_ENOMEM;
  m->cap = B;
  return GRIM_OK;
}

// One forward + backward pass over the gathered batch; leaves the parameter
// gradient in m->grad and adds the batch loss to *m->loss.
static cudaError_t mlp_forward_backward(grim_mlp* m, int B, cudaStream_t st) {
  cudaError_t e;
  const int T = 256;
  // forward
  const __nv_bfloat16* in = m->xb;
  int nin = MLP_IN;
  int wboff = 0;
  int wboffs[4];
  for (int l = 0; l < 4; l++) {
    wboffs[l] = wboff;
    const int no = mlp_nout(l);
    if ((e = gemm(B, no, nin, in, nin, m->wb + wboff, nin, m->z[l], no, st)) != cudaSuccess) return e;
    if (l < 3) {
      mlp_bias_silu<<<(unsigned)(((long long)B * no + T - 1) / T), T, 0, st>>>(m->z[l], m->params + mlp_boff(l), B, no,
                                                                              m->a[l], m->at[l]);
      in = m->a[l];
      nin = no;
    }
    wboff += no * mlp_nin(l);
  }
  // loss and dL/d(head) -> g (bf16 [B][80]), gt ([80][B]), dA (float [B][80])
  mlp_head_loss<<<(B + T - 1) / T, T, 0, st>>>(m->z[3], m->params + mlp_boff(3), m->yb, m->xh, B, m->g, m->gt, m->dA,
                                               m->loss);
  // backward
  for (int l = 3; l >= 0; l--) {
    const int no = mlp_nout(l), ni = mlp_nin(l);
    // dW_l [no][ni] = g^T [no][B] x a_{l-1} [B][ni]  ->  A = gt (K = B contiguous), B-operand = a_{l-1}^T [ni][B]
    const __nv_bfloat16* actT = (l == 0) ? m->xbt : m->at[l - 1];
    if ((e = gemm(no, ni, B, m->gt, B, actT, B, m->grad + mlp_woff(l), ni, st)) != cudaSuccess) return e;
    // db_l = column sums of the output-side gradient (float copy in dA)
    mlp_colsum<<<no, 256, 0, st>>>(m->dA, B, no, m->grad + mlp_boff(l));
    if (l == 0) break;
    // dA_{l-1} [B][ni] = g [B][no] x W_l [no][ni]  ->  B-operand = W_l^T [ni][no];
    // dA is reused: the bias gradient above has consumed it in stream order
    if ((e = gemm(B, ni, no, m->g, no, m->wbt + wboffs[l], no, m->dA, ni, st)) != cudaSuccess) return e;
    // dZ_{l-1} = dA * SiLU'(z_{l-1}) -> g, gt, and its float copy back into dA
    mlp_silu_back<<<(unsigned)(((long long)B * ni + T - 1) / T), T, 0, st>>>(m->dA, m->z[l - 1], B, ni, m->g, m->gt,
                                                                            m->dA);
  }
  return cudaGetLastError();
}

extern "C" {

int grim_mlp_create(unsigned long long seed, grim_mlp** out) {
  if (!out) return GRIM_EINVAL;
  *out = nullptr;
  grim_mlp* m = new grim_mlp();
  const size_t np = MLP_NPARAM;
  int nw = 0;
  for (int l = 0; l < 4; l++) nw += mlp_nout(l) * mlp_nin(l);
  bool ok = cudaMalloc(&m->params, 4 * np) == cudaSuccess && cudaMalloc(&m->m, 4 * np) == cudaSuccess &&
            cudaMalloc(&m->v, 4 * np) == cudaSuccess && cudaMalloc(&m->grad, 4 * np) == cudaSuccess &&
            cudaMalloc(&m->wb, 2 * nw) == cudaSuccess && cudaMalloc(&m->wbt, 2 * nw) == cudaSuccess &&
            cudaMalloc(&m->norm, 4 * (2 * MLP_IN + 2 * MLP_Y)) == cudaSuccess &&
            cudaMalloc(&m->loss, 4) == cudaSuccess;
  if (!ok) {
    grim_mlp_destroy(m);
    return GRIM_ENOMEM;
  }
  cudaMemset(m->m, 0, 4 * np);
  cudaMemset(m->v, 0, 4 * np);
  std::vector<float> nrm(2 * MLP_IN + 2 * MLP_Y, 0.f);
  for (int i = 0; i < MLP_IN; i++) nrm[MLP_IN + i] = 1.f;
  for (int i = 0; i < MLP_Y; i++) nrm[2 * MLP_IN + MLP_Y + i] = 1.f;
  cudaMemcpy(m->norm, nrm.data(), 4 * nrm.size(), cudaMemcpyHostToDevice);
  mlp_init_params<<<(MLP_NPARAM + 255) / 256, 256>>>(m->params, seed);
  mlp_refresh_bf16<<<(nw + 255) / 256, 256>>>(m->params, m->wb, m->wbt);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    grim_mlp_destroy(m);
    return GRIM_ECUDA;
  }
  *out = m;
  return GRIM_OK;
}

void grim_mlp_destroy(grim_mlp* m) {
  if (!m) return;
  void* ps[] = {m->params, m->m, m->v, m->wb, m->wbt, m->norm, m->xb, m->xbt, m->yb, m->xh, m->g, m->gt, m->dA, m->grad,
                m->loss, m->z[0], m->z[1], m->z[2], m->z[3], m->a[0], m->a[1], m->a[2], m->at[0], m->at[1], m->at[2]};
  for (void* p : ps) cudaFree(p);
  delete m;
}

int grim_mlp_param_count() { return MLP_NPARAM; }

int grim_mlp_get_params(grim_mlp* m, float* host, float* norm_host) {
  if (!m) return GRIM_EINVAL;
  if (host && cudaMemcpy(host, m->params, 4 * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess) return GRIM_ECUDA;
  if (norm_host &&
      cudaMemcpy(norm_host, m->norm, 4 * (2 * MLP_IN + 2 * MLP_Y), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GRIM_ECUDA;
  return GRIM_OK;
}

int grim_mlp_set_params(grim_mlp* m, const float* host, const float* norm_host) {
  if (!m) return GRIM_EINVAL;
  if (host && cudaMemcpy(m->params, host, 4 * MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return GRIM_ECUDA;
  if (norm_host &&
      cudaMemcpy(m->norm, norm_host, 4 * (2 * MLP_IN + 2 * MLP_Y), cudaMemcpyHostToDevice) != cudaSuccess)
    return GRIM_ECUDA;
  int nw = 0;
  for (int l = 0; l < 4; l++) nw += mlp_nout(l) * mlp_nin(l);
  mlp_refresh_bf16<<<(nw + 255) / 256, 256>>>(m->params, m->wb, m->wbt);
  cudaMemset(m->m, 0, 4 * MLP_NPARAM);
  cudaMemset(m->v, 0, 4 * MLP_NPARAM);
  m->adam_t = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? GRIM_OK : GRIM_ECUDA;
}

int grim_mlp_fit_norm(grim_mlp* m, const float* X, const float* Y, long long M) {
  if (!m || !X || !Y || M < 2) return GRIM_EINVAL;
  double* acc = nullptr;
  if (cudaMalloc(&acc, sizeof(double) * 2 * (MLP_IN + MLP_Y)) != cudaSuccess) return GRIM_ENOMEM;
  cudaMemset(acc, 0, sizeof(double) * 2 * (MLP_IN + MLP_Y));
  mlp_colstats<<<dim3(256, MLP_IN), 256>>>(X, M, MLP_IN, acc);
  mlp_colstats<<<dim3(256, MLP_Y), 256>>>(Y, M, MLP_Y, acc + 2 * MLP_IN);
  std::vector<double> h(2 * (MLP_IN + MLP_Y));
  cudaError_t e = cudaMemcpy(h.data(), acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost);
  cudaFree(acc);
  if (e != cudaSuccess) return GRIM_ECUDA;
  std::vector<float> nrm(2 * MLP_IN + 2 * MLP_Y);
  for (int c = 0; c < MLP_IN + MLP_Y; c++) {
    const double mean = h[2 * c] / M;
    double var = h[2 * c + 1] / M - mean * mean;
    double sd = var > 0 ? std::sqrt(var) : 0.0;
    // a constant feature standardises to 0; a constant target (a field the
    // workload never changes, e.g. u^3 in a 2-D box) is predicted as its mean
    if (sd < 1e-12 * (1.0 + std::fabs(mean))) sd = c < MLP_IN ? 1.0 : 0.0;
    if (c < MLP_IN) { nrm[c] = (float)mean; nrm[MLP_IN + c] = (float)sd; }
    else { const int o = c - MLP_IN; nrm[2 * MLP_IN + o] = (float)mean; nrm[2 * MLP_IN + MLP_Y + o] = (float)sd; }
  }
  return cudaMemcpy(m->norm, nrm.data(), 4 * nrm.size(), cudaMemcpyHostToDevice) == cudaSuccess ? GRIM_OK
                                                                                                : GRIM_ECUDA;
}

int grim_mlp_train(grim_mlp* m, const float* X, const float* Y, long long M, int batch, int steps, double lr,
                   unsigned long long seed, double* mean_loss) {
  if (!m || !X || !Y || M < 1 || batch < 16 || batch % 64 || steps < 0) return GRIM_EINVAL;
  int rc = mlp_alloc_batch(m, batch);
  if (rc) return rc;
  // row permutation: r_i = (off + i * stride) mod M with stride coprime to M
  long long stride = (long long)(0.6180339887498949 * M) | 1;
  auto gcd = [](long long a, long long b) { while (b) { long long t = a % b; a = b; b = t; } return a; };
  while (gcd(stride, M) != 1) stride += 2;
  cudaMemset(m->loss, 0, 4);
  int nw = 0;
  for (int l = 0; l < 4; l++) nw += mlp_nout(l) * mlp_nin(l);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  long long off = (long long)(seed % (unsigned long long)M);
  for (int s = 0; s < steps; s++) {
    mlp_gather<<<(batch + 255) / 256, 256>>>(X, Y, M, off, stride, batch, m->norm, m->xb, m->xbt, m->yb, m->xh);
    off = (off + (long long)batch * stride) % M;
    cudaError_t e = mlp_forward_backward(m, batch, 0);
    if (e != cudaSuccess) return GRIM_ECUDA;
    m->adam_t++;
    const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
    mlp_adam<<<(MLP_NPARAM + 255) / 256, 256>>>(m->params, m->m, m->v, m->grad, MLP_NPARAM, (float)lr, b1, b2, eps, c1,
                                                c2);
    mlp_refresh_bf16<<<(nw + 255) / 256, 256>>>(m->params, m->wb, m->wbt);
  }
  float l = 0.f;
  if (cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GRIM_ECUDA;
  if (mean_loss) *mean_loss = steps ? (double)l / steps : 0.0;
  return GRIM_OK;
}

int grim_mlp_gradient(grim_mlp* m, const float* X, const float* Y, long long M, float* grad_host, double* loss) {
  if (!m || !X || !Y || M < 64 || M % 64 || !grad_host) return GRIM_EINVAL;
  const int B = (int)M;
  int rc = mlp_alloc_batch(m, B);
  if (rc) return rc;
  cudaMemset(m->loss, 0, 4);
  mlp_gather<<<(B + 255) / 256, 256>>>(X, Y, M, 0, 1, B, m->norm, m->xb, m->xbt, m->yb, m->xh);
  if (mlp_forward_backward(m, B, 0) != cudaSuccess) return GRIM_ECUDA;
  float l = 0.f;
  if (cudaMemcpy(grad_host, m->grad, 4 * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return GRIM_ECUDA;
  if (loss) *loss = l;
  return GRIM_OK;
}

}  // extern "C"

namespace grim {
cudaError_t launch_mlp_features(const Params& p, const double* K, const double* Pn, const double* Pc, float* X,
                                float* Y, cudaStream_t st) {
  mlp_features<<<(unsigned)((p.N + 127) / 128), 128, 0, st>>>(p, K, Pn, Pc, X, Y);
  return cudaGetLastError();
}

// gc: the centre geometry table of a general metric (its first ten planes
// are g_{mu nu}), or NULL for Minkowski space.
cudaError_t launch_mlp_guess(const Params& p, const float* feat, const double* Pn, const grim_mlp* m, double* P0,
                             const double* gc, cudaStream_t st) {
  static PerDevice once;
  int sms = 0;
  cudaError_t e = once.get(
      [](int* v) {
        cudaError_t r = cudaFuncSetAttribute(mlp_guess, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(InferSmem));
        int dev = 0;
        if (r == cudaSuccess) r = cudaGetDevice(&dev);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        return r;
      },
      &sms);
  if (e != cudaSuccess) return e;
  long long tiles = (p.N + 16 * INF_WARPS - 1) / (16 * INF_WARPS);
  long long grid = sms;  // persistent: one block (and one copy of the weights) per SM
  if (grid > tiles) grid = tiles;
  mlp_guess<<<(unsigned)grid, INF_WARPS * 32, sizeof(InferSmem), st>>>(p, feat, Pn, m->wb, m->params, m->norm, P0,
                                                                        gc);
  return cudaGetLastError();
}
}  // namespace grim
