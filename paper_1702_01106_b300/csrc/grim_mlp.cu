// Learned initial guess for the Newton solve: a small MLP that maps a zone's
// features to the change of its primitives over a stage, P_conv - P_n.
// (The paper starts Newton from P_n; the learned start and its fallback to
// P_n are this library's additions.)
//
// Network: 30 features -> 128 -> 128 -> 128 -> head, SiLU after each hidden
// layer, bfloat16 weights and activations, float32 accumulation and biases,
// on the tensor cores (inference: tcgen05 with TMEM accumulators; training
// GEMMs: mma.sync m16n8k16).  The head (80 outputs, 77 used)
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
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>

#include "grim_tc.cuh"
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
  float* ws = nullptr;                                   // split-K partial tiles, partial bias sums
  unsigned long long* stalls = nullptr;                  // training GEMM CTAs that gave up waiting
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

// ---------------------------------------------------------------- tensor-core GEMM (training)
// C[M][N] (float32, ldc) = A[M][K] B[N][K]^T, A and B bfloat16 row-major
// with K contiguous (lda, ldb elements).  One CTA of 128 threads per tile
// of 128 rows x bn columns (bn <= 128, a multiple of 16): thread 0 has TMA
// copy K-chunks of 64 columns of both operands into a four-stage ring in
// shared memory and issues the tcgen05 MMAs (K = 16 each) that accumulate
// the tile in float32 in 128 TMEM columns; then each warp reads its 32 TMEM
// lanes (rows) back and stores them.  Rows, columns and K past the ends
// arrive as zeros (the tensor maps' out-of-bounds fill).  A split along K
// (blockIdx.z) stores its partial tile into its own slice of a workspace,
// and gemm_splitk_sum adds the slices in a fixed order, so that results do
// not depend on timing.
//
// An operand tile of R rows x 64 columns in shared memory: the eight groups
// of 8 columns one after another, each R rows x 16 bytes (what one TMA box
// of 8 x R elements writes), so element (r, k) lies at byte
//   (k / 8) * R * 16 + r * 16 + (k % 8) * 2,
// the no-swizzle K-major layout with LBO = R * 16 (core matrices adjacent
// along K) and SBO = 128 (8-row groups).
constexpr int GT_BM = 128, GT_BK = 64, GT_STAGES = 4, GT_THREADS = 128, GT_COLS = 128;
constexpr int GT_A_BYTES = GT_BM * GT_BK * 2;   // 16 KB; B takes at most as much
constexpr int GT_STAGE_BYTES = 2 * GT_A_BYTES;
constexpr int GT_SMEM = GT_STAGES * GT_STAGE_BYTES + 1024 + 128;  // ring, alignment slack, barriers
constexpr uint32_t GT_WAIT_LIMIT = 1u << 22;  // mbarrier polls before the kernel gives up
constexpr int GT_MAX_SPLITS = 16;
constexpr long long GT_WS_FLOATS = (long long)GT_MAX_SPLITS * 128 * 128;

__global__ void __launch_bounds__(GT_THREADS, 1)
    gemm_nt_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                 int bn, int chunks_per_split, float* __restrict__ C, int ldc, long long split_stride,
                 unsigned long long* __restrict__ stalls) {
  extern __shared__ unsigned char gsm_raw[];
  // the TMA destinations want 128-byte alignment: round the base up to 1 KB
  unsigned char* gsm = gsm_raw + ((1024u - (tc::smem_addr(gsm_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(gsm + GT_STAGES * GT_STAGE_BYTES);
  uint64_t* empty = full + GT_STAGES;
  uint64_t* done = empty + GT_STAGES;
  uint32_t* taddr = reinterpret_cast<uint32_t*>(done + 1);
  int* abort = reinterpret_cast<int*>(taddr + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GT_BM, n0 = blockIdx.x * bn;
  const int nchunks = (K + GT_BK - 1) / GT_BK;
  const int c0 = blockIdx.z * chunks_per_split;
  const int nc = min(c0 + chunks_per_split, nchunks) - c0;  // >= 1 by the launcher's choice of splits
  if (tid == 0) {
    for (int s = 0; s < GT_STAGES; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    *abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(taddr, GT_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *taddr;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(GT_BM, bn);
    const uint32_t a_lbo = GT_BM * 16, b_lbo = bn * 16;
    const uint32_t tx = (uint32_t)(GT_BK * 2) * (uint32_t)(GT_BM + bn);  // bytes of one chunk of A and B
    int issued = 0, used = 0;
    bool ok = true;
    auto load = [&](int i) {
      const int s = i % GT_STAGES;
      unsigned char* sa = gsm + s * GT_STAGE_BYTES;
      unsigned char* sb = sa + GT_A_BYTES;
      tc::mbar_arrive_expect_tx(&full[s], tx);
      const int k = (c0 + i) * GT_BK;
#pragma unroll
      for (int j = 0; j < GT_BK / 8; j++) {
        tc::tma_load_2d(sa + j * a_lbo, &ta, k + 8 * j, m0, &full[s]);
        tc::tma_load_2d(sb + j * b_lbo, &tb, k + 8 * j, n0, &full[s]);
      }
    };
    for (; issued < nc && issued < GT_STAGES; issued++) load(issued);
    for (; used < nc; used++) {
      const int s = used % GT_STAGES;
      const uint32_t ph = (uint32_t)(used / GT_STAGES) & 1u;
      if (!tc::mbar_wait(&full[s], ph, GT_WAIT_LIMIT)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_addr(gsm + s * GT_STAGE_BYTES), sb = sa + GT_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < GT_BK / 16; kk++)
        tc::mma_bf16(tm, tc::smem_desc(sa + 2 * kk * a_lbo, a_lbo, 128), tc::smem_desc(sb + 2 * kk * b_lbo, b_lbo, 128),
                     idesc, (uint32_t)(used | kk));
      tc::commit(&empty[s]);
      if (issued < nc) {
        // refill the stage once the MMAs that read it have completed
        if (!tc::mbar_wait(&empty[s], ph, GT_WAIT_LIMIT)) {
          ok = false;
          used++;
          break;
        }
        load(issued++);
      }
    }
    tc::commit(done);  // one arrival when every MMA issued above has completed
    if (!ok) {
      // the copies still in flight land before the kernel gives up
      for (int i = used; i < issued; i++)
        tc::mbar_wait(&full[i % GT_STAGES], (uint32_t)(i / GT_STAGES) & 1u, GT_WAIT_LIMIT);
      *abort = 1;
    }
  }
  __syncwarp();
  if (!tc::mbar_wait(done, 0, GT_WAIT_LIMIT)) *abort = 1;
  __syncthreads();
  if (*abort == 0) {
    tc::fence_after_sync();
    const int row = m0 + warp * 32 + lane;
    float* out = C + blockIdx.z * split_stride + (long long)row * ldc + n0;
    for (int c = 0; c < bn; c += 16) {
      float v[16];
      tc::ld_x16(tm + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (row < M && n0 + c < N) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(out + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  } else if (tid == 0) {
    atomicAdd(stalls, 1ull);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, GT_COLS);
}

// C[r][c] = sum over the splits z, in order, of the partial tiles ws[z][r][c].
__global__ void gemm_splitk_sum(const float* __restrict__ ws, int splits, long long slice, int M, int N,
                                float* __restrict__ C, int ldc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)M * N) return;
  float s = 0.f;
  for (int z = 0; z < splits; z++) s += ws[z * slice + i];
  C[(i / N) * ldc + i % N] = s;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of a bfloat16 matrix [rows][K] with row stride ld elements,
// copied in boxes of 8 columns x box_rows rows, zeros outside.
static bool tmap_kmajor(CUtensorMap* t, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows) {
  const EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)ld * 2u};
  const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  return f(t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dim, stride, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches C = A B^T (see gemm_nt_bf16).  Requirements, checked here:
// N a multiple of 16; lda, ldb multiples of 8 and >= K (16-byte TMA
// strides); ldc a multiple of 4 and >= N; A, B, C 16-byte aligned.
// splits: the number of K-splits, or 0 to choose (only when K spans at
// least 8 chunks of 64 and the tiles leave SMs idle; needs ws of
// splits * M * N floats, else no split).  stalls: device counter raised when
// a CTA gave up waiting for its copies or MMAs.
static cudaError_t gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                        float* C, int ldc, float* ws, long long ws_floats, unsigned long long* stalls,
                        cudaStream_t st, int splits = 0) {
  auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  if (M < 1 || N < 16 || K < 1 || N % 16 || lda % 8 || ldb % 8 || lda < K || ldb < K || ldc % 4 || ldc < N ||
      misaligned(A) || misaligned(B) || misaligned(C) || splits < 0 || !stalls)
    return cudaErrorInvalidValue;
  static PerDevice once;
  int sms = 0;
  cudaError_t e = once.get(
      [](int* v) {
        cudaError_t r = cudaFuncSetAttribute(gemm_nt_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        int dev = 0;
        if (r == cudaSuccess) r = cudaGetDevice(&dev);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        return r;
      },
      &sms);
  if (e != cudaSuccess) return e;
  const int bn = N < 128 ? N : 128;
  const int gx = (N + bn - 1) / bn, gy = (M + GT_BM - 1) / GT_BM;
  const int nchunks = (K + GT_BK - 1) / GT_BK;
  int s = splits;
  if (s == 0) {
    s = 1;
    const int idle = sms / (gx * gy);
    if (nchunks >= 8 && idle > 1) s = std::min(std::min(GT_MAX_SPLITS, nchunks / 4), idle);
  }
  s = std::min(s, nchunks);
  const int cps = (nchunks + s - 1) / s;
  s = (nchunks + cps - 1) / cps;  // every split gets at least one chunk
  const long long slice = (long long)M * N;
  if (s > 1 && (!ws || misaligned(ws) || (long long)s * slice > ws_floats)) {
    if (splits) return cudaErrorInvalidValue;
    s = 1;
  }
  const int cps_final = (nchunks + s - 1) / s;
  CUtensorMap ta, tb;
  if (!tmap_kmajor(&ta, A, M, K, lda, GT_BM) || !tmap_kmajor(&tb, B, N, K, ldb, bn)) return cudaErrorInvalidValue;
  const dim3 grid(gx, gy, s);
  if (s == 1) {
    gemm_nt_bf16<<<grid, GT_THREADS, GT_SMEM, st>>>(ta, tb, M, N, K, bn, cps_final, C, ldc, 0, stalls);
    return cudaGetLastError();
  }
  gemm_nt_bf16<<<grid, GT_THREADS, GT_SMEM, st>>>(ta, tb, M, N, K, bn, cps_final, ws, N, slice, stalls);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gemm_splitk_sum<<<(unsigned)((slice + 255) / 256), 256, 0, st>>>(ws, s, slice, M, N, C, ldc);
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
// Column sums of a float matrix g [B][n] (the bias gradient) in two passes
// with coalesced reads: mlp_colsum_part sums slice s of MLP_CS_SLICES row
// slices for 32 columns per block (threads (c, r): rows r, r + 8, ...),
// mlp_colsum_final adds the slices in order, so the sum is reproducible.
constexpr int MLP_CS_SLICES = 32;
__global__ void mlp_colsum_part(const float* __restrict__ g, int B, int n, float* __restrict__ part) {
  __shared__ float acc[8][33];
  const int c = threadIdx.x, r = threadIdx.y, col = blockIdx.x * 32 + c, sl = blockIdx.y;
  const int rows = (B + MLP_CS_SLICES - 1) / MLP_CS_SLICES;
  const int r0 = sl * rows, r1 = min(B, r0 + rows);
  float s = 0.f;
  if (col < n)
    for (int i = r0 + r; i < r1; i += 8) s += g[(long long)i * n + col];
  acc[r][c] = s;
  __syncthreads();
  if (r == 0 && col < n) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) t += acc[k][c];
    part[(long long)sl * n + col] = t;
  }
}
__global__ void mlp_colsum_final(const float* __restrict__ part, int n, float* __restrict__ out) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  float t = 0.f;
  for (int sl = 0; sl < MLP_CS_SLICES; sl++) t += part[(long long)sl * n + col];
  out[col] = t;
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
// The learned start on the fifth-generation tensor cores (tcgen05): one
// persistent CTA per SM keeps the bfloat16 weights in shared memory and runs
// tiles of 128 zones through the network in four independent streams of
// tiles, one per warpgroup, each with its own activation buffer, mbarrier
// and 128 TMEM columns, so that the epilogues of some streams overlap the
// MMAs and the global loads of the others.  Each layer is a 128 x N x K
// product issued by one thread as K/16 tcgen05.mma instructions (A: the
// tile's activations, B: the layer's weights, both in shared memory; D:
// float32 in tensor memory, one TMEM lane per zone); its completion arrives
// on the stream's mbarrier.  The epilogue reads each zone's row back from
// TMEM (tcgen05.ld: warp w of a warpgroup reads lanes 32 (w % 4) ..), adds
// the bias, applies SiLU and writes the bfloat16 activations over the
// layer's own A operand (complete by then).  The thread of a TMEM lane is
// the thread of that zone throughout, so the head's ten float32 inputs
// x_U stay in its registers.  The head's 80 outputs give y = M x_U + c per
// zone, and the start P_n + y (in the learned start's units) replaces the
// non-magnetic components of the Newton start P0.
constexpr int TC_ROWS = 128;      // zones per tile: the MMA's M and the TMEM lanes
constexpr int TC_STREAMS = 4;     // warpgroups, each with its own stream of tiles
constexpr int TC_THREADS = 128 * TC_STREAMS;
constexpr uint32_t TC_COLS = 128; // TMEM columns of one warpgroup's accumulator
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;  // mbarrier polls before the kernel gives up

// What one warpgroup's tile stream owns: the activations of its tile, in
// the core-matrix K-major layout.  The standardised features (the first
// layer's A operand, 128 x 32) occupy the start of the same buffer: the
// first epilogue overwrites them only after the first layer's MMAs are done.
struct TcStream {
  __align__(128) unsigned char h[TC_ROWS * MLP_H * 2];
  uint64_t mbar;                                           // completion of the stream's MMAs
};
struct TcSmem {
  __align__(128) unsigned char w0[MLP_H * MLP_IN * 2];     // W_1 [128][32], core-matrix K-major
  __align__(128) unsigned char w1[MLP_H * MLP_H * 2];      // W_2 [128][128]
  __align__(128) unsigned char w2[MLP_H * MLP_H * 2];      // W_3 [128][128]
  __align__(128) unsigned char w3[MLP_HEAD * MLP_H * 2];   // W_4 [80][128]
  TcStream st[TC_STREAMS];
  __align__(16) float hb[3 * MLP_H];                      // halved hidden biases
  __align__(16) float b4[MLP_HEAD];                       // head bias
  float norm[2 * MLP_IN + 2 * MLP_Y];                      // x mean, 1/x std, y mean, y std
  uint32_t taddr;
  int abort[TC_STREAMS];
};

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&h);
}

// A row-major bfloat16 matrix [rows][kc] (global) into the core-matrix
// K-major layout (shared), 16 bytes at a time.
__device__ __forceinline__ void tc_load_tile(unsigned char* dst, const __nv_bfloat16* src, int rows, int kc) {
  const int chunks = rows * (kc / 8);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int r = c / (kc / 8), k8 = c % (kc / 8);
    const uint4 v = *reinterpret_cast<const uint4*>(src + (long long)r * kc + k8 * 8);
    *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(r, k8 * 8, kc)) = v;
  }
}

// The 32 features of zone z (see the file header), standardised: all 32 as
// bfloat16 into row `row` of the stream's A tile, the first ten also as
// float32 into xu for the head.  Rows past the grid get the feature means
// (standardised zeros).
// Little float64 work here: the metric comes from a float copy of the
// centre table, and the P_n features are formed in float.
__device__ __forceinline__ void tc_features(const Params& p, const float* feat, const double* Pn, const float* gf,
                                            long long z, const TcSmem& S, TcStream& T, int row, float xu[MLP_XU]) {
  const long long N = p.N;
  float xf[MLP_IN];
  if (z < N) {
#pragma unroll
    for (int a = 0; a < NV; a++) xf[a] = __ldg(feat + a * N + z);
    if (gf) {  // the zone's g_{mu nu} from the float centre table of a general metric
      const long long nc = (long long)(p.n1 + 2) * (p.n2 + 2);
      const int zi = (int)(z % p.n1), zj = p.dim >= 2 ? (int)((z / p.n1) % p.n2) : 0;
      const float* gz = gf + (long long)(zj + 1) * (p.n1 + 2) + (zi + 1);
#pragma unroll
      for (int a = 0; a < 10; a++) xf[NV + a] = __ldg(gz + a * nc);
    } else {
      const float eta[10] = {-1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f};  // Minkowski g_{mu nu}
#pragma unroll
      for (int a = 0; a < 10; a++) xf[NV + a] = eta[a];
    }
    const float rho = (float)__ldg(Pn + z);
#pragma unroll
    for (int a = 0; a < NV; a++) xf[2 * NV + a] = mlp_pn_feature_f(a, a == 0 ? rho : (float)__ldg(Pn + a * N + z), rho);
    xf[30] = xf[31] = 0.f;
  } else {
#pragma unroll
    for (int a = 0; a < MLP_IN; a++) xf[a] = S.norm[a];
  }
  float xs[MLP_IN];
#pragma unroll
  for (int a = 0; a < MLP_IN; a++) xs[a] = (xf[a] - S.norm[a]) * S.norm[MLP_IN + a];
#pragma unroll
  for (int a = 0; a < MLP_XU; a++) xu[a] = xs[a];
#pragma unroll
  for (int c = 0; c < MLP_IN / 8; c++) {
    uint4 v;
    v.x = pack_bf16(xs[8 * c + 0], xs[8 * c + 1]);
    v.y = pack_bf16(xs[8 * c + 2], xs[8 * c + 3]);
    v.z = pack_bf16(xs[8 * c + 4], xs[8 * c + 5]);
    v.w = pack_bf16(xs[8 * c + 6], xs[8 * c + 7]);
    *reinterpret_cast<uint4*>(T.h + tc::kmajor_offset(row, 8 * c, MLP_IN)) = v;
  }
}

// Issue the MMAs of layer l for the tile (one thread) and commit them to
// the stream's mbarrier.
__device__ __forceinline__ void tc_issue_layer(const TcSmem& S, TcStream& T, int l, uint32_t tmem) {
  const unsigned char* B = l == 0 ? S.w0 : l == 1 ? S.w1 : l == 2 ? S.w2 : S.w3;
  const uint32_t kc = l == 0 ? MLP_IN : MLP_H;
  const uint32_t n = l == 3 ? MLP_HEAD : MLP_H;
  const uint32_t a0 = tc::smem_addr(T.h), b0 = tc::smem_addr(B), sbo = kc * 16u;
  const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, n);
  for (uint32_t s = 0; s < kc / 16; s++)  // K = 16 per MMA: two core matrices along K
    tc::mma_bf16(tmem, tc::smem_desc(a0 + 256u * s, 128u, sbo), tc::smem_desc(b0 + 256u * s, 128u, sbo), idesc,
                 s > 0);
  tc::commit(&T.mbar);
}

// Named barrier of one warpgroup (ids 1..4; 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1) mlp_guess_tc(const __grid_constant__ Params p,
                                                               const float* __restrict__ feat,
                                                               const double* __restrict__ Pn,
                                                               const __nv_bfloat16* __restrict__ wb,
                                                               const float* __restrict__ params,
                                                               const float* __restrict__ norm,
                                                               double* __restrict__ P0,
                                                               const float* __restrict__ gf,
                                                               unsigned long long* __restrict__ stalls) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = warp >> 2;                           // warpgroup: the tile stream of this thread
  const int row = (warp & 3) * 32 + (tid & 31);      // the tile row (zone) of this thread's TMEM lane
  TcStream& T = S.st[g];
  // weights, biases and standardisation into shared memory (all threads)
  tc_load_tile(S.w0, wb, MLP_H, MLP_IN);
  tc_load_tile(S.w1, wb + MLP_H * MLP_IN, MLP_H, MLP_H);
  tc_load_tile(S.w2, wb + MLP_H * MLP_IN + MLP_H * MLP_H, MLP_H, MLP_H);
  tc_load_tile(S.w3, wb + MLP_H * MLP_IN + 2 * MLP_H * MLP_H, MLP_HEAD, MLP_H);
  for (int i = tid; i < 3 * MLP_H; i += TC_THREADS) S.hb[i] = 0.5f * params[mlp_boff(i / MLP_H) + i % MLP_H];
  if (tid < MLP_HEAD) S.b4[tid] = params[mlp_boff(3) + tid];
  if (tid < 2 * MLP_IN + 2 * MLP_Y) S.norm[tid] = (tid >= MLP_IN && tid < 2 * MLP_IN) ? 1.0f / norm[tid] : norm[tid];
  if (tid < TC_STREAMS) {
    tc::mbar_init(&S.st[tid].mbar, 1);
    S.abort[tid] = 0;
  }
  if (warp == 0) tc::tmem_alloc(&S.taddr, TC_COLS * TC_STREAMS);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.taddr + TC_COLS * (uint32_t)g;             // this stream's accumulator
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lane quarter
  const bool issuer = (tid & 127) == 0;
  uint32_t phase = 0;
  const long long N = p.N;
  const long long tiles = (N + TC_ROWS - 1) / TC_ROWS;
  const long long tstep = (long long)gridDim.x * TC_STREAMS;
  for (long long t = (long long)blockIdx.x * TC_STREAMS + g; t < tiles; t += tstep) {
    const long long z = t * TC_ROWS + row;
    float xu[MLP_XU];
    tc_features(p, feat, Pn, gf, z, S, T, row, xu);
    tc::fence_async_smem();
    tc::fence_before_sync();
    wg_sync(g);
    for (int l = 0; l < MLP_NLAYER; l++) {
      if (issuer) {
        tc::fence_after_sync();
        tc_issue_layer(S, T, l, tmem);
      }
      // warp-uniform, since the TMEM loads below are warp-collective
      const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&T.mbar, phase, TC_WAIT_LIMIT));
      phase ^= 1u;
      if (!ok) S.abort[g] = 1;
      tc::fence_after_sync();
      uint32_t r[2][16];
      if (ok && l < MLP_NLAYER - 1) {
        // bias, SiLU, bfloat16 of this thread's zone, all 128 columns, 16 at
        // a time: the load of the next 16 is in flight while these are
        // processed
        const float4* hb4 = reinterpret_cast<const float4*>(S.hb + l * MLP_H);
        tc::ld_x16_issue(tlane, r[0]);
#pragma unroll
        for (int q = 0; q < MLP_H / 16; q++) {
          tc::ld_wait16(r[q & 1]);
          if (q + 1 < MLP_H / 16) tc::ld_x16_issue(tlane + (uint32_t)(16 * (q + 1)), r[(q + 1) & 1]);
          uint32_t u[8];
#pragma unroll
          for (int e4 = 0; e4 < 4; e4++) {
            const float4 b = hb4[4 * q + e4];
            const uint32_t* v = r[q & 1] + 4 * e4;
            u[2 * e4] = pack_bf16(silu_of_half(fmaf(__uint_as_float(v[0]), 0.5f, b.x)),
                                  silu_of_half(fmaf(__uint_as_float(v[1]), 0.5f, b.y)));
            u[2 * e4 + 1] = pack_bf16(silu_of_half(fmaf(__uint_as_float(v[2]), 0.5f, b.z)),
                                      silu_of_half(fmaf(__uint_as_float(v[3]), 0.5f, b.w)));
          }
          *reinterpret_cast<uint4*>(T.h + tc::kmajor_offset(row, 16 * q, MLP_H)) = make_uint4(u[0], u[1], u[2], u[3]);
          *reinterpret_cast<uint4*>(T.h + tc::kmajor_offset(row, 16 * q + 8, MLP_H)) =
              make_uint4(u[4], u[5], u[6], u[7]);
        }
      } else if (ok) {
        // head: y_i = sum_j M_ij x_j + c_i (M_ij in column 10 i + j, c_i in
        // column 70 + i), 16 columns at a time as above; then the start of
        // the zone (the loads are warp-collective: every lane takes part,
        // rows past the grid write nothing)
        const float4* b44 = reinterpret_cast<const float4*>(S.b4);
        float y[MLP_NP];
#pragma unroll
        for (int i = 0; i < MLP_NP; i++) y[i] = 0.f;
        tc::ld_x16_issue(tlane, r[0]);
#pragma unroll
        for (int q = 0; q < MLP_HEAD / 16; q++) {
          tc::ld_wait16(r[q & 1]);
          if (q + 1 < MLP_HEAD / 16) tc::ld_x16_issue(tlane + (uint32_t)(16 * (q + 1)), r[(q + 1) & 1]);
#pragma unroll
          for (int e4 = 0; e4 < 4; e4++) {
            const float4 b = b44[4 * q + e4];
            const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const int c = 16 * q + 4 * e4 + e;
              const float o = __uint_as_float(r[q & 1][4 * e4 + e]) + bb[e];
              if (c < MLP_NP * MLP_XU) y[c / MLP_XU] = fmaf(o, xu[c % MLP_XU], y[c / MLP_XU]);
              else if (c < MLP_NP * (MLP_XU + 1)) y[c - MLP_NP * MLP_XU] += o;
            }
          }
        }
        if (z < N) {
          const double rho = __ldg(Pn + z);
#pragma unroll
          for (int i = 0; i < MLP_NP; i++) {
            const int f = mlp_field(i);
            const double d = (double)(y[i] * S.norm[2 * MLP_IN + MLP_Y + f] + S.norm[2 * MLP_IN + f]);
            P0[f * N + z] = mlp_apply(f, f == 0 ? rho : __ldg(Pn + f * N + z), d, rho);
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      wg_sync(g);
      if (S.abort[g]) break;
    }
    if (S.abort[g]) break;
  }
  if (S.abort[g] && issuer) {
    // a layer's MMAs did not complete in time: wait (bounded) for them once
    // more before the tensor memory is released; the zones not reached keep
    // the plain start the zone-constant kernel wrote
    tc::mbar_wait(&T.mbar, phase ^ 1u, TC_WAIT_LIMIT);
    atomicAdd(stalls, 1ull);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(S.taddr, TC_COLS * TC_STREAMS);
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

// Reads and clears the training GEMM's stall counter (synchronous); true
// when a CTA gave up waiting (its tile was not written) or the read failed.
static bool mlp_take_stalls(grim_mlp* m) {
  unsigned long long n = 0;
  if (cudaMemcpy(&n, m->stalls, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
  if (n) cudaMemset(m->stalls, 0, sizeof(n));
  return n != 0;
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
    if ((e = gemm(B, no, nin, in, nin, m->wb + wboff, nin, m->z[l], no, m->ws, GT_WS_FLOATS, m->stalls, st)) !=
        cudaSuccess)
      return e;
    if (l < 3) {
      mlp_bias_silu<<<(unsigned)(((long long)B * no + T - 1) / T), T, 0, st>>>(m->z[l], m->params + mlp_boff(l), B, no,
                                                                              m->a[l], m->at[l]);
      in = m->a[l];
      nin = no;
    }
    wboff += no * mlp_nin(l);
  }
  // loss and dL/d(head) -> g (bf16 [B][80]), gt ([80][B]), dA (float [B][80])
  // one warp per block: a thread per row, spread over as many SMs as possible
  mlp_head_loss<<<(B + 31) / 32, 32, 0, st>>>(m->z[3], m->params + mlp_boff(3), m->yb, m->xh, B, m->g, m->gt, m->dA,
                                               m->loss);
  // backward
  for (int l = 3; l >= 0; l--) {
    const int no = mlp_nout(l), ni = mlp_nin(l);
    // dW_l [no][ni] = g^T [no][B] x a_{l-1} [B][ni]  ->  A = gt (K = B contiguous), B-operand = a_{l-1}^T [ni][B]
    const __nv_bfloat16* actT = (l == 0) ? m->xbt : m->at[l - 1];
    if ((e = gemm(no, ni, B, m->gt, B, actT, B, m->grad + mlp_woff(l), ni, m->ws, GT_WS_FLOATS, m->stalls, st)) !=
        cudaSuccess)
      return e;
    // db_l = column sums of the output-side gradient (float copy in dA)
    mlp_colsum_part<<<dim3((no + 31) / 32, MLP_CS_SLICES), dim3(32, 8), 0, st>>>(m->dA, B, no, m->ws);
    mlp_colsum_final<<<1, 128, 0, st>>>(m->ws, no, m->grad + mlp_boff(l));
    if (l == 0) break;
    // dA_{l-1} [B][ni] = g [B][no] x W_l [no][ni]  ->  B-operand = W_l^T [ni][no];
    // dA is reused: the bias gradient above has consumed it in stream order
    if ((e = gemm(B, ni, no, m->g, no, m->wbt + wboffs[l], no, m->dA, ni, m->ws, GT_WS_FLOATS, m->stalls, st)) !=
        cudaSuccess)
      return e;
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
            cudaMalloc(&m->loss, 4) == cudaSuccess && cudaMalloc(&m->ws, 4 * GT_WS_FLOATS) == cudaSuccess &&
            cudaMalloc(&m->stalls, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    grim_mlp_destroy(m);
    return GRIM_ENOMEM;
  }
  cudaMemset(m->m, 0, 4 * np);
  cudaMemset(m->v, 0, 4 * np);
  cudaMemset(m->stalls, 0, sizeof(unsigned long long));
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
                m->loss, m->z[0], m->z[1], m->z[2], m->z[3], m->a[0], m->a[1], m->a[2], m->at[0], m->at[1], m->at[2],
                m->ws, m->stalls};
  for (void* p : ps) cudaFree(p);
  delete m;
}

int grim_gemm_nt_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                      int splits) {
  if (!A || !B || !C || splits < 0 || splits > GT_MAX_SPLITS) return GRIM_EINVAL;
  float* ws = nullptr;
  unsigned long long* stalls = nullptr;
  const long long ws_floats = splits > 1 ? (long long)splits * M * N : 0;
  if (cudaMalloc(&stalls, sizeof(unsigned long long)) != cudaSuccess ||
      (ws_floats && cudaMalloc(&ws, 4 * ws_floats) != cudaSuccess)) {
    cudaFree(stalls);
    return GRIM_ENOMEM;
  }
  int rc = GRIM_OK;
  unsigned long long n = 0;
  if (cudaMemset(stalls, 0, sizeof(n)) != cudaSuccess) rc = GRIM_ECUDA;
  if (!rc) {
    const cudaError_t e = gemm(M, N, K, static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B),
                               ldb, C, ldc, ws, ws_floats, stalls, 0, splits ? splits : 1);
    if (e == cudaErrorInvalidValue) rc = GRIM_EINVAL;
    else if (e != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
             cudaMemcpy(&n, stalls, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess || n)
      rc = GRIM_ECUDA;
  }
  cudaFree(ws);
  cudaFree(stalls);
  return rc;
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
    mlp_gather<<<(batch + 31) / 32, 32>>>(X, Y, M, off, stride, batch, m->norm, m->xb, m->xbt, m->yb, m->xh);
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
  if (mlp_take_stalls(m)) return GRIM_ECUDA;
  if (mean_loss) *mean_loss = steps ? (double)l / steps : 0.0;
  return GRIM_OK;
}

int grim_mlp_gradient(grim_mlp* m, const float* X, const float* Y, long long M, float* grad_host, double* loss) {
  if (!m || !X || !Y || M < 64 || M % 64 || !grad_host) return GRIM_EINVAL;
  const int B = (int)M;
  int rc = mlp_alloc_batch(m, B);
  if (rc) return rc;
  cudaMemset(m->loss, 0, 4);
  mlp_gather<<<(B + 31) / 32, 32>>>(X, Y, M, 0, 1, B, m->norm, m->xb, m->xbt, m->yb, m->xh);
  if (mlp_forward_backward(m, B, 0) != cudaSuccess) return GRIM_ECUDA;
  float l = 0.f;
  if (cudaMemcpy(grad_host, m->grad, 4 * MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost) != cudaSuccess || mlp_take_stalls(m))
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

// float copy of the first n entries of a float64 table (the metric planes
// the learned start reads)
__global__ void mlp_table_f32(const double* __restrict__ in, long long n, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}
cudaError_t launch_mlp_metric_table(const Params& p, const double* gc, float* gf, cudaStream_t st) {
  const long long n = 10LL * (p.n1 + 2) * (p.n2 + 2);
  mlp_table_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gc, n, gf);
  return cudaGetLastError();
}

// gf: float copy of the first ten planes (g_{mu nu}) of the centre geometry
// table of a general metric (launch_mlp_metric_table), or NULL for
// Minkowski space.  stalls: a device counter raised when the kernel gave up
// waiting for its tensor-core work.
cudaError_t launch_mlp_guess(const Params& p, const float* feat, const double* Pn, const grim_mlp* m, double* P0,
                             const float* gf, unsigned long long* stalls, cudaStream_t st) {
  static PerDevice once;
  int sms = 0;
  cudaError_t e = once.get(
      [](int* v) {
        cudaError_t r = cudaFuncSetAttribute(mlp_guess_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(TcSmem));
        int dev = 0;
        if (r == cudaSuccess) r = cudaGetDevice(&dev);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        return r;
      },
      &sms);
  if (e != cudaSuccess) return e;
  const long long tiles = (p.N + TC_ROWS - 1) / TC_ROWS;
  long long grid = sms;  // persistent: one block (one copy of the weights, 256 TMEM columns) per SM
  if (grid > (tiles + TC_STREAMS - 1) / TC_STREAMS) grid = (tiles + TC_STREAMS - 1) / TC_STREAMS;
  mlp_guess_tc<<<(unsigned)grid, TC_THREADS, sizeof(TcSmem), st>>>(p, feat, Pn, m->wb, m->params, m->norm, P0, gf,
                                                                   stalls);
  return cudaGetLastError();
}
}  // namespace grim
