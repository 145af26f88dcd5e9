// rd_mlp.cu -- the surrogate network of delayed-acceptance sampling (not in
// the paper; Christen & Fox 2005): an MLP
//   x -> SiLU(W1 x + b1) -> SiLU(W2 . + b2) -> SiLU(W3 . + b3) -> W4 . + b4
// with x_i = (log theta_i - mu_i) / s_i (padded to 16 inputs), width 256,
// BF16 weights and activations into FP32-accumulating tcgen05 GEMMs, FP32
// master weights, Adam with decoupled weight decay, and the output mapped to
// a log-likelihood by Phi~ = floor + exp(shift + scale * net(x)).
//
// GEMM kernel: D[M][N] = sum_k A[m][k] B[n][k] for one 128-row tile of M and
// all N <= 256 columns per CTA; K is staged 64 at a time into 128B-swizzled
// shared memory (K-major or MN-major per operand, matching how the operand is
// stored in global memory), one thread issues the M=128 kind::f16 MMAs (BF16
// inputs, FP32 accumulator in TMEM) and four warps run the fused epilogue
// (bias + SiLU, SiLU', or a plain FP32 store) from TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rd_common.cuh"
#include "rd_internal.h"
#include "rd_tc_ptx.cuh"

namespace rd {
namespace mlp {

using namespace tc;

constexpr int kIn = 16;        // padded input features
constexpr int kGemmThreads = 128;
constexpr int kKChunk = 64;    // K elements staged per round (one 128-byte swizzle atom)

enum Epi { EPI_FWD_SILU = 0, EPI_BWD_SILU = 1, EPI_F32 = 2 };

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;  // K-major: A[m * lda + k]; MN-major: A[k * lda + m]
  int lda;
  const __nv_bfloat16* B;  // K-major: B[n * ldb + k]; MN-major: B[k * ldb + n]
  int ldb;
  const float* bias;       // EPI_FWD_SILU: [N]
  const float* zprev;      // EPI_BWD_SILU: [M][N] pre-activations
  float* out_f32;          // EPI_FWD_SILU: Z [M][N]; EPI_F32: D [M][N]
  __nv_bfloat16* out_bf16; // EPI_FWD_SILU: SiLU(Z); EPI_BWD_SILU: dZ
  int* err;
};

// Stages rows [0, rows) x K columns [k0, k0 + kc) of a K-major matrix into a
// 128B-swizzled tile with `rows` rows (columns beyond kc are zero).
__device__ __forceinline__ void stage_kmajor(uint8_t* tile, const __nv_bfloat16* g, int ld,
                                             int rows, int row0, int rows_valid, int k0, int kc) {
  for (int i = threadIdx.x; i < rows * 8; i += kGemmThreads) {
    const int r = i >> 3, c8 = (i & 7) * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < rows_valid && c8 < kc)
      v = *reinterpret_cast<const uint4*>(g + (size_t)(row0 + r) * ld + k0 + c8);
    *reinterpret_cast<uint4*>(tile + sw128_offset(rows, r, c8)) = v;
  }
}

// Stages K rows [k0, k0 + kc) x MN columns [mn0, mn0 + cols) of an MN-major
// matrix (g[k * ld + mn]) into a swizzled tile of 64 K rows (rows beyond kc
// are zero).
__device__ __forceinline__ void stage_mnmajor(uint8_t* tile, const __nv_bfloat16* g, int ld,
                                              int cols, int mn0, int k0, int kc) {
  const int per_row = cols / 8;
  for (int i = threadIdx.x; i < kKChunk * per_row; i += kGemmThreads) {
    const int r = i / per_row, c8 = (i - r * per_row) * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < kc) v = *reinterpret_cast<const uint4*>(g + (size_t)(k0 + r) * ld + mn0 + c8);
    *reinterpret_cast<uint4*>(tile + sw128_offset(kKChunk, r, c8)) = v;
  }
}

template <int EPI, int A_MN, int B_MN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_bf16(GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* ta = base;                 // A tile: 128 x 64 (16 KB)
  uint8_t* tb = base + 16384;         // B tile: up to 256 x 64 (32 KB)
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int N = g.N;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 256);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(128, N, A_MN, B_MN);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < g.K && ok; k0 += kKChunk) {
    const int kc = min(kKChunk, g.K - k0);
    if (A_MN)
      stage_mnmajor(ta, g.A, g.lda, 128, m0, k0, kc);
    else
      stage_kmajor(ta, g.A, g.lda, 128, m0, g.M - m0, k0, kc);
    if (B_MN)
      stage_mnmajor(tb, g.B, g.ldb, N, 0, k0, kc);
    else
      stage_kmajor(tb, g.B, g.ldb, N, 0, N, k0, kc);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint64_t ad = sdesc_sw128(smem_u32(ta), A_MN ? 128u * 64u : 16u, 1024u);
      const uint64_t bd = sdesc_sw128(smem_u32(tb), B_MN ? 128u * 64u : 16u, 1024u);
      for (int kk = 0; kk < kc / 16; ++kk) {
        const uint64_t off = (uint64_t)(A_MN ? kk * 2048 : kk * 32) >> 4;
        const uint64_t offb = (uint64_t)(B_MN ? kk * 2048 : kk * 32) >> 4;
        mma_f16(tmem, ad + off, bd + offb, idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar);
    }
    // the tiles are overwritten next round: wait for the MMAs to finish
    ok = mbar_wait_bounded(&bar, phase & 1u, &abort_flag);
    ++phase;
    tc_fence_after();
    __syncthreads();
  }
  if (ok) {
    const int m = m0 + 32 * warp + lane;  // TMEM lane = row of the tile
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    for (int n0 = 0; n0 < N; n0 += 8) {
      float v[8];
      __syncwarp();
      tmem_ld8(trow + (uint32_t)n0, v);
      tmem_wait_ld();
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const size_t o = (size_t)m * N + n0 + j;
        if (EPI == EPI_FWD_SILU) {
          const float z = v[j] + g.bias[n0 + j];
          g.out_f32[o] = z;
          g.out_bf16[o] = __float2bfloat16_rn(silu(z));
        } else if (EPI == EPI_BWD_SILU) {
          g.out_bf16[o] = __float2bfloat16_rn(v[j] * silu_grad(g.zprev[o]));
        } else {
          g.out_f32[o] = v[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
  if (threadIdx.x == 0 && abort_flag) atomicOr(g.err, 1);
}

// The tiles need 49 KB; asking for 100 KB keeps at most two CTAs (two
// 256-column TMEM allocations) on an SM, so an allocation never waits.
constexpr size_t kGemmSmem = 100 * 1024;

template <int EPI, int A_MN, int B_MN>
static cudaError_t gemm(const GemmArgs& a, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<EPI, A_MN, B_MN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_gemm_bf16<EPI, A_MN, B_MN><<<(a.M + 127) / 128, kGemmThreads, kGemmSmem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small CUDA-core kernels
// ---------------------------------------------------------------------------
struct Norm {
  double in_mu[RD_NPARAM], in_sd[RD_NPARAM];
  double floor, shift, scale;
};

// Features x_i = (log theta_i - mu_i) / s_i as BF16, zero-padded to 16.
__global__ void k_features(int B, int P, const double* theta, Norm nm, __nv_bfloat16* X) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int j = 0; j < kIn; ++j) {
    float v = 0.f;
    if (j < P) {
      const double t = theta[(size_t)b * P + j];
      v = (float)((log(t > 0.0 ? t : 1e-300) - nm.in_mu[j]) / nm.in_sd[j]);
    }
    X[(size_t)b * kIn + j] = __float2bfloat16_rn(v);
  }
}

// Last layer out[b] = sum_j H3[b][j] W4[j] + b4 (FP32), one warp per row; with
// a target, also dOut[b] = 2 (out - z) / B and the squared error.
__global__ void k_head_fwd(int B, int W, const __nv_bfloat16* H3, const float* W4,
                           const float* b4, float* out, const float* target, float* dout,
                           double* sq_err) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  float s = 0.f;
  for (int j = lane; j < W; j += 32) s += __bfloat162float(H3[(size_t)warp * W + j]) * W4[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float y = s + b4[0];
    out[warp] = y;
    if (target) {
      const float e = y - target[warp];
      dout[warp] = 2.f * e / (float)B;
      atomicAdd(sq_err, (double)e * (double)e);
    }
  }
}

// dZ3[b][j] = dOut[b] W4[j] SiLU'(Z3[b][j]) (BF16)
__global__ void k_head_bwd(int B, int W, const float* dout, const float* W4, const float* Z3,
                           __nv_bfloat16* dZ3) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * W) return;
  const int b = (int)(i / W), j = (int)(i - (size_t)b * W);
  dZ3[i] = __float2bfloat16_rn(dout[b] * W4[j] * silu_grad(Z3[i]));
}

// Column sums: g[j] = sum_b D[b][j] for a BF16 (dZ) or FP32 matrix, and for
// the head dW4[j] = sum_b dOut[b] H3[b][j], db4 = sum_b dOut[b].
__global__ void k_colsum_bf16(int B, int W, const __nv_bfloat16* D, float* g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= W) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += __bfloat162float(D[(size_t)b * W + j]);
  g[j] = s;
}

__global__ void k_head_wgrad(int B, int W, const float* dout, const __nv_bfloat16* H3, float* gW4,
                             float* gb4) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < W) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dout[b] * __bfloat162float(H3[(size_t)b * W + j]);
    gW4[j] = s;
  }
  if (j == 0) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dout[b];
    gb4[0] = s;
  }
}

// Adam with bias correction and decoupled weight decay on the weights (mask
// = 1) but not the biases; refreshes the BF16 copies of W1..W3.
struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  const uint8_t* decay_mask;
  int n;
  float lr, b1, b2, eps, wd, c1, c2;
};
__global__ void k_adam(AdamArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float gi = a.g[i];
  const float m = a.m[i] = a.b1 * a.m[i] + (1.f - a.b1) * gi;
  const float v = a.v[i] = a.b2 * a.v[i] + (1.f - a.b2) * gi * gi;
  float p = a.p[i];
  if (a.decay_mask[i]) p -= a.lr * a.wd * p;
  p -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
  a.p[i] = p;
}

__global__ void k_to_bf16(int n, const float* src, __nv_bfloat16* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Phi~ = floor + exp(shift + scale * out) in FP64.
__global__ void k_output(int B, const float* out, Norm nm, double* phit) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) phit[b] = nm.floor + exp(nm.shift + nm.scale * (double)out[b]);
}

}  // namespace mlp
}  // namespace rd

// ---------------------------------------------------------------------------
// Host side: the surrogate object, forward/backward, training, prediction
// ---------------------------------------------------------------------------
namespace rd {
namespace mlp {

// FP32 parameter layout: W1 [W][16], b1 [W], W2 [W][W], b2, W3 [W][W], b3, W4 [W], b4 [1].
struct Layout {
  int W;
  size_t oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, total;
  explicit Layout(int w) : W(w) {
    oW1 = 0;
    ob1 = oW1 + (size_t)W * kIn;
    oW2 = ob1 + W;
    ob2 = oW2 + (size_t)W * W;
    oW3 = ob2 + W;
    ob3 = oW3 + (size_t)W * W;
    oW4 = ob3 + W;
    ob4 = oW4 + W;
    total = ob4 + 1;
  }
};

}  // namespace mlp
}  // namespace rd

struct rd_surrogate {
  rd_problem* pb = nullptr;
  int P = 0;
  int W = 256;
  rd::mlp::Norm norm{};
  float* params = nullptr;
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  uint8_t* decay_mask = nullptr;
  __nv_bfloat16* Wb = nullptr;  // BF16 copies of W1, W2, W3 (packed like params)
  int adam_t = 0;
  // activations for up to `cap` rows
  int cap = 0;
  __nv_bfloat16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr;
  __nv_bfloat16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *out = nullptr, *dout = nullptr,
        *target = nullptr;
  double* sqerr = nullptr;
};

namespace rd {
namespace mlp {

static void free_acts(rd_surrogate* s) {
  void* ptrs[] = {s->X, s->H1, s->H2, s->H3, s->dZ1, s->dZ2, s->dZ3, s->Z1,
                  s->Z2, s->Z3, s->out, s->dout, s->target, s->sqerr};
  for (void* p : ptrs) cudaFree(p);
  s->X = s->H1 = s->H2 = s->H3 = s->dZ1 = s->dZ2 = s->dZ3 = nullptr;
  s->Z1 = s->Z2 = s->Z3 = s->out = s->dout = s->target = nullptr;
  s->sqerr = nullptr;
  s->cap = 0;
}

cudaError_t ensure_rows(rd_surrogate* s, int rows) {
  if (rows <= s->cap) return cudaSuccess;
  cudaStreamSynchronize(s->pb->stream);
  free_acts(s);
  const int cap = ((rows + 127) / 128) * 128;
  const size_t W = (size_t)s->W;
  cudaError_t e;
#define RD_ALLOC(ptr, bytes) \
  if ((e = cudaMalloc(&(ptr), (bytes))) != cudaSuccess) return e;
  RD_ALLOC(s->X, sizeof(__nv_bfloat16) * cap * kIn);
  RD_ALLOC(s->H1, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->H2, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->H3, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->dZ1, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->dZ2, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->dZ3, sizeof(__nv_bfloat16) * cap * W);
  RD_ALLOC(s->Z1, sizeof(float) * cap * W);
  RD_ALLOC(s->Z2, sizeof(float) * cap * W);
  RD_ALLOC(s->Z3, sizeof(float) * cap * W);
  RD_ALLOC(s->out, sizeof(float) * cap);
  RD_ALLOC(s->dout, sizeof(float) * cap);
  RD_ALLOC(s->target, sizeof(float) * cap);
  RD_ALLOC(s->sqerr, sizeof(double));
#undef RD_ALLOC
  s->cap = cap;
  s->pb->generation++;  // captured graphs may hold the old buffers
  return cudaSuccess;
}

static cudaError_t refresh_bf16(rd_surrogate* s, cudaStream_t st) {
  const Layout L(s->W);
  const int n = (int)L.ob4 + 1;
  k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(n, s->params, s->Wb);
  return cudaGetLastError();
}

// Forward pass for B rows of theta (device [B][P]) into s->out; with a
// target (device [B], normalised), also dOut and the summed squared error.
cudaError_t forward(rd_surrogate* s, int B, const double* theta, bool with_target,
                    cudaStream_t st) {
  const Layout L(s->W);
  const int W = s->W;
  int* err = s->pb->ws.err;
  k_features<<<(B + 127) / 128, 128, 0, st>>>(B, s->P, theta, s->norm, s->X);
  GemmArgs g{};
  g.err = err;
  g.M = B;
  g.N = W;
  g.K = kIn;
  g.A = s->X;
  g.lda = kIn;
  g.B = s->Wb + L.oW1;
  g.ldb = kIn;
  g.bias = s->params + L.ob1;
  g.out_f32 = s->Z1;
  g.out_bf16 = s->H1;
  cudaError_t e = gemm<EPI_FWD_SILU, 0, 0>(g, st);
  if (e != cudaSuccess) return e;
  g.K = W;
  g.A = s->H1;
  g.lda = W;
  g.B = s->Wb + L.oW2;
  g.ldb = W;
  g.bias = s->params + L.ob2;
  g.out_f32 = s->Z2;
  g.out_bf16 = s->H2;
  if ((e = gemm<EPI_FWD_SILU, 0, 0>(g, st)) != cudaSuccess) return e;
  g.A = s->H2;
  g.B = s->Wb + L.oW3;
  g.bias = s->params + L.ob3;
  g.out_f32 = s->Z3;
  g.out_bf16 = s->H3;
  if ((e = gemm<EPI_FWD_SILU, 0, 0>(g, st)) != cudaSuccess) return e;
  if (with_target) {
    if ((e = cudaMemsetAsync(s->sqerr, 0, sizeof(double), st)) != cudaSuccess) return e;
  }
  k_head_fwd<<<(B * 32 + 255) / 256, 256, 0, st>>>(
      B, W, s->H3, s->params + L.oW4, s->params + L.ob4, s->out,
      with_target ? s->target : nullptr, s->dout, s->sqerr);
  return cudaGetLastError();
}

// Backward pass of the mean-squared error after forward(with_target): all
// parameter gradients into s->grads.
cudaError_t backward(rd_surrogate* s, int B, cudaStream_t st) {
  const Layout L(s->W);
  const int W = s->W;
  int* err = s->pb->ws.err;
  const size_t nW = (size_t)B * W;
  k_head_bwd<<<(unsigned)((nW + 255) / 256), 256, 0, st>>>(B, W, s->dout, s->params + L.oW4,
                                                           s->Z3, s->dZ3);
  k_head_wgrad<<<(W + 127) / 128, 128, 0, st>>>(B, W, s->dout, s->H3, s->grads + L.oW4,
                                                s->grads + L.ob4);
  const __nv_bfloat16* Hs[3] = {s->X, s->H1, s->H2};  // inputs of layers 1..3
  __nv_bfloat16* dZs[3] = {s->dZ1, s->dZ2, s->dZ3};
  const float* Zs[3] = {s->Z1, s->Z2, s->Z3};
  const size_t oW[3] = {L.oW1, L.oW2, L.oW3}, ob[3] = {L.ob1, L.ob2, L.ob3};
  const int in[3] = {kIn, W, W};
  cudaError_t e;
  for (int l = 2; l >= 0; --l) {
    // dW_l = dZ_l^T H_{l-1}: M = W (outputs), N = in_l, K = B
    GemmArgs g{};
    g.err = err;
    g.M = W;
    g.N = in[l];
    g.K = B;
    g.A = dZs[l];
    g.lda = W;
    g.B = Hs[l];
    g.ldb = in[l];
    g.out_f32 = s->grads + oW[l];
    if ((e = gemm<EPI_F32, 1, 1>(g, st)) != cudaSuccess) return e;
    k_colsum_bf16<<<(W + 127) / 128, 128, 0, st>>>(B, W, dZs[l], s->grads + ob[l]);
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) o SiLU'(Z_{l-1}): M = B, N = W, K = W
    GemmArgs h{};
    h.err = err;
    h.M = B;
    h.N = W;
    h.K = W;
    h.A = dZs[l];
    h.lda = W;
    h.B = s->Wb + oW[l];
    h.ldb = W;
    h.zprev = Zs[l - 1];
    h.out_bf16 = dZs[l - 1];
    if ((e = gemm<EPI_BWD_SILU, 0, 1>(h, st)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t adam_step(rd_surrogate* s, double lr, double b1, double b2, double eps, double wd,
                      cudaStream_t st) {
  const Layout L(s->W);
  s->adam_t += 1;
  AdamArgs a;
  a.p = s->params;
  a.g = s->grads;
  a.m = s->adam_m;
  a.v = s->adam_v;
  a.decay_mask = s->decay_mask;
  a.n = (int)L.total;
  a.lr = (float)lr;
  a.b1 = (float)b1;
  a.b2 = (float)b2;
  a.eps = (float)eps;
  a.wd = (float)wd;
  a.c1 = (float)(1.0 - pow(b1, s->adam_t));
  a.c2 = (float)(1.0 - pow(b2, s->adam_t));
  k_adam<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return refresh_bf16(s, st);
}

cudaError_t predict(rd_surrogate* s, int B, const double* theta, double* phit, cudaStream_t st) {
  cudaError_t e = forward(s, B, theta, false, st);
  if (e != cudaSuccess) return e;
  k_output<<<(B + 127) / 128, 128, 0, st>>>(B, s->out, s->norm, phit);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace rd

using namespace rd;

#define RD_SCHECK(cond, code, msg) \
  do {                             \
    if (!(cond)) {                 \
      rd::set_error(msg);          \
      return code;                 \
    }                              \
  } while (0)
#define RD_SCUDA(call)                                                     \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      rd::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return RD_ECUDA;                                                     \
    }                                                                      \
  } while (0)

extern "C" {

rd_status rd_surrogate_destroy(rd_surrogate* s) {
  if (!s) return RD_OK;
  if (s->pb) cudaStreamSynchronize(s->pb->stream);
  rd::mlp::free_acts(s);
  cudaFree(s->params);
  cudaFree(s->grads);
  cudaFree(s->adam_m);
  cudaFree(s->adam_v);
  cudaFree(s->decay_mask);
  cudaFree(s->Wb);
  delete s;
  return RD_OK;
}

rd_status rd_surrogate_create(rd_problem* p, uint64_t seed, rd_surrogate** out) {
  RD_SCHECK(p && out, RD_EINVAL, "NULL argument");
  *out = nullptr;
  rd_surrogate* s = new rd_surrogate();
  s->pb = p;
  s->P = p->desc.n_params;
  s->W = RD_SURROGATE_WIDTH;
  const mlp::Layout L(s->W);
  // He-uniform initial weights (bound sqrt(6 / fan_in)); last layer scaled by
  // 0.1; biases zero.  A 64-bit linear congruential stream seeded by `seed`.
  std::vector<float> h(L.total, 0.f);
  std::vector<uint8_t> mask(L.total, 0);
  uint64_t state = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(state >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](size_t off, int rows, int cols, int fan_in, double scale) {
    const double bound = sqrt(6.0 / fan_in) * scale;
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        h[off + (size_t)r * cols + c] = (float)((2.0 * uni() - 1.0) * bound);
        mask[off + (size_t)r * cols + c] = 1;
      }
  };
  fill(L.oW1, s->W, mlp::kIn, s->P, 1.0);
  for (int r = 0; r < s->W; ++r)  // padded inputs carry no weight
    for (int c = s->P; c < mlp::kIn; ++c) h[L.oW1 + (size_t)r * mlp::kIn + c] = 0.f;
  fill(L.oW2, s->W, s->W, s->W, 1.0);
  fill(L.oW3, s->W, s->W, s->W, 1.0);
  fill(L.oW4, 1, s->W, s->W, 0.1);
  for (int j = 0; j < RD_NPARAM; ++j) {
    s->norm.in_mu[j] = 0.0;
    s->norm.in_sd[j] = 1.0;
  }
  s->norm.floor = 0.0;
  s->norm.shift = 0.0;
  s->norm.scale = 1.0;
  bool ok = cudaMalloc(&s->params, sizeof(float) * L.total) == cudaSuccess &&
            cudaMalloc(&s->grads, sizeof(float) * L.total) == cudaSuccess &&
            cudaMalloc(&s->adam_m, sizeof(float) * L.total) == cudaSuccess &&
            cudaMalloc(&s->adam_v, sizeof(float) * L.total) == cudaSuccess &&
            cudaMalloc(&s->decay_mask, L.total) == cudaSuccess &&
            cudaMalloc(&s->Wb, sizeof(__nv_bfloat16) * (L.ob4 + 1)) == cudaSuccess;
  ok = ok && cudaMemcpy(s->params, h.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(s->decay_mask, mask.data(), L.total, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(s->grads, 0, sizeof(float) * L.total) == cudaSuccess &&
       cudaMemset(s->adam_m, 0, sizeof(float) * L.total) == cudaSuccess &&
       cudaMemset(s->adam_v, 0, sizeof(float) * L.total) == cudaSuccess &&
       mlp::refresh_bf16(s, p->stream) == cudaSuccess &&
       cudaStreamSynchronize(p->stream) == cudaSuccess;
  if (!ok) {
    rd_surrogate_destroy(s);
    set_error("surrogate allocation failed");
    return RD_ENOMEM;
  }
  *out = s;
  return RD_OK;
}

rd_status rd_surrogate_get_params(rd_surrogate* s, float* host, size_t cap, size_t* n,
                                  double* norm) {
  RD_SCHECK(s && n, RD_EINVAL, "NULL argument");
  const mlp::Layout L(s->W);
  *n = L.total;
  if (host) {
    RD_SCHECK(cap >= L.total, RD_EINVAL, "parameter buffer too small");
    RD_SCUDA(cudaStreamSynchronize(s->pb->stream));
    RD_SCUDA(cudaMemcpy(host, s->params, sizeof(float) * L.total, cudaMemcpyDeviceToHost));
  }
  if (norm) {
    for (int j = 0; j < RD_NPARAM; ++j) {
      norm[j] = s->norm.in_mu[j];
      norm[RD_NPARAM + j] = s->norm.in_sd[j];
    }
    norm[2 * RD_NPARAM] = s->norm.floor;
    norm[2 * RD_NPARAM + 1] = s->norm.shift;
    norm[2 * RD_NPARAM + 2] = s->norm.scale;
  }
  return RD_OK;
}

rd_status rd_surrogate_set_params(rd_surrogate* s, const float* host, size_t n,
                                  const double* norm) {
  RD_SCHECK(s, RD_EINVAL, "NULL argument");
  const mlp::Layout L(s->W);
  if (host) {
    RD_SCHECK(n == L.total, RD_EINVAL, "parameter count mismatch");
    RD_SCUDA(cudaStreamSynchronize(s->pb->stream));
    RD_SCUDA(cudaMemcpy(s->params, host, sizeof(float) * L.total, cudaMemcpyHostToDevice));
    RD_SCUDA(mlp::refresh_bf16(s, s->pb->stream));
    RD_SCUDA(cudaStreamSynchronize(s->pb->stream));
  }
  if (norm) {
    for (int j = 0; j < RD_NPARAM; ++j) {
      RD_SCHECK(norm[RD_NPARAM + j] > 0, RD_EINVAL, "input scales must be positive");
      s->norm.in_mu[j] = norm[j];
      s->norm.in_sd[j] = norm[RD_NPARAM + j];
    }
    s->norm.floor = norm[2 * RD_NPARAM];
    s->norm.shift = norm[2 * RD_NPARAM + 1];
    s->norm.scale = norm[2 * RD_NPARAM + 2];
    s->pb->generation++;  // captured sampler graphs hold the normalisation by value
  }
  return RD_OK;
}

rd_status rd_surrogate_loss_grad(rd_surrogate* s, int B, const double* theta,
                                 const float* target, double* loss, float* grads) {
  RD_SCHECK(s && theta && target && loss, RD_EINVAL, "NULL argument");
  RD_SCHECK(B >= 128 && B % 128 == 0, RD_EINVAL, "B must be a positive multiple of 128");
  cudaStream_t st = s->pb->stream;
  RD_SCUDA(mlp::ensure_rows(s, B));
  RD_SCUDA(cudaMemcpyAsync(s->target, target, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
  RD_SCUDA(mlp::forward(s, B, theta, true, st));
  RD_SCUDA(mlp::backward(s, B, st));
  double se = 0.0;
  RD_SCUDA(cudaMemcpyAsync(&se, s->sqerr, sizeof(double), cudaMemcpyDeviceToHost, st));
  const mlp::Layout L(s->W);
  if (grads)
    RD_SCUDA(cudaMemcpyAsync(grads, s->grads, sizeof(float) * L.total, cudaMemcpyDeviceToDevice, st));
  RD_SCUDA(cudaStreamSynchronize(st));
  *loss = se / B;
  return RD_OK;
}

rd_status rd_surrogate_predict(rd_surrogate* s, int B, const double* theta, double* phi_tilde) {
  RD_SCHECK(s && theta && phi_tilde, RD_EINVAL, "NULL argument");
  RD_SCHECK(B >= 0, RD_EINVAL, "B must be >= 0");
  if (B == 0) return RD_OK;
  RD_SCUDA(mlp::ensure_rows(s, B));
  RD_SCUDA(mlp::predict(s, B, theta, phi_tilde, s->pb->stream));
  return RD_OK;
}

rd_status rd_surrogate_train(rd_surrogate* s, int n, const double* theta, const double* phi,
                             const rd_train_desc* td, double* report) {
  RD_SCHECK(s && theta && phi && td, RD_EINVAL, "NULL argument");
  RD_SCHECK(td->batch >= 128 && td->batch % 128 == 0, RD_EINVAL,
            "batch must be a positive multiple of 128");
  RD_SCHECK(td->epochs >= 1 && td->lr > 0, RD_EINVAL, "epochs >= 1 and lr > 0 required");
  cudaStream_t st = s->pb->stream;
  const int P = s->P;
  // host copies: normalisation and the shuffled order need them once
  std::vector<double> th((size_t)n * P), ph(n);
  RD_SCUDA(cudaStreamSynchronize(st));
  RD_SCUDA(cudaMemcpy(th.data(), theta, sizeof(double) * th.size(), cudaMemcpyDeviceToHost));
  RD_SCUDA(cudaMemcpy(ph.data(), phi, sizeof(double) * ph.size(), cudaMemcpyDeviceToHost));
  std::vector<int> keep;
  keep.reserve(n);
  double pmin = INFINITY;
  for (int i = 0; i < n; ++i) {
    bool ok = std::isfinite(ph[i]);
    for (int j = 0; j < P && ok; ++j) ok = th[(size_t)i * P + j] > 0;
    if (ok) {
      keep.push_back(i);
      pmin = std::min(pmin, ph[i]);
    }
  }
  RD_SCHECK((int)keep.size() >= 2 * td->batch, RD_EINVAL,
            "too few finite training pairs for two batches");
  // normalisation: inputs by the mean/sd of log theta, targets
  // z = log(phi - floor) standardised, floor = min phi - 1
  mlp::Norm nm{};
  for (int j = 0; j < RD_NPARAM; ++j) {
    nm.in_mu[j] = 0.0;
    nm.in_sd[j] = 1.0;
  }
  for (int j = 0; j < P; ++j) {
    double m = 0, v = 0;
    for (int i : keep) m += log(th[(size_t)i * P + j]);
    m /= keep.size();
    for (int i : keep) {
      const double d = log(th[(size_t)i * P + j]) - m;
      v += d * d;
    }
    nm.in_mu[j] = m;
    nm.in_sd[j] = std::max(sqrt(v / keep.size()), 1e-12);
  }
  nm.floor = pmin - 1.0;
  double zm = 0, zv = 0;
  for (int i : keep) zm += log(ph[i] - nm.floor);
  zm /= keep.size();
  for (int i : keep) {
    const double d = log(ph[i] - nm.floor) - zm;
    zv += d * d;
  }
  nm.shift = zm;
  nm.scale = std::max(sqrt(zv / keep.size()), 1e-12);
  s->norm = nm;
  s->pb->generation++;
  // seeded shuffle, hold-out split
  uint64_t state = td->seed * 2862933555777941757ull + 3037000493ull;
  auto next = [&]() {
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    return state >> 33;
  };
  for (size_t i = keep.size() - 1; i > 0; --i) std::swap(keep[i], keep[next() % (i + 1)]);
  const int n_hold = std::max(td->batch, (int)(td->holdout_frac * keep.size()) / td->batch * td->batch);
  const int n_train = ((int)keep.size() - n_hold) / td->batch * td->batch;
  RD_SCHECK(n_train >= td->batch, RD_EINVAL, "too few training pairs after the hold-out split");
  std::vector<double> th_s((size_t)(n_train + n_hold) * P);
  std::vector<float> z_s(n_train + n_hold);
  for (int r = 0; r < n_train + n_hold; ++r) {
    const int i = keep[r];
    for (int j = 0; j < P; ++j) th_s[(size_t)r * P + j] = th[(size_t)i * P + j];
    z_s[r] = (float)((log(ph[i] - nm.floor) - nm.shift) / nm.scale);
  }
  double* d_th = nullptr;
  float* d_z = nullptr;
  RD_SCUDA(cudaMalloc(&d_th, sizeof(double) * th_s.size()));
  RD_SCUDA(cudaMalloc(&d_z, sizeof(float) * z_s.size()));
  RD_SCUDA(cudaMemcpy(d_th, th_s.data(), sizeof(double) * th_s.size(), cudaMemcpyHostToDevice));
  RD_SCUDA(cudaMemcpy(d_z, z_s.data(), sizeof(float) * z_s.size(), cudaMemcpyHostToDevice));
  RD_SCUDA(mlp::ensure_rows(s, td->batch));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  const int nb = n_train / td->batch;
  double train_mse = 0.0;
  std::vector<double> ep_se(nb);
  for (int ep = 0; ep < td->epochs; ++ep) {
    // batches in a seeded order each epoch
    std::vector<int> order(nb);
    for (int b = 0; b < nb; ++b) order[b] = b;
    for (int b = nb - 1; b > 0; --b) std::swap(order[b], order[next() % (b + 1)]);
    double se = 0.0;
    for (int k = 0; k < nb; ++k) {
      const int b = order[k];
      RD_SCUDA(cudaMemcpyAsync(s->target, d_z + (size_t)b * td->batch, sizeof(float) * td->batch,
                               cudaMemcpyDeviceToDevice, st));
      RD_SCUDA(mlp::forward(s, td->batch, d_th + (size_t)b * td->batch * P, true, st));
      RD_SCUDA(mlp::backward(s, td->batch, st));
      RD_SCUDA(mlp::adam_step(s, td->lr, td->beta1, td->beta2, 1e-8, td->weight_decay, st));
      if (ep == td->epochs - 1) {
        double v = 0.0;
        RD_SCUDA(cudaMemcpyAsync(&v, s->sqerr, sizeof(double), cudaMemcpyDeviceToHost, st));
        RD_SCUDA(cudaStreamSynchronize(st));
        se += v;
      }
    }
    if (ep == td->epochs - 1) train_mse = se / n_train;
  }
  // hold-out error in target units and in Phi units
  double hold_se = 0.0, hold_abs = 0.0;
  std::vector<float> outv(td->batch);
  for (int off = n_train; off + td->batch <= n_train + n_hold; off += td->batch) {
    RD_SCUDA(cudaMemcpyAsync(s->target, d_z + off, sizeof(float) * td->batch,
                             cudaMemcpyDeviceToDevice, st));
    RD_SCUDA(mlp::forward(s, td->batch, d_th + (size_t)off * P, true, st));
    double v = 0.0;
    RD_SCUDA(cudaMemcpyAsync(&v, s->sqerr, sizeof(double), cudaMemcpyDeviceToHost, st));
    RD_SCUDA(cudaMemcpyAsync(outv.data(), s->out, sizeof(float) * td->batch, cudaMemcpyDeviceToHost, st));
    RD_SCUDA(cudaStreamSynchronize(st));
    hold_se += v;
    for (int r = 0; r < td->batch; ++r) {
      const double pt = nm.floor + exp(nm.shift + nm.scale * (double)outv[r]);
      const double pe = nm.floor + exp(nm.shift + nm.scale * (double)z_s[off + r]);
      hold_abs += fabs(pt - pe) / pe;
    }
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_th);
  cudaFree(d_z);
  int err = 0;
  RD_SCUDA(cudaMemcpy(&err, s->pb->ws.err, sizeof(int), cudaMemcpyDeviceToHost));
  RD_SCHECK(!err, RD_ETIMEOUT, "a training kernel's bounded wait gave up");
  if (report) {
    report[0] = train_mse;
    report[1] = hold_se / std::max(n_hold, 1);
    report[2] = hold_abs / std::max(n_hold, 1);
    report[3] = ms * 1e-3;
  }
  return RD_OK;
}

}  // extern "C"
