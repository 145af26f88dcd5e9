// rd_simt_common.cuh -- CUDA-core building blocks of the 2-D FP32 solves
// (rd_solve_simt.cu, rd_solve_cg.cu): shared-memory GEMMs of the eigenbasis
// (DCT-II) diagonalisation of [alpha I - beta Lap_h] and a CTA-wide FP64 sum.
#pragma once

#include <cuda_runtime.h>

#include "rd_tc_ptx.cuh"

namespace rd {

constexpr int kSimtThreads = 256;

template <int N>
constexpr size_t simt_smem_bytes() {
  return (size_t)3 * N * (N + 1) * sizeof(float);
}

// acc[i][j] = sum_k A(ty + 16 i, k) B(k, tx + 16 j), A(m, k) = pa[m*SAM + k*SAK],
// B(k, n) = pb[k*SBK + n*SBN].
template <int N, int SAM, int SAK, int SBK, int SBN>
__device__ __forceinline__ void smem_gemm(const float* __restrict__ pa,
                                          const float* __restrict__ pb,
                                          float (&acc)[N / 16][N / 16], int ty,
                                          int tx) {
  constexpr int TM = N / 16;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int k = 0; k < N; ++k) {
    float av[TM], bv[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) av[i] = pa[(ty + 16 * i) * SAM + k * SAK];
#pragma unroll
    for (int j = 0; j < TM; ++j) bv[j] = pb[k * SBK + (tx + 16 * j) * SBN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

template <int N>
__device__ __forceinline__ void store_tile(float* W, const float (&acc)[N / 16][N / 16],
                                           int ty, int tx) {
  constexpr int TM = N / 16, NP = N + 1;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) W[(ty + 16 * i) * NP + tx + 16 * j] = acc[i][j];
}

// In place: W <- [alpha I - beta Lap_h]^-1 W.
template <int N>
__device__ __forceinline__ void implicit_solve_simt(float* W, const float* Cm,
                                                    float alpha, float beta,
                                                    const float (&mur)[N / 16],
                                                    const float (&muc)[N / 16],
                                                    int ty, int tx) {
  constexpr int TM = N / 16, NP = N + 1;
  float acc[TM][TM];
  // P[y][k] = sum_x W[y][x] C[k][x]
  smem_gemm<N, NP, 1, 1, NP>(W, Cm, acc, ty, tx);
  __syncthreads();
  store_tile<N>(W, acc, ty, tx);
  __syncthreads();
  // Q[l][k] = sum_y C[l][y] P[y][k];  S = Q / (alpha + beta (mu_l + mu_k))
  smem_gemm<N, NP, 1, NP, 1>(Cm, W, acc, ty, tx);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] *= tc::recip_nr(fmaf(beta, mur[i] + muc[j], alpha));
  __syncthreads();
  store_tile<N>(W, acc, ty, tx);
  __syncthreads();
  // W1[y][k] = sum_l C[l][y] S[l][k]
  smem_gemm<N, 1, NP, NP, 1>(Cm, W, acc, ty, tx);
  __syncthreads();
  store_tile<N>(W, acc, ty, tx);
  __syncthreads();
  // W[y][x] = sum_k W1[y][k] C[k][x]
  smem_gemm<N, NP, 1, NP, 1>(W, Cm, acc, ty, tx);
  __syncthreads();
  store_tile<N>(W, acc, ty, tx);
  __syncthreads();
}

// FP64 sum over the CTA; result valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

// FP64 sum over the CTA, returned to every thread.
__device__ __forceinline__ double cta_sum_all(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

}  // namespace rd
