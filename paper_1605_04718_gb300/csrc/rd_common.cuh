// rd_common.cuh -- device-side problem description, work queues, Philox.
// Internal to the library; the public interface is include/rdbayes.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rdbayes.h"

namespace rd {

constexpr int kMaxSizes = RD_MAX_SIZES;
constexpr int kMaxObs = RD_MAX_OBS;
constexpr int kNParam = RD_NPARAM;

// One grid size of a problem: its initial state, observations and the
// constant tables of its implicit solve.
struct DevSize {
  int n;                    // grid points per side
  int npts;                 // n (1-D) or n*n (2-D)
  int n_obs;                // observation times
  int obs_steps[kMaxObs];   // step indices 1..n_steps, increasing
  int field_mask;           // bit 0: u observed, bit 1: v observed
  double inv_two_sigma2;    // 1 / (2 sigma^2)
  const float* u0f;         // FP32 initial state [npts] (2-D)
  const float* v0f;
  const double* u0d;        // FP64 initial state [npts] (1-D)
  const double* v0d;
  const float* yf;          // FP32 observations [n_obs][fields][npts] (2-D)
  const double* yd;         // FP64 observations (1-D)
  float ref_u, ref_v;       // reference state: spatial mean of the initial state
  const float* cmat;        // orthonormal DCT-II matrix C[k][i], FP32 [n][n]
  const float* mu;          // 4 sin^2(pi k / (2n)), FP32 [n]
};

struct DevProblem {
  int dim;
  int n_sizes;
  int n_steps;
  int precision;
  int growth;
  int n_params;
  int max_n;
  double tau;
  double w_max;
  int param_map[kNParam];
  double fixed[kNParam];
  int prior_kind[kNParam];
  double prior_p0[kNParam];
  double prior_p1[kNParam];
  int step_space[kNParam];
  int turing;  // prior restricted to the Turing space of (a, b, d)
  int scheme;  // RD_SCHEME_*: 1-D step with the reaction explicit or linearised implicit
  DevSize sz[kMaxSizes];
};

// Work queue for the persistent solve kernels: one list of proposal indices
// per grid size, each with an append counter and a pop counter.  Lives in the
// library's device workspace; counts/pops are zeroed before each fill.
struct WorkQueue {
  int* items;   // [n_sizes][capacity]
  int capacity;
  int* counts;  // [kMaxSizes] appended
  int* pops;    // [kMaxSizes] popped
  int order[kMaxSizes];  // size indices, largest grid first
  int n_sizes;
};

// Full parameter vector (a, b, d, gamma, r) of inferred values th[0..P).
__device__ __forceinline__ void full_theta(const DevProblem& pb,
                                           const double* th, double out[5]) {
#pragma unroll
  for (int i = 0; i < kNParam; ++i) out[i] = pb.fixed[i];
  for (int j = 0; j < pb.n_params; ++j) out[pb.param_map[j]] = th[j];
  if (!pb.growth) out[4] = 0.0;
}

// Pops the next work item; returns the proposal index or -1 when every list
// is exhausted.  *size_out receives the item's size index.
__device__ __forceinline__ int queue_pop(const WorkQueue& q, int* size_out) {
  for (int k = 0; k < q.n_sizes; ++k) {
    int s = q.order[k];
    int cnt = *((volatile int*)&q.counts[s]);
    if (*((volatile int*)&q.pops[s]) >= cnt) continue;
    int i = atomicAdd(&q.pops[s], 1);
    if (i < cnt) {
      *size_out = s;
      return q.items[(size_t)s * q.capacity + i];
    }
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplications mixed with the counter and key words, the key
// advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c[0];
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Eight uniforms in (0, 1) of chain `chain` at MCMC step `step`: the words of
// the Philox blocks at counters (chain, step, 0, point) and (chain, step, 1,
// point) with key (seed low, seed high), each mapped to (w + 1/2) 2^-32.
// point = 0 except for the points of a multi-proposal step (Algorithm 2).
__device__ __forceinline__ void chain_uniforms(uint64_t seed, uint32_t chain,
                                               uint32_t step, double u[8],
                                               uint32_t point = 0u) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t c0[4] = {chain, step, 0u, point};
  uint32_t c1[4] = {chain, step, 1u, point};
  philox4x32_10(c0, k0, k1);
  philox4x32_10(c1, k0, k1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u[i] = ((double)c0[i] + 0.5) * (1.0 / 4294967296.0);
    u[4 + i] = ((double)c1[i] + 0.5) * (1.0 / 4294967296.0);
  }
}

}  // namespace rd
