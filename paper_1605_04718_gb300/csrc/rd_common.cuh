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
constexpr int kNPhys = RD_NPHYS;

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
  unsigned long long wait_ns;  // limit of the solve kernels' bounded waits
  int stall_step;  // >= 0: tensor-core issuers stall at this step (failure-path test aid)
  double ss_tol;   // > 0: solve to a steady state (time-derivative L2 norm below this)
  int ss_confirm;  // steady state: also require |w(2T) - w(T)| < ss_tol
  int param_map[kNParam];
  double fixed[kNPhys];   // model parameters not inferred
  double rho_T;           // RD_GROWTH_POLY4: rho(T)
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

// Full model parameter vector (a, b, d, gamma, r, p1, p2, p3) of inferred
// values th[0..P).
__device__ __forceinline__ void full_theta(const DevProblem& pb,
                                           const double* th, double out[kNPhys]) {
#pragma unroll
  for (int i = 0; i < kNPhys; ++i) out[i] = pb.fixed[i];
  for (int j = 0; j < pb.n_params; ++j) out[pb.param_map[j]] = th[j];
  if (pb.growth != RD_GROWTH_EXP) out[4] = 0.0;
}

// rho(t) and rho'(t) / rho(t) of the problem's growth law at time t (FP64;
// T = n_steps tau for the polynomial law of Example 1).
__device__ __forceinline__ void growth_at(const DevProblem& pb, const double th[kNPhys],
                                          double t, double& rho, double& q) {
  if (pb.growth == RD_GROWTH_POLY4) {
    const double T = (double)pb.n_steps * pb.tau;
    const double p1 = th[5], p2 = th[6], p3 = th[7];
    const double p4 = pb.rho_T - 1.0 - p1 - p2 - p3;
    const double s = t / T;
    rho = 1.0 + s * (p1 + s * (p2 + s * (p3 + s * p4)));
    q = (p1 + s * (2.0 * p2 + s * (3.0 * p3 + s * 4.0 * p4))) / T / rho;
  } else {
    rho = exp(th[4] * t);
    q = th[4];
  }
}

// growth_at with explicitly rounded FP64 operations (no fused multiply-add),
// in the order written, for the bit-reproducible semi-implicit step.
__device__ __forceinline__ void growth_at_rn(const DevProblem& pb, const double th[kNPhys],
                                             double t, double& rho, double& q) {
  if (pb.growth == RD_GROWTH_POLY4) {
    const double T = __dmul_rn((double)pb.n_steps, pb.tau);
    const double p1 = th[5], p2 = th[6], p3 = th[7];
    const double p4 = __dsub_rn(__dsub_rn(__dsub_rn(__dsub_rn(pb.rho_T, 1.0), p1), p2), p3);
    const double s = __ddiv_rn(t, T);
    rho = __dadd_rn(1.0, __dmul_rn(s, __dadd_rn(p1, __dmul_rn(s, __dadd_rn(p2,
              __dmul_rn(s, __dadd_rn(p3, __dmul_rn(s, p4))))))));
    const double drds = __dadd_rn(p1, __dmul_rn(s, __dadd_rn(__dmul_rn(2.0, p2),
              __dmul_rn(s, __dadd_rn(__dmul_rn(3.0, p3), __dmul_rn(__dmul_rn(s, 4.0), p4))))));
    q = __ddiv_rn(__ddiv_rn(drds, T), rho);
  } else {
    rho = exp(__dmul_rn(th[4], t));
    q = th[4];
  }
}

// Support of the polynomial growth law: rho > 0 at s = k / 1000, k = 0..1000.
__device__ __forceinline__ bool poly4_positive(const DevProblem& pb, const double th[kNPhys]) {
  const double p1 = th[5], p2 = th[6], p3 = th[7];
  const double p4 = pb.rho_T - 1.0 - p1 - p2 - p3;
  for (int k = 0; k <= 1000; ++k) {
    const double s = (double)k / 1000.0;
    if (!(1.0 + s * (p1 + s * (p2 + s * (p3 + s * p4))) > 0.0)) return false;
  }
  return true;
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
