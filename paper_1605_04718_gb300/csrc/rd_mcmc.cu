// rd_mcmc.cu -- lock-step random-walk Metropolis chains on the device.
//
// One step of Algorithm 1 for every chain: draw a proposal from the symmetric
// Gaussian random walk, evaluate the prior, solve the forward problem for the
// proposals inside the prior's support, and accept with probability
// min(1, exp(-Phi(x_bar) + log mu0(x_bar) + Phi(x) - log mu0(x))).  The prior
// ratio is the paper's rule for a non-flat prior (eq. (bayes)); parameters
// stepped in log space carry the Jacobian theta in their density.
// Random numbers: Philox4x32-10 at counters (chain, step, 0|1, 0), key = seed;
// u_0..u_5 -> Box-Muller normals, u_6 -> acceptance uniform (stage-1 uniform
// under delayed acceptance), u_7 -> stage-2 uniform.
//
// Algorithm 2 (multi-proposal parallel Metropolis-Hastings, Sec. 2.1): see
// k_pmh_propose / k_pmh_select below.
//
// Delayed acceptance (Christen & Fox 2005, not in the paper): a surrogate
// Phi~ screens each proposal; only stage-1 survivors are solved, and the
// second test min(1, exp(Phi(x) - Phi(x_bar) + Phi~(x_bar) - Phi~(x))) keeps
// the chain's stationary distribution the exact posterior.
#include <cuda_runtime.h>
#include <math.h>

#include "rd_common.cuh"
#include "rd_internal.h"

namespace rd {

struct ChainView {
  int C, P;
  uint64_t seed;
  uint32_t first;  // global index of chain 0 in the Philox counters
  double chol[kNParam * kNParam];  // lower-triangular proposal factor
  double* theta;
  double* phi;
  double* phit;
  double* lp;
  const int* size_idx;
  double* prop;
  double* prop_phi;
  double* prop_phit;
  double* prop_lp;
  uint32_t* prop_status;
  double* samples;
  unsigned long long* counters;
  int* ctl;
  int N;  // proposals per chain and step of Algorithm 2 (0: Algorithm 1)
  double* pmh_prop;
  double* pmh_phi;
  double* pmh_lp;
  uint32_t* pmh_status;
};

static ChainView view_of(const rd_chains* c) {
  ChainView v;
  v.C = c->C;
  v.P = c->P;
  v.seed = c->seed;
  v.first = c->first_chain;
  for (int j = 0; j < kNParam * kNParam; ++j) v.chol[j] = c->chol[j];
  v.theta = c->theta;
  v.phi = c->phi;
  v.phit = c->phit;
  v.lp = c->lp;
  v.size_idx = c->size_idx;
  v.prop = c->prop;
  v.prop_phi = c->prop_phi;
  v.prop_phit = c->prop_phit;
  v.prop_lp = c->prop_lp;
  v.prop_status = c->prop_status;
  v.samples = c->samples;
  v.counters = c->counters;
  v.ctl = c->ctl;
  v.N = c->pmh_n;
  v.pmh_prop = c->pmh_prop;
  v.pmh_phi = c->pmh_phi;
  v.pmh_lp = c->pmh_lp;
  v.pmh_status = c->pmh_status;
  return v;
}

// The Turing space of the Schnakenberg kinetics (eq. (turing)) at the
// homogeneous steady state: f_u + g_v < 0, f_u g_v - f_v g_u > 0,
// d f_u + g_v > 0, (d f_u + g_v)^2 - 4 d (f_u g_v - f_v g_u) > 0 with
// f_u = (b - a)/(b + a), g_v = -(a + b)^2, f_u g_v - f_v g_u = (a + b)^2.
__device__ bool in_turing_space(const DevProblem& pb, const double* th) {
  double full[kNPhys];
  full_theta(pb, th, full);
  const double a = full[0], b = full[1], d = full[2];
  const double s = a + b;
  if (!(s > 0.0)) return false;
  const double fu = (b - a) / s, gv = -s * s, det = s * s;
  const double e = d * fu + gv;
  return fu + gv < 0.0 && det > 0.0 && e > 0.0 && e * e - 4.0 * d * det > 0.0;
}

// log mu0(theta) + sum of log |d theta / d eta| over log-stepped parameters;
// -inf outside the support.  Constants are dropped.
__device__ double log_prior_eta(const DevProblem& pb, const double* th) {
  double lp = 0.0;
  for (int j = 0; j < pb.n_params; ++j) {
    const double t = th[j];
    double lpj;
    if (pb.prior_kind[j] == RD_PRIOR_UNIFORM) {
      lpj = (t >= pb.prior_p0[j] && t <= pb.prior_p1[j]) ? 0.0 : -(double)INFINITY;
    } else {
      if (t > 0.0) {
        const double lt = log(t);
        const double z = (lt - log(pb.prior_p0[j])) / pb.prior_p1[j];
        lpj = -lt - 0.5 * z * z;
      } else {
        lpj = -(double)INFINITY;
      }
    }
    if (pb.step_space[j] == RD_STEP_LOG) lpj = lpj + log(t > 0.0 ? t : 1.0);
    lp += lpj;
  }
  if (pb.turing && !in_turing_space(pb, th)) lp = -(double)INFINITY;
  if (pb.growth == RD_GROWTH_POLY4 && isfinite(lp)) {
    double full[kNPhys];
    full_theta(pb, th, full);
    if (!poly4_positive(pb, full)) lp = -(double)INFINITY;
  }
  return lp;
}

__device__ __forceinline__ void chain_normals(const double u[8], double xi[6]) {
  const double two_pi = 6.283185307179586476925286766559;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double rad = sqrt(-2.0 * log(u[2 * j]));
    const double ang = two_pi * u[2 * j + 1];
    xi[2 * j] = rad * cos(ang);
    xi[2 * j + 1] = rad * sin(ang);
  }
}

__device__ __forceinline__ void queue_push(const WorkQueue& q, int s, int item) {
  const int i = atomicAdd(&q.counts[s], 1);
  q.items[(size_t)s * q.capacity + i] = item;
}

__global__ void k_chain_init(DevProblem pb, WorkQueue q, ChainView v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  double th[kNParam];
  for (int j = 0; j < v.P; ++j) th[j] = v.theta[(size_t)c * v.P + j];
  const double lp = log_prior_eta(pb, th);
  v.lp[c] = lp;
  if (isfinite(lp)) {
    v.phi[c] = (double)INFINITY;  // pending until the solve writes it
    v.prop_status[c] = RD_P_NOT_SOLVED;
    queue_push(q, v.size_idx[c], c);
  } else {
    v.phi[c] = (double)INFINITY;
    v.prop_status[c] = RD_P_OUT_OF_SUPPORT;
  }
}

// Stage-1 rejection marker (internal; never returned to callers).
constexpr uint32_t kStage1Reject = 0x100u;

// push = 0 (delayed acceptance): candidates are queued after stage 1.
__global__ void k_chain_propose(DevProblem pb, WorkQueue q, ChainView v, int push) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  const uint32_t step = (uint32_t)v.ctl[0];
  double u[8], xi[6];
  chain_uniforms(v.seed, v.first + (uint32_t)c, step, u);
  chain_normals(u, xi);
  double th[kNParam];
  for (int j = 0; j < v.P; ++j) {
    const double t = v.theta[(size_t)c * v.P + j];
    double inc = 0.0;  // (L xi)_j
    for (int i = 0; i <= j; ++i) inc += v.chol[j * kNParam + i] * xi[i];
    double tb;
    if (pb.step_space[j] == RD_STEP_LOG)
      tb = exp(log(t) + inc);
    else
      tb = t + inc;
    th[j] = tb;
    v.prop[(size_t)c * v.P + j] = tb;
  }
  const double lp = log_prior_eta(pb, th);
  v.prop_lp[c] = lp;
  if (isfinite(lp)) {
    v.prop_status[c] = 0u;
    if (push) {  // pending until the solve writes Phi and the status
      v.prop_status[c] = RD_P_NOT_SOLVED;
      v.prop_phi[c] = (double)INFINITY;
      queue_push(q, v.size_idx[c], c);
    }
  } else {
    v.prop_status[c] = RD_P_OUT_OF_SUPPORT;
    v.prop_phi[c] = (double)INFINITY;
  }
}

// Stage 1 of delayed acceptance: accept to stage 2 with probability
// min(1, exp(-Phi~(x_bar) + lp(x_bar) + Phi~(x) - lp(x))); survivors are queued
// for the exact solve.
__global__ void k_chain_stage1(WorkQueue q, ChainView v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  if (v.prop_status[c] != 0u) return;  // outside the prior's support
  double u[8];
  chain_uniforms(v.seed, v.first + (uint32_t)c, (uint32_t)v.ctl[0], u);
  const double la1 = (-v.prop_phit[c] + v.prop_lp[c]) - (-v.phit[c] + v.lp[c]);
  if (log(u[6]) < la1) {
    v.prop_status[c] = RD_P_NOT_SOLVED;  // pending until the solve writes it
    v.prop_phi[c] = (double)INFINITY;
    queue_push(q, v.size_idx[c], c);
  } else {
    v.prop_status[c] = kStage1Reject;
    v.prop_phi[c] = (double)INFINITY;
  }
}

// Stage 2: exact test on the survivors, then record the state.
__global__ void k_chain_accept_da(ChainView v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  const int slot = v.ctl[1];
  double u[8];
  chain_uniforms(v.seed, v.first + (uint32_t)c, (uint32_t)v.ctl[0], u);
  const uint32_t st = v.prop_status[c];
  const bool pass1 = (st != RD_P_OUT_OF_SUPPORT && st != kStage1Reject);
  bool acc = false;
  if (st == 0u) {
    const double la2 = (v.phi[c] - v.prop_phi[c]) + (v.prop_phit[c] - v.phit[c]);
    acc = log(u[7]) < la2;
  }
  if (acc) {
    for (int j = 0; j < v.P; ++j)
      v.theta[(size_t)c * v.P + j] = v.prop[(size_t)c * v.P + j];
    v.phi[c] = v.prop_phi[c];
    v.lp[c] = v.prop_lp[c];
    v.phit[c] = v.prop_phit[c];
  }
  for (int j = 0; j < v.P; ++j)
    v.samples[((size_t)slot * v.P + j) * v.C + c] = v.theta[(size_t)c * v.P + j];
  v.counters[c] += 1ull;
  v.counters[(size_t)v.C + c] += pass1 ? 1ull : 0ull;
  v.counters[(size_t)2 * v.C + c] += acc ? 1ull : 0ull;
  v.counters[(size_t)3 * v.C + c] += pass1 ? 1ull : 0ull;
}

__global__ void k_chain_accept(DevProblem pb, ChainView v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  const uint32_t step = (uint32_t)v.ctl[0];
  const int slot = v.ctl[1];
  double u[8];
  chain_uniforms(v.seed, v.first + (uint32_t)c, step, u);
  const uint32_t st = v.prop_status[c];
  bool acc = false;
  if (st == 0u) {
    const double la = (-v.prop_phi[c] + v.prop_lp[c]) - (-v.phi[c] + v.lp[c]);
    acc = log(u[6]) < la;
  }
  if (acc) {
    for (int j = 0; j < v.P; ++j)
      v.theta[(size_t)c * v.P + j] = v.prop[(size_t)c * v.P + j];
    v.phi[c] = v.prop_phi[c];
    v.lp[c] = v.prop_lp[c];
  }
  for (int j = 0; j < v.P; ++j)
    v.samples[((size_t)slot * v.P + j) * v.C + c] = v.theta[(size_t)c * v.P + j];
  v.counters[c] += 1ull;
  v.counters[(size_t)v.C + c] += (st != RD_P_OUT_OF_SUPPORT) ? 1ull : 0ull;
  v.counters[(size_t)2 * v.C + c] += acc ? 1ull : 0ull;
  v.counters[(size_t)3 * v.C + c] += (st != RD_P_OUT_OF_SUPPORT) ? 1ull : 0ull;
}

// ---------------------------------------------------------------- Algorithm 2
// Proposal t (1..N) of chain c: z = x + L xi_0 (the auxiliary point, random
// numbers of point 0), proposal = z + L xi_t (point t), both in step space.
__global__ void k_pmh_propose(DevProblem pb, WorkQueue q, ChainView v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.C * v.N) return;
  const int c = i / v.N, t = i - c * v.N + 1;
  const uint32_t step = (uint32_t)v.ctl[0];
  double u[8], xi0[6], xi[6];
  chain_uniforms(v.seed, v.first + (uint32_t)c, step, u, 0u);
  chain_normals(u, xi0);
  chain_uniforms(v.seed, v.first + (uint32_t)c, step, u, (uint32_t)t);
  chain_normals(u, xi);
  double th[kNParam];
  for (int j = 0; j < v.P; ++j) {
    const double x = v.theta[(size_t)c * v.P + j];
    double inc0 = 0.0, inc = 0.0;
    for (int k = 0; k <= j; ++k) {
      inc0 += v.chol[j * kNParam + k] * xi0[k];
      inc += v.chol[j * kNParam + k] * xi[k];
    }
    const bool lg = pb.step_space[j] == RD_STEP_LOG;
    const double eta = (lg ? log(x) : x) + inc0 + inc;
    th[j] = lg ? exp(eta) : eta;
    v.pmh_prop[(size_t)i * v.P + j] = th[j];
  }
  const double lp = log_prior_eta(pb, th);
  v.pmh_lp[i] = lp;
  if (isfinite(lp)) {
    v.pmh_status[i] = RD_P_NOT_SOLVED;  // pending until the solve writes it
    v.pmh_phi[i] = (double)INFINITY;
    queue_push(q, v.size_idx[c], i);
  } else {
    v.pmh_status[i] = RD_P_OUT_OF_SUPPORT;
    v.pmh_phi[i] = (double)INFINITY;
  }
}

// The N+1 points' stationary distribution and the N draws of one chain.
__global__ void k_pmh_select(ChainView v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.C) return;
  constexpr int M = RD_PMH_MAX_PROPOSALS + 1;
  const int N = v.N, n1 = N + 1;
  const uint32_t step = (uint32_t)v.ctl[0];
  const int slot = v.ctl[1];
  // log target of each point (-inf outside the support or for a failed solve)
  double lt[M];
  lt[0] = (isfinite(v.phi[c]) && isfinite(v.lp[c])) ? -v.phi[c] + v.lp[c] : -(double)INFINITY;
  int n_in = 0;
  for (int t = 1; t <= N; ++t) {
    const size_t i = (size_t)c * N + t - 1;
    const bool ok = v.pmh_status[i] == 0u && isfinite(v.pmh_phi[i]);
    n_in += v.pmh_status[i] != RD_P_OUT_OF_SUPPORT;
    lt[t] = ok ? -v.pmh_phi[i] + v.pmh_lp[i] : -(double)INFINITY;
  }
  // M = A^T - I with the last equation replaced by sum(pi) = 1, where
  // A(i, j) = min(1, exp(lt_j - lt_i)) / N (j != i), A(i, i) = 1 - row rest
  double a[M][M + 1];
  for (int i = 0; i < n1; ++i) {
    double rest = 0.0;
    for (int j = 0; j < n1; ++j) {
      if (j == i) continue;
      double r;
      if (lt[j] == -(double)INFINITY)
        r = 0.0;
      else if (lt[i] == -(double)INFINITY)
        r = 1.0;
      else
        r = fmin(1.0, exp(lt[j] - lt[i]));
      a[j][i] = r / N;  // transposed
      rest += r / N;
    }
    a[i][i] = (1.0 - rest) - 1.0;
  }
  for (int j = 0; j < n1; ++j) {
    a[n1 - 1][j] = 1.0;
    a[j][n1] = 0.0;
  }
  a[n1 - 1][n1] = 1.0;
  // Gaussian elimination with partial pivoting, then back substitution
  for (int k = 0; k < n1; ++k) {
    int piv = k;
    for (int i = k + 1; i < n1; ++i)
      if (fabs(a[i][k]) > fabs(a[piv][k])) piv = i;
    if (piv != k)
      for (int j = k; j <= n1; ++j) {
        const double tmp = a[k][j];
        a[k][j] = a[piv][j];
        a[piv][j] = tmp;
      }
    for (int i = k + 1; i < n1; ++i) {
      const double f = a[i][k] / a[k][k];
      for (int j = k; j <= n1; ++j) a[i][j] -= f * a[k][j];
    }
  }
  double pi[M];
  for (int i = n1 - 1; i >= 0; --i) {
    double s = a[i][n1];
    for (int j = i + 1; j < n1; ++j) s -= a[i][j] * pi[j];
    pi[i] = s / a[i][i];
  }
  double cum[M];
  double acc_sum = 0.0;
  for (int i = 0; i < n1; ++i) {
    acc_sum += pi[i];
    cum[i] = acc_sum;
  }
  // N draws; draw t (1..N) uses u_6 of point t
  int moved = 0, last = 0;
  for (int t = 1; t <= N; ++t) {
    double u[8];
    chain_uniforms(v.seed, v.first + (uint32_t)c, step, u, (uint32_t)t);
    const double x = u[6] * cum[n1 - 1];
    int k = 0;
    while (k < N && !(x < cum[k])) ++k;
    moved += k != 0;
    last = k;
    for (int j = 0; j < v.P; ++j) {
      const double th = k == 0 ? v.theta[(size_t)c * v.P + j]
                               : v.pmh_prop[((size_t)c * N + k - 1) * v.P + j];
      v.samples[((size_t)(slot + t - 1) * v.P + j) * v.C + c] = th;
    }
  }
  if (last != 0) {
    const size_t i = (size_t)c * N + last - 1;
    for (int j = 0; j < v.P; ++j) v.theta[(size_t)c * v.P + j] = v.pmh_prop[i * v.P + j];
    v.phi[c] = v.pmh_phi[i];
    v.lp[c] = v.pmh_lp[i];
  }
  v.counters[c] += (unsigned long long)N;
  v.counters[(size_t)v.C + c] += (unsigned long long)n_in;
  v.counters[(size_t)2 * v.C + c] += (unsigned long long)moved;
  v.counters[(size_t)3 * v.C + c] += (unsigned long long)n_in;
}

// Ends one MCMC step: advances the step counter and the sample ring by the
// step's samples, and empties the work lists for the next step.
__global__ void k_chain_advance(WorkQueue q, int* ctl, int rows) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl[0] += 1;
    ctl[1] += rows;
  }
  if (threadIdx.x < 2 * kMaxSizes) q.counts[threadIdx.x] = 0;  // counts, pops
}

cudaError_t launch_chain_init(rd_chains* c) {
  rd_problem* p = c->pb;
  WorkQueue q = make_queue(p);
  ChainView v = view_of(c);
  cudaError_t e = cudaMemsetAsync(q.counts, 0, 2 * kMaxSizes * sizeof(int), p->stream);
  if (e != cudaSuccess) return e;
  k_chain_init<<<(c->C + 127) / 128, 128, 0, p->stream>>>(p->dev, q, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = launch_solve(p, c->theta, c->phi, c->prop_status, nullptr);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(q.counts, 0, 2 * kMaxSizes * sizeof(int), p->stream);
}

// Enqueues one full MCMC step (propose, exact solves, accept, advance).
cudaError_t launch_chain_step(rd_chains* c) {
  rd_problem* p = c->pb;
  WorkQueue q = make_queue(p);
  ChainView v = view_of(c);
  const int blocks = (c->C + 127) / 128;
  // the work lists may hold counts from an rd_evaluate_batch call in between
  cudaError_t e = cudaMemsetAsync(q.counts, 0, 2 * kMaxSizes * sizeof(int), p->stream);
  if (e != cudaSuccess) return e;
  if (c->pmh_n > 0) {  // Algorithm 2
    const int n = c->C * c->pmh_n;
    k_pmh_propose<<<(n + 127) / 128, 128, 0, p->stream>>>(p->dev, q, v);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_solve(p, c->pmh_prop, c->pmh_phi, c->pmh_status, nullptr);
    if (e != cudaSuccess) return e;
    k_pmh_select<<<blocks, 128, 0, p->stream>>>(v);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_chain_advance<<<1, 32, 0, p->stream>>>(q, c->ctl, c->pmh_n);
    return cudaGetLastError();
  }
  const int da = c->sur != nullptr;
  k_chain_propose<<<blocks, 128, 0, p->stream>>>(p->dev, q, v, da ? 0 : 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (da) {
    e = mlp::predict(c->sur, c->C, c->prop, c->prop_phit, p->stream);
    if (e != cudaSuccess) return e;
    k_chain_stage1<<<blocks, 128, 0, p->stream>>>(q, v);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  e = launch_solve(p, c->prop, c->prop_phi, c->prop_status, nullptr);
  if (e != cudaSuccess) return e;
  if (da)
    k_chain_accept_da<<<blocks, 128, 0, p->stream>>>(v);
  else
    k_chain_accept<<<blocks, 128, 0, p->stream>>>(p->dev, v);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_chain_advance<<<1, 32, 0, p->stream>>>(q, c->ctl, 1);
  return cudaGetLastError();
}

}  // namespace rd
