// rd_solve_simt.cu -- forward solve G(p) and log-likelihood Phi(p; y) on CUDA
// cores: the 1-D FP64 Thomas path and the 2-D FP32 eigenbasis path.
//
// Both follow the IMEX Euler step of Sec. 3.1.1 with the reaction explicit
// and diffusion plus the dilution term of eq. (schnakenberg) implicit:
//   r_u = u + tau gamma (a - u + u^2 v),   r_v = v + tau gamma (b - u^2 v)
//   [(1 + tau m r) I - tau D rho_n^-2 Lap_h] w^{n+1} = r_w,  D = 1 (u), d (v)
// with the cell-centred Neumann Laplacian, and accumulate
// Phi = sum (y - w)^2 / (2 sigma^2) (eq. (logl)) at the observation steps.
// Growth factors rho_n = exp(r n tau) are formed in FP64 once per step and
// rounded once to the field precision.
//
// The persistent kernels pop proposals from per-size work lists (largest grid
// first) until the lists are empty, so one launch covers any mix of sizes.
#include <cuda_runtime.h>
#include <math.h>

#include "rd_common.cuh"
#include "rd_internal.h"
#include "rd_simt_common.cuh"
#include "rd_tc_ptx.cuh"

namespace rd {

// ---------------------------------------------------------------------------
// 1-D, FP64, one thread per proposal: Thomas algorithm on the tridiagonal
// Neumann matrix (diagonal alpha + 2 beta, alpha + beta in the two boundary
// rows, off-diagonals -beta).
// ---------------------------------------------------------------------------
// Factors of the Thomas elimination for [alpha I - beta Lap_h]: inverse
// pivots inv[i] and modified super-diagonal cp[i] = -beta inv[i].
template <int NMAX>
__device__ __forceinline__ void thomas_factors(int n, double alpha, double beta,
                                               double (&cp)[NMAX], double (&inv)[NMAX]) {
  double prev = 0.0;
  for (int i = 0; i < n; ++i) {
    const double diag = alpha + ((i == 0 || i == n - 1) ? beta : 2.0 * beta);
    const double den = diag + beta * prev;
    inv[i] = 1.0 / den;
    cp[i] = -beta * inv[i];
    prev = cp[i];
  }
}

// Steady-state mode (pb.ss_tol > 0, fixed domain, Sec. 3.1.2): the step loop
// stops at the first step T whose discrete time derivative has
//   (h^dim sum over both fields ((w^{T} - w^{T-1}) / tau)^2)^(1/2) < ss_tol,
// at most n_steps; the single observation is taken at T.  With ss_confirm the
// solve goes on to 2T and requires (h^dim sum (w(2T) - w(T))^2)^(1/2) < ss_tol;
// the reported state stays w(T).  Either failure is RD_P_NOT_CONVERGED.
// steps_out (may be null) receives T (0 when none was reached).
template <int NMAX>
__device__ void solve1d_item(const DevProblem& pb, const DevSize& S,
                             const double th[kNPhys], double* phi_out,
                             uint32_t* st_out, double* fields_out, int* steps_out) {
  double u[NMAX], v[NMAX], ru[NMAX], rv[NMAX];
  double cu[NMAX], cv[NMAX], iu[NMAX], iv[NMAX];
  double up[NMAX], vp[NMAX];  // steady-state mode: previous step, then w(T)
  const int n = S.n;
  for (int i = 0; i < n; ++i) {
    u[i] = S.u0d[i];
    v[i] = S.v0d[i];
  }
  const double a = th[0], b = th[1], d = th[2], g = th[3], r = th[4];
  const double tau = pb.tau, h2inv = (double)n * n, tg = tau * g;
  const int nfo = (S.field_mask & 1) + ((S.field_mask >> 1) & 1);
  const bool grow = (r != 0.0) || pb.growth == RD_GROWTH_POLY4;
  double phi = 0.0;
  bool bad = false;
  int next_obs = 0;
  double alpha = 1.0, bu = tau * h2inv, bv = tau * d * h2inv;
  thomas_factors<NMAX>(n, alpha, bu, cu, iu);
  thomas_factors<NMAX>(n, alpha, bv, cv, iv);
  const bool steady = pb.ss_tol > 0.0;
  int t_ss = 0, phase = 0;  // steady state: 0 seek T, 1 confirm to 2T
  bool conv = !steady;
  for (int step = 0; steady || step < pb.n_steps; ++step) {
    if (steady) {
      if (phase == 0 && step >= pb.n_steps) break;
      if (phase == 0)
        for (int i = 0; i < n; ++i) {
          up[i] = u[i];
          vp[i] = v[i];
        }
    }
    if (pb.scheme == RD_SCHEME_PICARD) {
      // the paper's semi-implicit step: the reaction linearised with u^n, v^n
      // and implicit, so the diagonal varies by node (Thomas, eliminated in
      // place: cu / cv hold c'_i, ru / rv hold d'_i).  Every operation is an
      // explicitly rounded FP64 one (no fused multiply-add) in a fixed order:
      // on a growing domain at large gamma the pattern reached after millions
      // of steps depends on the rounding of each step, so the step is kept
      // reproducible to the bit.
      double rho, q;  // rho_n and rho'/rho at t_n, FP64
      growth_at_rn(pb, th, __dmul_rn((double)step, tau), rho, q);
      if (!(rho > 0.0)) {
        bad = true;
        break;
      }
      const double al = __dadd_rn(1.0, __dmul_rn(__dmul_rn(tau, 1.0), q));  // m = 1 in 1-D
      const double h = __ddiv_rn(1.0, (double)n), hh = __dmul_rn(h, h);
      const double rr = __dmul_rn(rho, rho);
      const double bu1 = __ddiv_rn(__ddiv_rn(__dmul_rn(tau, 1.0), rr), hh);
      const double bv1 = __ddiv_rn(__ddiv_rn(__dmul_rn(tau, d), rr), hh);
      for (int i = 0; i < n; ++i) {
        const double aui = __dadd_rn(al, __dmul_rn(tg, __dsub_rn(1.0, __dmul_rn(u[i], v[i]))));
        const double avi = __dadd_rn(al, __dmul_rn(__dmul_rn(tg, u[i]), u[i]));
        const double rU = __dadd_rn(u[i], __dmul_rn(tg, a));
        const double rV = __dadd_rn(v[i], __dmul_rn(tg, b));
        const double edge = (i == 0 || i == n - 1) ? 1.0 : 2.0;
        const double du = __dadd_rn(__dadd_rn(aui, __dmul_rn(edge, bu1)),
                                    i > 0 ? __dmul_rn(bu1, cu[i - 1]) : 0.0);
        const double dv = __dadd_rn(__dadd_rn(avi, __dmul_rn(edge, bv1)),
                                    i > 0 ? __dmul_rn(bv1, cv[i - 1]) : 0.0);
        cu[i] = (i < n - 1) ? __ddiv_rn(-bu1, du) : 0.0;
        cv[i] = (i < n - 1) ? __ddiv_rn(-bv1, dv) : 0.0;
        ru[i] = __ddiv_rn(__dadd_rn(rU, i > 0 ? __dmul_rn(bu1, ru[i - 1]) : 0.0), du);
        rv[i] = __ddiv_rn(__dadd_rn(rV, i > 0 ? __dmul_rn(bv1, rv[i - 1]) : 0.0), dv);
      }
      u[n - 1] = ru[n - 1];
      v[n - 1] = rv[n - 1];
      for (int i = n - 2; i >= 0; --i) {
        u[i] = __dsub_rn(ru[i], __dmul_rn(cu[i], u[i + 1]));
        v[i] = __dsub_rn(rv[i], __dmul_rn(cv[i], v[i + 1]));
      }
    } else {
    if (grow) {  // rho_n = rho(t_n): the matrix changes every step
      double rho, q;
      growth_at(pb, th, (double)step * tau, rho, q);
      if (!(rho > 0.0)) {
        bad = true;
        break;
      }
      alpha = 1.0 + tau * 1.0 * q;  // m = 1 in 1-D
      bu = tau / (rho * rho) * h2inv;
      bv = tau * d / (rho * rho) * h2inv;
      thomas_factors<NMAX>(n, alpha, bu, cu, iu);
      thomas_factors<NMAX>(n, alpha, bv, cv, iv);
    }
    // explicit reaction fused with the forward elimination
    double pu = 0.0, pv = 0.0;
    for (int i = 0; i < n; ++i) {
      const double uu = u[i], vv = v[i];
      const double u2v = uu * uu * vv;
      const double rU = uu + tg * (a - uu + u2v);
      const double rV = vv + tg * (b - u2v);
      pu = (rU + bu * pu) * iu[i];
      pv = (rV + bv * pv) * iv[i];
      ru[i] = pu;
      rv[i] = pv;
    }
    u[n - 1] = ru[n - 1];
    v[n - 1] = rv[n - 1];
    for (int i = n - 2; i >= 0; --i) {
      u[i] = ru[i] - cu[i] * u[i + 1];
      v[i] = rv[i] - cv[i] * v[i + 1];
    }
    }
    bool observe = !steady && next_obs < S.n_obs && step + 1 == S.obs_steps[next_obs];
    if (steady) {
      double s2 = 0.0;
      for (int i = 0; i < n; ++i)
        s2 += (u[i] - up[i]) * (u[i] - up[i]) + (v[i] - vp[i]) * (v[i] - vp[i]);
      const double h = 1.0 / n;
      if (phase == 0) {
        if (sqrt(h * s2) / tau < pb.ss_tol) {
          t_ss = step + 1;
          observe = true;
          if (!pb.ss_confirm) {
            conv = true;
          } else {
            phase = 1;
            for (int i = 0; i < n; ++i) {
              up[i] = u[i];
              vp[i] = v[i];
            }
          }
        }
      } else if (step + 1 == 2 * t_ss) {
        conv = sqrt(h * s2) < pb.ss_tol;
        for (int i = 0; i < n; ++i) {
          u[i] = up[i];
          v[i] = vp[i];
        }
      }
    }
    if (observe) {
      const double* yo = S.yd + (size_t)next_obs * nfo * n;
      int fo = 0;
      for (int f = 0; f < 2; ++f) {
        if (!(S.field_mask & (1 << f))) continue;
        const double* w = f ? v : u;
        for (int i = 0; i < n; ++i) {
          if (!isfinite(w[i]) || fabs(w[i]) > pb.w_max) bad = true;
          const double e = yo[(size_t)fo * n + i] - w[i];
          phi += e * e;
        }
        ++fo;
      }
      ++next_obs;
    }
    if (steady && ((phase == 0 && t_ss > 0) || (phase == 1 && step + 1 == 2 * t_ss))) break;
  }
  const uint32_t st = (bad ? (uint32_t)RD_P_NONFINITE : 0u) |
                      (conv ? 0u : (uint32_t)RD_P_NOT_CONVERGED);
  *st_out = st;
  *phi_out = st ? (double)INFINITY : phi * S.inv_two_sigma2;
  if (steps_out) *steps_out = t_ss;
  if (fields_out) {
    for (int i = 0; i < n; ++i) {
      fields_out[i] = u[i];
      fields_out[n + i] = v[i];
    }
  }
}

template <int NMAX>
__global__ void k_solve1d_f64(DevProblem pb, WorkQueue q, const double* theta,
                              double* phi, uint32_t* status, double* fields,
                              size_t field_stride, int* steps_out) {
  for (;;) {
    int s;
    const int b = queue_pop(q, &s);
    if (b < 0) break;
    double th[kNPhys];
    full_theta(pb, theta + (size_t)b * pb.n_params, th);
    double* fo = fields ? fields + (size_t)b * field_stride : nullptr;
    solve1d_item<NMAX>(pb, pb.sz[s], th, &phi[b], &status[b], fo,
                       steps_out ? &steps_out[b] : nullptr);
  }
}

// ---------------------------------------------------------------------------
// 2-D, FP32 fields, one CTA of 256 threads per proposal with u, v and the DCT
// matrix resident in shared memory for the whole time loop.
//
// The fields are held as deviations du = u - u_ref, dv = v - v_ref from the
// spatial mean of the initial state.  The solve is linear and constants are
// in the kernel of the Laplacian, so the step for the deviations is
//   [alpha I - beta Lap_h] dw^{n+1} = dw^n + tau gamma kin(u, v) + (1 - alpha) w_ref,
// the same step as for w.  FP32 rounding then acts on |dw| (about 0.01 while
// a Turing pattern grows from the initial noise) instead of on |w| ~ 1,
// which keeps the small unstable modes accurate.
//
// Implicit solve by diagonalisation in the Neumann eigenbasis (orthonormal
// DCT-II, C[k][i] = c_k cos(pi k (i + 1/2) / N)):
//   P = W C^T, Q = C P, S = Q / (alpha + beta (mu_l + mu_k)), W1 = C^T S,
//   W = W1 C,   mu_k = 4 sin^2(pi k / (2N)), beta = tau D / (rho^2 h^2).
// Each product is an N x N x N GEMM from shared memory with 16 x 16 threads,
// thread (ty, tx) owning rows ty + 16 i and columns tx + 16 j.  Rows are
// padded to N + 1 floats so that every operand load is conflict-free.
// ---------------------------------------------------------------------------
// STEADY: the steady-state mode of solve1d_item (rd_solve_simt.cu, above),
// with the previous step (then w(T)) in two more shared-memory arrays.
template <int N, bool STEADY>
__device__ void solve2d_simt_item(const DevProblem& pb, const DevSize& S,
                                  const double th[kNPhys], float* sm, double* red,
                                  double* phi_out, uint32_t* st_out,
                                  float* fields_out, int* steps_out) {
  constexpr int TM = N / 16, NP = N + 1, NPTS = N * N;
  float* U = sm;  // u - ref_u
  float* V = sm + N * NP;  // v - ref_v
  float* Cm = sm + 2 * N * NP;
  float* Up = sm + 3 * N * NP;  // STEADY only
  float* Vp = sm + 4 * N * NP;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const float ref_u = S.ref_u, ref_v = S.ref_v;
  for (int i = tid; i < NPTS; i += kSimtThreads) {
    const int r = i / N, c = i - r * N;
    Cm[r * NP + c] = S.cmat[i];
    U[r * NP + c] = S.u0f[i] - ref_u;
    V[r * NP + c] = S.v0f[i] - ref_v;
  }
  float mur[TM], muc[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    mur[i] = S.mu[ty + 16 * i];
    muc[i] = S.mu[tx + 16 * i];
  }
  const double d = th[2], r = th[4], tau = pb.tau;
  const float fa = (float)th[0], fb = (float)th[1], ftg = (float)(tau * th[3]);
  const float w_max = (float)pb.w_max;
  const double h2inv = (double)N * N;
  const int nfo = (S.field_mask & 1) + ((S.field_mask >> 1) & 1);
  double phi = 0.0;
  int bad = 0;
  int next_obs = 0;
  int t_ss = 0, phase = 0;  // steady state: 0 seek T, 1 confirm to 2T
  bool conv = !STEADY;
  __syncthreads();
  for (int step = 0; STEADY || step < pb.n_steps; ++step) {
    if (STEADY && phase == 0) {
      if (step >= pb.n_steps) break;
      for (int i = tid; i < NPTS; i += kSimtThreads) {  // the reaction pass below
        const int o = (i / N) * NP + i % N;            // reads the same points
        Up[o] = U[o];
        Vp[o] = V[o];
      }
    }
    const double rho = exp(r * (double)step * tau);
    const double rho2inv = 1.0 / (rho * rho);
    const float alpha = (float)(1.0 + tau * 2.0 * r);  // m = 2 in 2-D
    const float bu = (float)(tau * rho2inv * h2inv);
    const float bv = (float)(tau * d * rho2inv * h2inv);
    const float cu = (float)(-tau * 2.0 * r * (double)ref_u);  // (1 - alpha) ref
    const float cv = (float)(-tau * 2.0 * r * (double)ref_v);
    for (int i = tid; i < NPTS; i += kSimtThreads) {
      const int y = i / N, x = i - y * N, o = y * NP + x;
      const float du = U[o], dv = V[o];
      const float uu = ref_u + du, vv = ref_v + dv;
      const float u2v = uu * uu * vv;
      U[o] = fmaf(ftg, fa - uu + u2v, du) + cu;
      V[o] = fmaf(ftg, fb - u2v, dv) + cv;
    }
    __syncthreads();
    implicit_solve_simt<N>(U, Cm, alpha, bu, mur, muc, ty, tx);
    implicit_solve_simt<N>(V, Cm, alpha, bv, mur, muc, ty, tx);
    bool observe = !STEADY && next_obs < S.n_obs && step + 1 == S.obs_steps[next_obs];
    bool stop = false;
    if (STEADY) {
      double part = 0.0;
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        const double eu = (double)U[o] - (double)Up[o], ev = (double)V[o] - (double)Vp[o];
        part += eu * eu + ev * ev;
      }
      const double h2 = 1.0 / ((double)N * N), s2 = cta_sum_all(part, red);
      if (phase == 0) {
        if (sqrt(h2 * s2) / tau < pb.ss_tol) {
          t_ss = step + 1;
          observe = true;
          if (!pb.ss_confirm) {
            conv = true;
            stop = true;
          } else {
            phase = 1;
            for (int i = tid; i < NPTS; i += kSimtThreads) {
              const int o = (i / N) * NP + i % N;
              Up[o] = U[o];
              Vp[o] = V[o];
            }
          }
        }
      } else if (step + 1 == 2 * t_ss) {
        conv = sqrt(h2 * s2) < pb.ss_tol;
        stop = true;
        for (int i = tid; i < NPTS; i += kSimtThreads) {
          const int o = (i / N) * NP + i % N;
          U[o] = Up[o];
          V[o] = Vp[o];
        }
      }
      __syncthreads();
    }
    if (observe) {
      const float* yo = S.yf + (size_t)next_obs * nfo * NPTS;
      int fo = 0;
      for (int f = 0; f < 2; ++f) {
        if (!(S.field_mask & (1 << f))) continue;
        const float* W = f ? V : U;
        const double ref = f ? (double)ref_v : (double)ref_u;
        const float* yf = yo + (size_t)fo * NPTS;
        for (int i = tid; i < NPTS; i += kSimtThreads) {
          const int y = i / N, x = i - y * N;
          const double w = ref + (double)W[y * NP + x];
          if (!(fabs(w) <= (double)w_max)) bad = 1;  // also catches NaN
          const double e = (double)yf[i] - w;
          phi += e * e;
        }
        ++fo;
      }
      ++next_obs;
    }
    if (stop) break;
  }
  const double tot = cta_sum(phi, red);
  const int any_bad = __syncthreads_or(bad);
  if (tid == 0) {
    const uint32_t st = (any_bad ? (uint32_t)RD_P_NONFINITE : 0u) |
                        (conv ? 0u : (uint32_t)RD_P_NOT_CONVERGED);
    *st_out = st;
    *phi_out = st ? (double)INFINITY : tot * S.inv_two_sigma2;
    if (steps_out) *steps_out = t_ss;
  }
  if (fields_out) {
    for (int i = tid; i < NPTS; i += kSimtThreads) {
      const int y = i / N, x = i - y * N;
      fields_out[i] = ref_u + U[y * NP + x];
      fields_out[NPTS + i] = ref_v + V[y * NP + x];
    }
  }
  __syncthreads();
}

#define RD_SIMT_CASE(NN)                                                      \
  case NN:                                                                    \
    if constexpr (NN <= NMAX)                                                 \
      solve2d_simt_item<NN, STEADY>(pb, S, th, sm, red, &phi[b], &status[b], fo, \
                                    steps_out ? &steps_out[b] : nullptr);     \
    break;

// NMAX: largest grid of the problem; sizes up to NMAX share one launch.
template <int NMAX, int MINB, bool STEADY>
__global__ void __launch_bounds__(kSimtThreads, MINB)
    k_solve2d_simt(DevProblem pb, WorkQueue q, const double* theta, double* phi,
                   uint32_t* status, float* fields, size_t field_stride, int* steps_out) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[kSimtThreads / 32];
  __shared__ int s_item, s_size;
  for (;;) {
    if (threadIdx.x == 0) {
      int s = 0;
      s_item = queue_pop(q, &s);
      s_size = s;
    }
    __syncthreads();
    const int b = s_item, s = s_size;
    __syncthreads();
    if (b < 0) break;
    double th[kNPhys];
    full_theta(pb, theta + (size_t)b * pb.n_params, th);
    const DevSize& S = pb.sz[s];
    float* fo = fields ? fields + (size_t)b * field_stride : nullptr;
    switch (S.n) {
      RD_SIMT_CASE(16)
      RD_SIMT_CASE(32)
      RD_SIMT_CASE(48)
      RD_SIMT_CASE(64)
      RD_SIMT_CASE(80)
      RD_SIMT_CASE(96)
      RD_SIMT_CASE(112)
      RD_SIMT_CASE(128)
      default:
        break;
    }
  }
}
#undef RD_SIMT_CASE

size_t simt2d_smem_bytes(int n, bool steady) {
  return (size_t)(steady ? 5 : 3) * n * (n + 1) * sizeof(float);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
__global__ void k_fill_queue(WorkQueue q, int B, const int* size_idx,
                             double* phi, uint32_t* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int s = size_idx ? size_idx[b] : 0;
  if (s < 0 || s >= q.n_sizes) {
    phi[b] = (double)INFINITY;
    status[b] = RD_P_OUT_OF_SUPPORT;
    return;
  }
  // pending until a solve kernel writes the result
  phi[b] = (double)INFINITY;
  status[b] = RD_P_NOT_SOLVED;
  const int i = atomicAdd(&q.counts[s], 1);
  q.items[(size_t)s * q.capacity + i] = b;
}

cudaError_t launch_fill_queue(const WorkQueue& q, int B, const int* size_idx,
                              double* phi, uint32_t* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(q.counts, 0, 2 * kMaxSizes * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (B > 0) k_fill_queue<<<(B + 255) / 256, 256, 0, st>>>(q, B, size_idx, phi, status);
  return cudaGetLastError();
}

// Kernel variant for a problem whose largest grid is max_n: the 1-D bucket
// (local arrays of 64 or 256 doubles) or the 2-D NMAX instantiation with the
// CTAs-per-SM hint that its shared memory allows (steady-state mode: the
// variant with the previous step's copy, N <= 96).
template <typename F>
static auto with_simt_kernel(int dim, int max_n, bool steady, F&& f) {
  if (dim == 1) {
    if (max_n <= 64) return f((const void*)k_solve1d_f64<64>, 0);
    return f((const void*)k_solve1d_f64<256>, 0);
  }
  if (steady) {
    if (max_n <= 32) return f((const void*)k_solve2d_simt<32, 2, true>, 32);
    if (max_n <= 64) return f((const void*)k_solve2d_simt<64, 2, true>, 64);
    return f((const void*)k_solve2d_simt<96, 1, true>, 96);
  }
  if (max_n <= 32) return f((const void*)k_solve2d_simt<32, 4, false>, 32);
  if (max_n <= 64) return f((const void*)k_solve2d_simt<64, 4, false>, 64);
  if (max_n <= 96) return f((const void*)k_solve2d_simt<96, 2, false>, 96);
  return f((const void*)k_solve2d_simt<128, 1, false>, 128);
}

cudaError_t launch_solve_simt(const DevProblem& pb, const WorkQueue& q,
                              const double* theta, double* phi, uint32_t* status,
                              void* fields, int grid, cudaStream_t st, int* steps_out) {
  const size_t stride = (size_t)2 * (pb.dim == 1 ? pb.max_n : pb.max_n * pb.max_n);
  const double* th = theta;
  void* fo = fields;
  DevProblem pbv = pb;
  WorkQueue qv = q;
  size_t stride_v = stride;
  int* so = steps_out;
  const bool steady = pb.ss_tol > 0.0;
  return with_simt_kernel(pb.dim, pb.max_n, steady, [&](const void* fn, int nmax) {
    const size_t smem = pb.dim == 1 ? 0 : simt2d_smem_bytes(nmax, steady);
    const int threads = pb.dim == 1 ? 128 : kSimtThreads;
    void* args[] = {&pbv, &qv, (void*)&th, &phi, &status, &fo, &stride_v, &so};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st);
  });
}

cudaError_t setup_solve_simt(int dim, int max_n, bool steady) {
  return with_simt_kernel(dim, max_n, steady, [&](const void* fn, int nmax) {
    if (dim == 1) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)simt2d_smem_bytes(nmax, steady));
  });
}

int grid_solve_simt(int dim, int max_n, int n_sm, bool steady) {
  return with_simt_kernel(dim, max_n, steady, [&](const void* fn, int nmax) {
    int per_sm = 0;
    const size_t smem = dim == 1 ? 0 : simt2d_smem_bytes(nmax, steady);
    const int threads = dim == 1 ? 128 : kSimtThreads;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    return n_sm * per_sm;
  });
}

}  // namespace rd
