// rd_solve_cg.cu -- forward solves by conjugate gradients on CUDA cores: the
// IMEX step with plain CG (the paper's linear solver) and the paper's
// semi-implicit step (Sec. 3.1.1, Example 1) in 2-D with preconditioned CG.
#include <cuda_runtime.h>
#include <math.h>

#include "rd_common.cuh"
#include "rd_internal.h"
#include "rd_simt_common.cuh"

namespace rd {

// ---------------------------------------------------------------------------
// 2-D, FP32, conjugate gradients on CUDA cores: one CTA of 256 threads per
// proposal with every vector resident in shared memory (rows padded to N + 1).
//
//  * RD_KERNEL_CG, IMEX step: each implicit system [alpha I - beta Lap_h] w =
//    r_w is solved by plain CG (the paper's own linear solver, Sec. 3.1.1)
//    from w^n, to a relative residual of 1e-6.  Vectors U, V, the rhs of v,
//    R, P, Q: N <= 96.
//  * RD_SCHEME_PICARD, the paper's semi-implicit step (Sec. 3.1.1,
//    Example 1): the reaction linearised with u^n, v^n makes the diagonal
//    node-dependent,
//      [D_u - beta_u Lap_h] u^{n+1} = u^n + tau gamma a,
//        D_u = 1 + tau m r + tau gamma (1 - u^n v^n),
//      [D_v - beta_v Lap_h] v^{n+1} = v^n + tau gamma b,
//        D_v = 1 + tau m r + tau gamma (u^n)^2,
//    solved by CG preconditioned with the eigenbasis solve of the operator
//    with the mean diagonal (the DCT-II diagonalisation, dense transforms from
//    shared memory).  Vectors U, V, the DCT matrix, the new u, R, Z, P, Q:
//    N <= 80.
// Fields are held as deviations from the initial-state mean as in the
// eigenbasis kernel; for the Picard step that turns the rhs into
// w^n - ref + tau gamma c + ref (1 - D).  Dot products are FP64.  A solve
// that reaches its iteration cap marks the proposal RD_P_NOT_CONVERGED.
// ---------------------------------------------------------------------------
constexpr int kCgMaxIter = 300;     // IMEX: plain CG
constexpr int kPcgMaxIter = 40;     // Picard: preconditioned CG
constexpr double kCgTol = 1e-6;     // relative residual

// Q = diag(dg) P - beta Lap_h P (5-point, Neumann by mirroring) at every
// point; dg(o) gives the diagonal at padded offset o.
template <int N, class Dg>
__device__ __forceinline__ void apply_op(const float* P, float* Q, float beta, Dg dg) {
  constexpr int NP = N + 1;
  for (int i = threadIdx.x; i < N * N; i += kSimtThreads) {
    const int y = i / N, x = i - y * N, o = y * NP + x;
    const float c = P[o];
    const float l = x > 0 ? P[o - 1] : c, r = x < N - 1 ? P[o + 1] : c;
    const float d = y > 0 ? P[o - NP] : c, u = y < N - 1 ? P[o + NP] : c;
    Q[o] = fmaf(dg(o), c, -beta * ((l + r) + (d + u) - 4.f * c));
  }
}

// CG on [diag(dg) - beta Lap_h] X = b from the X given, R = b - A X on entry;
// P, Q scratch; bb = |b|^2.  Returns false at the iteration cap.
template <int N, class Dg>
__device__ bool cg_solve(float* X, float* R, float* P, float* Q, float beta, Dg dg, double bb,
                         double* red) {
  constexpr int NP = N + 1;
  const int tid = threadIdx.x;
  double part = 0.0;
  for (int i = tid; i < N * N; i += kSimtThreads) {
    const int o = (i / N) * NP + i % N;
    P[o] = R[o];
    part += (double)R[o] * (double)R[o];
  }
  double rr = cta_sum_all(part, red);
  const double stop = kCgTol * kCgTol * bb;
  for (int it = 0; it < kCgMaxIter; ++it) {
    if (rr <= stop) return true;
    apply_op<N>(P, Q, beta, dg);
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      part += (double)P[o] * (double)Q[o];
    }
    const double pq = cta_sum_all(part, red);
    const float al = (float)(rr / pq);
    part = 0.0;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      X[o] = fmaf(al, P[o], X[o]);
      const float r = fmaf(-al, Q[o], R[o]);
      R[o] = r;
      part += (double)r * (double)r;
    }
    const double rr_new = cta_sum_all(part, red);
    const float be = (float)(rr_new / rr);
    rr = rr_new;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      P[o] = fmaf(be, P[o], R[o]);
    }
    __syncthreads();
  }
  return rr <= stop;
}

// Preconditioned CG on [diag(dg) - beta Lap_h] X = b, M = [dm I - beta
// Lap_h] solved in the eigenbasis; R = b on entry.  X = M^-1 b first.
template <int N, class Dg>
__device__ bool pcg_solve(float* X, float* R, float* Z, float* P, float* Q, const float* Cm,
                          float beta, float dm, Dg dg, const float (&mur)[N / 16],
                          const float (&muc)[N / 16], double* red) {
  constexpr int NP = N + 1;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double part = 0.0;
  for (int i = tid; i < N * N; i += kSimtThreads) {
    const int o = (i / N) * NP + i % N;
    Z[o] = R[o];
    part += (double)R[o] * (double)R[o];
  }
  const double bb = cta_sum_all(part, red);
  implicit_solve_simt<N>(Z, Cm, dm, beta, mur, muc, ty, tx);  // x0 = M^-1 b
  for (int i = tid; i < N * N; i += kSimtThreads) {
    const int o = (i / N) * NP + i % N;
    X[o] = Z[o];
  }
  __syncthreads();
  apply_op<N>(X, Q, beta, dg);
  __syncthreads();
  part = 0.0;
  for (int i = tid; i < N * N; i += kSimtThreads) {
    const int o = (i / N) * NP + i % N;
    const float r = R[o] - Q[o];
    R[o] = r;
    Z[o] = r;
    part += (double)r * (double)r;
  }
  double rr = cta_sum_all(part, red);
  const double stop = kCgTol * kCgTol * bb;
  if (rr <= stop) return true;
  implicit_solve_simt<N>(Z, Cm, dm, beta, mur, muc, ty, tx);
  part = 0.0;
  for (int i = tid; i < N * N; i += kSimtThreads) {
    const int o = (i / N) * NP + i % N;
    P[o] = Z[o];
    part += (double)R[o] * (double)Z[o];
  }
  double rz = cta_sum_all(part, red);
  for (int it = 0; it < kPcgMaxIter; ++it) {
    apply_op<N>(P, Q, beta, dg);
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      part += (double)P[o] * (double)Q[o];
    }
    const double pq = cta_sum_all(part, red);
    const float al = (float)(rz / pq);
    part = 0.0;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      X[o] = fmaf(al, P[o], X[o]);
      const float r = fmaf(-al, Q[o], R[o]);
      R[o] = r;
      Z[o] = r;
      part += (double)r * (double)r;
    }
    rr = cta_sum_all(part, red);
    if (rr <= stop) return true;
    implicit_solve_simt<N>(Z, Cm, dm, beta, mur, muc, ty, tx);
    part = 0.0;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      part += (double)R[o] * (double)Z[o];
    }
    const double rz_new = cta_sum_all(part, red);
    const float be = (float)(rz_new / rz);
    rz = rz_new;
    for (int i = tid; i < N * N; i += kSimtThreads) {
      const int o = (i / N) * NP + i % N;
      P[o] = fmaf(be, P[o], Z[o]);
    }
    __syncthreads();
  }
  return false;
}

template <int N, bool PICARD>
__device__ void solve2d_cg_item(const DevProblem& pb, const DevSize& S, const double th[kNPhys],
                                float* sm, double* red, double* phi_out, uint32_t* st_out,
                                float* fields_out) {
  constexpr int TM = N / 16, NP = N + 1, NPTS = N * N, VS = N * NP;
  float* U = sm;
  float* V = sm + VS;
  float* R = sm + 2 * VS;
  float* P = sm + 3 * VS;
  float* Q = sm + 4 * VS;
  float* W = sm + 5 * VS;  // IMEX: rhs of v; Picard: the new u
  float* Z = sm + 6 * VS;  // Picard only
  float* Cm = sm + 7 * VS; // Picard only
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const float ref_u = S.ref_u, ref_v = S.ref_v;
  for (int i = tid; i < NPTS; i += kSimtThreads) {
    const int y = i / N, x = i - y * N, o = y * NP + x;
    U[o] = S.u0f[i] - ref_u;
    V[o] = S.v0f[i] - ref_v;
    if (PICARD) Cm[o] = S.cmat[i];
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
  bool conv = true;
  int next_obs = 0;
  __syncthreads();
  for (int step = 0; step < pb.n_steps; ++step) {
    const double rho = exp(r * (double)step * tau);
    const double rho2inv = 1.0 / (rho * rho);
    const float alpha = (float)(1.0 + tau * 2.0 * r);  // m = 2 in 2-D
    const float bu = (float)(tau * rho2inv * h2inv);
    const float bv = (float)(tau * d * rho2inv * h2inv);
    if (!PICARD) {
      // IMEX: r_u - A u^n into R and the rhs r_v into W, from u^n, v^n
      const float cu = (float)(-tau * 2.0 * r * (double)ref_u);
      const float cv = (float)(-tau * 2.0 * r * (double)ref_v);
      auto dga = [alpha](int) { return alpha; };
      apply_op<N>(U, Q, bu, dga);
      __syncthreads();
      double part = 0.0;
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        const float du = U[o], dv = V[o];
        const float uu = ref_u + du, vv = ref_v + dv;
        const float u2v = uu * uu * vv;
        const float rhs_u = fmaf(ftg, fa - uu + u2v, du) + cu;
        W[o] = fmaf(ftg, fb - u2v, dv) + cv;
        R[o] = rhs_u - Q[o];
        part += (double)rhs_u * (double)rhs_u;
      }
      const double bbu = cta_sum_all(part, red);
      conv &= cg_solve<N>(U, R, P, Q, bu, dga, bbu, red);
      apply_op<N>(V, Q, bv, dga);
      __syncthreads();
      part = 0.0;
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        R[o] = W[o] - Q[o];
        part += (double)W[o] * (double)W[o];
      }
      const double bbv = cta_sum_all(part, red);
      conv &= cg_solve<N>(V, R, P, Q, bv, dga, bbv, red);
    } else {
      // Picard: diagonals from u^n, v^n; mean diagonal for the preconditioner
      auto dg_u = [=](int o) {
        return alpha + ftg * (1.f - (ref_u + U[o]) * (ref_v + V[o]));
      };
      auto dg_v = [=](int o) {
        const float uu = ref_u + U[o];
        return alpha + ftg * uu * uu;
      };
      double su = 0.0, sv = 0.0;
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        const float du = dg_u(o);
        su += du;
        sv += dg_v(o);
        R[o] = U[o] + ftg * fa + ref_u * (1.f - du);
      }
      const float mu_u = (float)(cta_sum_all(su, red) / NPTS);
      const float mu_v = (float)(cta_sum_all(sv, red) / NPTS);
      conv &= pcg_solve<N>(W, R, Z, P, Q, Cm, bu, mu_u, dg_u, mur, muc, red);
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        R[o] = V[o] + ftg * fb + ref_v * (1.f - dg_v(o));
      }
      __syncthreads();
      // v^{n+1} into V: its diagonal needs only u^n, which U still holds
      conv &= pcg_solve<N>(V, R, Z, P, Q, Cm, bv, mu_v, dg_v, mur, muc, red);
      for (int i = tid; i < NPTS; i += kSimtThreads) {
        const int o = (i / N) * NP + i % N;
        U[o] = W[o];
      }
      __syncthreads();
    }
    if (next_obs < S.n_obs && step + 1 == S.obs_steps[next_obs]) {
      const float* yo = S.yf + (size_t)next_obs * nfo * NPTS;
      int fo = 0;
      for (int f = 0; f < 2; ++f) {
        if (!(S.field_mask & (1 << f))) continue;
        const float* Wf = f ? V : U;
        const double ref = f ? (double)ref_v : (double)ref_u;
        const float* yf = yo + (size_t)fo * NPTS;
        for (int i = tid; i < NPTS; i += kSimtThreads) {
          const int y = i / N, x = i - y * N;
          const double w = ref + (double)Wf[y * NP + x];
          if (!(fabs(w) <= (double)w_max)) bad = 1;  // also catches NaN
          const double e = (double)yf[i] - w;
          phi += e * e;
        }
        ++fo;
      }
      ++next_obs;
    }
  }
  const double tot = cta_sum(phi, red);
  const int any_bad = __syncthreads_or(bad);
  if (tid == 0) {
    const uint32_t st = (any_bad ? (uint32_t)RD_P_NONFINITE : 0u) |
                        (conv ? 0u : (uint32_t)RD_P_NOT_CONVERGED);
    *st_out = st;
    *phi_out = st ? (double)INFINITY : tot * S.inv_two_sigma2;
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

#define RD_CG_CASE(NN)                                                              \
  case NN:                                                                          \
    if constexpr (NN <= NMAX)                                                       \
      solve2d_cg_item<NN, PICARD>(pb, S, th, sm, red, &phi[b], &status[b], fo);     \
    break;

template <int NMAX, bool PICARD>
__global__ void __launch_bounds__(kSimtThreads, 1)
    k_solve2d_cg(DevProblem pb, WorkQueue q, const double* theta, double* phi,
                 uint32_t* status, float* fields, size_t field_stride) {
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
      RD_CG_CASE(16)
      RD_CG_CASE(32)
      RD_CG_CASE(48)
      RD_CG_CASE(64)
      RD_CG_CASE(80)
      RD_CG_CASE(96)
      default:
        break;
    }
  }
}
#undef RD_CG_CASE

size_t cg_smem_bytes(int n, bool picard) {
  return (size_t)(picard ? 8 : 6) * n * (n + 1) * sizeof(float);
}

template <typename F>
static auto with_cg_kernel(int max_n, bool picard, F&& f) {
  if (picard) {
    if (max_n <= 32) return f((const void*)k_solve2d_cg<32, true>, 32);
    if (max_n <= 64) return f((const void*)k_solve2d_cg<64, true>, 64);
    return f((const void*)k_solve2d_cg<80, true>, 80);
  }
  if (max_n <= 32) return f((const void*)k_solve2d_cg<32, false>, 32);
  if (max_n <= 64) return f((const void*)k_solve2d_cg<64, false>, 64);
  return f((const void*)k_solve2d_cg<96, false>, 96);
}

bool cg_applicable(int n, bool picard) { return n <= (picard ? 80 : 96); }

cudaError_t setup_solve_cg(int max_n, bool picard) {
  return with_cg_kernel(max_n, picard, [&](const void* fn, int nmax) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cg_smem_bytes(nmax, picard));
  });
}

int grid_solve_cg(int max_n, bool picard, int n_sm) {
  return with_cg_kernel(max_n, picard, [&](const void* fn, int nmax) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSimtThreads,
                                                      cg_smem_bytes(nmax, picard)) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    return n_sm * per_sm;
  });
}

cudaError_t launch_solve_cg(const DevProblem& pb, const WorkQueue& q, const double* theta,
                            double* phi, uint32_t* status, void* fields, bool picard, int grid,
                            cudaStream_t st) {
  const double* th = theta;
  void* fo = fields;
  DevProblem pbv = pb;
  WorkQueue qv = q;
  size_t stride_v = (size_t)2 * pb.max_n * pb.max_n;
  return with_cg_kernel(pb.max_n, picard, [&](const void* fn, int nmax) {
    void* args[] = {&pbv, &qv, (void*)&th, &phi, &status, &fo, &stride_v};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSimtThreads), args,
                            cg_smem_bytes(nmax, picard), st);
  });
}

}  // namespace rd
