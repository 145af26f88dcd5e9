// rd_api.cu -- the extern "C" entry points declared in include/rdbayes.h.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rd_common.cuh"
#include "rd_internal.h"

namespace rd {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

#define RD_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      rd::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return RD_ECUDA;                                                     \
    }                                                                      \
  } while (0)

#define RD_CHECK(cond, code, msg) \
  do {                            \
    if (!(cond)) {                \
      rd::set_error(msg);         \
      return code;                \
    }                             \
  } while (0)

WorkQueue make_queue(const rd_problem* p) {
  WorkQueue q;
  q.items = p->ws.queue_items;
  q.capacity = p->ws.capacity;
  q.counts = p->ws.queue_counters;
  q.pops = p->ws.queue_counters + kMaxSizes;
  q.n_sizes = p->desc.n_sizes;
  std::vector<int> order(p->desc.n_sizes);
  for (int s = 0; s < p->desc.n_sizes; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return p->desc.nx[x] > p->desc.nx[y]; });
  for (int k = 0; k < kMaxSizes; ++k) q.order[k] = k < (int)order.size() ? order[k] : 0;
  return q;
}

bool uses_tc(const rd_problem* p) {
  if (p->desc.dim != 2) return false;
  for (int s = 0; s < p->desc.n_sizes; ++s)
    if (kernel_for_size(p, s) == RD_KERNEL_TC_STACKED ||
        kernel_for_size(p, s) == RD_KERNEL_TC_RESIDENT)
      return true;
  return false;
}

int kernel_for_size(const rd_problem* p, int s) {
  if (p->desc.dim != 2) return RD_KERNEL_SIMT;
  const int k = p->kernel_of_size[s];
  if (k != RD_KERNEL_DEFAULT) return k;
  if (p->desc.solver == RD_SOLVER_DCT_SIMT) return RD_KERNEL_SIMT;
  return p->desc.nx[s] == 128 ? RD_KERNEL_TC_RESIDENT : RD_KERNEL_TC_STACKED;
}

// Persistent CTAs of a kernel kind's launch when every SM holds as many as fit.
static int grid_max_of(const rd_problem* p, int kind) {
  switch (kind) {
    case RD_KERNEL_TC_RESIDENT: return grid_solve_tc128(p->n_sm);
    case RD_KERNEL_TC_STACKED: return grid_solve_tc(p->dev.max_n, p->n_sm);
    case RD_KERNEL_CG: return grid_solve_cg(p->dev.max_n, false, p->n_sm);
    default: return grid_solve_simt(p->desc.dim, p->dev.max_n, p->n_sm);
  }
}

cudaError_t launch_solve_queue(rd_problem* p, const WorkQueue& q, const double* theta,
                               double* phi, uint32_t* status, void* fields, cudaStream_t st,
                               int* steps_out) {
  if (p->dev.ss_tol > 0.0)  // steady-state mode: every size, CUDA cores, one launch
    return launch_solve_simt(p->dev, q, theta, phi, status, fields,
                             grid_solve_simt(p->desc.dim, p->dev.max_n, p->n_sm, true), st,
                             steps_out);
  if (p->desc.dim == 2 && p->dev.scheme == RD_SCHEME_PICARD)  // every size: one launch
    return launch_solve_cg(p->dev, q, theta, phi, status, fields, true,
                           grid_solve_cg(p->dev.max_n, true, p->n_sm), st);
  static const int kinds[4] = {RD_KERNEL_TC_RESIDENT, RD_KERNEL_TC_STACKED, RD_KERNEL_SIMT,
                               RD_KERNEL_CG};
  for (int kind : kinds) {
    WorkQueue sub = q;  // the sizes of this kernel, largest grid first
    sub.n_sizes = 0;
    int want = 0;  // CTAs per SM: the largest any of these sizes asks for
    for (int k = 0; k < q.n_sizes; ++k)
      if (kernel_for_size(p, q.order[k]) == kind) {
        sub.order[sub.n_sizes++] = q.order[k];
        want = std::max(want, p->ctas_per_sm[q.order[k]]);
      }
    if (sub.n_sizes == 0) continue;
    const int gmax = grid_max_of(p, kind);
    const int grid = (want > 0 && want * p->n_sm < gmax) ? want * p->n_sm : gmax;
    cudaError_t e;
    if (kind == RD_KERNEL_TC_RESIDENT)
      e = launch_solve_tc128(p->dev, sub, theta, phi, status, fields, grid, p->ws.err, st);
    else if (kind == RD_KERNEL_TC_STACKED)
      e = launch_solve_tc(p->dev, sub, theta, phi, status, fields, grid, p->ws.err, st);
    else if (kind == RD_KERNEL_CG)
      e = launch_solve_cg(p->dev, sub, theta, phi, status, fields, false, grid, st);
    else
      e = launch_solve_simt(p->dev, sub, theta, phi, status, fields, grid, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_solve_on(rd_problem* p, const double* theta, double* phi,
                            uint32_t* status, void* fields, cudaStream_t st) {
  return launch_solve_queue(p, make_queue(p), theta, phi, status, fields, st);
}

cudaError_t launch_solve(rd_problem* p, const double* theta, double* phi,
                         uint32_t* status, void* fields) {
  return launch_solve_on(p, theta, phi, status, fields, p->stream);
}

static rd_status ensure_capacity(rd_problem* p, int need) {
  if (need <= p->ws.capacity) return RD_OK;
  int cap = std::max(need, std::max(1024, 2 * p->ws.capacity));
  RD_CUDA(cudaStreamSynchronize(p->stream));
  if (p->ws.queue_items) RD_CUDA(cudaFree(p->ws.queue_items));
  p->ws.queue_items = nullptr;
  RD_CUDA(cudaMalloc(&p->ws.queue_items, sizeof(int) * (size_t)cap * p->desc.n_sizes));
  p->ws.capacity = cap;
  p->generation++;
  return RD_OK;
}

static rd_status validate_desc(const rd_problem_desc* d) {
  RD_CHECK(d, RD_EINVAL, "desc is NULL");
  RD_CHECK(d->dim == 1 || d->dim == 2, RD_EINVAL, "dim must be 1 or 2");
  RD_CHECK(d->n_sizes >= 1 && d->n_sizes <= RD_MAX_SIZES, RD_EINVAL,
           "n_sizes must be in 1..4");
  for (int s = 0; s < d->n_sizes; ++s) {
    const int n = d->nx[s];
    if (d->dim == 1) {
      RD_CHECK(n >= 2 && n <= 256, RD_EINVAL, "1-D grid size must be in 2..256");
    } else {
      RD_CHECK(n >= 16 && n <= 128 && n % 16 == 0, RD_EINVAL,
               "2-D grid size must be a multiple of 16 in 16..128");
    }
  }
  RD_CHECK(d->tau > 0 && isfinite(d->tau), RD_EINVAL, "tau must be positive");
  RD_CHECK(d->n_steps >= 1, RD_EINVAL, "n_steps must be >= 1");
  RD_CHECK((d->dim == 1 && d->precision == RD_PREC_F64) ||
               (d->dim == 2 && d->precision == RD_PREC_F32),
           RD_EINVAL, "precision must be F64 for 1-D and F32 for 2-D problems");
  RD_CHECK(d->solver == RD_SOLVER_AUTO || (d->dim == 1 && d->solver == RD_SOLVER_THOMAS) ||
               (d->dim == 2 && (d->solver == RD_SOLVER_DCT_SIMT || d->solver == RD_SOLVER_DCT_TC)),
           RD_EINVAL, "solver not available for this dimension");
  RD_CHECK(d->n_params >= 1 && d->n_params <= RD_NPARAM, RD_EINVAL,
           "n_params must be in 1..5");
  RD_CHECK(d->growth >= RD_GROWTH_NONE && d->growth <= RD_GROWTH_POLY4, RD_EINVAL,
           "unknown growth law");
  RD_CHECK(d->growth != RD_GROWTH_POLY4 || d->dim == 1, RD_EINVAL,
           "the polynomial growth law is built for 1-D problems");
  RD_CHECK(d->growth != RD_GROWTH_POLY4 || (d->rho_T > 0 && isfinite(d->rho_T)), RD_EINVAL,
           "the polynomial growth law needs rho_T > 0");
  for (int j = 0; j < d->n_params; ++j) {
    const int hi = d->growth == RD_GROWTH_POLY4 ? RD_NPHYS : RD_NPARAM;
    RD_CHECK(d->param_map[j] >= 0 && d->param_map[j] < hi, RD_EINVAL,
             "param_map entry out of range");
    for (int k = 0; k < j; ++k)
      RD_CHECK(d->param_map[k] != d->param_map[j], RD_EINVAL, "param_map repeats a parameter");
    RD_CHECK(d->prior_kind[j] == RD_PRIOR_UNIFORM || d->prior_kind[j] == RD_PRIOR_LOGNORMAL,
             RD_EINVAL, "unknown prior kind");
    if (d->prior_kind[j] == RD_PRIOR_UNIFORM)
      RD_CHECK(d->prior_p0[j] <= d->prior_p1[j], RD_EINVAL, "uniform prior needs lo <= hi");
    else
      RD_CHECK(d->prior_p0[j] > 0 && d->prior_p1[j] > 0, RD_EINVAL,
               "log-normal prior needs median > 0 and sigma > 0");
    RD_CHECK(d->step_space[j] == RD_STEP_LINEAR || d->step_space[j] == RD_STEP_LOG,
             RD_EINVAL, "unknown step space");
  }
  return RD_OK;
}

}  // namespace rd

using namespace rd;

extern "C" {

const char* rd_last_error(void) { return g_err.c_str(); }

rd_status rd_problem_create(const rd_problem_desc* desc, void* cuda_stream,
                            rd_problem** out) {
  RD_CHECK(out, RD_EINVAL, "out is NULL");
  *out = nullptr;
  rd_status vs = validate_desc(desc);
  if (vs != RD_OK) return vs;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("no CUDA device available");
    return RD_ECUDA;
  }
  rd_problem* p = new rd_problem();
  p->desc = *desc;
  if (p->desc.w_max <= 0) p->desc.w_max = 100.0;
  p->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    set_error("cannot query the CUDA device");
    return RD_ECUDA;
  }
  {
    const rd_status ns = noalloc_prepare(p->device);
    if (ns != RD_OK) {
      delete p;
      return ns;
    }
  }
  DevProblem& dv = p->dev;
  memset(&dv, 0, sizeof(dv));
  dv.dim = desc->dim;
  dv.n_sizes = desc->n_sizes;
  dv.n_steps = desc->n_steps;
  dv.precision = desc->precision;
  dv.growth = desc->growth;
  dv.n_params = desc->n_params;
  dv.tau = desc->tau;
  dv.w_max = p->desc.w_max;
  dv.wait_ns = 4000000000ull;
  dv.stall_step = -1;
  for (int j = 0; j < kNParam; ++j) {
    dv.param_map[j] = desc->param_map[j];
    dv.fixed[j] = desc->fixed[j];
    dv.prior_kind[j] = desc->prior_kind[j];
    dv.prior_p0[j] = desc->prior_p0[j];
    dv.prior_p1[j] = desc->prior_p1[j];
    dv.step_space[j] = desc->step_space[j];
  }
  for (int j = 0; j < 3; ++j) dv.fixed[kNParam + j] = desc->fixed_poly[j];
  dv.rho_T = desc->rho_T;
  dv.max_n = 0;
  const double pi = 3.14159265358979323846264338327950288;
  for (int s = 0; s < desc->n_sizes; ++s) {
    const int n = desc->nx[s];
    dv.max_n = std::max(dv.max_n, n);
    dv.sz[s].n = n;
    dv.sz[s].npts = desc->dim == 1 ? n : n * n;
    if (desc->dim == 2) {
      std::vector<float> c((size_t)n * n), mu(n);
      for (int k = 0; k < n; ++k) {
        const double ck = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
        for (int i = 0; i < n; ++i) c[(size_t)k * n + i] = (float)(ck * cos(pi * k * (i + 0.5) / n));
        const double sk = sin(pi * k / (2.0 * n));
        mu[k] = (float)(4.0 * sk * sk);
      }
      if (cudaMalloc(&p->cmat[s], sizeof(float) * c.size()) != cudaSuccess ||
          cudaMalloc(&p->mu[s], sizeof(float) * mu.size()) != cudaSuccess ||
          cudaMemcpy(p->cmat[s], c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(p->mu[s], mu.data(), sizeof(float) * mu.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        rd_problem_destroy(p);
        set_error("device allocation of solver tables failed");
        return RD_ENOMEM;
      }
      dv.sz[s].cmat = p->cmat[s];
      dv.sz[s].mu = p->mu[s];
    }
  }
  if (cudaMalloc(&p->ws.queue_counters, sizeof(int) * 2 * kMaxSizes) != cudaSuccess ||
      cudaMemset(p->ws.queue_counters, 0, sizeof(int) * 2 * kMaxSizes) != cudaSuccess ||
      cudaMalloc(&p->ws.err, sizeof(int)) != cudaSuccess ||
      cudaMemset(p->ws.err, 0, sizeof(int)) != cudaSuccess) {
    rd_problem_destroy(p);
    set_error("device allocation of the work queue failed");
    return RD_ENOMEM;
  }
  if (ensure_capacity(p, 1024) != RD_OK) {
    rd_problem_destroy(p);
    return RD_ENOMEM;
  }
  bool has128 = false;
  for (int k = 0; k < desc->n_sizes; ++k) has128 = has128 || (desc->dim == 2 && desc->nx[k] == 128);
  if (setup_solve_simt(desc->dim, dv.max_n) != cudaSuccess ||
      (desc->dim == 2 && setup_solve_tc(dv.max_n) != cudaSuccess) ||
      (desc->dim == 2 && cg_applicable(dv.max_n, false) &&
       setup_solve_cg(dv.max_n, false) != cudaSuccess) ||
      (has128 && setup_solve_tc128() != cudaSuccess)) {
    rd_problem_destroy(p);
    set_error("cannot configure the solve kernels' shared memory");
    return RD_ECUDA;
  }
  *out = p;
  return RD_OK;
}

rd_status rd_problem_destroy(rd_problem* p) {
  if (!p) return RD_OK;
  cudaStreamSynchronize(p->stream);
  for (int s = 0; s < RD_MAX_SIZES; ++s) {
    cudaFree(p->ic[s]);
    cudaFree(p->obs[s]);
    cudaFree(p->cmat[s]);
    cudaFree(p->mu[s]);
  }
  cudaFree(p->ws.queue_items);
  cudaFree(p->ws.queue_counters);
  cudaFree(p->ws.err);
  cudaFree(p->h2d_theta);
  cudaFree(p->h2d_size);
  cudaFree(p->d2h_phi);
  cudaFree(p->d2h_status);
  delete p;
  return RD_OK;
}

rd_status rd_set_stream(rd_problem* p, void* cuda_stream) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  p->stream = (cudaStream_t)cuda_stream;
  return RD_OK;
}

rd_status rd_set_initial_state(rd_problem* p, int size_idx, const double* u0,
                               const double* v0) {
  RD_CHECK(p && u0 && v0, RD_EINVAL, "NULL argument");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  DevSize& S = p->dev.sz[size_idx];
  const size_t npts = (size_t)S.npts;
  RD_CUDA(cudaStreamSynchronize(p->stream));
  cudaFree(p->ic[size_idx]);
  p->ic[size_idx] = nullptr;
  if (p->desc.precision == RD_PREC_F64) {
    RD_CUDA(cudaMalloc(&p->ic[size_idx], sizeof(double) * 2 * npts));
    double* d = (double*)p->ic[size_idx];
    RD_CUDA(cudaMemcpy(d, u0, sizeof(double) * npts, cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(d + npts, v0, sizeof(double) * npts, cudaMemcpyHostToDevice));
    S.u0d = d;
    S.v0d = d + npts;
  } else {
    // FP32 fields are stored as deviations from the spatial mean of the
    // initial state (see the 2-D solve kernel)
    double mu_u = 0.0, mu_v = 0.0;
    for (size_t i = 0; i < npts; ++i) {
      mu_u += u0[i];
      mu_v += v0[i];
    }
    S.ref_u = (float)(mu_u / (double)npts);
    S.ref_v = (float)(mu_v / (double)npts);
    std::vector<float> h(2 * npts);
    for (size_t i = 0; i < npts; ++i) {
      h[i] = (float)u0[i];
      h[npts + i] = (float)v0[i];
    }
    RD_CUDA(cudaMalloc(&p->ic[size_idx], sizeof(float) * 2 * npts));
    float* d = (float*)p->ic[size_idx];
    RD_CUDA(cudaMemcpy(d, h.data(), sizeof(float) * 2 * npts, cudaMemcpyHostToDevice));
    S.u0f = d;
    S.v0f = d + npts;
  }
  p->ic_set[size_idx] = true;
  p->generation++;
  return RD_OK;
}

rd_status rd_set_observations(rd_problem* p, int size_idx, int n_times,
                              const int* obs_steps, int field_mask,
                              const double* y, double sigma) {
  RD_CHECK(p && obs_steps && y, RD_EINVAL, "NULL argument");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  RD_CHECK(n_times >= 1 && n_times <= RD_MAX_OBS, RD_EINVAL, "n_times must be in 1..8");
  RD_CHECK(field_mask >= 1 && field_mask <= 3, RD_EINVAL, "field_mask must be 1, 2 or 3");
  RD_CHECK(sigma > 0 && isfinite(sigma), RD_EINVAL, "sigma must be positive");
  for (int o = 0; o < n_times; ++o) {
    RD_CHECK(obs_steps[o] >= 1 && obs_steps[o] <= p->desc.n_steps, RD_EINVAL,
             "observation step outside 1..n_steps");
    RD_CHECK(o == 0 || obs_steps[o] > obs_steps[o - 1], RD_EINVAL,
             "observation steps must increase");
  }
  DevSize& S = p->dev.sz[size_idx];
  const int nf = (field_mask & 1) + ((field_mask >> 1) & 1);
  const size_t nval = (size_t)n_times * nf * S.npts;
  RD_CUDA(cudaStreamSynchronize(p->stream));
  cudaFree(p->obs[size_idx]);
  p->obs[size_idx] = nullptr;
  if (p->desc.precision == RD_PREC_F64) {
    RD_CUDA(cudaMalloc(&p->obs[size_idx], sizeof(double) * nval));
    RD_CUDA(cudaMemcpy(p->obs[size_idx], y, sizeof(double) * nval, cudaMemcpyHostToDevice));
    S.yd = (const double*)p->obs[size_idx];
  } else {
    std::vector<float> h(nval);
    for (size_t i = 0; i < nval; ++i) h[i] = (float)y[i];
    RD_CUDA(cudaMalloc(&p->obs[size_idx], sizeof(float) * nval));
    RD_CUDA(cudaMemcpy(p->obs[size_idx], h.data(), sizeof(float) * nval, cudaMemcpyHostToDevice));
    S.yf = (const float*)p->obs[size_idx];
  }
  S.n_obs = n_times;
  for (int o = 0; o < RD_MAX_OBS; ++o) S.obs_steps[o] = o < n_times ? obs_steps[o] : 0;
  S.field_mask = field_mask;
  S.inv_two_sigma2 = 1.0 / (2.0 * sigma * sigma);
  p->obs_set[size_idx] = true;
  p->generation++;
  return RD_OK;
}

static rd_status check_ready(rd_problem* p) {
  for (int s = 0; s < p->desc.n_sizes; ++s) {
    RD_CHECK(p->ic_set[s] && p->obs_set[s], RD_ESTATE,
             "initial state and observations must be set for every grid size");
    RD_CHECK(p->dev.ss_tol <= 0.0 || p->dev.sz[s].n_obs == 1, RD_ESTATE,
             "steady-state mode observes once: set exactly one observation time");
  }
  return RD_OK;
}

rd_status rd_evaluate_batch(rd_problem* p, int B, const double* theta,
                            const int* size_idx, double* loglik,
                            uint32_t* status, void* fields) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(B >= 0, RD_EINVAL, "B must be >= 0");
  if (B == 0) return RD_OK;
  RD_CHECK(theta && loglik && status, RD_EINVAL, "NULL argument");
  rd_status r = check_ready(p);
  if (r != RD_OK) return r;
  if ((r = ensure_capacity(p, B)) != RD_OK) return r;
  WorkQueue q = make_queue(p);
  RD_CUDA(launch_fill_queue(q, B, size_idx, loglik, status, p->stream));
  RD_CUDA(launch_solve(p, theta, loglik, status, fields));
  return RD_OK;
}

rd_status rd_set_steady_state(rd_problem* p, double threshold, int confirm) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(threshold >= 0.0 && isfinite(threshold), RD_EINVAL, "threshold must be >= 0");
  if (threshold > 0.0) {
    RD_CHECK(!p->desc.growth, RD_EINVAL, "steady states are sought on a fixed domain");
    RD_CHECK(p->desc.dim == 1 || p->dev.max_n <= 96, RD_EINVAL,
             "steady-state mode in 2-D needs every grid at N <= 96");
    RD_CUDA(setup_solve_simt(p->desc.dim, p->dev.max_n, true));
  }
  p->dev.ss_tol = threshold;
  p->dev.ss_confirm = confirm ? 1 : 0;
  ++p->generation;  // captured chain steps hold the problem by value
  return RD_OK;
}

rd_status rd_evaluate_batch_steady(rd_problem* p, int B, const double* theta,
                                   const int* size_idx, double* loglik, uint32_t* status,
                                   void* fields, int* steps) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(p->dev.ss_tol > 0.0, RD_ESTATE, "steady-state mode is off (rd_set_steady_state)");
  RD_CHECK(B >= 0, RD_EINVAL, "B must be >= 0");
  if (B == 0) return RD_OK;
  RD_CHECK(theta && loglik && status, RD_EINVAL, "NULL argument");
  rd_status r = check_ready(p);
  if (r != RD_OK) return r;
  if ((r = ensure_capacity(p, B)) != RD_OK) return r;
  WorkQueue q = make_queue(p);
  RD_CUDA(launch_fill_queue(q, B, size_idx, loglik, status, p->stream));
  RD_CUDA(launch_solve_queue(p, q, theta, loglik, status, fields, p->stream, steps));
  return RD_OK;
}

rd_status rd_set_size_kernel(rd_problem* p, int size_idx, int kernel) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(p->desc.dim == 2, RD_EINVAL, "1-D problems always use the Thomas solve");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  RD_CHECK(kernel >= RD_KERNEL_DEFAULT && kernel <= RD_KERNEL_CG, RD_EINVAL,
           "unknown kernel");
  RD_CHECK(kernel != RD_KERNEL_CG || cg_applicable(p->dev.max_n, false), RD_EINVAL,
           "RD_KERNEL_CG needs every grid of the problem at N <= 96");
  RD_CHECK(kernel != RD_KERNEL_TC_RESIDENT || p->desc.nx[size_idx] == 128, RD_EINVAL,
           "RD_KERNEL_TC_RESIDENT needs N = 128");
  if (p->kernel_of_size[size_idx] != kernel) {
    p->kernel_of_size[size_idx] = kernel;
    ++p->generation;  // captured chain steps hold the old launches
  }
  return RD_OK;
}

rd_status rd_set_scheme(rd_problem* p, int scheme) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(scheme == RD_SCHEME_IMEX || scheme == RD_SCHEME_PICARD, RD_EINVAL, "unknown scheme");
  RD_CHECK(scheme == RD_SCHEME_IMEX || p->desc.dim == 1 || cg_applicable(p->dev.max_n, true),
           RD_EINVAL, "the semi-implicit scheme in 2-D needs every grid at N <= 80");
  if (scheme == RD_SCHEME_PICARD && p->desc.dim == 2)
    RD_CUDA(setup_solve_cg(p->dev.max_n, true));
  p->dev.scheme = scheme;
  ++p->generation;  // captured chain steps hold the problem by value
  return RD_OK;
}

rd_status rd_set_turing_prior(rd_problem* p, int enable) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  p->dev.turing = enable ? 1 : 0;
  ++p->generation;  // captured chain steps hold the problem by value
  return RD_OK;
}

rd_status rd_set_wait_limit(rd_problem* p, double seconds) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(seconds > 0 && seconds <= 60.0, RD_EINVAL, "wait limit must be in (0, 60] seconds");
  const unsigned long long ns = (unsigned long long)(seconds * 1e9);
  p->dev.wait_ns = ns > 0 ? ns : 1ull;
  ++p->generation;  // captured chain steps hold the problem by value
  return RD_OK;
}

rd_status rd_debug_stall_at_step(rd_problem* p, int step) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(step >= -1, RD_EINVAL, "step must be >= -1");
  p->dev.stall_step = step;
  ++p->generation;  // captured chain steps hold the problem by value
  return RD_OK;
}

rd_status rd_set_size_schedule(rd_problem* p, int size_idx, int ctas_per_sm) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  RD_CHECK(ctas_per_sm >= 0 && ctas_per_sm <= 32, RD_EINVAL, "ctas_per_sm must be in 0..32");
  if (p->ctas_per_sm[size_idx] != ctas_per_sm) {
    p->ctas_per_sm[size_idx] = ctas_per_sm;
    ++p->generation;  // captured chain steps hold the old launches
  }
  return RD_OK;
}

rd_status rd_get_size_schedule(const rd_problem* p, int size_idx, int* ctas_per_sm) {
  RD_CHECK(p && ctas_per_sm, RD_EINVAL, "NULL argument");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  const int gmax = grid_max_of(p, kernel_for_size(p, size_idx)) / p->n_sm;
  const int want = p->ctas_per_sm[size_idx];
  *ctas_per_sm = (want > 0 && want < gmax) ? want : gmax;
  return RD_OK;
}

rd_status rd_get_size_kernel(const rd_problem* p, int size_idx, int* kernel) {
  RD_CHECK(p && kernel, RD_EINVAL, "NULL argument");
  RD_CHECK(size_idx >= 0 && size_idx < p->desc.n_sizes, RD_EINVAL, "size_idx out of range");
  *kernel = kernel_for_size(p, size_idx);
  return RD_OK;
}

rd_status rd_evaluate_batch_host(rd_problem* p, int B, const double* theta,
                                 const int* size_idx, double* loglik,
                                 uint32_t* status) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CHECK(B >= 0, RD_EINVAL, "B must be >= 0");
  if (B == 0) return RD_OK;
  RD_CHECK(theta && loglik && status, RD_EINVAL, "NULL argument");
  if (B > p->staging_cap) {
    RD_CUDA(cudaStreamSynchronize(p->stream));
    cudaFree(p->h2d_theta);
    cudaFree(p->h2d_size);
    cudaFree(p->d2h_phi);
    cudaFree(p->d2h_status);
    p->h2d_theta = nullptr;
    p->h2d_size = nullptr;
    p->d2h_phi = nullptr;
    p->d2h_status = nullptr;
    p->staging_cap = 0;
    RD_CUDA(cudaMalloc(&p->h2d_theta, sizeof(double) * (size_t)B * p->desc.n_params));
    RD_CUDA(cudaMalloc(&p->h2d_size, sizeof(int) * (size_t)B));
    RD_CUDA(cudaMalloc(&p->d2h_phi, sizeof(double) * (size_t)B));
    RD_CUDA(cudaMalloc(&p->d2h_status, sizeof(uint32_t) * (size_t)B));
    p->staging_cap = B;
  }
  RD_CUDA(cudaMemcpyAsync(p->h2d_theta, theta, sizeof(double) * (size_t)B * p->desc.n_params,
                          cudaMemcpyHostToDevice, p->stream));
  if (size_idx)
    RD_CUDA(cudaMemcpyAsync(p->h2d_size, size_idx, sizeof(int) * (size_t)B,
                            cudaMemcpyHostToDevice, p->stream));
  rd_status r = rd_evaluate_batch(p, B, p->h2d_theta, size_idx ? p->h2d_size : nullptr,
                                  p->d2h_phi, p->d2h_status, nullptr);
  if (r != RD_OK) return r;
  RD_CUDA(cudaMemcpyAsync(loglik, p->d2h_phi, sizeof(double) * (size_t)B,
                          cudaMemcpyDeviceToHost, p->stream));
  RD_CUDA(cudaMemcpyAsync(status, p->d2h_status, sizeof(uint32_t) * (size_t)B,
                          cudaMemcpyDeviceToHost, p->stream));
  return rd_sync(p);  // waits, then reports a bounded wait that gave up
}

rd_status rd_sync(rd_problem* p) {
  RD_CHECK(p, RD_EINVAL, "problem is NULL");
  RD_CUDA(cudaStreamSynchronize(p->stream));
  int err = 0;
  RD_CUDA(cudaMemcpy(&err, p->ws.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    RD_CUDA(cudaMemset(p->ws.err, 0, sizeof(int)));
    set_error("a solve kernel's bounded wait gave up; its results are invalid");
    return RD_ETIMEOUT;
  }
  return RD_OK;
}

// ------------------------------------------------------------------ autotuning
rd_status rd_autotune(rd_problem* p, int B, const double* theta, int n_trials, int probe_steps,
                      double* times_out) {
  RD_CHECK(p && theta, RD_EINVAL, "NULL argument");
  RD_CHECK(p->desc.dim == 2, RD_EINVAL, "autotuning applies to 2-D problems");
  RD_CHECK(B > 0 && n_trials > 0 && probe_steps >= 0, RD_EINVAL,
           "B and n_trials must be > 0, probe_steps >= 0");
  rd_status r = check_ready(p);
  if (r != RD_OK) return r;
  if ((r = ensure_capacity(p, B)) != RD_OK) return r;
  const int P = p->desc.n_params, ns = p->desc.n_sizes;
  static const int kinds[4] = {RD_KERNEL_SIMT, RD_KERNEL_TC_STACKED, RD_KERNEL_TC_RESIDENT,
                               RD_KERNEL_CG};
  double times[RD_MAX_SIZES][4];
  double* d_theta = nullptr;
  double* d_phi = nullptr;
  uint32_t* d_st = nullptr;
  int* d_size = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int saved_steps = p->dev.n_steps;
  int saved_kernel[RD_MAX_SIZES], saved_ctas[RD_MAX_SIZES];
  for (int s = 0; s < RD_MAX_SIZES; ++s) {
    saved_kernel[s] = p->kernel_of_size[s];
    saved_ctas[s] = p->ctas_per_sm[s];
  }
  std::string fail;
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && fail.empty()) fail = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  bool ok = cu(cudaMalloc(&d_theta, sizeof(double) * (size_t)B * P), "cudaMalloc") &&
            cu(cudaMalloc(&d_phi, sizeof(double) * (size_t)B), "cudaMalloc") &&
            cu(cudaMalloc(&d_st, sizeof(uint32_t) * (size_t)B), "cudaMalloc") &&
            cu(cudaMalloc(&d_size, sizeof(int) * (size_t)B), "cudaMalloc") &&
            cu(cudaEventCreate(&e0), "cudaEventCreate") &&
            cu(cudaEventCreate(&e1), "cudaEventCreate") &&
            cu(cudaMemcpyAsync(d_theta, theta, sizeof(double) * (size_t)B * P,
                               cudaMemcpyHostToDevice, p->stream), "cudaMemcpyAsync");
  if (ok && probe_steps > 0 && probe_steps < saved_steps) p->dev.n_steps = probe_steps;
  std::vector<int> sizes((size_t)B);
  for (int s = 0; ok && s < ns; ++s) {
    std::fill(sizes.begin(), sizes.end(), s);
    ok = cu(cudaMemcpyAsync(d_size, sizes.data(), sizeof(int) * (size_t)B, cudaMemcpyHostToDevice,
                            p->stream), "cudaMemcpyAsync") &&
         cu(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    int best = -1, best_ctas = 0;
    double best_t = INFINITY;
    for (int k = 0; ok && k < 4; ++k) {
      times[s][k] = NAN;
      if (kinds[k] == RD_KERNEL_TC_RESIDENT && p->desc.nx[s] != 128) continue;
      if (kinds[k] == RD_KERNEL_CG && !cg_applicable(p->dev.max_n, false)) continue;
      p->kernel_of_size[s] = kinds[k];
      // schedule axis: 1, 2, 4, ... persistent CTAs per SM up to what fits
      const int per_max = std::max(1, grid_max_of(p, kinds[k]) / p->n_sm);
      for (int ctas = 1; ok && ctas <= per_max; ctas *= 2) {
      p->ctas_per_sm[s] = ctas;
      std::vector<float> ms;
      for (int t = 0; ok && t <= n_trials; ++t) {  // trial 0 warms up
        const WorkQueue q = make_queue(p);
        ok = cu(cudaEventRecord(e0, p->stream), "cudaEventRecord") &&
             cu(launch_fill_queue(q, B, d_size, d_phi, d_st, p->stream), "fill") &&
             cu(launch_solve(p, d_theta, d_phi, d_st, nullptr), "solve") &&
             cu(cudaEventRecord(e1, p->stream), "cudaEventRecord") &&
             cu(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float m = 0.f;
        if (ok && t > 0 && cu(cudaEventElapsedTime(&m, e0, e1), "cudaEventElapsedTime"))
          ms.push_back(m);
      }
      int err = 0;
      if (ok) ok = cu(cudaMemcpy(&err, p->ws.err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
      if (ok && err) {
        cudaMemset(p->ws.err, 0, sizeof(int));
        fail = "a solve kernel's bounded wait gave up during autotuning";
        ok = false;
      }
      if (!ok) break;
      std::sort(ms.begin(), ms.end());
      const double t_sec = 1e-3 * (double)ms[ms.size() / 2] / B;  // seconds per proposal
      if (!(times[s][k] <= t_sec)) times[s][k] = t_sec;  // best schedule of this kind
      if (t_sec < best_t) {
        best_t = t_sec;
        best = k;
        best_ctas = ctas;
      }
      }
    }
    if (ok) {
      saved_kernel[s] = kinds[best];
      saved_ctas[s] = best_ctas;
    }
  }
  p->dev.n_steps = saved_steps;
  for (int s = 0; s < RD_MAX_SIZES; ++s) {
    p->kernel_of_size[s] = saved_kernel[s];
    p->ctas_per_sm[s] = saved_ctas[s];
  }
  ++p->generation;  // captured chain steps hold the old launches
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_theta);
  cudaFree(d_phi);
  cudaFree(d_st);
  cudaFree(d_size);
  if (!ok) {
    set_error("rd_autotune: " + fail);
    return fail.find("bounded wait") != std::string::npos ? RD_ETIMEOUT : RD_ECUDA;
  }
  if (times_out)
    for (int s = 0; s < ns; ++s)
      for (int k = 0; k < 4; ++k) times_out[4 * s + k] = times[s][k];
  return RD_OK;
}

// ------------------------------------------------------------------ chains
rd_status rd_chains_destroy(rd_chains* c) {
  if (!c) return RD_OK;
  if (c->pb) cudaStreamSynchronize(c->pb->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  cudaFree(c->theta);
  cudaFree(c->phi);
  cudaFree(c->phit);
  cudaFree(c->lp);
  cudaFree(c->size_idx);
  cudaFree(c->prop);
  cudaFree(c->prop_phi);
  cudaFree(c->prop_phit);
  cudaFree(c->prop_lp);
  cudaFree(c->prop_status);
  cudaFree(c->samples);
  cudaFree(c->counters);
  cudaFree(c->ctl);
  cudaFree(c->pmh_prop);
  cudaFree(c->pmh_phi);
  cudaFree(c->pmh_lp);
  cudaFree(c->pmh_status);
  delete c;
  return RD_OK;
}

rd_status rd_chains_create(rd_problem* p, int n_chains, const double* theta0,
                           uint64_t seed, const double* step,
                           const int* size_idx, int capacity, rd_chains** out) {
  RD_CHECK(p && theta0 && step && out, RD_EINVAL, "NULL argument");
  *out = nullptr;
  RD_CHECK(n_chains >= 1, RD_EINVAL, "n_chains must be >= 1");
  RD_CHECK(capacity >= 1, RD_EINVAL, "capacity must be >= 1");
  rd_status r = check_ready(p);
  if (r != RD_OK) return r;
  if (size_idx)
    for (int i = 0; i < n_chains; ++i)
      RD_CHECK(size_idx[i] >= 0 && size_idx[i] < p->desc.n_sizes, RD_EINVAL,
               "size_idx out of range");
  if ((r = ensure_capacity(p, n_chains)) != RD_OK) return r;
  rd_chains* c = new rd_chains();
  c->pb = p;
  c->C = n_chains;
  c->P = p->desc.n_params;
  c->seed = seed;
  c->capacity = capacity;
  for (int j = 0; j < c->P; ++j) {
    c->step[j] = step[j];
    c->chol[j * RD_NPARAM + j] = step[j];
  }
  const size_t C = (size_t)n_chains, P = (size_t)c->P;
  bool ok = cudaMalloc(&c->theta, sizeof(double) * C * P) == cudaSuccess &&
            cudaMalloc(&c->phi, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->phit, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->lp, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->size_idx, sizeof(int) * C) == cudaSuccess &&
            cudaMalloc(&c->prop, sizeof(double) * C * P) == cudaSuccess &&
            cudaMalloc(&c->prop_phi, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->prop_phit, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->prop_lp, sizeof(double) * C) == cudaSuccess &&
            cudaMalloc(&c->prop_status, sizeof(uint32_t) * C) == cudaSuccess &&
            cudaMalloc(&c->samples, sizeof(double) * (size_t)capacity * P * C) == cudaSuccess &&
            cudaMalloc(&c->counters, sizeof(unsigned long long) * 4 * C) == cudaSuccess &&
            cudaMalloc(&c->ctl, sizeof(int) * 4) == cudaSuccess;
  if (!ok) {
    rd_chains_destroy(c);
    set_error("device allocation for chains failed");
    return RD_ENOMEM;
  }
  std::vector<int> sz(C, 0);
  if (size_idx) sz.assign(size_idx, size_idx + C);
  if (cudaMemcpy(c->theta, theta0, sizeof(double) * C * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->size_idx, sz.data(), sizeof(int) * C, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->counters, 0, sizeof(unsigned long long) * 4 * C) != cudaSuccess ||
      cudaMemset(c->ctl, 0, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(c->phit, 0, sizeof(double) * C) != cudaSuccess) {
    rd_chains_destroy(c);
    set_error("initialising chain state failed");
    return RD_ECUDA;
  }
  if (launch_chain_init(c) != cudaSuccess) {
    rd_chains_destroy(c);
    set_error("launching the initial solves failed");
    return RD_ECUDA;
  }
  *out = c;
  return RD_OK;
}

static rd_status capture_step_graph(rd_chains* c) {
  cudaStream_t cs;
  RD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = c->pb->stream;
  c->pb->stream = cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaError_t e2 = e == cudaSuccess ? launch_chain_step(c) : e;
  cudaError_t e3 = e == cudaSuccess ? cudaStreamEndCapture(cs, &g) : e;
  c->pb->stream = saved;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error(std::string("capturing the MCMC step graph failed: ") +
              cudaGetErrorString(e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3)));
    return RD_ECUDA;
  }
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error(std::string("instantiating the MCMC step graph failed: ") + cudaGetErrorString(e));
    return RD_ECUDA;
  }
  c->graph_ready = true;
  c->graph_generation = c->pb->generation;
  return RD_OK;
}

rd_status rd_chains_run(rd_chains* c, int n_steps) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  RD_CHECK(n_steps >= 0, RD_EINVAL, "n_steps must be >= 0");
  const long long rows = (long long)n_steps * (c->pmh_n > 0 ? c->pmh_n : 1);
  RD_CHECK(c->ring_host + rows <= c->capacity, RD_ESTATE,
           "sample buffer full: call rd_chains_read_samples first");
  if (!c->graph_ready || c->graph_generation != c->pb->generation) {
    RD_CUDA(cudaStreamSynchronize(c->pb->stream));
    rd_status r = capture_step_graph(c);
    if (r != RD_OK) return r;
  }
  for (int s = 0; s < n_steps; ++s) RD_CUDA(cudaGraphLaunch(c->graph, c->pb->stream));
  c->ring_host += (int)rows;
  return RD_OK;
}

rd_status rd_chains_set_proposal(rd_chains* c, const double* L) {
  RD_CHECK(c && L, RD_EINVAL, "NULL argument");
  for (int j = 0; j < c->P; ++j)
    for (int i = 0; i < RD_NPARAM; ++i) {
      const double v = (i <= j && i < c->P) ? L[j * c->P + i] : 0.0;
      RD_CHECK(isfinite(v), RD_EINVAL, "proposal factor must be finite");
      c->chol[j * RD_NPARAM + i] = v;
    }
  c->graph_ready = false;  // captured kernels hold the factor by value
  return RD_OK;
}

rd_status rd_chains_set_first_chain(rd_chains* c, uint32_t first) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  RD_CHECK((uint64_t)first + (uint64_t)c->C <= 0x100000000ull, RD_EINVAL,
           "first + n_chains must fit the 32-bit chain counter");
  c->first_chain = first;
  c->graph_ready = false;  // captured kernels hold it by value
  return RD_OK;
}

rd_status rd_chains_set_parallel_proposals(rd_chains* c, int n_prop) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  RD_CHECK(n_prop >= 0 && n_prop <= RD_PMH_MAX_PROPOSALS, RD_EINVAL,
           "n_prop must be in 0..RD_PMH_MAX_PROPOSALS");
  RD_CHECK(n_prop == 0 || c->sur == nullptr, RD_EINVAL,
           "multi-proposal steps do not combine with a surrogate");
  RD_CUDA(cudaStreamSynchronize(c->pb->stream));
  cudaFree(c->pmh_prop);
  cudaFree(c->pmh_phi);
  cudaFree(c->pmh_lp);
  cudaFree(c->pmh_status);
  c->pmh_prop = nullptr;
  c->pmh_phi = nullptr;
  c->pmh_lp = nullptr;
  c->pmh_status = nullptr;
  c->pmh_n = 0;
  c->graph_ready = false;
  if (n_prop == 0) return RD_OK;
  const size_t n = (size_t)c->C * n_prop;
  rd_status r = ensure_capacity(c->pb, (int)n);
  if (r != RD_OK) return r;
  RD_CUDA(cudaMalloc(&c->pmh_prop, sizeof(double) * n * c->P));
  RD_CUDA(cudaMalloc(&c->pmh_phi, sizeof(double) * n));
  RD_CUDA(cudaMalloc(&c->pmh_lp, sizeof(double) * n));
  RD_CUDA(cudaMalloc(&c->pmh_status, sizeof(uint32_t) * n));
  c->pmh_n = n_prop;
  return RD_OK;
}

rd_status rd_chains_set_surrogate(rd_chains* c, rd_surrogate* s) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  RD_CHECK(s == nullptr || c->pmh_n == 0, RD_EINVAL,
           "delayed acceptance works with single-proposal steps only");
  RD_CUDA(cudaStreamSynchronize(c->pb->stream));
  c->sur = s;
  c->graph_ready = false;  // the step graph differs with and without stage 1
  if (s) {
    RD_CUDA(mlp::ensure_rows(s, c->C));
    RD_CUDA(mlp::predict(s, c->C, c->theta, c->phit, c->pb->stream));
    RD_CUDA(cudaStreamSynchronize(c->pb->stream));
  }
  return RD_OK;
}

rd_status rd_chains_read_samples(rd_chains* c, double* out, size_t cap_steps,
                                 size_t* n_written, double* counters) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  cudaStream_t st = c->pb->stream;
  const size_t per = (size_t)c->P * c->C;
  size_t n = std::min((size_t)c->ring_host, out ? cap_steps : 0);
  if (n > 0) RD_CUDA(cudaMemcpyAsync(out, c->samples, sizeof(double) * per * n,
                                     cudaMemcpyDeviceToHost, st));
  if (counters) {
    std::vector<unsigned long long> h(4 * (size_t)c->C);
    RD_CUDA(cudaMemcpyAsync(h.data(), c->counters, sizeof(unsigned long long) * h.size(),
                            cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int i = 0; i < c->C; ++i) s += (double)h[(size_t)k * c->C + i];
      counters[k] = s;
    }
  }
  RD_CUDA(cudaStreamSynchronize(st));
  if (n < (size_t)c->ring_host && n > 0) {
    // move the unread tail to the front of the ring in chunks of n samples,
    // so that no copy has overlapping source and destination
    for (size_t k = n; k < (size_t)c->ring_host; k += n) {
      const size_t len = std::min(n, (size_t)c->ring_host - k);
      RD_CUDA(cudaMemcpyAsync(c->samples + per * (k - n), c->samples + per * k,
                              sizeof(double) * per * len, cudaMemcpyDeviceToDevice, st));
    }
  }
  c->ring_host -= (int)n;
  const int ring = c->ring_host;
  RD_CUDA(cudaMemcpyAsync(c->ctl + 1, &ring, sizeof(int), cudaMemcpyHostToDevice, st));
  RD_CUDA(cudaStreamSynchronize(st));
  if (n_written) *n_written = n;
  return RD_OK;
}

rd_status rd_chains_get_state(rd_chains* c, double* theta, double* phi) {
  RD_CHECK(c, RD_EINVAL, "chains is NULL");
  cudaStream_t st = c->pb->stream;
  if (theta)
    RD_CUDA(cudaMemcpyAsync(theta, c->theta, sizeof(double) * c->C * c->P,
                            cudaMemcpyDeviceToHost, st));
  if (phi) RD_CUDA(cudaMemcpyAsync(phi, c->phi, sizeof(double) * c->C, cudaMemcpyDeviceToHost, st));
  RD_CUDA(cudaStreamSynchronize(st));
  return RD_OK;
}

namespace {
struct CkptHeader {
  uint32_t magic;  // 'RDCK'
  uint32_t version;
  int32_t C, P;
  uint64_t seed;
  int32_t step;
  int32_t pad;
};
}  // namespace

rd_status rd_chains_checkpoint(rd_chains* c, void* buf, size_t cap, size_t* n) {
  RD_CHECK(c && n, RD_EINVAL, "NULL argument");
  const size_t C = (size_t)c->C, P = (size_t)c->P;
  const size_t need = sizeof(CkptHeader) + sizeof(double) * (C * P + 3 * C) +
                      sizeof(unsigned long long) * 4 * C;
  *n = need;
  if (!buf) return RD_OK;
  RD_CHECK(cap >= need, RD_EINVAL, "checkpoint buffer too small");
  cudaStream_t st = c->pb->stream;
  CkptHeader h;
  int ctl[4];
  RD_CUDA(cudaMemcpyAsync(ctl, c->ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
  char* q = (char*)buf + sizeof(CkptHeader);
  RD_CUDA(cudaMemcpyAsync(q, c->theta, sizeof(double) * C * P, cudaMemcpyDeviceToHost, st));
  q += sizeof(double) * C * P;
  RD_CUDA(cudaMemcpyAsync(q, c->phi, sizeof(double) * C, cudaMemcpyDeviceToHost, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(q, c->phit, sizeof(double) * C, cudaMemcpyDeviceToHost, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(q, c->lp, sizeof(double) * C, cudaMemcpyDeviceToHost, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(q, c->counters, sizeof(unsigned long long) * 4 * C,
                          cudaMemcpyDeviceToHost, st));
  RD_CUDA(cudaStreamSynchronize(st));
  h.magic = 0x4B434452u;
  h.version = 1;
  h.C = c->C;
  h.P = c->P;
  h.seed = c->seed;
  h.step = ctl[0];
  h.pad = 0;
  memcpy(buf, &h, sizeof(h));
  return RD_OK;
}

rd_status rd_chains_restore(rd_chains* c, const void* buf, size_t n) {
  RD_CHECK(c && buf, RD_EINVAL, "NULL argument");
  const size_t C = (size_t)c->C, P = (size_t)c->P;
  const size_t need = sizeof(CkptHeader) + sizeof(double) * (C * P + 3 * C) +
                      sizeof(unsigned long long) * 4 * C;
  RD_CHECK(n >= need, RD_EINVAL, "checkpoint too short");
  CkptHeader h;
  memcpy(&h, buf, sizeof(h));
  RD_CHECK(h.magic == 0x4B434452u && h.version == 1, RD_EINVAL, "not a chain checkpoint");
  RD_CHECK(h.C == c->C && h.P == c->P && h.seed == c->seed, RD_EINVAL,
           "checkpoint is for different chains (C, P or seed differ)");
  cudaStream_t st = c->pb->stream;
  const char* q = (const char*)buf + sizeof(CkptHeader);
  RD_CUDA(cudaMemcpyAsync(c->theta, q, sizeof(double) * C * P, cudaMemcpyHostToDevice, st));
  q += sizeof(double) * C * P;
  RD_CUDA(cudaMemcpyAsync(c->phi, q, sizeof(double) * C, cudaMemcpyHostToDevice, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(c->phit, q, sizeof(double) * C, cudaMemcpyHostToDevice, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(c->lp, q, sizeof(double) * C, cudaMemcpyHostToDevice, st));
  q += sizeof(double) * C;
  RD_CUDA(cudaMemcpyAsync(c->counters, q, sizeof(unsigned long long) * 4 * C,
                          cudaMemcpyHostToDevice, st));
  int ctl[4] = {h.step, 0, 0, 0};
  RD_CUDA(cudaMemcpyAsync(c->ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, st));
  RD_CUDA(cudaStreamSynchronize(st));
  c->ring_host = 0;
  return RD_OK;
}

}  // extern "C"
