// rd_internal.h -- host-side objects behind the C ABI handles and the kernel
// launchers shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rdbayes.h"
#include "rd_common.cuh"

namespace rd {

void set_error(const std::string& msg);
// Looks up (once per device, that device current) the device address of the
// fixed scratch of rd_evaluate_batch_noalloc (rd_noalloc.cu).
rd_status noalloc_prepare(int device);

// Problem-level device workspace: work lists and per-proposal outputs of the
// chain sampler's exact solves.
struct Workspace {
  int* queue_items = nullptr;   // [n_sizes][capacity]
  int* queue_counters = nullptr;  // [2 * kMaxSizes]: counts, pops
  int* err = nullptr;             // set by a kernel whose bounded wait gave up
  int capacity = 0;
};

}  // namespace rd

struct rd_problem {
  rd_problem_desc desc;
  rd::DevProblem dev;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;
  bool ic_set[RD_MAX_SIZES] = {false, false, false, false};
  bool obs_set[RD_MAX_SIZES] = {false, false, false, false};
  // per-size device buffers (owned)
  void* ic[RD_MAX_SIZES] = {nullptr, nullptr, nullptr, nullptr};
  void* obs[RD_MAX_SIZES] = {nullptr, nullptr, nullptr, nullptr};
  float* cmat[RD_MAX_SIZES] = {nullptr, nullptr, nullptr, nullptr};
  float* mu[RD_MAX_SIZES] = {nullptr, nullptr, nullptr, nullptr};
  rd::Workspace ws;
  // bumped whenever a device buffer that a captured graph may reference is
  // replaced; chains re-capture their step graph when it changes
  int generation = 0;
  // RD_KERNEL_* of each size; RD_KERNEL_DEFAULT follows desc.solver
  int kernel_of_size[RD_MAX_SIZES] = {0, 0, 0, 0};
  // persistent CTAs per SM of each size's launch (0 = the kernel's maximum)
  int ctas_per_sm[RD_MAX_SIZES] = {0, 0, 0, 0};
  // staging for rd_evaluate_batch_host
  double* h2d_theta = nullptr;
  int* h2d_size = nullptr;
  double* d2h_phi = nullptr;
  uint32_t* d2h_status = nullptr;
  int staging_cap = 0;
};

struct rd_chains {
  rd_problem* pb = nullptr;
  int C = 0;
  int P = 0;
  uint64_t seed = 0;
  uint32_t first_chain = 0;  // global index of chain 0 in the Philox counters
  int capacity = 0;
  int ring_host = 0;  // samples in the device ring (host mirror)
  double step[RD_NPARAM] = {0, 0, 0, 0, 0};
  double chol[RD_NPARAM * RD_NPARAM] = {};  // proposal increments L xi (row-major)
  // device state
  double* theta = nullptr;      // [C][P]
  double* phi = nullptr;        // [C]
  double* phit = nullptr;       // [C] surrogate Phi~ (DA only)
  double* lp = nullptr;         // [C] log prior (+ log Jacobian) in step space
  int* size_idx = nullptr;      // [C]
  double* prop = nullptr;       // [C][P] proposals
  double* prop_phi = nullptr;   // [C]
  double* prop_phit = nullptr;  // [C]
  double* prop_lp = nullptr;    // [C]
  uint32_t* prop_status = nullptr;  // [C]
  double* samples = nullptr;    // [capacity][P][C]
  unsigned long long* counters = nullptr;  // [4][C]: proposals, pass1, accepted, solves
  int* ctl = nullptr;           // [0]: step index, [1]: ring fill
  cudaGraphExec_t graph = nullptr;
  bool graph_ready = false;
  int graph_generation = -1;
  rd_surrogate* sur = nullptr;  // delayed acceptance when set
  // multi-proposal steps (Algorithm 2): N proposals per chain and step
  int pmh_n = 0;
  double* pmh_prop = nullptr;        // [C][N][P]
  double* pmh_phi = nullptr;         // [C][N]
  double* pmh_lp = nullptr;          // [C][N]
  uint32_t* pmh_status = nullptr;    // [C][N]
};

namespace rd {

cudaError_t launch_fill_queue(const WorkQueue& q, int B, const int* size_idx,
                              double* phi, uint32_t* status, cudaStream_t st);
// CUDA-core kernels (rd_solve_simt.cu); steady: the steady-state-mode variant
// (pb.ss_tol > 0), whose steps_out (may be null) receives each proposal's T.
cudaError_t launch_solve_simt(const DevProblem& pb, const WorkQueue& q,
                              const double* theta, double* phi, uint32_t* status,
                              void* fields, int grid, cudaStream_t st,
                              int* steps_out = nullptr);
cudaError_t setup_solve_simt(int dim, int max_n, bool steady = false);
cudaError_t setup_solve_tc(int max_n);
int grid_solve_tc(int max_n, int n_sm);
cudaError_t launch_solve_tc(const DevProblem& pb, const WorkQueue& q, const double* theta,
                            double* phi, uint32_t* status, void* fields, int grid, int* err,
                            cudaStream_t st);
size_t tc_smem_bytes_host(int max_n);
// 128^2-only tensor-core solve with the DCT matrices resident in TMEM
// (rd_solve_tc2.cu): every size in its queue must be a 2-D 128^2 grid.
bool tc128_applicable(const DevProblem& pb, int size_idx);
cudaError_t setup_solve_tc128();
int grid_solve_tc128(int n_sm);
cudaError_t launch_solve_tc128(const DevProblem& pb, const WorkQueue& q, const double* theta,
                               double* phi, uint32_t* status, void* fields, int grid, int* err,
                               cudaStream_t st);
// CUDA-core conjugate-gradient solves (rd_solve_simt.cu): the IMEX step by
// plain CG (RD_KERNEL_CG, N <= 96) or the paper's semi-implicit step by
// preconditioned CG (picard, N <= 80).
bool cg_applicable(int n, bool picard);
cudaError_t setup_solve_cg(int max_n, bool picard);
int grid_solve_cg(int max_n, bool picard, int n_sm);
cudaError_t launch_solve_cg(const DevProblem& pb, const WorkQueue& q, const double* theta,
                            double* phi, uint32_t* status, void* fields, bool picard, int grid,
                            cudaStream_t st);
bool uses_tc(const rd_problem* p);
int grid_solve_simt(int dim, int max_n, int n_sm, bool steady = false);
size_t simt2d_smem_bytes(int n, bool steady = false);

WorkQueue make_queue(const rd_problem* p);
int kernel_for_size(const rd_problem* p, int size_idx);
// Launches the solve kernels over the queue's sizes, one persistent launch
// per kernel kind in use (sizes grouped by kernel_for_size).
cudaError_t launch_solve_queue(rd_problem* p, const WorkQueue& q, const double* theta,
                               double* phi, uint32_t* status, void* fields, cudaStream_t st,
                               int* steps_out = nullptr);
cudaError_t launch_solve(rd_problem* p, const double* theta, double* phi,
                         uint32_t* status, void* fields);

namespace mlp {
cudaError_t predict(rd_surrogate* s, int B, const double* theta, double* phit, cudaStream_t st);
cudaError_t ensure_rows(rd_surrogate* s, int rows);
}  // namespace mlp

// chains
cudaError_t launch_chain_init(rd_chains* c);
cudaError_t launch_chain_step(rd_chains* c);

}  // namespace rd
