/*
 * rdbayes.h -- C ABI of the GB300 library for Bayesian identification of the
 * parameters of the Schnakenberg reaction-diffusion system (arXiv:1605.04718).
 *
 * The method (Sec. 2): data y = G(p) + eta with Gaussian noise (eq.
 * (meas_model)); log-likelihood Phi(p; y) = -log rho(y - G(p)) (eq. (logl));
 * posterior mu^y(p) proportional to exp(-Phi(p; y)) mu_0(p) (eq. (bayes));
 * sampled by Metropolis-Hastings (Algorithm 1) over many independent chains,
 * with burn-in and pooling as in Sec. 2.1.  G solves the system of eq.
 * (schnakenberg) with the kinetics of eq. (reactions),
 *     u_t + m r u = rho^-2 Lap u + gamma (a - u + u^2 v),
 *     v_t + m r v = d rho^-2 Lap v + gamma (b - u^2 v),
 * on the unit interval or square with Neumann boundaries, rho(t) = exp(r t)
 * (rho = 1 on a fixed domain), by the finite-difference IMEX Euler step of
 * Sec. 3.1.1 with the reaction explicit and diffusion plus dilution implicit.
 *
 * Conventions for every call:
 *  - Returns an rd_status; never aborts.  rd_last_error() gives a message
 *    for the calling thread.
 *  - Parameter vectors are in natural units, in the order of the inferred
 *    model parameters (a, b, d, gamma, r, p1, p2, p3) that
 *    rd_problem_desc.param_map lists.
 *  - "device" pointers are CUDA device addresses on the problem's device;
 *    "host" pointers are ordinary host memory.  The caller owns every pointer
 *    it passes; the library copies or consumes inputs in stream order and
 *    never keeps a caller pointer after the call's work has completed.
 *  - All GPU work is enqueued on the problem's CUDA stream (cudaStream_t passed
 *    as void*; NULL = the legacy default stream).  Calls marked "async" return
 *    before the work is done; rd_sync waits for it.
 *  - Per-proposal failures are status bits with Phi = +inf, not call errors
 *    (the paper's requirement that the log-likelihood be robust, Sec. 2).
 *  - There is no CPU fallback: without a CUDA device every call that needs one
 *    returns RD_ECUDA.
 */
#ifndef RDBAYES_H
#define RDBAYES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rd_problem rd_problem;
typedef struct rd_chains rd_chains;
typedef struct rd_surrogate rd_surrogate;

typedef enum {
  RD_OK = 0,
  RD_EINVAL = 1,   /* invalid argument (message in rd_last_error) */
  RD_ENOMEM = 2,   /* device or host allocation failed */
  RD_ECUDA = 3,    /* a CUDA runtime call failed, or no device */
  RD_ESTATE = 4,   /* call out of order (e.g. no observations set) */
  RD_ETIMEOUT = 5  /* a bounded device wait gave up */
} rd_status;

/* Per-proposal status bits. */
enum {
  RD_P_OK = 0,
  RD_P_OUT_OF_SUPPORT = 1, /* prior density zero: rejected without a solve */
  RD_P_NONFINITE = 2,      /* non-finite or |w| > w_max at an observation */
  RD_P_NOT_CONVERGED = 4,  /* iterative solve hit its iteration cap */
  RD_P_NOT_SOLVED = 8      /* queued, but no solve kernel finished it (a bounded
                              wait gave up: the call reports RD_ETIMEOUT) */
};

/* Implicit-diffusion solver of the IMEX step. */
enum {
  RD_SOLVER_AUTO = 0,      /* autotuned per grid size (2-D), Thomas (1-D) */
  RD_SOLVER_THOMAS = 1,    /* 1-D tridiagonal (FP64) */
  RD_SOLVER_DCT_SIMT = 2,  /* 2-D eigenbasis solve, FP32 CUDA-core GEMMs */
  RD_SOLVER_DCT_TC = 3     /* 2-D eigenbasis solve, split-FP16 tcgen05 GEMMs */
};

/* Solve kernel of one 2-D grid size (rd_set_size_kernel, rd_autotune).  All
 * compute the same IMEX step; they differ in how the eigenbasis transforms of
 * the implicit solve run on the GPU. */
enum {
  RD_KERNEL_DEFAULT = 0,     /* from desc.solver: SIMT for RD_SOLVER_DCT_SIMT;
                                otherwise TC_RESIDENT at N = 128, else
                                TC_STACKED */
  RD_KERNEL_SIMT = 1,        /* FP32 CUDA-core GEMMs, one proposal per CTA */
  RD_KERNEL_TC_STACKED = 2,  /* split-FP16 tcgen05, DCT matrix in shared memory,
                                floor(128/N) proposals stacked per MMA tile */
  RD_KERNEL_TC_RESIDENT = 3, /* split-FP16 tcgen05, DCT matrices resident in
                                tensor memory; N = 128 only */
  RD_KERNEL_CG = 4           /* each implicit system by plain conjugate gradients
                                (the paper's linear solver, Sec. 3.1.1) from the
                                previous step, FP32 on CUDA cores, vectors in
                                shared memory; every grid of the problem N <= 96 */
};

/* Time step of the forward problem (rd_set_scheme). */
enum {
  RD_SCHEME_IMEX = 0,   /* reaction explicit, diffusion + dilution implicit */
  RD_SCHEME_PICARD = 1  /* the paper's semi-implicit step (Sec. 3.1.1, Example 1):
                           reaction linearised with one Picard iterate and
                           implicit too; 1-D, or 2-D with every grid N <= 80 */
};

enum { RD_PRIOR_UNIFORM = 0, RD_PRIOR_LOGNORMAL = 1 };
/* Domain growth law rho(t) of eq. (schnakenberg) (rd_problem_desc.growth). */
enum {
  RD_GROWTH_NONE = 0,  /* fixed domain, rho = 1 */
  RD_GROWTH_EXP = 1,   /* rho = exp(r t), m = dim (r = model parameter 4) */
  RD_GROWTH_POLY4 = 2  /* Example 1 (Sec. 3.1.1): rho(s), s = t / T, T = n_steps tau,
                          = 1 + p1 s + p2 s^2 + p3 s^3 + p4 s^4 with
                          p4 = rho_T - 1 - p1 - p2 - p3, so rho(0) = 1 and
                          rho(T) = rho_T; p1..p3 = model parameters 5..7;
                          1-D only.  The prior also requires rho > 0 at
                          s = k / 1000, k = 0..1000 */
};
enum { RD_STEP_LINEAR = 0, RD_STEP_LOG = 1 };
enum { RD_PREC_F64 = 0, RD_PREC_F32 = 1 };

#define RD_MAX_SIZES 4
#define RD_MAX_OBS 8
#define RD_NPARAM 5  /* inferred parameters at most */
#define RD_NPHYS 8   /* model parameters (a, b, d, gamma, r, p1, p2, p3) */
#define RD_NOALLOC_MAX_BATCH 65536
#define RD_PMH_MAX_PROPOSALS 16 /* N of rd_chains_set_parallel_proposals */
#define RD_SURROGATE_WIDTH 256

/*
 * Problem description.  Grid: cell-centred, x_i = (i + 1/2)/N, h = 1/N, in
 * each dimension.  One problem may hold up to RD_MAX_SIZES grid sizes (each
 * with its own initial state and observations) whose proposals are batched
 * together in one launch.
 */
typedef struct {
  int dim;                    /* 1 or 2 */
  int n_sizes;                /* 1..RD_MAX_SIZES */
  int nx[RD_MAX_SIZES];       /* grid points per side; 2-D: multiple of 16, 16..128;
                                 1-D: 2..256 */
  double tau;                 /* time step */
  int n_steps;                /* steps to the final time T = n_steps * tau */
  int precision;              /* RD_PREC_F64 (1-D) or RD_PREC_F32 (2-D fields) */
  int solver;                 /* RD_SOLVER_* */
  int growth;                 /* RD_GROWTH_*: 0 fixed domain (r ignored), 1 exponential,
                                 2 Example 1's polynomial */
  int n_params;               /* number of inferred parameters P, 1..5 */
  int param_map[RD_NPARAM];   /* index in (a, b, d, gamma, r, p1, p2, p3) of inferred
                                 parameter j (5..7 only with RD_GROWTH_POLY4) */
  double fixed[RD_NPARAM];    /* values of the model parameters 0..4 that are not
                                 inferred */
  int prior_kind[RD_NPARAM];  /* per inferred parameter: RD_PRIOR_* */
  double prior_p0[RD_NPARAM]; /* uniform: lower bound; log-normal: median */
  double prior_p1[RD_NPARAM]; /* uniform: upper bound; log-normal: sigma of log */
  int step_space[RD_NPARAM];  /* per inferred parameter: RD_STEP_* */
  double w_max;               /* divergence bound (<= 0: default 100) */
  double fixed_poly[3];       /* RD_GROWTH_POLY4: values of p1..p3 not inferred */
  double rho_T;               /* RD_GROWTH_POLY4: the known final size rho(T) */
} rd_problem_desc;

/* Creates a problem on the current CUDA device and stream `cuda_stream`.
 * Allocates the library's device workspace.  EINVAL on an invalid desc. */
rd_status rd_problem_create(const rd_problem_desc* desc, void* cuda_stream,
                            rd_problem** out);
rd_status rd_problem_destroy(rd_problem* p);
rd_status rd_set_stream(rd_problem* p, void* cuda_stream);

/* Initial state u0, v0 of grid size `size_idx` (host, N^dim values each,
 * row-major with the first index along y).  The same fixed, known initial
 * state is used for every proposal (Sec. 3.1.2).  Copied; stream-ordered. */
rd_status rd_set_initial_state(rd_problem* p, int size_idx, const double* u0,
                               const double* v0);

/* Observations of size `size_idx`: n_times (1..RD_MAX_OBS) step indices
 * obs_steps (increasing, in 1..n_steps), observed fields field_mask (1 = u,
 * 2 = v, 3 = both), data y (host, [n_times][observed fields][N^dim]) and
 * noise standard deviation sigma.  Phi = sum (y - w)^2 / (2 sigma^2) over all
 * observed values (eq. (logl) with Gaussian noise).  Copied; stream-ordered. */
rd_status rd_set_observations(rd_problem* p, int size_idx, int n_times,
                              const int* obs_steps, int field_mask,
                              const double* y, double sigma);

/* Forward solves + log-likelihoods for B proposals (async).
 * theta:    device, [B][n_params] inferred parameters (natural units)
 * size_idx: device, [B] grid-size index of each proposal, or NULL (all 0)
 * loglik:   device, [B] Phi (+inf when status != 0)
 * status:   device, [B] RD_P_* bits
 * fields:   device or NULL, [B][2][maxN^dim] final u, v (float for F32
 *           problems, double for F64), each proposal at stride 2*maxN^dim
 *           with its own N^dim values first. */
rd_status rd_evaluate_batch(rd_problem* p, int B, const double* theta,
                            const int* size_idx, double* loglik,
                            uint32_t* status, void* fields);

/* As rd_evaluate_batch with HOST theta/size_idx/loglik/status: copies in,
 * solves, copies out, and returns when the results are in host memory;
 * RD_ETIMEOUT as rd_sync. */
rd_status rd_evaluate_batch_host(rd_problem* p, int B, const double* theta,
                                 const int* size_idx, double* loglik,
                                 uint32_t* status);

/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory while they run -- e.g. a host whose device memory is
 * all reserved by another allocator, or a time-critical loop that must not
 * stall on the device-wide synchronisation of cudaFree -- because
 * rd_evaluate_batch may grow the problem's workspace (cudaFree + cudaMalloc)
 * when it sees a larger batch than before.
 * Same arguments, results and stream behaviour as rd_evaluate_batch, but the
 * call allocates nothing: the solve kernels' work lists live in one fixed
 * device array of the library (about 1 MiB, held on every GPU that loads the
 * library until the process exits), so B may be at most RD_NOALLOC_MAX_BATCH
 * (EINVAL beyond).  The problem's device must be current.  rd_problem_create
 * looks up that array's device address once per device (which loads the array
 * onto the device), so the first call on a device is allocation-free too and
 * needs no set-up of its own.  All calls share the array and
 * each clears its counters before use, so calls whose GPU work overlaps (for
 * example on two streams at once) race and must be serialised by the caller. */
rd_status rd_evaluate_batch_noalloc(rd_problem* p, int B, const double* theta,
                                    const int* size_idx, double* loglik,
                                    uint32_t* status, void* fields);

/* Time-stepping scheme of the forward solves (RD_SCHEME_*; default IMEX).
 * RD_SCHEME_PICARD: per step
 *   [(1 + tau m r + tau gamma (1 - u^n v^n)) I - tau / rho_n^2 Lap_h] u^{n+1}
 *       = u^n + tau gamma a,
 *   [(1 + tau m r + tau gamma (u^n)^2) I - tau d / rho_n^2 Lap_h] v^{n+1}
 *       = v^n + tau gamma b,
 * each a system with a node-dependent diagonal: in 1-D tridiagonal (FP64
 * Thomas); in 2-D (FP32 fields) solved by conjugate gradients preconditioned
 * with the eigenbasis solve of the operator with the mean diagonal, to a
 * relative residual of 1e-6 (a proposal whose solve reaches the iteration
 * cap gets RD_P_NOT_CONVERGED), all sizes in one CUDA-core launch whatever
 * kernel each size has.  EINVAL for an unknown scheme or PICARD on a 2-D
 * problem with a grid above 80. */
rd_status rd_set_scheme(rd_problem* p, int scheme);

/* Steady-state forward map (the measurement protocol of Sec. 3.1.2: the data
 * are the stationary pattern).  With threshold > 0 every forward solve runs
 * until the first step T at which the L2 norm of the discrete time
 * derivative, (h^dim sum over both fields and all nodes of
 * ((w^T - w^{T-1}) / tau)^2)^(1/2), is below threshold (1e-5 in the paper),
 * at most n_steps steps; the misfit is taken against the problem's single
 * observation (each size must have exactly one observation time, whose step
 * index is then ignored) at T, and the final fields are w(T).  With
 * confirm != 0 the solve continues to 2T and requires the same norm of
 * w(2T) - w(T) to be below threshold (the paper's check that the state is
 * stationary).  A solve that reaches neither gets RD_P_NOT_CONVERGED.
 * Fixed domains only (EINVAL with growth); 2-D problems need every grid
 * N <= 96 and run on the CUDA-core eigenbasis kernel (the tensor-core
 * kernels hold no copy of the previous step), 1-D on the FP64 Thomas kernel.
 * threshold = 0 turns the mode off.  Takes effect at the next launch. */
rd_status rd_set_steady_state(rd_problem* p, double threshold, int confirm);

/* rd_evaluate_batch in steady-state mode that also writes T per proposal
 * (device int [B]; 0 where no steady state was reached).  ESTATE when the
 * mode is off. */
rd_status rd_evaluate_batch_steady(rd_problem* p, int B, const double* theta,
                                   const int* size_idx, double* loglik,
                                   uint32_t* status, void* fields, int* steps);

/* Restricts the prior to the Turing space of the kinetics (Sec. 3.1.2 Case 2,
 * eq. (turing)): with enable != 0, log mu0 = -inf unless (a, b, d) -- each
 * inferred or fixed -- satisfies f_u + g_v < 0, f_u g_v - f_v g_u > 0,
 * d f_u + g_v > 0 and (d f_u + g_v)^2 - 4 d (f_u g_v - f_v g_u) > 0 at the
 * homogeneous steady state; inside, the per-parameter priors apply (uniform
 * boxes give the paper's uniform prior on the Turing space).  Proposals
 * outside are rejected without a solve.  Default off. */
rd_status rd_set_turing_prior(rd_problem* p, int enable);

/* Kernel that solves the proposals of grid size `size_idx` (RD_KERNEL_*).
 * Sizes that share a kernel run in one persistent launch; a batch whose sizes
 * use different kernels runs one launch per kernel, in stream order.  EINVAL
 * for a 1-D problem (always the Thomas solve), an unknown kernel, or
 * TC_RESIDENT at N != 128.  Takes effect at the next launch (captured chain
 * steps are re-captured). */
rd_status rd_set_size_kernel(rd_problem* p, int size_idx, int kernel);
/* The kernel size `size_idx` runs with, RD_KERNEL_DEFAULT resolved. */
rd_status rd_get_size_kernel(const rd_problem* p, int size_idx, int* kernel);

/* Schedule of grid size `size_idx`'s persistent launch: CTAs per SM
 * (0..32; 0 = as many as fit, the default).  Sizes sharing a kernel launch
 * run with the largest value any of them sets, capped at what fits.  Takes
 * effect at the next launch. */
rd_status rd_set_size_schedule(rd_problem* p, int size_idx, int ctas_per_sm);
/* The CTAs per SM that size's launch uses (default and cap resolved). */
rd_status rd_get_size_schedule(const rd_problem* p, int size_idx, int* ctas_per_sm);

/* Timed search of the solve kernel of every grid size of a 2-D problem:
 * for each size s, solves the B proposals theta (host, [B][n_params], the
 * same batch for every candidate) as size s with each kernel that supports
 * it, one warm-up and n_trials timed launches (CUDA events on the problem's
 * stream), probe_steps IMEX steps per solve (0 = the problem's n_steps), and
 * sets the kernel and schedule with the lowest median time
 * (rd_set_size_kernel, rd_set_size_schedule): every kernel is timed at 1, 2,
 * 4, ... persistent CTAs per SM up to what fits on an SM.  Sizes
 * of a problem run one persistent launch per kernel kind, so the choice per
 * size stays within one batched evaluation.  times_out (host, may be NULL):
 * [n_sizes][4] seconds per proposal for RD_KERNEL_SIMT, TC_STACKED,
 * TC_RESIDENT and CG at each one's best schedule, NaN where a kernel does
 * not apply.  Allocates scratch for the
 * batch; synchronises the stream.  EINVAL for a 1-D problem; on a failed
 * launch the previous choices are kept. */
rd_status rd_autotune(rd_problem* p, int B, const double* theta, int n_trials, int probe_steps,
                      double* times_out);

/* Chains: n_chains independent random-walk Metropolis chains advanced in
 * lock-step, one proposal per chain per step (Algorithm 1).
 * theta0:   host [C][n_params] starting points
 * seed:     Philox key; chain c at its step s draws from counters (c, s, 0|1, 0)
 * step:     host [n_params] random-walk standard deviations in step space
 * size_idx: host [C] grid size of each chain, or NULL (all 0)
 * capacity: samples kept on the device before rd_chains_read_samples must be
 *           called (each sample = [n_params][C] doubles). */
rd_status rd_chains_create(rd_problem* p, int n_chains, const double* theta0,
                           uint64_t seed, const double* step,
                           const int* size_idx, int capacity,
                           rd_chains** out);
rd_status rd_chains_destroy(rd_chains* c);

/* Replaces the random-walk increments by a correlated Gaussian: the proposal
 * in step space is eta + L xi with L (host, [n_params][n_params], row-major,
 * lower-triangular; entries above the diagonal are ignored) and xi the chain's
 * standard normals.  The walk stays symmetric, so Algorithm 1's acceptance is
 * unchanged.  L = diag(step) is the sampler rd_chains_create sets up. */
rd_status rd_chains_set_proposal(rd_chains* c, const double* L);

/* Global index of this object's chain 0 in the random-number counters
 * (default 0): chain i draws at step s from counters (first + i, s, 0|1, 0).
 * Chains split over several objects -- one per GPU, each taking a contiguous
 * range of a run's chains with first = the range's start and the same seed --
 * then draw exactly the numbers the chains of one object of the total size
 * would (Sec. 2.1: many independent chains, pooled afterwards).  Set it
 * before the first rd_chains_run; it is not part of a checkpoint.  EINVAL if
 * first + n_chains exceeds 2^32. */
rd_status rd_chains_set_first_chain(rd_chains* c, uint32_t first);

/* Switches the chains to the multi-proposal parallel Metropolis-Hastings step
 * of Sec. 2.1 (Algorithm 2) with n_prop = N proposals per chain and step
 * (1..RD_PMH_MAX_PROPOSALS; 0 = back to Algorithm 1).  Per step and chain:
 * an auxiliary point z = x_k + L xi_0, N proposals z + L xi_t (t = 1..N, the
 * random numbers of point t at counters (chain, step, 0|1, t)), their
 * forward solves in the same batched launch as every other chain's, the
 * stationary distribution of the (N+1)-state chain
 * A(i, j) = min(1, target(x^j) / target(x^i)) / N (j != i), A(i, i) = 1 - the
 * row's other entries (solved in FP64), and N draws from it (draw t uses u_6
 * of point t); the draws are the step's N samples and the last is the new
 * state.  Proposals drawn around z rather than x_k make the N+1 points'
 * proposal symmetric, as the method needs to leave the posterior invariant.
 * Each step then writes N samples to the ring (capacity counts samples), and
 * rd_chains_read_samples' counters count N proposals per chain-step,
 * accepted = draws other than x_k.  Allocates the step's buffers; EINVAL with
 * a surrogate set (delayed acceptance works with Algorithm 1 only). */
rd_status rd_chains_set_parallel_proposals(rd_chains* c, int n_prop);

/* Advances every chain by n_steps (async; graph-replayed per step).
 * ESTATE if the sample buffer would overflow. */
rd_status rd_chains_run(rd_chains* c, int n_steps);

/* Copies the samples accumulated since the last read into out (host,
 * [n][n_params][C]; n <= cap_steps), sets *n_written, and fills
 * counters[4] (if non-NULL) with the totals since creation: proposals,
 * stage-1 survivors, accepted, exact solves.  Synchronises the stream. */
rd_status rd_chains_read_samples(rd_chains* c, double* out, size_t cap_steps,
                                 size_t* n_written, double* counters);

/* Current state: theta (host [C][n_params]), phi (host [C]); either may be
 * NULL.  Synchronises the stream. */
rd_status rd_chains_get_state(rd_chains* c, double* theta, double* phi);

/* Checkpoint of the full chain state (theta, Phi, surrogate Phi~, log prior,
 * step counter, counters) into host memory; *n = bytes needed.  With
 * buf == NULL only *n is set.  Restoring it into chains created with the same
 * problem, C and seed continues the chains bit-identically. */
rd_status rd_chains_checkpoint(rd_chains* c, void* buf, size_t cap, size_t* n);
rd_status rd_chains_restore(rd_chains* c, const void* buf, size_t n);

/*
 * Learned surrogate for delayed-acceptance sampling (not in the paper; the
 * two-stage acceptance of Christen & Fox 2005, which keeps the posterior
 * exact for any surrogate).  Network: x -> SiLU(W1 x + b1) -> SiLU(W2 . + b2)
 * -> SiLU(W3 . + b3) -> W4 . + b4, width RD_SURROGATE_WIDTH, inputs
 * x_j = (log theta_j - mu_j) / s_j for the n_params inferred parameters
 * (padded to 16), output Phi~ = floor + exp(shift + scale * net).  BF16
 * weights and activations, FP32 accumulation on the tensor cores, FP32 master
 * weights.  Parameters (FP32, host order): W1 [W][16], b1 [W], W2 [W][W], b2,
 * W3 [W][W], b3, W4 [W], b4 [1].  Normalisation vector (13 doubles):
 * mu[5], s[5], floor, shift, scale.
 */
typedef struct {
  int epochs;          /* passes over the training pairs (>= 1) */
  int batch;           /* minibatch rows, a positive multiple of 128 */
  double lr, beta1, beta2, weight_decay;  /* Adam with decoupled weight decay */
  double holdout_frac; /* fraction of pairs held out for the error report */
  uint64_t seed;       /* shuffling */
} rd_train_desc;

/* Creates a surrogate for problem p with seeded He-uniform initial weights. */
rd_status rd_surrogate_create(rd_problem* p, uint64_t seed, rd_surrogate** out);
rd_status rd_surrogate_destroy(rd_surrogate* s);

/* Trains on n pairs (device theta [n][n_params], device Phi [n]; pairs with
 * non-finite Phi are skipped): sets the normalisation from the data (inputs:
 * mean/sd of log theta; targets: z = log(Phi - floor), floor = min Phi - 1,
 * standardised), then minimises the mean squared error on z with Adam.
 * report (host, may be NULL) [4]: final-epoch training MSE, hold-out MSE,
 * hold-out mean relative |Phi~ - Phi| / Phi, wall seconds.  Synchronous. */
rd_status rd_surrogate_train(rd_surrogate* s, int n, const double* theta,
                             const double* phi, const rd_train_desc* td,
                             double* report);

/* Phi~ for B parameter vectors (device theta [B][n_params], device out [B]);
 * async on the problem's stream. */
rd_status rd_surrogate_predict(rd_surrogate* s, int B, const double* theta,
                               double* phi_tilde);

/* Mean squared error of the network output against normalised targets
 * (device float [B]) for B rows of theta (B a multiple of 128), and its
 * gradient with respect to every parameter (device float, parameter order;
 * may be NULL).  *loss is written on the host.  Synchronous. */
rd_status rd_surrogate_loss_grad(rd_surrogate* s, int B, const double* theta,
                                 const float* target, double* loss,
                                 float* grads);

/* Parameters (host FP32, *n = count; buf may be NULL to query) and the
 * normalisation (host, 13 doubles; may be NULL). */
rd_status rd_surrogate_get_params(rd_surrogate* s, float* buf, size_t cap,
                                  size_t* n, double* norm);
rd_status rd_surrogate_set_params(rd_surrogate* s, const float* buf, size_t n,
                                  const double* norm);

/* Switches chains to delayed acceptance with surrogate s (NULL: back to plain
 * Metropolis).  Each step then draws the proposal, evaluates Phi~ for every
 * chain, accepts to stage 2 with probability
 * min(1, exp(-Phi~(x_bar) + log mu0(x_bar) + Phi~(x) - log mu0(x))) (uniform
 * u_6), solves the forward problem only for stage-2 candidates, and accepts
 * with min(1, exp(Phi(x) - Phi(x_bar) + Phi~(x_bar) - Phi~(x))) (uniform
 * u_7).  The surrogate must outlive its use by the chains. */
rd_status rd_chains_set_surrogate(rd_chains* c, rd_surrogate* s);

/* Blocks until all work enqueued on the problem's stream has finished, then
 * returns RD_ETIMEOUT (and clears the flag) if a solve kernel's bounded wait
 * gave up since the last check: its unsolved proposals keep status
 * RD_P_NOT_SOLVED and Phi = +inf. */
rd_status rd_sync(rd_problem* p);

/* Limit of every bounded wait inside the tensor-core solve kernels (default
 * 4 s; (0, 60] seconds).  A healthy wait lasts microseconds; a wait that runs
 * out makes the kernel's CTA stop popping work, drain the MMAs it issued,
 * free its tensor memory and raise the problem's error flag, which rd_sync and
 * rd_evaluate_batch_host report as RD_ETIMEOUT.  The context stays usable.
 * Takes effect at the next launch (captured chain steps are re-captured). */
rd_status rd_set_wait_limit(rd_problem* p, double seconds);

/* Test aid for the failure path above (not part of the method): with
 * step >= 0, the MMA-issuing warp of every tensor-core solve CTA, after
 * issuing stage 1 of IMEX step `step` of its first proposal, waits on a
 * barrier that nothing completes instead of going on.  That wait, and then
 * every other wait of the CTA, runs out after the wait limit, so the launch
 * ends in bounded time with RD_ETIMEOUT and every proposal of the batch left
 * RD_P_NOT_SOLVED.  step = -1 (the default) turns it off.  CUDA-core kernels
 * have no waits and ignore it. */
rd_status rd_debug_stall_at_step(rd_problem* p, int step);

/* Message of the last failed call on this thread ("" if none). */
const char* rd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RDBAYES_H */
