/*
 * rd_oracle.c -- plain, slow FP64 CPU oracle for the Bayesian identification
 * of Schnakenberg reaction-diffusion parameters (Campillo-Funollet,
 * Venkataraman, Madzvamuse, arXiv:1605.04718).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * do.  It shares no source with the CUDA library.
 *
 * What it computes, step by step and in the paper's notation:
 *   - the forward model G (Sec. 3.1, eq. (schnakenberg) with the kinetics of
 *     eq. (reactions)), discretised with the 3/5-point Neumann Laplacian of
 *     Sec. 3.1.1 on a cell-centred grid x_i = (i + 1/2) h, h = 1/N, and a
 *     first-order IMEX Euler step: reaction explicit, diffusion and the
 *     linear dilution term implicit;
 *   - the implicit solve: in 1-D by the Thomas algorithm on the tridiagonal
 *     Neumann matrix, in 2-D by diagonalising the Neumann Laplacian in its
 *     eigenbasis (the orthonormal DCT-II, applied as plain dense sums), with a
 *     conjugate-gradient solve (the paper's own linear solver, Sec. 3.1.1) kept
 *     as an independent 2-D cross-check;
 *   - the Gaussian log-likelihood Phi(p; y) = -log rho(y - G(p)) of eq. (logl),
 *     i.e. sum (y - G)^2 / (2 sigma^2);
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
 *     generator both sides implement from its published definition, and the
 *     Box-Muller transform.
 *
 * Status bits per forward solve: 2 = non-finite or |w| > w_max at an
 * observation time (the "robust" log-likelihood of Sec. 2: such a parameter
 * gets Phi = +inf and is rejected).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ST_OUT_OF_SUPPORT 1u
#define ORC_ST_NONFINITE 2u
#define ORC_ST_NOT_CONVERGED 4u
#define ORC_NPHYS 8 /* (a, b, d, gamma, r, p1, p2, p3) */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of the 4x32 S-box            */
/* built from two 32x32->64 multiplications, key bumped by the Weyl           */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

/* Uniform in the open interval (0, 1): (w + 1/2) * 2^-32. */
static double word_to_uniform(uint32_t w) {
  return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/*
 * Random numbers of one chain at one MCMC step.  Two Philox blocks with
 * counters (first + chain, step, 0, point) and (first + chain, step, 1,
 * point) -- first = the global index of chain 0 when the chains are split
 * over several processes, 0 otherwise; point = 0 for Algorithm 1, the point's
 * index 0..N under the multi-proposal Algorithm 2 -- key = the 64-bit seed
 * split into (low, high) words, give 8 uniforms u_0..u_7:
 *   u_0..u_5 -> three Box-Muller pairs -> standard normals xi_0..xi_5
 *               (xi_{2j} = sqrt(-2 ln u_{2j}) cos(2 pi u_{2j+1}),
 *                xi_{2j+1} = sqrt(-2 ln u_{2j}) sin(2 pi u_{2j+1}));
 *   u_6       -> the Metropolis (or delayed-acceptance stage-1) uniform;
 *   u_7       -> the delayed-acceptance stage-2 uniform.
 */
void orc_chain_randoms_pt(uint64_t seed, uint32_t first, int n_chains, uint32_t step,
                          uint32_t point, double* normals /* [n_chains][6] */,
                          double* uniforms /* [n_chains][2] */) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int c = 0; c < n_chains; ++c) {
    uint32_t w[8];
    uint32_t ctr0[4] = {first + (uint32_t)c, step, 0u, point};
    uint32_t ctr1[4] = {first + (uint32_t)c, step, 1u, point};
    orc_philox4x32_10(ctr0, key, w);
    orc_philox4x32_10(ctr1, key, w + 4);
    double u[8];
    for (int i = 0; i < 8; ++i) u[i] = word_to_uniform(w[i]);
    for (int j = 0; j < 3; ++j) {
      double rad = sqrt(-2.0 * log(u[2 * j]));
      double ang = two_pi * u[2 * j + 1];
      normals[(size_t)c * 6 + 2 * j] = rad * cos(ang);
      normals[(size_t)c * 6 + 2 * j + 1] = rad * sin(ang);
    }
    uniforms[(size_t)c * 2 + 0] = u[6];
    uniforms[(size_t)c * 2 + 1] = u[7];
  }
}

void orc_chain_randoms_from(uint64_t seed, uint32_t first, int n_chains, uint32_t step,
                            double* normals, double* uniforms) {
  orc_chain_randoms_pt(seed, first, n_chains, step, 0u, normals, uniforms);
}

void orc_chain_randoms(uint64_t seed, int n_chains, uint32_t step, double* normals,
                       double* uniforms) {
  orc_chain_randoms_pt(seed, 0u, n_chains, step, 0u, normals, uniforms);
}

/* ------------------------------------------------------------------------ */
/* Implicit solves of  [alpha I - beta_h Lap_h] w = rhs  with the Neumann     */
/* Laplacian of Sec. 3.1.1 on a cell-centred grid (ghost values mirror the    */
/* boundary values).  beta_h = tau D / (rho^2 h^2) multiplies the stencil     */
/* weights (w_{i-1} - 2 w_i + w_{i+1}).                                       */
/* ------------------------------------------------------------------------ */

/* 1-D: Thomas algorithm on the tridiagonal matrix with diagonal
 * alpha + 2 beta_h (alpha + beta_h in the two boundary rows) and
 * off-diagonals -beta_h. */
void orc_solve1d_thomas(int n, double alpha, double beta_h, const double* rhs,
                        double* x) {
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (n == 1) {
    x[0] = rhs[0] / alpha;
    free(cp);
    free(dp);
    return;
  }
  for (int i = 0; i < n; ++i) {
    double diag = alpha + ((i == 0 || i == n - 1) ? beta_h : 2.0 * beta_h);
    double lower = (i > 0) ? -beta_h : 0.0;
    double upper = (i < n - 1) ? -beta_h : 0.0;
    double denom = diag - (i > 0 ? lower * cp[i - 1] : 0.0);
    cp[i] = upper / denom;
    dp[i] = (rhs[i] - (i > 0 ? lower * dp[i - 1] : 0.0)) / denom;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
}

/* 1-D: Thomas algorithm for [diag(alpha_i) - beta_h Lap_h] x = rhs (a
 * node-dependent alpha, as the linearised reaction terms of the paper's
 * semi-implicit scheme give). */
void orc_solve1d_thomas_var(int n, const double* alpha, double beta_h, const double* rhs,
                            double* x) {
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (n == 1) {
    x[0] = rhs[0] / alpha[0];
    free(cp);
    free(dp);
    return;
  }
  for (int i = 0; i < n; ++i) {
    double diag = alpha[i] + ((i == 0 || i == n - 1) ? beta_h : 2.0 * beta_h);
    double lower = (i > 0) ? -beta_h : 0.0;
    double upper = (i < n - 1) ? -beta_h : 0.0;
    double denom = diag - (i > 0 ? lower * cp[i - 1] : 0.0);
    cp[i] = upper / denom;
    dp[i] = (rhs[i] - (i > 0 ? lower * dp[i - 1] : 0.0)) / denom;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
}

/* Orthonormal DCT-II matrix: C[k][i] = c_k cos(pi k (i + 1/2) / N),
 * c_0 = sqrt(1/N), c_k = sqrt(2/N).  Its rows are the eigenvectors of the
 * cell-centred Neumann Laplacian; the eigenvalue of -Lap_h (times h^2) for
 * row k is 4 sin^2(pi k / (2N)). */
void orc_dct_matrix(int n, double* c) {
  const double pi = 3.14159265358979323846264338327950288;
  for (int k = 0; k < n; ++k) {
    double ck = (k == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    for (int i = 0; i < n; ++i)
      c[(size_t)k * n + i] = ck * cos(pi * k * (i + 0.5) / n);
  }
}

double orc_laplacian_eig(int n, int k) {
  const double pi = 3.14159265358979323846264338327950288;
  double s = sin(pi * k / (2.0 * n));
  return 4.0 * s * s;
}

/* 2-D solve by diagonalisation: w_hat = C rhs C^T, divide mode (l, k) by
 * alpha + beta_h (mu_l + mu_k), w = C^T w_hat C.  rhs and x are [N][N] with
 * the first index along y.  c = orc_dct_matrix, mu[k] = orc_laplacian_eig,
 * t and s are N*N scratch arrays.  x may alias rhs. */
static void solve2d_dct_ws(int n, double alpha, double beta_h, const double* c,
                           const double* mu, double* t, double* s,
                           const double* rhs, double* x) {
  size_t nn = (size_t)n * n;
  /* t[y][k] = sum_x rhs[y][x] C[k][x] */
  for (int y = 0; y < n; ++y)
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int xx = 0; xx < n; ++xx)
        acc += rhs[(size_t)y * n + xx] * c[(size_t)k * n + xx];
      t[(size_t)y * n + k] = acc;
    }
  /* s[l][k] = sum_y C[l][y] t[y][k]  (loop order keeps the inner loop
   * contiguous; each s[l][k] is still the plain sum over y in order) */
  memset(s, 0, sizeof(double) * nn);
  for (int l = 0; l < n; ++l)
    for (int y = 0; y < n; ++y) {
      double cly = c[(size_t)l * n + y];
      for (int k = 0; k < n; ++k) s[(size_t)l * n + k] += cly * t[(size_t)y * n + k];
    }
  for (int l = 0; l < n; ++l)
    for (int k = 0; k < n; ++k)
      s[(size_t)l * n + k] /= alpha + beta_h * (mu[l] + mu[k]);
  /* t[y][k] = sum_l C[l][y] s[l][k] */
  memset(t, 0, sizeof(double) * nn);
  for (int y = 0; y < n; ++y)
    for (int l = 0; l < n; ++l) {
      double cly = c[(size_t)l * n + y];
      for (int k = 0; k < n; ++k) t[(size_t)y * n + k] += cly * s[(size_t)l * n + k];
    }
  /* x[y][x] = sum_k t[y][k] C[k][x] */
  for (int y = 0; y < n; ++y) {
    double* row = x + (size_t)y * n;
    for (int xx = 0; xx < n; ++xx) row[xx] = 0.0;
    for (int k = 0; k < n; ++k) {
      double tyk = t[(size_t)y * n + k];
      for (int xx = 0; xx < n; ++xx) row[xx] += tyk * c[(size_t)k * n + xx];
    }
  }
}

void orc_solve2d_dct(int n, double alpha, double beta_h, const double* rhs,
                     double* x) {
  size_t nn = (size_t)n * n;
  double* c = (double*)malloc(sizeof(double) * nn);
  double* t = (double*)malloc(sizeof(double) * nn);
  double* s = (double*)malloc(sizeof(double) * nn);
  double* mu = (double*)malloc(sizeof(double) * (size_t)n);
  orc_dct_matrix(n, c);
  for (int k = 0; k < n; ++k) mu[k] = orc_laplacian_eig(n, k);
  solve2d_dct_ws(n, alpha, beta_h, c, mu, t, s, rhs, x);
  free(c);
  free(t);
  free(s);
  free(mu);
}

/* Apply A = alpha I - beta_h Lap_h (5-point, Neumann by mirroring). */
static void apply_op2d(int n, double alpha, double beta_h, const double* w,
                       double* out) {
  for (int y = 0; y < n; ++y)
    for (int xx = 0; xx < n; ++xx) {
      double c0 = w[(size_t)y * n + xx];
      double wl = xx > 0 ? w[(size_t)y * n + xx - 1] : c0;
      double wr = xx < n - 1 ? w[(size_t)y * n + xx + 1] : c0;
      double wd = y > 0 ? w[(size_t)(y - 1) * n + xx] : c0;
      double wu = y < n - 1 ? w[(size_t)(y + 1) * n + xx] : c0;
      out[(size_t)y * n + xx] =
          alpha * c0 - beta_h * (wl + wr + wd + wu - 4.0 * c0);
    }
}

/* 2-D solve by plain conjugate gradients (the paper's linear solver), from a
 * zero start, to a relative residual of rtol.  Returns the iteration count,
 * or -1 if max_iter was reached. */
int orc_solve2d_cg(int n, double alpha, double beta_h, const double* rhs,
                   double* x, double rtol, int max_iter) {
  size_t nn = (size_t)n * n;
  double* r = (double*)malloc(sizeof(double) * nn);
  double* p = (double*)malloc(sizeof(double) * nn);
  double* q = (double*)malloc(sizeof(double) * nn);
  double bnorm2 = 0.0, rr = 0.0;
  for (size_t i = 0; i < nn; ++i) {
    x[i] = 0.0;
    r[i] = rhs[i];
    p[i] = rhs[i];
    bnorm2 += rhs[i] * rhs[i];
  }
  rr = bnorm2;
  int it = 0;
  int done = (bnorm2 == 0.0);
  while (!done && it < max_iter) {
    apply_op2d(n, alpha, beta_h, p, q);
    double pq = 0.0;
    for (size_t i = 0; i < nn; ++i) pq += p[i] * q[i];
    double step = rr / pq;
    double rr_new = 0.0;
    for (size_t i = 0; i < nn; ++i) {
      x[i] += step * p[i];
      r[i] -= step * q[i];
      rr_new += r[i] * r[i];
    }
    ++it;
    if (rr_new <= rtol * rtol * bnorm2) done = 1;
    double beta_cg = rr_new / rr;
    rr = rr_new;
    for (size_t i = 0; i < nn; ++i) p[i] = r[i] + beta_cg * p[i];
  }
  free(r);
  free(p);
  free(q);
  return done ? it : -1;
}

/* Apply A = diag(alpha_i) - beta_h Lap_h (5-point, Neumann by mirroring):
 * the operator of the paper's semi-implicit step, whose linearised reaction
 * terms make the diagonal depend on the node. */
static void apply_op2d_var(int n, const double* alpha, double beta_h, const double* w,
                           double* out) {
  for (int y = 0; y < n; ++y)
    for (int xx = 0; xx < n; ++xx) {
      size_t i = (size_t)y * n + xx;
      double c0 = w[i];
      double wl = xx > 0 ? w[i - 1] : c0;
      double wr = xx < n - 1 ? w[i + 1] : c0;
      double wd = y > 0 ? w[i - n] : c0;
      double wu = y < n - 1 ? w[i + n] : c0;
      out[i] = alpha[i] * c0 - beta_h * (wl + wr + wd + wu - 4.0 * c0);
    }
}

/* 2-D solve of [diag(alpha_i) - beta_h Lap_h] x = rhs by plain conjugate
 * gradients (the paper's linear solver), from a zero start, to a relative
 * residual of rtol.  Returns the iteration count, or -1 if max_iter was
 * reached. */
int orc_solve2d_cg_var(int n, const double* alpha, double beta_h, const double* rhs,
                       double* x, double rtol, int max_iter) {
  size_t nn = (size_t)n * n;
  double* r = (double*)malloc(sizeof(double) * nn);
  double* p = (double*)malloc(sizeof(double) * nn);
  double* q = (double*)malloc(sizeof(double) * nn);
  double bnorm2 = 0.0;
  for (size_t i = 0; i < nn; ++i) {
    x[i] = 0.0;
    r[i] = rhs[i];
    p[i] = rhs[i];
    bnorm2 += rhs[i] * rhs[i];
  }
  double rr = bnorm2;
  int it = 0;
  int done = (bnorm2 == 0.0);
  while (!done && it < max_iter) {
    apply_op2d_var(n, alpha, beta_h, p, q);
    double pq = 0.0;
    for (size_t i = 0; i < nn; ++i) pq += p[i] * q[i];
    double step = rr / pq;
    double rr_new = 0.0;
    for (size_t i = 0; i < nn; ++i) {
      x[i] += step * p[i];
      r[i] -= step * q[i];
      rr_new += r[i] * r[i];
    }
    ++it;
    if (rr_new <= rtol * rtol * bnorm2) done = 1;
    double beta_cg = rr_new / rr;
    rr = rr_new;
    for (size_t i = 0; i < nn; ++i) p[i] = r[i] + beta_cg * p[i];
  }
  free(r);
  free(p);
  free(q);
  return done ? it : -1;
}

/* ------------------------------------------------------------------------ */
/* Forward model and log-likelihood                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dim;               /* 1 or 2 */
  int n;                 /* grid points per side */
  int n_steps;           /* time steps to the final time T = n_steps * tau */
  double tau;            /* time step */
  int m_growth;          /* m of eq. (schnakenberg): the spatial dimension */
  int n_obs;             /* number of observation times */
  const int* obs_steps;  /* [n_obs] step indices in 1..n_steps, increasing */
  int field_mask;        /* bit 0: u observed, bit 1: v observed */
  const double* y;       /* [n_obs][observed fields][n^dim] */
  double sigma;          /* noise standard deviation */
  const double* u0;      /* [n^dim] initial condition */
  const double* v0;
  double w_max;          /* |w| above this at an observation => divergent */
  int solver;            /* 2-D only: 0 = DCT diagonalisation, 1 = CG */
  int scheme;            /* 0 = IMEX (reaction explicit), 1 = the paper's
                            semi-implicit scheme (one Picard iterate) */
  int growth_kind;       /* ORC_GROWTH_*: the law of rho(t) (orc_growth) */
  double rho_T;          /* polynomial law: the known final size rho(T) */
  double logistic_K;     /* logistic law: the carrying capacity */
} orc_problem;

/* Domain growth laws rho(t) of eq. (schnakenberg), rho(0) = 1:
 *  ORC_GROWTH_EXP:      rho = exp(r t), r = theta[4] (r = 0: fixed domain);
 *  ORC_GROWTH_POLY4:    the finite-dimensional approximation of Example 1
 *    (Sec. 3.1.1): a degree-4 polynomial in s = t / T with the coefficients of
 *    order 0 and 4 fixed by rho(0) = 1 and rho(T) = rho_T, so three degrees
 *    of freedom p1, p2, p3 = theta[5..7]:
 *      rho = 1 + p1 s + p2 s^2 + p3 s^3 + p4 s^4,  p4 = rho_T - 1 - p1 - p2 - p3;
 *  ORC_GROWTH_LOGISTIC: eq. (grates)' logistic law with rate lambda = theta[4]
 *    and carrying capacity K, rho = e^{lambda t} / (1 + (e^{lambda t} - 1) / K),
 *    the solution of rho' = lambda rho (1 - rho / K). */
#define ORC_GROWTH_EXP 0
#define ORC_GROWTH_POLY4 1
#define ORC_GROWTH_LOGISTIC 2

/* rho(t) and rho'(t) / rho(t) of the law `kind` (T = final time). */
void orc_growth(int kind, const double* theta, double rho_T, double K, double T, double t,
                double* rho, double* rdot_over_rho) {
  if (kind == ORC_GROWTH_POLY4) {
    const double p1 = theta[5], p2 = theta[6], p3 = theta[7];
    const double p4 = rho_T - 1.0 - p1 - p2 - p3;
    const double sv = t / T;
    const double r = 1.0 + sv * (p1 + sv * (p2 + sv * (p3 + sv * p4)));
    const double drds = p1 + sv * (2.0 * p2 + sv * (3.0 * p3 + sv * 4.0 * p4));
    *rho = r;
    *rdot_over_rho = drds / T / r;
  } else if (kind == ORC_GROWTH_LOGISTIC) {
    const double lam = theta[4];
    const double e = exp(lam * t);
    const double r = e / (1.0 + (e - 1.0) / K);
    *rho = r;
    *rdot_over_rho = lam * (1.0 - r / K);
  } else {
    *rho = exp(theta[4] * t);
    *rdot_over_rho = theta[4];
  }
}

/*
 * One forward solve G(p) and its log-likelihood Phi(p; y).
 * theta = (a, b, d, gamma, r, p1, p2, p3): kinetics of eq. (reactions),
 * diffusion ratio d, scale gamma, and the growth law's parameters (orc_growth;
 * r = 0 with the exponential law: fixed domain).
 * Step n -> n+1 (t_n = n tau, rho_n = rho(t_n), q_n = rho'(t_n) / rho(t_n)):
 *   ru = u + tau gamma (a - u + u^2 v),   rv = v + tau gamma (b - u^2 v)
 *   [(1 + tau m q_n) I - tau / rho_n^2 Lap_h] u^{n+1} = ru
 *   [(1 + tau m q_n) I - tau d / rho_n^2 Lap_h] v^{n+1} = rv
 * With scheme = 1 the step is the paper's semi-implicit one (Sec. 3.1.1,
 * Example 1): diffusion, dilution and the linearised reaction implicit, one
 * Picard iterate (u^n, v^n in the nonlinear coefficients), each system
 * solved by the Thomas algorithm (1-D) or plain CG to 1e-14 (2-D):
 *   [(1 + tau m q_n + tau gamma (1 - u^n v^n)) I - tau / rho_n^2 Lap_h] u^{n+1}
 *       = u^n + tau gamma a
 *   [(1 + tau m q_n + tau gamma (u^n)^2) I - tau d / rho_n^2 Lap_h] v^{n+1}
 *       = v^n + tau gamma b
 * At each observation step the misfit (y - w)^2 / (2 sigma^2) of the observed
 * fields is added to Phi.  A growth law that reaches rho <= 0 flags the solve
 * non-finite.  Returns the status bits; Phi = +inf if nonzero.
 */
uint32_t orc_forward(const orc_problem* pb, const double* theta, double* phi_out,
                     double* u_out, double* v_out, double* obs_out) {
  const double a = theta[0], b = theta[1], d = theta[2], g = theta[3],
               r = theta[4];
  const int n = pb->n;
  const size_t npts = (pb->dim == 1) ? (size_t)n : (size_t)n * n;
  const double h = 1.0 / n;
  const double tau = pb->tau;
  double* u = (double*)malloc(sizeof(double) * npts);
  double* v = (double*)malloc(sizeof(double) * npts);
  double* ru = (double*)malloc(sizeof(double) * npts);
  double* rv = (double*)malloc(sizeof(double) * npts);
  double* t_au = (double*)malloc(sizeof(double) * npts);
  double* t_av = (double*)malloc(sizeof(double) * npts);
  memcpy(u, pb->u0, sizeof(double) * npts);
  memcpy(v, pb->v0, sizeof(double) * npts);
  double *c = NULL, *mu = NULL, *t = NULL, *s = NULL;
  if (pb->dim == 2) {
    c = (double*)malloc(sizeof(double) * npts);
    t = (double*)malloc(sizeof(double) * npts);
    s = (double*)malloc(sizeof(double) * npts);
    mu = (double*)malloc(sizeof(double) * (size_t)n);
    orc_dct_matrix(n, c);
    for (int k = 0; k < n; ++k) mu[k] = orc_laplacian_eig(n, k);
  }
  double phi = 0.0;
  uint32_t status = 0;
  int next_obs = 0;
  const int nf_obs = ((pb->field_mask & 1) ? 1 : 0) + ((pb->field_mask & 2) ? 1 : 0);
  const double T_final = (double)pb->n_steps * tau;
  for (int step = 0; step < pb->n_steps; ++step) {
    double t_n = (double)step * tau;
    double rho = exp(r * t_n);
    double alpha = 1.0 + tau * pb->m_growth * r;
    if (pb->growth_kind != ORC_GROWTH_EXP) {
      double q;
      orc_growth(pb->growth_kind, theta, pb->rho_T, pb->logistic_K, T_final, t_n, &rho, &q);
      if (!(rho > 0.0)) {
        status |= ORC_ST_NONFINITE;
        break;
      }
      alpha = 1.0 + tau * pb->m_growth * q;
    }
    double bu = tau * 1.0 / (rho * rho) / (h * h);
    double bv = tau * d / (rho * rho) / (h * h);
    if (pb->scheme == 1) {
      for (size_t i = 0; i < npts; ++i) {
        t_au[i] = alpha + tau * g * (1.0 - u[i] * v[i]);
        t_av[i] = alpha + tau * g * u[i] * u[i];
        ru[i] = u[i] + tau * g * a;
        rv[i] = v[i] + tau * g * b;
      }
      if (pb->dim == 1) {
        orc_solve1d_thomas_var(n, t_au, bu, ru, u);
        orc_solve1d_thomas_var(n, t_av, bv, rv, v);
      } else if (orc_solve2d_cg_var(n, t_au, bu, ru, u, 1e-14, 50 * n * n) < 0 ||
                 orc_solve2d_cg_var(n, t_av, bv, rv, v, 1e-14, 50 * n * n) < 0) {
        status |= ORC_ST_NOT_CONVERGED;
      }
    } else {  /* IMEX: reaction explicit */
      for (size_t i = 0; i < npts; ++i) {
        double uu = u[i], vv = v[i];
        double u2v = uu * uu * vv;
        ru[i] = uu + tau * g * (a - uu + u2v);
        rv[i] = vv + tau * g * (b - u2v);
      }
      if (pb->dim == 1) {
        orc_solve1d_thomas(n, alpha, bu, ru, u);
        orc_solve1d_thomas(n, alpha, bv, rv, v);
      } else if (pb->solver == 1) {
        if (orc_solve2d_cg(n, alpha, bu, ru, u, 1e-14, 50 * n * n) < 0 ||
            orc_solve2d_cg(n, alpha, bv, rv, v, 1e-14, 50 * n * n) < 0)
          status |= ORC_ST_NOT_CONVERGED;
      } else {
        solve2d_dct_ws(n, alpha, bu, c, mu, t, s, ru, u);
        solve2d_dct_ws(n, alpha, bv, c, mu, t, s, rv, v);
      }
    }
    if (next_obs < pb->n_obs && pb->obs_steps[next_obs] == step + 1) {
      const double* yo = pb->y + (size_t)next_obs * nf_obs * npts;
      int fo = 0;
      for (int f = 0; f < 2; ++f) {
        if (!(pb->field_mask & (1 << f))) continue;
        const double* w = (f == 0) ? u : v;
        const double* yf = yo + (size_t)fo * npts;
        if (obs_out)
          memcpy(obs_out + ((size_t)next_obs * nf_obs + fo) * npts, w,
                 sizeof(double) * npts);
        for (size_t i = 0; i < npts; ++i) {
          if (!isfinite(w[i]) || fabs(w[i]) > pb->w_max) status |= ORC_ST_NONFINITE;
          double e = yf[i] - w[i];
          phi += e * e / (2.0 * pb->sigma * pb->sigma);
        }
        ++fo;
      }
      ++next_obs;
    }
  }
  if (status) phi = INFINITY;
  *phi_out = phi;
  if (u_out) memcpy(u_out, u, sizeof(double) * npts);
  if (v_out) memcpy(v_out, v, sizeof(double) * npts);
  free(u);
  free(v);
  free(ru);
  free(rv);
  free(t_au);
  free(t_av);
  free(c);
  free(mu);
  free(t);
  free(s);
  return status;
}

typedef struct {
  const orc_problem* pb;
  const double* theta;
  double* phi;
  uint32_t* status;
  double* fields;
  int begin, end;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* j = (batch_job*)arg;
  size_t npts = (j->pb->dim == 1) ? (size_t)j->pb->n : (size_t)j->pb->n * j->pb->n;
  for (int i = j->begin; i < j->end; ++i) {
    double* uo = j->fields ? j->fields + (size_t)i * 2 * npts : NULL;
    double* vo = j->fields ? uo + npts : NULL;
    j->status[i] = orc_forward(j->pb, j->theta + (size_t)i * ORC_NPHYS, &j->phi[i], uo, vo,
                               NULL);
  }
  return NULL;
}

/* Forward solves for B parameter vectors ([B][ORC_NPHYS]) on n_threads host threads,
 * one proposal per thread at a time. */
void orc_forward_batch(const orc_problem* pb, int B, const double* theta,
                       double* phi, uint32_t* status, double* fields,
                       int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > B) n_threads = B > 0 ? B : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  batch_job* jobs = (batch_job*)malloc(sizeof(batch_job) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].pb = pb;
    jobs[t].theta = theta;
    jobs[t].phi = phi;
    jobs[t].status = status;
    jobs[t].fields = fields;
    jobs[t].begin = (int)((long)B * t / n_threads);
    jobs[t].end = (int)((long)B * (t + 1) / n_threads);
    pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}
