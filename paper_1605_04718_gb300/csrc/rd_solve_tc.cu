// rd_solve_tc.cu -- 2-D forward solve on the tensor cores (tcgen05, TMEM).
//
// Same IMEX step as the CUDA-core path (Sec. 3.1.1 scheme with the reaction
// explicit, diffusion and dilution implicit, fields held as deviations from
// the initial-state mean), with the implicit solve done as four dense
// transforms in the Neumann eigenbasis (orthonormal DCT-II matrix C):
//   stage 1  P    = R  C^T        (transform along x)
//   stage 2  Q^T  = P^T C^T       (transform along y, result transposed)
//   scale    S^T  = Q^T o L,      L[k][l] = 1 / (alpha + beta (mu_k + mu_l))
//   stage 3  W1^T = S^T C         (inverse along y)
//   stage 4  W    = W1 C          (inverse along x)
// Every stage is one M = 128 tcgen05.mma (kind::f16, FP32 accumulation in
// TMEM) with the data as operand A and C as operand B.  Operand A alternates
// between K-major (stages 1, 3) and MN-major (stages 2, 4) so that the TMEM
// lane a thread reads is always the row it writes next.  floor(128 / N)
// proposals of an N x N grid are stacked along M and share one CTA.
//
// Precision: each FP32 operand x is split into FP16 hi + lo and each product
// is formed as hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32
// resolution), giving about 22 significant bits per element.  The data's lo
// part is stored negated (one instruction less per pair in the split) and
// the MMAs that read it negate it back (descriptor bit).  The small
// hi*lo and lo*hi products are issued before the hi*hi ones and each stage's
// output is scaled by 1 + n 2^-29 against the tensor core's round-toward-zero
// accumulation (tc_rz_comp).  Power-of-two
// stage scales keep every operand inside the FP16 normal range for field
// deviations between 0.01 and 100:
//   R' = 256 r, C' = 8 C  -> P' = 2048 P;   P'' = P' / 128 = 16 P
//   Q' = 128 Q;  S'' = Q' L / 64 = 2 S;     W1' = 16 W1;  W' = 128 W.
// The FP32 state (W' = 128 dw) and the tables L stay in TMEM for the whole
// time loop; only the operands of the next MMA live in shared memory.
//
// Warp roles (288 threads): warps 0-3 convert field u, warps 4-7 field v
// (warp w reads TMEM lanes 32 (w % 4) ...), warp 8 allocates TMEM and issues
// the MMAs, one thread, in the order u1 v1 u2 v2 ... u4 v4, so that they
// also complete in that order.  Hand-offs use mbarriers (one arrival per
// warp); every wait is bounded and a timed-out wait makes the whole CTA
// leave, free its TMEM and raise the error flag.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "rd_common.cuh"
#include "rd_internal.h"
#include "rd_tc_ptx.cuh"

namespace rd {

using namespace tc;

constexpr int kTcThreads = 288;
constexpr int kTcMaxStack = 8;  // proposals per CTA (128 / 16)

struct TcCtrl {
  uint64_t mma_done[2];   // stage MMAs of field f completed (tcgen05.commit)
  uint64_t op_ready[2];   // operand of the next stage of field f written (4 warps)
  uint64_t rx_ready;      // both fields' stage-1 operands written (8 warps)
  uint64_t fin;           // drain of in-flight MMAs at exit
  uint64_t never;         // completed by nothing (failure-path test aid)
  uint32_t tmem_base;
  int abort;
  int size;
  int n_items;
  int items[kTcMaxStack];
  int bad[kTcMaxStack];
  double phi[kTcMaxStack];
  double th[kTcMaxStack][kNPhys];
  float mu[128];
};

__host__ __device__ constexpr int tc_nblk(int n) { return (n + 63) / 64; }
__host__ __device__ constexpr uint32_t tc_tile_c(int n) { return (uint32_t)n * 128u * tc_nblk(n); }
__host__ __device__ constexpr uint32_t tc_tile_op(int n) {
  return (uint32_t)(128 * 128 * tc_nblk(n)) > (uint32_t)(n * 128 * 2)
             ? (uint32_t)(128 * 128 * tc_nblk(n))
             : (uint32_t)(n * 128 * 2);
}
// Offsets from the 1024-aligned base: C hi, C lo, then (field, hi/lo) tiles.
__host__ __device__ constexpr uint32_t tc_off_c(int nmax, int hl) { return hl * tc_tile_c(nmax); }
__host__ __device__ constexpr uint32_t tc_off_op(int nmax, int f, int hl) {
  return 2 * tc_tile_c(nmax) + (uint32_t)(2 * f + hl) * tc_tile_op(nmax);
}
__host__ __device__ constexpr uint32_t tc_off_ctrl(int nmax) {
  return 2 * tc_tile_c(nmax) + 4 * tc_tile_op(nmax);
}
// dynamic shared memory: alignment slack + tiles + control block + a guard
__host__ __device__ constexpr uint32_t tc_smem_bytes(int nmax) {
  return 1024 + tc_off_ctrl(nmax) + (uint32_t)((sizeof(TcCtrl) + 1023) / 1024 * 1024) + 4096;
}
__host__ __device__ constexpr uint32_t tc_tmem_cols(int nmax) {
  return 4 * nmax <= 32 ? 32 : 4 * nmax <= 64 ? 64 : 4 * nmax <= 128 ? 128 : 4 * nmax <= 256 ? 256 : 512;
}

// Stores 8 consecutive columns c..c+7 (c % 8 == 0) of row r, each times
// scale, as FP16 hi and negated lo parts into a swizzled tile pair (the
// split on pairs of values with the paired FP32 instructions).
__device__ __forceinline__ void store_split8(uint8_t* hi_tile, uint8_t* lo_tile, int rows,
                                             int r, int c, const float* x, float scale) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split_f16x2_neglo_scaled(x[2 * j], x[2 * j + 1], scale, h[j], l[j]);
  const uint32_t off = sw128_offset(rows, r, c);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// As store_split8 without a scale.
__device__ __forceinline__ void store_split8n(uint8_t* hi_tile, uint8_t* lo_tile, int rows,
                                              int r, int c, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split_f16x2_neglo(x[2 * j], x[2 * j + 1], h[j], l[j]);
  const uint32_t off = sw128_offset(rows, r, c);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// As store_split8 with one scale per value.
__device__ __forceinline__ void store_split8v(uint8_t* hi_tile, uint8_t* lo_tile, int rows,
                                              int r, int c, const float* x, const float* s8) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    split_f16x2_neglo_scaled2(x[2 * j], x[2 * j + 1], s8[2 * j], s8[2 * j + 1], h[j], l[j]);
  const uint32_t off = sw128_offset(rows, r, c);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Runs fn(c, v) over this lane's n accumulator columns at t_acc in chunks of
// 16 (v = the chunk's values), the next chunk's TMEM load in flight while
// the current one is converted.  n is a multiple of 16 and warp-uniform.
template <class F>
__device__ __forceinline__ void convert_cols(uint32_t t_acc, int n, F&& fn) {
  float b0[16], b1[16];
  const int nq = n / 16;
  __syncwarp();
  tmem_ld16(t_acc, b0);
  tmem_wait_ld();
#pragma unroll 1
  for (int q = 0; q < nq; q += 2) {
    const bool has1 = q + 1 < nq, has2 = q + 2 < nq;
    if (has1) tmem_ld16(t_acc + (uint32_t)(16 * (q + 1)), b1);
    fn(16 * q, b0);
    if (has1) {
      tmem_wait_ld();
      if (has2) tmem_ld16(t_acc + (uint32_t)(16 * (q + 2)), b0);
      fn(16 * (q + 1), b1);
      if (has2) tmem_wait_ld();
    }
  }
}

__device__ __forceinline__ void store_zero8(uint8_t* hi_tile, uint8_t* lo_tile, int rows, int r,
                                            int c) {
  const uint32_t off = sw128_offset(rows, r, c);
  *reinterpret_cast<uint4*>(hi_tile + off) = make_uint4(0, 0, 0, 0);
  *reinterpret_cast<uint4*>(lo_tile + off) = make_uint4(0, 0, 0, 0);
}

// Compensation of the tensor core's round-toward-zero accumulation: each
// MMA's sum is truncated toward zero, about 0.72 * 2^-24 of the accumulator
// per MMA; with the correction products issued first (small accumulator) the
// n / 16 main products of a stage leave a shrink of about (n / 16) * 0.5 *
// 2^-24 (partial sums average about 0.7 of the final value), undone by
// scaling each stage's output by 1 + kappa.
__device__ __forceinline__ float tc_rz_comp(int n) { return (float)n * 0x1p-29f; }

// Issues one stage of field f (3 split products over K = n in steps of 16):
// the correction products (hi*lo, lo*hi) of every K block first, while the
// accumulator is small, then the main products (hi*hi).
__device__ __forceinline__ void issue_stage(uint8_t* base, int nmax, int n, int stage, int f,
                                            uint32_t d_tmem) {
  const int a_mn = (stage == 2 || stage == 4) ? 1 : 0;
  const int b_mn = (stage == 3 || stage == 4) ? 1 : 0;
  const uint32_t idesc = idesc_f16_f32(128, n, a_mn, b_mn);
  const uint32_t idesc_na = idesc_f16_f32(128, n, a_mn, b_mn, 0, 1);  // A = the negated lo
  const uint32_t a_hi = smem_u32(base + tc_off_op(nmax, f, 0));
  const uint32_t a_lo = smem_u32(base + tc_off_op(nmax, f, 1));
  const uint32_t b_hi = smem_u32(base + tc_off_c(nmax, 0));
  const uint32_t b_lo = smem_u32(base + tc_off_c(nmax, 1));
  const uint32_t cstride = (uint32_t)n * 128u;  // C tile and MN-major data tile block stride
  const uint32_t a_lbo = a_mn ? cstride : 16u, b_lbo = b_mn ? cstride : 16u;
  for (int kk = 0; kk < n / 16; ++kk) {
    const uint32_t a_off = a_mn ? (uint32_t)kk * 2048u : (uint32_t)(kk >> 2) * 16384u + (kk & 3) * 32u;
    const uint32_t b_off = b_mn ? (uint32_t)kk * 2048u : (uint32_t)(kk >> 2) * cstride + (kk & 3) * 32u;
    const uint64_t ah = sdesc_sw128(a_hi + a_off, a_lbo, 1024u);
    const uint64_t al = sdesc_sw128(a_lo + a_off, a_lbo, 1024u);
    const uint64_t bh = sdesc_sw128(b_hi + b_off, b_lbo, 1024u);
    const uint64_t bl = sdesc_sw128(b_lo + b_off, b_lbo, 1024u);
    mma_f16(d_tmem, ah, bl, idesc, kk > 0 ? 1u : 0u);
    mma_f16(d_tmem, al, bh, idesc_na, 1u);
  }
  for (int kk = 0; kk < n / 16; ++kk) {  // main products last (see tc_rz_comp)
    const uint32_t a_off = a_mn ? (uint32_t)kk * 2048u : (uint32_t)(kk >> 2) * 16384u + (kk & 3) * 32u;
    const uint32_t b_off = b_mn ? (uint32_t)kk * 2048u : (uint32_t)(kk >> 2) * cstride + (kk & 3) * 32u;
    mma_f16(d_tmem, sdesc_sw128(a_hi + a_off, a_lbo, 1024u), sdesc_sw128(b_hi + b_off, b_lbo, 1024u),
            idesc, 1u);
  }
}

// Pops up to floor(128 / n_s) proposals of one grid size.
__device__ __forceinline__ void tc_pop_group(const DevProblem& pb, const WorkQueue& q,
                                             TcCtrl* ctl) {
  ctl->n_items = 0;
  for (int k = 0; k < q.n_sizes; ++k) {
    const int s = q.order[k];
    const int cnt = *((volatile int*)&q.counts[s]);
    if (*((volatile int*)&q.pops[s]) >= cnt) continue;
    const int sp = 128 / pb.sz[s].n;
    const int i = atomicAdd(&q.pops[s], sp);
    if (i >= cnt) continue;
    const int m = min(sp, cnt - i);
    for (int j = 0; j < m; ++j) ctl->items[j] = q.items[(size_t)s * q.capacity + i + j];
    ctl->n_items = m;
    ctl->size = s;
    return;
  }
}

// One converter thread: field f, TMEM lane l (stacked row).  Runs the
// reaction / observation pass and the three stage conversions of every step.
__device__ bool tc_converter(const DevProblem& pb, const DevSize& S, TcCtrl* ctl, uint8_t* base,
                             int nmax, int n, uint32_t tmem, int f, int warp, int lane,
                             uint32_t& ph_done, float* fields,
                             size_t field_stride) {
  volatile int* abort = &ctl->abort;
  const int l = 32 * (warp & 3) + lane;
  const int sp = 128 / n;
  const int p = l / n, row = l - p * n;
  const bool lane_used = p < sp;
  const bool valid = lane_used && p < ctl->n_items;
  const int pp = lane_used ? p : 0;
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t t_acc_u = tmem + lane_off, t_acc_v = tmem + lane_off + (uint32_t)n;
  const uint32_t t_acc_f = f ? t_acc_v : t_acc_u;
  const uint32_t t_lam = tmem + lane_off + (uint32_t)(2 * n + f * n);
  uint8_t* op_hi[2] = {base + tc_off_op(nmax, 0, 0), base + tc_off_op(nmax, 1, 0)};
  uint8_t* op_lo[2] = {base + tc_off_op(nmax, 0, 1), base + tc_off_op(nmax, 1, 1)};
  const double* th = ctl->th[pp];
  const double tau = pb.tau;
  const float fa = (float)th[0], fb = (float)th[1], ftg = (float)(tau * th[3]);
  const double r = th[4], dcoef = th[2];
  const float ref_u = S.ref_u, ref_v = S.ref_v;
  const int c0 = f ? n / 2 : 0, c1 = f ? n : n / 2;
  const int nfo = (S.field_mask & 1) + ((S.field_mask >> 1) & 1);
  const float mu_row = ctl->mu[row];
  const double h2inv = (double)n * n;
  double phi = 0.0;
  int bad = 0;
  int next_obs = 0;
  const float kap = tc_rz_comp(n);
  for (int step = 0;; ++step) {
    if (step > 0) {
      // stage 4 of both fields done: the fourth commit of a step completes an
      // odd phase of each mma_done, and the other field's stage-4 phase is the
      // one pending or just completed (the MMAs complete in issue order)
      if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
      ++ph_done;
      if (!mbar_wait_bounded(&ctl->mma_done[f ^ 1], 1u, abort, pb.wait_ns)) return false;
      tc_fence_after();
    }
    const bool last = (step == pb.n_steps);
    const bool obs = next_obs < S.n_obs && step == S.obs_steps[next_obs];
    const float kap_w = step > 0 ? kap : 0.f;  // the initial state is exact
    // growth factors of this step (FP64, rounded once)
    float alpha = 1.f, cu = 0.f, cv = 0.f, beta_f = 0.f;
    if (pb.growth) {
      const double rho2inv = exp(-2.0 * r * (double)step * tau);
      alpha = (float)(1.0 + tau * 2.0 * r);
      cu = (float)(-tau * 2.0 * r * (double)ref_u);
      cv = (float)(-tau * 2.0 * r * (double)ref_v);
      beta_f = (float)(tau * (f ? dcoef : 1.0) * rho2inv * h2inv);
    }
    // ---- reaction (and observation) over columns [c0, c1) of both fields
    for (int x = c0; x < c1; x += 8) {
      float wu[8], wv[8];
      __syncwarp();
      tmem_ld8(t_acc_u + (uint32_t)x, wu);
      tmem_ld8(t_acc_v + (uint32_t)x, wv);
      tmem_wait_ld();
      float du[8], dv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        du[j] = fmaf(wu[j] * (1.f / 128.f), kap_w, wu[j] * (1.f / 128.f));
        dv[j] = fmaf(wv[j] * (1.f / 128.f), kap_w, wv[j] * (1.f / 128.f));
      }
      if (valid && (obs || last)) {
        if (obs) {
          const float* yo = S.yf + (size_t)next_obs * nfo * S.npts + (size_t)row * n + x;
          int fo = 0;
          for (int ff = 0; ff < 2; ++ff) {
            if (!(S.field_mask & (1 << ff))) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const double w = ff ? (double)ref_v + (double)dv[j] : (double)ref_u + (double)du[j];
              if (!(fabs(w) <= pb.w_max)) bad = 1;
              const double e = (double)yo[(size_t)fo * S.npts + j] - w;
              phi += e * e;
            }
            ++fo;
          }
        }
        if (last && fields) {
          float* fo = fields + (size_t)ctl->items[p] * field_stride;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            fo[(size_t)row * n + x + j] = ref_u + du[j];
            fo[(size_t)S.npts + (size_t)row * n + x + j] = ref_v + dv[j];
          }
        }
      }
      if (last) continue;
      if (!lane_used) {
        store_zero8(op_hi[0], op_lo[0], 128, l, x);
        store_zero8(op_hi[1], op_lo[1], 128, l, x);
        continue;
      }
      // 256 r (the operand scale, applied through the constants: exact)
      float ru[8], rv[8];
      const float ftg8 = 256.f * ftg, cu8 = 256.f * cu, cv8 = 256.f * cv;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float uu = ref_u + du[j], vv = ref_v + dv[j];
        const float u2v = uu * uu * vv;
        ru[j] = fmaf(ftg8, fa - uu + u2v, fmaf(du[j], 256.f, cu8));
        rv[j] = fmaf(ftg8, fb - u2v, fmaf(dv[j], 256.f, cv8));
      }
      store_split8n(op_hi[0], op_lo[0], 128, l, x, ru);
      store_split8n(op_hi[1], op_lo[1], 128, l, x, rv);
    }
    if (obs) ++next_obs;
    if (last) break;
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->rx_ready);

    // ---- stage 1 -> MN-major operand of stage 2 (row y, columns p n + k)
    if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
    ++ph_done;
    tc_fence_after();
    {
      const float sc1 = (1.f / 128.f) * (1.f + kap);
      convert_cols(t_acc_f, n, [&](int k, const float* v) {
        if (!lane_used) return;
        store_split8(op_hi[f], op_lo[f], n, row, p * n + k, v, sc1);
        store_split8(op_hi[f], op_lo[f], n, row, p * n + k + 8, v + 8, sc1);
      });
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->op_ready[f]);

    // ---- stage 2 -> scale by L -> K-major operand of stage 3 (row l)
    if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
    ++ph_done;
    tc_fence_after();
    if (!pb.growth) {  // L from its TMEM table, loaded with the accumulator
      for (int c = 0; c < n; c += 8) {
        float a8[8], l8[8];
        __syncwarp();
        tmem_ld8(t_acc_f + (uint32_t)c, a8);
        tmem_ld8(t_lam + (uint32_t)c, l8);
        tmem_wait_ld();
        if (!lane_used) {
          store_zero8(op_hi[f], op_lo[f], 128, l, c);
          continue;
        }
        store_split8v(op_hi[f], op_lo[f], 128, l, c, a8, l8);
      }
    } else {
      convert_cols(t_acc_f, n, [&](int c, const float* v) {
        if (!lane_used) {
          store_zero8(op_hi[f], op_lo[f], 128, l, c);
          store_zero8(op_hi[f], op_lo[f], 128, l, c + 8);
          return;
        }
        float l16[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          l16[j] = (1.f / 64.f) * recip_nr(fmaf(beta_f, ctl->mu[c + j] + mu_row, alpha));
          l16[j] = fmaf(l16[j], kap, l16[j]);
        }
        store_split8v(op_hi[f], op_lo[f], 128, l, c, v, l16);
        store_split8v(op_hi[f], op_lo[f], 128, l, c + 8, v + 8, l16 + 8);
      });
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->op_ready[f]);

    // ---- stage 3 -> MN-major operand of stage 4 (row k, columns p n + y)
    if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
    ++ph_done;
    tc_fence_after();
    {
      const float sc3 = 1.f + kap;
      convert_cols(t_acc_f, n, [&](int y, const float* v) {
        if (!lane_used) return;
        store_split8(op_hi[f], op_lo[f], n, row, p * n + y, v, sc3);
        store_split8(op_hi[f], op_lo[f], n, row, p * n + y + 8, v + 8, sc3);
      });
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->op_ready[f]);
  }
  if (valid) {
    atomicAdd(&ctl->phi[p], phi);
    if (bad) atomicOr(&ctl->bad[p], 1);
  }
  return true;
}

// The MMA-issuing warp: one step = stage 1 of both fields once the reaction
// pass is done, then stages 2-4 of each field as its operand is ready.
__device__ bool tc_issuer(const DevProblem& pb, TcCtrl* ctl, uint8_t* base, int nmax, int n,
                          uint32_t tmem, int lane, uint32_t& ph_rx, uint32_t (&ph_op)[2]) {
  volatile int* abort = &ctl->abort;
  const uint32_t d[2] = {tmem, tmem + (uint32_t)n};
  for (int step = 0; step < pb.n_steps; ++step) {
    if (!mbar_wait_bounded(&ctl->rx_ready, ph_rx & 1u, abort, pb.wait_ns)) return false;
    ++ph_rx;
    tc_fence_after();
    if (lane == 0) {
      for (int f = 0; f < 2; ++f) {
        issue_stage(base, nmax, n, 1, f, d[f]);
        mma_commit(&ctl->mma_done[f]);
      }
    }
    __syncwarp();
    if (step == pb.stall_step) {  // test aid: wait on a barrier nothing completes
      mbar_wait_bounded(&ctl->never, 0u, abort, pb.wait_ns);
      return false;
    }
    for (int stage = 2; stage <= 4; ++stage) {
      for (int f = 0; f < 2; ++f) {
        if (!mbar_wait_bounded(&ctl->op_ready[f], ph_op[f] & 1u, abort, pb.wait_ns)) return false;
        ++ph_op[f];
        tc_fence_after();
        if (lane == 0) {
          issue_stage(base, nmax, n, stage, f, d[f]);
          mma_commit(&ctl->mma_done[f]);
        }
        __syncwarp();
      }
    }
  }
  return true;
}

template <int NMAX>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_solve2d_tc(DevProblem pb, WorkQueue q, const double* theta, double* phi, uint32_t* status,
                 float* fields, size_t field_stride, int* err) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned start, derived from smem_raw so that the compiler keeps
  // the shared address space (plain shared loads and stores, not generic)
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  TcCtrl* ctl = reinterpret_cast<TcCtrl*>(base + tc_off_ctrl(NMAX));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kCols = tc_tmem_cols(NMAX);

  if (warp == 8) {
    tmem_alloc(&ctl->tmem_base, kCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&ctl->mma_done[0], 1);
    mbar_init(&ctl->mma_done[1], 1);
    mbar_init(&ctl->op_ready[0], 4);
    mbar_init(&ctl->op_ready[1], 4);
    mbar_init(&ctl->rx_ready, 8);
    mbar_init(&ctl->fin, 1);
    mbar_init(&ctl->never, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;

  uint32_t ph_done = 0, ph_rx = 0;
  uint32_t ph_op[2] = {0, 0};
  int cur_size = -1;
  for (;;) {
    if (tid == 0) {
      if (ctl->abort)
        ctl->n_items = 0;
      else
        tc_pop_group(pb, q, ctl);
      for (int j = 0; j < ctl->n_items; ++j) {
        full_theta(pb, theta + (size_t)ctl->items[j] * pb.n_params, ctl->th[j]);
        ctl->phi[j] = 0.0;
        ctl->bad[j] = 0;
      }
      for (int j = ctl->n_items; j < kTcMaxStack; ++j) {  // idle rows: pure diffusion
        ctl->th[j][0] = ctl->th[j][1] = ctl->th[j][3] = ctl->th[j][4] = 0.0;
        ctl->th[j][2] = 1.0;
      }
    }
    __syncthreads();
    if (ctl->n_items == 0) break;
    const int s = ctl->size;
    const DevSize& S = pb.sz[s];
    const int n = S.n;
    const int sp = 128 / n;
    if (s != cur_size) {  // DCT matrix tiles (8 C, split) and eigenvalues of this size
      uint8_t* chi = base + tc_off_c(NMAX, 0);
      uint8_t* clo = base + tc_off_c(NMAX, 1);
      for (int i = tid; i < n * n; i += kTcThreads) {
        const int rr = i / n, cc = i - rr * n;
        __half h, lo;
        split_f16(8.f * S.cmat[i], h, lo);
        const uint32_t off = sw128_offset(n, rr, cc);
        *reinterpret_cast<__half*>(chi + off) = h;
        *reinterpret_cast<__half*>(clo + off) = lo;
      }
      for (int i = tid; i < n; i += kTcThreads) ctl->mu[i] = S.mu[i];
      fence_proxy_async_smem();
      cur_size = s;
      __syncthreads();
    }
    // initial deviations (scaled by 128) and the tables L of fixed domains
    if (warp < 8) {
      const int f = warp >> 2;
      const int l = 32 * (warp & 3) + lane;
      const int p = l / n, row = l - p * n;
      const bool lane_used = p < sp;
      const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
      const float ref = f ? S.ref_v : S.ref_u;
      const float* w0 = f ? S.v0f : S.u0f;
      const double* th = ctl->th[lane_used ? p : 0];
      const float beta = (float)(pb.tau * (f ? th[2] : 1.0) * (double)n * n);
      const float mu_row = ctl->mu[row];
      for (int x = 0; x < n; x += 8) {
        float v8[8], l8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          v8[j] = lane_used ? (w0[(size_t)row * n + x + j] - ref) * 128.f : 0.f;
          l8[j] = (1.f / 64.f) / fmaf(beta, ctl->mu[x + j] + mu_row, 1.f);
          l8[j] = fmaf(l8[j], tc_rz_comp(n), l8[j]);
        }
        __syncwarp();
        tmem_st8(tmem + lane_off + (uint32_t)(f * n + x), v8);
        tmem_st8(tmem + lane_off + (uint32_t)(2 * n + f * n + x), l8);
      }
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp < 8) {
      tc_converter(pb, S, ctl, base, NMAX, n, tmem, warp >> 2, warp, lane, ph_done, fields,
                   field_stride);
    } else {
      tc_issuer(pb, ctl, base, NMAX, n, tmem, lane, ph_rx, ph_op);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!ctl->abort && tid < ctl->n_items) {
      const int b = ctl->items[tid];
      const bool bad = ctl->bad[tid] != 0;
      status[b] = bad ? (uint32_t)RD_P_NONFINITE : 0u;
      phi[b] = bad ? (double)INFINITY : ctl->phi[tid] * S.inv_two_sigma2;
    }
    __syncthreads();
  }
  // drain: every MMA this CTA issued must finish before its TMEM is freed
  if (warp == 8) {
    if (lane == 0) mma_commit(&ctl->fin);
    __syncwarp();
    volatile int never = 0;
    mbar_wait_bounded(&ctl->fin, 0, &never);
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
  if (tid == 0 && ctl->abort) atomicOr(err, 1);
}

// ---------------------------------------------------------------- host side
template <typename F>
static auto with_tc_kernel(int max_n, F&& f) {
  if (max_n <= 32) return f((const void*)k_solve2d_tc<32>, 32);
  if (max_n <= 64) return f((const void*)k_solve2d_tc<64>, 64);
  if (max_n <= 96) return f((const void*)k_solve2d_tc<96>, 96);
  return f((const void*)k_solve2d_tc<128>, 128);
}

cudaError_t setup_solve_tc(int max_n) {
  return with_tc_kernel(max_n, [&](const void* fn, int nmax) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes(nmax));
  });
}

int grid_solve_tc(int max_n, int n_sm) {
  return with_tc_kernel(max_n, [&](const void* fn, int nmax) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTcThreads,
                                                      tc_smem_bytes(nmax)) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const int by_tmem = (int)(512 / tc_tmem_cols(nmax));
    return n_sm * (per_sm < by_tmem ? per_sm : by_tmem);
  });
}

cudaError_t launch_solve_tc(const DevProblem& pb, const WorkQueue& q, const double* theta,
                            double* phi, uint32_t* status, void* fields, int grid, int* err,
                            cudaStream_t st) {
  const size_t stride = (size_t)2 * pb.max_n * pb.max_n;
  DevProblem pbv = pb;
  WorkQueue qv = q;
  const double* th = theta;
  void* fo = fields;
  size_t stride_v = stride;
  int* errv = err;
  return with_tc_kernel(pb.max_n, [&](const void* fn, int nmax) {
    void* args[] = {&pbv, &qv, (void*)&th, &phi, &status, &fo, &stride_v, &errv};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), args, tc_smem_bytes(nmax), st);
  });
}

size_t tc_smem_bytes_host(int max_n) {
  return with_tc_kernel(max_n, [&](const void*, int nmax) { return (size_t)tc_smem_bytes(nmax); });
}

}  // namespace rd
