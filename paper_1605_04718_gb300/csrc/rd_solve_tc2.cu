// rd_solve_tc2.cu -- the 128^2 forward solve on the tensor cores with the
// DCT matrices resident in TMEM.
//
// Same step and number format as k_solve2d_tc (rd_solve_tc.cu): explicit
// reaction, implicit diffusion by the four eigenbasis transforms (Sec. 3.1.1
// with the diagonal solve in the DCT-II basis), split-FP16 operands with
// three products, FP32 accumulation, state held as deviation from the
// initial-state mean.  The difference is the orientation: the constant
// matrix 8C (and its transpose) is operand A, read from TMEM, and each
// field's data is operand B in shared memory, so an MMA reads 4 KB of
// operands from shared memory instead of 8 KB.  With i the index on TMEM
// lanes and j the one on columns:
//   stage 1  D[k][i] = sum_j C[k][j] R[i][j]        (B = R, K-major)
//   stage 2  D[l][k] = sum_i C[l][i] P[k][i]        (B = P, K-major)
//   scale    S[l][k] = D[l][k] L[l][k]
//   stage 3  D[i][k] = sum_l C^T[i][l] S[l][k]      (B = S, MN-major)
//   stage 4  D[j][i] = sum_k C^T[j][k] E[i][k]      (B = E, K-major)
// so one step maps a state with i on the lanes to one with j on the lanes:
// the state is W (y on the lanes) after an even number of steps and W^T
// after an odd number.  L is symmetric, so the same code serves both.
//
// Pipelining.  The fields u and v run interleaved: while the tensor core
// works on one field's stage, the other field's converter warps turn the
// previous result into the next operand.  (Splitting a stage into two N = 64
// halves, to start on half an operand, cost more than it overlapped: an
// N = 64 MMA takes about 56 cycles against 64 for N = 128.)
//
// The diagonal factor L = 1 / (alpha + beta (mu_l + mu_k)) (times 1/64 and
// the compensation below) is computed where it is applied: the reciprocal by
// the hardware approximation (within one ulp), on pairs of columns with the
// paired FP32 instructions.  On a fixed domain L is the same every step, so
// its rounding error compounds in the slow modes: a cheaper reciprocal (one
// approximation for two values through their product) moved Phi by more
// than the posterior allows.  The converter warps are bound by throughput
// (their instructions, TMEM loads and shared-memory stores beside the MMAs'
// operand reads: twice the warps did not convert faster), and the tensor
// core waits on them, so the hot loops save instructions: the hi/lo
// split works on pairs with the paired FP32 instructions and stores the lo
// part negated (one mixed FP16/FP32 subtraction per value; the MMAs that
// read it set the negate bit of B), the operand scale 256 of the reaction
// is applied through its constants, and stage 3's compensation is folded
// into L.
//
// Accumulation order.  The tensor core rounds each MMA's sum toward zero, a
// bias of about 0.72 * 2^-24 of the accumulator per MMA that compounds over
// the chain.  Each stage therefore issues the small correction products
// (hi*lo, lo*hi) first, while the accumulator is small, and the 8 main
// products (hi*hi) last; the remaining shrink of about 8 * 0.5 * 2^-24 (the
// partial sums average about 0.7 of the final value) is compensated by
// multiplying each stage's output by 1 + 2^-22.
//
// TMEM (512 columns): 8C hi | 8C lo | 8C^T hi | 8C^T lo (64 columns each,
// two FP16 per column) | field u accumulator | field v accumulator.
// One 128^2 proposal per CTA, 544 threads: warps 0-7 convert field u,
// 8-15 field v (two warps per TMEM lane quadrant), warp 16 allocates TMEM
// and issues the MMAs, one thread, in the order u1 v1 u2 v2 ... u4 v4 (two
// issuing threads let both fields' MMAs share the tensor core at once: they
// then finish together and convert together, with nothing to overlap).  As
// the MMAs complete in that order, a converter starts the reaction once it
// has seen the stage-4 commit of both fields.  Barrier arrivals are one per
// warp.  Shared memory: the four operand tiles (u hi, u lo, v hi, v lo;
// 32 KB each) and control.
// Bounded waits as in rd_solve_tc.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "rd_common.cuh"
#include "rd_internal.h"
#include "rd_tc_ptx.cuh"

namespace rd {

using namespace tc;

namespace tc2 {

constexpr int N = 128;
constexpr uint32_t kColCHi = 0, kColCLo = 64, kColCtHi = 128, kColCtLo = 192;
constexpr uint32_t kColAcc = 256;  // + 128 f
constexpr uint32_t kTileBytes = 128 * 128 * 2;  // one FP16 operand tile
constexpr uint32_t kOffCtrl = 4 * kTileBytes;  // after the tiles u hi, u lo, v hi, v lo
constexpr uint32_t kSmemBytes = 1024 + kOffCtrl + 4096;
// stage output scales with the round-toward-zero compensation 1 + 2^-22
constexpr float kScale1 = 0x1p-7f + 0x1p-29f;   // stage 1: (1/128)(1 + 2^-22)
// stage 2: L (1/64)(1 + 2^-22)^2, the compensation of stage 3 included
// (the transforms are linear), so that stage 3's output is split unscaled
constexpr float kScaleL = 0x1p-6f + 0x1p-27f;
constexpr float kScaleW = 0x1p-7f + 0x1p-29f;   // stage 4 (state read): (1/128)(1 + 2^-22)

struct Ctrl {
  uint64_t mma_done[2];   // per field: its stage's MMAs completed
  uint64_t op_all[2];     // per field: the whole next operand written
  uint64_t rx_ready;      // reaction written (both fields)
  uint64_t fin;
  uint64_t never;         // completed by nothing (failure-path test aid)
  double phi;
  uint32_t tmem_base;
  int abort;
  int item;
  int size;
  int bad;
  double th[kNPhys];
  alignas(16) float mu[N];
};

__device__ __forceinline__ uint8_t* tile(uint8_t* base, int f, int hl) {
  return base + (uint32_t)(2 * f + hl) * kTileBytes;
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// K-major stage (1, 2, 4) of field f: the correction products of all K
// blocks first, then the main products.
__device__ __forceinline__ void issue_kmajor(uint8_t* base, uint32_t tmem, int stage, int f) {
  constexpr uint32_t idesc = idesc_f16_f32(128, N, 0, 0);
  constexpr uint32_t idesc_nb = idesc_f16_f32(128, N, 0, 0, 1);  // B = the negated lo
  const uint32_t a_hi = tmem + (stage <= 2 ? kColCHi : kColCtHi);
  const uint32_t a_lo = tmem + (stage <= 2 ? kColCLo : kColCtLo);
  const uint64_t bh = sdesc_sw128(smem_u32(tile(base, f, 0)), 16u, 1024u);
  const uint64_t bl = sdesc_sw128(smem_u32(tile(base, f, 1)), 16u, 1024u);
  const uint32_t d = tmem + kColAcc + (uint32_t)(128 * f);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t off = ((uint32_t)(kk >> 2) * 16384u + (uint32_t)(kk & 3) * 32u) >> 4;
    mma_ts(d, a_hi + (uint32_t)(kk * 8), bl + off, idesc_nb, kk > 0 ? 1u : 0u);
    mma_ts(d, a_lo + (uint32_t)(kk * 8), bh + off, idesc, 1u);
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t off = ((uint32_t)(kk >> 2) * 16384u + (uint32_t)(kk & 3) * 32u) >> 4;
    mma_ts(d, a_hi + (uint32_t)(kk * 8), bh + off, idesc, 1u);
  }
}

// Stage 3 of field f: B = the MN-major operand tile (K rows = lanes of the
// conversion, two 64-column N blocks 16 KB apart), corrections first.
__device__ __forceinline__ void issue_stage3(uint8_t* base, uint32_t tmem, int f) {
  constexpr uint32_t idesc = idesc_f16_f32(128, N, 0, 1);
  constexpr uint32_t idesc_nb = idesc_f16_f32(128, N, 0, 1, 1);  // B = the negated lo
  const uint32_t a_hi = tmem + kColCtHi, a_lo = tmem + kColCtLo;
  const uint64_t bh = sdesc_sw128(smem_u32(tile(base, f, 0)), 16384u, 1024u);
  const uint64_t bl = sdesc_sw128(smem_u32(tile(base, f, 1)), 16384u, 1024u);
  const uint32_t d = tmem + kColAcc + (uint32_t)(128 * f);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t off = ((uint32_t)kk * 2048u) >> 4;
    mma_ts(d, a_hi + (uint32_t)(kk * 8), bl + off, idesc_nb, kk > 0 ? 1u : 0u);
    mma_ts(d, a_lo + (uint32_t)(kk * 8), bh + off, idesc, 1u);
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t off = ((uint32_t)kk * 2048u) >> 4;
    mma_ts(d, a_hi + (uint32_t)(kk * 8), bh + off, idesc, 1u);
  }
}

// Splits 8 values (times scale) of row r, columns c..c+7 into the hi and
// negated lo tiles: one 16-byte store each.
__device__ __forceinline__ void store8(uint8_t* hi, uint8_t* lo, int r, int c, const float* x,
                                       float scale) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split_f16x2_neglo_scaled(x[2 * j], x[2 * j + 1], scale, h[j], l[j]);
  const uint32_t off = sw128_offset(128, r, c);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// As store8 without a scale.
__device__ __forceinline__ void store8n(uint8_t* hi, uint8_t* lo, int r, int c, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) split_f16x2_neglo(x[2 * j], x[2 * j + 1], h[j], l[j]);
  const uint32_t off = sw128_offset(128, r, c);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// As store8 with one scale per value.
__device__ __forceinline__ void store8s(uint8_t* hi, uint8_t* lo, int r, int c, const float* x,
                                        const float* s8) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    split_f16x2_neglo_scaled2(x[2 * j], x[2 * j + 1], s8[2 * j], s8[2 * j + 1], h[j], l[j]);
  const uint32_t off = sw128_offset(128, r, c);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Explicit reaction in place on 8 points: state (x 128) ->
// r_u = du + tau gamma (a - u + u^2 v) (+ cu), r_v = dv + tau gamma (b - u^2 v)
// (+ cv), as deviations from the reference state, times 256 (the operand
// scale, applied through the constants: exact).
__device__ __forceinline__ void react8(float* u, float* v, float sw, float ref_u, float ref_v,
                                       float fa, float fb, float ftg, float cu, float cv) {
  const float sw8 = 256.f * sw, ftg8 = 256.f * ftg, cu8 = 256.f * cu, cv8 = 256.f * cv;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float uu = fmaf(u[j], sw, ref_u), vv = fmaf(v[j], sw, ref_v);
    const float u2v = uu * uu * vv;
    u[j] = fmaf(ftg8, fa - uu + u2v, fmaf(u[j], sw8, cu8));
    v[j] = fmaf(ftg8, fb - u2v, fmaf(v[j], sw8, cv8));
  }
}

struct ObsCtx {
  const float* yo;  // this observation's data, or null
  float* fo;        // this proposal's output fields, or null
  bool odd;         // state transposed (x on the lanes)
};

// Observation misfit and final-field output of 8 points of row l, columns c..c+7.
__device__ __forceinline__ void observe8(const DevProblem& pb, const DevSize& S, const ObsCtx& o,
                                         int l, int c, const float* u, const float* v, float sw,
                                         double& phi, int& bad) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const size_t pt = o.odd ? (size_t)(c + j) * N + l : (size_t)l * N + c + j;  // y N + x
    const float du = u[j] * sw, dv = v[j] * sw;
    if (o.yo) {
      int k = 0;
      if (S.field_mask & 1) {
        const double w = (double)S.ref_u + (double)du;
        if (!(fabs(w) <= pb.w_max)) bad = 1;
        const double e = (double)o.yo[pt] - w;
        phi += e * e;
        ++k;
      }
      if (S.field_mask & 2) {
        const double w = (double)S.ref_v + (double)dv;
        if (!(fabs(w) <= pb.w_max)) bad = 1;
        const double e = (double)o.yo[(size_t)k * S.npts + pt] - w;
        phi += e * e;
      }
    }
    if (o.fo) {
      o.fo[pt] = S.ref_u + du;
      o.fo[(size_t)S.npts + pt] = S.ref_v + dv;
    }
  }
}

// One converter warp w (0 .. 8 WPF - 1), WPF warps per TMEM lane quadrant
// and field.  Stage conversions: field f = w / (4 WPF), columns
// [cw r, cw (r + 1)) of each half, cw = 64 / WPF, r = (w / 4) % WPF.
// Reaction: both fields at columns [xw p, xw (p + 1)) of each half,
// xw = 32 / WPF, p = w / 4.
template <int WPF>
__device__ bool converter(const DevProblem& pb, const DevSize& S, Ctrl* ctl, uint8_t* base,
                          uint32_t tmem, int warp, int lane, uint32_t& ph_done,
                          float* fields, size_t field_stride) {
  constexpr int CW = 64 / WPF;  // stage-conversion columns per half
  constexpr int XW = 32 / WPF;  // reaction columns per half
  volatile int* abort = &ctl->abort;
  const int f = warp / (4 * WPF);
  const int q = warp & 3;
  const int rr = (warp >> 2) % WPF;
  const int p = warp >> 2;
  const int l = 32 * q + lane;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t t_u = tmem + lane_off + kColAcc, t_v = t_u + 128u;
  const uint32_t t_f = f ? t_v : t_u;
  uint8_t* const hi_u = tile(base, 0, 0);
  uint8_t* const lo_u = tile(base, 0, 1);
  uint8_t* const hi_v = tile(base, 1, 0);
  uint8_t* const lo_v = tile(base, 1, 1);
  uint8_t* const hi_f = f ? hi_v : hi_u;
  uint8_t* const lo_f = f ? lo_v : lo_u;
  const double* th = ctl->th;
  const double tau = pb.tau;
  const float fa = (float)th[0], fb = (float)th[1], ftg = (float)(tau * th[3]);
  const double r = th[4];
  const float beta_fixed = (float)(tau * (f ? th[2] : 1.0) * (double)N * N);
  const float ref_u = S.ref_u, ref_v = S.ref_v;
  const int nfo = (S.field_mask & 1) + ((S.field_mask >> 1) & 1);
  const float mu_l = ctl->mu[l];
  double phi = 0.0;
  int bad = 0;
  int next_obs = 0;
  for (int step = 0;; ++step) {
    if (step > 0) {  // stage 4 of both fields done: the fourth commit of a step
      // completes an odd phase, and the other field's stage-4 phase is the one
      // pending or just completed (the MMAs complete in issue order)
      if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
      ++ph_done;
      if (!mbar_wait_bounded(&ctl->mma_done[f ^ 1], 1u, abort, pb.wait_ns)) return false;
      tc_fence_after();
    }
    const bool last = step == pb.n_steps;
    const float sw = step > 0 ? kScaleW : 0x1p-7f;
    const bool obs = next_obs < S.n_obs && step == S.obs_steps[next_obs];
    ObsCtx o;
    o.yo = obs ? S.yf + (size_t)next_obs * nfo * S.npts : nullptr;
    o.fo = (last && fields) ? fields + (size_t)ctl->item * field_stride : nullptr;
    o.odd = step & 1;
    if (obs) ++next_obs;
    float alpha = 1.f, cu = 0.f, cv = 0.f;
    float beta_f = beta_fixed;
    if (pb.growth) {  // FP64, rounded once per step
      const double rho2inv = exp(-2.0 * r * (double)step * tau);
      alpha = (float)(1.0 + tau * 2.0 * r);
      cu = (float)(-tau * 2.0 * r * (double)ref_u);
      cv = (float)(-tau * 2.0 * r * (double)ref_v);
      beta_f = (float)(tau * (f ? th[2] : 1.0) * rho2inv * (double)N * N);
    }
    // ---- observation / output, then the reaction -> stage-1 operands
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int x0 = 64 * half + XW * p;
      float uh[XW], vh[XW];  // all loads of the half in flight at once
      __syncwarp();
#pragma unroll
      for (int j = 0; j < XW; j += 8) {
        tmem_ld8(t_u + (uint32_t)(x0 + j), *reinterpret_cast<float(*)[8]>(uh + j));
        tmem_ld8(t_v + (uint32_t)(x0 + j), *reinterpret_cast<float(*)[8]>(vh + j));
      }
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < XW; j += 8) {
        if (o.yo || o.fo) observe8(pb, S, o, l, x0 + j, uh + j, vh + j, sw, phi, bad);
        if (last) continue;
        react8(uh + j, vh + j, sw, ref_u, ref_v, fa, fb, ftg, cu, cv);
        store8n(hi_u, lo_u, l, x0 + j, uh + j);
        store8n(hi_v, lo_v, l, x0 + j, vh + j);
      }
    }
    if (last) break;
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->rx_ready);

    // ---- stages 1-3 of field f -> operands of stages 2-4
#pragma unroll 1
    for (int stage = 1; stage <= 3; ++stage) {
      if (!mbar_wait_bounded(&ctl->mma_done[f], ph_done & 1u, abort, pb.wait_ns)) return false;
      ++ph_done;
      tc_fence_after();

      // this warp's 64 columns in 4 chunks of 16, the next chunk's TMEM load in
      // flight while the current one is converted
      constexpr int NQ = CW / 8;  // chunks of 16 columns, both halves
      int cols[NQ];
#pragma unroll
      for (int qq = 0; qq < NQ; ++qq)
        cols[qq] = 64 * (qq / (NQ / 2)) + CW * rr + 16 * (qq % (NQ / 2));
      float buf[2][16];
      __syncwarp();
      tmem_ld16(t_f + (uint32_t)cols[0], buf[0]);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float* a = buf[q & 1];
        if (q < NQ - 1) tmem_ld16(t_f + (uint32_t)cols[q + 1], buf[(q + 1) & 1]);
        const int c0 = cols[q];
        if (stage == 2) {  // S = D L, L from mu_l + mu_k two columns at a time
          const uint64_t ml2 = f2_pack(mu_l, mu_l), be2 = f2_pack(beta_f, beta_f);
          const uint64_t al2 = f2_pack(alpha, alpha), ks2 = f2_pack(kScaleL, kScaleL);
#pragma unroll
          for (int k = 0; k < 16; k += 8) {
            float lam8[8];
#pragma unroll
            for (int jj = 0; jj < 8; jj += 2) {
              const float2 mc = *reinterpret_cast<const float2*>(&ctl->mu[c0 + k + jj]);
              const uint64_t x2 = f2_fma(f2_add(ml2, f2_pack(mc.x, mc.y)), be2, al2);
              f2_unpack(f2_mul(f2_recip(x2), ks2), lam8[jj], lam8[jj + 1]);
            }
            store8s(hi_f, lo_f, l, c0 + k, a + k, lam8);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 16; k += 8) {
            if (stage == 1)
              store8(hi_f, lo_f, l, c0 + k, a + k, kScale1);
            else
              store8n(hi_f, lo_f, l, c0 + k, a + k);
          }
        }
        if (q < NQ - 1) tmem_wait_ld();
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->op_all[f]);
    }
  }
  atomicAdd(&ctl->phi, phi);
  if (bad) atomicOr(&ctl->bad, 1);
  return true;
}

__device__ bool issuer(const DevProblem& pb, Ctrl* ctl, uint8_t* base, uint32_t tmem, int lane,
                       uint32_t& ph_rx, uint32_t (&ph_all)[2]) {
  volatile int* abort = &ctl->abort;
  for (int step = 0; step < pb.n_steps; ++step) {
    if (!mbar_wait_bounded(&ctl->rx_ready, ph_rx & 1u, abort, pb.wait_ns)) return false;
    ++ph_rx;
    tc_fence_after();
    if (lane == 0) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        issue_kmajor(base, tmem, 1, f);
        mma_commit(&ctl->mma_done[f]);
      }
    }
    __syncwarp();
    if (step == pb.stall_step) {  // test aid: wait on a barrier nothing completes
      mbar_wait_bounded(&ctl->never, 0u, abort, pb.wait_ns);
      return false;
    }
#pragma unroll 1
    for (int stage = 2; stage <= 4; ++stage) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        if (!mbar_wait_bounded(&ctl->op_all[f], ph_all[f] & 1u, abort, pb.wait_ns)) return false;
        ++ph_all[f];
        tc_fence_after();
        if (lane == 0) {
          if (stage == 3)
            issue_stage3(base, tmem, f);
          else
            issue_kmajor(base, tmem, stage, f);
          mma_commit(&ctl->mma_done[f]);
        }
        __syncwarp();
      }
    }
  }
  return true;
}

}  // namespace tc2

template <int WPF>
__global__ void __launch_bounds__(32 * (8 * WPF + 1), 1)
    k_solve2d_tc128(DevProblem pb, WorkQueue q, const double* theta, double* phi,
                    uint32_t* status, float* fields, size_t field_stride, int* err) {
  using namespace tc2;
  constexpr int kConvWarps = 8 * WPF;
  constexpr int kThreads = 32 * (kConvWarps + 1);
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned start, derived from smem_raw so that the compiler keeps
  // the shared address space (plain shared loads and stores, not generic)
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  Ctrl* ctl = reinterpret_cast<Ctrl*>(base + kOffCtrl);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == kConvWarps) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int f = 0; f < 2; ++f) {
      mbar_init(&ctl->mma_done[f], 1);
      mbar_init(&ctl->op_all[f], kConvWarps / 2);
    }
    mbar_init(&ctl->rx_ready, kConvWarps);
    mbar_init(&ctl->fin, 1);
    mbar_init(&ctl->never, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  // every size in this kernel's queue is 128^2: one DCT matrix serves all
  const DevSize& S0 = pb.sz[q.order[0]];
  // 8C and 8C^T as split FP16 into TMEM (lane = output index), once per CTA:
  // the first half of the converter warps C, the second C^T
  if (warp < kConvWarps) {
    const bool tr = warp >= 4 * WPF;
    const int m = 32 * (warp & 3) + lane;
    const int cbase = (64 / WPF) * ((warp >> 2) % WPF);
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    for (int c0 = cbase; c0 < cbase + 64 / WPF; c0 += 8) {
      float vh[8], vl[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k0 = 2 * (c0 + j), k1 = k0 + 1;
        const float e0 = 8.f * (tr ? S0.cmat[(size_t)k0 * N + m] : S0.cmat[(size_t)m * N + k0]);
        const float e1 = 8.f * (tr ? S0.cmat[(size_t)k1 * N + m] : S0.cmat[(size_t)m * N + k1]);
        __half h0, l0, h1, l1;
        split_f16(e0, h0, l0);
        split_f16(e1, h1, l1);
        vh[j] = __uint_as_float((uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16));
        vl[j] = __uint_as_float((uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16));
      }
      __syncwarp();
      tmem_st8(tmem + lane_off + (tr ? kColCtHi : kColCHi) + (uint32_t)c0, vh);
      tmem_st8(tmem + lane_off + (tr ? kColCtLo : kColCLo) + (uint32_t)c0, vl);
    }
    tmem_wait_st();
  }
  for (int i = tid; i < N; i += kThreads) ctl->mu[i] = S0.mu[i];
  uint32_t ph_done = 0, ph_rx = 0;
  uint32_t ph_all[2] = {0, 0};
  for (;;) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      int sz = 0;
      ctl->item = ctl->abort ? -1 : queue_pop(q, &sz);
      ctl->size = sz;
      if (ctl->item >= 0) full_theta(pb, theta + (size_t)ctl->item * pb.n_params, ctl->th);
      ctl->phi = 0.0;
      ctl->bad = 0;
    }
    __syncthreads();
    if (ctl->item < 0) break;
    const DevSize& S = pb.sz[ctl->size];
    if (warp < kConvWarps) {  // initial deviations (x 128), y on the lanes
      const int l = 32 * (warp & 3) + lane;
      const int p = warp >> 2;
      const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
      for (int f = 0; f < 2; ++f) {
        const float ref = f ? S.ref_v : S.ref_u;
        const float* w0 = f ? S.v0f : S.u0f;
        for (int x = (32 / WPF) * p; x < N; x += 64) {
#pragma unroll
          for (int x8 = 0; x8 < 32 / WPF; x8 += 8) {
            float v8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v8[j] = (w0[(size_t)l * N + x + x8 + j] - ref) * 128.f;
            __syncwarp();
            tmem_st8(tmem + lane_off + kColAcc + (uint32_t)(128 * f + x + x8), v8);
          }
        }
      }
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp < kConvWarps)
      converter<WPF>(pb, S, ctl, base, tmem, warp, lane, ph_done, fields, field_stride);
    else
      issuer(pb, ctl, base, tmem, lane, ph_rx, ph_all);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && !ctl->abort) {
      const int b = ctl->item;
      status[b] = ctl->bad ? (uint32_t)RD_P_NONFINITE : 0u;
      phi[b] = ctl->bad ? (double)INFINITY : ctl->phi * S.inv_two_sigma2;
    }
  }
  if (warp == kConvWarps) {
    if (lane == 0) mma_commit(&ctl->fin);
    __syncwarp();
    volatile int never = 0;
    mbar_wait_bounded(&ctl->fin, 0, &never);
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (tid == 0 && ctl->abort) atomicOr(err, 1);
}

bool tc128_applicable(const DevProblem& pb, int size_idx) {
  return pb.dim == 2 && pb.sz[size_idx].n == 128;
}

// Converter warps per TMEM lane quadrant and field.
constexpr int kTc128Wpf = 2;

cudaError_t setup_solve_tc128() {
  return cudaFuncSetAttribute(k_solve2d_tc128<kTc128Wpf>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc2::kSmemBytes);
}

int grid_solve_tc128(int n_sm) { return n_sm; }

cudaError_t launch_solve_tc128(const DevProblem& pb, const WorkQueue& q, const double* theta,
                               double* phi, uint32_t* status, void* fields, int grid, int* err,
                               cudaStream_t st) {
  const size_t stride = (size_t)2 * pb.max_n * pb.max_n;
  k_solve2d_tc128<kTc128Wpf><<<grid, 32 * (8 * kTc128Wpf + 1), tc2::kSmemBytes, st>>>(
      pb, q, theta, phi, status, (float*)fields, stride, err);
  return cudaGetLastError();
}

}  // namespace rd
