// rd_tc_ptx.cuh -- inline-PTX wrappers for the tensor-core solve: mbarriers,
// tcgen05 (TMEM allocation, MMA, commit, TMEM loads/stores, fences) and the
// shared-memory / instruction descriptors of tcgen05.mma kind::f16.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace rd {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Waits for the phase with the given parity, suspending the thread (instead
// of spinning) for up to the hinted time; returns whether it completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Default limit of a bounded wait: 4 s of wall time.
constexpr uint64_t kWaitLimitNs = 4000000000ull;

// Bounded wait for the phase with the given parity.  Gives up (returns false)
// when *abort is set by another thread, or after limit_ns of wall time (or
// 2^30 polls), in which case it sets *abort itself so that every other waiter
// leaves too.  A healthy wait in these kernels lasts microseconds.  Every
// lane of a warp polls with the same instruction, so a warp leaves as one.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if ((it & 15u) == 15u &&
        (globaltimer_ns() - t0 > limit_ns || it > (1u << 30))) {
      *abort = 1;
      return false;
    }
  }
}

// ---------------------------------------------------------------- fences
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- TMEM
// Allocation by one whole warp; the TMEM address is written to *dst (smem).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 32 lanes x 32-bit, 8 consecutive columns: register j of lane i holds
// TMEM[lane base + i][column + j].
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 lanes x 32-bit, 32 consecutive columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 lanes x 32-bit, 16 consecutive columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- MMA
// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives once on the mbarrier when every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, A negated
// (bit 13) if neg_a, B negated (bit 14) if neg_b, A/B K-major (0) or
// MN-major (1), N >> 3 at bits 17..22, M >> 4 at bits 24..28.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N, int a_mn, int b_mn,
                                                     int neg_b = 0, int neg_a = 0) {
  return (1u << 4) | ((uint32_t)neg_a << 13) | ((uint32_t)neg_b << 14) |
         ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, 128-byte swizzle: start address, leading
// and stride byte offsets (16-byte units), version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Byte offset of element (r, c) of a 16-bit tile stored in 128-byte-swizzled
// column blocks of 64 elements: block c / 64 at c / 64 * rows * 128, row r at
// r * 128 within it, 16-byte chunk (c % 64) / 8 stored at position
// chunk ^ (r % 8).  Tiles start on 1024-byte boundaries.
__device__ __forceinline__ uint32_t sw128_offset(int rows, int r, int c) {
  return (uint32_t)((c >> 6) * rows * 128 + r * 128 + ((((c & 63) >> 3) ^ (r & 7)) << 4) +
                    ((c & 7) << 1));
}

// hi = fp16(x), lo = fp16(x - hi): x = hi + lo to about 22 significant bits
// while |x| stays inside the FP16 normal range.
__device__ __forceinline__ void split_f16(float x, __half& hi, __half& lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}

// 1/x to within about one ulp for normal x of moderate size (here
// 1 <= x < 2^20): the hardware reciprocal approximation refined by one
// Newton-Raphson step for f(r) = 1/r - x, r' = r + r (1 - x r).
__device__ __forceinline__ float recip_nr(float x) {
  const float r = __fdividef(1.f, x);
  return fmaf(r, fmaf(-x, r, 1.f), r);
}

// split_f16 of two values at once: .x holds a, .y holds b (a at the lower
// address when stored).
__device__ __forceinline__ void split_f16x2(float a, float b, __half2& hi, __half2& lo) {
  hi = __floats2half2_rn(a, b);
  const float2 h = __half22float2(hi);
  lo = __floats2half2_rn(a - h.x, b - h.y);
}

// ---------------------------------------------------------------- packed FP32
// Two FP32 values in one 64-bit register (first value in the low half),
// operated on by the paired FP32 instructions (add/sub/mul/fma .f32x2), each
// element rounded to nearest as by the scalar instruction.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// a * b + c, one rounding per element
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// 1/x of both elements: the hardware approximation (rcp.approx, at most one
// ulp from the exact reciprocal).
__device__ __forceinline__ uint64_t f2_recip(uint64_t x) {
  float x0, x1, r0, r1;
  f2_unpack(x, x0, x1);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(x1));
  return f2_pack(r0, r1);
}

// 1/x of both elements: the hardware approximation refined by one
// Newton-Raphson step r' = r + r (1 - x r), as recip_nr.
__device__ __forceinline__ uint64_t f2_recip_nr(uint64_t x) {
  float x0, x1, r0, r1;
  f2_unpack(x, x0, x1);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(x1));
  const uint64_t r = f2_pack(r0, r1);
  const uint64_t e = f2_fma(f2_sub(0ull, x), r, f2_pack(1.f, 1.f));
  return f2_fma(r, e, r);
}

// hi = {fp16(a sa), fp16(b sb)} and lo = the rounded remainders
// {fp16(a sa - hi_a), fp16(b sb - hi_b)}, each as one 32-bit word with the
// first value in the low half: split_f16 of the two scaled values, with the
// FP32 arithmetic done on the pair at once.
__device__ __forceinline__ void split_f16x2_scaled2(float a, float b, float sa, float sb,
                                                    uint32_t& hi, uint32_t& lo) {
  asm("{\n\t.reg .b64 x, y, r;\n\t.reg .f32 x0, x1, y0, y1, r0, r1;\n\t"
      ".reg .b16 h0, h1;\n\t"
      "mov.b64 x, {%2, %3};\n\t"
      "mov.b64 y, {%4, %5};\n\t"
      "mul.rn.f32x2 x, x, y;\n\t"
      "mov.b64 {x0, x1}, x;\n\t"
      "cvt.rn.f16x2.f32 %0, x1, x0;\n\t"
      "mov.b32 {h0, h1}, %0;\n\t"
      "cvt.f32.f16 y0, h0;\n\t"
      "cvt.f32.f16 y1, h1;\n\t"
      "mov.b64 y, {y0, y1};\n\t"
      "sub.rn.f32x2 r, x, y;\n\t"
      "mov.b64 {r0, r1}, r;\n\t"
      "cvt.rn.f16x2.f32 %1, r1, r0;\n\t}"
      : "=r"(hi), "=r"(lo)
      : "f"(a), "f"(b), "f"(sa), "f"(sb));
}
// As split_f16x2_scaled2, but nlo holds the negated remainders
// {fp16(hi_a - a sa), fp16(hi_b - b sb)}: each remainder is one
// mixed-precision subtraction (FP16 minus FP32, rounded to FP32; exact here)
// instead of a conversion back to FP32 and a subtraction.  Rounding to
// nearest is symmetric, so nlo is exactly the negated lo of
// split_f16x2_scaled2; an MMA that reads it sets its negate bit.
__device__ __forceinline__ void split_f16x2_neglo_scaled2(float a, float b, float sa, float sb,
                                                          uint32_t& hi, uint32_t& nlo) {
  asm("{\n\t.reg .b64 x, s;\n\t.reg .f32 x0, x1, r0, r1;\n\t"
      ".reg .b16 h0, h1;\n\t"
      "mov.b64 x, {%2, %3};\n\t"
      "mov.b64 s, {%4, %5};\n\t"
      "mul.rn.f32x2 x, x, s;\n\t"
      "mov.b64 {x0, x1}, x;\n\t"
      "cvt.rn.f16x2.f32 %0, x1, x0;\n\t"
      "mov.b32 {h0, h1}, %0;\n\t"
      "sub.rn.f32.f16 r0, h0, x0;\n\t"
      "sub.rn.f32.f16 r1, h1, x1;\n\t"
      "cvt.rn.f16x2.f32 %1, r1, r0;\n\t}"
      : "=r"(hi), "=r"(nlo)
      : "f"(a), "f"(b), "f"(sa), "f"(sb));
}
// split_f16x2_neglo_scaled2 of unscaled values: hi = {fp16(a), fp16(b)},
// nlo = {fp16(hi_a - a), fp16(hi_b - b)}.
__device__ __forceinline__ void split_f16x2_neglo(float a, float b, uint32_t& hi, uint32_t& nlo) {
  asm("{\n\t.reg .f32 r0, r1;\n\t.reg .b16 h0, h1;\n\t"
      "cvt.rn.f16x2.f32 %0, %3, %2;\n\t"
      "mov.b32 {h0, h1}, %0;\n\t"
      "sub.rn.f32.f16 r0, h0, %2;\n\t"
      "sub.rn.f32.f16 r1, h1, %3;\n\t"
      "cvt.rn.f16x2.f32 %1, r1, r0;\n\t}"
      : "=r"(hi), "=r"(nlo)
      : "f"(a), "f"(b));
}
__device__ __forceinline__ void split_f16x2_neglo_scaled(float a, float b, float s, uint32_t& hi,
                                                         uint32_t& nlo) {
  split_f16x2_neglo_scaled2(a, b, s, s, hi, nlo);
}
__device__ __forceinline__ void split_f16x2_scaled(float a, float b, float s, uint32_t& hi,
                                                   uint32_t& lo) {
  split_f16x2_scaled2(a, b, s, s, hi, lo);
}

}  // namespace tc
}  // namespace rd
