// Primitives shared by the tensor-core kernels (sm_103a): K-major 128-byte-swizzled operand
// tiles, shared-memory and instruction descriptors for tcgen05.mma, bounded mbarrier waits,
// commits, and the TF32 split.
#pragma once

#include <cstdint>

#include "../../include/dftfe_gb300.h"

namespace dftfe {
namespace tc {

constexpr long kSpinLimit = 40000000L;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, byte) in a K-major 128-byte-swizzled tile (rows of 128 bytes,
// 8-row atoms of 1024 bytes, 16-byte chunks XOR-ed with the row index mod 8)
__host__ __device__ __forceinline__ uint32_t sw128(uint32_t row, uint32_t b) {
  return (row >> 3) * 1024u + (row & 7u) * 128u + ((((b >> 4) ^ (row & 7u)) & 7u) << 4) + (b & 15u);
}

// shared-memory matrix descriptor: start, LBO 16 B (unused for swizzled K-major),
// SBO 1024 B (between 8-row atoms), version 1, layout SWIZZLE_128B
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D = F32, A/B format (BF16 = 1 under kind::f16, TF32 = 2 under
// kind::tf32), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count));
}

// bounded wait on a phase parity; false on time-out (recorded in *err and *abort) or when
// another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* err,
                                          long limit = kSpinLimit) {
  const uint32_t addr = smem_u32(b);
  for (long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}"
                 : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  *abort = 1;
  atomicExch(err, (int)DFTFE_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(b)) : "memory");
}

// one cta_group::1 MMA, D (TMEM) (+)= A B^T with A, B from shared memory descriptors
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// the same rounding (to 10 explicit mantissa bits, nearest, ties away from zero) on the bit
// pattern with two integer operations: adding half of the dropped unit carries into the kept
// bits exactly when the dropped part is at least half (and into the exponent on overflow);
// identical to cvt.rna.tf32.f32 for every finite input
__device__ __forceinline__ uint32_t tf32_rn_bits(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

// FP32 value -> TF32 hi + TF32 lo by integer rounding (f - hi is exact in FP32)
__device__ __forceinline__ void split_tf32_bits(uint32_t u, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rn_bits(u);
  lo = tf32_rn_bits(__float_as_uint(__uint_as_float(u) - __uint_as_float(hi)));
}

// FP64 value -> TF32 hi + TF32 lo (each rounded to nearest, ties away)
__device__ __forceinline__ void split_tf32(double v, uint32_t& hi, uint32_t& lo) {
  const float f = __double2float_rn(v);
  hi = tf32_rn(f);
  lo = tf32_rn(__double2float_rn(v - (double)__uint_as_float(hi)));
}

// FP32 value -> TF32 hi + TF32 lo, FP32 arithmetic only (f - hi is exact)
__device__ __forceinline__ void split_tf32f(float f, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rn(f);
  lo = tf32_rn(f - __uint_as_float(hi));
}

// exact FP32 -> FP64 widening with integer operations only (the FP64 pipe of this part is
// narrow); FP32 subnormals, which the accumulators here never hold, become zero
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)s);
  const uint64_t bits = s | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// FP64 -> FP32 with integer operations only, rounding to nearest with ties away from zero;
// magnitudes below the FP32 normal range become (signed) zero.  Used where an FP64 operand
// only feeds a split product of FP32 accuracy, to keep the conversion off the FP64 pipe.
__device__ __forceinline__ float narrow_f64(double v) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e <= 896) return __uint_as_float(s);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);      // top 23 fraction bits
  const uint32_t f = (((uint32_t)(e - 896) << 23) | mant) + ((lo >> 28) & 1u);
  return __uint_as_float(s | f);
}

// 32 consecutive 32-bit TMEM columns of this warp's 32 lanes (lane = row)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace dftfe
