// Blackwell tensor-core (tcgen05), tensor-memory, bulk-copy and mbarrier
// primitives as inline PTX, and the exact integer arithmetic that runs the
// BConv matrix product (Eq. 2; Sec. 4.2 treats BConv as a matrix product)
// on the fp16 tensor pipe.
//
// Exactness. A centered residue y (|y| < 2^30) is written as four balanced
// signed bytes, y = sum_a d_a 2^(8a) with d_a in [-128, 128); the byte
// weights are folded into the matrix, m'_(k,a) = [m_k 2^(8a)]_p centered, and
// each m' is split the same way into four bytes e_(k,a,b) ("planes" b). Every
// byte is an exact fp16 value and every product d e (|d e| <= 2^14) an exact
// fp32 value, and plane b's sum over the K sources and 4 digits,
// P_b = sum_(k,a) d_(k,a) e_(k,a,b), stays below 2^22 in magnitude for
// K <= 63, so the fp32 accumulation is exact in any order. Then
// S = sum_b P_b 2^(8b) = sum_k y_k m_k + (multiple of p), |S| < 2^46, and one
// signed Montgomery reduction (Alg. 2) gives the same residue as the
// CUDA-core lazy sum.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "arith.cuh"

namespace ckks {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05), no swizzling: the operand is a
// grid of core matrices of 8 rows x 16 bytes (128 contiguous bytes each);
// lbo = byte distance between core matrices adjacent along K, sbo = between
// core matrices adjacent along M (or N). Bits 46-48 hold the fixed value 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= 1ull << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: A and B fp16, D fp32,
// both operands K-major, M x N tile (M = 128: N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A * B^T, issued by one thread; completion is tracked with
// commit().
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The mbarrier at mbar receives one arrival when every tcgen05.mma issued so
// far by this thread has completed.
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Tensor-memory allocation: executed by one whole warp; the base address is
// written to shared memory at slot. ncols is a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane (the warp reads the
// 32 lanes of its quadrant, warp id mod 4); taddr carries the quadrant's
// first lane in its upper half.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Generic-proxy shared-memory writes become visible to the async proxy
// (tensor core, bulk copies).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Non-blocking test / potentially blocking try of the phase with the given
// parity.
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true once the phase completed, false after `limit` SM clock
// cycles without completion. Limits below 1024 cycles poll with the
// non-blocking test only (a blocking try may sleep past such a limit), so a
// limit of a few cycles expires whenever the phase is still pending at the
// call; longer limits let the hardware suspend the waiting warp.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  if (mbar_test(mbar, parity)) return true;
  const long long t0 = clock64();
  if (limit < 1024) {
    while (clock64() - t0 <= limit)
      if (mbar_test(mbar, parity)) return true;
    return false;
  }
  while (clock64() - t0 <= limit)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

// One arrival that also expects `bytes` of transaction (bulk-copy) data.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bulk copy global -> shared of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) that completes on mbar's transaction count. The source is
// this GPU's own memory; the destination is this CTA's shared memory.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Status word bits written by bounded waits that expired (read back by the
// host as CKKS_ETIMEOUT).
constexpr uint32_t kStatusTimeout = 1u;
// Set by the range checks of the checked launch mode (a residue >= its prime).
constexpr uint32_t kStatusRange = 2u;

__device__ __forceinline__ void report_timeout(uint32_t* status) {
  if (status) atomicOr(status, kStatusTimeout);
}

// Four balanced signed-byte digits of a centered residue (|y| < 2^30) as two
// fp16 pairs, in order d0 d1 | d2 d3: with z = y + 0x808080 the low three
// bytes of z are d_a + 128 (a < 3) and z >> 24 = d3 in [-64, 64]. Each byte u
// becomes the fp16 1024 + u by placing 0x64 above it; subtracting 1152 then
// leaves u - 128 exactly.
__device__ __forceinline__ uint2 digits_f16(int32_t y) {
  const uint32_t z = (uint32_t)(y + 0x808080);
  uint32_t lo = __byte_perm(z, 0x64646464u, 0x4140);
  uint32_t hi = __byte_perm(z, 0x64646464u, 0x4342) ^ 0x00800000u;
  const __half2 off = __halves2half2(__ushort_as_half((unsigned short)0x6480), __ushort_as_half((unsigned short)0x6480));
  __half2 a = __hsub2(*reinterpret_cast<__half2*>(&lo), off);
  __half2 b = __hsub2(*reinterpret_cast<__half2*>(&hi), off);
  return make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
}

// Residue in [0, p) of an output from its four plane sums (fp32 bit patterns
// of exact integers with |v| < 2^22): adding 1.5 2^23 puts v + 0x4B400000 in
// the float's bit pattern; S = sum_b v_b 2^(8b) is assembled from two 32-bit
// halves t0 = v0 + 2^8 v1, t1 = v2 + 2^8 v3 (each fits int32), then
// S 2^-32 mod p by SMR (the matrix carries the 2^32).
__device__ __forceinline__ uint32_t planes_residue(uint32_t f0, uint32_t f1, uint32_t f2, uint32_t f3, uint32_t p,
                                                   uint32_t m) {
  const float kMagic = 12582912.0f;
  const uint32_t b0 = __float_as_uint(__fadd_rn(__uint_as_float(f0), kMagic));
  const uint32_t b1 = __float_as_uint(__fadd_rn(__uint_as_float(f1), kMagic));
  const uint32_t b2 = __float_as_uint(__fadd_rn(__uint_as_float(f2), kMagic));
  const uint32_t b3 = __float_as_uint(__fadd_rn(__uint_as_float(f3), kMagic));
  constexpr uint32_t kBias = 0x4B400000u * 257u;  // (1 + 2^8) times the magic's pattern, mod 2^32
  const int32_t t0 = (int32_t)(b0 + (b1 << 8) - kBias);
  const int32_t t1 = (int32_t)(b2 + (b3 << 8) - kBias);
  const int64_t S = (int64_t)t0 + ((int64_t)t1 << 16);
  return fix_signed(smr(S, p, m), p);
}

}  // namespace tc
}  // namespace ckks
