// The modular multiplication methods compared in Table 3 (Sec. 4.1), run on
// this GPU: every thread advances eight independent chains a <- a * b mod q
// for `rounds` steps with one reduction method, so the kernel time measures
// the method's throughput. Each step returns a value in [0, q), so all
// methods compute a * b^rounds mod q exactly and must agree bit for bit.
#include <vector>

#include "internal.h"

namespace ckks {
namespace {

struct MulConsts {
  uint32_t q, b;
  uint64_t mu;        // Barrett: floor(2^64 / q)
  uint32_t qinv_neg;  // Montgomery: -q^-1 mod 2^32
  uint32_t b_mont;    // b 2^32 mod q (Montgomery and signed-Montgomery operand)
  uint32_t b_sh;      // Shoup companion floor(b 2^32 / q)
  uint32_t m;         // signed Montgomery: q^-1 mod 2^32
};

// Barrett (64-bit): z = a b, estimated quotient floor(z mu / 2^64) is at most
// one below floor(z / q) because z < 2^62, so z - qhat q is in [0, 2q).
__device__ __forceinline__ uint32_t mm_barrett(uint32_t a, const MulConsts& c) {
  const uint64_t z = (uint64_t)a * c.b;
  const uint64_t qh = __umul64hi(z, c.mu);
  return csub((uint32_t)(z - qh * c.q), c.q);
}

// Montgomery (unsigned, Montgomery 1985): t = (z + (z q' mod 2^32) q) / 2^32
// with b in Montgomery form; t is in [0, 2q).
__device__ __forceinline__ uint32_t mm_montgomery(uint32_t a, const MulConsts& c) {
  const uint64_t z = (uint64_t)a * c.b_mont;
  const uint32_t mq = (uint32_t)z * c.qinv_neg;
  return csub((uint32_t)((z + (uint64_t)mq * c.q) >> 32), c.q);
}

__device__ __forceinline__ uint32_t mm_shoup(uint32_t a, const MulConsts& c) {
  return csub(shoup(a, c.b, c.b_sh, c.q), c.q);
}

// Signed Montgomery reduction (Alg. 2) of a b~, result in (-q, q), then [0, q).
__device__ __forceinline__ uint32_t mm_smr(uint32_t a, const MulConsts& c) {
  return fix_signed(mont_mul(a, c.b_mont, c.q, c.m), c.q);
}

template <int M>
__device__ __forceinline__ uint32_t mm(uint32_t a, const MulConsts& c) {
  if (M == CKKS_MODMUL_BARRETT) return mm_barrett(a, c);
  if (M == CKKS_MODMUL_MONTGOMERY) return mm_montgomery(a, c);
  if (M == CKKS_MODMUL_SHOUP) return mm_shoup(a, c);
  return mm_smr(a, c);
}

constexpr int kChains = 8;

template <int M>
__global__ void k_modmul_chain(MulConsts c, const uint32_t* in, uint32_t* out, int n, int rounds) {
  const int base = (blockIdx.x * blockDim.x + threadIdx.x) * kChains;
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = base + k < n ? in[base + k] : 0;
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = mm<M>(a[k], c);
  }
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    if (base + k < n) out[base + k] = a[k];
}

// Integer multiply issue rates: 16 independent dependent chains per thread of
// one instruction form (mad.lo, mad.hi, mad.wide), enough warps for every
// scheduler; the chains' xor is stored so that nothing is removed.
template <int OP>
__global__ void k_intop_chain(uint32_t c, uint32_t d, uint32_t* out, int rounds) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[16];
  uint64_t w[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    x[k] = tid * 16 + k;
    w[k] = (uint64_t)(tid * 16 + k) << 7;
  }
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (OP == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(c), "r"(d));
      if (OP == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(c), "r"(d));
      if (OP == 2) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[k]) : "r"((uint32_t)(w[k] >> 16)), "r"(c));
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc ^= x[k] ^ (uint32_t)w[k] ^ (uint32_t)(w[k] >> 32);
  out[tid] = acc;
}

uint32_t inv_pow2_32(uint32_t q) {  // q^-1 mod 2^32 for odd q (Newton iteration)
  uint32_t x = q;
  for (int i = 0; i < 5; ++i) x *= 2u - q * x;
  return x;
}

}  // namespace
}  // namespace ckks

using namespace ckks;

extern "C" int ckks_bench_modmul(ckks_ctx* ctx, int method, int prime_id, uint32_t b, const uint32_t* a_host,
                                 int n, int rounds, uint32_t* out_host, float* ms) {
  if (!ctx || !a_host || !out_host || !ms || n < 1 || rounds < 0) return CKKS_EINVAL;
  if (method < CKKS_MODMUL_BARRETT || method > CKKS_MODMUL_SMR) return CKKS_EINVAL;
  if (prime_id < 0 || prime_id >= (int)ctx->pc_host.size()) return CKKS_EINVAL;
  MulConsts c{};
  c.q = ctx->pc_host[prime_id].q;
  if (b >= c.q) return CKKS_EINVAL;
  c.b = b;
  c.mu = (uint64_t)(((unsigned __int128)1 << 64) / c.q);
  c.m = inv_pow2_32(c.q);
  c.qinv_neg = 0u - c.m;
  c.b_mont = (uint32_t)(((uint64_t)b << 32) % c.q);
  c.b_sh = (uint32_t)(((uint64_t)b << 32) / c.q);
  for (int i = 0; i < n; ++i)
    if (a_host[i] >= c.q) return CKKS_EINVAL;
  uint32_t *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, (size_t)n * 4) != cudaSuccess) return CKKS_ENOMEM;
  if (cudaMalloc(&dout, (size_t)n * 4) != cudaSuccess) {
    cudaFree(din);
    return CKKS_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t st = ctx->stream;
  cudaMemcpyAsync(din, a_host, (size_t)n * 4, cudaMemcpyHostToDevice, st);
  const int threads = 256, per = threads * kChains, blocks = (n + per - 1) / per;
  auto run = [&]() {
    switch (method) {
      case CKKS_MODMUL_BARRETT: k_modmul_chain<CKKS_MODMUL_BARRETT><<<blocks, threads, 0, st>>>(c, din, dout, n, rounds); break;
      case CKKS_MODMUL_MONTGOMERY: k_modmul_chain<CKKS_MODMUL_MONTGOMERY><<<blocks, threads, 0, st>>>(c, din, dout, n, rounds); break;
      case CKKS_MODMUL_SHOUP: k_modmul_chain<CKKS_MODMUL_SHOUP><<<blocks, threads, 0, st>>>(c, din, dout, n, rounds); break;
      default: k_modmul_chain<CKKS_MODMUL_SMR><<<blocks, threads, 0, st>>>(c, din, dout, n, rounds); break;
    }
    count_launch(1);
  };
  run();  // warm-up
  cudaEventRecord(e0, st);
  run();
  cudaEventRecord(e1, st);
  cudaMemcpyAsync(out_host, dout, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  float t = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  *ms = t;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(din);
  cudaFree(dout);
  if (e != cudaSuccess) {
    ctx->err = std::string("bench_modmul: ") + cudaGetErrorString(e);
    return CKKS_ECUDA;
  }
  return CKKS_OK;
}

extern "C" int ckks_bench_intop(ckks_ctx* ctx, int op, int rounds, double* ops, float* ms) {
  if (!ctx || !ops || !ms || op < CKKS_INTOP_MAD_LO || op > CKKS_INTOP_MAD_WIDE || rounds < 1) return CKKS_EINVAL;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  uint32_t* dout = nullptr;
  if (cudaMalloc(&dout, (size_t)threads * blocks * 4) != cudaSuccess) return CKKS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t st = ctx->stream;
  const uint32_t c = 0x9E3779B1u, d = 0x7F4A7C15u;
  auto run = [&]() {
    switch (op) {
      case CKKS_INTOP_MAD_LO: k_intop_chain<0><<<blocks, threads, 0, st>>>(c, d, dout, rounds); break;
      case CKKS_INTOP_MAD_HI: k_intop_chain<1><<<blocks, threads, 0, st>>>(c, d, dout, rounds); break;
      default: k_intop_chain<2><<<blocks, threads, 0, st>>>(c, d, dout, rounds); break;
    }
    count_launch(1);
  };
  run();  // warm-up
  cudaEventRecord(e0, st);
  run();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaStreamSynchronize(st);
  float t = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  *ms = t;
  *ops = (double)threads * blocks * 16 * rounds;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dout);
  if (e != cudaSuccess) {
    ctx->err = std::string("bench_intop: ") + cudaGetErrorString(e);
    return CKKS_ECUDA;
  }
  return CKKS_OK;
}
