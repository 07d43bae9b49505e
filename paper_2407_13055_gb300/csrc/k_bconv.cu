// Fast basis conversion (Eq. 2) on coefficient-domain limbs, two bit-identical
// variants:
//  * CUDA cores: centered inputs, the paper's lazy 64-bit accumulation and one
//    signed Montgomery reduction per output (Sec. 4.2);
//  * INT8 tensor cores: unsigned residues u_k in [0, q_k) split into bytes,
//    multiplied with the byte planes of the matrix by mma.sync (u8 x u8 ->
//    s32, exact), then recombined modulo p. The centered form is recovered
//    exactly by subtracting c [Q]_p, c = number of inputs above q_k / 2, which
//    enters the product as one more input limb.
#include "internal.h"

namespace ckks {

// ---------------------------------------------------------------------------
// CUDA-core variant: one coefficient per thread.
// ---------------------------------------------------------------------------
__global__ void k_bconv_core(DevParams dp, const uint32_t* __restrict__ in, int k, const int* src_ids,
                             const uint2* cin, const int32_t* mat, uint32_t* out, int m, const int* dst_ids) {
  const int n = 1 << dp.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int32_t y[64];
  for (int i = 0; i < k; ++i) {
    const uint32_t q = dp.pc[src_ids[i]].q;
    const uint2 w = cin[i];
    y[i] = centered(csub(shoup(in[(size_t)i * n + c], w.x, w.y, q), q), q);
  }
  for (int t = 0; t < m; ++t) {
    const PrimeConst P = dp.pc[dst_ids[t]];
    const int64_t lim = (int64_t)P.q << 31, wrap = (int64_t)P.q << 32;
    int64_t acc = 0;
    int since = 0, batch = 8;
    for (int i = 0; i < k; ++i) {
      acc += (int64_t)y[i] * (int64_t)mat[(size_t)t * k + i];
      if (++since == batch) {
        acc = acc >= lim ? acc - wrap : (acc < -lim ? acc + wrap : acc);
        since = 0;
        batch = 4;
      }
    }
    acc = acc >= lim ? acc - wrap : (acc < -lim ? acc + wrap : acc);
    out[(size_t)t * n + c] = fix_signed(smr(acc, P.q, P.m), P.q);
  }
}

// ---------------------------------------------------------------------------
// INT8 tensor-core variant.
//
// GEMM shape: rows (t, s) = 7 t + s for the m targets and the seven byte
// weights 2^(8s); columns = coefficients; reduction index (kk, a) = 4 kk + a
// over the k inputs plus the count limb (kk = k) and the four bytes a of u.
// abytes[(t,s)][(kk,a)] = byte (s - a) of Bt[t][kk] (zero outside 0..3),
// Bt[t][kk] = [(Qs/s_kk) 2^64]_{p_t} and Bt[t][k] = [-Qs 2^64]_{p_t}. Then
// D_s = sum_(kk,a) abytes * byte_a(u_kk) is exact in int32 and
//   acc = sum_s D_s 2^(8s) = lo + hi 2^32  (lo = s 0..3, hi = s 4..6),
// acc = 2^64 (sum_kk y_kk Qs/s_kk) mod p, so SMR(SMR(lo) + hi) is the result.
// ---------------------------------------------------------------------------
constexpr int TC_WARPS = 4;

__device__ __forceinline__ void mma_u8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(32 * TC_WARPS) k_bconv_tc(DevParams dp, const uint32_t* __restrict__ in, int k,
                                                            const int* src_ids, const uint2* cin,
                                                            const uint8_t* abytes, int mp, int kp, uint32_t* out,
                                                            int m, const int* dst_ids) {
  extern __shared__ uint32_t sm[];
  const int n = 1 << dp.log_n;
  uint8_t* A = reinterpret_cast<uint8_t*>(sm);                     // [mp][kp] bytes
  int* cst = reinterpret_cast<int*>(sm + (mp * kp) / 4) + (threadIdx.x / 32) * mp * 8;  // per warp [mp][8]
  for (int i = threadIdx.x; i < mp * kp / 4; i += blockDim.x) sm[i] = reinterpret_cast<const uint32_t*>(abytes)[i];
  __syncthreads();
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int g = lane >> 2, tig = lane & 3;
  const int ks_n = kp / 32;
  const int tiles = n / 8;
  for (int tile = blockIdx.x * TC_WARPS + warp; tile < tiles; tile += gridDim.x * TC_WARPS) {
    const int col = tile * 8 + g;
    // B fragments: b0 of k-step ks holds u_(8 ks + tig), b1 holds u_(8 ks + 4 + tig).
    uint32_t u[2 * 9];
    int cnt = 0;
    for (int ks = 0; ks < ks_n; ++ks)
      for (int h = 0; h < 2; ++h) {
        const int kk = 8 * ks + 4 * h + tig;
        uint32_t v = 0;
        if (kk < k) {
          const uint32_t q = dp.pc[src_ids[kk]].q;
          const uint2 w = cin[kk];
          v = csub(shoup(in[(size_t)kk * n + col], w.x, w.y, q), q);
          cnt += v > (q >> 1);
        }
        u[2 * ks + h] = v;
      }
    cnt += __shfl_xor_sync(0xffffffffu, cnt, 1);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, 2);
    for (int ks = 0; ks < ks_n; ++ks)
      for (int h = 0; h < 2; ++h)
        if (8 * ks + 4 * h + tig == k) u[2 * ks + h] = (uint32_t)cnt;
    for (int mb = 0; mb < mp / 16; ++mb) {
      int acc[4] = {0, 0, 0, 0};
      for (int ks = 0; ks < ks_n; ++ks) {
        const uint8_t* r0 = A + (size_t)(16 * mb + g) * kp + 32 * ks + 4 * tig;
        const uint8_t* r1 = r0 + 8 * kp;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(r0);
        a[1] = *reinterpret_cast<const uint32_t*>(r1);
        a[2] = *reinterpret_cast<const uint32_t*>(r0 + 16);
        a[3] = *reinterpret_cast<const uint32_t*>(r1 + 16);
        mma_u8(acc, a, u[2 * ks], u[2 * ks + 1]);
      }
      cst[(16 * mb + g) * 8 + 2 * tig] = acc[0];
      cst[(16 * mb + g) * 8 + 2 * tig + 1] = acc[1];
      cst[(16 * mb + g + 8) * 8 + 2 * tig] = acc[2];
      cst[(16 * mb + g + 8) * 8 + 2 * tig + 1] = acc[3];
    }
    __syncwarp();
    for (int t = tig; t < m; t += 4) {
      const PrimeConst P = dp.pc[dst_ids[t]];
      uint64_t d[7];
#pragma unroll
      for (int s = 0; s < 7; ++s) d[s] = (uint32_t)cst[(7 * t + s) * 8 + g];
      const uint64_t lo = d[0] + (d[1] << 8) + (d[2] << 16) + (d[3] << 24);
      const uint64_t hi = d[4] + (d[5] << 8) + (d[6] << 16);
      const int64_t x = (int64_t)smr((int64_t)lo, P.q, P.m) + (int64_t)hi;
      out[(size_t)t * n + col] = fix_signed(smr(x, P.q, P.m), P.q);
    }
    __syncwarp();
  }
}

void launch_bconv(const DevParams& dp, const uint32_t* in, int k, const int* src_ids, const uint2* cin,
                  const int32_t* mat, uint32_t* out, int m, const int* dst_ids, int variant, const uint8_t* abytes,
                  int mp, int kp, cudaStream_t st) {
  const int n = 1 << dp.log_n;
  if (variant == 0) {
    k_bconv_core<<<(n + 127) / 128, 128, 0, st>>>(dp, in, k, src_ids, cin, mat, out, m, dst_ids);
  } else {
    const size_t smem = (size_t)mp * kp + (size_t)TC_WARPS * mp * 8 * sizeof(int);
    cudaFuncSetAttribute(k_bconv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = (n / 8 + TC_WARPS - 1) / TC_WARPS;
    if (blocks > 4 * dp.sms) blocks = 4 * dp.sms;
    k_bconv_tc<<<blocks, 32 * TC_WARPS, smem, st>>>(dp, in, k, src_ids, cin, abytes, mp, kp, out, m, dst_ids);
  }
}

}  // namespace ckks
