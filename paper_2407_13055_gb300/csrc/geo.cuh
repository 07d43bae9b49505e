// Launch geometry of the row/column kernels for each supported ring degree.
#pragma once
#include "ntt.cuh"

namespace ckks {

// EC, ER: values per thread in the column and row phases; H = EC^2 rows of
// W = ER^2 words. Supported: N = 2^8 (4, 4), 2^12 (8, 8), 2^16 (8, 32).
template <int EC_, int ER_>
struct Geo {
  static constexpr int EC = EC_, ER = ER_;
  static constexpr int H = EC * EC, W = ER * ER, N = H * W;
  static constexpr int RPC = (128 / ER < H) ? 128 / ER : H;  // rows per row-kernel block
  static constexpr int RT = RPC * ER;                         // row-kernel threads
  static constexpr int TC = 16;                               // columns per column-kernel block
  static constexpr int CT = TC * EC;                          // column-kernel threads
  static constexpr int ROWBUF = W + ER;                       // words per row transpose buffer
  static constexpr int COLBUF = (H + EC) * TC;                // words per column transpose buffer
};

#define CKKS_DISPATCH_LOGN(log_n, ...)                    \
  do {                                                    \
    switch (log_n) {                                      \
      case 8: {                                           \
        using G = ::ckks::Geo<4, 4>;                      \
        __VA_ARGS__;                                      \
      } break;                                            \
      case 12: {                                          \
        using G = ::ckks::Geo<8, 8>;                      \
        __VA_ARGS__;                                      \
      } break;                                            \
      case 16: {                                          \
        using G = ::ckks::Geo<8, 32>;                     \
        __VA_ARGS__;                                      \
      } break;                                            \
      default:                                            \
        break;                                            \
    }                                                     \
  } while (0)

__device__ __forceinline__ uint32_t brev_n(uint32_t v, int log_n) { return __brev(v) >> (32 - log_n); }

// Source position (internal bit-reversed layout) of destination position p
// under the NTT-domain automorphism out[j] = in[((2j+1)k mod 2N - 1)/2] (Eq. 4).
__device__ __forceinline__ uint32_t auto_src(uint32_t p, uint32_t k, int log_n) {
  uint32_t j = brev_n(p, log_n);
  uint32_t mask = (2u << log_n) - 1;
  uint32_t jp = (((2 * j + 1) * k) & mask) >> 1;
  return brev_n(jp, log_n);
}

}  // namespace ckks
