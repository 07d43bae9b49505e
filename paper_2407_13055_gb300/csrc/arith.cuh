// Device-side 32-bit modular arithmetic for primes q < 2^31 (Sec. 3, Sec. 4.1).
#pragma once
#include <cstdint>

namespace ckks {

// Per-prime constants, one entry per prime id (ciphertext primes first, then
// the auxiliary primes).
struct PrimeConst {
  uint32_t q;        // the prime, q = 1 mod 2N, q < 2^31
  uint32_t m;        // q^-1 mod 2^32 (signed Montgomery reduction, Alg. 2)
  int32_t r2c;       // 2^64 mod q, centered: turns a Montgomery product into a plain one
  int32_t r1c;       // 2^32 mod q, centered: BConv matrix entry of a one-prime conversion
  uint32_t ninv;     // N^-1 mod q
  uint32_t ninv_sh;  // Shoup companion floor(ninv 2^32 / q)
  uint32_t mont;     // 2^32 mod q (to Montgomery form)
  uint32_t mont_sh;
};

// a in [0, 2b) -> [0, b): min(a, a - b) on unsigned values.
__device__ __forceinline__ uint32_t csub(uint32_t a, uint32_t b) { return min(a, a - b); }

// Signed Montgomery reduction (Alg. 2): for x in [-q 2^31, q 2^31),
// y = x 2^-32 mod q with y in (-q, q): one low and one high signed product.
__device__ __forceinline__ int32_t smr(int64_t x, uint32_t q, uint32_t m) {
  uint32_t lo = (uint32_t)x;
  int32_t hi = (int32_t)(x >> 32);
  int32_t z = (int32_t)(lo * m);
  return hi - __mulhi(z, (int32_t)q);
}

// Shoup's product by a constant w < q with companion wsh = floor(w 2^32 / q):
// any 32-bit a -> a w mod q in [0, 2q).
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t wsh, uint32_t q) {
  uint32_t h = __umulhi(a, wsh);
  return a * w - h * q;
}

// Exact a * b mod q for a, b in [0, q): two signed Montgomery reductions,
// the second by 2^64 mod q to remove the 2^-32 factors. Result in [0, q).
__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, const PrimeConst& P) {
  int32_t t = smr((int64_t)((uint64_t)a * b), P.q, P.m);
  int32_t u = smr((int64_t)t * P.r2c, P.q, P.m);
  return (uint32_t)(u + ((u >> 31) & (int32_t)P.q));
}

// Montgomery product with one operand in Montgomery form (b~ = b 2^32 mod q):
// a in [0, 2^31) -> a b mod q in (-q, q).
__device__ __forceinline__ int32_t mont_mul(uint32_t a, uint32_t bm, uint32_t q, uint32_t m) {
  return smr((int64_t)((uint64_t)a * bm), q, m);
}

// 64-bit sum folded below 2^32 q: lo + hi [2^32]_q (r32 = 2^32 mod q).
__device__ __forceinline__ uint64_t fold64(uint64_t s, uint32_t r32) {
  return (uint64_t)(uint32_t)s + (uint64_t)(uint32_t)(s >> 32) * r32;
}

// Unsigned Montgomery reduction (Montgomery 1985) of s < 2^32 q: s 2^-32 mod
// q in [0, 2q]; m = q^-1 mod 2^32 (t = -lo q^-1 makes lo + t q = 0 mod 2^32,
// with a carry exactly when lo != 0).
__device__ __forceinline__ uint32_t redc64(uint64_t s, uint32_t q, uint32_t m) {
  const uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32);
  const uint32_t t = 0u - lo * m;
  return hi + __umulhi(t, q) + (lo != 0u);
}

// (-q, q) -> [0, q)
__device__ __forceinline__ uint32_t fix_signed(int32_t v, uint32_t q) {
  return (uint32_t)(v + ((v >> 31) & (int32_t)q));
}

// Harvey-style lazy butterflies with Shoup twiddles (w, wsh).
// LAZY (q < 2^30): forward inputs/outputs in [0, 4q); inverse in [0, 2q).
// !LAZY (q < 2^31): forward and inverse values in [0, 2q).
template <bool LAZY>
__device__ __forceinline__ void ct_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wsh, uint32_t q) {
  if (LAZY) {
    const uint32_t q2 = 2 * q;
    x = csub(x, q2);
    uint32_t t = shoup(y, w, wsh, q);
    y = x - t + q2;
    x = x + t;
  } else {
    x = csub(x, q);
    uint32_t t = csub(shoup(y, w, wsh, q), q);
    y = x - t + q;
    x = x + t;
  }
}

template <bool LAZY>
__device__ __forceinline__ void gs_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wsh, uint32_t q) {
  if (LAZY) {
    const uint32_t q2 = 2 * q;
    uint32_t s = x + y;
    uint32_t d = x - y + q2;
    x = csub(s, q2);
    y = shoup(d, w, wsh, q);
  } else {
    x = csub(x, q);
    y = csub(y, q);
    uint32_t s = x + y;
    uint32_t d = x - y + q;
    x = s;
    y = shoup(d, w, wsh, q);
  }
}

// Reduce a lazily reduced value to [0, q).
template <bool LAZY>
__device__ __forceinline__ uint32_t normalize(uint32_t x, uint32_t q) {
  if (LAZY) x = csub(x, 2 * q);
  return csub(x, q);
}

// Centered representative of x in [0, q): (-(q-1)/2 .. (q-1)/2).
__device__ __forceinline__ int32_t centered(uint32_t x, uint32_t q) {
  return x > (q >> 1) ? (int32_t)(x - q) : (int32_t)x;
}

}  // namespace ckks
