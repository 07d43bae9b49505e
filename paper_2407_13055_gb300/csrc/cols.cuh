// Column phase of the key switch: every ModSwitch (iNTT -> BConv -> NTT,
// Alg. 1) runs its coefficient-domain middle inside one column kernel. A block
// holds a tile of TC columns x H rows; its slices of TC * EC threads share the
// tile's centered inputs in shared memory and convert the targets between
// them. Launch shapes (tile width, slices, target split, targets per pass)
// are chosen at run time; the launchers are instantiated per geometry in
// separate translation units (k_cols_*.cu) so that the variants compile in
// parallel.
#pragma once
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "geo.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tc.cuh"

namespace ckks {

namespace {

__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, uint32_t q) { return csub(a + b, q); }

// Prime id of extended limb t at a level whose window starts at prime base.
__device__ __forceinline__ int prime_of(int t, int n, int L, int base) { return t < n ? base + t : L + (t - n); }

// BConv of EC coefficient-domain values per thread: out[i] = sum_k y[k][i] *
// mat[k] reduced modulo p (Eq. 2 with the 2^32 factor folded into mat).
// y is in shared memory: y4[(k * EC/4 + i/4) * NT + pos]. Lazy reduction as
// in Sec. 4.2: |y|, |mat| < p/2 bound each product by 2^29 p, so eight of
// them and then four more after each range reduction stay below 2^63. The
// range reduction folds the high word back with 2^32 = r1c (mod p):
// acc = lo + hi * r1c, |acc| < 2^30 p + 2^32, which also meets the signed
// Montgomery reduction's input range [-p 2^31, p 2^31).
__device__ __forceinline__ int64_t fold(int64_t a, int32_t r1c) {
  return (int64_t)(uint32_t)a + (int64_t)(int32_t)(a >> 32) * (int64_t)r1c;
}

template <int EC, int NT>
__device__ __forceinline__ void mac4(int64_t (&acc)[EC], const int4* __restrict__ y4, int pos, int k, int64_t b) {
#pragma unroll
  for (int i4 = 0; i4 < EC / 4; ++i4) {
    const int4 v = y4[(k * (EC / 4) + i4) * NT + pos];
    acc[4 * i4 + 0] += (int64_t)v.x * b;
    acc[4 * i4 + 1] += (int64_t)v.y * b;
    acc[4 * i4 + 2] += (int64_t)v.z * b;
    acc[4 * i4 + 3] += (int64_t)v.w * b;
  }
}

// Sum of the sources' centered bounds, sum_k (s_k - 1) / 2 (float: it is only
// compared with 2^63 at a margin far above its rounding error).
__device__ __forceinline__ float src_bound(const DevParams& dp, int K, int id0, const int2* idtab = nullptr) {
  float s = 0.f;
  for (int k = 0; k < K; ++k) s += (float)(dp.pc[idtab ? idtab[k].y : id0 + k].q >> 1);
  return s;
}

// With |y_k| <= (s_k - 1)/2 and |mat_k| <= (p - 1)/2, the whole sum stays
// below 2^63 when sum_k (s_k - 1)/2 * (p - 1)/2 does, and then only the final
// range reduction is needed (2^63 = 9.22e18).
__device__ __forceinline__ bool no_fold(float sy, uint32_t p) { return sy * (float)(p >> 1) < 9.0e18f; }

// Chunks of four products, unrolled. Without the bound above (nofold false),
// 2^29 p per product allows eight before the first range reduction and four
// after each one, so the fold runs after every chunk but the first, and once
// at the end.
template <int EC, int NT>
__device__ __forceinline__ void bconv_accumulate(const int4* __restrict__ y4, int pos, int K,
                                                 const int32_t* __restrict__ mat, const PrimeConst& P,
                                                 uint32_t (&out)[EC], bool nofold) {
  int64_t acc[EC];
#pragma unroll
  for (int i = 0; i < EC; ++i) acc[i] = 0;
  int k = 0;
  if (nofold) {
    for (; k + 4 <= K; k += 4) {
      const int64_t b0 = __ldg(mat + k), b1 = __ldg(mat + k + 1), b2 = __ldg(mat + k + 2), b3 = __ldg(mat + k + 3);
      mac4<EC, NT>(acc, y4, pos, k, b0);
      mac4<EC, NT>(acc, y4, pos, k + 1, b1);
      mac4<EC, NT>(acc, y4, pos, k + 2, b2);
      mac4<EC, NT>(acc, y4, pos, k + 3, b3);
    }
  }
  for (; k + 4 <= K; k += 4) {
    const int64_t b0 = __ldg(mat + k), b1 = __ldg(mat + k + 1), b2 = __ldg(mat + k + 2), b3 = __ldg(mat + k + 3);
    mac4<EC, NT>(acc, y4, pos, k, b0);
    mac4<EC, NT>(acc, y4, pos, k + 1, b1);
    mac4<EC, NT>(acc, y4, pos, k + 2, b2);
    mac4<EC, NT>(acc, y4, pos, k + 3, b3);
    if (k >= 4) {
#pragma unroll
      for (int i = 0; i < EC; ++i) acc[i] = fold(acc[i], P.r1c);
    }
  }
  for (; k < K; ++k) mac4<EC, NT>(acc, y4, pos, k, (int64_t)__ldg(mat + k));
#pragma unroll
  for (int i = 0; i < EC; ++i) out[i] = fix_signed(smr(fold(acc[i], P.r1c), P.q, P.m), P.q);
}

// Two targets per pass: each shared-memory read of y feeds both sums, which
// halves the shared-memory traffic of the conversion at the cost of a second
// set of accumulators.
template <int EC, int NT>
__device__ __forceinline__ void mac4x2(int64_t (&a0)[EC], int64_t (&a1)[EC], const int4* __restrict__ y4, int pos,
                                       int k, int64_t b0, int64_t b1) {
#pragma unroll
  for (int i4 = 0; i4 < EC / 4; ++i4) {
    const int4 v = y4[(k * (EC / 4) + i4) * NT + pos];
    a0[4 * i4 + 0] += (int64_t)v.x * b0;
    a0[4 * i4 + 1] += (int64_t)v.y * b0;
    a0[4 * i4 + 2] += (int64_t)v.z * b0;
    a0[4 * i4 + 3] += (int64_t)v.w * b0;
    a1[4 * i4 + 0] += (int64_t)v.x * b1;
    a1[4 * i4 + 1] += (int64_t)v.y * b1;
    a1[4 * i4 + 2] += (int64_t)v.z * b1;
    a1[4 * i4 + 3] += (int64_t)v.w * b1;
  }
}

template <int EC, int NT>
__device__ __forceinline__ void bconv_accumulate2(const int4* __restrict__ y4, int pos, int K,
                                                  const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                                                  const PrimeConst& P0, const PrimeConst& P1, uint32_t (&o0)[EC],
                                                  uint32_t (&o1)[EC], bool nofold) {
  int64_t a0[EC], a1[EC];
#pragma unroll
  for (int i = 0; i < EC; ++i) a0[i] = a1[i] = 0;
  int k = 0;
  if (nofold) {
    for (; k + 4 <= K; k += 4) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mac4x2<EC, NT>(a0, a1, y4, pos, k + kk, (int64_t)__ldg(m0 + k + kk), (int64_t)__ldg(m1 + k + kk));
    }
  }
  for (; k + 4 <= K; k += 4) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mac4x2<EC, NT>(a0, a1, y4, pos, k + kk, (int64_t)__ldg(m0 + k + kk), (int64_t)__ldg(m1 + k + kk));
    if (k >= 4) {
#pragma unroll
      for (int i = 0; i < EC; ++i) {
        a0[i] = fold(a0[i], P0.r1c);
        a1[i] = fold(a1[i], P1.r1c);
      }
    }
  }
  for (; k < K; ++k) mac4x2<EC, NT>(a0, a1, y4, pos, k, (int64_t)__ldg(m0 + k), (int64_t)__ldg(m1 + k));
#pragma unroll
  for (int i = 0; i < EC; ++i) {
    o0[i] = fix_signed(smr(fold(a0[i], P0.r1c), P0.q, P0.m), P0.q);
    o1[i] = fix_signed(smr(fold(a1[i], P1.r1c), P1.q, P1.m), P1.q);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Column kernels
// ---------------------------------------------------------------------------

// Column kernels. A block covers a tile of TC columns x H rows and is split
// into GS slices of CT = TC * EC threads; position pos = (jj, c) of a slice
// owns EC elements of one column. The slices share the coefficient-domain
// tile: slice s finishes the iNTT of input limbs k = s, s + GS, ..., then
// (after one block barrier) handles targets m = s, s + GS, ...; each slice
// synchronizes its own transposes with a named barrier.
template <class G, int TC>
struct ColTile {
  static constexpr int EC = G::EC, H = G::H, W = G::W;
  static constexpr int CT = TC * EC;
  static constexpr int BUF = (H + EC) * TC;
};

template <class G, int TC>
__device__ __forceinline__ void col_inputs(const DevParams& dp, const uint32_t* src, size_t src_stride, int K,
                                           int id0, const uint2* cin, int4* y4, uint32_t* colbuf, int l, int jj,
                                           int c, int pos, int slice, int GS, uint32_t* ycopy = nullptr,
                                           const int2* idtab = nullptr) {
  using CTL = ColTile<G, TC>;
  // the next source's loads are issued before this one's iNTT columns
  uint32_t nx[G::EC];
  if (slice < K) {
#pragma unroll
    for (int i = 0; i < G::EC; ++i) nx[i] = src[slice * src_stride + (G::EC * jj + i) * G::W + l];
  }
  for (int k = slice; k < K; k += GS) {
    const int id = idtab ? idtab[k].y : id0 + k;
    const uint32_t q = dp.pc[id].q;
    const uint2* itw = dp.itw + ((size_t)id << dp.log_n);
    uint32_t x[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) x[i] = nx[i];
    if (k + GS < K) {
      const uint32_t* s = src + (k + GS) * src_stride;
#pragma unroll
      for (int i = 0; i < G::EC; ++i) nx[i] = s[(G::EC * jj + i) * G::W + l];
    }
    if (q < (1u << 30)) col_inv<G::EC, TC, true>(x, colbuf, itw, jj, c, q, slice + 1, CTL::CT);
    else col_inv<G::EC, TC, false>(x, colbuf, itw, jj, c, q, slice + 1, CTL::CT);
    const uint2 w = cin[k];
    int32_t y[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) y[i] = centered(csub(shoup(x[i], w.x, w.y, q), q), q);
#pragma unroll
    for (int i4 = 0; i4 < G::EC / 4; ++i4)
      y4[(k * (G::EC / 4) + i4) * CTL::CT + pos] = make_int4(y[4 * i4], y[4 * i4 + 1], y[4 * i4 + 2], y[4 * i4 + 3]);
    if (ycopy) {
      uint32_t* yc = ycopy + ((size_t)k << dp.log_n);
#pragma unroll
      for (int i = 0; i < G::EC; ++i) yc[(jj + G::EC * i) * G::W + l] = (uint32_t)y[i];
    }
  }
}

// NTT column phase of one converted target; store B layout (lazy range).
template <class G, int TC>
__device__ __forceinline__ void col_ntt_store(const DevParams& dp, uint32_t (&x)[G::EC], int id, uint32_t* dst,
                                              uint32_t* colbuf, int l, int jj, int c, int slice) {
  using CTL = ColTile<G, TC>;
  const uint32_t q = dp.pc[id].q;
  const uint2* tw = dp.tw + ((size_t)id << dp.log_n);
  if (q < (1u << 30)) col_fwd<G::EC, TC, true>(x, colbuf, tw, jj, c, q, slice + 1, CTL::CT);
  else col_fwd<G::EC, TC, false>(x, colbuf, tw, jj, c, q, slice + 1, CTL::CT);
#pragma unroll
  for (int i = 0; i < G::EC; ++i) dst[(G::EC * jj + i) * G::W + l] = x[i];
}

// BConv each target m = m0, m0 + step, ... (mat row, prime id, destination
// from tgt), then its NTT column phase; TP = 2 converts targets in pairs.
template <class G, int TC, int TP, class Target>
__device__ __forceinline__ void col_targets(const DevParams& dp, const int4* y4, int K, int M, int m0, int step,
                                            Target tgt, uint32_t* colbuf, int l, int jj, int c, int pos,
                                            int slice, float sy) {
  using CTL = ColTile<G, TC>;
  int m = m0;
  if (TP == 2) {
    for (; m + step < M; m += 2 * step) {
      const int32_t *r0, *r1;
      int i0, i1;
      uint32_t *d0, *d1;
      tgt(m, r0, i0, d0);
      tgt(m + step, r1, i1, d1);
      const PrimeConst P0 = dp.pc[i0], P1 = dp.pc[i1];
      uint32_t x0[G::EC], x1[G::EC];
      bconv_accumulate2<G::EC, CTL::CT>(y4, pos, K, r0, r1, P0, P1, x0, x1, no_fold(sy, P0.q) && no_fold(sy, P1.q));
      col_ntt_store<G, TC>(dp, x0, i0, d0, colbuf, l, jj, c, slice);
      col_ntt_store<G, TC>(dp, x1, i1, d1, colbuf, l, jj, c, slice);
    }
  }
  for (; m < M; m += step) {
    const int32_t* row;
    int id;
    uint32_t* dst;
    tgt(m, row, id, dst);
    const PrimeConst P = dp.pc[id];
    uint32_t x[G::EC];
    bconv_accumulate<G::EC, CTL::CT>(y4, pos, K, row, P, x, no_fold(sy, P.q));
    col_ntt_store<G, TC>(dp, x, id, dst, colbuf, l, jj, c, slice);
  }
}

// Launch shape (section "Launch shapes" below): SL slices per block; blockIdx.z
// of gridDim.z blocks per column tile takes targets m = slice + SL z (mod
// SL gridDim.z), all of them recomputing the shared input iNTT columns.

// C1: ModUp column kernel. grid (W/TC, digits, Z), block SL * CT.
template <class G, int TC, int SL, int TP>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_ks_modup_cols(DevParams dp, int n, int base, int tix,
                                                                               const uint32_t* S, uint32_t* T) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int j = blockIdx.y;  // j-th active digit of the window
  const int alpha = dp.alpha, L = dp.L, ext = n + alpha;
  const int g = base / alpha + j;
  const int lo = max(0, g * alpha - base), hi = min(n, (g + 1) * alpha - base), K = hi - lo;
  const int2 off = dp.ks.up_off[tix * dp.dnum + j];
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)alpha * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  col_inputs<G, TC>(dp, S + ((size_t)lo << dp.log_n), (size_t)1 << dp.log_n, K, base + lo, dp.ks.up_cin + off.x,
                    y4, colbuf, l, jj, c, pos, slice, SL);
  __syncthreads();
  const int M = ext - K;
  auto tgt = [&](int m, const int32_t*& row, int& id, uint32_t*& dst) {
    const int t = m < lo ? m : m + K;  // skip the digit's own limbs
    row = dp.ks.up_mat + off.y + t * K;
    id = prime_of(t, n, L, base);
    dst = T + ((size_t)(j * ext + t) << dp.log_n);
  };
  col_targets<G, TC, TP>(dp, y4, K, M, slice + SL * blockIdx.z, SL * gridDim.z, tgt, colbuf, l, jj, c, pos, slice,
                         src_bound(dp, K, base + lo));
}

// C2: ModDown column kernel. grid (W/TC, 2 polys, Z). Input S [2][alpha][N]
// (P limbs after the row-phase iNTT); output T [2][n][N].
template <class G, int TC, int SL, int TP>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_ks_moddown_cols(DevParams dp, int n, int base,
                                                                                 const uint32_t* S, uint32_t* T) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int u = blockIdx.y;
  const int alpha = dp.alpha;
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)alpha * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  col_inputs<G, TC>(dp, S + ((size_t)(u * alpha) << dp.log_n), (size_t)1 << dp.log_n, alpha, dp.L, dp.ks.dn_cin,
                    y4, colbuf, l, jj, c, pos, slice, SL);
  __syncthreads();
  auto tgt = [&](int i, const int32_t*& row, int& id, uint32_t*& dst) {
    row = dp.ks.dn_mat + (base + i) * alpha;
    id = base + i;
    dst = T + ((size_t)(u * n + i) << dp.log_n);
  };
  col_targets<G, TC, TP>(dp, y4, alpha, n, slice + SL * blockIdx.z, SL * gridDim.z, tgt, colbuf, l, jj, c, pos,
                         slice, src_bound(dp, alpha, dp.L));
}


// Top limb of the ModDown fused with rescaling, on one column tile of
// polynomial u (every thread of the block calls it). S holds the P limbs of
// both polynomials through their iNTT rows and, after them, E_u = A_u[l] P^-1
// + extra_u[l] (l = n - 1) through its iNTT rows. The P limbs' iNTT columns
// give their centered coefficients y (sources 0 .. alpha - 1 in y4); E's iNTT
// columns and the conversion z = BConv(P -> q_l) give the top limb's ModDown
// output V = E - z P^-1 = iNTT((A_l - z_l) P^-1 + d_l) in the coefficient
// domain, whose centered value c_l becomes source alpha. With Yu the y and
// c_l are also stored ([alpha + 1][N], A layout along h).
template <class G, int TC>
__device__ __forceinline__ void top_limb_sources(const DevParams& dp, int n, const uint32_t* S, int4* y4,
                                                 uint32_t* colbuf, int l, int jj, int c, int pos, int slice, int SL,
                                                 int u, uint32_t* Yu) {
  using CTL = ColTile<G, TC>;
  const int alpha = dp.alpha, top = n - 1;
  col_inputs<G, TC>(dp, S + ((size_t)(u * alpha) << dp.log_n), (size_t)1 << dp.log_n, alpha, dp.L, dp.ks.dn_cin,
                    y4, colbuf, l, jj, c, pos, slice, SL, Yu);
  const PrimeConst Pt = dp.pc[top];
  if (slice == SL - 1) {
    // E_u: iNTT columns, times N^-1, kept in [0, q_l) in source slot alpha
    const uint2* itw = dp.itw + ((size_t)top << dp.log_n);
    const uint32_t* s = S + ((size_t)(2 * alpha + u) << dp.log_n);
    uint32_t x[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) x[i] = s[(G::EC * jj + i) * G::W + l];
    if (Pt.q < (1u << 30)) col_inv<G::EC, TC, true>(x, colbuf, itw, jj, c, Pt.q, slice + 1, CTL::CT);
    else col_inv<G::EC, TC, false>(x, colbuf, itw, jj, c, Pt.q, slice + 1, CTL::CT);
    int32_t e[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) e[i] = (int32_t)csub(shoup(x[i], Pt.ninv, Pt.ninv_sh, Pt.q), Pt.q);
#pragma unroll
    for (int i4 = 0; i4 < G::EC / 4; ++i4)
      y4[(alpha * (G::EC / 4) + i4) * CTL::CT + pos] = make_int4(e[4 * i4], e[4 * i4 + 1], e[4 * i4 + 2], e[4 * i4 + 3]);
  }
  __syncthreads();
  if (slice == 0) {
    uint32_t z[G::EC];
    bconv_accumulate<G::EC, CTL::CT>(y4, pos, alpha, dp.ks.dn_mat + top * alpha, Pt, z,
                                     no_fold(src_bound(dp, alpha, dp.L), Pt.q));
    const uint2 pinv = dp.ks.dn_pinv[top];
#pragma unroll
    for (int i4 = 0; i4 < G::EC / 4; ++i4) {
      int4& slot = y4[(alpha * (G::EC / 4) + i4) * CTL::CT + pos];
      const int4 e = slot;
      const uint32_t ev[4] = {(uint32_t)e.x, (uint32_t)e.y, (uint32_t)e.z, (uint32_t)e.w};
      int32_t cl[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t zp = csub(shoup(z[4 * i4 + k], pinv.x, pinv.y, Pt.q), Pt.q);
        cl[k] = centered(csub(ev[k] + Pt.q - zp, Pt.q), Pt.q);
      }
      slot = make_int4(cl[0], cl[1], cl[2], cl[3]);
      if (Yu) {
        uint32_t* yc = Yu + ((size_t)alpha << dp.log_n);
#pragma unroll
        for (int k = 0; k < 4; ++k) yc[(jj + G::EC * (4 * i4 + k)) * G::W + l] = (uint32_t)cl[k];
      }
    }
  }
  __syncthreads();
}

// Top limb of the fused ModDown + rescale alone (the tensor-core form of the
// rescale conversion takes its sources from Y = [2][alpha + 1][N]).
// grid (W/TC, 2 polys).
template <class G, int TC, int SL>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_ks_moddown_cols_top(DevParams dp, int n,
                                                                                        const uint32_t* S,
                                                                                        uint32_t* Y) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int u = blockIdx.y, alpha = dp.alpha;
  uint32_t* colbuf =
      reinterpret_cast<uint32_t*>(smem4 + (size_t)(alpha + 1) * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  top_limb_sources<G, TC>(dp, n, S, smem4, colbuf, l, jj, c, pos, slice, SL, u,
                          Y + ((size_t)(u * (alpha + 1)) << dp.log_n));
}

// ModDown fused with rescaling, one column kernel per tile: the top limb's
// sources (top_limb_sources: the P limbs' centered coefficients and c_l, K =
// alpha + 1) convert to every q_i, i < l (matrix rs_mat: the ModDown row plus
// [P]_{q_i}) as w_i = z_i + P [c_l]_{q_i}; then the NTT columns. The top
// limb's ModDown needs only the coefficients of its own column positions, so
// it happens inside the tile. grid (W/TC, 2 polys, Z).
template <class G, int TC, int SL, int TP>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_rs_cols_fused(DevParams dp, int n, const uint32_t* S,
                                                                                  uint32_t* T) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int u = blockIdx.y;
  const int alpha = dp.alpha, top = n - 1, K = alpha + 1;
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)K * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  top_limb_sources<G, TC>(dp, n, S, y4, colbuf, l, jj, c, pos, slice, SL, u, nullptr);
  auto tgt = [&](int i, const int32_t*& row, int& id, uint32_t*& dst) {
    row = dp.ks.rs_mat + i * K;
    id = i;
    dst = T + ((size_t)(u * top + i) << dp.log_n);
  };
  col_targets<G, TC, TP>(dp, y4, K, top, slice + SL * blockIdx.z, SL * gridDim.z, tgt, colbuf, l, jj, c, pos, slice,
                         src_bound(dp, alpha, dp.L) + (float)(dp.pc[top].q >> 1));
}

// ModDown merged into the rescaling (Sec. 6), column kernel: the K source
// limbs of polynomial u (P primes, then the dropped window primes; row-phase
// iNTT already applied, S = [2][K]) finish their iNTT columns and are scaled
// by cin; BConv (Eq. 2, centered) to the n1 primes of the new window, then
// the NTT columns into T = [2][n1]. grid (W/TC, 2 polys, Z).
template <class G, int TC, int SL, int TP>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_mm_cols(DevParams dp, MmArgs m, const uint32_t* S,
                                                                    uint32_t* T) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int u = blockIdx.y;
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)m.K * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  col_inputs<G, TC>(dp, S + ((size_t)(u * m.K) << dp.log_n), (size_t)1 << dp.log_n, m.K, 0, m.cin, y4, colbuf, l,
                    jj, c, pos, slice, SL, nullptr, m.rows);
  __syncthreads();
  auto tgt = [&](int t, const int32_t*& row, int& id, uint32_t*& dst) {
    row = m.mat + t * m.K;
    id = m.s1 + t;
    dst = T + ((size_t)(u * m.n1 + t) << dp.log_n);
  };
  col_targets<G, TC, TP>(dp, y4, m.K, m.n1, slice + SL * blockIdx.z, SL * gridDim.z, tgt, colbuf, l, jj, c, pos,
                         slice, src_bound(dp, m.K, 0, m.rows));
}

template <class G, int TC, int SL>
static size_t col_smem_bytes(int K) {
  using CTL = ColTile<G, TC>;
  return (size_t)K * (G::EC / 4) * CTL::CT * sizeof(int4) + (size_t)SL * CTL::BUF * sizeof(uint32_t);
}

// Raise a kernel's dynamic shared-memory limit once per process (and only
// when a larger size is needed), so that steady-state launches and graph
// captures issue no attribute calls.
static void set_col_smem(const void* f, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = done[f];
  if (bytes > cur) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cur = bytes;
  }
}

// ---------------------------------------------------------------------------
// Launch shapes of the column kernels
//
// A shape is (tc, sl, z): column-tile width, slices per block and blocks per
// tile. Every shape computes the same values (only the division of targets
// among threads changes), so the choice affects time alone. The default
// follows a fixed rule; ckks_tune times every candidate at a level and
// records the fastest in the context's tuning table, which launches read.
// ---------------------------------------------------------------------------

template <int V>
using IC = std::integral_constant<int, V>;

}  // namespace ckks
#include "cols_tc.cuh"
namespace ckks {

// Calls f(IC<TC>, IC<SL>, IC<TP>) for a shape's compile-time parameters.
template <class F>
static bool with_shape(const ColShape& s, F f) {
  auto sl_tp = [&](auto tc) {
    switch (s.sl * 4 + s.tp) {
      case 2 * 4 + 1: f(tc, IC<2>{}, IC<1>{}); return true;
      case 4 * 4 + 1: f(tc, IC<4>{}, IC<1>{}); return true;
      case 8 * 4 + 1: f(tc, IC<8>{}, IC<1>{}); return true;
      case 2 * 4 + 2: f(tc, IC<2>{}, IC<2>{}); return true;
      case 4 * 4 + 2: f(tc, IC<4>{}, IC<2>{}); return true;
      case 8 * 4 + 2: f(tc, IC<8>{}, IC<2>{}); return true;
      default: return false;
    }
  };
  if (s.tc == 8) return sl_tp(IC<8>{});
  if (s.tc == 4) return sl_tp(IC<4>{});
  return false;
}

// Default shape: 8 columns (32-byte row segments) when that already gives
// two blocks per SM, else 4 to double the block count; four slices; no split.
template <class G>
static ColShape default_shape(int blocks_per_tile_column, int sms) {
  ColShape s;
  s.tc = ((G::W / 8) * blocks_per_tile_column >= 2 * sms || G::W / 4 < 16) ? 8 : 4;
  s.sl = 4;
  s.z = 1;
  s.tp = 1;
  return s;
}

// A shape is launchable when the tile width divides the row, a slice is a
// whole number of warps (each slice synchronizes its transposes with a named
// barrier, whose thread count must be a multiple of the warp size) and the
// parameters are among the compiled ones.
template <class G>
static bool tc_shape_ok(const ColShape& s);

template <class G>
static bool shape_ok(const ColShape& s) {
  if (s.tp == 8 || s.tp == 16) return tc_shape_ok<G>(s);
  return (s.tc == 4 || s.tc == 8) && G::W % s.tc == 0 && (s.tc * G::EC) % 32 == 0 &&
         (s.sl == 2 || s.sl == 4 || s.sl == 8) && s.z >= 1 && s.z <= 4 && (s.tp == 1 || s.tp == 2);
}

template <class G>
static ColShape pick_shape(const Scratch& sc, ColKernel k, int n, const ColShape& def) {
  if (sc.tune) {
    const ColShape s = sc.tune->get(k, n);
    if (s.valid() && shape_ok<G>(s)) return s;
  }
  return def;
}


template <class G>
void launch_modup_cols(const DevParams& dp, int n, int base, int tix, int digits, const Scratch& sc,
                       const ColShape& s0, cudaStream_t st) {
  if (is_tc_shape(s0) && dp.ks.tc_img && dp.alpha <= kTcMaxSources &&
      with_tc_shape<G>(s0, [&](auto tc, auto sl, auto nc) {
        constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, NC = decltype(nc)::value;
        using SH = TcShape<G, TC, SL, NC>;
        int mmax = 0;
        for (int j = 0; j < digits; ++j) {
          const int g = base / dp.alpha + j;
          const int k = std::min(n, (g + 1) * dp.alpha - base) - std::max(0, g * dp.alpha - base);
          mmax = std::max(mmax, n + dp.alpha - k);
        }
        const int kr = tc_kr(dp.alpha);
        const size_t sm = tc_smem<SH, NC>(kr, mmax).total;
        set_col_smem((const void*)k_ks_modup_cols_tc<G, TC, SL, NC>, sm);
        launch_pdl(dp.pdl, k_ks_modup_cols_tc<G, TC, SL, NC>, dim3(G::W / TC, digits), dim3(SH::NT), sm, st, dp, n,
                   base, tix, kr, mmax, (const uint32_t*)sc.S, sc.T);
        count_launch(1);
      }))
    return;
  const ColShape s = is_tc_shape(s0) ? default_shape<G>(digits, dp.sms) : s0;
  with_shape(s, [&](auto tc, auto sl, auto tp) {
    constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, TP = decltype(tp)::value;
    const size_t sm = col_smem_bytes<G, TC, SL>(dp.alpha);
    set_col_smem((const void*)k_ks_modup_cols<G, TC, SL, TP>, sm);
    launch_pdl(dp.pdl, k_ks_modup_cols<G, TC, SL, TP>, dim3(G::W / TC, digits, s.z), dim3(SL * ColTile<G, TC>::CT), sm, st,
               dp, n, base, tix, (const uint32_t*)sc.S, sc.T);
    count_launch(1);
  });
}

template <class G>
void launch_moddown_cols(const DevParams& dp, int n, int base, int tix, const Scratch& sc, const ColShape& s0,
                         cudaStream_t st) {
  if (is_tc_shape(s0) && dp.ks.tc_img && dp.alpha <= kTcMaxSources &&
      with_tc_shape<G>(s0, [&](auto tc, auto sl, auto nc) {
        constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, NC = decltype(nc)::value;
        using SH = TcShape<G, TC, SL, NC>;
        const int kr = tc_kr(dp.alpha);
        const size_t sm = tc_smem<SH, NC>(kr, n).total;
        set_col_smem((const void*)k_ks_moddown_cols_tc<G, TC, SL, NC>, sm);
        launch_pdl(dp.pdl, k_ks_moddown_cols_tc<G, TC, SL, NC>, dim3(G::W / TC, 2), dim3(SH::NT), sm, st, dp, n, base,
                   tix, kr, (const uint32_t*)sc.S, sc.T);
        count_launch(1);
      }))
    return;
  const ColShape s = is_tc_shape(s0) ? default_shape<G>(2, dp.sms) : s0;
  with_shape(s, [&](auto tc, auto sl, auto tp) {
    constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, TP = decltype(tp)::value;
    const size_t sm = col_smem_bytes<G, TC, SL>(dp.alpha);
    set_col_smem((const void*)k_ks_moddown_cols<G, TC, SL, TP>, sm);
    launch_pdl(dp.pdl, k_ks_moddown_cols<G, TC, SL, TP>, dim3(G::W / TC, 2, s.z), dim3(SL * ColTile<G, TC>::CT), sm, st,
               dp, n, base, (const uint32_t*)sc.S, sc.T);
    count_launch(1);
  });
}

template <class G>
void launch_moddown_cols_top(const DevParams& dp, int n, const Scratch& sc, uint32_t* Y, cudaStream_t st) {
  ColShape s = default_shape<G>(2, dp.sms);
  with_shape(s, [&](auto tc, auto sl, auto) {
    constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value;
    const size_t sm = col_smem_bytes<G, TC, SL>(dp.alpha + 1);
    set_col_smem((const void*)k_ks_moddown_cols_top<G, TC, SL>, sm);
    launch_pdl(dp.pdl, k_ks_moddown_cols_top<G, TC, SL>, dim3(G::W / TC, 2), dim3(SL * ColTile<G, TC>::CT), sm, st, dp,
               n, (const uint32_t*)sc.S, Y);
    count_launch(1);
  });
}

template <class G>
void launch_rs_cols_fused(const DevParams& dp, int n, const Scratch& sc, uint32_t* T3, const ColShape& s0,
                          cudaStream_t st) {
  if (is_tc_shape(s0) && dp.ks.tc_img && dp.alpha + 1 <= kTcMaxSources &&
      with_tc_shape<G>(s0, [&](auto tc, auto sl, auto nc) {
        constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, NC = decltype(nc)::value;
        using SH = TcShape<G, TC, SL, NC>;
        // top limb first (its sources go through Y), then the conversion on
        // the tensor cores
        launch_moddown_cols_top<G>(dp, n, sc, sc.U, st);
        const int kr = tc_kr(dp.alpha + 1);
        const size_t sm = tc_smem<SH, NC>(kr, n - 1).total;
        set_col_smem((const void*)k_rs_cols_fused_tc<G, TC, SL, NC>, sm);
        launch_pdl(dp.pdl, k_rs_cols_fused_tc<G, TC, SL, NC>, dim3(G::W / TC, 2), dim3(SH::NT), sm, st, dp, n, kr,
                   (const uint32_t*)sc.U, T3);
        count_launch(1);
      }))
    return;
  const ColShape s = is_tc_shape(s0) ? default_shape<G>(2, dp.sms) : s0;
  with_shape(s, [&](auto tc, auto sl, auto tp) {
    constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, TP = decltype(tp)::value;
    const size_t sm = col_smem_bytes<G, TC, SL>(dp.alpha + 1);
    set_col_smem((const void*)k_rs_cols_fused<G, TC, SL, TP>, sm);
    launch_pdl(dp.pdl, k_rs_cols_fused<G, TC, SL, TP>, dim3(G::W / TC, 2, s.z), dim3(SL * ColTile<G, TC>::CT), sm, st, dp,
               n, (const uint32_t*)sc.S, T3);
    count_launch(1);
  });
}

template <class G>
void launch_mm_cols(const DevParams& dp, const MmArgs& m, const Scratch& sc, const ColShape& s0, cudaStream_t st) {
  const ColShape s = is_tc_shape(s0) ? default_shape<G>(2, dp.sms) : s0;
  with_shape(s, [&](auto tc, auto sl, auto tp) {
    constexpr int TC = decltype(tc)::value, SL = decltype(sl)::value, TP = decltype(tp)::value;
    const size_t sm = col_smem_bytes<G, TC, SL>(m.K);
    set_col_smem((const void*)k_mm_cols<G, TC, SL, TP>, sm);
    launch_pdl(dp.pdl, k_mm_cols<G, TC, SL, TP>, dim3(G::W / TC, 2, s.z), dim3(SL * ColTile<G, TC>::CT), sm, st, dp,
               m, (const uint32_t*)sc.S, sc.T);
    count_launch(1);
  });
}


// Rational rescaling, column kernel (Sec. 3.1, Sec. 5.1): the K dropped
// limbs (row-phase iNTT already applied, S = [K][2]) finish their iNTT
// columns and are scaled by N^-1 [T_add (T_drop/d_k)^-1]_{d_k}; BConv (Eq. 2,
// centered) to every prime of the new window, then the NTT columns into
// T = [2][n1]. grid (W/TC, 2 polys), block SL * CT.
template <class G, int TC, int SL>
__global__ void __launch_bounds__(SL* ColTile<G, TC>::CT) k_rr_cols(DevParams dp, RrArgs r, const uint32_t* S,
                                                                    uint32_t* T) {
  pdl_wait();
  pdl_trigger();
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int u = blockIdx.y;
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)r.K * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  col_inputs<G, TC>(dp, S + ((size_t)u << dp.log_n), (size_t)2 << dp.log_n, r.K, 0, r.cin, y4, colbuf, l, jj, c,
                    pos, slice, SL, nullptr, r.drop);
  __syncthreads();
  auto tgt = [&](int i, const int32_t*& row, int& id, uint32_t*& dst) {
    row = r.mat + i * r.K;
    id = r.s1 + i;
    dst = T + ((size_t)(u * r.n1 + i) << dp.log_n);
  };
  col_targets<G, TC, 1>(dp, y4, r.K, r.n1, slice, SL, tgt, colbuf, l, jj, c, pos, slice,
                        src_bound(dp, r.K, 0, r.drop));
}

template <class G>
void launch_rr_cols(const DevParams& dp, const RrArgs& r, const Scratch& sc, cudaStream_t st) {
  constexpr int TC = 8, SL = 4;
  const size_t sm = col_smem_bytes<G, TC, SL>(r.K);
  set_col_smem((const void*)k_rr_cols<G, TC, SL>, sm);
  launch_pdl(dp.pdl, k_rr_cols<G, TC, SL>, dim3(G::W / TC, 2), dim3(SL * ColTile<G, TC>::CT), sm, st, dp, r,
             (const uint32_t*)sc.S, sc.T);
  count_launch(1);
}

}  // namespace ckks
