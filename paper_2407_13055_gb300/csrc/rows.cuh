// Row phase of the NTT / iNTT as standalone kernels over a list of limbs.
//
// Each warp-group of ER threads owns one row of W = ER^2 words. All global
// loads a thread needs (its row elements and the twiddles of its second
// register pass, which are specific to the thread) are issued before the
// first butterfly, so a warp waits for memory once instead of once per stage.
#pragma once
#include "geo.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace ckks {

// Limb list of a row launch: launch index y -> (data limb index, prime id).
// Rule (no table): y = u * pl + r selects limb first + r of polynomial u,
// whose limbs start at data limb u * ps; that limb's extended index
// t = (first + r) % per is q_(base + t) for t < n, else p_(t - n) (base: the
// first prime of the level's window).
struct LimbMap {
  const int2* tab;  // explicit table, or null for the rule
  int first;
  int per, n, L;
  int pl = 1 << 30, ps = 0;
  int fixed = -1;   // >= 0: every limb uses this prime id
  int base = 0;
  __device__ __forceinline__ int2 operator()(int y) const {
    if (tab) return tab[y];
    const int u = y / pl, r = y % pl;
    const int t = (first + r) % per;
    return make_int2(u * ps + first + r, fixed >= 0 ? fixed : (t < n ? base + t : L + (t - n)));
  }
};

// Register-resident twiddles of one pass: tw[(1 << s) - 1 + b] for local
// stage s and block b (2^s blocks).
template <int E, bool LAZY>
__device__ __forceinline__ void ct_pass_reg(uint32_t (&x)[E], const uint2 (&tw)[E - 1], uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = 0; s < e; ++s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = tw[(1 << s) - 1 + b];
#pragma unroll
      for (int r = 0; r < half; ++r) {
        const int i0 = b * 2 * half + r;
        ct_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

template <int E, bool LAZY>
__device__ __forceinline__ void gs_pass_reg(uint32_t (&x)[E], const uint2 (&tw)[E - 1], uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = e - 1; s >= 0; --s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = tw[(1 << s) - 1 + b];
#pragma unroll
      for (int r = 0; r < half; ++r) {
        const int i0 = b * 2 * half + r;
        gs_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

// First-pass twiddles of row h (the same for every thread of the row):
// local stage s, block b uses index (H + h) 2^s + b; the row's ER threads
// stage them in the row's own shared slice at (2^s - 1) + b and sync with a
// warp barrier (a row never spans two warps).
template <int E, int H>
__device__ __forceinline__ void stage_row_twiddles(uint2* sm, const uint2* __restrict__ t, int h, int jj) {
  for (int idx = jj; idx < E - 1; idx += E) {
    const int s = 31 - __clz(idx + 1);
    const int b = idx + 1 - (1 << s);
    sm[idx] = __ldg(t + ((uint32_t)(H + h) << s) + b);
  }
  __syncwarp();
}

template <int E, bool LAZY>
__device__ __forceinline__ void ct_pass_sm(uint32_t (&x)[E], const uint2* sm, uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = 0; s < e; ++s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = sm[(1 << s) - 1 + b];
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        ct_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

template <int E, bool LAZY>
__device__ __forceinline__ void gs_pass_sm(uint32_t (&x)[E], const uint2* sm, uint32_t q) {
  constexpr int e = Log2<E>::v;
#pragma unroll
  for (int s = e - 1; s >= 0; --s) {
    const int half = E >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w = sm[(1 << s) - 1 + b];
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        gs_bfly<LAZY>(x[i0], x[i0 + half], w.x, w.y, q);
      }
    }
  }
}

// Second-pass twiddles of thread jj in row h: indices ((H + h) E + jj) 2^s + b,
// contiguous for each stage, so stages s >= 1 load with 16-byte vectors.
template <int E, int H>
__device__ __forceinline__ void load_pass_b_twiddles(uint2 (&tw)[E - 1], const uint2* __restrict__ t, int h,
                                                     int jj) {
  constexpr int e = Log2<E>::v;
  const uint32_t base = (uint32_t)(H + h) * E + jj;
  tw[0] = __ldg(t + base);
#pragma unroll
  for (int s = 1; s < e; ++s) {
    const uint4* p = reinterpret_cast<const uint4*>(t + (base << s));
#pragma unroll
    for (int b2 = 0; b2 < (1 << (s - 1)); ++b2) {
      const uint4 v = __ldg(p + b2);
      tw[(1 << s) - 1 + 2 * b2] = make_uint2(v.x, v.y);
      tw[(1 << s) + 2 * b2] = make_uint2(v.z, v.w);
    }
  }
}

// Where a forward row phase puts its results, and where an inverse row phase
// gets its inputs. A thread holds the E consecutive device positions
// pos0 .. pos0 + E - 1 of its row (B layout: pos0 = h W + E jj) of launch
// limb y, whose data limb and prime are lm = map(y). The plain forms store to
// / load from a limb array; the key-switch kernels supply fused ones (input
// preparation before the iNTT, ModDown and rescale epilogues after the NTT).
struct RowStore {
  uint32_t* dst;
  int compact;  // write launch limb y at dst + y N instead of at data limb lm.x
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2 lm,
                                             uint32_t pos0) const {
    const size_t dl = compact ? (size_t)y : (size_t)lm.x;
    store_vec<E>(dst + (dl << dp.log_n) + pos0, x);
  }
};

struct RowLoad {
  const uint32_t* src;
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int, int2 lm,
                                             uint32_t pos0) const {
    load_vec<E>(x, src + ((size_t)lm.x << dp.log_n) + pos0);
  }
};

// Forward row phase: src in A layout (column-phase output, natural
// positions); the epilogue receives the B-layout results normalized to
// [0, q). Launched with programmatic dependent launch: the twiddles are
// loaded before waiting for the previous kernel.
template <class G, class Epi>
__global__ void __launch_bounds__(G::RT) k_rows_fwd_t(DevParams dp, const uint32_t* src, Epi epi, LimbMap map) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  __shared__ uint2 twa[G::RPC * (G::ER - 1)];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  const uint2* tw = dp.tw + ((size_t)lm.y << dp.log_n);
  uint2 twb[G::ER - 1];
  load_pass_b_twiddles<G::ER, G::H>(twb, tw, h, jj);
  uint2* tr = twa + r * (G::ER - 1);
  stage_row_twiddles<G::ER, G::H>(tr, tw, h, jj);
  pdl_wait();
  pdl_trigger();
  const uint32_t* s = src + ((size_t)lm.x << dp.log_n) + (size_t)h * G::W;
  uint32_t x[G::ER];
#pragma unroll
  for (int i = 0; i < G::ER; ++i) x[i] = s[jj + G::ER * i];
  uint32_t* b = buf + r * G::ROWBUF;
  if (q < (1u << 30)) {
    ct_pass_sm<G::ER, true>(x, tr, q);
    row_a_to_b<G::ER>(x, b, jj);
    ct_pass_reg<G::ER, true>(x, twb, q);
#pragma unroll
    for (int i = 0; i < G::ER; ++i) x[i] = normalize<true>(x[i], q);
  } else {
    ct_pass_sm<G::ER, false>(x, tr, q);
    row_a_to_b<G::ER>(x, b, jj);
    ct_pass_reg<G::ER, false>(x, twb, q);
#pragma unroll
    for (int i = 0; i < G::ER; ++i) x[i] = normalize<false>(x[i], q);
  }
  epi(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * G::W + G::ER * jj));
}

// Inverse row phase: the source gives B-layout values in [0, q) (NTT domain);
// dst in A layout, lazy range [0, 2q) (the column phase that follows accepts
// it). dst_compact: write limb y at dst + y N instead of at data limb lm.x.
template <class G, class Src>
__global__ void __launch_bounds__(G::RT) k_rows_inv_t(DevParams dp, Src src, uint32_t* dst, LimbMap map,
                                                      int dst_compact) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  __shared__ uint2 twa[G::RPC * (G::ER - 1)];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  const uint2* itw = dp.itw + ((size_t)lm.y << dp.log_n);
  uint2 twb[G::ER - 1];
  load_pass_b_twiddles<G::ER, G::H>(twb, itw, h, jj);
  uint2* tr = twa + r * (G::ER - 1);
  stage_row_twiddles<G::ER, G::H>(tr, itw, h, jj);
  pdl_wait();
  pdl_trigger();
  uint32_t x[G::ER];
  src(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * G::W + G::ER * jj));
  uint32_t* b = buf + r * G::ROWBUF;
  if (q < (1u << 30)) {
    gs_pass_reg<G::ER, true>(x, twb, q);
    row_b_to_a<G::ER>(x, b, jj);
    gs_pass_sm<G::ER, true>(x, tr, q);
  } else {
    gs_pass_reg<G::ER, false>(x, twb, q);
    row_b_to_a<G::ER>(x, b, jj);
    gs_pass_sm<G::ER, false>(x, tr, q);
  }
  const size_t dl = dst_compact ? (size_t)blockIdx.y : (size_t)lm.x;
  uint32_t* o = dst + (dl << dp.log_n) + (size_t)h * G::W;
#pragma unroll
  for (int i = 0; i < G::ER; ++i) o[jj + G::ER * i] = x[i];
}

template <class G, class Epi>
inline void launch_rows_fwd(const DevParams& dp, const uint32_t* src, const Epi& epi, int limbs, LimbMap map,
                            cudaStream_t st) {
  if (limbs <= 0) return;
  launch_pdl(dp.pdl, k_rows_fwd_t<G, Epi>, dim3(G::H / G::RPC, limbs), dim3(G::RT), 0, st, dp, src, epi, map);
  count_launch(1);
}

template <class G, class Src>
inline void launch_rows_inv(const DevParams& dp, const Src& srcf, uint32_t* dst, int limbs, LimbMap map,
                            bool dst_compact, cudaStream_t st) {
  if (limbs <= 0) return;
  launch_pdl(dp.pdl, k_rows_inv_t<G, Src>, dim3(G::H / G::RPC, limbs), dim3(G::RT), 0, st, dp, srcf, dst, map,
             dst_compact ? 1 : 0);
  count_launch(1);
}

template <class G>
inline void launch_rows_g(const DevParams& dp, bool inverse, const uint32_t* src, uint32_t* dst, int limbs,
                          LimbMap map, bool dst_compact, cudaStream_t st) {
  if (inverse) launch_rows_inv<G>(dp, RowLoad{src}, dst, limbs, map, dst_compact, st);
  else launch_rows_fwd<G>(dp, src, RowStore{dst, dst_compact ? 1 : 0}, limbs, map, st);
}

}  // namespace ckks
