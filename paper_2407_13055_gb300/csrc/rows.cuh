// Row phase of the NTT / iNTT as standalone kernels over a list of limbs.
//
// Each warp-group of ER threads owns one row of W = ER^2 words. All global
// loads a thread needs (its row elements and the twiddles of its second
// register pass, which are specific to the thread) are issued before the
// first butterfly, so a warp waits for memory once instead of once per stage.
#pragma once
#include <type_traits>

#include "geo.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tc.cuh"

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
  int tail = 1 << 30, tail_prime = 0;  // launch limbs y >= tail: (y, tail_prime)
  __device__ __forceinline__ int2 operator()(int y) const {
    if (y >= tail) return make_int2(y, tail_prime);
    if (tab) return tab[y];
    const int u = y / pl, r = y % pl;
    const int t = (first + r) % per;
    return make_int2(u * ps + first + r, fixed >= 0 ? fixed : (t < n ? base + t : L + (t - n)));
  }
};

// Epilogues that read operands after the transform may name them up front
// (a method prefetch(dp, y, pos0)): the row kernel asks for them to be moved
// into L2 before it starts its passes, so the epilogue's loads find them there.
template <class Epi, class = void>
struct HasPrefetch : std::false_type {};
template <class Epi>
struct HasPrefetch<Epi, std::void_t<decltype(&Epi::prefetch)>> : std::true_type {};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

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

// ---------------------------------------------------------------------------
// Rows of W = 1024 words (N = 2^16) in three register passes of 4, 3 and 3
// stages on 64 threads per row, 16 values per thread, so that a thread keeps
// 16 values and 21 twiddle pairs (7 shared by its pass-B groups, 14 for its
// two pass-C groups) instead of 32 values and 31 pairs: twice the resident
// warps of the two-pass form. Element e of the row (0 .. 1023) sits at
//   A layout (pass A):  thread t, value i < 16:         e = t + 64 i
//   B layout (pass B):  thread t, group g < 2, i < 8:   e = 64 (t >> 2) + 8 i + 2 (t & 3) + g
//   C layout (pass C):  thread t, group g < 2, i < 8:   e = 16 t + 8 g + i
// so the row's forward output (C layout) is the same B-layout run of 16
// consecutive words per thread that the epilogues expect. Forward stage k
// (0 .. 9 of the row) uses twiddle (H + h) 2^k + (e >> (10 - k)); pass A's
// 15 depend on the row only and are staged in shared memory, pass B's on
// o = t >> 2 (base (H + h) 16 + o), pass C's on the group (base (H + h) 128
// + 2 t + g). Launch bounds of 6 blocks of 4 warps per SM (80 registers):
// 24 resident warps, against 16 for the two-pass form at 128 registers.
// Transposes go through one 1024-word buffer per row with an XOR
// swizzle of the bank bits by bits 5-8 of e, conflict-free for the three
// access patterns (32 consecutive e; fixed i, g over a warp in B; fixed i
// over a warp in C).
// ---------------------------------------------------------------------------

__device__ __forceinline__ int row3_swz(int e) {
  const int b5 = (e >> 5) & 1, b6 = (e >> 6) & 1, b7 = (e >> 7) & 1, b8 = (e >> 8) & 1;
  return e ^ ((b8 << 4) | (b7 << 3) | (b5 << 2) | (b8 << 1) | b6);
}
__device__ __forceinline__ int row3_eb(int t, int g, int i) { return 64 * (t >> 2) + 8 * i + 2 * (t & 3) + g; }

// Pass-B and pass-C twiddles of thread t in row h: local stage s, block b at
// entry (2^s - 1) + b, global index base 2^s + b.
template <int H>
__device__ __forceinline__ void row3_load_twiddles(uint2 (&tb)[7], uint2 (&tc)[2][7], const uint2* __restrict__ t,
                                                   int h, int tid) {
  const uint32_t bb = (uint32_t)(H + h) * 16 + (tid >> 2);
  tb[0] = __ldg(t + bb);
  {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + 2 * bb));
    tb[1] = make_uint2(v.x, v.y);
    tb[2] = make_uint2(v.z, v.w);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + 4 * bb) + k);
    tb[3 + 2 * k] = make_uint2(v.x, v.y);
    tb[4 + 2 * k] = make_uint2(v.z, v.w);
  }
  // pass C: the two groups' blocks are adjacent, so each stage is one run
  const uint32_t bc = (uint32_t)(H + h) * 128 + 2 * tid;
  {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + bc));
    tc[0][0] = make_uint2(v.x, v.y);
    tc[1][0] = make_uint2(v.z, v.w);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {  // stage 1: entries 2 bc + 2 g + b
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + 2 * bc) + k);
    tc[k][1] = make_uint2(v.x, v.y);
    tc[k][2] = make_uint2(v.z, v.w);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // stage 2: entries 4 bc + 4 g + b
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + 4 * bc) + k);
    tc[k >> 1][3 + 2 * (k & 1)] = make_uint2(v.x, v.y);
    tc[k >> 1][4 + 2 * (k & 1)] = make_uint2(v.z, v.w);
  }
}

// Pass-A twiddles of row h (15 entries, shared by its 64 threads).
template <int H>
__device__ __forceinline__ void row3_stage_a(uint2* sm, const uint2* __restrict__ t, int h, int tid) {
  if (tid < 15) {
    const int s = 31 - __clz(tid + 1);
    const int b = tid + 1 - (1 << s);
    sm[tid] = __ldg(t + ((uint32_t)(H + h) << s) + b);
  }
}

template <class G, class Epi>
__global__ void __launch_bounds__(128, 6) k_rows3_fwd_t(DevParams dp, const uint32_t* src, Epi epi, LimbMap map) {
  static_assert(G::W == 1024, "three-pass rows are for W = 1024");
  __shared__ uint32_t buf[2][1024];
  __shared__ uint2 twa[2][15];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int h = blockIdx.x * 2 + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  const uint2* tw = dp.tw + ((size_t)lm.y << dp.log_n);
  uint2 tb[7], tc[2][7];
  row3_load_twiddles<G::H>(tb, tc, tw, h, t);
  row3_stage_a<G::H>(twa[r], tw, h, t);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  if constexpr (HasPrefetch<Epi>::value) epi.prefetch(dp, (int)blockIdx.y, (uint32_t)(h * 1024 + 16 * t));
  const uint32_t* s = src + ((size_t)lm.x << dp.log_n) + (size_t)h * 1024;
  uint32_t x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = s[t + 64 * i];
  uint32_t* b = buf[r];
  uint32_t y0[8], y1[8];
  if (q < (1u << 30)) ct_pass_sm<16, true>(x, twa[r], q);
  else ct_pass_sm<16, false>(x, twa[r], q);
#pragma unroll
  for (int i = 0; i < 16; ++i) b[row3_swz(t + 64 * i)] = x[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(row3_eb(t, 0, i))];
    y1[i] = b[row3_swz(row3_eb(t, 1, i))];
  }
  __syncthreads();
  if (q < (1u << 30)) {
    ct_pass_reg<8, true>(y0, tb, q);
    ct_pass_reg<8, true>(y1, tb, q);
  } else {
    ct_pass_reg<8, false>(y0, tb, q);
    ct_pass_reg<8, false>(y1, tb, q);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(row3_eb(t, 0, i))] = y0[i];
    b[row3_swz(row3_eb(t, 1, i))] = y1[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(16 * t + i)];
    y1[i] = b[row3_swz(16 * t + 8 + i)];
  }
  if (q < (1u << 30)) {
    ct_pass_reg<8, true>(y0, tc[0], q);
    ct_pass_reg<8, true>(y1, tc[1], q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = normalize<true>(y0[i], q);
      x[8 + i] = normalize<true>(y1[i], q);
    }
  } else {
    ct_pass_reg<8, false>(y0, tc[0], q);
    ct_pass_reg<8, false>(y1, tc[1], q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = normalize<false>(y0[i], q);
      x[8 + i] = normalize<false>(y1[i], q);
    }
  }
  epi(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * 1024 + 16 * t));
}

template <class G, class Src>
__global__ void __launch_bounds__(128, 6) k_rows3_inv_t(DevParams dp, Src src, uint32_t* dst, LimbMap map,
                                                     int dst_compact) {
  static_assert(G::W == 1024, "three-pass rows are for W = 1024");
  __shared__ uint32_t buf[2][1024];
  __shared__ uint2 twa[2][15];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int h = blockIdx.x * 2 + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  const uint2* itw = dp.itw + ((size_t)lm.y << dp.log_n);
  uint2 tb[7], tc[2][7];
  row3_load_twiddles<G::H>(tb, tc, itw, h, t);
  row3_stage_a<G::H>(twa[r], itw, h, t);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  uint32_t x[16];
  src(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * 1024 + 16 * t));
  uint32_t* b = buf[r];
  uint32_t y0[8], y1[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = x[i];
    y1[i] = x[8 + i];
  }
  if (q < (1u << 30)) {
    gs_pass_reg<8, true>(y0, tc[0], q);
    gs_pass_reg<8, true>(y1, tc[1], q);
  } else {
    gs_pass_reg<8, false>(y0, tc[0], q);
    gs_pass_reg<8, false>(y1, tc[1], q);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(16 * t + i)] = y0[i];
    b[row3_swz(16 * t + 8 + i)] = y1[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(row3_eb(t, 0, i))];
    y1[i] = b[row3_swz(row3_eb(t, 1, i))];
  }
  __syncthreads();
  if (q < (1u << 30)) {
    gs_pass_reg<8, true>(y0, tb, q);
    gs_pass_reg<8, true>(y1, tb, q);
  } else {
    gs_pass_reg<8, false>(y0, tb, q);
    gs_pass_reg<8, false>(y1, tb, q);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(row3_eb(t, 0, i))] = y0[i];
    b[row3_swz(row3_eb(t, 1, i))] = y1[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = b[row3_swz(t + 64 * i)];
  if (q < (1u << 30)) gs_pass_sm<16, true>(x, twa[r], q);
  else gs_pass_sm<16, false>(x, twa[r], q);
  const size_t dl = dst_compact ? (size_t)blockIdx.y : (size_t)lm.x;
  uint32_t* o = dst + (dl << dp.log_n) + (size_t)h * 1024;
#pragma unroll
  for (int i = 0; i < 16; ++i) o[t + 64 * i] = x[i];
}

// ---------------------------------------------------------------------------
// Three-pass rows with the twiddles in shared memory. The same passes, layouts
// and twiddle indices as k_rows3_fwd_t / k_rows3_inv_t, but the pass-B and
// pass-C twiddles (21 pairs per thread, 42 registers there) are copied into
// shared memory with asynchronous copies (cp.async: no registers, the copies
// land while the thread loads its row and runs its first pass) and read from
// there at each stage. A thread then keeps little more than its 16 values, so
// the kernel fits 8 blocks of 4 warps per SM (64 registers, 25 KB of shared
// memory per block): 32 resident warps against 24.
// Layouts per row: pass A as before (15 pairs, entry (2^s - 1) + b); pass B per
// group o = t >> 2, entry (1 << s) + b (entry 0 unused), 10 entries per group
// so that the 8 groups of a warp fall in distinct banks; pass C per thread as
// 7 16-byte pairs in pair-major order (pair p of thread t at [p][t]): pair 0 =
// stage 0 of groups 0 and 1, pairs 1 + g = stage 1 of group g, pairs 3 + 2g and
// 4 + 2g = stage 2 of group g (blocks 0-1 and 2-3), each read as one 16-byte
// word by the thread, conflict-free across the warp.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct Row3Tw {
  uint2 a[2][15];        // pass A, per row
  uint2 b[2][16][10];    // pass B, per row and group o
  uint4 c[2][7][64];     // pass C, per row, pair, thread
};

// Copies of thread t of row r (row h of the limb's table t): pass A by the
// first 15 threads, pass B by the four threads of each group (one stage part
// each), pass C by every thread (its own 7 pairs). Two commit groups: pass A,
// then passes B and C (order `a_first`), or pass C then passes B and A.
template <int H>
__device__ __forceinline__ void row3s_copy_twiddles(Row3Tw& sw, const uint2* __restrict__ tw, int r, int h, int t,
                                                    bool a_first) {
  auto copy_a = [&]() {
    if (t < 15) {
      const int s = 31 - __clz(t + 1);
      const int b = t + 1 - (1 << s);
      cp_async8(&sw.a[r][t], tw + ((uint32_t)(H + h) << s) + b);
    }
  };
  auto copy_b = [&]() {
    const int o = t >> 2, part = t & 3;
    const uint32_t bb = (uint32_t)(H + h) * 16 + o;
    if (part == 0) cp_async8(&sw.b[r][o][1], tw + bb);
    else if (part == 1) cp_async16(&sw.b[r][o][2], tw + 2 * bb);
    else cp_async16(&sw.b[r][o][4 + 2 * (part - 2)], tw + 4 * bb + 2 * (part - 2));
  };
  auto copy_c = [&]() {
    const uint32_t bc = (uint32_t)(H + h) * 128 + 2 * t;
    cp_async16(&sw.c[r][0][t], tw + bc);
#pragma unroll
    for (int k = 0; k < 2; ++k) cp_async16(&sw.c[r][1 + k][t], tw + 2 * bc + 2 * k);
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async16(&sw.c[r][3 + k][t], tw + 4 * bc + 2 * k);
  };
  if (a_first) {
    copy_a();
    cp_async_commit();
    copy_b();
    copy_c();
  } else {
    copy_c();
    cp_async_commit();
    copy_b();
    copy_a();
  }
  cp_async_commit();
}

// Pass B on both groups, twiddle of stage s, block b at w[(1 << s) + b].
template <bool LAZY>
__device__ __forceinline__ void row3s_ct_b(uint32_t (&y0)[8], uint32_t (&y1)[8], const uint2* w, uint32_t q) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int half = 8 >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 tw = w[(1 << s) + b];
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        ct_bfly<LAZY>(y0[i0], y0[i0 + half], tw.x, tw.y, q);
        ct_bfly<LAZY>(y1[i0], y1[i0 + half], tw.x, tw.y, q);
      }
    }
  }
}

template <bool LAZY>
__device__ __forceinline__ void row3s_gs_b(uint32_t (&y0)[8], uint32_t (&y1)[8], const uint2* w, uint32_t q) {
#pragma unroll
  for (int s = 2; s >= 0; --s) {
    const int half = 8 >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 tw = w[(1 << s) + b];
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        gs_bfly<LAZY>(y0[i0], y0[i0 + half], tw.x, tw.y, q);
        gs_bfly<LAZY>(y1[i0], y1[i0 + half], tw.x, tw.y, q);
      }
    }
  }
}

// Twiddle pair of group g, stage s, block b from the thread's pass-C pairs
// (c[p * 64] = pair p).
__device__ __forceinline__ uint2 row3s_c_tw(const uint4* c, int g, int s, int b) {
  const uint4 v = s == 0 ? c[0] : s == 1 ? c[(1 + g) * 64] : c[(3 + 2 * g + (b >> 1)) * 64];
  const bool hi = s == 0 ? g == 1 : (b & 1) == 1;
  return hi ? make_uint2(v.z, v.w) : make_uint2(v.x, v.y);
}

template <bool LAZY>
__device__ __forceinline__ void row3s_ct_c(uint32_t (&y0)[8], uint32_t (&y1)[8], const uint4* c, uint32_t q) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int half = 8 >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w0 = row3s_c_tw(c, 0, s, b), w1 = row3s_c_tw(c, 1, s, b);
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        ct_bfly<LAZY>(y0[i0], y0[i0 + half], w0.x, w0.y, q);
        ct_bfly<LAZY>(y1[i0], y1[i0 + half], w1.x, w1.y, q);
      }
    }
  }
}

template <bool LAZY>
__device__ __forceinline__ void row3s_gs_c(uint32_t (&y0)[8], uint32_t (&y1)[8], const uint4* c, uint32_t q) {
#pragma unroll
  for (int s = 2; s >= 0; --s) {
    const int half = 8 >> (s + 1);
#pragma unroll
    for (int b = 0; b < (1 << s); ++b) {
      const uint2 w0 = row3s_c_tw(c, 0, s, b), w1 = row3s_c_tw(c, 1, s, b);
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = b * 2 * half + k;
        gs_bfly<LAZY>(y0[i0], y0[i0 + half], w0.x, w0.y, q);
        gs_bfly<LAZY>(y1[i0], y1[i0 + half], w1.x, w1.y, q);
      }
    }
  }
}

template <class G, class Epi>
__global__ void __launch_bounds__(128, 8) k_rows3s_fwd_t(DevParams dp, const uint32_t* src, Epi epi, LimbMap map) {
  static_assert(G::W == 1024, "three-pass rows are for W = 1024");
  __shared__ uint32_t buf[2][1024];
  __shared__ __align__(16) Row3Tw sw;
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int h = blockIdx.x * 2 + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  row3s_copy_twiddles<G::H>(sw, dp.tw + ((size_t)lm.y << dp.log_n), r, h, t, true);
  pdl_wait();
  pdl_trigger();
  const uint32_t* s = src + ((size_t)lm.x << dp.log_n) + (size_t)h * 1024;
  uint32_t x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = s[t + 64 * i];
  cp_async_wait<1>();
  __syncthreads();
  uint32_t* b = buf[r];
  uint32_t y0[8], y1[8];
  const bool lazy = q < (1u << 30);
  if (lazy) ct_pass_sm<16, true>(x, sw.a[r], q);
  else ct_pass_sm<16, false>(x, sw.a[r], q);
#pragma unroll
  for (int i = 0; i < 16; ++i) b[row3_swz(t + 64 * i)] = x[i];
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(row3_eb(t, 0, i))];
    y1[i] = b[row3_swz(row3_eb(t, 1, i))];
  }
  __syncthreads();
  const uint2* wb = sw.b[r][t >> 2];
  if (lazy) row3s_ct_b<true>(y0, y1, wb, q);
  else row3s_ct_b<false>(y0, y1, wb, q);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(row3_eb(t, 0, i))] = y0[i];
    b[row3_swz(row3_eb(t, 1, i))] = y1[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(16 * t + i)];
    y1[i] = b[row3_swz(16 * t + 8 + i)];
  }
  const uint4* wc = &sw.c[r][0][t];
  if (lazy) {
    row3s_ct_c<true>(y0, y1, wc, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = normalize<true>(y0[i], q);
      x[8 + i] = normalize<true>(y1[i], q);
    }
  } else {
    row3s_ct_c<false>(y0, y1, wc, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = normalize<false>(y0[i], q);
      x[8 + i] = normalize<false>(y1[i], q);
    }
  }
  epi(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * 1024 + 16 * t));
}

template <class G, class Src>
__global__ void __launch_bounds__(128, 8) k_rows3s_inv_t(DevParams dp, Src src, uint32_t* dst, LimbMap map,
                                                      int dst_compact) {
  static_assert(G::W == 1024, "three-pass rows are for W = 1024");
  __shared__ uint32_t buf[2][1024];
  __shared__ __align__(16) Row3Tw sw;
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int h = blockIdx.x * 2 + r;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  row3s_copy_twiddles<G::H>(sw, dp.itw + ((size_t)lm.y << dp.log_n), r, h, t, false);
  pdl_wait();
  pdl_trigger();
  uint32_t x[16];
  src(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * 1024 + 16 * t));
  uint32_t* b = buf[r];
  uint32_t y0[8], y1[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = x[i];
    y1[i] = x[8 + i];
  }
  const bool lazy = q < (1u << 30);
  cp_async_wait<1>();  // own pass-C pairs (read by this thread only)
  const uint4* wc = &sw.c[r][0][t];
  if (lazy) row3s_gs_c<true>(y0, y1, wc, q);
  else row3s_gs_c<false>(y0, y1, wc, q);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(16 * t + i)] = y0[i];
    b[row3_swz(16 * t + 8 + i)] = y1[i];
  }
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    y0[i] = b[row3_swz(row3_eb(t, 0, i))];
    y1[i] = b[row3_swz(row3_eb(t, 1, i))];
  }
  __syncthreads();
  const uint2* wb = sw.b[r][t >> 2];
  if (lazy) row3s_gs_b<true>(y0, y1, wb, q);
  else row3s_gs_b<false>(y0, y1, wb, q);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[row3_swz(row3_eb(t, 0, i))] = y0[i];
    b[row3_swz(row3_eb(t, 1, i))] = y1[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = b[row3_swz(t + 64 * i)];
  if (lazy) gs_pass_sm<16, true>(x, sw.a[r], q);
  else gs_pass_sm<16, false>(x, sw.a[r], q);
  const size_t dl = dst_compact ? (size_t)blockIdx.y : (size_t)lm.x;
  uint32_t* o = dst + (dl << dp.log_n) + (size_t)h * 1024;
#pragma unroll
  for (int i = 0; i < 16; ++i) o[t + 64 * i] = x[i];
}

// Three-pass forward rows with the input staged by bulk copies: a block
// takes RP consecutive row pairs of one limb; the next pairs' 8 KB of input
// (two contiguous rows) stream into a second shared buffer with
// cp.async.bulk (one thread issues, an mbarrier counts the bytes) while the
// current pair is transformed, so the loads' latency overlaps the
// arithmetic. The staging buffer of a pair also holds its transposes. Every
// wait is bounded by dp.wait_limit (expired: status word, the block stops
// after draining its own copies). In-place use (src == the epilogue's
// destination) is safe: a block reads and writes only its own rows.
template <class G, class Epi, int RP>
__global__ void __launch_bounds__(128, 5) k_rows3_fwd_bulk(DevParams dp, const uint32_t* src, Epi epi, LimbMap map) {
  static_assert(G::W == 1024, "three-pass rows are for W = 1024");
  __shared__ __align__(128) uint32_t buf[2][2][1024];
  __shared__ uint2 twa[2][15];
  __shared__ __align__(8) uint64_t bar[2];
  const int r = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int2 lm = map(blockIdx.y);
  const uint32_t q = dp.pc[lm.y].q;
  const uint2* tw = dp.tw + ((size_t)lm.y << dp.log_n);
  const uint32_t* s0 = src + ((size_t)lm.x << dp.log_n);
  const int pair0 = blockIdx.x * RP;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar[0]), 1);
    tc::mbar_init(tc::smem_u32(&bar[1]), 1);
    tc::mbar_init_fence();
  }
  uint2 tb[7], tc_[2][7];
  row3_load_twiddles<G::H>(tb, tc_, tw, 2 * pair0 + r, t);
  row3_stage_a<G::H>(twa[r], tw, 2 * pair0 + r, t);
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  uint32_t issued = 0;  // thread 0: copies issued (pair k goes to buffer k & 1)
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2 && k < RP; ++k) {
      const uint32_t b = tc::smem_u32(&bar[k]);
      tc::mbar_expect_tx(b, 8192);
      tc::bulk_g2s(tc::smem_u32(buf[k]), s0 + (size_t)(pair0 + k) * 2048, 8192, b);
      ++issued;
    }
  }
  uint32_t waited = 0;
  for (int k = 0; k < RP; ++k) {
    const int h = 2 * (pair0 + k) + r;
    if (k > 0) {
      row3_load_twiddles<G::H>(tb, tc_, tw, h, t);
      row3_stage_a<G::H>(twa[r], tw, h, t);
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&bar[k & 1]), (uint32_t)((k >> 1) & 1), dp.wait_limit);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) tc::report_timeout(dp.status);
      break;
    }
    ++waited;
    uint32_t* b = buf[k & 1][r];
    uint32_t x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = b[t + 64 * i];
    uint32_t y0[8], y1[8];
    if (q < (1u << 30)) ct_pass_sm<16, true>(x, twa[r], q);
    else ct_pass_sm<16, false>(x, twa[r], q);
    __syncthreads();  // every thread read its input before the transposes overwrite it
#pragma unroll
    for (int i = 0; i < 16; ++i) b[row3_swz(t + 64 * i)] = x[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      y0[i] = b[row3_swz(row3_eb(t, 0, i))];
      y1[i] = b[row3_swz(row3_eb(t, 1, i))];
    }
    __syncthreads();
    if (q < (1u << 30)) {
      ct_pass_reg<8, true>(y0, tb, q);
      ct_pass_reg<8, true>(y1, tb, q);
    } else {
      ct_pass_reg<8, false>(y0, tb, q);
      ct_pass_reg<8, false>(y1, tb, q);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      b[row3_swz(row3_eb(t, 0, i))] = y0[i];
      b[row3_swz(row3_eb(t, 1, i))] = y1[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      y0[i] = b[row3_swz(16 * t + i)];
      y1[i] = b[row3_swz(16 * t + 8 + i)];
    }
    // the buffer and the pass-A twiddles are free once every thread has read
    // them: the next copy into this buffer may start
    tc::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0 && k + 2 < RP) {
      const uint32_t bb = tc::smem_u32(&bar[k & 1]);
      tc::mbar_expect_tx(bb, 8192);
      tc::bulk_g2s(tc::smem_u32(buf[k & 1]), s0 + (size_t)(pair0 + k + 2) * 2048, 8192, bb);
      ++issued;
    }
    if (q < (1u << 30)) {
      ct_pass_reg<8, true>(y0, tc_[0], q);
      ct_pass_reg<8, true>(y1, tc_[1], q);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        x[i] = normalize<true>(y0[i], q);
        x[8 + i] = normalize<true>(y1[i], q);
      }
    } else {
      ct_pass_reg<8, false>(y0, tc_[0], q);
      ct_pass_reg<8, false>(y1, tc_[1], q);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        x[i] = normalize<false>(y0[i], q);
        x[8 + i] = normalize<false>(y1[i], q);
      }
    }
    epi(dp, x, (int)blockIdx.y, lm, (uint32_t)(h * 1024 + 16 * t));
  }
  // after a timeout: let the copies still in flight land before the block's
  // shared memory is released
  if (threadIdx.x == 0)
    for (uint32_t k = waited; k < issued; ++k)
      tc::mbar_wait(tc::smem_u32(&bar[k & 1]), (k >> 1) & 1, 1ll << 32);
}

template <class G, class Epi>
inline void launch_rows_fwd(const DevParams& dp, const uint32_t* src, const Epi& epi, int limbs, LimbMap map,
                            cudaStream_t st) {
  if (limbs <= 0) return;
  bool three = false;
  if constexpr (G::W == 1024) {
    if (dp.rows_passes == 4 || dp.rows_passes == 5) {
      if (dp.rows_passes == 4)
        launch_pdl(dp.pdl, k_rows3_fwd_bulk<G, Epi, 2>, dim3(G::H / 4, limbs), dim3(128), 0, st, dp, src, epi, map);
      else
        launch_pdl(dp.pdl, k_rows3_fwd_bulk<G, Epi, 4>, dim3(G::H / 8, limbs), dim3(128), 0, st, dp, src, epi, map);
      three = true;
    } else if (dp.rows_passes == 6) {
      launch_pdl(dp.pdl, k_rows3s_fwd_t<G, Epi>, dim3(G::H / 2, limbs), dim3(128), 0, st, dp, src, epi, map);
      three = true;
    } else if (dp.rows_passes != 2) {
      launch_pdl(dp.pdl, k_rows3_fwd_t<G, Epi>, dim3(G::H / 2, limbs), dim3(128), 0, st, dp, src, epi, map);
      three = true;
    }
  }
  if (!three)
    launch_pdl(dp.pdl, k_rows_fwd_t<G, Epi>, dim3(G::H / G::RPC, limbs), dim3(G::RT), 0, st, dp, src, epi, map);
  count_launch(1);
}

template <class G, class Src>
inline void launch_rows_inv(const DevParams& dp, const Src& srcf, uint32_t* dst, int limbs, LimbMap map,
                            bool dst_compact, cudaStream_t st) {
  if (limbs <= 0) return;
  bool three = false;
  if constexpr (G::W == 1024) {
    if (dp.rows_passes == 6) {
      launch_pdl(dp.pdl, k_rows3s_inv_t<G, Src>, dim3(G::H / 2, limbs), dim3(128), 0, st, dp, srcf, dst, map,
                 dst_compact ? 1 : 0);
      three = true;
    } else if (dp.rows_passes != 2) {
      launch_pdl(dp.pdl, k_rows3_inv_t<G, Src>, dim3(G::H / 2, limbs), dim3(128), 0, st, dp, srcf, dst, map,
                 dst_compact ? 1 : 0);
      three = true;
    }
  }
  if (!three)
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
