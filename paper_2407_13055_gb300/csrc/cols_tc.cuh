// Column kernels with the BConv on the tensor cores (tcgen05, kind::f16).
//
// The column phase of a ModSwitch (iNTT columns -> BConv, Eq. 2 -> NTT
// columns, Alg. 1) holds a tile of TC columns x H rows. Here the conversion
// of the whole tile to a chunk of NC targets is one exact matrix product
// (tc.cuh):
//   A (shared memory, M = the tile's TC*H coefficients in 128-row tiles,
//      K = 4 digits per source): balanced signed-byte digits of the centered
//      sources, written by the slices that finish the sources' iNTT columns;
//   B (shared memory, N = 4 planes per target): the conversion matrix with
//      the byte weights folded in, split into byte planes; built once per
//      context on the host and brought in with one bulk copy;
//   D (tensor memory, two buffers): four exact fp32 plane sums per output.
// All warps then read D (one TMEM lane = one coefficient), turn each output's
// four plane sums into its residue (one signed Montgomery reduction), and
// stage the residues in shared memory, from where the slices run each
// target's NTT columns as in the CUDA-core kernels. While the slices run the
// NTT columns of one chunk, the tensor core computes the next one.
//
// Every mbarrier wait is bounded by dp.wait_limit clock cycles. When one
// expires the block records the timeout in dp.status, stops its work, waits
// (bounded) for its own bulk copy and MMAs still in flight, frees its tensor
// memory and returns; the host reports CKKS_ETIMEOUT at the next
// synchronizing call.
#pragma once
#include "tc.cuh"

namespace ckks {

// Launch geometry of a tensor-core column block.
template <class G, int TC, int SL, int NC>
struct TcShape {
  static constexpr int EC = G::EC, H = G::H;
  static constexpr int CT = TC * EC;            // threads per slice
  static constexpr int NT = SL * CT;            // threads per block
  static constexpr int NW = NT / 32;            // warps per block
  static constexpr int TCH = TC * H;            // coefficients per tile
  static constexpr int MT = TCH / 128;          // 128-row M tiles
  static constexpr int BUF = (H + EC) * TC;     // words of one slice's column transpose buffer
  static constexpr uint32_t TMEM_COLS = 2u * MT * NC * 4;  // two buffers of MT x (NC targets x 4 planes)
  static_assert(TCH % 128 == 0, "a tile is a whole number of 128-row M tiles");
  static_assert(NT % 128 == 0, "the epilogue needs every TMEM lane quadrant covered by whole warps");
  static_assert(TMEM_COLS >= 32 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0,
                "tensor memory is allocated in powers of two up to 512 columns");
};

// K extent of the product for K sources: four digits each, in steps of 16
// (one kind::f16 instruction).
__host__ __device__ inline int tc_kr(int K) { return 16 * ((K + 3) / 4); }

// Largest source count of the tensor-core kernels (K extent 64).
constexpr int kTcMaxSources = 16;

// Shared-memory layout of a block (byte offsets), for K extent kr and at
// most mmax targets.
struct TcSmem {
  uint32_t a, b, r, cbuf, prm, bar, flag, slot, total;
};

template <class SH, int NC>
__host__ __device__ inline TcSmem tc_smem(int kr, int mmax) {
  TcSmem s;
  s.a = 0;
  s.b = s.a + (uint32_t)SH::MT * 128u * kr * 2u;
  s.r = s.b + 4u * (uint32_t)((mmax + 3) & ~3) * kr * 2u;
  s.cbuf = s.r + (uint32_t)NC * SH::TCH * 4u;
  s.prm = s.cbuf + (uint32_t)(SH::NT / SH::CT) * SH::BUF * 4u;
  s.bar = (s.prm + (uint32_t)mmax * 8u + 15u) & ~15u;
  s.flag = s.bar + 3u * 8u;
  s.slot = s.flag + 4u;
  s.total = s.slot + 12u;
  return s;
}

// Byte offset in A of coefficient ci (= row * TC + column of the tile) and
// source k: M tile ci / 128, row ci % 128 in core matrices of 8 rows x 16
// bytes (two sources' four fp16 digits per row), 8-row groups kr * 16 bytes
// apart.
__device__ __forceinline__ uint32_t tc_a_off(int ci, int k, int kr) {
  const int mt = ci >> 7, r = ci & 127;
  return (uint32_t)(mt * 128 * kr * 2 + (r >> 3) * (kr * 16) + (k >> 1) * 128 + (r & 7) * 16 + (k & 1) * 8);
}

constexpr long long kTcDrainLimit = 1ll << 32;  // cycles to wait for own copies / MMAs after a timeout

template <class G, int TC, int SL, int NC>
struct TcBlock {
  using SH = TcShape<G, TC, SL, NC>;
  uint8_t* sm;
  TcSmem lay;
  int kr;
  uint32_t tmem = 0;
  // thread 0: work in flight (bit 0: the plane copy; bit 1 + b: MMA buffer b)
  // and the last chunk committed to each buffer
  uint32_t pending = 0;
  int last0 = 0, last1 = 0;

  __device__ TcBlock(uint8_t* s, const TcSmem& l, int k) : sm(s), lay(l), kr(k) {}

  __device__ uint32_t bar(int i) const { return tc::smem_u32(sm + lay.bar + 8 * i); }  // 0: planes, 1/2: MMA buffers
  __device__ volatile int* flag() const { return reinterpret_cast<volatile int*>(sm + lay.flag); }
  __device__ uint32_t* colbuf(int slice) const {
    return reinterpret_cast<uint32_t*>(sm + lay.cbuf) + (size_t)slice * SH::BUF;
  }

  // Tensor memory, barriers, the plane copy, the targets' prime constants and
  // the zero digits of the unused source slots. Reads only the context's
  // tables, so it may run before the programmatic-dependent-launch wait.
  template <class Tgt>
  __device__ void begin(const DevParams& dp, const uint8_t* img, uint32_t img_bytes, int K, int M, Tgt target) {
    const int tid = threadIdx.x;
    if (tid < 32) tc::tmem_alloc(tc::smem_u32(sm + lay.slot), SH::TMEM_COLS);
    if (tid == 0) {
      for (int i = 0; i < 3; ++i) tc::mbar_init(bar(i), 1);
      tc::mbar_init_fence();
      *flag() = 0;
      tc::mbar_expect_tx(bar(0), img_bytes);
      tc::bulk_g2s(tc::smem_u32(sm + lay.b), img, img_bytes, bar(0));
      pending = 1;
    }
    uint2* prm = reinterpret_cast<uint2*>(sm + lay.prm);
    for (int m = tid; m < M; m += SH::NT) {
      int id;
      uint32_t* d;
      target(m, id, d);
      prm[m] = make_uint2(dp.pc[id].q, dp.pc[id].m);
    }
    const int slots = kr / 4 - K;
    for (int i = tid; i < slots * SH::TCH; i += SH::NT)
      *reinterpret_cast<uint2*>(sm + lay.a + tc_a_off(i % SH::TCH, K + i / SH::TCH, kr)) = make_uint2(0u, 0u);
  }

  // Digits of source k for the thread's EC coefficients (rows jj + EC i of
  // column c: the layout the column iNTT leaves).
  __device__ __forceinline__ void put(int k, const int32_t (&y)[G::EC], int jj, int c) const {
#pragma unroll
    for (int i = 0; i < G::EC; ++i)
      *reinterpret_cast<uint2*>(sm + lay.a + tc_a_off((jj + G::EC * i) * TC + c, k, kr)) = tc::digits_f16(y[i]);
  }

  // Thread 0: the MMAs of chunk ch (targets ch NC ..) into buffer ch & 1.
  __device__ void issue(int ch, int M) {
    const int bf = ch & 1, mc = min(NC, M - ch * NC), n = 4 * ((mc + 3) & ~3);
    const uint32_t id = tc::idesc_f16(128, n), sbo = (uint32_t)kr * 16u;
    const uint32_t a0 = tc::smem_u32(sm + lay.a), b0 = tc::smem_u32(sm + lay.b) + (uint32_t)(ch * NC * kr * 8);
#pragma unroll
    for (int mt = 0; mt < SH::MT; ++mt) {
      const uint32_t d = tmem + (uint32_t)((bf * SH::MT + mt) * NC * 4);
      for (int s = 0; s < kr / 16; ++s)
        tc::mma_f16(d, tc::sdesc(a0 + (uint32_t)(mt * 128 * kr * 2 + s * 256), 128, sbo),
                    tc::sdesc(b0 + (uint32_t)(s * 256), 128, sbo), id, s > 0);
    }
    tc::commit(bar(1 + bf));
    pending |= 2u << bf;
    if (bf) last1 = ch;
    else last0 = ch;
  }

  // Residues of chunk ch: warp w reads TMEM lane quadrant w % 4 (coefficients
  // mt * 128 + 32 (w % 4) + lane), the warps of a quadrant splitting the
  // chunk's targets in groups of four; R[t][ci] in shared memory.
  __device__ void epilogue(int ch, int M) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, qd = warp & 3;
    const int mc = min(NC, M - ch * NC), g4n = (mc + 3) >> 2;
    const uint32_t t0 = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)((ch & 1) * SH::MT * NC * 4);
    const uint2* prm = reinterpret_cast<const uint2*>(sm + lay.prm) + ch * NC;
    uint32_t* R = reinterpret_cast<uint32_t*>(sm + lay.r);
    for (int g4 = warp >> 2; g4 < g4n; g4 += SH::NW / 4) {
      uint32_t v[SH::MT][16];
#pragma unroll
      for (int mt = 0; mt < SH::MT; ++mt) tc::tmem_ld16(t0 + (uint32_t)(mt * NC * 4 + g4 * 16), v[mt]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int tg = g4 * 4 + t;
        if (tg >= mc) break;
        const uint2 qm = prm[tg];
#pragma unroll
        for (int mt = 0; mt < SH::MT; ++mt)
          R[tg * SH::TCH + mt * 128 + qd * 32 + lane] =
              tc::planes_residue(v[mt][4 * t], v[mt][4 * t + 1], v[mt][4 * t + 2], v[mt][4 * t + 3], qm.x, qm.y);
      }
    }
  }

  // After the sources: the chunks' products, residues and NTT columns.
  // target(m, id, dst): prime id and destination limb of target m.
  template <class Tgt>
  __device__ void convert(const DevParams& dp, int M, Tgt target, int l, int jj, int c, int slice) {
    const int tid = threadIdx.x, lane = tid & 31;
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem = *reinterpret_cast<volatile uint32_t*>(sm + lay.slot);
    const int nch = (M + NC - 1) / NC;
    if (tid == 0) {
      if (tc::mbar_wait(bar(0), 0, dp.wait_limit)) {
        pending &= ~1u;
        issue(0, M);
        if (nch > 1) issue(1, M);
      } else {
        *flag() = 1;
        tc::report_timeout(dp.status);
      }
    }
    __syncthreads();
    const uint32_t* R = reinterpret_cast<const uint32_t*>(sm + lay.r);
    for (int ch = 0; ch < nch && !*flag(); ++ch) {
      const int bf = ch & 1;
      const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar(1 + bf), (uint32_t)((ch >> 1) & 1), dp.wait_limit));
      if (ok) {
        if (tid == 0) pending &= ~(2u << bf);
        tc::fence_after_sync();
        epilogue(ch, M);
      } else {
        *flag() = 1;
        if (lane == 0) tc::report_timeout(dp.status);
      }
      tc::fence_before_sync();
      __syncthreads();
      if (*flag()) break;
      if (tid == 0 && ch + 2 < nch) {
        tc::fence_after_sync();
        issue(ch + 2, M);
      }
      const int mc = min(NC, M - ch * NC);
      for (int tg = slice; tg < mc; tg += SL) {
        uint32_t x[G::EC];
#pragma unroll
        for (int i = 0; i < G::EC; ++i) x[i] = R[tg * SH::TCH + (jj + G::EC * i) * TC + c];
        int id;
        uint32_t* dst;
        target(ch * NC + tg, id, dst);
        col_ntt_store<G, TC>(dp, x, id, dst, colbuf(slice), l, jj, c, slice);
      }
      __syncthreads();
    }
    // teardown: nothing of this block may still write shared or tensor memory
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && pending) {
      if (pending & 1u) tc::mbar_wait(bar(0), 0, kTcDrainLimit);
      if (pending & 2u) tc::mbar_wait(bar(1), (uint32_t)((last0 >> 1) & 1), kTcDrainLimit);
      if (pending & 4u) tc::mbar_wait(bar(2), (uint32_t)((last1 >> 1) & 1), kTcDrainLimit);
    }
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, SH::TMEM_COLS);
  }
};

// Source phase of the tensor-core kernels: slice s finishes the iNTT columns
// of sources k = s, s + GS, ..., multiplies by cin[k] (N^-1 folded) and
// writes the centered values' digits (and, with ycopy, the centered values
// themselves to global memory).
template <class G, int TC, class Blk>
__device__ __forceinline__ void col_inputs_tc(const DevParams& dp, const uint32_t* src, size_t src_stride, int K,
                                              int id0, const uint2* cin, const Blk& blk, uint32_t* colbuf, int l,
                                              int jj, int c, int slice, int GS, uint32_t* ycopy = nullptr,
                                              const int2* idtab = nullptr) {
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
    constexpr int CT = TC * G::EC;
    if (q < (1u << 30)) col_inv<G::EC, TC, true>(x, colbuf, itw, jj, c, q, slice + 1, CT);
    else col_inv<G::EC, TC, false>(x, colbuf, itw, jj, c, q, slice + 1, CT);
    const uint2 w = cin[k];
    int32_t y[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) y[i] = centered(csub(shoup(x[i], w.x, w.y, q), q), q);
    blk.put(k, y, jj, c);
    if (ycopy) {
      uint32_t* yc = ycopy + ((size_t)k << dp.log_n);
#pragma unroll
      for (int i = 0; i < G::EC; ++i) yc[(jj + G::EC * i) * G::W + l] = (uint32_t)y[i];
    }
  }
}

// ModUp, tensor-core form of k_ks_modup_cols (same grid, same results).
template <class G, int TC, int SL, int NC>
__global__ void __launch_bounds__(TcShape<G, TC, SL, NC>::NT, 1)
    k_ks_modup_cols_tc(DevParams dp, int n, int base, int tix, int kr_max, int mmax, const uint32_t* S, uint32_t* T) {
  using SH = TcShape<G, TC, SL, NC>;
  extern __shared__ __align__(128) uint8_t tc_sm[];
  const int tid = threadIdx.x, slice = tid / SH::CT, pos = tid % SH::CT;
  const int c = pos % TC, jj = pos / TC, l = blockIdx.x * TC + c, j = blockIdx.y;
  const int alpha = dp.alpha, L = dp.L, ext = n + alpha, g = base / alpha + j;
  const int lo = max(0, g * alpha - base), hi = min(n, (g + 1) * alpha - base), K = hi - lo, M = ext - K;
  const int2 off = dp.ks.up_off[tix * dp.dnum + j];
  const int2 img = dp.ks.up_img[tix * dp.dnum + j];
  auto target = [&](int m, int& id, uint32_t*& dst) {
    const int t = m < lo ? m : m + K;  // skip the digit's own limbs
    id = prime_of(t, n, L, base);
    dst = T + ((size_t)(j * ext + t) << dp.log_n);
  };
  TcBlock<G, TC, SL, NC> blk(tc_sm, tc_smem<SH, NC>(kr_max, mmax), tc_kr(K));
  blk.begin(dp, dp.ks.tc_img + img.x, (uint32_t)img.y, K, M, target);
  pdl_wait();
  pdl_trigger();
  col_inputs_tc<G, TC>(dp, S + ((size_t)lo << dp.log_n), (size_t)1 << dp.log_n, K, base + lo, dp.ks.up_cin + off.x,
                       blk, blk.colbuf(slice), l, jj, c, slice, SL);
  blk.convert(dp, M, target, l, jj, c, slice);
}

// ModDown, tensor-core form of k_ks_moddown_cols.
template <class G, int TC, int SL, int NC>
__global__ void __launch_bounds__(TcShape<G, TC, SL, NC>::NT, 1)
    k_ks_moddown_cols_tc(DevParams dp, int n, int base, int tix, int kr_max, const uint32_t* S, uint32_t* T) {
  using SH = TcShape<G, TC, SL, NC>;
  extern __shared__ __align__(128) uint8_t tc_sm[];
  const int tid = threadIdx.x, slice = tid / SH::CT, pos = tid % SH::CT;
  const int c = pos % TC, jj = pos / TC, l = blockIdx.x * TC + c, u = blockIdx.y;
  const int alpha = dp.alpha;
  const int2 img = dp.ks.dn_img[tix];
  auto target = [&](int i, int& id, uint32_t*& dst) {
    id = base + i;
    dst = T + ((size_t)(u * n + i) << dp.log_n);
  };
  TcBlock<G, TC, SL, NC> blk(tc_sm, tc_smem<SH, NC>(kr_max, n), tc_kr(alpha));
  blk.begin(dp, dp.ks.tc_img + img.x, (uint32_t)img.y, alpha, n, target);
  pdl_wait();
  pdl_trigger();
  col_inputs_tc<G, TC>(dp, S + ((size_t)(u * alpha) << dp.log_n), (size_t)1 << dp.log_n, alpha, dp.L, dp.ks.dn_cin,
                       blk, blk.colbuf(slice), l, jj, c, slice, SL);
  blk.convert(dp, n, target, l, jj, c, slice);
}

// ModDown fused with rescaling, second column kernel, tensor-core form of
// k_rs_cols_fused: K = alpha + 1 stored sources (the centered P-limb
// coefficients and the top limb's c_l, Y = [2][alpha + 1][N]), targets i < l.
template <class G, int TC, int SL, int NC>
__global__ void __launch_bounds__(TcShape<G, TC, SL, NC>::NT, 1)
    k_rs_cols_fused_tc(DevParams dp, int n, int kr_max, const uint32_t* Y, uint32_t* T) {
  using SH = TcShape<G, TC, SL, NC>;
  extern __shared__ __align__(128) uint8_t tc_sm[];
  const int tid = threadIdx.x, slice = tid / SH::CT, pos = tid % SH::CT;
  const int c = pos % TC, jj = pos / TC, l = blockIdx.x * TC + c, u = blockIdx.y;
  const int alpha = dp.alpha, top = n - 1, K = alpha + 1;
  const int2 img = dp.ks.rs_img[n];
  auto target = [&](int i, int& id, uint32_t*& dst) {
    id = i;
    dst = T + ((size_t)(u * top + i) << dp.log_n);
  };
  TcBlock<G, TC, SL, NC> blk(tc_sm, tc_smem<SH, NC>(kr_max, top), tc_kr(K));
  blk.begin(dp, dp.ks.tc_img + img.x, (uint32_t)img.y, K, top, target);
  pdl_wait();
  pdl_trigger();
  for (int k = slice; k < K; k += SL) {
    const uint32_t* yk = Y + ((size_t)(u * K + k) << dp.log_n);
    int32_t y[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) y[i] = (int32_t)yk[(jj + G::EC * i) * G::W + l];
    blk.put(k, y, jj, c);
  }
  blk.convert(dp, top, target, l, jj, c, slice);
}

// ---------------------------------------------------------------------------
// Launch shapes of the tensor-core kernels: (tc, sl, tp) with tp = NC, the
// targets per MMA chunk (8 or 16); z = 1.
// ---------------------------------------------------------------------------

// Calls f(IC<TC>, IC<SL>, IC<NC>) for a tensor-core shape.
template <class G, class F>
static bool with_tc_shape(const ColShape& s, F f) {
  if constexpr (G::H != 64) {
    return false;
  } else {
    switch (s.tc * 1000 + s.sl * 100 + s.tp) {
      case 8000 + 200 + 8: f(IC<8>{}, IC<2>{}, IC<8>{}); return true;
      case 8000 + 200 + 16: f(IC<8>{}, IC<2>{}, IC<16>{}); return true;
      case 8000 + 400 + 8: f(IC<8>{}, IC<4>{}, IC<8>{}); return true;
      case 8000 + 400 + 16: f(IC<8>{}, IC<4>{}, IC<16>{}); return true;
      case 4000 + 400 + 8: f(IC<4>{}, IC<4>{}, IC<8>{}); return true;
      case 4000 + 400 + 16: f(IC<4>{}, IC<4>{}, IC<16>{}); return true;
      case 4000 + 800 + 8: f(IC<4>{}, IC<8>{}, IC<8>{}); return true;
      case 4000 + 800 + 16: f(IC<4>{}, IC<8>{}, IC<16>{}); return true;
      default: return false;
    }
  }
}

inline bool is_tc_shape(const ColShape& s) { return s.tp == 8 || s.tp == 16; }

template <class G>
static bool tc_shape_ok(const ColShape& s) {
  bool ok = false;
  if (s.z == 1) with_tc_shape<G>(s, [&](auto, auto, auto) { ok = true; });
  return ok;
}

}  // namespace ckks
