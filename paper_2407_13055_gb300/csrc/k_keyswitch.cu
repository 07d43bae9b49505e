// Fused hybrid key switching (Sec. 2.3: ModUp -> KeyMult -> MAC -> ModDown)
// and single rescaling (Sec. 2.1), built from alternating row and column
// kernels so that every ModSwitch (iNTT -> BConv -> NTT, Alg. 1) is split at
// its coefficient-domain midpoint:
//
//   R1 (rows)  : input (d, a1*a2 or phi_k(a)) -> iNTT row phase          -> S
//   C1 (cols)  : iNTT col phase, * N^-1 (Q_j/q_i)^-1, BConv Eq. 2 to every
//                prime outside digit j, NTT col phase                    -> T
//   R2 (rows)  : NTT row phase, KeyMult + MAC over the digits with evk;
//                Q limbs -> A, P limbs -> iNTT row phase                 -> S
//   C2 (cols)  : iNTT col phase, * N^-1 (P/p_k)^-1, BConv P -> Q, NTT col -> T
//   R3 (rows)  : NTT row phase, (acc - z) P^-1 + (d0, d1) or (phi(b), 0)  -> out
//
// Constants are folded as in the paper's Seq. 2 (N^-1 into the BConv
// constant, 2^32 into the BConv matrix so that the signed Montgomery
// reduction of the lazily accumulated sum needs no correction). The BConv
// matrix product uses the paper's lazy reduction (Sec. 4.2): centered inputs
// and entries, eight 64-bit products, then +-2^32 p range fixes every four.
#include "geo.cuh"
#include "internal.h"

namespace ckks {

namespace {

__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, uint32_t q) { return csub(a + b, q); }

__device__ __forceinline__ int prime_of(int t, int n, int L) { return t < n ? t : L + (t - n); }

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
__device__ __forceinline__ void bconv_accumulate(const int4* __restrict__ y4, int pos, int K,
                                                 const int32_t* __restrict__ mat, const PrimeConst& P,
                                                 uint32_t (&out)[EC]) {
  int64_t acc[EC];
#pragma unroll
  for (int i = 0; i < EC; ++i) acc[i] = 0;
  int since = 0, batch = 8;
  for (int k = 0; k < K; ++k) {
    const int32_t b = __ldg(mat + k);
#pragma unroll
    for (int i4 = 0; i4 < EC / 4; ++i4) {
      const int4 v = y4[(k * (EC / 4) + i4) * NT + pos];
      acc[4 * i4 + 0] += (int64_t)v.x * (int64_t)b;
      acc[4 * i4 + 1] += (int64_t)v.y * (int64_t)b;
      acc[4 * i4 + 2] += (int64_t)v.z * (int64_t)b;
      acc[4 * i4 + 3] += (int64_t)v.w * (int64_t)b;
    }
    if (++since == batch) {
#pragma unroll
      for (int i = 0; i < EC; ++i) acc[i] = fold(acc[i], P.r1c);
      since = 0;
      batch = 4;
    }
  }
#pragma unroll
  for (int i = 0; i < EC; ++i) out[i] = fix_signed(smr(fold(acc[i], P.r1c), P.q, P.m), P.q);
}

}  // namespace

// ---------------------------------------------------------------------------
// R1: key-switch input -> iNTT row phase -> S [n][N] (A layout stores)
// ---------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ void load_ks_input_row(const DevParams& dp, const KsArgs& a, int i, int h, int jj,
                                                  uint32_t* b, uint32_t (&x)[G::ER]) {
  const size_t rowoff = ((size_t)i << dp.log_n) + (size_t)h * G::W;
  if (a.mode == KS_PLAIN) {
    load_vec<G::ER>(x, a.x0 + rowoff + G::ER * jj);
  } else if (a.mode == KS_TENSOR) {
    const PrimeConst P = dp.pc[i];
    uint32_t a1[G::ER], a2[G::ER];
    load_vec<G::ER>(a1, a.x0 + a.poly_stride0 + rowoff + G::ER * jj);
    load_vec<G::ER>(a2, a.x1 + a.poly_stride1 + rowoff + G::ER * jj);
#pragma unroll
    for (int r = 0; r < G::ER; ++r) x[r] = mulmod(a1[r], a2[r], P);
  } else {
    // phi_k(a): destination row h reads one source row (Eq. 4 keeps the high
    // bits of the bit-reversed position together); stage it in shared memory.
    const uint32_t src_row = auto_src((uint32_t)h * G::W, a.galois, dp.log_n) / G::W;
    const uint32_t* s = a.x0 + a.poly_stride0 + ((size_t)i << dp.log_n) + (size_t)src_row * G::W;
#pragma unroll
    for (int r = 0; r < G::ER; ++r) {
      const int l = jj + G::ER * r;
      b[l + l / G::ER] = s[l];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < G::ER; ++r) {
      const uint32_t l = G::ER * jj + r;
      const uint32_t ls = auto_src((uint32_t)h * G::W + l, a.galois, dp.log_n) % G::W;
      x[r] = b[ls + ls / G::ER];
    }
    __syncwarp();
  }
}

template <class G>
__global__ void __launch_bounds__(G::RT) k_ks_in(DevParams dp, KsArgs a, uint32_t* S) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int i = blockIdx.y;
  uint32_t* b = buf + r * G::ROWBUF;
  uint32_t x[G::ER];
  load_ks_input_row<G>(dp, a, i, h, jj, b, x);
  const uint32_t q = dp.pc[i].q;
  const uint2* itw = dp.itw + ((size_t)i << dp.log_n);
  if (q < (1u << 30)) row_inv<G::ER, G::H, true>(x, b, itw, h, jj, q);
  else row_inv<G::ER, G::H, false>(x, b, itw, h, jj, q);
  uint32_t* o = S + ((size_t)i << dp.log_n) + (size_t)h * G::W;
#pragma unroll
  for (int k = 0; k < G::ER; ++k) o[jj + G::ER * k] = x[k];
}

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
                                           int c, int pos, int slice, int GS) {
  using CTL = ColTile<G, TC>;
  for (int k = slice; k < K; k += GS) {
    const int id = id0 + k;
    const uint32_t q = dp.pc[id].q;
    const uint2* itw = dp.itw + ((size_t)id << dp.log_n);
    const uint32_t* s = src + k * src_stride;
    uint32_t x[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) x[i] = s[(G::EC * jj + i) * G::W + l];
    if (q < (1u << 30)) col_inv<G::EC, TC, true>(x, colbuf, itw, jj, c, q, slice + 1, CTL::CT);
    else col_inv<G::EC, TC, false>(x, colbuf, itw, jj, c, q, slice + 1, CTL::CT);
    const uint2 w = cin[k];
    int32_t y[G::EC];
#pragma unroll
    for (int i = 0; i < G::EC; ++i) y[i] = centered(csub(shoup(x[i], w.x, w.y, q), q), q);
#pragma unroll
    for (int i4 = 0; i4 < G::EC / 4; ++i4)
      y4[(k * (G::EC / 4) + i4) * CTL::CT + pos] = make_int4(y[4 * i4], y[4 * i4 + 1], y[4 * i4 + 2], y[4 * i4 + 3]);
  }
}

// BConv one target and run its NTT column phase; store B layout (lazy range).
template <class G, int TC>
__device__ __forceinline__ void col_target(const DevParams& dp, const int4* y4, int K, const int32_t* mat_row,
                                           int id, uint32_t* dst, uint32_t* colbuf, int l, int jj, int c, int pos,
                                           int slice) {
  using CTL = ColTile<G, TC>;
  const PrimeConst P = dp.pc[id];
  uint32_t x[G::EC];
  bconv_accumulate<G::EC, CTL::CT>(y4, pos, K, mat_row, P, x);
  const uint2* tw = dp.tw + ((size_t)id << dp.log_n);
  if (P.q < (1u << 30)) col_fwd<G::EC, TC, true>(x, colbuf, tw, jj, c, P.q, slice + 1, CTL::CT);
  else col_fwd<G::EC, TC, false>(x, colbuf, tw, jj, c, P.q, slice + 1, CTL::CT);
#pragma unroll
  for (int i = 0; i < G::EC; ++i) dst[(G::EC * jj + i) * G::W + l] = x[i];
}

constexpr int kSlices = 4;

// C1: ModUp column kernel. grid (W/TC, digits), block kSlices * CT.
template <class G, int TC>
__global__ void __launch_bounds__(kSlices* ColTile<G, TC>::CT) k_ks_modup_cols(DevParams dp, int n,
                                                                               const uint32_t* S, uint32_t* T) {
  using CTL = ColTile<G, TC>;
  extern __shared__ int4 smem4[];
  const int slice = threadIdx.x / CTL::CT, pos = threadIdx.x % CTL::CT;
  const int c = pos % TC, jj = pos / TC;
  const int l = blockIdx.x * TC + c;
  const int j = blockIdx.y;
  const int alpha = dp.alpha, L = dp.L, ext = n + alpha;
  const int lo = j * alpha, hi = min(n, lo + alpha), K = hi - lo;
  const int2 off = dp.ks.up_off[n * dp.dnum + j];
  int4* y4 = smem4;
  uint32_t* colbuf = reinterpret_cast<uint32_t*>(smem4 + (size_t)alpha * (G::EC / 4) * CTL::CT) + slice * CTL::BUF;
  col_inputs<G, TC>(dp, S + ((size_t)lo << dp.log_n), (size_t)1 << dp.log_n, K, lo, dp.ks.up_cin + off.x, y4,
                    colbuf, l, jj, c, pos, slice, kSlices);
  __syncthreads();
  const int M = ext - K;
  for (int m = slice; m < M; m += kSlices) {
    const int t = m < lo ? m : m + K;  // skip the digit's own limbs
    uint32_t* dst = T + ((size_t)(j * ext + t) << dp.log_n);
    col_target<G, TC>(dp, y4, K, dp.ks.up_mat + off.y + t * K, prime_of(t, n, L), dst, colbuf, l, jj, c, pos,
                      slice);
  }
}

// C2: ModDown column kernel. grid (W/TC, 2 polys). Input S [2][alpha][N]
// (P limbs after the row-phase iNTT); output T [2][n][N].
template <class G, int TC>
__global__ void __launch_bounds__(kSlices* ColTile<G, TC>::CT) k_ks_moddown_cols(DevParams dp, int n,
                                                                                 const uint32_t* S, uint32_t* T) {
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
                    y4, colbuf, l, jj, c, pos, slice, kSlices);
  __syncthreads();
  for (int i = slice; i < n; i += kSlices) {
    uint32_t* dst = T + ((size_t)(u * n + i) << dp.log_n);
    col_target<G, TC>(dp, y4, alpha, dp.ks.dn_mat + i * alpha, i, dst, colbuf, l, jj, c, pos, slice);
  }
}

// ---------------------------------------------------------------------------
// R2: KeyMult + MAC (Par. 1: one kernel for all digits and both key halves)
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(G::RT, 3) k_ks_keymult(DevParams dp, KsArgs a, const uint32_t* T, uint32_t* S,
                                                     uint32_t* A, int km_out, uint32_t* km_dst) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int t = blockIdx.y;
  const int n = a.n, alpha = dp.alpha, L = dp.L, ext = n + alpha, ext_top = L + alpha;
  const int id = prime_of(t, n, L);
  const int key_limb = t < n ? t : L + (t - n);
  const PrimeConst P = dp.pc[id];
  const bool lazy = P.q < (1u << 30);
  const uint2* tw = dp.tw + ((size_t)id << dp.log_n);
  uint32_t* b = buf + r * G::ROWBUF;
  const size_t rowoff = (size_t)h * G::W;
  const int digits = (n + alpha - 1) / alpha;
  uint32_t acc0[G::ER], acc1[G::ER];
#pragma unroll
  for (int i = 0; i < G::ER; ++i) acc0[i] = acc1[i] = 0;
  for (int j = 0; j < digits; ++j) {
    const int lo = j * alpha, hi = min(n, lo + alpha);
    uint32_t x[G::ER];
    if (t >= lo && t < hi) {
      load_ks_input_row<G>(dp, a, t, h, jj, b, x);  // the digit's own limb: ModUp copies it
    } else {
      const uint32_t* s = T + ((size_t)(j * ext + t) << dp.log_n) + rowoff;
#pragma unroll
      for (int i = 0; i < G::ER; ++i) x[i] = s[jj + G::ER * i];
      if (lazy) {
        row_fwd<G::ER, G::H, true>(x, b, tw, h, jj, P.q);
#pragma unroll
        for (int i = 0; i < G::ER; ++i) x[i] = csub(x[i], 2 * P.q);  // [0, 2q) < 2^31
      } else {
        row_fwd<G::ER, G::H, false>(x, b, tw, h, jj, P.q);
#pragma unroll
        for (int i = 0; i < G::ER; ++i) x[i] = csub(x[i], P.q);      // [0, q)
      }
    }
    if (km_out == KM_MODUP) {
#pragma unroll
      for (int i = 0; i < G::ER; ++i) x[i] = csub(x[i], P.q);
      store_vec<G::ER>(km_dst + ((size_t)(j * ext + t) << dp.log_n) + rowoff + G::ER * jj, x);
      continue;
    }
    const uint32_t* e0 = a.evk + ((size_t)((j * 2 + 0) * ext_top + key_limb) << dp.log_n) + rowoff + G::ER * jj;
    const uint32_t* e1 = a.evk + ((size_t)((j * 2 + 1) * ext_top + key_limb) << dp.log_n) + rowoff + G::ER * jj;
#pragma unroll
    for (int i4 = 0; i4 < G::ER / 4; ++i4) {
      uint32_t k0[4], k1[4];
      load_vec_stream<4>(k0, e0 + 4 * i4);
      load_vec_stream<4>(k1, e1 + 4 * i4);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = 4 * i4 + v;
        acc0[i] = addm(acc0[i], fix_signed(mont_mul(x[i], k0[v], P.q, P.m), P.q), P.q);
        acc1[i] = addm(acc1[i], fix_signed(mont_mul(x[i], k1[v], P.q, P.m), P.q), P.q);
      }
    }
  }
  if (km_out == KM_MODUP) return;
  if (km_out == KM_ACC_ALL) {
    store_vec<G::ER>(km_dst + ((size_t)t << dp.log_n) + rowoff + G::ER * jj, acc0);
    store_vec<G::ER>(km_dst + ((size_t)(ext + t) << dp.log_n) + rowoff + G::ER * jj, acc1);
    return;
  }
  if (t < n) {
    store_vec<G::ER>(A + ((size_t)t << dp.log_n) + rowoff + G::ER * jj, acc0);
    store_vec<G::ER>(A + ((size_t)(n + t) << dp.log_n) + rowoff + G::ER * jj, acc1);
  } else {
    const int k = t - n;
    const uint2* itw = dp.itw + ((size_t)id << dp.log_n);
    if (lazy) {
      row_inv<G::ER, G::H, true>(acc0, b, itw, h, jj, P.q);
      row_inv<G::ER, G::H, true>(acc1, b, itw, h, jj, P.q);
    } else {
      row_inv<G::ER, G::H, false>(acc0, b, itw, h, jj, P.q);
      row_inv<G::ER, G::H, false>(acc1, b, itw, h, jj, P.q);
    }
    uint32_t* o0 = S + ((size_t)k << dp.log_n) + rowoff;
    uint32_t* o1 = S + ((size_t)(alpha + k) << dp.log_n) + rowoff;
#pragma unroll
    for (int i = 0; i < G::ER; ++i) {
      o0[jj + G::ER * i] = acc0[i];
      o1[jj + G::ER * i] = acc1[i];
    }
  }
}

// ---------------------------------------------------------------------------
// R3: ModDown epilogue. out_u[i] = (A_u[i] - NTT(T_u[i])) P^-1 + extra_u[i]
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(G::RT, 3) k_ks_out(DevParams dp, KsArgs a, const uint32_t* T, const uint32_t* A,
                                                 size_t a_stride) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int i = blockIdx.y;
  const int n = a.n;
  const PrimeConst P = dp.pc[i];
  const bool lazy = P.q < (1u << 30);
  const uint2* tw = dp.tw + ((size_t)i << dp.log_n);
  const uint2 pinv = dp.ks.dn_pinv[i];
  uint32_t* b = buf + r * G::ROWBUF;
  const size_t rowoff = ((size_t)i << dp.log_n) + (size_t)h * G::W;
  for (int u = 0; u < 2; ++u) {
    uint32_t z[G::ER];
    const uint32_t* s = T + ((size_t)(u * n + i) << dp.log_n) + (size_t)h * G::W;
#pragma unroll
    for (int k = 0; k < G::ER; ++k) z[k] = s[jj + G::ER * k];
    if (lazy) {
      row_fwd<G::ER, G::H, true>(z, b, tw, h, jj, P.q);
#pragma unroll
      for (int k = 0; k < G::ER; ++k) z[k] = normalize<true>(z[k], P.q);
    } else {
      row_fwd<G::ER, G::H, false>(z, b, tw, h, jj, P.q);
#pragma unroll
      for (int k = 0; k < G::ER; ++k) z[k] = normalize<false>(z[k], P.q);
    }
    uint32_t acc[G::ER];
    load_vec<G::ER>(acc, A + u * a_stride + rowoff + G::ER * jj);
#pragma unroll
    for (int k = 0; k < G::ER; ++k) z[k] = csub(shoup(acc[k] - z[k] + P.q, pinv.x, pinv.y, P.q), P.q);
    if (a.extra == 1) {
      // HMult: d0 = b1 b2, d1 = a1 b2 + a2 b1 recomputed from the inputs,
      // four elements at a time.
      const uint32_t* pb1 = a.x0 + rowoff + G::ER * jj;
      const uint32_t* pb2 = a.x1 + rowoff + G::ER * jj;
#pragma unroll
      for (int k4 = 0; k4 < G::ER / 4; ++k4) {
        uint32_t b1[4], b2[4];
        load_vec<4>(b1, pb1 + 4 * k4);
        load_vec<4>(b2, pb2 + 4 * k4);
        if (u == 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) z[4 * k4 + v] = addm(z[4 * k4 + v], mulmod(b1[v], b2[v], P), P.q);
        } else {
          uint32_t a1[4], a2[4];
          load_vec<4>(a1, pb1 + a.poly_stride0 + 4 * k4);
          load_vec<4>(a2, pb2 + a.poly_stride1 + 4 * k4);
#pragma unroll
          for (int v = 0; v < 4; ++v)
            z[4 * k4 + v] =
                addm(z[4 * k4 + v], addm(mulmod(a1[v], b2[v], P), mulmod(a2[v], b1[v], P), P.q), P.q);
        }
      }
    } else if (a.extra == 2 && u == 0) {
      // HRot: add phi_k(b).
      const uint32_t src_row = auto_src((uint32_t)h * G::W, a.galois, dp.log_n) / G::W;
      const uint32_t* sb = a.x0 + ((size_t)i << dp.log_n) + (size_t)src_row * G::W;
#pragma unroll
      for (int k = 0; k < G::ER; ++k) {
        const int l = jj + G::ER * k;
        b[l + l / G::ER] = sb[l];
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < G::ER; ++k) {
        const uint32_t l = G::ER * jj + k;
        const uint32_t ls = auto_src((uint32_t)h * G::W + l, a.galois, dp.log_n) % G::W;
        z[k] = addm(z[k], b[ls + ls / G::ER], P.q);
      }
      __syncwarp();
    }
    store_vec<G::ER>(a.out + u * a.out_stride + rowoff + G::ER * jj, z);
  }
}

// ---------------------------------------------------------------------------
// Rescale (single rescaling): iNTT of the top limb, centered, reduced into
// every lower prime, NTT, then (c_i - r_i) q_l^-1.
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(G::RT) k_rs_in(DevParams dp, const uint32_t* in, size_t sin, int n,
                                                uint32_t* S) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int u = blockIdx.y, l = n - 1;
  const uint32_t q = dp.pc[l].q;
  const uint2* itw = dp.itw + ((size_t)l << dp.log_n);
  uint32_t* b = buf + r * G::ROWBUF;
  uint32_t x[G::ER];
  load_vec<G::ER>(x, in + u * sin + ((size_t)l << dp.log_n) + (size_t)h * G::W + G::ER * jj);
  if (q < (1u << 30)) row_inv<G::ER, G::H, true>(x, b, itw, h, jj, q);
  else row_inv<G::ER, G::H, false>(x, b, itw, h, jj, q);
  uint32_t* o = S + ((size_t)u << dp.log_n) + (size_t)h * G::W;
#pragma unroll
  for (int k = 0; k < G::ER; ++k) o[jj + G::ER * k] = x[k];
}

template <class G>
__global__ void __launch_bounds__(G::CT) k_rs_cols(DevParams dp, int n, const uint32_t* S, uint32_t* T,
                                                  int groups) {
  __shared__ uint32_t colbuf[G::COLBUF];
  const int c = threadIdx.x % G::TC, jj = threadIdx.x / G::TC;
  const int l = blockIdx.x * G::TC + c;
  const int u = blockIdx.y, top = n - 1;
  const PrimeConst Pt = dp.pc[top];
  const uint2* itw = dp.itw + ((size_t)top << dp.log_n);
  uint32_t x[G::EC];
  const uint32_t* s = S + ((size_t)u << dp.log_n);
#pragma unroll
  for (int i = 0; i < G::EC; ++i) x[i] = s[(G::EC * jj + i) * G::W + l];
  if (Pt.q < (1u << 30)) col_inv<G::EC, G::TC, true>(x, colbuf, itw, jj, c, Pt.q);
  else col_inv<G::EC, G::TC, false>(x, colbuf, itw, jj, c, Pt.q);
  int32_t v[G::EC];
#pragma unroll
  for (int i = 0; i < G::EC; ++i) v[i] = centered(csub(shoup(x[i], Pt.ninv, Pt.ninv_sh, Pt.q), Pt.q), Pt.q);
  const int per = (top + groups - 1) / groups;
  const int m0 = blockIdx.z * per, m1 = min(top, m0 + per);
  for (int i = m0; i < m1; ++i) {
    const PrimeConst P = dp.pc[i];
    uint32_t y[G::EC];
#pragma unroll
    for (int k = 0; k < G::EC; ++k) y[k] = fix_signed(smr((int64_t)v[k] * P.r1c, P.q, P.m), P.q);
    const uint2* tw = dp.tw + ((size_t)i << dp.log_n);
    if (P.q < (1u << 30)) col_fwd<G::EC, G::TC, true>(y, colbuf, tw, jj, c, P.q);
    else col_fwd<G::EC, G::TC, false>(y, colbuf, tw, jj, c, P.q);
    uint32_t* d = T + ((size_t)(u * top + i) << dp.log_n);
#pragma unroll
    for (int k = 0; k < G::EC; ++k) d[(G::EC * jj + k) * G::W + l] = y[k];
  }
}

template <class G>
__global__ void __launch_bounds__(G::RT) k_rs_out(DevParams dp, const uint32_t* in, size_t sin, int n,
                                                 const uint32_t* T, uint32_t* out, size_t sout) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int top = n - 1;
  const int u = blockIdx.y / top, i = blockIdx.y % top;
  const PrimeConst P = dp.pc[i];
  const uint2 qinv = dp.ks.rs_qinv[top * dp.L + i];
  const uint2* tw = dp.tw + ((size_t)i << dp.log_n);
  uint32_t* b = buf + r * G::ROWBUF;
  uint32_t z[G::ER];
  const uint32_t* s = T + ((size_t)(u * top + i) << dp.log_n) + (size_t)h * G::W;
#pragma unroll
  for (int k = 0; k < G::ER; ++k) z[k] = s[jj + G::ER * k];
  if (P.q < (1u << 30)) {
    row_fwd<G::ER, G::H, true>(z, b, tw, h, jj, P.q);
#pragma unroll
    for (int k = 0; k < G::ER; ++k) z[k] = normalize<true>(z[k], P.q);
  } else {
    row_fwd<G::ER, G::H, false>(z, b, tw, h, jj, P.q);
#pragma unroll
    for (int k = 0; k < G::ER; ++k) z[k] = normalize<false>(z[k], P.q);
  }
  const size_t rowoff = ((size_t)i << dp.log_n) + (size_t)h * G::W + G::ER * jj;
  uint32_t cv[G::ER];
  load_vec<G::ER>(cv, in + u * sin + rowoff);
#pragma unroll
  for (int k = 0; k < G::ER; ++k) z[k] = csub(shoup(cv[k] - z[k] + P.q, qinv.x, qinv.y, P.q), P.q);
  store_vec<G::ER>(out + u * sout + rowoff, z);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static int groups_for(int blocks_per_group, int max_groups) {
  const int want = 2 * 152;  // aim for two blocks per SM
  int g = (want + blocks_per_group - 1) / blocks_per_group;
  if (g > max_groups) g = max_groups;
  return g < 1 ? 1 : g;
}

template <class G, int TC>
static size_t col_smem_bytes(int K) {
  using CTL = ColTile<G, TC>;
  return (size_t)K * (G::EC / 4) * CTL::CT * sizeof(int4) + (size_t)kSlices * CTL::BUF * sizeof(uint32_t);
}

static void set_col_smem(const void* f, size_t bytes) {
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Column-tile width: 8 columns (32-byte row segments) when that already
// gives two blocks per SM, else 4 to double the block count.
template <class G, class F8, class F4>
static void with_tc(int blocks_per_tile_column, F8 f8, F4 f4) {
  if ((G::W / 8) * blocks_per_tile_column >= 2 * 152 || G::W / 4 < 16) f8();
  else f4();
}

template <class G, int TC>
static void launch_modup_cols(const DevParams& dp, int n, int digits, const Scratch& sc, cudaStream_t st) {
  const size_t sm = col_smem_bytes<G, TC>(dp.alpha);
  set_col_smem((const void*)k_ks_modup_cols<G, TC>, sm);
  k_ks_modup_cols<G, TC><<<dim3(G::W / TC, digits), kSlices * ColTile<G, TC>::CT, sm, st>>>(dp, n, sc.S, sc.T);
}

template <class G, int TC>
static void launch_moddown_cols(const DevParams& dp, int n, const Scratch& sc, cudaStream_t st) {
  const size_t sm = col_smem_bytes<G, TC>(dp.alpha);
  set_col_smem((const void*)k_ks_moddown_cols<G, TC>, sm);
  k_ks_moddown_cols<G, TC><<<dim3(G::W / TC, 2), kSlices * ColTile<G, TC>::CT, sm, st>>>(dp, n, sc.S, sc.T);
}

void launch_keyswitch(const DevParams& dp, const Scratch& sc, const KsArgs& a, int km_out, uint32_t* km_dst,
                      cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha, ext = n + alpha;
  const int digits = (n + alpha - 1) / alpha;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    const dim3 rows_in(G::H / G::RPC, n), rows_ext(G::H / G::RPC, ext);
    prof_mark(sc, st, -1);
    k_ks_in<G><<<rows_in, G::RT, 0, st>>>(dp, a, sc.S);
    prof_mark(sc, st, P_KS_IN);
    with_tc<G>(digits, [&] { launch_modup_cols<G, 8>(dp, n, digits, sc, st); },
               [&] { launch_modup_cols<G, 4>(dp, n, digits, sc, st); });
    prof_mark(sc, st, P_MODUP_COLS);
    k_ks_keymult<G><<<rows_ext, G::RT, 0, st>>>(dp, a, sc.T, sc.S, sc.A, km_out, km_dst);
    prof_mark(sc, st, P_KEYMULT);
    if (km_out == KM_KEYSWITCH) {
      with_tc<G>(2, [&] { launch_moddown_cols<G, 8>(dp, n, sc, st); },
                 [&] { launch_moddown_cols<G, 4>(dp, n, sc, st); });
      prof_mark(sc, st, P_MODDOWN_COLS);
      k_ks_out<G><<<rows_in, G::RT, 0, st>>>(dp, a, sc.T, sc.A, (size_t)n << dp.log_n);
      prof_mark(sc, st, P_KS_OUT);
    }
  });
}

void launch_moddown(const DevParams& dp, const Scratch& sc, const uint32_t* acc, int n, uint32_t* out,
                    cudaStream_t st) {
  const int alpha = dp.alpha, ext = n + alpha;
  const size_t limb = (size_t)1 << dp.log_n;
  // S <- P limbs of both polynomials, then their row-phase iNTT in place.
  for (int u = 0; u < 2; ++u)
    cudaMemcpyAsync(sc.S + (size_t)u * alpha * limb, acc + ((size_t)u * ext + n) * limb,
                    (size_t)alpha * limb * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  KsArgs a{};
  a.n = n;
  a.out = out;
  a.out_stride = (size_t)n * limb;
  a.extra = 0;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    launch_rows_inv_only(dp, sc.S, 2 * alpha, IdMap{nullptr, alpha, 0, dp.L}, st);
    with_tc<G>(2, [&] { launch_moddown_cols<G, 8>(dp, n, sc, st); },
               [&] { launch_moddown_cols<G, 4>(dp, n, sc, st); });
    count_launch(1);
    k_ks_out<G><<<dim3(G::H / G::RPC, n), G::RT, 0, st>>>(dp, a, sc.T, acc, (size_t)ext * limb);
    count_launch(1);
  });
}

void launch_rescale(const DevParams& dp, const Scratch& sc, const uint32_t* in, size_t sin, int n,
                    uint32_t* out, size_t sout, cudaStream_t st) {
  const int top = n - 1;
  if (top < 1) return;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    k_rs_in<G><<<dim3(G::H / G::RPC, 2), G::RT, 0, st>>>(dp, in, sin, n, sc.S);
    prof_mark(sc, st, P_RS_IN);
    const int tiles = G::W / G::TC;
    const int g = groups_for(tiles * 2, top);
    k_rs_cols<G><<<dim3(tiles, 2, g), G::CT, 0, st>>>(dp, n, sc.S, sc.T, g);
    prof_mark(sc, st, P_RS_COLS);
    k_rs_out<G><<<dim3(G::H / G::RPC, 2 * top), G::RT, 0, st>>>(dp, in, sin, n, sc.T, out, sout);
    prof_mark(sc, st, P_RS_OUT);
  });
}

}  // namespace ckks
