// Hybrid key switching (Sec. 2.3: ModUp -> KeyMult -> MAC -> ModDown) and
// single rescaling (Sec. 2.1). Every ModSwitch (iNTT -> BConv -> NTT, Alg. 1)
// is split at its coefficient-domain midpoint, which only exists between the
// two column phases, so the pipeline alternates:
//
//   prep    (stream): input d, a1*a2 (tensor) or phi_k(a) (automorphism)    -> S
//   rows^-1 (rows)  : iNTT row phase of S, in place
//   C1      (cols)  : iNTT col phase, * N^-1 (Q_j/q_i)^-1, BConv (Eq. 2) to
//                     every prime outside digit j, NTT col phase            -> T
//   rows    (rows)  : NTT row phase of every T limb, in place
//   KeyMult (stream): acc_u = sum_j ModUp_j * evk_j[u] (Par. 1)            -> A
//   rows^-1 (rows)  : iNTT row phase of the P limbs of A                     -> S
//   C2      (cols)  : iNTT col phase, * N^-1 (P/p_k)^-1, BConv P -> Q, NTT col -> T
//   rows    (rows)  : NTT row phase of T, in place
//   epilogue(stream): (acc - z) P^-1 + (d0, d1) or (phi(b), 0)              -> out
//
// Row kernels (rows.cuh) hold W-word rows in registers with their twiddles
// loaded up front; column kernels hold a tile of TC columns; streaming kernels
// do the NTT-domain element-wise work with 128-bit accesses at full
// occupancy. Constants are folded as in the paper's Seq. 2 (N^-1 into the
// BConv constant, 2^32 into the BConv matrix). The BConv product uses the
// paper's lazy reduction (Sec. 4.2).
#include "geo.cuh"
#include "internal.h"
#include "rows.cuh"

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
// Rescale column kernel: iNTT cols of the top limb, centered, reduced into
// every lower prime, NTT cols.
// ---------------------------------------------------------------------------
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


// ---------------------------------------------------------------------------
// Streaming kernels: grid (N / (4 * threads), limbs), four consecutive
// positions per thread.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t stream_pos() { return 4 * (blockIdx.x * blockDim.x + threadIdx.x); }

// Four NTT-domain values of the key-switched polynomial at limb i.
__device__ __forceinline__ void ks_input4(const DevParams& dp, const KsArgs& a, int i, uint32_t p0,
                                          uint32_t (&v)[4]) {
  const size_t off = ((size_t)i << dp.log_n) + p0;
  if (a.mode == KS_PLAIN) {
    load_vec<4>(v, a.x0 + off);
  } else if (a.mode == KS_TENSOR) {
    const PrimeConst P = dp.pc[i];
    uint32_t a1[4], a2[4];
    load_vec<4>(a1, a.x0 + a.poly_stride0 + off);
    load_vec<4>(a2, a.x1 + a.poly_stride1 + off);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = mulmod(a1[k], a2[k], P);
  } else {
    const uint32_t* s = a.x0 + a.poly_stride0 + ((size_t)i << dp.log_n);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __ldg(s + auto_src(p0 + k, a.galois, dp.log_n));
  }
}

__global__ void k_ks_prep(DevParams dp, KsArgs a, uint32_t* S) {
  const int i = blockIdx.y;
  const uint32_t p0 = stream_pos();
  uint32_t v[4];
  ks_input4(dp, a, i, p0, v);
  store_vec<4>(S + ((size_t)i << dp.log_n) + p0, v);
}

// KeyMult + MAC over the D digits for extended limb t (Par. 1): the digit's
// own limbs are the input itself (ModUp copies them), the others come from
// the NTT'd ModUp output T[j][t]. All loads of a thread are issued before any
// product so that one memory latency covers the whole sum. A = [2][n + alpha][N].
template <int D>
__global__ void k_ks_keymult(DevParams dp, KsArgs a, const uint32_t* T, uint32_t* A, int km_out,
                             uint32_t* km_dst) {
  const int t = blockIdx.y;
  const int n = a.n, alpha = dp.alpha, L = dp.L, ext = n + alpha, ext_top = L + alpha;
  const int id = prime_of(t, n, L);
  const int key_limb = t < n ? t : L + (t - n);
  const PrimeConst P = dp.pc[id];
  const uint32_t p0 = stream_pos();
  uint32_t x[D][4], e0[D][4], e1[D][4];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int lo = j * alpha, hi = min(n, lo + alpha);
    if (t >= lo && t < hi) ks_input4(dp, a, t, p0, x[j]);
    else load_vec<4>(x[j], T + ((size_t)(j * ext + t) << dp.log_n) + p0);
  }
  if (km_out == KM_MODUP) {
#pragma unroll
    for (int j = 0; j < D; ++j) store_vec<4>(km_dst + ((size_t)(j * ext + t) << dp.log_n) + p0, x[j]);
    return;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    load_vec_stream<4>(e0[j], a.evk + ((size_t)((j * 2 + 0) * ext_top + key_limb) << dp.log_n) + p0);
    load_vec_stream<4>(e1[j], a.evk + ((size_t)((j * 2 + 1) * ext_top + key_limb) << dp.log_n) + p0);
  }
  uint32_t acc0[4] = {0, 0, 0, 0}, acc1[4] = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc0[k] = addm(acc0[k], fix_signed(mont_mul(x[j][k], e0[j][k], P.q, P.m), P.q), P.q);
      acc1[k] = addm(acc1[k], fix_signed(mont_mul(x[j][k], e1[j][k], P.q, P.m), P.q), P.q);
    }
  uint32_t* dst = km_out == KM_ACC_ALL ? km_dst : A;
  store_vec<4>(dst + ((size_t)t << dp.log_n) + p0, acc0);
  store_vec<4>(dst + ((size_t)(ext + t) << dp.log_n) + p0, acc1);
}

static void launch_keymult(int digits, dim3 g, int th, cudaStream_t st, const DevParams& dp, const KsArgs& a,
                           const uint32_t* T, uint32_t* A, int km_out, uint32_t* km_dst) {
  switch (digits) {
#define CKKS_KM(D) \
  case D: k_ks_keymult<D><<<g, th, 0, st>>>(dp, a, T, A, km_out, km_dst); break;
    CKKS_KM(1) CKKS_KM(2) CKKS_KM(3) CKKS_KM(4) CKKS_KM(5) CKKS_KM(6) CKKS_KM(7) CKKS_KM(8)
#undef CKKS_KM
    default:
      break;
  }
}

// ModDown epilogue: out_u[i] = (A_u[i] - T_u[i]) P^-1 + extra_u[i], with
// extra = (d0, d1) recomputed from the inputs (HMult) or (phi_k(b), 0) (HRot).
__global__ void k_ks_epilogue(DevParams dp, KsArgs a, const uint32_t* T, const uint32_t* A, size_t a_stride) {
  const int n = a.n;
  const int u = blockIdx.y / n, i = blockIdx.y % n;
  const PrimeConst P = dp.pc[i];
  const uint2 pinv = dp.ks.dn_pinv[i];
  const uint32_t p0 = stream_pos();
  const size_t off = ((size_t)i << dp.log_n) + p0;
  uint32_t z[4], acc[4];
  load_vec<4>(z, T + ((size_t)(u * n + i) << dp.log_n) + p0);
  load_vec<4>(acc, A + u * a_stride + off);
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = csub(shoup(acc[k] - z[k] + P.q, pinv.x, pinv.y, P.q), P.q);
  if (a.extra == 1) {
    uint32_t b1[4], b2[4];
    load_vec<4>(b1, a.x0 + off);
    load_vec<4>(b2, a.x1 + off);
    if (u == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) z[k] = addm(z[k], mulmod(b1[k], b2[k], P), P.q);
    } else {
      uint32_t a1[4], a2[4];
      load_vec<4>(a1, a.x0 + a.poly_stride0 + off);
      load_vec<4>(a2, a.x1 + a.poly_stride1 + off);
#pragma unroll
      for (int k = 0; k < 4; ++k) z[k] = addm(z[k], addm(mulmod(a1[k], b2[k], P), mulmod(a2[k], b1[k], P), P.q), P.q);
    }
  } else if (a.extra == 2 && u == 0) {
    const uint32_t* sb = a.x0 + ((size_t)i << dp.log_n);
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = addm(z[k], __ldg(sb + auto_src(p0 + k, a.galois, dp.log_n)), P.q);
  }
  store_vec<4>(a.out + u * a.out_stride + off, z);
}

// Rescale epilogue: out_u[i] = (c_u[i] - r_u[i]) q_l^-1, r = NTT of the
// centered top limb reduced modulo q_i.
__global__ void k_rs_epilogue(DevParams dp, const uint32_t* in, size_t sin, int n, const uint32_t* T,
                              uint32_t* out, size_t sout) {
  const int top = n - 1;
  const int u = blockIdx.y / top, i = blockIdx.y % top;
  const PrimeConst P = dp.pc[i];
  const uint2 qinv = dp.ks.rs_qinv[top * dp.L + i];
  const uint32_t p0 = stream_pos();
  const size_t off = ((size_t)i << dp.log_n) + p0;
  uint32_t z[4], c[4];
  load_vec<4>(z, T + ((size_t)(u * top + i) << dp.log_n) + p0);
  load_vec<4>(c, in + u * sin + off);
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = csub(shoup(c[k] - z[k] + P.q, qinv.x, qinv.y, P.q), P.q);
  store_vec<4>(out + u * sout + off, z);
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
    count_launch(1);
}

template <class G, int TC>
static void launch_moddown_cols(const DevParams& dp, int n, const Scratch& sc, cudaStream_t st) {
  const size_t sm = col_smem_bytes<G, TC>(dp.alpha);
  set_col_smem((const void*)k_ks_moddown_cols<G, TC>, sm);
  k_ks_moddown_cols<G, TC><<<dim3(G::W / TC, 2), kSlices * ColTile<G, TC>::CT, sm, st>>>(dp, n, sc.S, sc.T);
    count_launch(1);
}

// Streaming grid: four positions per thread.
static void stream_grid(int log_n, int limbs, dim3& grid, int& threads) {
  const int quads = (1 << log_n) / 4;
  threads = quads < 256 ? quads : 256;
  grid = dim3(quads / threads, limbs);
}

// Offset and count of the level's entries in the ModUp limb table (the
// NTT'd ModUp limbs (j, t), t outside digit j).
static void modup_rows_range(int n, int alpha, int& off, int& cnt) {
  auto count = [&](int m) { return ((m + alpha - 1) / alpha) * (m + alpha) - m; };
  off = 0;
  for (int m = 1; m < n; ++m) off += count(m);
  cnt = count(n);
}

// ModDown from the accumulators A = [2][n + alpha][N] (a_stride between
// polys): P-limb iNTT rows (into S), C2, NTT rows, epilogue.
template <class G>
static void moddown_tail(const DevParams& dp, const Scratch& sc, const KsArgs& a, const uint32_t* A,
                         size_t a_stride, cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha;
  const size_t limb = (size_t)1 << dp.log_n;
  // P limbs n .. n+alpha-1 of both accumulators -> S [2][alpha] (compact)
  launch_rows_g<G>(dp, true, A, sc.S, 2 * alpha,
                   LimbMap{nullptr, n, n + alpha, n, dp.L, alpha, (int)(a_stride >> dp.log_n)}, true, st);
  prof_mark(sc, st, P_MODDOWN_IN_ROWS);
  with_tc<G>(2, [&] { launch_moddown_cols<G, 8>(dp, n, sc, st); },
             [&] { launch_moddown_cols<G, 4>(dp, n, sc, st); });
  prof_mark(sc, st, P_MODDOWN_COLS);
  launch_rows_g<G>(dp, false, sc.T, sc.T, 2 * n, LimbMap{nullptr, 0, n, n, dp.L}, false, st);
  prof_mark(sc, st, P_MODDOWN_ROWS);
  dim3 g;
  int th;
  stream_grid(dp.log_n, 2 * n, g, th);
  k_ks_epilogue<<<g, th, 0, st>>>(dp, a, sc.T, A, a_stride);
    count_launch(1);
  prof_mark(sc, st, P_KS_EPILOGUE);
}

void launch_keyswitch(const DevParams& dp, const Scratch& sc, const KsArgs& a, int km_out, uint32_t* km_dst,
                      cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha, ext = n + alpha;
  const int digits = (n + alpha - 1) / alpha;
  const size_t limb = (size_t)1 << dp.log_n;
  dim3 g;
  int th;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    stream_grid(dp.log_n, n, g, th);
    k_ks_prep<<<g, th, 0, st>>>(dp, a, sc.S);
    count_launch(1);
    prof_mark(sc, st, P_KS_PREP);
    launch_rows_g<G>(dp, true, sc.S, sc.S, n, LimbMap{nullptr, 0, n, n, dp.L}, false, st);
    prof_mark(sc, st, P_KS_IN_ROWS);
    with_tc<G>(digits, [&] { launch_modup_cols<G, 8>(dp, n, digits, sc, st); },
               [&] { launch_modup_cols<G, 4>(dp, n, digits, sc, st); });
    prof_mark(sc, st, P_MODUP_COLS);
    int off, cnt;
    modup_rows_range(n, alpha, off, cnt);
    launch_rows_g<G>(dp, false, sc.T, sc.T, cnt, LimbMap{dp.ks.up_rows + off, 0, 1, 0, 0}, false, st);
    prof_mark(sc, st, P_MODUP_ROWS);
    stream_grid(dp.log_n, ext, g, th);
    launch_keymult(digits, g, th, st, dp, a, sc.T, sc.A, km_out, km_dst);
    count_launch(1);
    prof_mark(sc, st, P_KEYMULT);
    if (km_out == KM_KEYSWITCH) moddown_tail<G>(dp, sc, a, sc.A, (size_t)ext * limb, st);
  });
}

void launch_moddown(const DevParams& dp, const Scratch& sc, const uint32_t* acc, int n, uint32_t* out,
                    cudaStream_t st) {
  KsArgs a{};
  a.n = n;
  a.out = out;
  a.out_stride = (size_t)n << dp.log_n;
  a.extra = 0;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    moddown_tail<G>(dp, sc, a, acc, (size_t)(n + dp.alpha) << dp.log_n, st);
  });
}

void launch_rescale(const DevParams& dp, const Scratch& sc, const uint32_t* in, size_t sin, int n,
                    uint32_t* out, size_t sout, cudaStream_t st) {
  const int top = n - 1;
  if (top < 1) return;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    // top limb of both polynomials -> S [2] (compact)
    launch_rows_g<G>(dp, true, in, sc.S, 2, LimbMap{nullptr, top, n, n, dp.L, 1, (int)(sin >> dp.log_n)}, true, st);
    prof_mark(sc, st, P_RS_IN_ROWS);
    const int tiles = G::W / G::TC;
    const int gr = groups_for(tiles * 2, top);
    k_rs_cols<G><<<dim3(tiles, 2, gr), G::CT, 0, st>>>(dp, n, sc.S, sc.T, gr);
    count_launch(1);
    prof_mark(sc, st, P_RS_COLS);
    launch_rows_g<G>(dp, false, sc.T, sc.T, 2 * top, LimbMap{nullptr, 0, top, top, dp.L}, false, st);
    prof_mark(sc, st, P_RS_ROWS);
    dim3 g;
    int th;
    stream_grid(dp.log_n, 2 * top, g, th);
    k_rs_epilogue<<<g, th, 0, st>>>(dp, in, sin, n, sc.T, out, sout);
    count_launch(1);
    prof_mark(sc, st, P_RS_EPILOGUE);
  });
}

}  // namespace ckks
