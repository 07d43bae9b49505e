// Hybrid key switching (Sec. 2.3: ModUp -> KeyMult -> MAC -> ModDown) and
// single rescaling (Sec. 2.1). Every ModSwitch (iNTT -> BConv -> NTT, Alg. 1)
// is split at its coefficient-domain midpoint, which only exists between the
// two column phases, so the pipeline alternates:
//
//   rows^-1 (rows)  : input d, a1*a2 (tensor) or phi_k(a) (automorphism)
//                     formed while loading, iNTT row phase                  -> S
//   C1      (cols)  : iNTT col phase, * N^-1 (Q_j/q_i)^-1, BConv (Eq. 2) to
//                     every prime outside digit j, NTT col phase            -> T
//   rows    (rows)  : NTT row phase of every T limb, in place
//   KeyMult (stream): acc_u = sum_j ModUp_j * evk_j[u] (Par. 1)            -> A
//   rows^-1 (rows)  : iNTT row phase of the P limbs of A                     -> S
//   C2      (cols)  : iNTT col phase, * N^-1 (P/p_k)^-1, BConv P -> Q, NTT col -> T
//   rows    (rows)  : NTT row phase of T, then the epilogue
//                     (acc - z) P^-1 + (d0, d1) or (phi(b), 0)               -> out
//
// HMult with rescaling by q_l fuses the ModDown into the rescale: the P limbs'
// iNTT rows also take E = acc_l P^-1 + d_l of the top limb; one column kernel
// finishes, per column tile, the top limb's ModDown output V = E - BConv(P ->
// q_l) P^-1 in the coefficient domain and converts the P limbs' and V's
// centered coefficients to every q_i, i < l; the NTT rows' epilogue forms
// (acc_i - w_i)(P q_l)^-1 + d_i q_l^-1.
//
// Row kernels (rows.cuh) hold W-word rows in registers with their twiddles
// loaded up front, and take the element-wise step before (input preparation)
// or after (ModDown and rescale epilogues) the transform as a functor, so
// those values never make a round trip through memory; column kernels hold a
// tile of TC columns; the KeyMult kernel streams the evaluation key with
// 128-bit accesses at full occupancy. Constants are folded as in the paper's Seq. 2 (N^-1 into the
// BConv constant, 2^32 into the BConv matrix). The BConv product uses the
// paper's lazy reduction (Sec. 4.2).
#include <functional>

#include "cols.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "rows.cuh"

namespace ckks {

// The column launchers are instantiated in k_cols_*.cu.
using G16 = Geo<8, 32>;
using G12 = Geo<8, 8>;
using G8 = Geo<4, 4>;
#define CKKS_COL_DECL(G)                                                                                        \
  extern template void launch_modup_cols<G>(const DevParams&, int, int, int, int, const Scratch&, const ColShape&, \
                                            cudaStream_t);                                                      \
  extern template void launch_moddown_cols<G>(const DevParams&, int, int, int, const Scratch&, const ColShape&,      \
                                              cudaStream_t);                                                    \
  extern template void launch_rs_cols_fused<G>(const DevParams&, int, const Scratch&, uint32_t*,                \
                                               const ColShape&, cudaStream_t);                                  \
  extern template void launch_mm_cols<G>(const DevParams&, const MmArgs&, const Scratch&, const ColShape&,     \
                                         cudaStream_t);
CKKS_COL_DECL(G16)
CKKS_COL_DECL(G12)
CKKS_COL_DECL(G8)
#undef CKKS_COL_DECL

bool col_shape_supported(int log_n, int tc, int sl, int z, int tp) {
  const ColShape s{tc, sl, z, tp};
  bool ok = false;
  CKKS_DISPATCH_LOGN(log_n, { ok = shape_ok<G>(s); });
  return ok;
}


// ---------------------------------------------------------------------------
// Rescale column kernel: iNTT cols of the top limb, centered, reduced into
// every lower prime, NTT cols.
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(G::CT) k_rs_cols(DevParams dp, int n, const uint32_t* S, uint32_t* T,
                                                  int groups) {
  pdl_wait();
  pdl_trigger();
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
    const PrimeConst P = dp.pc[a.base + i];
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

// KeyMult + MAC over the D digits for extended limb t (Par. 1), positions
// p0 .. p0 + 3: the digit's own limbs are the input itself (ModUp copies
// them), the others come from the NTT'd ModUp output T[j][t]. All loads of a
// thread are issued before any product so that one memory latency covers the
// whole sum. A = [2][n + alpha][N]. With wait_dep the programmatic-dependent-
// launch wait sits after the index arithmetic and before the first load.
template <int D>
__device__ __forceinline__ void keymult_quad(const DevParams& dp, const KsArgs& a, const uint32_t* T, uint32_t* A,
                                             int t, uint32_t p0, int km_out, uint32_t* km_dst, bool wait_dep) {
  const int n = a.n, alpha = dp.alpha, L = dp.L, ext = n + alpha, ext_top = L + alpha;
  const int id = prime_of(t, n, L, a.base);
  const int key_limb = id;  // keys cover every prime: limb = global prime index
  const int g0 = a.base / alpha;  // first active digit of the window
  const PrimeConst P = dp.pc[id];
  uint32_t x[D][4], e0[D][4], e1[D][4];
  // (streaming the key before the wait kept every key word live across it:
  // 86 registers and a third of the occupancy, so the wait comes first)
  if (wait_dep) {
    pdl_wait();
    pdl_trigger();
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int lo = max(0, (g0 + j) * alpha - a.base), hi = min(n, (g0 + j + 1) * alpha - a.base);
    const uint32_t* tj = T + ((size_t)(j * ext + t) << dp.log_n);
    if (t >= lo && t < hi) {
      ks_input4(dp, a, t, p0, x[j]);
    } else if (a.hoisted) {
      // ModUp commutes with the automorphism exactly (centered BConv), so
      // phi(ModUp(a)) is a gather from the ModUp limbs of a
#pragma unroll
      for (int k = 0; k < 4; ++k) x[j][k] = __ldg(tj + auto_src(p0 + k, a.galois, dp.log_n));
    } else {
      load_vec<4>(x[j], tj + p0);
    }
  }
  if (km_out == KM_MODUP) {
#pragma unroll
    for (int j = 0; j < D; ++j) store_vec<4>(km_dst + ((size_t)(j * ext + t) << dp.log_n) + p0, x[j]);
    return;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    load_vec_stream<4>(e0[j], a.evk + ((size_t)(((g0 + j) * 2 + 0) * ext_top + key_limb) << dp.log_n) + p0);
    load_vec_stream<4>(e1[j], a.evk + ((size_t)(((g0 + j) * 2 + 1) * ext_top + key_limb) << dp.log_n) + p0);
  }
  // acc_u = sum_j x_j e_j[u] 2^-32 mod q with one reduction per output: the
  // products (x < 2^31, e < q) are summed in 64 bits, three of them at most
  // (< 3 2^62) before the sum is folded with 2^32 = mont (mod q) to below
  // 2^32 q, and again after each further product; one unsigned Montgomery
  // reduction of the folded sum gives a value below 2q (the key's Montgomery
  // factor cancels the 2^-32).
  uint32_t acc0[4], acc1[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint64_t s0 = 0, s1 = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      s0 += (uint64_t)x[j][k] * e0[j][k];
      s1 += (uint64_t)x[j][k] * e1[j][k];
      if (j >= 2) {
        s0 = fold64(s0, P.mont);
        s1 = fold64(s1, P.mont);
      }
    }
    acc0[k] = csub(csub(redc64(s0, P.q, P.m), P.q), P.q);
    acc1[k] = csub(csub(redc64(s1, P.q, P.m), P.q), P.q);
  }
  uint32_t* dst = km_out == KM_ACC_ALL ? km_dst : A;
  store_vec<4>(dst + ((size_t)t << dp.log_n) + p0, acc0);
  store_vec<4>(dst + ((size_t)(ext + t) << dp.log_n) + p0, acc1);
}

template <int D>
__global__ void k_ks_keymult(DevParams dp, KsArgs a, const uint32_t* T, uint32_t* A, int km_out,
                             uint32_t* km_dst) {
  keymult_quad<D>(dp, a, T, A, blockIdx.y, stream_pos(), km_out, km_dst, true);
}

static void launch_keymult(int digits, dim3 g, int th, cudaStream_t st, const DevParams& dp, const KsArgs& a,
                           const uint32_t* T, uint32_t* A, int km_out, uint32_t* km_dst) {
  switch (digits) {
#define CKKS_KM(D) \
  case D: launch_pdl(dp.pdl, k_ks_keymult<D>, g, dim3(th), 0, st, dp, a, T, A, km_out, km_dst); break;
    CKKS_KM(1) CKKS_KM(2) CKKS_KM(3) CKKS_KM(4) CKKS_KM(5) CKKS_KM(6) CKKS_KM(7) CKKS_KM(8)
#undef CKKS_KM
    default:
      break;
  }
}

// Linear transform, KeyMult + MAC of every rotated term in one kernel
// (Par. 5): for extended limb t,
//   acc_u[t] = sum_i pt_i[t] (.) sum_j phi_i(ModUp_j(a))[t] (.) evk_i[j][u][t],
// the automorphism read as a gather from the shared ModUp limbs of a (own
// digit limbs: from a itself). The plaintexts are in the extended basis, so
// the sum stays in Q_l P until one ModDown. A = [2][n + alpha][N].
template <int D>
__global__ void k_lt_keymult(DevParams dp, KsArgs a, LtArgs lt, const uint32_t* T, uint32_t* A) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.y;
  const int n = a.n, alpha = dp.alpha, L = dp.L, ext = n + alpha, ext_top = L + alpha;
  const int id = prime_of(t, n, L, a.base);
  const int key_limb = id;
  const int g0 = a.base / alpha;
  const PrimeConst P = dp.pc[id];
  const uint32_t p0 = stream_pos();
  const uint32_t* ain = a.x0 + a.poly_stride0 + ((size_t)t << dp.log_n);
  uint32_t acc0[4] = {0, 0, 0, 0}, acc1[4] = {0, 0, 0, 0};
  for (int i = 0; i < lt.count; ++i) {
    const uint32_t* evk = lt.evk[i];
    if (!evk) continue;
    const uint32_t g = lt.galois[i];
    uint32_t x[D][4], e0[D][4], e1[D][4], w[4];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int lo = max(0, (g0 + j) * alpha - a.base), hi = min(n, (g0 + j + 1) * alpha - a.base);
      const uint32_t* src = (t >= lo && t < hi) ? ain : T + ((size_t)(j * ext + t) << dp.log_n);
#pragma unroll
      for (int k = 0; k < 4; ++k) x[j][k] = __ldg(src + auto_src(p0 + k, g, dp.log_n));
      load_vec_stream<4>(e0[j], evk + ((size_t)(((g0 + j) * 2 + 0) * ext_top + key_limb) << dp.log_n) + p0);
      load_vec_stream<4>(e1[j], evk + ((size_t)(((g0 + j) * 2 + 1) * ext_top + key_limb) << dp.log_n) + p0);
    }
    const int pl = t < n ? t : lt.pt_p[i] + (t - n);
    load_vec<4>(w, lt.pt[i] + ((size_t)pl << dp.log_n) + p0);
    uint32_t s0[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        s0[k] = addm(s0[k], fix_signed(mont_mul(x[j][k], e0[j][k], P.q, P.m), P.q), P.q);
        s1[k] = addm(s1[k], fix_signed(mont_mul(x[j][k], e1[j][k], P.q, P.m), P.q), P.q);
      }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc0[k] = addm(acc0[k], mulmod(s0[k], w[k], P), P.q);
      acc1[k] = addm(acc1[k], mulmod(s1[k], w[k], P), P.q);
    }
  }
  store_vec<4>(A + ((size_t)t << dp.log_n) + p0, acc0);
  store_vec<4>(A + ((size_t)(ext + t) << dp.log_n) + p0, acc1);
}

static void launch_lt_keymult(int digits, dim3 g, int th, cudaStream_t st, const DevParams& dp, const KsArgs& a,
                              const LtArgs& lt, const uint32_t* T, uint32_t* A) {
  switch (digits) {
#define CKKS_LT(D) \
  case D: launch_pdl(dp.pdl, k_lt_keymult<D>, g, dim3(th), 0, st, dp, a, lt, T, A); break;
    CKKS_LT(1) CKKS_LT(2) CKKS_LT(3) CKKS_LT(4) CKKS_LT(5) CKKS_LT(6) CKKS_LT(7) CKKS_LT(8)
#undef CKKS_LT
    default:
      break;
  }
}

// Linear transform epilogue, limb i of output poly u:
//   out_0 = (A_0 - Z_0) P^-1 + sum_i pt_i (.) phi_i(b)      (accumulated automorphisms, Par. 4)
//   out_1 = (A_1 - Z_1) P^-1 + sum_{i: r_i = 0} pt_i (.) a
// ks = 0 (no rotated term): the key-switch part is zero and A, Z are not read.
__global__ void k_lt_epilogue(DevParams dp, KsArgs a, LtArgs lt, const uint32_t* Z, const uint32_t* A,
                              size_t a_stride, int ks) {
  pdl_wait();
  pdl_trigger();
  const int n = a.n;
  const int u = blockIdx.y / n, i = blockIdx.y % n;
  const PrimeConst P = dp.pc[a.base + i];
  const uint32_t p0 = stream_pos();
  const size_t off = ((size_t)i << dp.log_n) + p0;
  uint32_t z[4] = {0, 0, 0, 0};
  if (ks) {
    const uint2 pinv = dp.ks.dn_pinv[a.base + i];
    uint32_t acc[4];
    load_vec<4>(z, Z + ((size_t)(u * n + i) << dp.log_n) + p0);
    load_vec<4>(acc, A + u * a_stride + off);
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = csub(shoup(acc[k] - z[k] + P.q, pinv.x, pinv.y, P.q), P.q);
  }
  const uint32_t* src = a.x0 + u * a.poly_stride0 + ((size_t)i << dp.log_n);
  for (int t = 0; t < lt.count; ++t) {
    const bool plain = lt.evk[t] == nullptr;
    if (u == 1 && !plain) continue;
    uint32_t w[4], v[4];
    load_vec<4>(w, lt.pt[t] + off);
    if (plain) {
      load_vec<4>(v, src + p0);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldg(src + auto_src(p0 + k, lt.galois[t], dp.log_n));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = addm(z[k], mulmod(w[k], v[k], P), P.q);
  }
  store_vec<4>(a.out + u * a.out_stride + off, z);
}

// Extra term of the ModDown output at limb i (HMult: d0 or d1; HRot: phi(b)).
__device__ __forceinline__ void ks_extra4(const DevParams& dp, const KsArgs& a, int u, int i, uint32_t p0,
                                          const PrimeConst& P, uint32_t (&e)[4]) {
  const size_t off = ((size_t)i << dp.log_n) + p0;
#pragma unroll
  for (int k = 0; k < 4; ++k) e[k] = 0;
  if (a.extra == 1) {
    uint32_t b1[4], b2[4];
    load_vec<4>(b1, a.x0 + off);
    load_vec<4>(b2, a.x1 + off);
    if (u == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) e[k] = mulmod(b1[k], b2[k], P);
    } else {
      uint32_t a1[4], a2[4];
      load_vec<4>(a1, a.x0 + a.poly_stride0 + off);
      load_vec<4>(a2, a.x1 + a.poly_stride1 + off);
#pragma unroll
      for (int k = 0; k < 4; ++k) e[k] = addm(mulmod(a1[k], b2[k], P), mulmod(a2[k], b1[k], P), P.q);
    }
  } else if (a.extra == 2 && u == 0) {
    const uint32_t* sb = a.x0 + ((size_t)i << dp.log_n);
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = __ldg(sb + auto_src(p0 + k, a.galois, dp.log_n));
  }
}

// ---------------------------------------------------------------------------
// Row-kernel sources and epilogues (the streaming steps fused into the row
// phases): a thread handles positions pos0 .. pos0 + E - 1 of launch limb y,
// four at a time.
// ---------------------------------------------------------------------------

// Key-switch input before the iNTT rows: d, a1 a2 or phi_k(a) at limb y.
struct SrcKsInput {
  KsArgs a;
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      uint32_t v[4];
      ks_input4(dp, a, y, pos0 + 4 * c, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) x[4 * c + k] = v[k];
    }
  }
};

// ModDown epilogue after the NTT rows of z (launch limb y = u n + i):
// out_u[i] = (A_u[i] - z) P^-1 + extra_u[i].
// L2 prefetch of the operands an HMult epilogue reads at limb i (poly u,
// positions p0 ..): the tensor inputs d0 / d1 are formed from.
__device__ __forceinline__ void prefetch_tensor_inputs(const DevParams& dp, const KsArgs& a, int u, int i,
                                                       uint32_t p0) {
  if (a.extra != 1) return;
  const size_t off = ((size_t)i << dp.log_n) + p0;
  prefetch_l2(a.x0 + off);
  prefetch_l2(a.x1 + off);
  if (u == 1) {
    prefetch_l2(a.x0 + a.poly_stride0 + off);
    prefetch_l2(a.x1 + a.poly_stride1 + off);
  }
}

struct EpiModDown {
  KsArgs a;
  const uint32_t* A;
  size_t a_stride;
  __device__ __forceinline__ void prefetch(const DevParams& dp, int y, uint32_t pos0) const {
    const int u = y / a.n, i = y % a.n;
    prefetch_l2(A + u * a_stride + ((size_t)i << dp.log_n) + pos0);
    prefetch_tensor_inputs(dp, a, u, i, pos0);
  }
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    const int n = a.n, u = y / n, i = y % n;
    const PrimeConst P = dp.pc[a.base + i];
    const uint2 pinv = dp.ks.dn_pinv[a.base + i];
    const size_t limb = (size_t)i << dp.log_n;
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      const uint32_t p = pos0 + 4 * c;
      uint32_t acc[4], e[4], z[4];
      load_vec<4>(acc, A + u * a_stride + limb + p);
      ks_extra4(dp, a, u, i, p, P, e);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        z[k] = addm(csub(shoup(acc[k] - x[4 * c + k] + P.q, pinv.x, pinv.y, P.q), P.q), e[k], P.q);
      store_vec<4>(a.out + u * a.out_stride + limb + p, z);
    }
  }
};

// Inputs of the fused ModDown + rescale's iNTT rows: launch limbs y < 2 alpha
// are the P limbs of the two accumulators (data limb lm.x of A); limb
// 2 alpha + u is the top limb's E_u = A_u[l] P^-1 + extra_u[l] (l = n - 1, NTT
// domain, formed while loading), so that the top limb's ModDown output
// V_u = (A_u[l] - z) P^-1 + extra_u[l] = E_u - z P^-1 can be finished in the
// coefficient domain by the column kernel that converts z = BConv(P -> q_l).
struct SrcModDownTop {
  KsArgs a;
  const uint32_t* A;
  size_t a_stride;
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2 lm,
                                             uint32_t pos0) const {
    const int two_alpha = 2 * dp.alpha;
    if (y < two_alpha) {
      load_vec<E>(x, A + ((size_t)lm.x << dp.log_n) + pos0);
      return;
    }
    const int u = y - two_alpha, top = a.n - 1;
    const PrimeConst P = dp.pc[top];
    const uint2 pinv = dp.ks.dn_pinv[top];
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      const uint32_t p = pos0 + 4 * c;
      uint32_t acc[4], e[4];
      load_vec<4>(acc, A + u * a_stride + ((size_t)top << dp.log_n) + p);
      ks_extra4(dp, a, u, top, p, P, e);
#pragma unroll
      for (int k = 0; k < 4; ++k) x[4 * c + k] = addm(csub(shoup(acc[k], pinv.x, pinv.y, P.q), P.q), e[k], P.q);
    }
  }
};

// HMult's d0 = b1 b2 (u = 0) or d1 = a1 b2 + a2 b1 (u = 1) at limb i, times
// 2^-32: the 64-bit product (or sum of two, below 2 q^2 < 2^32 q) through one
// unsigned Montgomery reduction, in [0, 2q]; the caller's constant carries
// the 2^32 back.
__device__ __forceinline__ void tensor_d4_mont(const DevParams& dp, const KsArgs& a, int u, int i, uint32_t p0,
                                               const PrimeConst& P, uint32_t (&e)[4]) {
  const size_t off = ((size_t)i << dp.log_n) + p0;
  uint32_t b1[4], b2[4];
  load_vec<4>(b1, a.x0 + off);
  load_vec<4>(b2, a.x1 + off);
  if (u == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = redc64((uint64_t)b1[k] * b2[k], P.q, P.m);
  } else {
    uint32_t a1[4], a2[4];
    load_vec<4>(a1, a.x0 + a.poly_stride0 + off);
    load_vec<4>(a2, a.x1 + a.poly_stride1 + off);
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = redc64((uint64_t)a1[k] * b2[k] + (uint64_t)a2[k] * b1[k], P.q, P.m);
  }
}

// Output of the fused ModDown + rescale after the NTT rows of the conversion
// w (launch limb y = u top + i, top = l): out_u[i] = (A_u[i] - w)(P q_l)^-1 +
// extra_u[i] q_l^-1, d0/d1 re-formed from the four input limbs (at the
// three-pass rows' 24 warps per SM their loads hide: 39 us against 23 + 23
// us as rows then a streaming kernel). For HMult (extra = 1) the products are
// reduced once (tensor_d4_mont) and q_l^-1 2^32 restores their scale.
struct EpiRsOut {
  KsArgs a;
  const uint32_t* A;
  size_t a_stride;
  __device__ __forceinline__ void prefetch(const DevParams& dp, int y, uint32_t pos0) const {
    const int top = a.n - 1, u = y / top, i = y % top;
    prefetch_l2(A + u * a_stride + ((size_t)i << dp.log_n) + pos0);
    prefetch_tensor_inputs(dp, a, u, i, pos0);
  }
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    const int top = a.n - 1, u = y / top, i = y % top;
    const PrimeConst P = dp.pc[i];
    const bool mont = a.extra == 1;
    const uint2 pq = dp.ks.dn_pqinv[top * dp.L + i],
                qi = mont ? dp.ks.rs_qinv_r[top * dp.L + i] : dp.ks.rs_qinv[top * dp.L + i];
    const size_t limb = (size_t)i << dp.log_n;
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      const uint32_t p = pos0 + 4 * c;
      uint32_t acc[4], e[4], z[4];
      load_vec<4>(acc, A + u * a_stride + limb + p);
      if (mont) tensor_d4_mont(dp, a, u, i, p, P, e);
      else ks_extra4(dp, a, u, i, p, P, e);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        z[k] = addm(csub(shoup(acc[k] - x[4 * c + k] + P.q, pq.x, pq.y, P.q), P.q),
                    csub(shoup(e[k], qi.x, qi.y, P.q), P.q), P.q);
      store_vec<4>(a.out + u * a.out_stride + limb + p, z);
    }
  }
};

// Output of the merged ModDown + rescaling after the NTT rows of X (launch
// limb y = u n1 + t): out_u[t] = A_u[t'] c1 + extra_u[t'] c2 - X c3.
struct EpiMmOut {
  KsArgs a;
  MmArgs m;
  const uint32_t* A;
  size_t a_stride;
  __device__ __forceinline__ void prefetch(const DevParams& dp, int y, uint32_t pos0) const {
    const int u = y / m.n1, t = y % m.n1;
    const int old_limb = m.epi[t].old_limb;
    if (old_limb < 0) return;
    prefetch_l2(A + u * a_stride + ((size_t)old_limb << dp.log_n) + pos0);
    prefetch_tensor_inputs(dp, a, u, old_limb, pos0);
  }
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    const int u = y / m.n1, t = y % m.n1;
    const MmEpi e = m.epi[t];
    const PrimeConst P = dp.pc[m.s1 + t];
    const uint32_t q = P.q;
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      const uint32_t p = pos0 + 4 * c;
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] = csub(q - csub(shoup(x[4 * c + k], e.c3.x, e.c3.y, q), q), q);
      if (e.old_limb >= 0) {
        uint32_t acc[4], ex[4];
        load_vec<4>(acc, A + u * a_stride + ((size_t)e.old_limb << dp.log_n) + p);
        ks_extra4(dp, a, u, e.old_limb, p, P, ex);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          w[k] = addm(addm(w[k], csub(shoup(acc[k], e.c1.x, e.c1.y, q), q), q),
                      csub(shoup(ex[k], e.c2.x, e.c2.y, q), q), q);
      }
      store_vec<4>(a.out + u * a.out_stride + ((size_t)t << dp.log_n) + p, w);
    }
  }
};

// Rescale after the NTT rows of r (launch limb y = u top + i):
// out_u[i] = (c_u[i] - r) q_l^-1.
struct EpiRescale {
  const uint32_t* in;
  size_t sin;
  int top;
  uint32_t* out;
  size_t sout;
  __device__ __forceinline__ void prefetch(const DevParams& dp, int y, uint32_t pos0) const {
    prefetch_l2(in + (y / top) * sin + ((size_t)(y % top) << dp.log_n) + pos0);
  }
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    const int u = y / top, i = y % top;
    const PrimeConst P = dp.pc[i];
    const uint2 qinv = dp.ks.rs_qinv[top * dp.L + i];
    const size_t limb = (size_t)i << dp.log_n;
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      const uint32_t p = pos0 + 4 * c;
      uint32_t cv[4], z[4];
      load_vec<4>(cv, in + u * sin + limb + p);
#pragma unroll
      for (int k = 0; k < 4; ++k) z[k] = csub(shoup(cv[k] - x[4 * c + k] + P.q, qinv.x, qinv.y, P.q), P.q);
      store_vec<4>(out + u * sout + limb + p, z);
    }
  }
};

// Sources of the merged ModDown + rescaling before the iNTT rows (launch
// limb y = u K + k, accumulator limb lm.x = u ext + t): a P limb as it is; a
// dropped window limb t as Y P^-1 = A_u[t] P^-1 + extra_u[t].
struct SrcMerged {
  KsArgs a;
  const uint32_t* A;
  int ext;
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int, int2 lm,
                                             uint32_t pos0) const {
    load_vec<E>(x, A + ((size_t)lm.x << dp.log_n) + pos0);
    const int u = lm.x / ext, t = lm.x % ext;
    if (t >= a.n) return;
    const PrimeConst P = dp.pc[lm.y];
    const uint2 pinv = dp.ks.dn_pinv[lm.y];
#pragma unroll
    for (int c = 0; c < E / 4; ++c) {
      uint32_t e[4];
      ks_extra4(dp, a, u, t, pos0 + 4 * c, P, e);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        x[4 * c + k] = addm(csub(shoup(x[4 * c + k], pinv.x, pinv.y, P.q), P.q), e[k], P.q);
    }
  }
};

// Dropped limbs of a rational rescaling before the iNTT rows: launch limb
// y = 2k + u is limb drop[k].x of polynomial u.
struct SrcDrop {
  const uint32_t* in;
  size_t sin;
  const int2* drop;
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    load_vec<E>(x, in + (y & 1) * sin + ((size_t)drop[y >> 1].x << dp.log_n) + pos0);
  }
};

// Rational rescaling after the NTT rows of X (launch limb y = u n1 + i):
// out_u[i] = (c_u[i] T_add - X) T_drop^-1 mod t_i, c_u[i] taken from the old
// window (0 for an added prime).
struct EpiRational {
  RrArgs r;
  const uint32_t* in;
  size_t sin;
  uint32_t* out;
  size_t sout;
  __device__ __forceinline__ void prefetch(const DevParams& dp, int y, uint32_t pos0) const {
    const int old_limb = r.epi[y % r.n1].old_limb;
    if (old_limb >= 0) prefetch_l2(in + (y / r.n1) * sin + ((size_t)old_limb << dp.log_n) + pos0);
  }
  template <int E>
  __device__ __forceinline__ void operator()(const DevParams& dp, uint32_t (&x)[E], int y, int2,
                                             uint32_t pos0) const {
    const int u = y / r.n1, i = y % r.n1;
    const uint32_t q = dp.pc[r.s1 + i].q;
    const RrEpi e = r.epi[i];
    const uint32_t* c = e.old_limb >= 0 ? in + u * sin + ((size_t)e.old_limb << dp.log_n) : nullptr;
    uint32_t* o = out + u * sout + ((size_t)i << dp.log_n);
#pragma unroll
    for (int k4 = 0; k4 < E / 4; ++k4) {
      const uint32_t p = pos0 + 4 * k4;
      uint32_t cv[4] = {0, 0, 0, 0}, z[4];
      if (c) load_vec<4>(cv, c + p);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t a = csub(shoup(cv[k], e.ta_tdi.x, e.ta_tdi.y, q), q);
        const uint32_t b = csub(shoup(x[4 * k4 + k], e.tdi.x, e.tdi.y, q), q);
        z[k] = csub(a + q - b, q);
      }
      store_vec<4>(o + p, z);
    }
  }
};

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static int groups_for(int blocks_per_group, int max_groups, int sms) {
  const int want = 2 * sms;  // aim for two blocks per SM
  int g = (want + blocks_per_group - 1) / blocks_per_group;
  if (g > max_groups) g = max_groups;
  return g < 1 ? 1 : g;
}

// Streaming grid: four positions per thread.
static void stream_grid(int log_n, int limbs, dim3& grid, int& threads) {
  const int quads = (1 << log_n) / 4;
  threads = quads < 256 ? quads : 256;
  grid = dim3(quads / threads, limbs);
}

// Digits active at the level: the fixed groups of alpha primes that meet the
// window [base, base + n).
static int active_digits(const KsArgs& a, int alpha) { return (a.base + a.n - 1) / alpha - a.base / alpha + 1; }

// Row map of the level's n ciphertext limbs (window primes).
static LimbMap window_map(const KsArgs& a, int L) {
  LimbMap m{nullptr, 0, a.n, a.n, L};
  m.base = a.base;
  return m;
}

// ModDown fused with rescaling by q_l (l = n - 1): out gets n - 1 limbs.
template <class G>
static void moddown_rescale_tail(const DevParams& dp, const Scratch& sc, const KsArgs& a, const uint32_t* A,
                                 size_t a_stride, cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha, top = n - 1;
  uint32_t* T3 = sc.T;   // [2][top] fused conversions
  // iNTT rows of the P limbs and of E_u (SrcModDownTop), compact in S
  LimbMap in_map{nullptr, n, n + alpha, n, dp.L, alpha, (int)(a_stride >> dp.log_n)};
  in_map.tail = 2 * alpha;
  in_map.tail_prime = top;
  launch_rows_inv<G>(dp, SrcModDownTop{a, A, a_stride}, sc.S, 2 * alpha + 2, in_map, true, st);
  prof_mark(sc, st, P_MODDOWN_IN_ROWS);
  launch_rs_cols_fused<G>(dp, n, sc, T3, pick_shape<G>(sc, CK_RS_FUSED, a.tix, default_shape<G>(2, dp.sms)), st);
  prof_mark(sc, st, P_RS_COLS);
  launch_rows_fwd<G>(dp, T3, EpiRsOut{a, A, a_stride}, 2 * top, LimbMap{nullptr, 0, top, top, dp.L}, st);
  prof_mark(sc, st, P_RS_ROWS);
}

// ModDown merged into the rescaling (Sec. 6): one conversion from P and the
// dropped primes replaces the ModDown conversion, the top limb's NTT and
// iNTT, and the rescale conversion of moddown_rescale_tail.
template <class G>
static void merged_tail(const DevParams& dp, const Scratch& sc, const KsArgs& a, const uint32_t* A,
                        size_t a_stride, cudaStream_t st) {
  const MmArgs& m = *a.mm;
  const int ext = a.n + dp.alpha;
  launch_rows_inv<G>(dp, SrcMerged{a, A, ext}, sc.S, 2 * m.K, LimbMap{m.rows, 0, 0, 0, 0}, true, st);
  prof_mark(sc, st, P_MODDOWN_IN_ROWS);
  launch_mm_cols<G>(dp, m, sc, pick_shape<G>(sc, CK_RS_FUSED, a.tix, default_shape<G>(2, dp.sms)), st);
  prof_mark(sc, st, P_RS_COLS);
  LimbMap out_map{nullptr, 0, m.n1, m.n1, dp.L};
  out_map.base = m.s1;
  launch_rows_fwd<G>(dp, sc.T, EpiMmOut{a, m, A, a_stride}, 2 * m.n1, out_map, st);
  prof_mark(sc, st, P_RS_ROWS);
}

template <class G>
static void moddown_tail(const DevParams& dp, const Scratch& sc, const KsArgs& a, const uint32_t* A,
                         size_t a_stride, cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha;
  const size_t limb = (size_t)1 << dp.log_n;
  // P limbs n .. n+alpha-1 of both accumulators -> S [2][alpha] (compact)
  launch_rows_g<G>(dp, true, A, sc.S, 2 * alpha,
                   LimbMap{nullptr, n, n + alpha, n, dp.L, alpha, (int)(a_stride >> dp.log_n)}, true, st);
  prof_mark(sc, st, P_MODDOWN_IN_ROWS);
  launch_moddown_cols<G>(dp, n, a.base, a.tix, sc, pick_shape<G>(sc, CK_MODDOWN, a.tix, default_shape<G>(2, dp.sms)), st);
  prof_mark(sc, st, P_MODDOWN_COLS);
  launch_rows_fwd<G>(dp, sc.T, EpiModDown{a, A, a_stride}, 2 * n, window_map(a, dp.L), st);
  prof_mark(sc, st, P_MODDOWN_ROWS);
}

// The row-phase form the fine-tuner chose for the level (N = 2^16: two or
// three register passes), else the three-pass default.
static DevParams tuned_rows(const DevParams& dp, const Scratch& sc, int tix) {
  DevParams d = dp;
  if (sc.tune) {
    const ColShape s = sc.tune->get(CK_ROWS, tix);
    if (s.tc >= 2 && s.tc <= 6) d.rows_passes = s.tc;
  }
  return d;
}

// ModUp half of a key switch: input rows (d, a1 a2 or phi_k(a)), ModUp
// columns and ModUp NTT rows; sc.T receives the ModUp limbs (own-digit limbs
// excepted: KeyMult reads those from the input).
void launch_ks_modup(const DevParams& dp0, const Scratch& sc, const KsArgs& a, cudaStream_t st) {
  const DevParams dp = tuned_rows(dp0, sc, a.tix);
  const int digits = active_digits(a, dp.alpha);
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    launch_rows_inv<G>(dp, SrcKsInput{a}, sc.S, a.n, window_map(a, dp.L), true, st);
    prof_mark(sc, st, P_KS_IN_ROWS);
    launch_modup_cols<G>(dp, a.n, a.base, a.tix, digits, sc,
                         pick_shape<G>(sc, CK_MODUP, a.tix, default_shape<G>(digits, dp.sms)), st);
    prof_mark(sc, st, P_MODUP_COLS);
    launch_rows_g<G>(dp, false, sc.T, sc.T, a.rows_cnt, LimbMap{dp.ks.up_rows + a.rows_off, 0, 1, 0, 0}, false, st);
    prof_mark(sc, st, P_MODUP_ROWS);
  });
}

// ModDown half from the accumulators A ([2][n + alpha][N], poly stride
// a_stride words): ModDown (+ the HMult or HRot epilogue), fused with or
// merged into the rescaling when a.rescale is set.
void launch_ks_tail(const DevParams& dp0, const Scratch& sc, const KsArgs& a, const uint32_t* A, size_t a_stride,
                    cudaStream_t st) {
  const DevParams dp = tuned_rows(dp0, sc, a.tix);
  CKKS_DISPATCH_LOGN(dp.log_n, {
    if (a.rescale && a.mm) merged_tail<G>(dp, sc, a, A, a_stride, st);
    else if (a.rescale) moddown_rescale_tail<G>(dp, sc, a, A, a_stride, st);
    else moddown_tail<G>(dp, sc, a, A, a_stride, st);
  });
}

void launch_keyswitch(const DevParams& dp0, const Scratch& sc, const KsArgs& a, int km_out, uint32_t* km_dst,
                      cudaStream_t st) {
  const DevParams dp = tuned_rows(dp0, sc, a.tix);
  const int ext = a.n + dp.alpha;
  const int digits = active_digits(a, dp.alpha);
  const size_t limb = (size_t)1 << dp.log_n;
  launch_ks_modup(dp0, sc, a, st);
  dim3 g;
  int th;
  stream_grid(dp.log_n, ext, g, th);
  launch_keymult(digits, g, th, st, dp, a, sc.T, sc.A, km_out, km_dst);
  count_launch(1);
  prof_mark(sc, st, P_KEYMULT);
  if (km_out == KM_KEYSWITCH) launch_ks_tail(dp0, sc, a, sc.A, (size_t)ext * limb, st);
}

// KeyMult + MAC alone (the unfused form, k_unfused.cu): T the ModUp limbs,
// A [2][n + alpha][N] the accumulators.
void launch_keyswitch_keymult_only(const DevParams& dp, const KsArgs& a, const uint32_t* T, uint32_t* A,
                                   cudaStream_t st) {
  dim3 g;
  int th;
  stream_grid(dp.log_n, a.n + dp.alpha, g, th);
  launch_keymult(active_digits(a, dp.alpha), g, th, st, dp, a, T, A, KM_KEYSWITCH, nullptr);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// Persistent streaming stage of a batch (stage-major form, batch.cu): one
// launch runs the KeyMult + MAC (Par. 1) of every key-switching operation of
// the batch and every element-wise operation (HAdd, PAdd, PMult). Its blocks
// take work items (operation, limb) from a device queue by atomic increment
// until the queue is empty. An item runs once its operation has been
// admitted: the admitted-operation count lives in host-mapped memory and may
// be raised by the host while the kernel runs. A wait for admission is
// bounded by dp.wait_limit; when it expires the block marks the status word
// and the queue's abort flag, and every block stops at its next item. KeyMult
// items come limb-major (all operations' limb t, then limb t + 1), so the
// evaluation-key rows of a limb are read from HBM once and reused from L2 by
// every operation that uses the same key.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int load_sys_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int D>
__device__ __forceinline__ void pers_keymult(const DevParams& dp, const PersOp& o, int t) {
  for (uint32_t p0 = 4 * threadIdx.x; p0 < (1u << dp.log_n); p0 += 4 * blockDim.x)
    keymult_quad<D>(dp, o.ks, o.T, o.A, t, p0, KM_KEYSWITCH, nullptr, false);
}

// Element-wise item y = u n + i of HAdd (x + y), PAdd ((x_0 + pt, x_1)) or
// PMult (x (.) pt) at limb i of the window.
__device__ __forceinline__ void pers_elementwise(const DevParams& dp, const PersOp& o, int y) {
  const int u = y / o.n, i = y % o.n;
  const PrimeConst P = dp.pc[o.base + i];
  const size_t off = (size_t)i << dp.log_n;
  const uint32_t* x = o.x + u * o.sx + off;
  const uint32_t* w = o.y + (o.kind == PK_HADD ? u * o.sy : 0) + off;
  uint32_t* out = o.out + u * o.so + off;
  for (uint32_t p0 = 4 * threadIdx.x; p0 < (1u << dp.log_n); p0 += 4 * blockDim.x) {
    uint32_t a[4], b[4];
    load_vec<4>(a, x + p0);
    if (o.kind == PK_PADD && u == 1) {
      store_vec<4>(out + p0, a);
      continue;
    }
    load_vec<4>(b, w + p0);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = o.kind == PK_PMULT ? mulmod(a[k], b[k], P) : addm(a[k], b[k], P.q);
    store_vec<4>(out + p0, a);
  }
}

__global__ void __launch_bounds__(256) k_persistent(DevParams dp, const PersOp* ops, const int2* items, int n_items,
                                                    int* q, const int* admitted) {
  __shared__ int s_it;
  int known = 0;  // thread 0: admitted count last read
  for (;;) {
    if (threadIdx.x == 0) {
      int it = atomicAdd(&q[0], 1);
      if (it >= n_items || *(volatile int*)&q[1]) {
        it = -1;
      } else {
        const int op = items[it].x;
        if (known <= op) known = load_sys_relaxed(admitted);
        if (known <= op) {
          const long long t0 = clock64();
          for (;;) {
            __nanosleep(200);
            known = load_sys_relaxed(admitted);
            if (known > op) break;
            if (*(volatile int*)&q[1]) {
              it = -1;
              break;
            }
            if (clock64() - t0 > dp.wait_limit) {
              tc::report_timeout(dp.status);
              atomicExch(&q[1], 1);
              it = -1;
              break;
            }
          }
        }
      }
      s_it = it;
    }
    __syncthreads();
    const int it = s_it;
    __syncthreads();
    if (it < 0) return;
    const int2 w = items[it];
    const PersOp& o = ops[w.x];
    if (o.kind == PK_KEYMULT) {
      switch (o.digits) {
#define CKKS_PK(D) \
  case D: pers_keymult<D>(dp, o, w.y); break;
        CKKS_PK(1) CKKS_PK(2) CKKS_PK(3) CKKS_PK(4) CKKS_PK(5) CKKS_PK(6) CKKS_PK(7) CKKS_PK(8)
#undef CKKS_PK
        default:
          break;
      }
    } else {
      pers_elementwise(dp, o, w.y);
    }
  }
}

void launch_persistent(const DevParams& dp, const PersOp* ops, const int2* items, int n_items, int* q,
                       const int* admitted, int blocks, cudaStream_t st) {
  k_persistent<<<blocks, 256, 0, st>>>(dp, ops, items, n_items, q, admitted);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// Software fine-tuner for the column kernels (Sec. 4.2, "Fine-tuning"): for
// the level with n limbs, time every candidate shape of each kernel (reps
// launches per shape, CUDA events on st) and record the fastest. The kernels
// run on the lane's scratch exactly as inside an operation; they read what
// the scratch holds (their time does not depend on the values) and write
// only scratch.
// ---------------------------------------------------------------------------

template <class G>
static std::vector<ColShape> shape_candidates(int targets, const ColShape& def, bool tensor) {
  std::vector<ColShape> v;
  if (tensor)
    for (int tc : {8, 4})
      for (int sl : {2, 4, 8})
        for (int nc : {8, 16}) {
          const ColShape c{tc, sl, 1, nc};
          if (tc_shape_ok<G>(c)) v.push_back(c);
        }
  for (int tc : {8, 4}) {
    if (G::W % tc != 0) continue;
    for (int sl : {2, 4, 8})
      for (int z = 1; z <= 4; ++z)
        for (int tp = 1; tp <= 2; ++tp) {
          const ColShape c{tc, sl, z, tp};
          const bool is_def = tc == def.tc && sl == def.sl && z == def.z && tp == def.tp;
          if (!shape_ok<G>(c)) continue;
          if (sl * z * tp > targets && !is_def) continue;  // some slices would have no target
          v.push_back(c);
        }
  }
  return v;
}

int tune_columns(const DevParams& dp, const Scratch& sc, Tuning& tu, const KsArgs& lvl, int reps, cudaStream_t st) {
  const int n = lvl.n, base = lvl.base, tix = lvl.tix;
  if (n < 1 || n > dp.L || reps < 1) return CKKS_EINVAL;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CKKS_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CKKS_ECUDA;
  }
  int rc = CKKS_OK;
  const size_t limb = (size_t)1 << dp.log_n;
  const int alpha = dp.alpha, digits = active_digits(lvl, alpha);
  CKKS_DISPATCH_LOGN(dp.log_n, {
    for (int k = 0; k < CK_COUNT && rc == CKKS_OK; ++k) {
      if (k == CK_RS_FUSED && (n < 2 || base != 0)) continue;  // single rescaling only
      ColShape def;
      int targets;
      const bool tensor =
          dp.tune_tensor && dp.ks.tc_img != nullptr && dp.alpha + (k == CK_RS_FUSED ? 1 : 0) <= kTcMaxSources;
      std::function<void(const ColShape&)> run;
      if (k == CK_MODUP) {
        def = default_shape<G>(digits, dp.sms);
        targets = n;  // fewest targets of a digit: n + alpha - (digit size)
        run = [&](const ColShape& s) { launch_modup_cols<G>(dp, n, base, tix, digits, sc, s, st); };
      } else if (k == CK_MODDOWN) {
        def = default_shape<G>(2, dp.sms);
        targets = n;
        run = [&](const ColShape& s) { launch_moddown_cols<G>(dp, n, base, tix, sc, s, st); };
      } else {
        def = default_shape<G>(2, dp.sms);
        targets = n - 1;
        run = [&](const ColShape& s) {
          launch_rs_cols_fused<G>(dp, n, sc, sc.T, s, st);
        };
      }
      ColShape best = def;
      float best_ms = -1.f;
      for (const ColShape& s : shape_candidates<G>(targets, def, tensor)) {
        run(s);  // first launch: attributes, instruction cache
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) run(s);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = CKKS_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
          best_ms = ms;
          best = s;
        }
      }
      if (rc == CKKS_OK) tu.set(k, tix, best, 1e3f * best_ms / reps);
    }
    // row phase at N = 2^16: two or three register passes, timed on the
    // level's ModUp NTT rows (in place on the scratch, like the columns)
    if constexpr (G::W == 1024) {
      int best_p = 3;
      float best_ms = -1.f;
      for (int passes : {3, 2, 4, 5}) {  // form 6 (twiddles in shared memory): by hand only
        if (rc != CKKS_OK || lvl.rows_cnt < 1) break;
        DevParams dv = dp;
        dv.rows_passes = passes;
        auto run = [&]() {
          launch_rows_g<G>(dv, false, sc.T, sc.T, lvl.rows_cnt, LimbMap{dp.ks.up_rows + lvl.rows_off, 0, 1, 0, 0},
                           false, st);
        };
        run();
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) run();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = CKKS_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
          best_ms = ms;
          best_p = passes;
        }
      }
      if (rc == CKKS_OK && best_ms >= 0.f) tu.set(CK_ROWS, tix, ColShape{best_p, 1, 1, 1}, 1e3f * best_ms / reps);
    }
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == CKKS_OK && cudaGetLastError() != cudaSuccess) rc = CKKS_ECUDA;
  return rc;
}

// Hoisted rotations of one ciphertext (Par. 5): ModUp of its a part once
// (iNTT rows straight from the ciphertext, ModUp columns, NTT rows), then for
// each rotation KeyMult with phi_k applied while loading the ModUp limbs,
// ModDown and the epilogue adding phi_k(b). The ModDown conversions use the
// scratch after the ModUp limbs so that those stay intact for the next
// rotation. Bit-identical to one full key switch per rotation.
void launch_hoisted_rotations(const DevParams& dp0, const Scratch& sc, const KsArgs* rots, int count,
                              cudaStream_t st) {
  if (count < 1) return;
  const KsArgs& a0 = rots[0];
  const DevParams dp = tuned_rows(dp0, sc, a0.tix);
  const int n = a0.n, alpha = dp.alpha, ext = n + alpha;
  const int digits = active_digits(a0, alpha);
  const size_t limb = (size_t)1 << dp.log_n;
  Scratch down = sc;
  down.T = sc.T + (size_t)digits * ext * limb;
  dim3 g;
  int th;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    launch_rows_g<G>(dp, true, a0.x0 + a0.poly_stride0, sc.S, n, window_map(a0, dp.L), true, st);
    prof_mark(sc, st, P_KS_IN_ROWS);
    launch_modup_cols<G>(dp, n, a0.base, a0.tix, digits, sc,
                         pick_shape<G>(sc, CK_MODUP, a0.tix, default_shape<G>(digits, dp.sms)), st);
    prof_mark(sc, st, P_MODUP_COLS);
    launch_rows_g<G>(dp, false, sc.T, sc.T, a0.rows_cnt, LimbMap{dp.ks.up_rows + a0.rows_off, 0, 1, 0, 0}, false,
                     st);
    prof_mark(sc, st, P_MODUP_ROWS);
    for (int i = 0; i < count; ++i) {
      stream_grid(dp.log_n, ext, g, th);
      launch_keymult(digits, g, th, st, dp, rots[i], sc.T, sc.A, KM_KEYSWITCH, nullptr);
      count_launch(1);
      prof_mark(sc, st, P_KEYMULT);
      moddown_tail<G>(dp, down, rots[i], sc.A, (size_t)ext * limb, st);
    }
  });
}

// Linear transform (Par. 5): ModUp of a once, KeyMult + MAC of all rotated
// terms with their extended plaintexts in one kernel, one ModDown of the
// sum, and the epilogue adding the plaintext-weighted automorphisms of b
// (and pt (.) a for unrotated terms).
void launch_linear_transform(const DevParams& dp0, const Scratch& sc, const KsArgs& a, const LtArgs& lt,
                             cudaStream_t st) {
  const DevParams dp = tuned_rows(dp0, sc, a.tix);
  const int n = a.n, alpha = dp.alpha, ext = n + alpha;
  const int digits = active_digits(a, alpha);
  const size_t limb = (size_t)1 << dp.log_n;
  Scratch down = sc;
  down.T = sc.T + (size_t)digits * ext * limb;
  dim3 g;
  int th;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    if (lt.rotated > 0) {
      launch_rows_g<G>(dp, true, a.x0 + a.poly_stride0, sc.S, n, window_map(a, dp.L), true, st);
      prof_mark(sc, st, P_KS_IN_ROWS);
      launch_modup_cols<G>(dp, n, a.base, a.tix, digits, sc,
                           pick_shape<G>(sc, CK_MODUP, a.tix, default_shape<G>(digits, dp.sms)), st);
      prof_mark(sc, st, P_MODUP_COLS);
      launch_rows_g<G>(dp, false, sc.T, sc.T, a.rows_cnt, LimbMap{dp.ks.up_rows + a.rows_off, 0, 1, 0, 0}, false,
                       st);
      prof_mark(sc, st, P_MODUP_ROWS);
      stream_grid(dp.log_n, ext, g, th);
      launch_lt_keymult(digits, g, th, st, dp, a, lt, sc.T, sc.A);
      count_launch(1);
      prof_mark(sc, st, P_KEYMULT);
      const size_t a_stride = (size_t)ext * limb;
      launch_rows_g<G>(dp, true, sc.A, down.S, 2 * alpha,
                       LimbMap{nullptr, n, n + alpha, n, dp.L, alpha, (int)(a_stride >> dp.log_n)}, true, st);
      prof_mark(sc, st, P_MODDOWN_IN_ROWS);
      launch_moddown_cols<G>(dp, n, a.base, a.tix, down, pick_shape<G>(sc, CK_MODDOWN, a.tix, default_shape<G>(2, dp.sms)), st);
      prof_mark(sc, st, P_MODDOWN_COLS);
      launch_rows_g<G>(dp, false, down.T, down.T, 2 * n, window_map(a, dp.L), false, st);
      prof_mark(sc, st, P_MODDOWN_ROWS);
    }
    stream_grid(dp.log_n, 2 * n, g, th);
    launch_pdl(dp.pdl, k_lt_epilogue, g, dim3(th), 0, st, dp, a, lt, (const uint32_t*)down.T, (const uint32_t*)sc.A,
               (size_t)ext * limb, lt.rotated > 0 ? 1 : 0);
    count_launch(1);
    prof_mark(sc, st, P_KS_EPILOGUE);
  });
}

// Rational rescaling (Sec. 3.1, Sec. 3.2, Sec. 5.1): iNTT rows of each
// dropped limb of both polynomials (S = [K][2]), the conversion column
// kernel (T = [2][n1]), NTT rows with the epilogue. `in` is [2][n0] limbs of
// the old window (poly stride sin words), `out` [2][n1] of the new one.
void launch_rational_rescale(const DevParams& dp, const Scratch& sc, const RrArgs& r, const uint32_t* in,
                             size_t sin, uint32_t* out, size_t sout, cudaStream_t st) {
  CKKS_DISPATCH_LOGN(dp.log_n, {
    prof_mark(sc, st, -1);
    if (r.K > 0) {
      // every dropped limb of both polynomials: launch limb y = 2k + u -> S[y]
      launch_rows_inv<G>(dp, SrcDrop{in, sin, r.drop}, sc.S, 2 * r.K, LimbMap{r.rows, 0, 1, 0, 0}, true, st);
      prof_mark(sc, st, P_RS_IN_ROWS);
      launch_rr_cols<G>(dp, r, sc, st);
      prof_mark(sc, st, P_RS_COLS);
    }
    LimbMap m{nullptr, 0, r.n1, r.n1, dp.L};
    m.base = r.s1;
    launch_rows_fwd<G>(dp, sc.T, EpiRational{r, in, sin, out, sout}, 2 * r.n1, m, st);
    prof_mark(sc, st, P_RS_ROWS);
  });
}

void launch_moddown(const DevParams& dp, const Scratch& sc, const uint32_t* acc, int n, uint32_t* out,
                    cudaStream_t st) {
  KsArgs a{};
  a.n = n;
  a.tix = n;
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
    const int gr = groups_for(tiles * 2, top, dp.sms);
    launch_pdl(dp.pdl, k_rs_cols<G>, dim3(tiles, 2, gr), dim3(G::CT), 0, st, dp, n, (const uint32_t*)sc.S, sc.T, gr);
    count_launch(1);
    prof_mark(sc, st, P_RS_COLS);
    launch_rows_fwd<G>(dp, sc.T, EpiRescale{in, sin, top, out, sout}, 2 * top, LimbMap{nullptr, 0, top, top, dp.L},
                       st);
    prof_mark(sc, st, P_RS_ROWS);
  });
}

}  // namespace ckks
