// Unfused form of HMult (+ rescale), HRot and HConj: every step of the key
// switch (Sec. 2.3) as its own kernel launch with every intermediate in
// device memory, the one-operation-per-kernel mechanism baseline of the
// paper's fusion ablation (Sec. 5, Table 8): tensor, full iNTT of d2 (row
// and column launches), one BConv launch per ModUp digit (Eq. 2), full NTTs
// of the converted limbs, KeyMult + MAC, full iNTT of the P limbs, BConv
// P -> Q, full NTT, the ModDown epilogue, and for rescaling the iNTT of the
// top limb, its reduction into every lower prime, NTT and the rescale
// epilogue. Same arithmetic as the fused pipeline, so the residues are
// identical (CKKS_LAUNCH_UNFUSED).
#include <algorithm>

#include "geo.cuh"
#include "internal.h"

namespace ckks {

namespace {

__device__ __forceinline__ uint32_t uf_add(uint32_t a, uint32_t b, uint32_t q) { return csub(a + b, q); }

__device__ __forceinline__ uint32_t uf_pos() { return 4 * (blockIdx.x * blockDim.x + threadIdx.x); }

// d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 (Sec. 2.1) -> D [3][n].
__global__ void k_uf_tensor(DevParams dp, const uint32_t* c1, const uint32_t* c2, size_t s1, size_t s2, uint32_t* D,
                            int n) {
  const int i = blockIdx.y;
  const PrimeConst P = dp.pc[i];
  const size_t off = ((size_t)i << dp.log_n) + uf_pos(), poly = (size_t)n << dp.log_n;
  uint32_t b1[4], a1[4], b2[4], a2[4], d0[4], d1[4], d2[4];
  load_vec<4>(b1, c1 + off);
  load_vec<4>(a1, c1 + s1 + off);
  load_vec<4>(b2, c2 + off);
  load_vec<4>(a2, c2 + s2 + off);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d0[k] = mulmod(b1[k], b2[k], P);
    d1[k] = uf_add(mulmod(a1[k], b2[k], P), mulmod(a2[k], b1[k], P), P.q);
    d2[k] = mulmod(a1[k], a2[k], P);
  }
  store_vec<4>(D + off, d0);
  store_vec<4>(D + poly + off, d1);
  store_vec<4>(D + 2 * poly + off, d2);
}

// BConv (Eq. 2) of K coefficient-domain source limbs (prime ids src(k)) to
// the targets t of one launch: out limb t (prime dst(t)) = sum_k y_k mat[t][k]
// with y_k = centered([x_k (Q/q_k)^-1]_{q_k}); cin holds N^-1 (Q/q_k)^-1 as
// in the fused tables, so N is multiplied back (the standalone iNTT already
// applied N^-1). Lazy 64-bit sums with a range fold every four products.
// up_ix >= 0: the ModUp tables of entry up_ix (level table index * dnum +
// digit) of the device offset table; up_ix < 0: the ModDown tables.
__global__ void k_uf_bconv(DevParams dp, const uint32_t* in, int K, IdMap src, int up_ix, int mat_stride,
                           uint32_t* out, int M, IdMap dst, int skip_lo, int skip_hi) {
  const int n = 1 << dp.log_n;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const uint2* cin = dp.ks.dn_cin;
  const int32_t* mat = dp.ks.dn_mat;
  if (up_ix >= 0) {
    const int2 off = dp.ks.up_off[up_ix];
    cin = dp.ks.up_cin + off.x;
    mat = dp.ks.up_mat + off.y;
  }
  int32_t y[64];
  for (int k = 0; k < K; ++k) {
    const PrimeConst Q = dp.pc[src(k)];
    const uint32_t w = mulmod(cin[k].x, (uint32_t)n % Q.q, Q);
    y[k] = centered(mulmod(in[(size_t)k * n + c], w, Q), Q.q);
  }
  for (int t = 0; t < M; ++t) {
    if (t >= skip_lo && t < skip_hi) continue;
    const PrimeConst P = dp.pc[dst(t)];
    const int64_t lim = (int64_t)P.q << 31, wrap = (int64_t)P.q << 32;
    int64_t acc = 0;
    for (int k = 0; k < K; ++k) {
      acc += (int64_t)y[k] * (int64_t)mat[(size_t)t * mat_stride + k];
      if ((k & 3) == 3) acc = acc >= lim ? acc - wrap : (acc < -lim ? acc + wrap : acc);
    }
    acc = acc >= lim ? acc - wrap : (acc < -lim ? acc + wrap : acc);
    out[(size_t)t * n + c] = fix_signed(smr(acc, P.q, P.m), P.q);
  }
}

// ModDown epilogue: out_u[i] = (A_u[i] - Z_u[i]) P^-1 + E_u[i] (E optional).
__global__ void k_uf_moddown_epi(DevParams dp, const uint32_t* A, size_t a_stride, const uint32_t* Z, int n,
                                 const uint32_t* E, size_t e_stride, uint32_t* out, size_t o_stride) {
  const int u = blockIdx.y / n, i = blockIdx.y % n;
  const PrimeConst P = dp.pc[i];
  const uint2 pinv = dp.ks.dn_pinv[i];
  const size_t off = ((size_t)i << dp.log_n) + uf_pos();
  uint32_t a[4], z[4], e[4] = {0, 0, 0, 0};
  load_vec<4>(a, A + u * a_stride + off);
  load_vec<4>(z, Z + ((size_t)(u * n) << dp.log_n) + off);
  if (E) load_vec<4>(e, E + u * e_stride + off);
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = uf_add(csub(shoup(a[k] - z[k] + P.q, pinv.x, pinv.y, P.q), P.q), e[k], P.q);
  store_vec<4>(out + u * o_stride + off, a);
}

// Rescale, reduction step: W_u[i] = centered(R_u) mod q_i for i < top (R_u
// the coefficient-domain top limb of polynomial u).
__global__ void k_uf_rs_reduce(DevParams dp, const uint32_t* R, int top, uint32_t* W) {
  const int u = blockIdx.y / top, i = blockIdx.y % top;
  const uint32_t ql = dp.pc[top].q, qi = dp.pc[i].q;
  const uint32_t p0 = uf_pos();
  uint32_t r[4], w[4];
  load_vec<4>(r, R + ((size_t)u << dp.log_n) + p0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int64_t v = centered(r[k], ql) % (int64_t)qi;
    w[k] = (uint32_t)(v < 0 ? v + qi : v);
  }
  store_vec<4>(W + ((size_t)(u * top + i) << dp.log_n) + p0, w);
}

// Rescale epilogue: out_u[i] = (V_u[i] - W_u[i]) q_l^-1.
__global__ void k_uf_rs_epi(DevParams dp, const uint32_t* V, size_t v_stride, const uint32_t* W, int top,
                            uint32_t* out, size_t o_stride) {
  const int u = blockIdx.y / top, i = blockIdx.y % top;
  const PrimeConst P = dp.pc[i];
  const uint2 qinv = dp.ks.rs_qinv[top * dp.L + i];
  const size_t off = ((size_t)i << dp.log_n) + uf_pos();
  uint32_t v[4], w[4];
  load_vec<4>(v, V + u * v_stride + off);
  load_vec<4>(w, W + ((size_t)(u * top) << dp.log_n) + off);
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = csub(shoup(v[k] - w[k] + P.q, qinv.x, qinv.y, P.q), P.q);
  store_vec<4>(out + u * o_stride + off, v);
}

dim3 uf_grid(int log_n, int limbs) { return dim3(((1 << log_n) / 4 + 255) / 256, limbs); }
int uf_threads(int log_n) { return (1 << log_n) / 4 < 256 ? (1 << log_n) / 4 : 256; }

void uf_copy(uint32_t* dst, const uint32_t* src, size_t words, cudaStream_t st) {
  cudaMemcpyAsync(dst, src, words * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
}

}  // namespace

size_t unfused_scratch_words(const DevParams& dp) {
  const size_t limb = (size_t)1 << dp.log_n, L = dp.L, ext = dp.L + dp.alpha;
  // D [3][L] (+ NTT-domain copy of d2 [L]), T [dnum][ext], A [2][ext], S [2][alpha],
  // Z [2][L], V [2][L], R [2], W [2][L]
  return (4 * L + dp.dnum * ext + 2 * ext + 2 * dp.alpha + 6 * L + 2) * limb;
}

// a: the fused form's key-switch arguments (KS_TENSOR with extra = 1 for
// HMult, KS_AUTO with extra = 2 for HRot / HConj; a.rescale selects the
// rescaling of HMult); W: unfused_scratch_words(dp) words of device memory.
void launch_keyswitch_unfused(const DevParams& dp, const KsArgs& a, uint32_t* W, cudaStream_t st) {
  const int n = a.n, alpha = dp.alpha, L = dp.L, ext = n + alpha, log_n = dp.log_n;
  const size_t limb = (size_t)1 << log_n;
  const int digits = (n + alpha - 1) / alpha;
  uint32_t* D = W;                          // [3][n]: d0, d1, d2 (HMult); phi(b), -, phi(a) (HRot)
  uint32_t* D2n = D + 3 * (size_t)L * limb;  // NTT-domain copy of d2 / phi(a)
  uint32_t* T = D2n + (size_t)L * limb;      // [digits][ext]
  uint32_t* A = T + (size_t)dp.dnum * (L + alpha) * limb;  // [2][ext]
  uint32_t* S = A + 2 * (size_t)(L + alpha) * limb;         // [2][alpha]
  uint32_t* Z = S + 2 * (size_t)alpha * limb;              // [2][n]
  uint32_t* V = Z + 2 * (size_t)L * limb;                  // [2][n]
  uint32_t* R = V + 2 * (size_t)L * limb;                  // [2]
  uint32_t* Wr = R + 2 * limb;                             // [2][n - 1]
  const size_t poly = (size_t)n * limb;
  const int th = uf_threads(log_n);
  // input: d2 (HMult) or phi_k(a) (HRot); E: the ModDown epilogue's extra term
  const uint32_t* E = nullptr;
  size_t e_stride = 0;
  if (a.mode == KS_TENSOR) {
    k_uf_tensor<<<uf_grid(log_n, n), th, 0, st>>>(dp, a.x0, a.x1, a.poly_stride0, a.poly_stride1, D, n);
    count_launch(1);
    E = D;
    e_stride = poly;
  } else {
    launch_automorph(dp, a.x0, D, n, a.galois, st);                         // phi(b)
    launch_automorph(dp, a.x0 + a.poly_stride0, D + 2 * poly, n, a.galois, st);  // phi(a)
    E = D;
    e_stride = 0;  // only u = 0 gets phi(b): handled by two epilogue launches below
  }
  uint32_t* d2 = D + 2 * poly;
  uf_copy(D2n, d2, poly, st);
  launch_ntt(dp, d2, n, id_ct(n, L), true, st);
  // ModUp: per digit, BConv of its coefficient-domain limbs to every other
  // extended limb, then the NTT of those limbs (before and after the digit)
  for (int j = 0; j < digits; ++j) {
    const int lo = j * alpha, hi = std::min(n, (j + 1) * alpha), K = hi - lo;
    uint32_t* Tj = T + (size_t)j * ext * limb;
    IdMap src{nullptr, 1 << 30, 1 << 30, L, lo};
    k_uf_bconv<<<((int)limb + 127) / 128, 128, 0, st>>>(dp, d2 + (size_t)lo * limb, K, src, a.tix * dp.dnum + j,
                                                        K, Tj, ext, id_ext(n, L, alpha), lo, hi);
    count_launch(1);
    if (lo > 0) launch_ntt(dp, Tj, lo, IdMap{nullptr, lo, lo, L, 0}, false, st);
    launch_ntt(dp, Tj + (size_t)hi * limb, ext - hi, IdMap{nullptr, ext - hi, n - hi, L, hi}, false, st);
  }
  // KeyMult + MAC (own-digit limbs from the NTT-domain input)
  KsArgs km = a;
  km.mode = KS_PLAIN;
  km.x0 = D2n;
  km.hoisted = 0;
  launch_keyswitch_keymult_only(dp, km, T, A, st);
  // ModDown: iNTT of the P limbs, BConv P -> Q, NTT, epilogue
  const size_t a_stride = (size_t)ext * limb;
  for (int u = 0; u < 2; ++u) uf_copy(S + (size_t)u * alpha * limb, A + u * a_stride + poly, (size_t)alpha * limb, st);
  launch_ntt(dp, S, 2 * alpha, IdMap{nullptr, alpha, 0, L, 0}, true, st);
  for (int u = 0; u < 2; ++u) {
    k_uf_bconv<<<((int)limb + 127) / 128, 128, 0, st>>>(dp, S + (size_t)u * alpha * limb, alpha,
                                                        IdMap{nullptr, 1 << 30, 0, L, 0}, -1, alpha,
                                                        Z + (size_t)u * poly, n, id_ct(n, L), 0, 0);
    count_launch(1);
  }
  launch_ntt(dp, Z, 2 * n, id_ct(n, L), false, st);
  uint32_t* dst = a.rescale ? V : a.out;
  const size_t d_stride = a.rescale ? poly : a.out_stride;
  if (a.mode == KS_TENSOR) {
    k_uf_moddown_epi<<<uf_grid(log_n, 2 * n), th, 0, st>>>(dp, A, a_stride, Z, n, E, e_stride, dst, d_stride);
    count_launch(1);
  } else {
    // out_0 = (A_0 - Z_0) P^-1 + phi(b), out_1 = (A_1 - Z_1) P^-1
    k_uf_moddown_epi<<<uf_grid(log_n, n), th, 0, st>>>(dp, A, a_stride, Z, n, E, 0, dst, d_stride);
    k_uf_moddown_epi<<<uf_grid(log_n, n), th, 0, st>>>(dp, A + a_stride, 0, Z + poly, n, nullptr, 0,
                                                       dst + d_stride, 0);
    count_launch(2);
  }
  if (!a.rescale) return;
  // rescale: iNTT of the top limb of both polynomials, reduction into the
  // lower primes, NTT, (V - W) q_l^-1
  const int top = n - 1;
  for (int u = 0; u < 2; ++u) uf_copy(R + (size_t)u * limb, V + u * poly + (size_t)top * limb, limb, st);
  launch_ntt(dp, R, 2, IdMap{nullptr, 1, 1, L, top}, true, st);
  k_uf_rs_reduce<<<uf_grid(log_n, 2 * top), th, 0, st>>>(dp, R, top, Wr);
  count_launch(1);
  launch_ntt(dp, Wr, 2 * top, id_ct(top, L), false, st);
  k_uf_rs_epi<<<uf_grid(log_n, 2 * top), th, 0, st>>>(dp, V, poly, Wr, top, a.out, a.out_stride);
  count_launch(1);
}

}  // namespace ckks
