// Standalone transforms and element-wise kernels (Sec. 2.2 NTT, element-wise
// operations, Eq. 4 automorphism; Alg. 2 SMR).
#include "geo.cuh"
#include "internal.h"
#include "tc.cuh"

#include <atomic>

namespace ckks {

static std::atomic<uint64_t> g_launches{0};
uint64_t launch_count() { return g_launches.load(); }
void count_launch(int k) { g_launches += (uint64_t)k; }

void Prof::mark(cudaStream_t st, int id) {
  if (used == ev.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ev.push_back(e);
    ids.push_back(id);
  }
  ids[used] = id;
  cudaEventRecord(ev[used], st);
  ++used;
}

// ---------------------------------------------------------------------------
// Standalone NTT / iNTT, in place on [limbs][N]
// ---------------------------------------------------------------------------

template <class G>
__global__ void __launch_bounds__(G::CT) k_cols_fwd(DevParams dp, uint32_t* data, IdMap ids) {
  __shared__ uint32_t buf[G::COLBUF];
  const int c = threadIdx.x % G::TC, jj = threadIdx.x / G::TC;
  const int l = blockIdx.x * G::TC + c;
  const int limb = blockIdx.y, id = ids(limb);
  const uint32_t q = dp.pc[id].q;
  const uint2* tw = dp.tw + ((size_t)id << dp.log_n);
  uint32_t* d = data + ((size_t)limb << dp.log_n);
  uint32_t x[G::EC];
#pragma unroll
  for (int i = 0; i < G::EC; ++i) x[i] = d[(jj + G::EC * i) * G::W + l];
  if (q < (1u << 30)) col_fwd<G::EC, G::TC, true>(x, buf, tw, jj, c, q);
  else col_fwd<G::EC, G::TC, false>(x, buf, tw, jj, c, q);
#pragma unroll
  for (int i = 0; i < G::EC; ++i) d[(G::EC * jj + i) * G::W + l] = x[i];
}

template <class G>
__global__ void __launch_bounds__(G::RT) k_rows_fwd(DevParams dp, uint32_t* data, IdMap ids) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int limb = blockIdx.y, id = ids(limb);
  const uint32_t q = dp.pc[id].q;
  const uint2* tw = dp.tw + ((size_t)id << dp.log_n);
  uint32_t* row = data + ((size_t)limb << dp.log_n) + (size_t)h * G::W;
  uint32_t* b = buf + r * G::ROWBUF;
  uint32_t x[G::ER];
#pragma unroll
  for (int i = 0; i < G::ER; ++i) x[i] = row[jj + G::ER * i];
  if (q < (1u << 30)) {
    row_fwd<G::ER, G::H, true>(x, b, tw, h, jj, q);
#pragma unroll
    for (int i = 0; i < G::ER; ++i) x[i] = normalize<true>(x[i], q);
  } else {
    row_fwd<G::ER, G::H, false>(x, b, tw, h, jj, q);
#pragma unroll
    for (int i = 0; i < G::ER; ++i) x[i] = normalize<false>(x[i], q);
  }
  store_vec<G::ER>(row + G::ER * jj, x);
}

template <class G>
__global__ void __launch_bounds__(G::RT) k_rows_inv(DevParams dp, uint32_t* data, IdMap ids) {
  __shared__ uint32_t buf[G::RPC * G::ROWBUF];
  const int r = threadIdx.x / G::ER, jj = threadIdx.x % G::ER;
  const int h = blockIdx.x * G::RPC + r;
  const int limb = blockIdx.y, id = ids(limb);
  const uint32_t q = dp.pc[id].q;
  const uint2* itw = dp.itw + ((size_t)id << dp.log_n);
  uint32_t* row = data + ((size_t)limb << dp.log_n) + (size_t)h * G::W;
  uint32_t* b = buf + r * G::ROWBUF;
  uint32_t x[G::ER];
  load_vec<G::ER>(x, row + G::ER * jj);
  if (q < (1u << 30)) row_inv<G::ER, G::H, true>(x, b, itw, h, jj, q);
  else row_inv<G::ER, G::H, false>(x, b, itw, h, jj, q);
#pragma unroll
  for (int i = 0; i < G::ER; ++i) row[jj + G::ER * i] = x[i];
}

template <class G>
__global__ void __launch_bounds__(G::CT) k_cols_inv(DevParams dp, uint32_t* data, IdMap ids) {
  __shared__ uint32_t buf[G::COLBUF];
  const int c = threadIdx.x % G::TC, jj = threadIdx.x / G::TC;
  const int l = blockIdx.x * G::TC + c;
  const int limb = blockIdx.y, id = ids(limb);
  const PrimeConst P = dp.pc[id];
  const uint2* itw = dp.itw + ((size_t)id << dp.log_n);
  uint32_t* d = data + ((size_t)limb << dp.log_n);
  uint32_t x[G::EC];
#pragma unroll
  for (int i = 0; i < G::EC; ++i) x[i] = d[(G::EC * jj + i) * G::W + l];
  if (P.q < (1u << 30)) col_inv<G::EC, G::TC, true>(x, buf, itw, jj, c, P.q);
  else col_inv<G::EC, G::TC, false>(x, buf, itw, jj, c, P.q);
#pragma unroll
  for (int i = 0; i < G::EC; ++i)
    d[(jj + G::EC * i) * G::W + l] = csub(shoup(x[i], P.ninv, P.ninv_sh, P.q), P.q);
}

void launch_ntt(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, bool inverse, cudaStream_t st) {
  if (limbs <= 0) return;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    dim3 gc(G::W / G::TC, limbs), gr(G::H / G::RPC, limbs);
    if (!inverse) {
      k_cols_fwd<G><<<gc, G::CT, 0, st>>>(dp, data, ids);
      k_rows_fwd<G><<<gr, G::RT, 0, st>>>(dp, data, ids);
    } else {
      k_rows_inv<G><<<gr, G::RT, 0, st>>>(dp, data, ids);
      k_cols_inv<G><<<gc, G::CT, 0, st>>>(dp, data, ids);
    }
    count_launch(2);
  });
}

void launch_rows_inv_only(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, cudaStream_t st) {
  if (limbs <= 0) return;
  CKKS_DISPATCH_LOGN(dp.log_n, {
    k_rows_inv<G><<<dim3(G::H / G::RPC, limbs), G::RT, 0, st>>>(dp, data, ids);
    count_launch(1);
  });
}

// ---------------------------------------------------------------------------
// Layout permutation: internal (bit-reversed NTT order) <-> canonical. The
// bit reversal is an involution, so one kernel serves both directions.
// ---------------------------------------------------------------------------

// Bit-reversal permutation of each limb (an involution): out[p] = in[brev(p)].
// A position of log_n = 2K + m bits is p = (a, b, c) with a the top K bits, b
// the middle m and c the low K; brev(p) = (brev(c), brev(b), brev(a)). A block
// takes one b: it reads the 2^K x 2^K tile in[(a, b, c)] row by row (c runs
// over consecutive words) into shared memory and writes out[(r, brev(b), j)] =
// tile[brev(j)][brev(r)] row by row (j consecutive), so both sides move whole
// 2^K-word runs; the padded row makes the column reads conflict-free.
template <int K>
__global__ void __launch_bounds__(256) k_permute(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                 int log_n) {
  constexpr int T = 1 << K;
  __shared__ uint32_t tile[T][T + 1];
  const int m = log_n - 2 * K;
  const uint32_t b = blockIdx.x;
  const uint32_t bb = m > 0 ? brev_n(b, m) : 0u;
  const size_t base = (size_t)blockIdx.y << log_n;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int a = idx >> K, c = idx & (T - 1);
    tile[a][c] = in[base + ((size_t)a << (K + m)) + ((size_t)b << K) + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx >> K, j = idx & (T - 1);
    out[base + ((size_t)r << (K + m)) + ((size_t)bb << K) + j] = tile[brev_n(j, K)][brev_n(r, K)];
  }
}

void launch_permute(const DevParams& dp, const uint32_t* in, uint32_t* out, int limbs, bool, cudaStream_t st) {
  if (limbs <= 0) return;
  if (dp.log_n >= 10) k_permute<5><<<dim3(1u << (dp.log_n - 10), limbs), 256, 0, st>>>(in, out, dp.log_n);
  else k_permute<4><<<dim3(1u << (dp.log_n - 8), limbs), 256, 0, st>>>(in, out, dp.log_n);  // N = 2^8
}

// Range check of the checked launch mode: grid (N / 1024, polys * limbs),
// four residues per thread; one flag write per block that saw a violation.
__global__ void __launch_bounds__(256) k_check_range(DevParams dp, const uint32_t* __restrict__ d, size_t poly_stride,
                                                     int n_q, int n_ext, int base) {
  const int limbs = n_q + n_ext;
  const int u = blockIdx.y / limbs, t = blockIdx.y % limbs;
  const uint32_t q = dp.pc[t < n_q ? base + t : dp.L + (t - n_q)].q;
  const size_t off = u * poly_stride + ((size_t)t << dp.log_n) + 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const uint4 v = *reinterpret_cast<const uint4*>(d + off);
  const bool bad = v.x >= q || v.y >= q || v.z >= q || v.w >= q;
  if (__syncthreads_or(bad) && threadIdx.x == 0 && dp.status) atomicOr(dp.status, tc::kStatusRange);
}

void launch_check_range(const DevParams& dp, const uint32_t* d, size_t poly_stride, int polys, int n_q, int n_ext,
                        int base, cudaStream_t st) {
  const int limbs = n_q + n_ext;
  if (!d || polys <= 0 || limbs <= 0) return;
  const int quads = (1 << dp.log_n) / 4, threads = quads < 256 ? quads : 256;
  k_check_range<<<dim3(quads / threads, polys * limbs), threads, 0, st>>>(dp, d, poly_stride, n_q, n_ext, base);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// Element-wise kernels: blockIdx.y enumerates (poly, limb), x covers N / 4
// positions with 128-bit accesses.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, uint32_t q) { return csub(a + b, q); }

// Element-wise kernels over the n limbs of a level whose primes are
// q[base .. base + n).
__global__ void k_hadd(DevParams dp, const uint32_t* a, const uint32_t* b, uint32_t* out, int n, int base,
                       size_t sa, size_t sb, size_t so) {
  const int t = blockIdx.y / n, i = blockIdx.y % n;
  const uint32_t q = dp.pc[base + i].q;
  const size_t off = ((size_t)i << dp.log_n) + 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const uint4 x = *reinterpret_cast<const uint4*>(a + t * sa + off);
  const uint4 y = *reinterpret_cast<const uint4*>(b + t * sb + off);
  *reinterpret_cast<uint4*>(out + t * so + off) =
      make_uint4(addmod(x.x, y.x, q), addmod(x.y, y.y, q), addmod(x.z, y.z, q), addmod(x.w, y.w, q));
}

// PAdd: (b + pt, a) limb by limb.
__global__ void k_padd(DevParams dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base,
                       size_t sa, size_t so) {
  const int t = blockIdx.y / n, i = blockIdx.y % n;
  const uint32_t q = dp.pc[base + i].q;
  const size_t off = ((size_t)i << dp.log_n) + 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  uint4 x = *reinterpret_cast<const uint4*>(a + t * sa + off);
  if (t == 0) {
    const uint4 y = *reinterpret_cast<const uint4*>(pt + off);
    x = make_uint4(addmod(x.x, y.x, q), addmod(x.y, y.y, q), addmod(x.z, y.z, q), addmod(x.w, y.w, q));
  }
  *reinterpret_cast<uint4*>(out + t * so + off) = x;
}

__global__ void k_pmult(DevParams dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base,
                        size_t sa, size_t so) {
  const int t = blockIdx.y / n, i = blockIdx.y % n;
  const PrimeConst P = dp.pc[base + i];
  const size_t off = ((size_t)i << dp.log_n) + 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const uint4 x = *reinterpret_cast<const uint4*>(a + t * sa + off);
  const uint4 y = *reinterpret_cast<const uint4*>(pt + off);
  *reinterpret_cast<uint4*>(out + t * so + off) =
      make_uint4(mulmod(x.x, y.x, P), mulmod(x.y, y.y, P), mulmod(x.z, y.z, P), mulmod(x.w, y.w, P));
}

// d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 (Sec. 2.1 HMult before relinearization).
__global__ void k_tensor(DevParams dp, const uint32_t* c1, const uint32_t* c2, uint32_t* out, int n) {
  const int i = blockIdx.y;
  const PrimeConst P = dp.pc[i];
  const size_t poly = (size_t)n << dp.log_n;
  const size_t off = ((size_t)i << dp.log_n) + blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t b1 = c1[off], a1 = c1[poly + off], b2 = c2[off], a2 = c2[poly + off];
  out[off] = mulmod(b1, b2, P);
  out[poly + off] = addmod(mulmod(a1, b2, P), mulmod(a2, b1, P), P.q);
  out[2 * poly + off] = mulmod(a1, a2, P);
}

__global__ void k_automorph(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint32_t k, int log_n) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t base = (size_t)blockIdx.y << log_n;
  out[base + p] = in[base + auto_src(p, k, log_n)];
}

__global__ void k_small_to_res(DevParams dp, const int64_t* v, uint32_t* out, IdMap ids) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  const int limb = blockIdx.y;
  const uint32_t q = dp.pc[ids(limb)].q;
  int64_t r = v[c] % (int64_t)q;
  if (r < 0) r += q;
  out[((size_t)limb << dp.log_n) + c] = (uint32_t)r;
}

__global__ void k_lincomb(DevParams dp, const uint32_t* a, const uint32_t* s, int sign_as, const uint32_t* c,
                          const uint32_t* d, uint32_t* out, IdMap ids) {
  const int limb = blockIdx.y;
  const PrimeConst P = dp.pc[ids(limb)];
  const size_t off = ((size_t)limb << dp.log_n) + blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  if (a && s) {
    uint32_t as = mulmod(a[off], s[off], P);
    acc = sign_as < 0 ? (as ? P.q - as : 0) : as;
  }
  if (c) acc = addmod(acc, c[off], P.q);
  if (d) acc = addmod(acc, d[off], P.q);
  out[off] = acc;
}

__global__ void k_add_scaled(DevParams dp, const uint32_t* a, const uint2* g, const uint32_t* b, uint32_t* out,
                             IdMap ids) {
  const int limb = blockIdx.y;
  const uint32_t q = dp.pc[ids(limb)].q;
  const uint2 w = g[limb];
  const size_t off = ((size_t)limb << dp.log_n) + blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t v = csub(shoup(a[off], w.x, w.y, q), q);
  out[off] = addmod(v, b[off], q);
}

__global__ void k_to_mont(DevParams dp, uint32_t* data, IdMap ids) {
  const int limb = blockIdx.y;
  const PrimeConst P = dp.pc[ids(limb)];
  const size_t off = ((size_t)limb << dp.log_n) + blockIdx.x * blockDim.x + threadIdx.x;
  data[off] = csub(shoup(data[off], P.mont, P.mont_sh, P.q), P.q);
}

__global__ void k_smr(DevParams dp, const int64_t* x, int32_t* y, int n, int id) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = smr(x[i], dp.pc[id].q, dp.pc[id].m);
}

static dim3 grid_elems(const DevParams& dp, int per_thread, int rows, int threads) {
  return dim3(((1 << dp.log_n) / per_thread + threads - 1) / threads, rows);
}

void launch_hadd(const DevParams& dp, const uint32_t* a, const uint32_t* b, uint32_t* out, int n, int base,
                 size_t sa, size_t sb, size_t so, cudaStream_t st) {
  const int th = 64;
  k_hadd<<<grid_elems(dp, 4, 2 * n, th), th, 0, st>>>(dp, a, b, out, n, base, sa, sb, so);
  count_launch(1);
}

void launch_padd(const DevParams& dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base,
                 size_t sa, size_t so, cudaStream_t st) {
  const int th = 64;
  k_padd<<<grid_elems(dp, 4, 2 * n, th), th, 0, st>>>(dp, a, pt, out, n, base, sa, so);
  count_launch(1);
}

void launch_pmult(const DevParams& dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base,
                  size_t sa, size_t so, cudaStream_t st) {
  const int th = 64;
  k_pmult<<<grid_elems(dp, 4, 2 * n, th), th, 0, st>>>(dp, a, pt, out, n, base, sa, so);
  count_launch(1);
}

void launch_tensor(const DevParams& dp, const uint32_t* c1, const uint32_t* c2, uint32_t* out, int n,
                   cudaStream_t st) {
  const int th = 256;
  k_tensor<<<grid_elems(dp, 1, n, th), th, 0, st>>>(dp, c1, c2, out, n);
}

void launch_automorph(const DevParams& dp, const uint32_t* in, uint32_t* out, int limbs, uint32_t galois,
                      cudaStream_t st) {
  const int th = 256;
  k_automorph<<<grid_elems(dp, 1, limbs, th), th, 0, st>>>(in, out, galois, dp.log_n);
}

void launch_small_to_res(const DevParams& dp, const int64_t* v, uint32_t* out, int limbs, IdMap ids,
                         cudaStream_t st) {
  const int th = 256;
  k_small_to_res<<<grid_elems(dp, 1, limbs, th), th, 0, st>>>(dp, v, out, ids);
}

void launch_lincomb(const DevParams& dp, const uint32_t* a, const uint32_t* s, int sign_as, const uint32_t* c,
                    const uint32_t* d, uint32_t* out, int limbs, IdMap ids, cudaStream_t st) {
  const int th = 256;
  k_lincomb<<<grid_elems(dp, 1, limbs, th), th, 0, st>>>(dp, a, s, sign_as, c, d, out, ids);
}

void launch_add_scaled(const DevParams& dp, const uint32_t* a, const uint2* g, const uint32_t* b, uint32_t* out,
                       int limbs, IdMap ids, cudaStream_t st) {
  const int th = 256;
  k_add_scaled<<<grid_elems(dp, 1, limbs, th), th, 0, st>>>(dp, a, g, b, out, ids);
}

void launch_to_mont(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, cudaStream_t st) {
  const int th = 256;
  k_to_mont<<<grid_elems(dp, 1, limbs, th), th, 0, st>>>(dp, data, ids);
}

void launch_smr(const DevParams& dp, const int64_t* x, int32_t* y, int n, int prime_id, cudaStream_t st) {
  if (n <= 0) return;
  k_smr<<<(n + 255) / 256, 256, 0, st>>>(dp, x, y, n, prime_id);
}

}  // namespace ckks
