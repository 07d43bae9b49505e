// CPU oracle for the 32-bit-word RNS-CKKS key-switch path of the Cheddar paper
// (arxiv 2407.13055). TEST INFRASTRUCTURE ONLY: tests, the smoke check and the
// CPU-baseline leg of the benchmark call it; the CUDA library never does.
//
// Plain and slow on purpose: every modular product is (a*b) % q in 64-bit
// integers, every NTT is the textbook twist + cyclic radix-2 transform, and
// every constant is recomputed from its definition. It shares no code with
// the CUDA path.
//
// Conventions (the paper is silent on them; the readings are listed in the
// design notes):
//  * a polynomial at level l is an [n][N] array of residues in [0, q_i),
//    n = l + 1, limb i modulo q_i (Sec. 2.1, RNS);
//  * the NTT domain is the natural order: out[i] = sum_k a_k psi^((2i+1)k)
//    (Eq. 3 and Sec. 2.2), psi the smallest x in [2, q) with x^N = -1 mod q;
//  * an extended polynomial over PQ stores the n ciphertext limbs first,
//    then the alpha auxiliary limbs p_0 .. p_{alpha-1};
//  * digit j of the hybrid key switching gadget is the primes
//    q_{j*alpha} .. q_{j*alpha+alpha-1} (the last digit may be partial);
//  * an evaluation key is [dnum][2][L + alpha][N]: for each digit the pair
//    (b_j, a_j) over all L ciphertext primes and the alpha auxiliary primes.
//
// parity unpinned: none (every function is pinned by the CPU tests).
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

typedef uint32_t u32;
typedef uint64_t u64;
typedef int32_t i32;
typedef int64_t i64;

namespace {

u32 mul_mod(u32 a, u32 b, u32 q) { return (u32)((u64)a * b % q); }
u32 add_mod(u32 a, u32 b, u32 q) { return (u32)(((u64)a + b) % q); }
u32 sub_mod(u32 a, u32 b, u32 q) { return (u32)(((u64)a + q - b % q) % q); }

u32 pow_mod(u32 b, u64 e, u32 q) {
  u64 r = 1 % q, x = b % q;
  while (e) {
    if (e & 1) r = r * x % q;
    x = x * x % q;
    e >>= 1;
  }
  return (u32)r;
}

// Modular inverse by Fermat's little theorem (q prime).
u32 inv_mod(u32 a, u32 q) { return pow_mod(a, q - 2, q); }

// Residue of a signed integer.
u32 from_signed(i64 v, u32 q) {
  i64 r = v % (i64)q;
  if (r < 0) r += q;
  return (u32)r;
}

// Centered representative in [-(q-1)/2, (q-1)/2] of a residue in [0, q).
i64 centered(u32 x, u32 q) { return x > q / 2 ? (i64)x - (i64)q : (i64)x; }

// Miller-Rabin with bases {2, 7, 61}: deterministic for n < 4,759,123,141
// (Jaeschke 1993), which covers every 32-bit prime.
bool is_prime_u32(u64 n) {
  if (n < 2) return false;
  for (u64 sp : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 61ull})
    if (n % sp == 0) return n == sp;
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : {2ull, 7ull, 61ull}) {
    u64 x = pow_mod((u32)(a % n), d, (u32)n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = x * x % n;
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

// psi = the smallest x in [2, q) with x^N = -1 (mod q). Such an x has
// multiplicative order exactly 2N because 2N is a power of two (Eq. 3).
u32 find_psi(u32 q, int log_n) {
  static std::map<std::pair<u32, int>, u32> cache;
  auto key = std::make_pair(q, log_n);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  u64 n = 1ull << log_n;
  for (u32 x = 2; x < q; ++x) {
    if (pow_mod(x, n, q) == q - 1) {
      cache[key] = x;
      return x;
    }
  }
  return 0;
}

// Bit reversal of i over `bits` bits.
u32 bit_reverse(u32 i, int bits) {
  u32 r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1u) << (bits - 1 - b);
  return r;
}

// Cyclic DFT over Z_q of length N = 2^log_n with root w, in place, natural
// order in and out: A[i] = sum_k a[k] w^(i k). Iterative radix-2 with an
// explicit bit-reversal permutation (textbook Cooley-Tukey).
void cyclic_dft(u32* a, int log_n, u32 q, u32 w) {
  u32 n = 1u << log_n;
  for (u32 i = 0; i < n; ++i) {
    u32 j = bit_reverse(i, log_n);
    if (i < j) std::swap(a[i], a[j]);
  }
  for (u32 len = 2; len <= n; len <<= 1) {
    u32 wl = pow_mod(w, n / len, q);
    for (u32 s = 0; s < n; s += len) {
      u32 wk = 1;
      for (u32 j = 0; j < len / 2; ++j) {
        u32 u = a[s + j];
        u32 v = mul_mod(a[s + j + len / 2], wk, q);
        a[s + j] = add_mod(u, v, q);
        a[s + j + len / 2] = sub_mod(u, v, q);
        wk = mul_mod(wk, wl, q);
      }
    }
  }
}

// Negacyclic NTT (Sec. 2.2): out[i] = sum_k a_k psi^((2i+1)k), natural order.
// Written as a twist by psi^k followed by the cyclic DFT with w = psi^2.
void ntt_fast(u32* a, int log_n, u32 q) {
  u32 n = 1u << log_n, psi = find_psi(q, log_n);
  u32 pk = 1;
  for (u32 k = 0; k < n; ++k) {
    a[k] = mul_mod(a[k], pk, q);
    pk = mul_mod(pk, psi, q);
  }
  cyclic_dft(a, log_n, q, mul_mod(psi, psi, q));
}

// Inverse of ntt_fast: a_k = N^-1 psi^-k sum_i A_i w^(-i k).
void intt_fast(u32* a, int log_n, u32 q) {
  u32 n = 1u << log_n, psi = find_psi(q, log_n);
  u32 psi_inv = inv_mod(psi, q);
  cyclic_dft(a, log_n, q, mul_mod(psi_inv, psi_inv, q));
  u32 n_inv = inv_mod(n % q, q), pk = n_inv;
  for (u32 k = 0; k < n; ++k) {
    a[k] = mul_mod(a[k], pk, q);
    pk = mul_mod(pk, psi_inv, q);
  }
}

// q is the list of all L ciphertext primes in their fixed order; a
// polynomial at a level holds the n_q consecutive primes q[base ..
// base + n_q) (base = 0 for single rescaling; the 25-30 prime system of
// Sec. 3.2 uses other windows, see or_rescale_rational). Key-switching digits
// are the fixed groups q[j alpha .. (j+1) alpha) of that list, cut to the
// window, and a key limb is selected by its global prime index.
struct Params {
  int log_n, L, alpha, dnum;
  const u32* q;
  const u32* p;
  int base = 0;
  u32 n() const { return 1u << log_n; }
  // prime of limb t of an extended polynomial at level with n_q limbs
  u32 ext_prime(int t, int n_q) const { return t < n_q ? q[base + t] : p[t - n_q]; }
  int first_digit() const { return base / alpha; }
  // window limbs [lo, hi) of the j-th active digit
  void digit(int j, int n_q, int& lo, int& hi) const {
    int g = first_digit() + j;
    lo = std::max(0, g * alpha - base);
    hi = std::min(n_q, (g + 1) * alpha - base);
  }
  int key_limb(int t, int n_q) const { return t < n_q ? base + t : L + (t - n_q); }
};

// Fast basis conversion (Eq. 2) with centered y_j (reading of Sec. 4.2,
// "lazy reduction": the y_j are taken in (-q_j/2, q_j/2)):
//   y_j = centered([x_j * (Qs/s_j)^-1]_{s_j}),  out_i = sum_j y_j [Qs/s_j]_{d_i} mod d_i
// where Qs is the product of the K source primes s_j. Coefficient domain.
void bconv(const u32* x, int k_src, const u32* src, u32* out, int m_dst, const u32* dst, u32 n) {
  std::vector<u32> hat_inv(k_src);
  std::vector<u32> hat(size_t(k_src) * m_dst);
  for (int j = 0; j < k_src; ++j) {
    u32 h = 1;
    for (int jj = 0; jj < k_src; ++jj)
      if (jj != j) h = mul_mod(h, src[jj] % src[j], src[j]);
    hat_inv[j] = inv_mod(h, src[j]);
    for (int i = 0; i < m_dst; ++i) {
      u32 hd = 1;
      for (int jj = 0; jj < k_src; ++jj)
        if (jj != j) hd = mul_mod(hd, src[jj] % dst[i], dst[i]);
      hat[size_t(j) * m_dst + i] = hd;
    }
  }
  std::vector<i64> y(k_src);
  for (u32 c = 0; c < n; ++c) {
    for (int j = 0; j < k_src; ++j)
      y[j] = centered(mul_mod(x[size_t(j) * n + c], hat_inv[j], src[j]), src[j]);
    for (int i = 0; i < m_dst; ++i) {
      u32 acc = 0;
      for (int j = 0; j < k_src; ++j)
        acc = add_mod(acc, mul_mod(from_signed(y[j], dst[i]), hat[size_t(j) * m_dst + i], dst[i]), dst[i]);
      out[size_t(i) * n + c] = acc;
    }
  }
}

// Coefficient-domain automorphism X -> X^k (Eq. 4 stated on coefficients):
// a_t X^t -> a_t X^(t k mod 2N), negated when t k mod 2N >= N.
void automorph_coeff(const u32* a, u32* out, u32 n, u32 k, u32 q) {
  for (u32 t = 0; t < n; ++t) {
    u64 e = (u64)t * k % (2ull * n);
    if (e < n) out[e] = a[t];
    else out[e - n] = a[t] ? q - a[t] : 0;
  }
}

// NTT-domain automorphism in natural order (Eq. 4):
// out[j] = in[((2j+1) k mod 2N - 1) / 2].
void automorph_ntt(const u32* a, u32* out, u32 n, u32 k) {
  for (u32 j = 0; j < n; ++j) {
    u64 src = (((2ull * j + 1) * k) % (2ull * n) - 1) / 2;
    out[j] = a[src];
  }
}

// Number of digits active at a level with n_q ciphertext limbs from prime base.
// (Sec. 2.3: hybrid key switching splits Q_l into digits of alpha primes.)
int n_digits(int n_q, int alpha, int base = 0) { return (base + n_q - 1) / alpha - base / alpha + 1; }

// ModUp (Alg. 1 as ModSwitch Q_j -> PQ, Sec. 2.3): for every active digit j,
// bring its limbs to the coefficient domain, convert to every other prime of
// Q_l and P by Eq. 2, and return to the NTT domain. The digit's own limbs are
// copied. out is [n_digits][n_q + alpha][N].
void modup(const Params& P, const u32* d, int n_q, u32* out) {
  u32 n = P.n();
  int ext = n_q + P.alpha, nd = n_digits(n_q, P.alpha, P.base);
  for (int j = 0; j < nd; ++j) {
    int lo, hi;
    P.digit(j, n_q, lo, hi);
    int k_src = hi - lo;
    std::vector<u32> coef(size_t(k_src) * n);
    std::vector<u32> src(k_src);
    for (int s = 0; s < k_src; ++s) {
      src[s] = P.q[P.base + lo + s];
      std::memcpy(&coef[size_t(s) * n], d + size_t(lo + s) * n, n * 4);
      intt_fast(&coef[size_t(s) * n], P.log_n, src[s]);
    }
    std::vector<u32> dst;
    std::vector<int> dst_limb;
    for (int t = 0; t < ext; ++t) {
      if (t >= lo && t < hi) continue;
      dst.push_back(P.ext_prime(t, n_q));
      dst_limb.push_back(t);
    }
    std::vector<u32> conv(dst.size() * n);
    bconv(coef.data(), k_src, src.data(), conv.data(), (int)dst.size(), dst.data(), n);
    u32* oj = out + size_t(j) * ext * n;
    for (int t = lo; t < hi; ++t) std::memcpy(oj + size_t(t) * n, d + size_t(t) * n, n * 4);
    for (size_t i = 0; i < dst.size(); ++i) {
      ntt_fast(&conv[i * n], P.log_n, dst[i]);
      std::memcpy(oj + size_t(dst_limb[i]) * n, &conv[i * n], n * 4);
    }
  }
}

// KeyMult + MAC (Sec. 2.3): acc_t = sum_j ModUp_j * evk_j[t], t in {0,1},
// over the n_q active ciphertext limbs and the alpha auxiliary limbs; the
// top-level key is truncated by skipping limbs n_q .. L-1.
void keymult(const Params& P, const u32* up, int n_q, const u32* evk, u32* acc) {
  u32 n = P.n();
  int ext = n_q + P.alpha, nd = n_digits(n_q, P.alpha, P.base), ext_top = P.L + P.alpha;
  for (int t = 0; t < 2; ++t)
    for (int l = 0; l < ext; ++l) {
      u32 q = P.ext_prime(l, n_q);
      int key_limb = P.key_limb(l, n_q);
      for (u32 c = 0; c < n; ++c) {
        u32 s = 0;
        for (int j = 0; j < nd; ++j) {
          u32 x = up[(size_t(j) * ext + l) * n + c];
          u32 e = evk[((size_t(P.first_digit() + j) * 2 + t) * ext_top + key_limb) * n + c];
          s = add_mod(s, mul_mod(x, e, q), q);
        }
        acc[(size_t(t) * ext + l) * n + c] = s;
      }
    }
}

// ModDown (Sec. 2.3; hybrid key switching of Han-Ki): for each of the two
// polynomials, x_P = iNTT(acc[P]); z_i = NTT(BConv_{P -> q_i}(x_P));
// out_i = (acc[q_i] - z_i) * P^-1 mod q_i.
void moddown(const Params& P, const u32* acc, int n_q, u32* out) {
  u32 n = P.n();
  int ext = n_q + P.alpha;
  for (int t = 0; t < 2; ++t) {
    const u32* a = acc + size_t(t) * ext * n;
    std::vector<u32> xp(size_t(P.alpha) * n);
    for (int k = 0; k < P.alpha; ++k) {
      std::memcpy(&xp[size_t(k) * n], a + size_t(n_q + k) * n, n * 4);
      intt_fast(&xp[size_t(k) * n], P.log_n, P.p[k]);
    }
    std::vector<u32> z(size_t(n_q) * n);
    bconv(xp.data(), P.alpha, P.p, z.data(), n_q, P.q + P.base, n);
    for (int i = 0; i < n_q; ++i) {
      u32 q = P.q[P.base + i];
      ntt_fast(&z[size_t(i) * n], P.log_n, q);
      u32 pinv = 1;
      for (int k = 0; k < P.alpha; ++k) pinv = mul_mod(pinv, P.p[k] % q, q);
      pinv = inv_mod(pinv, q);
      for (u32 c = 0; c < n; ++c)
        out[(size_t(t) * n_q + i) * n + c] = mul_mod(sub_mod(a[size_t(i) * n + c], z[size_t(i) * n + c], q), pinv, q);
    }
  }
}

// Key switching of one polynomial d (NTT domain, n_q limbs) with evk:
// out = ModDown(KeyMult(ModUp(d), evk)), two polynomials of n_q limbs.
// (Sec. 2.3, the key-switching sequence.)
void keyswitch(const Params& P, const u32* d, int n_q, const u32* evk, u32* out) {
  u32 n = P.n();
  int ext = n_q + P.alpha, nd = n_digits(n_q, P.alpha, P.base);
  std::vector<u32> up(size_t(nd) * ext * n), acc(size_t(2) * ext * n);
  modup(P, d, n_q, up.data());
  keymult(P, up.data(), n_q, evk, acc.data());
  moddown(P, acc.data(), n_q, out);
}

}  // namespace

extern "C" {

// Primality for the prime rule (Eq. 3: the NTT primes are primes q = 1 mod 2N).
int or_is_prime(uint64_t v) { return is_prime_u32(v) ? 1 : 0; }

// Prime lists (Eq. 3: q = 1 mod 2N; Sec. 3: q < 2^31). Reading of the paper's
// silent choice: q_0 is the largest such prime below 2^31; q_1 .. q_{L-1} are
// the largest such primes below 2^30 in decreasing order; the auxiliary primes
// p_0 .. p_{alpha-1} are the next largest such primes below 2^31 after q_0.
int or_gen_primes(int log_n, int n_q, int n_p, uint32_t* q, uint32_t* p) {
  u64 m = 2ull << log_n;
  u64 c = ((1ull << 31) - 1) / m * m + 1;
  if (c >= (1ull << 31)) c -= m;
  int got_top = 0;
  std::vector<u32> top;
  for (; c > (1ull << 30) && got_top < 1 + n_p; c -= m)
    if (is_prime_u32(c)) { top.push_back((u32)c); ++got_top; }
  if (got_top < 1 + n_p) return -1;
  if (n_q > 0) q[0] = top[0];
  for (int i = 0; i < n_p; ++i) p[i] = top[1 + i];
  c = ((1ull << 30) - 1) / m * m + 1;
  if (c >= (1ull << 30)) c -= m;
  for (int i = 1; i < n_q; c -= m) {
    if (c < (1ull << 28)) return -1;
    if (is_prime_u32(c)) q[i++] = (u32)c;
  }
  return 0;
}

// psi of the negacyclic NTT (Eq. 3): the smallest x with x^N = -1 mod q.
uint32_t or_find_psi(uint32_t q, int log_n) { return find_psi(q, log_n); }

// 32-bit signed Montgomery reduction (Alg. 2): for x in [-q 2^31, q 2^31),
// returns y = x 2^-32 mod q with y in (-q, q), using m = q^-1 mod 2^32 as a
// signed 32-bit value, one low and one high signed 32-bit product.
int32_t or_smr(int64_t x, uint32_t q) {
  u32 m = 1;  // Newton iteration for q^-1 mod 2^32
  for (int i = 0; i < 5; ++i) m *= 2u - q * m;
  u32 x_lo = (u32)(u64)x;
  i32 x_hi = (i32)(x >> 32);
  i32 z = (i32)(x_lo * m);                      // mullo32
  i32 zh = (i32)(((i64)z * (i64)(i32)q) >> 32);  // mulhi32
  return x_hi - zh;
}

// Negacyclic NTT (Eq. 3) by its definition, O(N^2): out[i] = sum_k a_k psi^((2i+1)k).
void or_ntt_naive(const uint32_t* a, uint32_t* out, int log_n, uint32_t q) {
  u32 n = 1u << log_n, psi = find_psi(q, log_n);
  for (u32 i = 0; i < n; ++i) {
    u32 s = 0;
    for (u32 k = 0; k < n; ++k)
      s = add_mod(s, mul_mod(a[k], pow_mod(psi, (u64)(2 * i + 1) * k % (2 * n), q), q), q);
    out[i] = s;
  }
}

// Inverse NTT (Eq. 3) by its definition: a_k = N^-1 sum_i A_i psi^(-(2i+1)k).
void or_intt_naive(const uint32_t* a, uint32_t* out, int log_n, uint32_t q) {
  u32 n = 1u << log_n, psi_inv = inv_mod(find_psi(q, log_n), q);
  u32 n_inv = inv_mod(n % q, q);
  for (u32 k = 0; k < n; ++k) {
    u32 s = 0;
    for (u32 i = 0; i < n; ++i)
      s = add_mod(s, mul_mod(a[i], pow_mod(psi_inv, (u64)(2 * i + 1) * k % (2 * n), q), q), q);
    out[k] = mul_mod(s, n_inv, q);
  }
}

// Fast NTT / iNTT (Eq. 3, Sec. 2.2) over `limbs` limbs, limb i modulo primes[i], in place.
void or_ntt(uint32_t* a, int limbs, const uint32_t* primes, int log_n) {
  for (int i = 0; i < limbs; ++i) ntt_fast(a + (size_t(i) << log_n), log_n, primes[i]);
}
void or_intt(uint32_t* a, int limbs, const uint32_t* primes, int log_n) {
  for (int i = 0; i < limbs; ++i) intt_fast(a + (size_t(i) << log_n), log_n, primes[i]);
}

// Eq. 2, coefficient domain: x [k_src][N] modulo src -> out [m_dst][N] modulo dst.
void or_bconv(const uint32_t* x, int k_src, const uint32_t* src, uint32_t* out, int m_dst,
              const uint32_t* dst, int log_n) {
  bconv(x, k_src, src, out, m_dst, dst, 1u << log_n);
}

// Automorphism X -> X^k (Eq. 4) on NTT-domain limbs, and on coefficients.
void or_automorph_ntt(const uint32_t* a, uint32_t* out, int limbs, int log_n, uint32_t k) {
  u32 n = 1u << log_n;
  for (int i = 0; i < limbs; ++i) automorph_ntt(a + size_t(i) * n, out + size_t(i) * n, n, k);
}
void or_automorph_coeff(const uint32_t* a, uint32_t* out, int limbs, const uint32_t* primes, int log_n,
                        uint32_t k) {
  u32 n = 1u << log_n;
  for (int i = 0; i < limbs; ++i) automorph_coeff(a + size_t(i) * n, out + size_t(i) * n, n, k, primes[i]);
}

// Tensor product of two ciphertexts (Sec. 2.1, HMult before relinearization),
// NTT domain: d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2. ct = [2][n_q][N]
// (b then a); out = [3][n_q][N].
void or_tensor(const uint32_t* ct1, const uint32_t* ct2, int n_q, const uint32_t* q, int log_n,
               uint32_t* out) {
  u32 n = 1u << log_n;
  size_t poly = size_t(n_q) * n;
  for (int i = 0; i < n_q; ++i)
    for (u32 c = 0; c < n; ++c) {
      size_t o = size_t(i) * n + c;
      u32 b1 = ct1[o], a1 = ct1[poly + o], b2 = ct2[o], a2 = ct2[poly + o];
      out[o] = mul_mod(b1, b2, q[i]);
      out[poly + o] = add_mod(mul_mod(a1, b2, q[i]), mul_mod(a2, b1, q[i]), q[i]);
      out[2 * poly + o] = mul_mod(a1, a2, q[i]);
    }
}

// ModUp (Alg. 1, Eq. 2), KeyMult + MAC (Sec. 2.3, Par. 1) and ModDown
// (Sec. 2.3) as separate steps, for the step-by-step parity tests.
void or_modup(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
              const uint32_t* d, int n_q, uint32_t* out) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  modup(P, d, n_q, out);
}

void or_keymult(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
                const uint32_t* up, int n_q, const uint32_t* evk, uint32_t* acc) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  keymult(P, up, n_q, evk, acc);
}

void or_moddown(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
                const uint32_t* acc, int n_q, uint32_t* out) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  moddown(P, acc, n_q, out);
}

// Single rescaling (Sec. 2.1 "Rescaling"; c' = round(c / q_l)): for each of the
// `polys` polynomials, v = centered(iNTT(c_l)); for i < l:
// c'_i = (c_i - NTT(v mod q_i)) * q_l^-1 mod q_i. in [polys][n_q][N] -> out
// [polys][n_q-1][N].
void or_rescale(const uint32_t* in, int polys, int n_q, const uint32_t* q, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  int l = n_q - 1;
  for (int t = 0; t < polys; ++t) {
    const u32* c = in + size_t(t) * n_q * n;
    std::vector<u32> top(c + size_t(l) * n, c + size_t(l + 1) * n);
    intt_fast(top.data(), log_n, q[l]);
    std::vector<u32> r(n);
    for (int i = 0; i < l; ++i) {
      for (u32 k = 0; k < n; ++k) r[k] = from_signed(centered(top[k], q[l]), q[i]);
      ntt_fast(r.data(), log_n, q[i]);
      u32 qinv = inv_mod(q[l] % q[i], q[i]);
      for (u32 k = 0; k < n; ++k)
        out[(size_t(t) * l + i) * n + k] = mul_mod(sub_mod(c[size_t(i) * n + k], r[k], q[i]), qinv, q[i]);
    }
  }
}

// Rational rescaling between two windows of the prime list q (Sec. 3.1
// "Rational rescaling", Sec. 3.2, Sec. 5.1 with Fig. 4): the primes of the
// old window [s_old, s_old + n_old) that the new window [s_new, s_new +
// n_new) lacks are divided out (their product T_drop) and the primes the new
// window adds are multiplied in (T_add): c' = (c T_add - X) / T_drop with
// X = BConv_{drop -> new}([c T_add]_{T_drop}) (Eq. 2 with centered
// representatives). Steps, per polynomial: for every dropped prime d,
// x_d = iNTT(c_d) T_add mod d; X_t = BConv(x)_t for every prime t of the
// new window, back to the NTT domain; c'_t = (c_t T_add - X_t) T_drop^-1 mod
// t, where c_t T_add = 0 for an added prime. in [polys][n_old][N] ->
// out [polys][n_new][N], both in window order.
void or_rescale_rational(const uint32_t* in, int polys, const uint32_t* q, int s_old, int n_old, int s_new,
                         int n_new, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  auto in_old = [&](int g) { return g >= s_old && g < s_old + n_old; };
  auto in_new = [&](int g) { return g >= s_new && g < s_new + n_new; };
  std::vector<int> drop, add;
  for (int g = s_old; g < s_old + n_old; ++g)
    if (!in_new(g)) drop.push_back(g);
  for (int g = s_new; g < s_new + n_new; ++g)
    if (!in_old(g)) add.push_back(g);
  auto prod_mod = [&](const std::vector<int>& set, u32 m) {
    u32 r = 1 % m;
    for (int g : set) r = mul_mod(r, q[g] % m, m);
    return r;
  };
  const int K = (int)drop.size();
  std::vector<u32> src(K), dst(n_new);
  for (int k = 0; k < K; ++k) src[k] = q[drop[k]];
  for (int i = 0; i < n_new; ++i) dst[i] = q[s_new + i];
  for (int t = 0; t < polys; ++t) {
    const u32* c = in + size_t(t) * n_old * n;
    u32* o = out + size_t(t) * n_new * n;
    if (K == 0) {  // nothing dropped: only T_add multiplies in
      for (int i = 0; i < n_new; ++i) {
        int g = s_new + i;
        u32 qq = q[g], ta = prod_mod(add, qq);
        for (u32 k = 0; k < n; ++k) o[size_t(i) * n + k] = in_old(g) ? mul_mod(c[size_t(g - s_old) * n + k], ta, qq) : 0;
      }
      continue;
    }
    std::vector<u32> x(size_t(K) * n), conv(size_t(n_new) * n);
    for (int k = 0; k < K; ++k) {
      u32 d = src[k], ta = prod_mod(add, d);
      std::memcpy(&x[size_t(k) * n], c + size_t(drop[k] - s_old) * n, n * 4);
      intt_fast(&x[size_t(k) * n], log_n, d);
      for (u32 j = 0; j < n; ++j) x[size_t(k) * n + j] = mul_mod(x[size_t(k) * n + j], ta, d);
    }
    bconv(x.data(), K, src.data(), conv.data(), n_new, dst.data(), n);
    for (int i = 0; i < n_new; ++i) {
      int g = s_new + i;
      u32 qq = q[g];
      ntt_fast(&conv[size_t(i) * n], log_n, qq);
      u32 ta = prod_mod(add, qq), tdi = inv_mod(prod_mod(drop, qq), qq);
      for (u32 k = 0; k < n; ++k) {
        u32 ct = in_old(g) ? mul_mod(c[size_t(g - s_old) * n + k], ta, qq) : 0;
        o[size_t(i) * n + k] = mul_mod(sub_mod(ct, conv[size_t(i) * n + k], qq), tdi, qq);
      }
    }
  }
}

// HMult (Sec. 2.1): tensor, relinearize with evk (key switching of d2),
// optionally rescale. ct = [2][n_q][N]; out = [2][n_q][N] or [2][n_q-1][N].
void or_hmult(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
              const uint32_t* ct1, const uint32_t* ct2, int n_q, const uint32_t* evk, int rescale,
              uint32_t* out) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  u32 n = P.n();
  size_t poly = size_t(n_q) * n;
  std::vector<u32> d(3 * poly), ks(2 * poly), res(2 * poly);
  q += base;
  or_tensor(ct1, ct2, n_q, q, log_n, d.data());
  keyswitch(P, d.data() + 2 * poly, n_q, evk, ks.data());
  for (int t = 0; t < 2; ++t)
    for (int i = 0; i < n_q; ++i)
      for (u32 c = 0; c < n; ++c) {
        size_t o = size_t(i) * n + c;
        res[t * poly + o] = add_mod(d[t * poly + o], ks[t * poly + o], q[i]);
      }
  if (rescale) or_rescale(res.data(), 2, n_q, q, log_n, out);
  else std::memcpy(out, res.data(), 2 * poly * 4);
}

// HMult with ModDown merged into the rescaling (the merge the paper takes
// from MAD and extends to its prime system, Sec. 6). The level's window is
// q[base .. base + n_q) (Params.base), the next level's q[s_new .. s_new +
// n_new); D = primes leaving the window (T_drop their product), A = primes
// entering it (T_add; empty and 1 for the usual rescaling by q_l, Sec. 3.2
// for the rational one). With Y_u = KeyMult(ModUp(d2))_u + P d_u on the
// window and P (d_u the tensor's d0, d1; P d_u = 0 on the P limbs), one fast
// basis conversion (Eq. 2, centered) from the primes P and D gives
// X = BConv([Y T_add]_{P T_drop}) on the new window, and
//   out_t = (Y_t T_add - X_t) (P T_drop)^-1   (Y_t = 0 for t in A).
// This divides by P T_drop in one rounding instead of ModDown then rescale,
// so the result differs from the two-step one by a small polynomial.
// ct = [2][n_q][N]; out = [2][n_new][N].
void or_hmult_merged(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
                     const uint32_t* ct1, const uint32_t* ct2, int n_q, const uint32_t* evk, int s_new,
                     int n_new, uint32_t* out) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  u32 n = P.n();
  const int ext = n_q + alpha, nd = n_digits(n_q, alpha, base);
  size_t poly = size_t(n_q) * n;
  auto in_old = [&](int g) { return g >= base && g < base + n_q; };
  auto in_new = [&](int g) { return g >= s_new && g < s_new + n_new; };
  std::vector<int> drop, add;
  for (int g = base; g < base + n_q; ++g)
    if (!in_new(g)) drop.push_back(g);
  for (int g = s_new; g < s_new + n_new; ++g)
    if (!in_old(g)) add.push_back(g);
  auto pmod = [&](u32 m) {
    u32 r = 1 % m;
    for (int k = 0; k < alpha; ++k) r = mul_mod(r, p[k] % m, m);
    return r;
  };
  auto prod_mod = [&](const std::vector<int>& set, u32 m) {
    u32 r = 1 % m;
    for (int g : set) r = mul_mod(r, q[g] % m, m);
    return r;
  };
  std::vector<u32> d(3 * poly), up(size_t(nd) * ext * n), acc(size_t(2) * ext * n);
  or_tensor(ct1, ct2, n_q, q + base, log_n, d.data());
  modup(P, d.data() + 2 * poly, n_q, up.data());
  keymult(P, up.data(), n_q, evk, acc.data());
  const int K = alpha + (int)drop.size();
  std::vector<u32> src(K), dst(n_new);
  for (int k = 0; k < alpha; ++k) src[k] = p[k];
  for (size_t k = 0; k < drop.size(); ++k) src[alpha + k] = q[drop[k]];
  for (int t = 0; t < n_new; ++t) dst[t] = q[s_new + t];
  for (int u = 0; u < 2; ++u) {
    const u32* a = acc.data() + size_t(u) * ext * n;
    const u32* du = d.data() + size_t(u) * poly;
    // Y on window prime g (limb g - base): acc + [P]_g d
    auto y_at = [&](int g, u32 c) {
      u32 m = q[g];
      size_t o = size_t(g - base) * n + c;
      return add_mod(a[o], mul_mod(pmod(m), du[o], m), m);
    };
    // [Y T_add]_s on the sources, coefficient domain
    std::vector<u32> y(size_t(K) * n);
    for (int k = 0; k < K; ++k) {
      u32 m = src[k], ta = prod_mod(add, m);
      for (u32 c = 0; c < n; ++c) {
        u32 v = k < alpha ? a[size_t(n_q + k) * n + c] : y_at(drop[k - alpha], c);
        y[size_t(k) * n + c] = mul_mod(v, ta, m);
      }
      intt_fast(&y[size_t(k) * n], log_n, m);
    }
    std::vector<u32> x(size_t(n_new) * n);
    bconv(y.data(), K, src.data(), x.data(), n_new, dst.data(), n);
    for (int t = 0; t < n_new; ++t) {
      const int g = s_new + t;
      u32 m = q[g];
      ntt_fast(&x[size_t(t) * n], log_n, m);
      u32 ta = prod_mod(add, m), inv = inv_mod(mul_mod(pmod(m), prod_mod(drop, m), m), m);
      for (u32 c = 0; c < n; ++c) {
        u32 yt = in_old(g) ? mul_mod(y_at(g, c), ta, m) : 0;
        out[(size_t(u) * n_new + t) * n + c] = mul_mod(sub_mod(yt, x[size_t(t) * n + c], m), inv, m);
      }
    }
  }
}

// HRot / HConj (Sec. 2.3): out = (phi_k(b), 0) + KeySwitch(phi_k(a)) with the
// key for phi_k(s); k = 5^r mod 2N for a rotation by r, k = 2N - 1 for
// conjugation. Automorphism first (the equivalent order of the paper's
// ModUp -> KeyMult -> MAC -> automorphism -> ModDown; see the design notes).
void or_hrot(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum, int base,
             const uint32_t* ct, int n_q, uint32_t k, const uint32_t* evk, uint32_t* out) {
  Params P{log_n, L, alpha, dnum, q, p, base};
  u32 n = P.n();
  size_t poly = size_t(n_q) * n;
  q += base;
  std::vector<u32> rb(poly), ra(poly), ks(2 * poly);
  or_automorph_ntt(ct, rb.data(), n_q, log_n, k);
  or_automorph_ntt(ct + poly, ra.data(), n_q, log_n, k);
  keyswitch(P, ra.data(), n_q, evk, ks.data());
  for (int i = 0; i < n_q; ++i)
    for (u32 c = 0; c < n; ++c) {
      size_t o = size_t(i) * n + c;
      out[o] = add_mod(rb[o], ks[o], q[i]);
      out[poly + o] = ks[poly + o];
    }
}

// HAdd (Sec. 2.1): limb-wise modular addition of two ciphertexts [2][n_q][N].
void or_hadd(const uint32_t* x, const uint32_t* y, int n_q, const uint32_t* q, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  for (int t = 0; t < 2; ++t)
    for (int i = 0; i < n_q; ++i)
      for (u32 c = 0; c < n; ++c) {
        size_t o = (size_t(t) * n_q + i) * n + c;
        out[o] = add_mod(x[o], y[o], q[i]);
      }
}

// PMult (Sec. 2.1): ciphertext [2][n_q][N] times plaintext [n_q][N], NTT domain.
void or_pmult(const uint32_t* x, const uint32_t* pt, int n_q, const uint32_t* q, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  for (int t = 0; t < 2; ++t)
    for (int i = 0; i < n_q; ++i)
      for (u32 c = 0; c < n; ++c) {
        size_t o = (size_t(t) * n_q + i) * n + c;
        out[o] = mul_mod(x[o], pt[size_t(i) * n + c], q[i]);
      }
}

// Signed small coefficients -> residues modulo each prime (RNS, Sec. 2.1), then NTT (Eq. 3).
void or_small_to_ntt(const int64_t* v, int limbs, const uint32_t* primes, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  for (int i = 0; i < limbs; ++i) {
    for (u32 c = 0; c < n; ++c) out[size_t(i) * n + c] = from_signed(v[c], primes[i]);
    ntt_fast(out + size_t(i) * n, log_n, primes[i]);
  }
}

// Encryption (Eq. 1): (b, a) = (-a s + m + e, a), NTT domain over the n_q
// primes; s and e are small signed coefficient vectors, a is uniform
// (NTT domain), m the plaintext (NTT domain).
void or_encrypt(const int64_t* s, const uint32_t* a, const int64_t* e, const uint32_t* m, int n_q,
                const uint32_t* q, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  size_t poly = size_t(n_q) * n;
  std::vector<u32> sh(poly), eh(poly);
  or_small_to_ntt(s, n_q, q, log_n, sh.data());
  or_small_to_ntt(e, n_q, q, log_n, eh.data());
  for (int i = 0; i < n_q; ++i)
    for (u32 c = 0; c < n; ++c) {
      size_t o = size_t(i) * n + c;
      u32 as = mul_mod(a[o], sh[o], q[i]);
      out[o] = add_mod(sub_mod(m[o], as, q[i]), eh[o], q[i]);
      out[poly + o] = a[o];
    }
}

// Decryption (Sec. 2.1): m = b + a s (NTT domain).
void or_decrypt(const int64_t* s, const uint32_t* ct, int n_q, const uint32_t* q, int log_n, uint32_t* out) {
  u32 n = 1u << log_n;
  size_t poly = size_t(n_q) * n;
  std::vector<u32> sh(poly);
  or_small_to_ntt(s, n_q, q, log_n, sh.data());
  for (int i = 0; i < n_q; ++i)
    for (u32 c = 0; c < n; ++c) {
      size_t o = size_t(i) * n + c;
      out[o] = add_mod(ct[o], mul_mod(ct[poly + o], sh[o], q[i]), q[i]);
    }
}

// Key-switching key from s_from to s (Sec. 2.3, hybrid gadget; the paper
// cites Han-Ki for it): for each digit j, b_j = -a_j s + e_j + g_j s_from over all L
// ciphertext and alpha auxiliary primes, with g_j = [P]_{q_i} on the limbs of
// digit j and 0 on every other limb (including the auxiliary ones).
// s: ternary secret coefficients; s_from_ntt: [L+alpha][N] NTT domain;
// a: [dnum][L+alpha][N] uniform NTT domain; e: [dnum][N] coefficients.
// evk out: [dnum][2][L+alpha][N].
void or_keygen_ks(int log_n, int L, const uint32_t* q, int alpha, const uint32_t* p, int dnum,
                  const int64_t* s, const uint32_t* s_from_ntt, const uint32_t* a, const int64_t* e,
                  uint32_t* evk) {
  u32 n = 1u << log_n;
  int ext = L + alpha;
  std::vector<u32> primes(ext);
  for (int i = 0; i < ext; ++i) primes[i] = i < L ? q[i] : p[i - L];
  size_t poly = size_t(ext) * n;
  std::vector<u32> sh(poly), eh(poly);
  or_small_to_ntt(s, ext, primes.data(), log_n, sh.data());
  for (int j = 0; j < dnum; ++j) {
    or_small_to_ntt(e + size_t(j) * n, ext, primes.data(), log_n, eh.data());
    for (int i = 0; i < ext; ++i) {
      u32 pr = primes[i];
      u32 g = 0;
      if (i < L && i / alpha == j) {
        g = 1;
        for (int k = 0; k < alpha; ++k) g = mul_mod(g, p[k] % pr, pr);
      }
      for (u32 c = 0; c < n; ++c) {
        size_t o = size_t(i) * n + c;
        u32 aa = a[size_t(j) * poly + o];
        u32 b = sub_mod(eh[o], mul_mod(aa, sh[o], pr), pr);
        b = add_mod(b, mul_mod(g, s_from_ntt[o], pr), pr);
        evk[(size_t(j) * 2 + 0) * poly + o] = b;
        evk[(size_t(j) * 2 + 1) * poly + o] = aa;
      }
    }
  }
}

}  // extern "C"
