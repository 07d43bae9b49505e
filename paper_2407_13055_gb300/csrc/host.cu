// Host-side number theory, table construction, sampling and encoding.
#include <cmath>
#include <complex>
#include <cstring>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ckks {

namespace {

typedef unsigned __int128 u128;

uint32_t mulm(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)((uint64_t)a * b % q); }

uint32_t powm(uint32_t b, uint64_t e, uint32_t q) {
  uint64_t r = 1, x = b % q;
  for (; e; e >>= 1) {
    if (e & 1) r = r * x % q;
    x = x * x % q;
  }
  return (uint32_t)(r % q);
}

// Inverse by the extended Euclidean algorithm (a and q coprime).
uint32_t invm(uint32_t a, uint32_t q) {
  int64_t t = 0, nt = 1, r = q, nr = a % q;
  while (nr) {
    int64_t k = r / nr;
    int64_t tmp = t - k * nt;
    t = nt;
    nt = tmp;
    tmp = r - k * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += q;
  return (uint32_t)t;
}

uint32_t shoup_of(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }
uint2 shoup_pair(uint32_t w, uint32_t q) { return make_uint2(w, shoup_of(w, q)); }
int32_t centered_h(uint32_t x, uint32_t q) { return x > q / 2 ? (int32_t)((int64_t)x - q) : (int32_t)x; }

// fp16 bit pattern of an integer v with |v| <= 2048 (exact).
uint16_t f16_bits(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  uint32_t a = (uint32_t)(v < 0 ? -v : v);
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;
  return (uint16_t)(sign | (uint16_t)((e + 15) << 10) | (uint16_t)((a << (10 - e)) & 0x3FFu));
}

// Byte-plane image of a conversion matrix for the tensor-core BConv (the B
// operand of cols_tc.cuh): mat[t * K + k] (t < M targets with primes
// prime[t]) are centered [(...) 2^32]_{prime_t} entries. For each target and
// source, m'_a = [mat 2^(8a)]_{prime_t} centered (a < 4) is written as four
// balanced signed bytes (m'_a = sum_b e_b 2^(8b), e_b in [-128, 128) for
// b < 3); row 4 t + b of the image holds e_b of (k, a) at column 4 k + a, as
// fp16. Rows are padded to a multiple of 16 (zero targets), columns to
// kr = 16 ceil(K / 4), and the image is stored in the MMA's shared-memory
// layout: core matrices of 8 rows x 8 columns (128 bytes), column blocks of
// 8 adjacent (128 bytes apart), 8-row groups kr * 16 bytes apart. Returns
// (byte offset in img, bytes).
int2 append_planes(std::vector<uint8_t>& img, const int32_t* mat, int M, int K, const uint32_t* prime) {
  const int kr = 16 * ((K + 3) / 4);
  const int rows = 4 * ((M + 3) & ~3);
  const size_t off = img.size(), bytes = (size_t)rows * kr * 2;
  img.resize(off + bytes, 0);
  uint8_t* base = img.data() + off;
  for (int t = 0; t < M; ++t) {
    const uint32_t p = prime[t];
    for (int k = 0; k < K; ++k) {
      const int32_t m = mat[(size_t)t * K + k];
      const uint64_t mu = (uint64_t)(m < 0 ? (int64_t)m + p : (int64_t)m);
      for (int a = 0; a < 4; ++a) {
        int64_t v = centered_h((uint32_t)((mu << (8 * a)) % p), p);
        int e[4];
        for (int b = 0; b < 3; ++b) {
          e[b] = (int)(((v % 256) + 256 + 128) % 256) - 128;
          v = (v - e[b]) / 256;
        }
        e[3] = (int)v;
        for (int b = 0; b < 4; ++b) {
          const int n = 4 * t + b, c = 4 * k + a;
          const size_t o = (size_t)(n >> 3) * kr * 16 + (size_t)(c >> 3) * 128 + (n & 7) * 16 + (c & 7) * 2;
          const uint16_t h = f16_bits(e[b]);
          base[o] = (uint8_t)(h & 0xFF);
          base[o + 1] = (uint8_t)(h >> 8);
        }
      }
    }
  }
  return make_int2((int)off, (int)bytes);
}

uint32_t brev(uint32_t v, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i, v >>= 1) r = (r << 1) | (v & 1);
  return r;
}

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Miller-Rabin with bases 2, 3, 5, 7, 11, 13, 17: deterministic below 3.4e14.
bool host_is_prime(uint64_t n) {
  if (n < 2) return false;
  static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint64_t s : small) {
    if (n == s) return true;
    if (n % s == 0) return false;
  }
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  for (uint64_t a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull}) {
    u128 x = 1, base = a % n;
    for (uint64_t e = d; e; e >>= 1) {
      if (e & 1) x = x * base % n;
      base = base * base % n;
    }
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int i = 1; i < r && witness; ++i) {
      x = x * x % n;
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

uint32_t host_find_psi(uint32_t q, int log_n) {
  const uint64_t n = 1ull << log_n;
  for (uint32_t x = 2; x < q; ++x)
    if (powm(x, n, q) == q - 1) return x;
  return 0;
}

int host_gen_primes(int log_n, int n_q, int n_p, uint32_t* q, uint32_t* p) {
  const uint64_t step = 2ull << log_n;
  // Candidates 1 mod 2N below a bound, scanned downwards.
  auto scan = [&](uint64_t bound, uint32_t* out, int count, uint32_t skip) {
    uint64_t c = (bound - 1) / step * step + 1;
    int got = 0;
    while (got < count) {
      if (c <= step || c < (bound >> 2)) return false;
      if (c != skip && host_is_prime(c)) out[got++] = (uint32_t)c;
      c -= step;
    }
    return true;
  };
  if (n_q < 1 || n_p < 0) return CKKS_EINVAL;
  std::vector<uint32_t> top(1 + n_p);
  if (!scan(1ull << 31, top.data(), 1 + n_p, 0)) return CKKS_EINVAL;
  q[0] = top[0];
  for (int i = 0; i < n_p; ++i) p[i] = top[1 + i];
  if (n_q > 1 && !scan(1ull << 30, q + 1, n_q - 1, 0)) return CKKS_EINVAL;
  return CKKS_OK;
}

// The exemplar 25-30 prime system (Sec. 3.2, Table 2). `count` primes
// = 1 mod 2N nearest to 2^bits (by distance, the smaller first on a tie).
static std::vector<uint32_t> primes_near(int bits, int count, int log_n) {
  const uint64_t step = 2ull << log_n, c = 1ull << bits;
  uint64_t up = (c / step + 1) * step + 1, dn = (c / step) * step + 1;
  if (dn >= c) dn -= step;
  std::vector<uint64_t> found;
  while ((int)found.size() < count) {
    if (host_is_prime(dn)) found.push_back(dn);
    if (host_is_prime(up)) found.push_back(up);
    up += step;
    dn -= step;
  }
  std::sort(found.begin(), found.end(), [&](uint64_t a, uint64_t b) {
    const uint64_t da = a > c ? a - c : c - a, db = b > c ? b - c : c - b;
    return da != db ? da < db : a < b;
  });
  return std::vector<uint32_t>(found.begin(), found.begin() + count);
}

int host_gen_prime_system_2530(int log_n, int n_p, uint32_t* q, uint32_t* p, int* first, int* count) {
  if (log_n < 2 || log_n > 17 || n_p < 1) return CKKS_EINVAL;
  const std::vector<uint32_t> tau = primes_near(25, 4, log_n);
  double b[4];
  for (int i = 0; i < 4; ++i) b[i] = std::log2((double)tau[i]) - 25.0;
  const std::vector<uint32_t> pool = primes_near(30, 200, log_n);
  // deviations a_i = log2(q_i) - 30 that make every rescaling of the cycle
  // divide by exactly 2^40 (levels 1-4) or 2^55 (double rescaling, 5-8)
  const double sb = b[0] + b[1] + b[2] + b[3];
  const double target[11] = {-(b[2] + b[3]), sb / 2, sb / 2, -(b[0] + b[1]), (b[0] + b[1]) / 3,
                             (b[0] + b[1]) / 3, (b[0] + b[1]) / 3, -b[0], -b[1], -b[2], -b[3]};
  std::vector<bool> used(pool.size(), false);
  uint32_t qs[11];
  for (int i = 0; i < 11; ++i) {
    int best = -1;
    double bd = 0;
    for (size_t k = 0; k < pool.size(); ++k) {
      if (used[k]) continue;
      const double d = std::fabs(std::log2((double)pool[k]) - 30.0 - target[i]);
      if (best < 0 || d < bd || (d == bd && pool[k] < pool[best])) {
        best = (int)k;
        bd = d;
      }
    }
    used[best] = true;
    qs[i] = pool[best];
  }
  q[0] = tau[3];
  q[1] = tau[2];
  q[2] = tau[1];
  q[3] = tau[0];
  for (int i = 0; i < 11; ++i) q[4 + i] = qs[i];
  const uint64_t step = 2ull << log_n;
  uint64_t c = ((1ull << 31) - 1) / step * step + 1;
  for (int got = 0; got < n_p; c -= step) {
    if (c < (1ull << 30)) return CKKS_EINVAL;
    bool in_q = false;
    for (int i = 0; i < 15; ++i) in_q |= q[i] == c;
    if (!in_q && host_is_prime(c)) p[got++] = (uint32_t)c;
  }
  static const int kFirst[9] = {2, 4, 0, 2, 4, 3, 2, 1, 0}, kCount[9] = {2, 3, 5, 6, 7, 9, 11, 13, 15};
  for (int l = 0; l < 9; ++l) {
    first[l] = kFirst[l];
    count[l] = kCount[l];
  }
  return CKKS_OK;
}

// ---------------------------------------------------------------------------
// Sampler (SplitMix64, Steele-Lea-Flood 2014)
// ---------------------------------------------------------------------------
uint32_t Sampler::uniform(uint32_t q) {
  uint32_t mask = 1;
  while (mask < q - 1) mask = (mask << 1) | 1;
  for (;;) {
    uint32_t v = (uint32_t)(next() >> 32) & mask;
    if (v < q) return v;
  }
}

// Discrete Gaussian on [-bound, bound] by inversion of its cumulative table.
int64_t Sampler::gaussian(double sigma, int bound) {
  static double cached_sigma = -1;
  static int cached_bound = -1;
  static std::vector<double> cdf;
  if (sigma != cached_sigma || bound != cached_bound) {
    cdf.assign(2 * bound + 1, 0.0);
    double tot = 0;
    for (int v = -bound; v <= bound; ++v) tot += std::exp(-(double)v * v / (2 * sigma * sigma));
    double run = 0;
    for (int v = -bound; v <= bound; ++v) {
      run += std::exp(-(double)v * v / (2 * sigma * sigma)) / tot;
      cdf[v + bound] = run;
    }
    cached_sigma = sigma;
    cached_bound = bound;
  }
  const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
  for (int i = 0; i < 2 * bound; ++i)
    if (u < cdf[i]) return i - bound;
  return bound;
}

void Sampler::ternary(int64_t* s, int n, int hw) {
  if (hw <= 0) {
    for (int i = 0; i < n; ++i) {
      uint32_t v;
      do v = (uint32_t)(next() >> 62);
      while (v == 3);
      s[i] = (int64_t)v - 1;
    }
    return;
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i) s[i] = 0;
  for (int i = 0; i < hw && i < n; ++i) {
    int j = i + (int)(next() % (uint64_t)(n - i));
    std::swap(idx[i], idx[j]);
    s[idx[i]] = (next() >> 63) ? 1 : -1;
  }
}

// ---------------------------------------------------------------------------
// Encoding: slot j <-> zeta^(5^j mod 2N), zeta = exp(i pi / N)
// ---------------------------------------------------------------------------
namespace {
typedef std::complex<double> cd;

// In-place radix-2 FFT: A[k] = sum_j a[j] exp(sign 2 pi i jk / n).
void fft(std::vector<cd>& a, int sign) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const double ang = sign * 2 * M_PI / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        const cd w(std::cos(ang * k), std::sin(ang * k));
        const cd u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}
}  // namespace

void host_encode(const double* re_im, int log_n, double scale, std::vector<int64_t>& coeffs) {
  const int n = 1 << log_n;
  std::vector<cd> zo(n, 0.0);  // z at zeta^(2j+1), j < N
  uint64_t e = 1;
  for (int j = 0; j < n / 2; ++j) {
    const cd u(re_im[2 * j], re_im[2 * j + 1]);
    zo[(e - 1) / 2] = u;
    zo[(2 * n - e - 1) / 2] = std::conj(u);
    e = e * 5 % (2 * n);
  }
  fft(zo, -1);  // sum_j z_(2j+1) exp(-2 pi i jk / N)
  coeffs.resize(n);
  for (int k = 0; k < n; ++k) {
    const cd tw(std::cos(-M_PI * k / n), std::sin(-M_PI * k / n));
    const double v = (zo[k] * tw).real() / n * scale;
    coeffs[k] = (int64_t)(v < 0 ? -std::floor(-v + 0.5) : std::floor(v + 0.5));
  }
}

void host_decode(const uint32_t* res, int nl, const uint32_t* q, int log_n, double scale, double* re_im) {
  const int n = 1 << log_n;
  // Garner mixed-radix digits; inv[i][j] = q_j^-1 mod q_i.
  std::vector<uint32_t> inv((size_t)nl * nl);
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < i; ++j) inv[(size_t)i * nl + j] = invm(q[j] % q[i], q[i]);
  // mixed-radix digits of (Q-1)/2, whose residues are (q_i - 1)/2
  std::vector<uint32_t> half(nl), v(nl);
  for (int i = 0; i < nl; ++i) {
    uint32_t t = (q[i] - 1) / 2;
    for (int j = 0; j < i; ++j) t = mulm((t + q[i] - half[j] % q[i]) % q[i], inv[(size_t)i * nl + j], q[i]);
    half[i] = t;
  }
  std::vector<cd> m(n);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < nl; ++i) {
      uint32_t t = res[(size_t)i * n + k];
      for (int j = 0; j < i; ++j) t = mulm((t + q[i] - v[j] % q[i]) % q[i], inv[(size_t)i * nl + j], q[i]);
      v[i] = t;
    }
    bool neg = false;
    for (int i = nl - 1; i >= 0; --i) {
      if (v[i] != half[i]) {
        neg = v[i] > half[i];
        break;
      }
    }
    // value = d_0 + q_0 (d_1 + q_1 (d_2 + ...)), evaluated from the top digit
    // (Horner): the leading digits of a small value are 0 (or q_i - 1 for a
    // negative one), so nothing overflows however many limbs there are.
    double x = 0;
    if (!neg) {
      for (int i = nl - 1; i >= 0; --i) x = x * (double)q[i] + (double)v[i];
    } else {
      for (int i = nl - 1; i >= 0; --i) x = x * (double)q[i] + (double)(q[i] - 1 - v[i]);
      x = -(x + 1);
    }
    const cd tw(std::cos(M_PI * k / n), std::sin(M_PI * k / n));
    m[k] = x * tw;
  }
  fft(m, +1);  // sum_k m_k zeta^k exp(2 pi i jk / N) = value at zeta^(2j+1)
  uint64_t e = 1;
  for (int j = 0; j < n / 2; ++j) {
    const cd z = m[(e - 1) / 2] / scale;
    re_im[2 * j] = z.real();
    re_im[2 * j + 1] = z.imag();
    e = e * 5 % (2 * n);
  }
}

// ---------------------------------------------------------------------------
// Context tables
// ---------------------------------------------------------------------------
int build_context(ckks_ctx* ctx, const ckks_params* prm) {
  const int log_n = prm->log_n, L = prm->n_q, alpha = prm->n_p, dnum = prm->dnum;
  const int n = 1 << log_n, np = L + alpha;
  ctx->N = n;
  ctx->q.assign(prm->q, prm->q + L);
  ctx->p.assign(prm->p, prm->p + alpha);
  std::vector<uint32_t> pr(np);
  for (int i = 0; i < np; ++i) pr[i] = i < L ? prm->q[i] : prm->p[i - L];

  // per-prime constants
  ctx->pc_host.resize(np);
  for (int i = 0; i < np; ++i) {
    const uint32_t q = pr[i];
    PrimeConst& c = ctx->pc_host[i];
    c.q = q;
    uint32_t m = 1;
    for (int it = 0; it < 5; ++it) m *= 2u - q * m;  // Newton: q m = 1 mod 2^32
    c.m = m;
    const uint32_t r1 = (uint32_t)((1ull << 32) % q);
    const uint32_t r2 = mulm(r1, r1, q);
    c.r1c = centered_h(r1, q);
    c.r2c = centered_h(r2, q);
    c.ninv = invm((uint32_t)(n % q), q);
    c.ninv_sh = shoup_of(c.ninv, q);
    c.mont = r1;
    c.mont_sh = shoup_of(r1, q);
  }

  // levels: windows of the prime list (given) or prefixes (single rescaling)
  ctx->windowed = prm->n_levels > 0;
  if (ctx->windowed) {
    ctx->lvl_first.assign(prm->level_first, prm->level_first + prm->n_levels);
    ctx->lvl_count.assign(prm->level_count, prm->level_count + prm->n_levels);
  } else {
    ctx->lvl_first.assign(L, 0);
    ctx->lvl_count.resize(L);
    for (int l = 0; l < L; ++l) ctx->lvl_count[l] = l + 1;
  }
  const int nlev = ctx->n_levels();

  // key-switching constants, per level (table index tix = level + 1): the
  // level's window [s, s + nl) meets the fixed digits q[j alpha .. (j+1) alpha)
  // in the active digits j = s / alpha ..
  std::vector<uint2> up_cin;
  std::vector<int32_t> up_mat;
  std::vector<int2> up_off((size_t)(std::max(L, nlev) + 1) * dnum, make_int2(0, 0));
  std::vector<int2> up_rows;
  ctx->rows_off.assign(nlev + 1, 0);
  ctx->rows_cnt.assign(nlev + 1, 0);
  for (int tix = 1; tix <= nlev; ++tix) {
    const int s0 = ctx->lvl_first[tix - 1], nl = ctx->lvl_count[tix - 1];
    const int ext = nl + alpha;
    const int j0 = s0 / alpha, digits = (s0 + nl - 1) / alpha - j0 + 1;
    auto prime_of_t = [&](int t) { return t < nl ? s0 + t : L + (t - nl); };
    ctx->rows_off[tix] = (int)up_rows.size();
    for (int j = 0; j < digits; ++j) {
      const int g = j0 + j;
      const int lo = std::max(0, g * alpha - s0), hi = std::min(nl, (g + 1) * alpha - s0);
      up_off[(size_t)tix * dnum + j] = make_int2((int)up_cin.size(), (int)up_mat.size());
      for (int i = lo; i < hi; ++i) {
        const int pi = s0 + i;
        uint32_t hat = 1;  // Q_j / q_i mod q_i over the digit's primes in the window
        for (int i2 = lo; i2 < hi; ++i2)
          if (i2 != i) hat = mulm(hat, pr[s0 + i2] % pr[pi], pr[pi]);
        up_cin.push_back(shoup_pair(mulm(invm(hat, pr[pi]), ctx->pc_host[pi].ninv, pr[pi]), pr[pi]));
      }
      for (int t = 0; t < ext; ++t) {
        const int id = prime_of_t(t);
        const uint32_t d = pr[id];
        for (int i = lo; i < hi; ++i) {
          if (t >= lo && t < hi) {
            up_mat.push_back(0);
            continue;
          }
          uint32_t hat = 1;
          for (int i2 = lo; i2 < hi; ++i2)
            if (i2 != i) hat = mulm(hat, pr[s0 + i2] % d, d);
          up_mat.push_back(centered_h(mulm(hat, ctx->pc_host[id].mont, d), d));
        }
      }
      for (int t = 0; t < ext; ++t)
        if (t < lo || t >= hi) up_rows.push_back(make_int2(j * ext + t, prime_of_t(t)));
    }
    ctx->rows_cnt[tix] = (int)up_rows.size() - ctx->rows_off[tix];
  }
  std::vector<uint2> dn_cin(alpha), dn_pinv(L);
  std::vector<int32_t> dn_mat((size_t)L * alpha);
  for (int k = 0; k < alpha; ++k) {
    const uint32_t pk = pr[L + k];
    uint32_t hat = 1;
    for (int k2 = 0; k2 < alpha; ++k2)
      if (k2 != k) hat = mulm(hat, pr[L + k2] % pk, pk);
    dn_cin[k] = shoup_pair(mulm(invm(hat, pk), ctx->pc_host[L + k].ninv, pk), pk);
  }
  ctx->gadget_p.resize(np);
  for (int i = 0; i < np; ++i) {
    uint32_t P = 1;
    for (int k = 0; k < alpha; ++k) P = mulm(P, pr[L + k] % pr[i], pr[i]);
    ctx->gadget_p[i] = shoup_pair(P, pr[i]);
  }
  for (int i = 0; i < L; ++i) {
    const uint32_t q = pr[i];
    dn_pinv[i] = shoup_pair(invm(ctx->gadget_p[i].x, q), q);
    for (int k = 0; k < alpha; ++k) {
      uint32_t hat = 1;
      for (int k2 = 0; k2 < alpha; ++k2)
        if (k2 != k) hat = mulm(hat, pr[L + k2] % q, q);
      dn_mat[(size_t)i * alpha + k] = centered_h(mulm(hat, ctx->pc_host[i].mont, q), q);
    }
  }
  std::vector<int32_t> rs_mat((size_t)L * (alpha + 1));
  for (int i = 0; i < L; ++i) {
    for (int k = 0; k < alpha; ++k) rs_mat[(size_t)i * (alpha + 1) + k] = dn_mat[(size_t)i * alpha + k];
    rs_mat[(size_t)i * (alpha + 1) + alpha] =
        centered_h(mulm(ctx->gadget_p[i].x, ctx->pc_host[i].mont, pr[i]), pr[i]);
  }
  // byte-plane images of the ModUp, ModDown and fused-rescale matrices for
  // the tensor-core BConv (at most 16 sources: K extent 64)
  std::vector<uint8_t> tc_img;
  std::vector<int2> up_img((size_t)(std::max(L, nlev) + 1) * dnum, make_int2(0, 0));
  std::vector<int2> dn_img((size_t)nlev + 1, make_int2(0, 0)), rs_img((size_t)L + 1, make_int2(0, 0));
  const bool tc_ok = alpha <= 16;
  if (tc_ok) {
    std::vector<int32_t> rows;
    std::vector<uint32_t> tp;
    for (int tix = 1; tix <= nlev; ++tix) {
      const int s0 = ctx->lvl_first[tix - 1], nl = ctx->lvl_count[tix - 1];
      const int ext = nl + alpha;
      const int j0 = s0 / alpha, digits = (s0 + nl - 1) / alpha - j0 + 1;
      for (int j = 0; j < digits; ++j) {
        const int g = j0 + j;
        const int lo = std::max(0, g * alpha - s0), hi = std::min(nl, (g + 1) * alpha - s0), K = hi - lo;
        const int2 o = up_off[(size_t)tix * dnum + j];
        rows.clear();
        tp.clear();
        for (int t = 0; t < ext; ++t) {
          if (t >= lo && t < hi) continue;
          for (int k = 0; k < K; ++k) rows.push_back(up_mat[(size_t)o.y + (size_t)t * K + k]);
          tp.push_back(pr[t < nl ? s0 + t : L + (t - nl)]);
        }
        up_img[(size_t)tix * dnum + j] = append_planes(tc_img, rows.data(), ext - K, K, tp.data());
      }
      rows.assign(dn_mat.begin() + (size_t)s0 * alpha, dn_mat.begin() + (size_t)(s0 + nl) * alpha);
      dn_img[tix] = append_planes(tc_img, rows.data(), nl, alpha, pr.data() + s0);
    }
    if (alpha + 1 <= 16)
      for (int n = 2; n <= L; ++n) rs_img[n] = append_planes(tc_img, rs_mat.data(), n - 1, alpha + 1, pr.data());
  }
  std::vector<uint2> dn_pqinv((size_t)L * L, make_uint2(0, 0));
  for (int l = 1; l < L; ++l)
    for (int i = 0; i < l; ++i)
      dn_pqinv[(size_t)l * L + i] = shoup_pair(invm(mulm(ctx->gadget_p[i].x, pr[l] % pr[i], pr[i]), pr[i]), pr[i]);
  std::vector<uint2> rs_qinv((size_t)L * L, make_uint2(0, 0)), rs_qinv_r((size_t)L * L, make_uint2(0, 0));
  for (int l = 1; l < L; ++l)
    for (int i = 0; i < l; ++i) {
      const uint32_t inv = invm(pr[l] % pr[i], pr[i]);
      rs_qinv[(size_t)l * L + i] = shoup_pair(inv, pr[i]);
      rs_qinv_r[(size_t)l * L + i] = shoup_pair(mulm(inv, (uint32_t)((1ull << 32) % pr[i]), pr[i]), pr[i]);
    }

  // rational rescaling transitions l -> l - 1 (windowed levels only)
  std::vector<int2> rr_drop, rr_rows;
  std::vector<uint2> rr_cin;
  std::vector<int32_t> rr_mat;
  std::vector<RrEpi> rr_epi;
  struct RrOff {
    size_t drop, rows, cin, mat, epi;
  };
  std::vector<RrOff> rr_off(nlev);
  ctx->rr.assign(nlev, RrArgs{});
  if (ctx->windowed) {
    for (int l = 1; l < nlev; ++l) {
      const int s0 = ctx->lvl_first[l], n0 = ctx->lvl_count[l];
      const int s1 = ctx->lvl_first[l - 1], n1 = ctx->lvl_count[l - 1];
      std::vector<int> drop, add;
      for (int g = s0; g < s0 + n0; ++g)
        if (g < s1 || g >= s1 + n1) drop.push_back(g);
      for (int g = s1; g < s1 + n1; ++g)
        if (g < s0 || g >= s0 + n0) add.push_back(g);
      auto prod_mod = [&](const std::vector<int>& set, uint32_t m, int skip) {
        uint32_t r = 1 % m;
        for (int g : set)
          if (g != skip) r = mulm(r, pr[g] % m, m);
        return r;
      };
      const int K = (int)drop.size();
      rr_off[l] = RrOff{rr_drop.size(), rr_rows.size(), rr_cin.size(), rr_mat.size(), rr_epi.size()};
      for (int k = 0; k < K; ++k) {
        const int g = drop[k];
        const uint32_t d = pr[g];
        rr_drop.push_back(make_int2(g - s0, g));
        rr_rows.push_back(make_int2(0, g));
        rr_rows.push_back(make_int2(0, g));
        const uint32_t c = mulm(mulm(prod_mod(add, d, -1), invm(prod_mod(drop, d, g), d), d), ctx->pc_host[g].ninv, d);
        rr_cin.push_back(shoup_pair(c, d));
      }
      for (int i = 0; i < n1; ++i) {
        const int g = s1 + i;
        const uint32_t t = pr[g];
        for (int k = 0; k < K; ++k)
          rr_mat.push_back(centered_h(mulm(prod_mod(drop, t, drop[k]), ctx->pc_host[g].mont, t), t));
        const uint32_t tdi = K ? invm(prod_mod(drop, t, -1), t) : 1;
        RrEpi e;
        e.old_limb = (g >= s0 && g < s0 + n0) ? g - s0 : -1;
        e.ta_tdi = shoup_pair(mulm(prod_mod(add, t, -1), tdi, t), t);
        e.tdi = shoup_pair(tdi, t);
        rr_epi.push_back(e);
      }
      RrArgs& r = ctx->rr[l];
      r.K = K;
      r.s0 = s0;
      r.n0 = n0;
      r.s1 = s1;
      r.n1 = n1;
    }
  }

  // ModDown merged into the rescaling l -> l - 1 (Sec. 6), every level l >= 1:
  // sources p_0 .. p_(alpha-1) and the primes leaving the window, targets the
  // new window (constants as documented with MmArgs)
  std::vector<int2> mm_rows;
  std::vector<uint2> mm_cin;
  std::vector<int32_t> mm_mat;
  std::vector<MmEpi> mm_epi;
  struct MmOff {
    size_t rows, cin, mat, epi;
  };
  std::vector<MmOff> mm_off(nlev);
  ctx->mm.assign(nlev, MmArgs{});
  for (int l = 1; l < nlev; ++l) {
    const int s0 = ctx->lvl_first[l], n0 = ctx->lvl_count[l];
    const int s1 = ctx->lvl_first[l - 1], n1 = ctx->lvl_count[l - 1];
    std::vector<int> src, drop, add;  // prime ids
    for (int k = 0; k < alpha; ++k) src.push_back(L + k);
    for (int g = s0; g < s0 + n0; ++g)
      if (g < s1 || g >= s1 + n1) drop.push_back(g);
    for (int g = s1; g < s1 + n1; ++g)
      if (g < s0 || g >= s0 + n0) add.push_back(g);
    src.insert(src.end(), drop.begin(), drop.end());
    auto prod_ids = [&](const std::vector<int>& ids, uint32_t m, int skip) {
      uint32_t r = 1 % m;
      for (int id : ids)
        if (id != skip) r = mulm(r, pr[id] % m, m);
      return r;
    };
    const int K = (int)src.size();
    mm_off[l] = MmOff{mm_rows.size(), mm_cin.size(), mm_mat.size(), mm_epi.size()};
    for (int u = 0; u < 2; ++u)
      for (int id : src) {
        const int t = id >= L ? n0 + (id - L) : id - s0;
        mm_rows.push_back(make_int2(u * (n0 + alpha) + t, id));
      }
    for (int id : src) {
      const uint32_t m = pr[id];
      uint32_t c = mulm(prod_ids(add, m, -1), invm(prod_ids(src, m, id), m), m);
      if (id < L) c = mulm(c, ctx->gadget_p[id].x, m);
      mm_cin.push_back(shoup_pair(mulm(c, ctx->pc_host[id].ninv, m), m));
    }
    for (int t = 0; t < n1; ++t) {
      const int g = s1 + t;
      const uint32_t m = pr[g];
      for (int id : src) mm_mat.push_back(centered_h(mulm(prod_ids(src, m, id), ctx->pc_host[g].mont, m), m));
      const uint32_t ptd_inv = invm(prod_ids(src, m, -1), m), ta = prod_ids(add, m, -1);
      MmEpi e;
      e.old_limb = (g >= s0 && g < s0 + n0) ? g - s0 : -1;
      e.c1 = shoup_pair(mulm(ta, ptd_inv, m), m);
      e.c2 = shoup_pair(mulm(ta, invm(prod_ids(drop, m, -1), m), m), m);
      e.c3 = shoup_pair(ptd_inv, m);
      mm_epi.push_back(e);
    }
    MmArgs& a = ctx->mm[l];
    a.K = K;
    a.n0 = n0;
    a.s1 = s1;
    a.n1 = n1;
  }

  // twiddles: tw[id][k] = psi^brev(k), itw[id][k] = psi^-brev(k)
  std::vector<uint2> tw((size_t)np * n), itw((size_t)np * n);
  std::vector<uint32_t> pw(n), ipw(n);
  for (int i = 0; i < np; ++i) {
    const uint32_t q = pr[i];
    const uint32_t psi = host_find_psi(q, log_n);
    if (!psi) return CKKS_EINVAL;
    const uint32_t ipsi = invm(psi, q);
    pw[0] = ipw[0] = 1;
    for (int k = 1; k < n; ++k) {
      pw[k] = mulm(pw[k - 1], psi, q);
      ipw[k] = mulm(ipw[k - 1], ipsi, q);
    }
    for (int k = 0; k < n; ++k) {
      const uint32_t e = brev(k, log_n);
      tw[(size_t)i * n + k] = shoup_pair(pw[e], q);
      itw[(size_t)i * n + k] = shoup_pair(ipw[e], q);
    }
  }

  // one device allocation for all tables
  struct Part {
    const void* src;
    size_t bytes;
    size_t off;
  };
  std::vector<Part> parts = {
      {ctx->pc_host.data(), ctx->pc_host.size() * sizeof(PrimeConst), 0},
      {tw.data(), tw.size() * sizeof(uint2), 0},
      {itw.data(), itw.size() * sizeof(uint2), 0},
      {up_cin.data(), up_cin.size() * sizeof(uint2), 0},
      {up_mat.data(), up_mat.size() * sizeof(int32_t), 0},
      {up_off.data(), up_off.size() * sizeof(int2), 0},
      {dn_cin.data(), dn_cin.size() * sizeof(uint2), 0},
      {dn_mat.data(), dn_mat.size() * sizeof(int32_t), 0},
      {dn_pinv.data(), dn_pinv.size() * sizeof(uint2), 0},
      {rs_qinv.data(), rs_qinv.size() * sizeof(uint2), 0},
      {up_rows.data(), up_rows.size() * sizeof(int2), 0},
      {rs_mat.data(), rs_mat.size() * sizeof(int32_t), 0},
      {dn_pqinv.data(), dn_pqinv.size() * sizeof(uint2), 0},
      {rr_drop.data(), rr_drop.size() * sizeof(int2), 0},
      {rr_cin.data(), rr_cin.size() * sizeof(uint2), 0},
      {rr_mat.data(), rr_mat.size() * sizeof(int32_t), 0},
      {rr_epi.data(), rr_epi.size() * sizeof(RrEpi), 0},
      {rr_rows.data(), rr_rows.size() * sizeof(int2), 0},
      {mm_rows.data(), mm_rows.size() * sizeof(int2), 0},
      {mm_cin.data(), mm_cin.size() * sizeof(uint2), 0},
      {mm_mat.data(), mm_mat.size() * sizeof(int32_t), 0},
      {mm_epi.data(), mm_epi.size() * sizeof(MmEpi), 0},
      {tc_img.data(), tc_img.size(), 0},
      {up_img.data(), up_img.size() * sizeof(int2), 0},
      {dn_img.data(), dn_img.size() * sizeof(int2), 0},
      {rs_img.data(), rs_img.size() * sizeof(int2), 0},
      {rs_qinv_r.data(), rs_qinv_r.size() * sizeof(uint2), 0},
  };
  size_t total = 0;
  for (auto& p : parts) {
    p.off = total;
    total += align_up(std::max<size_t>(p.bytes, 16));
  }
  char* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) return CKKS_ENOMEM;
  for (auto& p : parts)
    if (p.bytes && cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(base);
      return CKKS_ECUDA;
    }
  ctx->d_tables = base;
  ctx->table_bytes = total;
  DevParams& dp = ctx->dp;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms < 1) sms = 1;
  dp.sms = sms;
  dp.log_n = log_n;
  dp.L = L;
  dp.alpha = alpha;
  dp.dnum = dnum;
  dp.pc = reinterpret_cast<const PrimeConst*>(base + parts[0].off);
  dp.tw = reinterpret_cast<const uint2*>(base + parts[1].off);
  dp.itw = reinterpret_cast<const uint2*>(base + parts[2].off);
  dp.ks.up_cin = reinterpret_cast<const uint2*>(base + parts[3].off);
  dp.ks.up_mat = reinterpret_cast<const int32_t*>(base + parts[4].off);
  dp.ks.up_off = reinterpret_cast<const int2*>(base + parts[5].off);
  dp.ks.dn_cin = reinterpret_cast<const uint2*>(base + parts[6].off);
  dp.ks.dn_mat = reinterpret_cast<const int32_t*>(base + parts[7].off);
  dp.ks.dn_pinv = reinterpret_cast<const uint2*>(base + parts[8].off);
  dp.ks.rs_qinv = reinterpret_cast<const uint2*>(base + parts[9].off);
  dp.ks.up_rows = reinterpret_cast<const int2*>(base + parts[10].off);
  dp.ks.rs_mat = reinterpret_cast<const int32_t*>(base + parts[11].off);
  dp.ks.dn_pqinv = reinterpret_cast<const uint2*>(base + parts[12].off);
  dp.ks.tc_img = tc_ok ? reinterpret_cast<const uint8_t*>(base + parts[22].off) : nullptr;
  dp.ks.up_img = reinterpret_cast<const int2*>(base + parts[23].off);
  dp.ks.dn_img = reinterpret_cast<const int2*>(base + parts[24].off);
  dp.ks.rs_img = reinterpret_cast<const int2*>(base + parts[25].off);
  dp.ks.rs_qinv_r = reinterpret_cast<const uint2*>(base + parts[26].off);
  for (int l = 1; l < nlev && ctx->windowed; ++l) {
    RrArgs& r = ctx->rr[l];
    r.drop = reinterpret_cast<const int2*>(base + parts[13].off) + rr_off[l].drop;
    r.cin = reinterpret_cast<const uint2*>(base + parts[14].off) + rr_off[l].cin;
    r.mat = reinterpret_cast<const int32_t*>(base + parts[15].off) + rr_off[l].mat;
    r.epi = reinterpret_cast<const RrEpi*>(base + parts[16].off) + rr_off[l].epi;
    r.rows = reinterpret_cast<const int2*>(base + parts[17].off) + rr_off[l].rows;
  }
  for (int l = 1; l < nlev; ++l) {
    MmArgs& a = ctx->mm[l];
    a.rows = reinterpret_cast<const int2*>(base + parts[18].off) + mm_off[l].rows;
    a.cin = reinterpret_cast<const uint2*>(base + parts[19].off) + mm_off[l].cin;
    a.mat = reinterpret_cast<const int32_t*>(base + parts[20].off) + mm_off[l].mat;
    a.epi = reinterpret_cast<const MmEpi*>(base + parts[21].off) + mm_off[l].epi;
  }

  ctx->owns_tables = true;
  const int rc = alloc_scratch(ctx);
  if (rc != CKKS_OK) {
    cudaFree(base);
    ctx->d_tables = nullptr;
  }
  return rc;
}

int alloc_status(ckks_ctx* ctx) {
  void* h = nullptr;
  if (cudaHostAlloc(&h, sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess) return CKKS_ENOMEM;
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaFreeHost(h);
    return CKKS_ECUDA;
  }
  *static_cast<volatile uint32_t*>(h) = 0;
  ctx->h_status = static_cast<uint32_t*>(h);
  ctx->dp.status = static_cast<uint32_t*>(d);
  return CKKS_OK;
}

void free_status(ckks_ctx* ctx) {
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  ctx->h_status = nullptr;
  ctx->dp.status = nullptr;
}

// Key-switching scratch of one context (one execution lane): S (row-phase
// iNTT outputs), T (column-phase outputs), A (accumulators), U (HMult result
// before rescaling).
int alloc_scratch(ckks_ctx* ctx) {
  const DevParams& dp = ctx->dp;
  const int L = dp.L, np = dp.L + dp.alpha;
  const size_t limb = (size_t)1 << dp.log_n;
  // windows are at most L primes; the fused ModDown + rescaling takes the 2
  // alpha P limbs and two top limbs, the merged one 2K limbs
  size_t s_limbs = std::max(L, 2 * dp.alpha + 2);
  for (const MmArgs& m : ctx->mm) s_limbs = std::max(s_limbs, 2 * (size_t)m.K);
  // T: the ModUp limbs (dnum (L + alpha)) followed by room for the ModDown
  // conversions (2L), so that hoisted rotations keep the ModUp limbs
  const size_t t_limbs = std::max((size_t)dp.dnum * np + 2 * (size_t)L, (size_t)2 * L + 4);
  // U holds the [2][alpha + 1] centered coefficients of the fused rescale
  const size_t a_limbs = 2 * (size_t)np, u_limbs = 2 * (size_t)std::max(L, dp.alpha + 1);
  const size_t words = (s_limbs + t_limbs + a_limbs + u_limbs) * limb;
  uint32_t* sc = nullptr;
  if (cudaMalloc(&sc, words * sizeof(uint32_t)) != cudaSuccess) return CKKS_ENOMEM;
  ctx->d_scratch = sc;
  ctx->scratch_bytes = words * sizeof(uint32_t);
  ctx->sc.S = sc;
  ctx->sc.T = ctx->sc.S + s_limbs * limb;
  ctx->sc.A = ctx->sc.T + t_limbs * limb;
  ctx->sc.U = ctx->sc.A + a_limbs * limb;
  return CKKS_OK;
}

}  // namespace ckks
