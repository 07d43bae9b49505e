// Host-side structures and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ckks.h"
#include "arith.cuh"

namespace ckks {

// Key-switching constants on the device (all built by host.cu).
struct KsTables {
  // ModUp (Alg. 1 Q_j -> PQ): for the level with n ciphertext limbs and digit
  // j, up_off[n * dnum + j] = (offset into up_cin, offset into up_mat).
  // up_cin[off + i]: Shoup pair of N^-1 [(Q_j/q_i)^-1]_{q_i} for the digit's
  // i-th prime; up_mat[off + t * a_j + i]: [(Q_j/q_i) 2^32]_{prime_t}
  // centered, t over all n + alpha extended limbs (own-digit rows unused).
  const uint2* up_cin;
  const int32_t* up_mat;
  const int2* up_off;
  // ModDown (P -> Q): dn_cin[k] = Shoup pair of N^-1 [(P/p_k)^-1]_{p_k};
  // dn_mat[i * alpha + k] = [(P/p_k) 2^32]_{q_i} centered; dn_pinv[i] = Shoup
  // pair of [P^-1]_{q_i}.
  const uint2* dn_cin;
  const int32_t* dn_mat;
  const uint2* dn_pinv;
  // Rescale: rs_qinv[l * L + i] = Shoup pair of [q_l^-1]_{q_i}, i < l;
  // rs_qinv_r the same for [q_l^-1 2^32]_{q_i} (applied to a Montgomery-reduced
  // product, which carries 2^-32).
  const uint2* rs_qinv;
  const uint2* rs_qinv_r;
  // ModUp output limbs that need the NTT row phase, per level n (in order of
  // n = 1 .. L): (limb index j (n + alpha) + t in the scratch, prime id) for
  // every digit j and every extended limb t outside the digit.
  const int2* up_rows;
  // ModDown fused with rescaling: rs_mat[i * (alpha + 1) + k] = dn_mat row i
  // followed by [P 2^32]_{q_i} (centered); dn_pqinv[l * L + i] = Shoup pair of
  // [(P q_l)^-1]_{q_i}, i < l.
  const int32_t* rs_mat;
  const uint2* dn_pqinv;
  // Tensor-core BConv (cols_tc.cuh): fp16 byte-plane images of the
  // conversion matrices in the shared-memory layout of the MMA's B operand,
  // one allocation tc_img; entries (byte offset, bytes) per conversion:
  // up_img[tix * dnum + j] (ModUp digit j), dn_img[tix] (ModDown),
  // rs_img[n] (fused ModDown + rescale at n limbs). Null tc_img: the
  // tensor-core kernels are not available (more than 16 sources).
  const uint8_t* tc_img;
  const int2* up_img;
  const int2* dn_img;
  const int2* rs_img;
};

struct DevParams {
  int log_n, L, alpha, dnum;
  const PrimeConst* pc;  // [L + alpha]
  const uint2* tw;       // [L + alpha][N] forward twiddles (w, Shoup companion)
  const uint2* itw;      // [L + alpha][N] inverse twiddles
  KsTables ks;
  int sms = 0;  // streaming multiprocessors of the context's device (grid sizing)
  int pdl;  // host-side launch option: key-switch kernels use programmatic dependent launch
  int tune_tensor = 0;  // host-side option: the fine-tuner also times the tensor-core column shapes
  int unfused = 0;      // host-side option: key-switching operations run the unfused one-step-per-launch form
  int checked = 0;      // host-side option: range checks of operands and results (CKKS_LAUNCH_CHECKED)
  int rows_passes = 3;  // host-side launch option at N = 2^16: row phase in 3 (16 values per
                        // thread, 64 threads per row) or 2 (32 values, 32 threads) passes
  // Bounded device-side waits (mbarrier waits of the tensor-core and bulk-copy
  // kernels): a wait gives up after wait_limit SM clock cycles and sets
  // tc::kStatusTimeout in *status (host-mapped memory of the context, read
  // back by the synchronizing calls as CKKS_ETIMEOUT).
  uint32_t* status = nullptr;
  long long wait_limit = 1ll << 32;
};

// Limb -> prime id. Either an explicit device array, or the extended-
// polynomial rule: limb t (mod per_poly) < n -> q_t, else p_{t - n}.
// Limb t of a polynomial whose ciphertext limbs are the window q[base ..
// base + n) of the prime list is q_(base + t) for t < n, else p_(t - n).
struct IdMap {
  const int* ids;
  int per_poly, n, L;
  int base = 0;
  __host__ __device__ int operator()(int limb) const {
    if (ids) return ids[limb];
    int t = limb % per_poly;
    return t < n ? base + t : L + (t - n);
  }
};

inline IdMap id_ct(int n, int L, int base = 0) { return IdMap{nullptr, n, n, L, base}; }
inline IdMap id_ext(int n, int L, int alpha, int base = 0) { return IdMap{nullptr, n + alpha, n, L, base}; }
inline IdMap id_arr(const int* d) { return IdMap{d, 1 << 30, 0, 0}; }

// Key-switch input modes (what polynomial is key-switched).
enum KsMode { KS_PLAIN = 0, KS_TENSOR = 1, KS_AUTO = 2 };
// What the KeyMult row kernel writes.
enum KmOut { KM_KEYSWITCH = 0, KM_ACC_ALL = 1, KM_MODUP = 2 };

struct MmArgs;

struct KsArgs {
  int n;                 // active ciphertext limbs
  int base;              // their primes are q[base .. base + n) (0 unless the levels are windows)
  int tix;               // level + 1: index of the level's key-switch tables and tuned shapes
  int rows_off, rows_cnt;  // the level's range in the ModUp row table (ks.up_rows)
  int mode;              // KsMode
  const uint32_t* x0;    // KS_PLAIN: d [n][N]; KS_TENSOR: ct1; KS_AUTO: ct
  const uint32_t* x1;    // KS_TENSOR: ct2
  size_t poly_stride0;   // words between b and a of x0 (ciphertexts)
  size_t poly_stride1;
  uint32_t galois;       // KS_AUTO
  const uint32_t* evk;   // [dnum][2][L + alpha][N], Montgomery form
  uint32_t* out;         // [2][n][N] (stride out_stride between polys); [2][n-1][N] with rescale
  size_t out_stride;
  int rescale;           // 1: ModDown fused with rescaling by q_(n-1) (HMult)
  int extra;             // ModDown epilogue: 0 none, 1 HMult (d0, d1), 2 HRot (phi(b), 0)
  int hoisted;           // 1: the ModUp limbs in scratch are of a itself (hoisted rotations), so
                         //    KeyMult applies the automorphism phi_galois while loading them
  const MmArgs* mm;      // with rescale: ModDown merged into the rescaling (host pointer, read by
                         // the launcher; null for ModDown then rescale)
};

// Terms of a linear transform sum_i pt_i (.) HRot_{r_i}(ct) (Par. 4, Par. 5),
// passed to the kernels by value. Term i: automorphism galois[i] (1 for
// r = 0), key evk[i] (null for r = 0: the term is pt_i (.) ct itself) and the
// extended plaintext pt[i] = [pt_level + 1 Q limbs][alpha P limbs], whose
// first P limb is at limb index pt_p[i].
constexpr int kLtMax = 64;
struct LtArgs {
  int count;      // number of terms
  int rotated;    // number of terms with a key
  uint32_t galois[kLtMax];
  const uint32_t* evk[kLtMax];
  const uint32_t* pt[kLtMax];
  int pt_p[kLtMax];
};

// Rational rescaling from the window of level l to that of level l - 1
// (Sec. 3.1, Sec. 3.2): K dropped primes (their product T_drop) are divided
// out and the added primes (T_add) multiplied in. Device tables of the
// transition: drop[k] = (limb of the old window, prime id) of dropped prime
// k; cin[k] = Shoup pair of N^-1 [T_add (T_drop/d_k)^-1]_{d_k}; mat[i K + k]
// = [(T_drop/d_k) 2^32]_{t_i} centered for prime t_i of the new window;
// epi[i] = (old limb of t_i or -1 if added, Shoup pair of [T_add T_drop^-1],
// Shoup pair of [T_drop^-1]) packed as below.
struct RrEpi {
  int old_limb;
  uint2 ta_tdi;  // [T_add T_drop^-1]_t, Shoup pair
  uint2 tdi;     // [T_drop^-1]_t, Shoup pair
};
// ModDown merged into the rescaling (Sec. 6), transition from level l to
// l - 1: one conversion from the alpha P primes and the K - alpha primes that
// leave the window (T_drop their product; T_add that of the entering ones,
// 1 for the usual rescaling by q_l) to the new window's n1 primes.
struct MmEpi {
  int old_limb;  // target's limb in the old window, or -1 for a prime that enters it
  uint2 c1;      // [T_add (P T_drop)^-1]_t, Shoup pair (accumulator limb)
  uint2 c2;      // [T_add T_drop^-1]_t (ModDown extra: d_u for HMult)
  uint2 c3;      // [(P T_drop)^-1]_t (conversion X)
};
struct MmArgs {
  int K;               // sources: p_0 .. p_(alpha-1), then the dropped primes
  int n0, s1, n1;      // old window size; new window start and size
  const int2* rows;    // [2K]: (limb u (n0 + alpha) + t of the accumulator, prime id) for u = 0, 1
  const uint2* cin;    // [K]: Shoup pair of N^-1 [T_add (P T_drop / s_k)^-1 m_k]_{s_k}, m_k = P for a
                       //      dropped prime (its row source is Y P^-1), 1 for p_k
  const int32_t* mat;  // [n1][K]: [(P T_drop / s_k) 2^32]_t, centered
  const MmEpi* epi;    // [n1]
};

struct RrArgs {
  int K;                  // dropped primes
  int s0, n0, s1, n1;     // old and new windows
  const int2* drop;
  const int2* rows;       // [2K]: (unused, prime id of drop[y / 2]) for the row kernels
  const uint2* cin;
  const int32_t* mat;
  const RrEpi* epi;
};

// Kernel ids of the key-switch and rescale pipelines (measurement support).
enum ProfId {
  P_KS_PREP = 0,      // input d, a1*a2 or phi(a) (streaming)
  P_KS_IN_ROWS,       // iNTT row phase of the input
  P_MODUP_COLS,       // iNTT cols, BConv Q_j -> PQ, NTT cols
  P_MODUP_ROWS,       // NTT row phase of the ModUp output
  P_KEYMULT,          // KeyMult + MAC (streaming)
  P_MODDOWN_IN_ROWS,  // iNTT row phase of the P limbs
  P_MODDOWN_COLS,     // iNTT cols, BConv P -> Q, NTT cols
  P_MODDOWN_ROWS,     // NTT row phase of the converted limbs
  P_KS_EPILOGUE,      // (acc - z) P^-1 + d0/d1 or phi(b) (streaming)
  P_RS_IN_ROWS,       // rescale: iNTT rows of the top limb
  P_RS_COLS,          // rescale: iNTT cols, reduce, NTT cols
  P_RS_ROWS,          // rescale: NTT rows
  P_RS_EPILOGUE,      // HMult rescale epilogue: fused into the rescale rows (no launches)
  P_COUNT
};

// Per-kernel timing with CUDA events recorded on the launching stream:
// mark(-1) before the first kernel of an operation, mark(id) after each
// kernel; the time between consecutive marks is charged to the later id.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ids;
  size_t used = 0;
  void mark(cudaStream_t st, int id);
};

// Kernels launched by this library in this process.
uint64_t launch_count();
void count_launch(int k);

// Column kernels with a tunable launch shape, and the table of tuned shapes
// (one per context, shared with its clones). A shape is (tc, sl, z): column
// tile width, slices per block, blocks per tile, plus tp, the conversion
// targets per pass. Entries are atomics so that
// lanes on other host threads may read while ckks_tune writes.
// CK_ROWS is not a column kernel: its entry's tc is the number of register
// passes of the row phase at N = 2^16 (2 or 3), chosen by the same tuner.
enum ColKernel { CK_MODUP = 0, CK_MODDOWN = 1, CK_RS_FUSED = 2, CK_ROWS = 3, CK_COUNT = 4 };

struct ColShape {
  int tc = 0, sl = 0, z = 0, tp = 1;  // tp: conversion targets per pass (1 or 2)
  bool valid() const { return tc > 0; }
};

struct Tuning {
  explicit Tuning(int max_n)
      : max_n(max_n),
        packed(new std::atomic<uint32_t>[CK_COUNT * (max_n + 1)]),
        us(new std::atomic<float>[CK_COUNT * (max_n + 1)]) {
    for (int i = 0; i < CK_COUNT * (max_n + 1); ++i) {
      packed[i].store(0);
      us[i].store(0.f);
    }
  }
  ColShape get(int k, int n) const {
    ColShape s;
    if (k < 0 || k >= CK_COUNT || n < 1 || n > max_n) return s;
    const uint32_t v = packed[k * (max_n + 1) + n].load(std::memory_order_relaxed);
    if (v) {
      s.tc = (int)(v & 0xff);
      s.sl = (int)((v >> 8) & 0xff);
      s.z = (int)((v >> 16) & 0xff);
      s.tp = (int)((v >> 24) & 0xff);
    }
    return s;
  }
  float time_us(int k, int n) const {
    return (k < 0 || k >= CK_COUNT || n < 1 || n > max_n) ? 0.f : us[k * (max_n + 1) + n].load();
  }
  void set(int k, int n, const ColShape& s, float t_us) {
    if (k < 0 || k >= CK_COUNT || n < 1 || n > max_n) return;
    const uint32_t v =
        s.valid() ? (uint32_t)s.tc | ((uint32_t)s.sl << 8) | ((uint32_t)s.z << 16) | ((uint32_t)s.tp << 24) : 0u;
    packed[k * (max_n + 1) + n].store(v, std::memory_order_relaxed);
    us[k * (max_n + 1) + n].store(t_us);
  }
  const int max_n;
  std::unique_ptr<std::atomic<uint32_t>[]> packed;
  std::unique_ptr<std::atomic<float>[]> us;
};

// Scratch buffers owned by the context.
struct Scratch {
  uint32_t* S;  // row-phase iNTT outputs (ModUp input, ModDown P-limbs)
  uint32_t* T;  // column-phase outputs [dnum][L + alpha][N] (ModUp), then [2][L][N] (ModDown)
  uint32_t* A;  // accumulators [2][n + alpha][N]
  uint32_t* U;  // centered coefficients of the fused ModDown + rescale [2][alpha + 1][N]; staged HMult output
  Prof* prof;   // optional stage timing (null or off: no events)
  const Tuning* tune = nullptr;  // tuned column-kernel shapes (null: default rule)
};

inline void prof_mark(const Scratch& sc, cudaStream_t st, int id) {
  if (sc.prof && sc.prof->on) sc.prof->mark(st, id);
}

// ---- launchers (k_basic.cu) ----
void launch_ntt(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, bool inverse, cudaStream_t st);
// Row phase of the iNTT only (the column phase is fused into a consumer).
void launch_rows_inv_only(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, cudaStream_t st);
void launch_permute(const DevParams& dp, const uint32_t* in, uint32_t* out, int limbs, bool to_internal,
                    cudaStream_t st);
// Range check (checked launch mode): every residue of `polys` polynomials
// (poly_stride words apart) of n_q window limbs (primes q[base ..]) followed
// by n_ext auxiliary limbs (p[0 ..]) must be below its prime; a violation sets
// tc::kStatusRange in dp.status.
void launch_check_range(const DevParams& dp, const uint32_t* d, size_t poly_stride, int polys, int n_q, int n_ext,
                        int base, cudaStream_t st);
void launch_hadd(const DevParams& dp, const uint32_t* a, const uint32_t* b, uint32_t* out, int n, int base, size_t sa,
                 size_t sb, size_t so, cudaStream_t st);
void launch_padd(const DevParams& dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base, size_t sa,
                 size_t so, cudaStream_t st);
void launch_pmult(const DevParams& dp, const uint32_t* a, const uint32_t* pt, uint32_t* out, int n, int base, size_t sa,
                  size_t so, cudaStream_t st);
void launch_tensor(const DevParams& dp, const uint32_t* c1, const uint32_t* c2, uint32_t* out, int n,
                   cudaStream_t st);
void launch_automorph(const DevParams& dp, const uint32_t* in, uint32_t* out, int limbs, uint32_t galois,
                      cudaStream_t st);
void launch_small_to_res(const DevParams& dp, const int64_t* v, uint32_t* out, int limbs, IdMap ids,
                         cudaStream_t st);
// out = sign_as * a * s + c + d (mod q), limb-wise; any pointer may be null (term skipped).
void launch_lincomb(const DevParams& dp, const uint32_t* a, const uint32_t* s, int sign_as, const uint32_t* c,
                    const uint32_t* d, uint32_t* out, int limbs, IdMap ids, cudaStream_t st);
// out = a * g_limb + b, with g_limb a per-limb constant (gadget) given as Shoup pairs.
void launch_add_scaled(const DevParams& dp, const uint32_t* a, const uint2* g, const uint32_t* b, uint32_t* out,
                       int limbs, IdMap ids, cudaStream_t st);
void launch_to_mont(const DevParams& dp, uint32_t* data, int limbs, IdMap ids, cudaStream_t st);
void launch_smr(const DevParams& dp, const int64_t* x, int32_t* y, int n, int prime_id, cudaStream_t st);

// ---- launchers (k_keyswitch.cu) ----
// Full key switch of one polynomial (mode), result written per a.extra.
bool col_shape_supported(int log_n, int tc, int sl, int z, int tp);
int tune_columns(const DevParams& dp, const Scratch& sc, Tuning& tu, const KsArgs& lvl, int reps, cudaStream_t st);
void launch_keyswitch(const DevParams& dp, const Scratch& sc, const KsArgs& a, int km_out, uint32_t* km_dst,
                      cudaStream_t st);
// The two halves of launch_keyswitch around KeyMult: ModUp into sc.T, and
// ModDown (with its epilogue / rescaling) from accumulators A.
void launch_ks_modup(const DevParams& dp, const Scratch& sc, const KsArgs& a, cudaStream_t st);
void launch_ks_tail(const DevParams& dp, const Scratch& sc, const KsArgs& a, const uint32_t* A, size_t a_stride,
                    cudaStream_t st);

// Unfused form (k_unfused.cu): every step of the key switch (and of the
// rescale of HMult) as its own launch, intermediates in W
// (unfused_scratch_words(dp) words); non-windowed levels only.
void launch_keyswitch_keymult_only(const DevParams& dp, const KsArgs& a, const uint32_t* T, uint32_t* A,
                                   cudaStream_t st);
size_t unfused_scratch_words(const DevParams& dp);
void launch_keyswitch_unfused(const DevParams& dp, const KsArgs& a, uint32_t* W, cudaStream_t st);

// Persistent streaming stage of a batch (k_keyswitch.cu): work items
// (operation index, limb) over a table of operations.
enum PersKind { PK_KEYMULT = 0, PK_HADD = 1, PK_PADD = 2, PK_PMULT = 3 };
struct PersOp {
  int kind;            // PersKind
  int digits;          // PK_KEYMULT: active digits
  KsArgs ks;           // PK_KEYMULT: the key switch (input, key, window)
  const uint32_t* T;   // PK_KEYMULT: ModUp limbs [digits][n + alpha][N]
  uint32_t* A;         // PK_KEYMULT: accumulators [2][n + alpha][N]
  const uint32_t* x;   // element-wise: ciphertext operand [2][n] (poly stride sx words)
  const uint32_t* y;   // second ciphertext (HAdd, poly stride sy) or plaintext [n] (PAdd, PMult)
  uint32_t* out;       // [2][n], poly stride so
  size_t sx, sy, so;
  int n, base;         // limbs and window start of the element-wise operation
};
// q: device [head, abort] (zeroed before the launch); admitted: host-mapped
// count of admitted operations (items of operation k run once admitted > k).
void launch_persistent(const DevParams& dp, const PersOp* ops, const int2* items, int n_items, int* q,
                       const int* admitted, int blocks, cudaStream_t st);
// ModDown only: acc [2][n + alpha][N] (internal layout) -> out [2][n][N].
void launch_hoisted_rotations(const DevParams& dp, const Scratch& sc, const KsArgs* rots, int count,
                              cudaStream_t st);
void launch_linear_transform(const DevParams& dp, const Scratch& sc, const KsArgs& a, const LtArgs& lt,
                             cudaStream_t st);
void launch_rational_rescale(const DevParams& dp, const Scratch& sc, const RrArgs& r, const uint32_t* in,
                             size_t sin, uint32_t* out, size_t sout, cudaStream_t st);
void launch_moddown(const DevParams& dp, const Scratch& sc, const uint32_t* acc, int n, uint32_t* out,
                    cudaStream_t st);
// Rescale: in [2][n][N] (stride sin) -> out [2][n-1][N] (stride sout).
void launch_rescale(const DevParams& dp, const Scratch& sc, const uint32_t* in, size_t sin, int n,
                    uint32_t* out, size_t sout, cudaStream_t st);

// ---- launchers (k_bconv.cu) ----
// Standalone coefficient-domain BConv, in [k][N] -> out [m][N]; cin: Shoup
// pairs of [(Qs/s_i)^-1]_{s_i} (k entries), mat: [m][k] centered
// [(Qs/s_i) 2^32]_{d_t} (variant 0); abytes: [mp][kp] byte planes of the
// tensor-core variant (variant 1, layout in k_bconv.cu); dst ids per output.
void launch_bconv(const DevParams& dp, const uint32_t* in, int k, const int* src_ids, const uint2* cin,
                  const int32_t* mat, uint32_t* out, int m, const int* dst_ids, int variant, const uint8_t* abytes,
                  int mp, int kp, cudaStream_t st);

}  // namespace ckks

// ---- objects ----
namespace ckks {
// Device bytes held by the objects of a context and its clones, and their
// optional limit (0 = none). Shared by a context, its clones and the objects
// charged to it.
struct MemBudget {
  std::atomic<size_t> used{0};
  std::atomic<size_t> limit{0};
};
}  // namespace ckks

struct ckks_obj {
  int kind;  // 1 ct, 2 pt, 3 sk, 4 evk
  ckks_ctx* ctx;
  size_t bytes = 0;                      // device bytes charged to mem
  std::shared_ptr<ckks::MemBudget> mem;  // the budget they are charged to
};

struct ckks_ctx {
  ckks::DevParams dp;
  int N;
  std::vector<uint32_t> q, p;  // host copies
  std::vector<ckks::PrimeConst> pc_host;
  double scale, sigma;
  int secret_hw;
  uint64_t seed;
  cudaStream_t stream;
  void* d_tables;
  size_t table_bytes;
  bool owns_tables;  // false for a clone (tables belong to the parent context)
  ckks::Scratch sc;
  ckks::Prof prof;
  std::shared_ptr<ckks::Tuning> tune;  // shared with clones
  void* d_scratch;
  size_t scratch_bytes;
  uint32_t* d_unfused = nullptr;  // scratch of the unfused form (allocated on its first use)
  // host-side key-switching constants needed for keygen (gadget P mod prime)
  std::vector<uint2> gadget_p;  // [L + alpha] Shoup pair of [P]_{prime}
  std::string err;
  int device;
  std::shared_ptr<ckks::MemBudget> mem;  // object memory budget, shared with clones
  uint32_t* h_status = nullptr;  // host-mapped status word (dp.status is its device address), shared by
                                 // a context and its clones; freed by the context that owns the tables
  // Levels: level l holds the primes q[lvl_first[l] .. lvl_first[l] +
  // lvl_count[l]). Single rescaling: lvl_first = 0, lvl_count = l + 1. With
  // given windows (the 25-30 prime system) rescaling is rational.
  bool windowed = false;
  std::vector<int> lvl_first, lvl_count;
  std::vector<int> rows_off, rows_cnt;  // per level + 1: ModUp row-table range
  std::vector<ckks::RrArgs> rr;         // per level l >= 1 (windowed): transition l -> l - 1
  std::vector<ckks::MmArgs> mm;         // per level l >= 1: merged ModDown + rescaling l -> l - 1
  int n_levels() const { return (int)lvl_count.size(); }
  int lvl_n(int level) const { return lvl_count[level]; }
  int lvl_base(int level) const { return lvl_first[level]; }
  int cap_limbs(int cap_level) const {
    int m = 0;
    for (int l = 0; l <= cap_level && l < n_levels(); ++l) m = lvl_count[l] > m ? lvl_count[l] : m;
    return m;
  }
  // key-switch level arguments (n, base, table index, ModUp row range)
  void set_level(ckks::KsArgs& k, int level) const {
    k.n = lvl_count[level];
    k.base = lvl_first[level];
    k.tix = level + 1;
    k.rows_off = rows_off[level + 1];
    k.rows_cnt = rows_cnt[level + 1];
  }
};

// Admission pool (ckks_pool_*): bytes granted to running requests, against
// a fixed budget.
struct ckks_pool {
  std::atomic<size_t> used{0};
  size_t budget = 0;
};

struct ckks_ct {
  ckks_obj h;
  uint32_t* d;
  int level, cap_level;
  double scale;
  bool borrowed;
  size_t poly_stride() const { return (size_t)h.ctx->cap_limbs(cap_level) << h.ctx->dp.log_n; }
};

struct ckks_pt {
  ckks_obj h;
  uint32_t* d;
  int level;
  double scale;
  int ext = 0;  // auxiliary (P) limbs stored after the level + 1 Q limbs (extended plaintexts)
};

struct ckks_sk {
  ckks_obj h;
  uint32_t* d_s;  // NTT-domain secret over all L + alpha primes (internal layout)
  std::vector<int64_t> coeffs;
};

struct ckks_evk {
  ckks_obj h;
  uint32_t* d;  // [dnum][2][L + alpha][N], internal layout, Montgomery form
  uint32_t galois;
};

// capi.cu: validation and key-switch arguments of the key-switching
// operations (out's level and scale are set), shared by the direct calls and
// the batched forms.
int prepare_hmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, const ckks_evk* evk, int flags, ckks_ct* out,
                  ckks::KsArgs& k, bool& staged);
int prepare_hauto(ckks_ctx* ctx, const ckks_ct* c, uint32_t galois, const ckks_evk* evk, ckks_ct* out,
                  ckks::KsArgs& k);
uint32_t galois_of_rotation(int r, int log_n);

// host.cu
namespace ckks {
int build_context(ckks_ctx* ctx, const ckks_params* p);
int alloc_scratch(ckks_ctx* ctx);
// Host-mapped status word of bounded device waits (dp.status); freed by free_status.
int alloc_status(ckks_ctx* ctx);
void free_status(ckks_ctx* ctx);
bool host_is_prime(uint64_t n);
uint32_t host_find_psi(uint32_t q, int log_n);
int host_gen_primes(int log_n, int n_q, int n_p, uint32_t* q, uint32_t* p);
int host_gen_prime_system_2530(int log_n, int n_p, uint32_t* q, uint32_t* p, int* first, int* count);
// Encoding (fp64): N/2 complex slots -> N rounded integer coefficients.
void host_encode(const double* re_im, int log_n, double scale, std::vector<int64_t>& coeffs);
// Decoding from canonical residues [n][N] (coefficient domain).
void host_decode(const uint32_t* res, int n, const uint32_t* q, int log_n, double scale, double* re_im);
// Sampler (SplitMix64 stream).
struct Sampler {
  uint64_t state;
  explicit Sampler(uint64_t seed) : state(seed) {}
  uint64_t next() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint32_t uniform(uint32_t q);  // rejection sampling in [0, q)
  int64_t gaussian(double sigma, int bound);
  void ternary(int64_t* s, int n, int hw);
};
}  // namespace ckks
