/*
 * ckks.h -- C ABI of the GB300 RNS-CKKS key-switch library (libckks_gb300.so).
 *
 * The library implements the data-parallel hot path of the 32-bit-word
 * RNS-CKKS scheme described in "Cheddar: A Swift Fully Homomorphic Encryption
 * Library Designed for GPU Architectures" (arxiv 2407.13055): homomorphic
 * multiplication and rotation with hybrid key switching, i.e. the negacyclic
 * NTT/iNTT (Sec. 2.2, Eq. 3), fast basis conversion (Eq. 2), ModUp/ModDown
 * (Sec. 2.3, Alg. 1), the evaluation-key inner product, tensor and
 * relinearization, automorphism (Eq. 4) and rescaling (Sec. 2.1).
 * Every step runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Status: every function returning int returns CKKS_OK (0) or a negative
 *    CKKS_E* code; ckks_last_error() gives a message for the last failure on
 *    that context.
 *  - Ownership: handles are opaque and created through a context. Free each
 *    with ckks_free() before ckks_ctx_destroy(). A ciphertext made by
 *    ckks_ct_wrap_device() borrows the caller's device buffer and never frees
 *    it.
 *  - Ordering: all operations are enqueued on the context's CUDA stream and
 *    are asynchronous unless stated; host buffers are read/written before the
 *    call returns (those calls synchronize the stream). Outputs may alias
 *    inputs only where stated.
 *  - Residues: a polynomial at level l has n = l + 1 limbs, limb i modulo
 *    q_i. Host ("canonical") layout is [limb][N] uint32 residues in [0, q_i)
 *    with the NTT domain in natural order: A[i] = sum_k a_k psi^((2i+1)k) with
 *    psi the smallest x in [2, q) with x^N = -1 mod q. A ciphertext is
 *    [2][n][N] (b then a, Eq. 1). Device buffers use the library's internal
 *    layout (NTT domain in bit-reversed order); only the import/export and
 *    ckks_step_* calls see the canonical layout.
 *  - Auxiliary limbs: an extended polynomial over PQ stores the n ciphertext
 *    limbs followed by the alpha auxiliary limbs p_0 .. p_{alpha-1}.
 *    Digit j of the key-switching gadget is q_{j*alpha} .. q_{j*alpha+alpha-1}.
 *  - Prime ids (ckks_step_*): 0 .. n_q-1 name q_0 .. q_{n_q-1},
 *    n_q .. n_q+n_p-1 name p_0 .. p_{n_p-1}.
 */
#ifndef CKKS_GB300_H
#define CKKS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CKKS_OK 0
#define CKKS_EINVAL (-1)   /* bad argument, shape or parameter */
#define CKKS_ELEVEL (-2)   /* level mismatch, or rescale at level 0 */
#define CKKS_ESCALE (-3)   /* scales differ by more than a relative 2^-20 */
#define CKKS_ENOKEY (-4)   /* missing or wrong kind of evaluation key */
#define CKKS_ENOMEM (-5)   /* device or host allocation failed */
#define CKKS_ECUDA (-6)    /* a CUDA call failed (message in ckks_last_error) */
#define CKKS_ETIMEOUT (-7) /* a bounded device-side wait expired */
#define CKKS_EBUSY (-8)    /* admission refused (memory footprint) */
#define CKKS_ERANGE (-9)   /* checked launch mode: a residue was not below its prime */

#define CKKS_RESCALE 1     /* ckks_hmult flag: rescale the product (Sec. 2.1) */
#define CKKS_RESCALE_MERGED 2 /* ckks_hmult flag: rescale with ModDown merged into it (Sec. 6) */

typedef struct ckks_ctx ckks_ctx;
typedef struct ckks_ct ckks_ct;
typedef struct ckks_pt ckks_pt;
typedef struct ckks_sk ckks_sk;
typedef struct ckks_evk ckks_evk;

/* Scheme parameters (Table 1 of the paper): N = 2^log_n; n_q ciphertext
 * primes q_0..q_{n_q-1}; n_p = alpha auxiliary primes; dnum digits with
 * dnum * alpha >= n_q. Every prime must satisfy q = 1 mod 2N (Eq. 3) and
 * q < 2^31 (Sec. 3). log_n must be 8, 12 or 16. scale is the default
 * encoding scale Delta; secret_hw is the Hamming weight of the ternary secret
 * drawn by ckks_keygen_secret (0 = uniform ternary); sigma is the error
 * standard deviation (3.2); seed seeds the library's own sampler.
 *
 * Levels. With n_levels = 0 (single rescaling), level l holds the primes
 * q_0..q_l and rescaling drops q_l. With n_levels > 0, level l holds the
 * contiguous window q[level_first[l] .. level_first[l] + level_count[l]) of
 * the prime list, as in the 25-30 prime system with its inverted-terminal
 * order (Sec. 3.2, Sec. 3.3), and rescaling from level l to l - 1 is
 * rational (Sec. 3.1): the primes the lower window lacks are divided out and
 * those it adds multiplied in. Key-switching digits are the fixed groups of
 * n_p consecutive primes of the whole list, and the evaluation keys cover
 * every prime, so one key serves every level (Sec. 3.2). */
typedef struct {
  int log_n;
  int n_q;
  const uint32_t* q;
  int n_p;
  const uint32_t* p;
  int dnum;
  double scale;
  int secret_hw;
  double sigma;
  uint64_t seed;
  int n_levels;
  const int* level_first;
  const int* level_count;
} ckks_params;

/* Library's prime rule (Eq. 3 with q < 2^31): q_0 is the largest prime below
 * 2^31 with q = 1 mod 2N, q_1..q_{n_q-1} the largest such primes below 2^30 in
 * decreasing order, p_0..p_{n_p-1} the next largest such primes below 2^31.
 * Host only. Returns CKKS_EINVAL if not enough primes exist. */
int ckks_gen_primes(int log_n, int n_q, int n_p, uint32_t* q_out, uint32_t* p_out);
/* The exemplar 25-30 prime system of Table 2 (Sec. 3.2): 15 ciphertext
 * primes in inverted-terminal order [tau_3, tau_2, tau_1, tau_0, q_0..q_10]
 * (tau_i = 1 mod 2N near 2^25, q_i = 1 mod 2N near 2^30) and 9 levels, each a
 * window of that list: levels 1-4 keep Delta ~ 2^40 by rational rescaling
 * (4 -> 3 and 3 -> 2 drop three q's and add two taus, 2 -> 1 drops four
 * taus and adds two q's, 1 -> 0 drops three q's and adds two taus), levels
 * 5-8 add {tau_i, q_(7+i)} for double rescaling at Delta ~ 2^55. The taus
 * are the four such primes nearest 2^25; each q_i is chosen so that every
 * rescaling of the cycle divides by as nearly 2^40 (2^55) as the primes
 * allow; the n_p auxiliary primes are the largest = 1 mod 2N below 2^31.
 * Writes q_out[15], p_out[n_p], level_first[9], level_count[9]. */
int ckks_gen_prime_system_2530(int log_n, int n_p, uint32_t* q_out, uint32_t* p_out, int* level_first,
                               int* level_count);

/* Context: validates the parameters, builds and uploads the per-prime tables
 * (twiddles, Montgomery/Shoup constants, BConv matrices for every level) and
 * allocates the key-switching scratch. cuda_stream is a cudaStream_t (NULL =
 * legacy default stream) on the current device, which must be an sm_103 GPU. */
int ckks_ctx_create(const ckks_params* params, void* cuda_stream, ckks_ctx** out);
void ckks_ctx_destroy(ckks_ctx* ctx);
/* Ciphertext limbs per polynomial at `level` (level + 1 with single
 * rescaling, the window size with level windows); CKKS_ELEVEL if out of
 * range. */
int ckks_level_limbs(ckks_ctx* ctx, int level);
/* Execution lane: a context that shares `parent`'s parameters and device
 * tables but has its own CUDA stream and key-switching scratch, so that
 * operations issued on different lanes can run concurrently on the GPU.
 * Objects (ciphertexts, keys) of the parent work with the clone; ordering
 * between lanes is the caller's (CUDA events). Destroy clones before their
 * parent. */
int ckks_ctx_clone(ckks_ctx* parent, void* cuda_stream, ckks_ctx** out);
const char* ckks_last_error(ckks_ctx* ctx);
int ckks_sync(ckks_ctx* ctx);            /* cudaStreamSynchronize on the context stream */
void ckks_free(void* handle);            /* any ckks_ct / ckks_pt / ckks_sk / ckks_evk */
/* Device bytes held by the context's tables and scratch (admission control). */
size_t ckks_ctx_device_bytes(ckks_ctx* ctx);
/* Object memory budget (not from the paper: admission control for serving).
 * The device memory of the objects created through a context and its clones
 * (ciphertexts, plaintexts, secret and evaluation keys) is counted together;
 * with a limit (bytes > 0) an allocation that would exceed it fails with
 * CKKS_ENOMEM before the CUDA allocator is called. 0 removes the limit.
 * ckks_memory_in_use returns the bytes those objects hold now. */
int ckks_set_memory_limit(ckks_ctx* ctx, size_t bytes);
size_t ckks_memory_in_use(ckks_ctx* ctx);
/* Device bytes one request of kind `op` (CKKS_OP_*) at `level` holds while it
 * runs on a lane: its input ciphertexts (a plaintext counted as half a
 * ciphertext), its output ciphertext and, for the operations that use it,
 * the lane's key-switching scratch. Resident evaluation keys are shared by
 * requests and are not included. 0 for an unknown op or level. */
size_t ckks_request_bytes(ckks_ctx* ctx, int op, int level);
/* Admission pool (host-side, thread-safe): requests acquire their bytes
 * before they start and release them when done. ckks_pool_acquire returns
 * CKKS_EBUSY (and acquires nothing) when the bytes would exceed the budget;
 * ckks_pool_release returns CKKS_EINVAL for more bytes than are held. */
typedef struct ckks_pool ckks_pool;
int ckks_pool_create(size_t budget_bytes, ckks_pool** out);
int ckks_pool_acquire(ckks_pool* pool, size_t bytes);
int ckks_pool_release(ckks_pool* pool, size_t bytes);
size_t ckks_pool_in_use(const ckks_pool* pool);
void ckks_pool_destroy(ckks_pool* pool);

/* --- keys (Sec. 2.1; hybrid key switching after Han-Ki, cited by the paper) --- */
/* Ternary secret drawn with the library's sampler (SplitMix64 stream). */
int ckks_keygen_secret(ckks_ctx* ctx, uint64_t seed, ckks_sk** out);
/* Secret from N signed coefficients in {-1, 0, 1} (host). */
int ckks_sk_import(ckks_ctx* ctx, const int64_t* coeffs, ckks_sk** out);
/* Relinearization key (s^2 -> s), rotation key (phi_{5^r}(s) -> s) and
 * conjugation key (phi_{2N-1}(s) -> s); dnum digit pairs over all n_q + n_p
 * primes, drawn with the library's sampler. */
int ckks_keygen_relin(ckks_ctx* ctx, const ckks_sk* sk, uint64_t seed, ckks_evk** out);
int ckks_keygen_rot(ckks_ctx* ctx, const ckks_sk* sk, int r, uint64_t seed, ckks_evk** out);
int ckks_keygen_conj(ckks_ctx* ctx, const ckks_sk* sk, uint64_t seed, ckks_evk** out);
/* Key from host residues [dnum][2][n_q + n_p][N] (canonical layout; pair j is
 * (b_j, a_j)). galois = 0 for a relinearization key, else the Galois element
 * k of phi_k (5^r mod 2N for a rotation by r, 2N - 1 for conjugation). */
int ckks_evk_import(ckks_ctx* ctx, const uint32_t* host, uint32_t galois, ckks_evk** out);

/* --- encoding and encryption --- */
/* Encode N/2 complex slots (interleaved re, im) at `level` with `scale`:
 * round(scale * sigma^-1(u)) (Sec. 2.1; slot j <-> zeta^(5^j), zeta =
 * exp(i pi / N)), then NTT on the device. */
int ckks_encode(ckks_ctx* ctx, const double* re_im, int level, double scale, ckks_pt** out);
/* Extended plaintext for ckks_linear_transform: the same integer
 * coefficients reduced modulo the level + 1 ciphertext primes and the n_p
 * auxiliary primes, stored [level + 1 Q limbs][n_p P limbs]. ckks_pmult and
 * ckks_pt_export use its Q limbs. */
int ckks_encode_ext(ckks_ctx* ctx, const double* re_im, int level, double scale, ckks_pt** out);
/* Decode: iNTT on the device, centered CRT lift and FFT on the host; writes
 * N/2 interleaved complex slots. Synchronizes. */
int ckks_decode(ckks_ctx* ctx, const ckks_pt* pt, double* re_im_out);
/* Eq. 1: (b, a) = (-a s + m + e, a) with a uniform and e Gaussian from the
 * library's sampler. */
int ckks_encrypt(ckks_ctx* ctx, const ckks_sk* sk, const ckks_pt* pt, uint64_t seed, ckks_ct** out);
/* Decryption (Sec. 2.1): m = b + a s, NTT domain; a new plaintext at the
 * ciphertext's level and scale. */
int ckks_decrypt(ckks_ctx* ctx, const ckks_sk* sk, const ckks_ct* ct, ckks_pt** out);

/* --- ciphertext and plaintext objects --- */
/* New ciphertext with room for `capacity_level` (capacity_level+1 limbs per
 * polynomial); its level and scale are set by the operation that writes it. */
int ckks_ct_create(ckks_ctx* ctx, int capacity_level, ckks_ct** out);
int ckks_ct_import(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_ct** out);
/* Copies [2][level+1][N] canonical residues to `host` (`words` = its size in
 * uint32). Synchronizes. */
int ckks_ct_export(ckks_ctx* ctx, const ckks_ct* ct, uint32_t* host, size_t words, int* level,
                   double* scale);
/* Re-import host residues into an existing ciphertext (no allocation). */
int ckks_ct_upload(ckks_ctx* ctx, ckks_ct* ct, const uint32_t* host, int level, double scale);
/* Asynchronous forms for pipelining host transfers with work on other
 * streams: they only enqueue the copy and the layout permutation on the
 * context stream (staged through the context's scratch, so in order with its
 * operations). `host` should be page-locked for the copy to be asynchronous;
 * the caller must keep it unchanged (upload) or not read it (export) until
 * the stream has passed the copy (ckks_sync or a CUDA event). */
int ckks_ct_upload_async(ckks_ctx* ctx, ckks_ct* ct, const uint32_t* host, int level, double scale);
int ckks_ct_export_async(ckks_ctx* ctx, const ckks_ct* ct, uint32_t* host, size_t words);
/* Borrow a device buffer of [2][level+1][N] uint32 in the internal layout. */
int ckks_ct_wrap_device(ckks_ctx* ctx, uint32_t* dev_ptr, int level, double scale, ckks_ct** out);
int ckks_ct_info(const ckks_ct* ct, int* level, double* scale, uint32_t** dev_ptr);
int ckks_pt_import(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_pt** out);
/* Extended plaintext from canonical residues [level + 1 + n_p][N] (Q limbs,
 * then P limbs). Synchronizes. */
int ckks_pt_import_ext(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_pt** out);
int ckks_pt_export(ckks_ctx* ctx, const ckks_pt* pt, uint32_t* host, size_t words, int* level,
                   double* scale);

/* --- homomorphic operations (Sec. 2.1), all asynchronous on the context stream --- */
/* HAdd (Sec. 2.1): limb-wise addition; levels must match, scales within
 * 2^-20 (else CKKS_ELEVEL / CKKS_ESCALE). out may alias a or b. */
int ckks_hadd(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out);
/* PAdd (Sec. 2.1): (b + pt, a) limb-wise; the plaintext's level must be >= the
 * ciphertext's and its scale equal within 2^-20. out may alias a. */
int ckks_padd(ckks_ctx* ctx, const ckks_ct* a, const ckks_pt* pt, ckks_ct* out);
/* PMult (Sec. 2.1): ciphertext times plaintext in the NTT domain; scale
 * multiplies. out may alias a. */
int ckks_pmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_pt* pt, ckks_ct* out);
/* HMult: tensor (d0, d1, d2), relinearize d2 with evk (ModUp, KeyMult,
 * ModDown; Sec. 2.3) and, with CKKS_RESCALE, rescale by q_l (rationally
 * with prime windows, Sec. 3.2). With CKKS_RESCALE_MERGED instead, ModDown
 * and the rescaling are one division by P T_drop (the merge of Sec. 6): one
 * basis conversion from P and the primes leaving the window of KeyMult +
 * P d. Its residues differ from CKKS_RESCALE's by a polynomial of a few
 * units, far below the encryption noise; level and scale are the same.
 * Other flag bits: CKKS_EINVAL. out must not alias a or b. */
int ckks_hmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, const ckks_evk* evk, int flags,
               ckks_ct* out);
/* Rescale (Sec. 2.1; rational with level windows, Sec. 3.1): c'_i =
 * (c_i - [c_l]_centered) * q_l^-1, scale /= q_l.
 * out must not alias in. */
int ckks_rescale(ckks_ctx* ctx, const ckks_ct* in, ckks_ct* out);
/* HRot by r slots to the left (Eq. 4 with k = 5^r mod 2N) with evk from
 * ckks_keygen_rot(r) or ckks_evk_import(galois = k). out must not alias ct. */
int ckks_hrot(ckks_ctx* ctx, const ckks_ct* ct, int r, const ckks_evk* evk, ckks_ct* out);
/* HConj (Sec. 2.1, Eq. 4 with k = 2N - 1) with evk from ckks_keygen_conj.
 * out must not alias ct. */
int ckks_hconj(ckks_ctx* ctx, const ckks_ct* ct, const ckks_evk* evk, ckks_ct* out);
/* Hoisted rotations (Par. 5, Fig. 5): outs[i] = HRot(ct, r[i]) under evks[i]
 * for i < count, sharing one ModUp of ct's a part. Because the BConv of the
 * ModUp is centered (odd), ModUp commutes with the automorphism exactly and
 * every output is bit-identical to a separate ckks_hrot. Each ModDown reads
 * the automorphism of the shared ModUp limbs while multiplying by the key.
 * Outputs must be distinct, must not alias ct and need capacity >= ct's
 * level. Asynchronous on the context stream; count = 0 does nothing. */
int ckks_hrot_hoisted(ckks_ctx* ctx, const ckks_ct* ct, int count, const int* r, const ckks_evk* const* evks,
                      ckks_ct* const* outs);
/* Linear transform (Par. 4, Par. 5): out = sum_{i < count} pts[i] (.) HRot(ct, r[i])
 * (r[i] = 0: pts[i] (.) ct, no key needed; evks[i] may be NULL there).
 * The rotated terms share one ModUp of ct's a part; their KeyMult + MAC,
 * each multiplied by its plaintext in the extended basis Q_l P, accumulate
 * in one kernel, and ONE ModDown of that sum follows (so the key-switch
 * rounding differs from summing separate HRot + PMult results, within the
 * same noise bound); the b parts enter as one accumulated sum of
 * plaintext-weighted automorphisms. pts[i]: extended plaintexts
 * (ckks_encode_ext / ckks_pt_import_ext) at a level >= ct's, all of one
 * scale. 1 <= count <= 64. out: level of ct, scale ct.scale * pt scale;
 * it must not alias ct. Asynchronous on the context stream. */
int ckks_linear_transform(ckks_ctx* ctx, const ckks_ct* ct, int count, const int* r, const ckks_evk* const* evks,
                          const ckks_pt* const* pts, ckks_ct* out);

/* --- batched form: many independent ciphertext operations at mixed levels ---
 * A batch is a list of independent operations (no operation's output may be
 * an input or output of another one in the same batch) issued across `lanes`
 * execution lanes (ckks_ctx_clone) that fork from and join into the context
 * stream. use_graph is a set of mode flags:
 *  CKKS_BATCH_GRAPH: the whole list is captured once into a CUDA graph and
 *    each ckks_batch_run is a single graph launch;
 *  CKKS_BATCH_PERSISTENT: stage-major form with a persistent kernel. Each
 *    key-switching operation (HMult, HRot, HConj) runs its ModUp on its lane
 *    into working memory of its own (the batch allocates (dnum + 2)(n + alpha)
 *    limbs per such operation at creation), the lanes join, ONE persistent
 *    kernel runs the KeyMult + MAC (Par. 1) of all of them and every HAdd,
 *    PAdd and PMult of the batch, taking (operation, limb) work items from a
 *    device queue (limb-major, so each evaluation-key limb is read once per
 *    batch and reused from L2 by every operation with that key), then the
 *    lanes run the ModDown tails. Rescale operations run whole on their lanes.
 *    The persistent kernel runs an operation's items only once the operation
 *    is admitted (ckks_batch_run_admit, ckks_batch_admit); a wait for
 *    admission is bounded by the context's wait limit (ckks_set_wait_limit),
 *    after which the kernel stops and the next synchronizing call returns
 *    CKKS_ETIMEOUT.
 * Operations follow the single-operation entry points (same checks, same
 * results, bit for bit in every mode). */
#define CKKS_BATCH_GRAPH 1
#define CKKS_BATCH_PERSISTENT 2
#define CKKS_OP_HMULT 1   /* ckks_hmult(a, b, evk, flags, out) */
#define CKKS_OP_HROT 2    /* ckks_hrot(a, r, evk, out) */
#define CKKS_OP_HCONJ 3   /* ckks_hconj(a, evk, out) */
#define CKKS_OP_PMULT 4   /* ckks_pmult(a, pt, out) */
#define CKKS_OP_RESCALE 5 /* ckks_rescale(a, out) */
#define CKKS_OP_HADD 6    /* ckks_hadd(a, b, out) */
#define CKKS_OP_PADD 7    /* ckks_padd(a, pt, out) */
typedef struct {
  int op;
  int flags;
  int r;
  const ckks_ct* a;
  const ckks_ct* b;
  const ckks_pt* pt;
  const ckks_evk* evk;
  ckks_ct* out;
} ckks_op;
typedef struct ckks_batch ckks_batch;
/* Validates the list by running it once (synchronizes), then captures it if
 * use_graph. The batch references (does not own) the operands. */
int ckks_batch_create(ckks_ctx* ctx, const ckks_op* ops, int count, int lanes, int use_graph, ckks_batch** out);
/* Enqueue the whole list on the context stream (asynchronous); a persistent
 * batch admits every operation. */
int ckks_batch_run(ckks_batch* batch);
/* Persistent batches only: enqueue the list with only operations
 * 0 .. admitted - 1 admitted to the persistent stage (0 <= admitted <=
 * count); the others' KeyMult / element-wise items wait, bounded, until
 * ckks_batch_admit raises the count (the host may do so while the batch runs,
 * which is how operations that arrive later join a running launch). A count
 * lower than the previous run's first waits for the batch's earlier runs.
 * The outputs of operations never admitted before the wait limit are
 * undefined, and the next synchronizing call returns CKKS_ETIMEOUT.
 * CKKS_EINVAL for a non-persistent batch or a count out of range. */
int ckks_batch_run_admit(ckks_batch* batch, int admitted);
/* Raises the admitted count of a persistent batch (never lowers it);
 * takes effect in the running persistent kernel. */
int ckks_batch_admit(ckks_batch* batch, int admitted);
void ckks_batch_destroy(ckks_batch* batch);

/* --- served form: continuous batching of single requests (not in the paper,
 * which runs one operation at a time; Sec. 5.2 names multi-query batching as
 * a different model) ---
 * A request is one HMult with rescaling (CKKS_OP_HMULT, flags CKKS_RESCALE)
 * or one HRot by r (CKKS_OP_HROT) that arrives arrival_s seconds after the
 * run starts. ckks_serve_run serves a list of them on n_lanes execution lanes
 * (contexts on their own streams, e.g. clones): a request is admitted, in
 * arrival order, once its arrival time has passed, a lane is idle and the
 * pool grants its `bytes` (its device footprint, ckks_request_bytes); it then
 * runs on that lane, so admitted requests overlap on the GPU, and requests
 * that arrive meanwhile are admitted as lanes and bytes free up. Completion
 * is a CUDA event recorded after the request on its lane; its bytes go back
 * to the pool. The loop runs on the calling thread (polling; it returns once
 * every request has completed). Times are host steady-clock seconds since
 * the start of the run. The lanes' device must be the current device; the
 * loop allocates no device memory (one CUDA event per lane).
 *  lanes:     n_lanes contexts (1 <= n_lanes <= 64), all of the same
 *             parameters; lane l's requests are enqueued on lanes[l]'s stream.
 *  pool:      admission pool; it may already hold bytes (resident keys).
 *  reqs:      n requests, sorted by arrival_s (CKKS_EINVAL otherwise); a
 *             request whose out is NULL writes to lane_outs[lane].
 *  lane_outs: n_lanes output ciphertexts, or NULL when every request has its
 *             own out.
 *  hooks:     NULL for the library's own issue and completion; non-NULL
 *             replaces both (host tests of the scheduling: issue(user, i,
 *             lane) starts request i on the lane and returns CKKS_OK or an
 *             error, query(user, lane) returns 1 once the lane's request has
 *             completed, 0 while it runs, a negative code on failure; lanes
 *             may then be NULL).
 *  done:      n records, filled by request index: admission and completion
 *             times, the lane (-1 for a request that was never admitted).
 *  order:     NULL or n request indices in completion order (after a
 *             failure only the completed requests' entries are written).
 * Errors: CKKS_EINVAL for bad arguments, or a request whose bytes exceed
 * what the pool can ever grant it (its budget less the bytes it held at the
 * start); the first failing issue or completion ends the run with that code
 * after waiting for the requests already running. */
typedef struct {
  int op;
  int r;
  double arrival_s;
  const ckks_ct* a;
  const ckks_ct* b;
  const ckks_evk* evk;
  ckks_ct* out;
  size_t bytes;
} ckks_request;
typedef struct {
  double start_s;
  double end_s;
  int lane;
} ckks_request_done;
typedef struct {
  int (*issue)(void* user, int request, int lane);
  int (*query)(void* user, int lane);
  void* user;
} ckks_serve_hooks;
int ckks_serve_run(ckks_ctx* const* lanes, int n_lanes, ckks_pool* pool, const ckks_request* reqs, int n,
                   ckks_ct* const* lane_outs, const ckks_serve_hooks* hooks, ckks_request_done* done, int* order);

/* --- rescale without allocation (the paper has no counterpart to this entry
 * point; it exists for callers that must not allocate device memory while
 * they run, such as a serving loop with a latency budget, where cudaMalloc can
 * synchronize the whole device or fail when memory is tight). --- */
/* Fixed size, in uint32 words, of the library's static device scratch used by
 * ckks_rescale_noalloc: 2^21 words = 8 MiB, held on every GPU that loads the
 * library until the process exits. */
#define CKKS_NOALLOC_SCRATCH_WORDS (1u << 21)
/* Same result as ckks_rescale (single rescaling, c'_i = (c_i - [c_l]) q_l^-1)
 * on caller-owned device buffers, with no allocation of any kind.
 *  in_dev:  [2][level+1][N] uint32 residues, internal layout (as a ciphertext
 *           created with capacity `level`; see ckks_ct_info).
 *  out_dev: [2][level][N] uint32, written in the same layout; must not
 *           overlap in_dev.
 * The scratch is a file-scope device array shared by every call: it needs
 * (2 + 2*level) * N <= CKKS_NOALLOC_SCRATCH_WORDS (at N = 2^16: level <= 15),
 * larger requests return CKKS_EINVAL with a message and launch nothing.
 * Calls whose kernels overlap on the GPU (other streams, other threads)
 * race on that array; calls in order on one stream do not. Every scratch word
 * is written before it is read in each call, so nothing needs clearing.
 * The context's device must be the current device (CKKS_EINVAL otherwise,
 * before any device work). The first call on each device looks up the
 * array's device address with that device current (cudaGetSymbolAddress);
 * make that first call before any stream capture. Asynchronous on the
 * context stream. */
int ckks_rescale_noalloc(ckks_ctx* ctx, const uint32_t* in_dev, int level, uint32_t* out_dev);

/* --- launch options ---
 * CKKS_LAUNCH_PDL (default on): the key-switch kernels use programmatic
 * dependent launch, so each one is scheduled and loads its twiddles and
 * constants while its predecessor on the stream finishes (lower latency for
 * one stream of operations). Its blocks then hold SM resources while they
 * wait, which can cost throughput when several lanes share the GPU. A clone
 * inherits its parent's flags when it is created. */
#define CKKS_LAUNCH_PDL 1
/* CKKS_TUNE_TENSOR (default off): ckks_tune also times the tensor-core
 * shapes of the column kernels (tp in {8, 16}, below). They are slower than
 * the CUDA-core shapes when several lanes share the GPU (their larger
 * shared-memory blocks crowd out the other lanes' kernels), while the tuner
 * times one kernel alone, so they are only candidates on request. */
#define CKKS_TUNE_TENSOR 2
/* CKKS_LAUNCH_UNFUSED (default off): HMult (with or without CKKS_RESCALE),
 * HRot and HConj run the unfused form instead, one kernel launch per step
 * with every intermediate in device memory (tensor or automorphism, full
 * iNTT, one BConv per ModUp digit, full NTTs, KeyMult, iNTT of the P limbs,
 * BConv P -> Q, NTT, ModDown epilogue, and for rescaling iNTT of the top
 * limb, reduction, NTT, epilogue): the mechanism baseline of the fusion
 * ablation (Sec. 5, Table 8), same residues. Single rescaling only (CKKS_EINVAL
 * on a windowed context; CKKS_RESCALE_MERGED is refused); the first such
 * operation allocates the form's scratch on the context. */
#define CKKS_LAUNCH_UNFUSED 4
/* CKKS_LAUNCH_CHECKED (default off): checked mode. Every homomorphic
 * operation first checks, on the device, that each residue of its ciphertext
 * and plaintext operands is below its prime (q_i of the level's window, p_k of
 * the auxiliary limbs), and checks its output the same way after it ran;
 * uploads and imports of ciphertexts, plaintexts and evaluation keys check
 * what they wrote. A violation marks the context's status word: the next
 * synchronizing call on the context or a clone (ckks_sync, exports, imports,
 * decryption) returns CKKS_ERANGE and clears the mark; the results of the
 * operations since the previous synchronizing call are then undefined, and
 * the context stays usable. The checks cost one extra read of every operand
 * and result. No kernel indexes memory by a residue, so residues out of range
 * give wrong values, never out-of-bounds accesses; the kernels' indices follow
 * from the launch geometry and host-checked arguments only. Operations of a
 * persistent stage-major batch (CKKS_BATCH_PERSISTENT) are not checked. */
#define CKKS_LAUNCH_CHECKED 8
int ckks_set_launch_flags(ckks_ctx* ctx, int flags);

/* Bounded device-side waits. The tensor-core and bulk-copy kernels wait on
 * shared-memory barriers (for their bulk copies and matrix products); each
 * wait gives up after `cycles` SM clock cycles (default 2^32, about two
 * seconds), marks the context's status word, frees what the block holds and
 * returns. The next synchronizing call on the context or any of its clones
 * (ckks_sync, exports, decryption, the step entry points) then returns
 * CKKS_ETIMEOUT and clears the mark; the outputs of the operations issued
 * since the previous synchronizing call are undefined, and the context stays
 * usable. The limit applies to kernels enqueued after the call; a clone
 * inherits the parent's limit when it is created. CKKS_EINVAL if cycles < 1.
 * (Not from the paper: a guard of this implementation's asynchronous
 * kernels.) */
int ckks_set_wait_limit(ckks_ctx* ctx, long long cycles);

/* --- launch-shape fine-tuning (Sec. 4.2, "Fine-tuning"; Sec. 6) ---
 * The three BConv column kernels (ModUp conversion, ModDown conversion,
 * fused ModDown + rescale conversion) can run in several launch shapes
 * (tc, sl, z, tp): column-tile width tc in {4, 8} columns, sl in {2, 4, 8}
 * thread slices per block sharing the tile, z in 1..4 blocks per tile
 * splitting the conversion targets, and tp in {1, 2} targets converted per
 * pass over the shared inputs with CUDA-core multiply-adds. tp in {8, 16}
 * selects the tensor-core form instead (N = 2^12 and 2^16, at most 16
 * conversion sources, z = 1; (tc, sl) in {(8, 2), (8, 4), (4, 4), (4, 8)}):
 * the conversion of a tile to tp targets at a time is one exact fp16 matrix
 * product on the tensor cores (tcgen05) over byte planes of the sources and
 * of the matrix (Eq. 2 as a matrix product, Sec. 4.2). Every shape computes
 * identical values; only time changes. A context and its clones share one
 * table of shapes per (kernel, level); levels without an entry use a fixed
 * rule. */
#define CKKS_COL_MODUP 0
#define CKKS_COL_MODDOWN 1
#define CKKS_COL_RS_FUSED 2
/* Not a column kernel: the row phase of the NTT at N = 2^16 runs as 2
 * register passes (32 values per thread, radix 2^5 x 2^5) or 3 (16 values,
 * 2^4 x 2^3 x 2^3); the entry's tc is the number of passes (sl = z = tp = 1),
 * tuned on the level's ModUp NTT rows and used by that level's key
 * switches. tc = 4 and 5 select the three-pass form whose forward rows take
 * 2 (4) and 4 (5) row pairs per block and stage each pair's input in shared
 * memory with bulk copies (cp.async.bulk) that overlap the previous pair's
 * arithmetic (bounded waits, see ckks_set_wait_limit). tc = 6 selects the
 * three-pass form with the second and third passes' twiddles copied into
 * shared memory by asynchronous copies (cp.async) instead of held in
 * registers (64 registers, 8 blocks of 4 warps per SM), forward and inverse
 * rows; ckks_tune does not time it (slower than form 3 on GB300, most of all
 * for the rows with fused epilogues), it is set by hand only. Without an
 * entry: 3. */
#define CKKS_ROW_PASSES 3
/* Times every candidate shape of the three kernels at `level` (reps launches
 * each, CUDA events on the context stream, on the context's scratch), and at
 * N = 2^16 both row-phase forms, and records the fastest. Synchronizes the stream: do not call it while the
 * stream is being captured. level in [0, n_q - 1] (the fused rescale kernel
 * is tuned for level >= 1). */
int ckks_tune(ckks_ctx* ctx, int level, int reps);
/* Tuned shape of `kernel` at `level` and its mean launch time in
 * microseconds; *tc = 0 when the level has no entry. */
int ckks_tune_get(ckks_ctx* ctx, int kernel, int level, int* tc, int* sl, int* z, int* tp, float* us);
/* Sets a shape by hand (tc in {4, 8}, sl in {2, 4, 8}, z in 1..4, tp in
 * {1, 2}; at N = 2^8 only tc = 8, since a slice must be whole warps; the
 * tensor-core shapes listed above; for CKKS_ROW_PASSES tc in 2 .. 6 at
 * N = 2^16), or clears the entry with tc = 0. A tensor-core shape for a
 * conversion with more than 16 sources runs the fixed CUDA-core rule.
 * Changes no value any operation computes. */
int ckks_tune_set(ckks_ctx* ctx, int kernel, int level, int tc, int sl, int z, int tp);

/* --- Table 3 on this GPU: modular multiplication methods (Sec. 4.1) ---
 * Runs out[i] = a[i] * b^rounds mod q (q = prime_id of the context) as eight
 * independent chains per thread with one reduction method per call, and
 * reports the timed kernel's milliseconds (one untimed warm-up run first).
 * Every method returns exactly the same values. Inputs must be < q.
 * Synchronous; allocates its own device buffers. */
#define CKKS_MODMUL_BARRETT 0    /* 64-bit Barrett: mulwide, mulhi64, mullo64 */
#define CKKS_MODMUL_MONTGOMERY 1 /* unsigned Montgomery: mulwide32, mullo32, mulwide32 + add64 */
#define CKKS_MODMUL_SHOUP 2      /* Shoup (constant operand): mulhi32, 2 mullo32 */
#define CKKS_MODMUL_SMR 3        /* signed Montgomery (Alg. 2): mulwide32, mullo32, mulhi32 */
int ckks_bench_modmul(ckks_ctx* ctx, int method, int prime_id, uint32_t b, const uint32_t* a, int n, int rounds,
                      uint32_t* out, float* ms);

/* Integer multiply issue rate of this GPU (the denominator of the integer-ALU
 * roofline): 8 blocks of 256 threads per SM, each thread advancing 16
 * independent dependent chains of one instruction form for `rounds` steps on
 * the context stream. *ops = instructions executed (per thread lane),
 * *ms = CUDA-event time of the timed launch (one untimed launch first).
 * CKKS_EINVAL on a bad argument. */
#define CKKS_INTOP_MAD_LO 0   /* mad.lo.u32 */
#define CKKS_INTOP_MAD_HI 1   /* mad.hi.u32 */
#define CKKS_INTOP_MAD_WIDE 2 /* mad.wide.u32 (32 x 32 + 64) */
int ckks_bench_intop(ckks_ctx* ctx, int op, int rounds, double* ops, float* ms);

/* --- measurement support --- */
/* Number of kernel ids reported by ckks_profile_read. */
#define CKKS_PROF_KERNELS 13
/* enable = 1: clear and start recording one CUDA event on the context stream
 * after every stage of the key-switch and rescale pipelines (input prep,
 * ModUp rows/columns/rows, KeyMult, ModDown rows/columns/rows, epilogue, and
 * the four rescale stages);
 * enable = 0: stop recording. */
int ckks_profile(ckks_ctx* ctx, int enable);
/* Synchronizes, then writes per kernel id the total device milliseconds
 * between the event before and the event after each launch, and the number
 * of launches (arrays of CKKS_PROF_KERNELS entries). */
int ckks_profile_read(ckks_ctx* ctx, double* total_ms, uint64_t* launches);
/* Name of a kernel id, or NULL when out of range. */
const char* ckks_profile_name(int id);
/* Kernels this library has launched in this process. */
uint64_t ckks_launch_count(void);

/* --- step-level entry points on host buffers (canonical layout; synchronous).
 * They run the same kernels as the operations above and exist so that each
 * step of the path can be compared with a reference on its own. --- */
/* Alg. 2 (signed Montgomery reduction) on n inputs x in [-q 2^31, q 2^31). */
int ckks_step_smr(ckks_ctx* ctx, const int64_t* x, int n, int prime_id, int32_t* y);
/* NTT (inverse = 0) or iNTT (inverse = 1) of `limbs` limbs in place;
 * prime_ids[i] names the prime of limb i. */
int ckks_step_ntt(ckks_ctx* ctx, uint32_t* data, int limbs, const int* prime_ids, int inverse);
/* Eq. 2 on coefficient-domain limbs: in [k][N] modulo src primes ->
 * out [m][N] modulo dst primes. variant 0 = CUDA-core lazy-SMR GEMM,
 * 1 = byte-split INT8 tensor-core GEMM (mma.sync, INT32 accumulation). */
int ckks_step_bconv(ckks_ctx* ctx, const uint32_t* in, int k, const int* src_ids, uint32_t* out,
                    int m, const int* dst_ids, int variant);
/* Tensor: ct1, ct2 [2][n_q][N] -> out [3][n_q][N] (d0, d1, d2). */
int ckks_step_tensor(ckks_ctx* ctx, const uint32_t* ct1, const uint32_t* ct2, int n_q, uint32_t* out);
/* NTT-domain automorphism out[j] = in[((2j+1)k mod 2N - 1)/2] (Eq. 4) on
 * `limbs` limbs. */
int ckks_step_automorph(ckks_ctx* ctx, const uint32_t* in, int limbs, uint32_t galois, uint32_t* out);
/* ModUp of d [n_q][N] (NTT domain): out [digits][n_q + n_p][N]. */
int ckks_step_modup(ckks_ctx* ctx, const uint32_t* d, int n_q, uint32_t* out);
/* ModUp fused with KeyMult+MAC: acc [2][n_q + n_p][N] = sum_j ModUp_j(d) * evk_j. */
int ckks_step_keyswitch_acc(ckks_ctx* ctx, const uint32_t* d, int n_q, const ckks_evk* evk, uint32_t* acc);
/* ModDown of acc [2][n_q + n_p][N] -> out [2][n_q][N]. */
int ckks_step_moddown(ckks_ctx* ctx, const uint32_t* acc, int n_q, uint32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* CKKS_GB300_H */
