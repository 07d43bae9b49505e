// C ABI of the library (declarations and documentation in include/ckks.h).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"
#include "tc.cuh"

using namespace ckks;

namespace {

const int K_CT = 1, K_PT = 2, K_SK = 3, K_EVK = 4;

int fail(ckks_ctx* ctx, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(ckks_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_check(ckks_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CKKS_OK;
  return fail(ctx, CKKS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Synchronizes the context stream, then reports a bounded device-side wait
// that expired since the last check (status word set by the kernels).
int sync_check(ckks_ctx* ctx, const char* what) {
  const int rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), what);
  if (rc != CKKS_OK) return rc;
  if (ctx->h_status) {
    volatile uint32_t* st = ctx->h_status;
    const uint32_t v = *st;
    if (v & ckks::tc::kStatusRange) {
      *st = 0;
      return fail(ctx, CKKS_ERANGE,
                  "%s: checked mode found a residue not below its prime; results of the operations since the "
                  "last synchronizing call are undefined",
                  what);
    }
    if (v) {
      *st = 0;
      return fail(ctx, CKKS_ETIMEOUT,
                  "%s: a bounded device-side wait expired (wait limit %lld cycles); results of the operations "
                  "since the last synchronizing call are undefined",
                  what, (long long)ctx->dp.wait_limit);
    }
  }
  return CKKS_OK;
}

// Status after enqueuing kernels: launch errors only (asynchronous faults
// surface at the next synchronizing call).
int launched(ckks_ctx* ctx, const char* what) { return cuda_check(ctx, cudaGetLastError(), what); }

// Checked launch mode (CKKS_LAUNCH_CHECKED): device-side range checks of a
// ciphertext's or plaintext's residues at its level, enqueued on the context
// stream; a violation surfaces as CKKS_ERANGE at the next synchronizing call.
static void check_ct(ckks_ctx* ctx, const ckks_ct* c) {
  if (ctx->dp.checked && c)
    launch_check_range(ctx->dp, c->d, c->poly_stride(), 2, ctx->lvl_n(c->level), 0, ctx->lvl_base(c->level),
                       ctx->stream);
}
static void check_pt(ckks_ctx* ctx, const ckks_pt* p) {
  if (ctx->dp.checked && p)
    launch_check_range(ctx->dp, p->d, 0, 1, ctx->lvl_n(p->level), p->ext, ctx->lvl_base(p->level), ctx->stream);
}

size_t limb_words(const ckks_ctx* ctx) { return (size_t)ctx->N; }

bool scales_match(double a, double b) { return std::fabs(a - b) <= std::ldexp(std::fabs(a), -20); }

template <class T>
T* new_obj(ckks_ctx* ctx, int kind) {
  T* o = new (std::nothrow) T();
  if (!o) return nullptr;
  o->h.kind = kind;
  o->h.ctx = ctx;
  return o;
}

// Device temporary freed at scope exit (step entry points only).
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

// Device memory of an object, charged to its context's budget: refused
// (cudaErrorMemoryAllocation, no CUDA call) when the context's objects would
// exceed the limit.
cudaError_t obj_malloc(ckks_ctx* ctx, ckks_obj* o, void** p, size_t bytes) {
  ckks::MemBudget& m = *ctx->mem;
  const size_t lim = m.limit.load();
  const size_t before = m.used.fetch_add(bytes);
  if (lim && before + bytes > lim) {
    m.used.fetch_sub(bytes);
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    m.used.fetch_sub(bytes);
    return e;
  }
  o->bytes += bytes;
  o->mem = ctx->mem;
  return cudaSuccess;
}

void obj_release(ckks_obj* o) {
  if (o->mem) o->mem->used.fetch_sub(o->bytes);
  o->bytes = 0;
  o->mem.reset();
}

uint32_t galois_rot(int r, int log_n) {
  const uint64_t two_n = 2ull << log_n;
  const int64_t slots = 1ll << (log_n - 1);
  int64_t e = ((int64_t)r % slots + slots) % slots;
  uint64_t k = 1, b = 5;
  for (; e; e >>= 1) {
    if (e & 1) k = k * b % two_n;
    b = b * b % two_n;
  }
  return (uint32_t)k;
}

}  // namespace

extern "C" {

int ckks_gen_primes(int log_n, int n_q, int n_p, uint32_t* q_out, uint32_t* p_out) {
  if (log_n < 2 || log_n > 20 || n_q < 1 || n_p < 0 || !q_out || (n_p && !p_out)) return CKKS_EINVAL;
  return host_gen_primes(log_n, n_q, n_p, q_out, p_out);
}

int ckks_gen_prime_system_2530(int log_n, int n_p, uint32_t* q_out, uint32_t* p_out, int* level_first,
                               int* level_count) {
  if (!q_out || !p_out || !level_first || !level_count) return CKKS_EINVAL;
  return host_gen_prime_system_2530(log_n, n_p, q_out, p_out, level_first, level_count);
}

int ckks_ctx_create(const ckks_params* prm, void* stream, ckks_ctx** out) {
  if (!prm || !out) return CKKS_EINVAL;
  *out = nullptr;
  ckks_ctx* ctx = new (std::nothrow) ckks_ctx();
  if (!ctx) return CKKS_ENOMEM;
  ctx->d_tables = nullptr;
  ctx->d_scratch = nullptr;
  ctx->stream = (cudaStream_t)stream;
  auto bad = [&](int code) {
    // keep the message reachable for the caller: print it, then free
    fprintf(stderr, "ckks_ctx_create: %s\n", ctx->err.c_str());
    delete ctx;
    return code;
  };
  const int log_n = prm->log_n, L = prm->n_q, alpha = prm->n_p;
  if (log_n != 8 && log_n != 12 && log_n != 16)
    return bad(fail(ctx, CKKS_EINVAL, "log_n must be 8, 12 or 16 (got %d)", log_n));
  if (L < 1 || alpha < 1 || !prm->q || !prm->p)
    return bad(fail(ctx, CKKS_EINVAL, "need at least one ciphertext and one auxiliary prime"));
  if (prm->dnum != (L + alpha - 1) / alpha)
    return bad(fail(ctx, CKKS_EINVAL, "dnum (%d) must equal ceil(n_q / n_p) = %d", prm->dnum,
                    (L + alpha - 1) / alpha));
  if (prm->dnum > 8) return bad(fail(ctx, CKKS_EINVAL, "dnum %d above the supported maximum of 8", prm->dnum));
  if (prm->n_levels < 0 || (prm->n_levels > 0 && (!prm->level_first || !prm->level_count)))
    return bad(fail(ctx, CKKS_EINVAL, "level windows: n_levels %d without tables", prm->n_levels));
  for (int l = 0; l < prm->n_levels; ++l)
    if (prm->level_first[l] < 0 || prm->level_count[l] < 1 || prm->level_first[l] + prm->level_count[l] > L)
      return bad(fail(ctx, CKKS_EINVAL, "level %d window [%d, +%d) outside the %d primes", l, prm->level_first[l],
                      prm->level_count[l], L));
  const uint64_t two_n = 2ull << log_n;
  std::vector<uint32_t> all(prm->q, prm->q + L);
  all.insert(all.end(), prm->p, prm->p + alpha);
  for (size_t i = 0; i < all.size(); ++i) {
    const uint32_t v = all[i];
    if (v >= (1u << 31) || v < (1u << 20) || v % two_n != 1 || !host_is_prime(v))
      return bad(fail(ctx, CKKS_EINVAL, "prime %zu (%u) is not a prime = 1 mod 2N in [2^20, 2^31)", i, v));
    for (size_t j = 0; j < i; ++j)
      if (all[j] == v) return bad(fail(ctx, CKKS_EINVAL, "prime %u repeated", v));
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return bad(fail(ctx, CKKS_ECUDA, "no CUDA device"));
  if (prop.major != 10 || prop.minor != 3)
    return bad(fail(ctx, CKKS_ECUDA, "library is built for sm_103 (GB300); device is sm_%d%d", prop.major,
                    prop.minor));
  ctx->device = dev;
  ctx->scale = prm->scale;
  ctx->sigma = prm->sigma > 0 ? prm->sigma : 3.2;
  ctx->secret_hw = prm->secret_hw;
  ctx->seed = prm->seed;
  int rc = build_context(ctx, prm);
  if (rc != CKKS_OK) return bad(fail(ctx, rc, "building tables failed (%d)", rc));
  rc = alloc_status(ctx);
  if (rc != CKKS_OK) {
    if (ctx->d_tables) cudaFree(ctx->d_tables);
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    return bad(fail(ctx, rc, "status word allocation failed"));
  }
  ctx->sc.prof = &ctx->prof;
  ctx->mem = std::make_shared<ckks::MemBudget>();
  ctx->tune = std::make_shared<ckks::Tuning>(L);
  ctx->sc.tune = ctx->tune.get();
  ctx->dp.pdl = 1;
  *out = ctx;
  return CKKS_OK;
}

int ckks_ctx_clone(ckks_ctx* parent, void* cuda_stream, ckks_ctx** out) {
  if (!parent || !out) return CKKS_EINVAL;
  *out = nullptr;
  ckks_ctx* c = new (std::nothrow) ckks_ctx();
  if (!c) return CKKS_ENOMEM;
  c->dp = parent->dp;
  c->N = parent->N;
  c->q = parent->q;
  c->p = parent->p;
  c->pc_host = parent->pc_host;
  c->scale = parent->scale;
  c->sigma = parent->sigma;
  c->secret_hw = parent->secret_hw;
  c->seed = parent->seed;
  c->stream = (cudaStream_t)cuda_stream;
  c->d_tables = parent->d_tables;
  c->table_bytes = 0;
  c->owns_tables = false;
  c->gadget_p = parent->gadget_p;
  c->device = parent->device;
  c->windowed = parent->windowed;
  c->lvl_first = parent->lvl_first;
  c->lvl_count = parent->lvl_count;
  c->rows_off = parent->rows_off;
  c->rows_cnt = parent->rows_cnt;
  c->rr = parent->rr;
  c->mm = parent->mm;
  c->d_scratch = nullptr;
  int rc = alloc_scratch(c);
  if (rc != CKKS_OK) {
    delete c;
    return fail(parent, rc, "clone: scratch allocation failed");
  }
  c->h_status = parent->h_status;  // shared with the parent (dp.status copied above)
  c->sc.prof = &c->prof;
  c->mem = parent->mem;
  c->tune = parent->tune;
  c->sc.tune = c->tune.get();
  *out = c;
  return CKKS_OK;
}

void ckks_ctx_destroy(ckks_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  if (ctx->d_tables && ctx->owns_tables) cudaFree(ctx->d_tables);
  if (ctx->d_scratch) cudaFree(ctx->d_scratch);
  if (ctx->d_unfused) cudaFree(ctx->d_unfused);
  if (ctx->owns_tables) free_status(ctx);
  for (cudaEvent_t e : ctx->prof.ev) cudaEventDestroy(e);
  delete ctx;
}

int ckks_set_launch_flags(ckks_ctx* ctx, int flags) {
  if (!ctx || (flags & ~(CKKS_LAUNCH_PDL | CKKS_TUNE_TENSOR | CKKS_LAUNCH_UNFUSED | CKKS_LAUNCH_CHECKED)))
    return CKKS_EINVAL;
  if ((flags & CKKS_LAUNCH_UNFUSED) && ctx->windowed)
    return fail(ctx, CKKS_EINVAL, "launch flags: the unfused form supports single rescaling only");
  ctx->dp.pdl = (flags & CKKS_LAUNCH_PDL) ? 1 : 0;
  ctx->dp.tune_tensor = (flags & CKKS_TUNE_TENSOR) ? 1 : 0;
  ctx->dp.unfused = (flags & CKKS_LAUNCH_UNFUSED) ? 1 : 0;
  ctx->dp.checked = (flags & CKKS_LAUNCH_CHECKED) ? 1 : 0;
  return CKKS_OK;
}

int ckks_set_wait_limit(ckks_ctx* ctx, long long cycles) {
  if (!ctx) return CKKS_EINVAL;
  if (cycles < 1) return fail(ctx, CKKS_EINVAL, "wait limit %lld: must be at least one cycle", cycles);
  ctx->dp.wait_limit = cycles;
  return CKKS_OK;
}

int ckks_tune(ckks_ctx* ctx, int level, int reps) {
  if (!ctx || !ctx->tune) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "tune: level %d out of range", level);
  if (reps < 1 || reps > 1000) return fail(ctx, CKKS_EINVAL, "tune: reps %d out of [1, 1000]", reps);
  KsArgs lvl{};
  ctx->set_level(lvl, level);
  const int rc = ckks::tune_columns(ctx->dp, ctx->sc, *ctx->tune, lvl, reps, ctx->stream);
  if (rc != CKKS_OK) return fail(ctx, rc, "tune: %s", cudaGetErrorString(cudaGetLastError()));
  return CKKS_OK;
}

int ckks_tune_get(ckks_ctx* ctx, int kernel, int level, int* tc, int* sl, int* z, int* tp, float* us) {
  if (!ctx || !ctx->tune || !tc || !sl || !z || !tp || !us) return CKKS_EINVAL;
  if (kernel < 0 || kernel >= ckks::CK_COUNT) return fail(ctx, CKKS_EINVAL, "tune: kernel %d unknown", kernel);
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "tune: level %d out of range", level);
  const ckks::ColShape s = ctx->tune->get(kernel, level + 1);
  *tc = s.tc;
  *sl = s.sl;
  *z = s.z;
  *tp = s.tp;
  *us = ctx->tune->time_us(kernel, level + 1);
  return CKKS_OK;
}

int ckks_tune_set(ckks_ctx* ctx, int kernel, int level, int tc, int sl, int z, int tp) {
  if (!ctx || !ctx->tune) return CKKS_EINVAL;
  if (kernel < 0 || kernel >= ckks::CK_COUNT) return fail(ctx, CKKS_EINVAL, "tune: kernel %d unknown", kernel);
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "tune: level %d out of range", level);
  ckks::ColShape s;
  if (tc != 0 && kernel == ckks::CK_ROWS) {
    if (ctx->dp.log_n != 16 || tc < 2 || tc > 6)
      return fail(ctx, CKKS_EINVAL, "tune: row passes %d not supported at N = 2^%d", tc, ctx->dp.log_n);
    s = ckks::ColShape{tc, 1, 1, 1};
  } else if (tc != 0) {
    if (!ckks::col_shape_supported(ctx->dp.log_n, tc, sl, z, tp))
      return fail(ctx, CKKS_EINVAL, "tune: shape (%d, %d, %d, %d) not supported at N = 2^%d", tc, sl, z, tp,
                  ctx->dp.log_n);
    s.tc = tc;
    s.sl = sl;
    s.z = z;
    s.tp = tp;
  }
  ctx->tune->set(kernel, level + 1, s, 0.f);
  return CKKS_OK;
}

int ckks_level_limbs(ckks_ctx* ctx, int level) {
  if (!ctx) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  return ctx->lvl_n(level);
}

int ckks_profile(ckks_ctx* ctx, int enable) {
  if (!ctx) return CKKS_EINVAL;
  if (enable) ctx->prof.used = 0;
  ctx->prof.on = enable != 0;
  return CKKS_OK;
}

int ckks_profile_read(ckks_ctx* ctx, double* total_ms, uint64_t* launches) {
  if (!ctx || !total_ms || !launches) return CKKS_EINVAL;
  int rc = sync_check(ctx, "profile");
  if (rc) return rc;
  for (int i = 0; i < P_COUNT; ++i) {
    total_ms[i] = 0;
    launches[i] = 0;
  }
  const Prof& p = ctx->prof;
  for (size_t i = 1; i < p.used; ++i) {
    const int id = p.ids[i];
    if (id < 0 || id >= P_COUNT) continue;
    float ms = 0;
    rc = cuda_check(ctx, cudaEventElapsedTime(&ms, p.ev[i - 1], p.ev[i]), "profile");
    if (rc) return rc;
    total_ms[id] += ms;
    launches[id] += 1;
  }
  return CKKS_OK;
}

const char* ckks_profile_name(int id) {
  static const char* names[P_COUNT] = {
      "ks_prep",      "ks_in_rows",       "modup_cols",   "modup_rows",    "keymult",
      "moddown_in_rows", "moddown_cols",  "moddown_rows", "ks_epilogue",   "rescale_in_rows",
      "rescale_cols", "rescale_rows",     "rescale_epilogue"};
  return id >= 0 && id < P_COUNT ? names[id] : nullptr;
}

uint64_t ckks_launch_count(void) { return launch_count(); }

const char* ckks_last_error(ckks_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ckks_sync(ckks_ctx* ctx) {
  if (!ctx) return CKKS_EINVAL;
  return sync_check(ctx, "stream synchronize");
}

size_t ckks_ctx_device_bytes(ckks_ctx* ctx) { return ctx ? ctx->table_bytes + ctx->scratch_bytes : 0; }

}  // extern "C"

// Admission pool of a server: a byte budget that requests acquire while
// they hold device memory (host-side accounting, thread-safe).
extern "C" {

int ckks_pool_create(size_t budget_bytes, ckks_pool** out) {
  if (!out) return CKKS_EINVAL;
  ckks_pool* p = new (std::nothrow) ckks_pool();
  if (!p) return CKKS_ENOMEM;
  p->budget = budget_bytes;
  *out = p;
  return CKKS_OK;
}

int ckks_pool_acquire(ckks_pool* pool, size_t bytes) {
  if (!pool) return CKKS_EINVAL;
  size_t cur = pool->used.load();
  for (;;) {
    if (bytes > pool->budget || cur > pool->budget - bytes) return CKKS_EBUSY;
    if (pool->used.compare_exchange_weak(cur, cur + bytes)) return CKKS_OK;
  }
}

int ckks_pool_release(ckks_pool* pool, size_t bytes) {
  if (!pool) return CKKS_EINVAL;
  size_t cur = pool->used.load();
  for (;;) {
    if (bytes > cur) return CKKS_EINVAL;
    if (pool->used.compare_exchange_weak(cur, cur - bytes)) return CKKS_OK;
  }
}

size_t ckks_pool_in_use(const ckks_pool* pool) { return pool ? pool->used.load() : 0; }

void ckks_pool_destroy(ckks_pool* pool) { delete pool; }

int ckks_set_memory_limit(ckks_ctx* ctx, size_t bytes) {
  if (!ctx || !ctx->mem) return CKKS_EINVAL;
  ctx->mem->limit.store(bytes);
  return CKKS_OK;
}

size_t ckks_memory_in_use(ckks_ctx* ctx) { return ctx && ctx->mem ? ctx->mem->used.load() : 0; }

size_t ckks_request_bytes(ckks_ctx* ctx, int op, int level) {
  if (!ctx || level < 0 || level >= ctx->n_levels()) return 0;
  const size_t ct = 2 * (size_t)ctx->cap_limbs(level) * limb_words(ctx) * sizeof(uint32_t);
  size_t inputs;
  switch (op) {
    case CKKS_OP_HMULT:
    case CKKS_OP_HADD:
      inputs = 2 * ct;
      break;
    case CKKS_OP_HROT:
    case CKKS_OP_HCONJ:
    case CKKS_OP_RESCALE:
      inputs = ct;
      break;
    case CKKS_OP_PMULT:
    case CKKS_OP_PADD:
      inputs = ct + ct / 2;
      break;
    default:
      return 0;
  }
  const bool ks = op == CKKS_OP_HMULT || op == CKKS_OP_HROT || op == CKKS_OP_HCONJ || op == CKKS_OP_RESCALE;
  return inputs + ct + (ks ? ctx->scratch_bytes : 0);
}

void ckks_free(void* handle) {
  if (!handle) return;
  ckks_obj* o = reinterpret_cast<ckks_obj*>(handle);
  switch (o->kind) {
    case K_CT: {
      ckks_ct* c = reinterpret_cast<ckks_ct*>(handle);
      if (c->d && !c->borrowed) cudaFree(c->d);
      obj_release(&c->h);
      delete c;
    } break;
    case K_PT: {
      ckks_pt* p = reinterpret_cast<ckks_pt*>(handle);
      if (p->d) cudaFree(p->d);
      obj_release(&p->h);
      delete p;
    } break;
    case K_SK: {
      ckks_sk* s = reinterpret_cast<ckks_sk*>(handle);
      if (s->d_s) cudaFree(s->d_s);
      obj_release(&s->h);
      delete s;
    } break;
    case K_EVK: {
      ckks_evk* e = reinterpret_cast<ckks_evk*>(handle);
      if (e->d) cudaFree(e->d);
      obj_release(&e->h);
      delete e;
    } break;
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------

int ckks_ct_create(ckks_ctx* ctx, int cap_level, ckks_ct** out) {
  if (!ctx || !out) return CKKS_EINVAL;
  if (cap_level < 0 || cap_level >= ctx->n_levels())
    return fail(ctx, CKKS_ELEVEL, "capacity level %d out of range", cap_level);
  ckks_ct* c = new_obj<ckks_ct>(ctx, K_CT);
  if (!c) return CKKS_ENOMEM;
  c->level = cap_level;
  c->cap_level = cap_level;
  c->scale = ctx->scale;
  c->borrowed = false;
  const size_t cbytes = 2 * (size_t)ctx->cap_limbs(cap_level) * limb_words(ctx) * sizeof(uint32_t);
  if (obj_malloc(ctx, &c->h, (void**)&c->d, cbytes) != cudaSuccess) {
    delete c;
    return fail(ctx, CKKS_ENOMEM, "ciphertext allocation failed (%zu bytes; objects of the context hold %zu of "
                "a limit of %zu, 0 = none)", cbytes, ctx->mem->used.load(), ctx->mem->limit.load());
  }
  *out = c;
  return CKKS_OK;
}

static int ct_upload(ckks_ctx* ctx, ckks_ct* c, const uint32_t* host, int level, double scale, bool sync) {
  if (!ctx || !c || !host) return CKKS_EINVAL;
  if (level < 0 || level > c->cap_level) return fail(ctx, CKKS_ELEVEL, "level %d exceeds capacity %d", level, c->cap_level);
  const int n = ctx->lvl_n(level);
  const size_t lw = limb_words(ctx);
  uint32_t* stage = ctx->sc.A;  // 2 L limbs of staging
  for (int u = 0; u < 2; ++u) {
    int rc = cuda_check(ctx,
                        cudaMemcpyAsync(stage + (size_t)u * n * lw, host + (size_t)u * n * lw,
                                        (size_t)n * lw * 4, cudaMemcpyHostToDevice, ctx->stream),
                        "upload");
    if (rc) return rc;
    launch_permute(ctx->dp, stage + (size_t)u * n * lw, c->d + u * c->poly_stride(), n, true, ctx->stream);
  }
  c->level = level;
  c->scale = scale;
  check_ct(ctx, c);
  int rc = launched(ctx, "permute");
  if (rc || !sync) return rc;
  return sync_check(ctx, "upload");
}

int ckks_ct_upload(ckks_ctx* ctx, ckks_ct* c, const uint32_t* host, int level, double scale) {
  return ct_upload(ctx, c, host, level, scale, true);
}

int ckks_ct_upload_async(ckks_ctx* ctx, ckks_ct* c, const uint32_t* host, int level, double scale) {
  return ct_upload(ctx, c, host, level, scale, false);
}

int ckks_ct_import(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_ct** out) {
  if (!ctx || !out) return CKKS_EINVAL;
  int rc = ckks_ct_create(ctx, level, out);
  if (rc) return rc;
  rc = ckks_ct_upload(ctx, *out, host, level, scale);
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

static int ct_export(ckks_ctx* ctx, const ckks_ct* c, uint32_t* host, size_t words, int* level, double* scale,
                     bool sync) {
  if (!ctx || !c || !host) return CKKS_EINVAL;
  const int n = ctx->lvl_n(c->level);
  const size_t lw = limb_words(ctx);
  if (words < 2 * (size_t)n * lw) return fail(ctx, CKKS_EINVAL, "export buffer too small");
  uint32_t* stage = ctx->sc.A;
  for (int u = 0; u < 2; ++u)
    launch_permute(ctx->dp, c->d + u * c->poly_stride(), stage + (size_t)u * n * lw, n, false, ctx->stream);
  int rc = launched(ctx, "permute");
  if (rc) return rc;
  rc = cuda_check(ctx, cudaMemcpyAsync(host, stage, 2 * (size_t)n * lw * 4, cudaMemcpyDeviceToHost, ctx->stream),
                  "export");
  if (rc) return rc;
  if (sync) rc = sync_check(ctx, "export");
  if (level) *level = c->level;
  if (scale) *scale = c->scale;
  return rc;
}

int ckks_ct_export(ckks_ctx* ctx, const ckks_ct* c, uint32_t* host, size_t words, int* level, double* scale) {
  return ct_export(ctx, c, host, words, level, scale, true);
}

int ckks_ct_export_async(ckks_ctx* ctx, const ckks_ct* c, uint32_t* host, size_t words) {
  return ct_export(ctx, c, host, words, nullptr, nullptr, false);
}

int ckks_ct_wrap_device(ckks_ctx* ctx, uint32_t* dev_ptr, int level, double scale, ckks_ct** out) {
  if (!ctx || !dev_ptr || !out) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  ckks_ct* c = new_obj<ckks_ct>(ctx, K_CT);
  if (!c) return CKKS_ENOMEM;
  c->d = dev_ptr;
  c->level = c->cap_level = level;  // the buffer holds [2][limbs of level][N]
  c->scale = scale;
  c->borrowed = true;
  *out = c;
  return CKKS_OK;
}

int ckks_ct_info(const ckks_ct* c, int* level, double* scale, uint32_t** dev_ptr) {
  if (!c) return CKKS_EINVAL;
  if (level) *level = c->level;
  if (scale) *scale = c->scale;
  if (dev_ptr) *dev_ptr = c->d;
  return CKKS_OK;
}

static int pt_alloc(ckks_ctx* ctx, int level, double scale, ckks_pt** out, int ext = 0) {
  ckks_pt* p = new_obj<ckks_pt>(ctx, K_PT);
  if (!p) return CKKS_ENOMEM;
  p->level = level;
  p->scale = scale;
  p->ext = ext;
  if (obj_malloc(ctx, &p->h, (void**)&p->d, (size_t)(ctx->lvl_n(level) + ext) * limb_words(ctx) * 4) != cudaSuccess) {
    delete p;
    return fail(ctx, CKKS_ENOMEM, "plaintext allocation failed");
  }
  *out = p;
  return CKKS_OK;
}

int ckks_pt_import(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_pt** out) {
  if (!ctx || !host || !out) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  int rc = pt_alloc(ctx, level, scale, out);
  if (rc) return rc;
  const int n = ctx->lvl_n(level);
  const size_t lw = limb_words(ctx);
  rc = cuda_check(ctx, cudaMemcpyAsync(ctx->sc.A, host, (size_t)n * lw * 4, cudaMemcpyHostToDevice, ctx->stream),
                  "upload");
  if (!rc) {
    launch_permute(ctx->dp, ctx->sc.A, (*out)->d, n, true, ctx->stream);
    check_pt(ctx, *out);
    rc = launched(ctx, "permute");
  }
  if (!rc) rc = sync_check(ctx, "upload");
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

int ckks_pt_import_ext(ckks_ctx* ctx, const uint32_t* host, int level, double scale, ckks_pt** out) {
  if (!ctx || !host || !out) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  const int alpha = ctx->dp.alpha;
  int rc = pt_alloc(ctx, level, scale, out, alpha);
  if (rc) return rc;
  const int n = ctx->lvl_n(level) + alpha;
  const size_t lw = limb_words(ctx);
  rc = cuda_check(ctx, cudaMemcpyAsync(ctx->sc.A, host, (size_t)n * lw * 4, cudaMemcpyHostToDevice, ctx->stream),
                  "upload");
  if (!rc) {
    launch_permute(ctx->dp, ctx->sc.A, (*out)->d, n, true, ctx->stream);
    check_pt(ctx, *out);
    rc = launched(ctx, "permute");
  }
  if (!rc) rc = sync_check(ctx, "upload");
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

int ckks_pt_export(ckks_ctx* ctx, const ckks_pt* p, uint32_t* host, size_t words, int* level, double* scale) {
  if (!ctx || !p || !host) return CKKS_EINVAL;
  const int n = ctx->lvl_n(p->level);
  const size_t lw = limb_words(ctx);
  if (words < (size_t)n * lw) return fail(ctx, CKKS_EINVAL, "export buffer too small");
  launch_permute(ctx->dp, p->d, ctx->sc.A, n, false, ctx->stream);
  int rc = launched(ctx, "permute");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(host, ctx->sc.A, (size_t)n * lw * 4, cudaMemcpyDeviceToHost, ctx->stream), "export");
  if (!rc) rc = sync_check(ctx, "export");
  if (level) *level = p->level;
  if (scale) *scale = p->scale;
  return rc;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------

static int sk_from_coeffs(ckks_ctx* ctx, const int64_t* coeffs, ckks_sk** out) {
  const int np = ctx->dp.L + ctx->dp.alpha;
  const size_t lw = limb_words(ctx);
  ckks_sk* s = new_obj<ckks_sk>(ctx, K_SK);
  if (!s) return CKKS_ENOMEM;
  s->coeffs.assign(coeffs, coeffs + lw);
  DevBuf tmp;
  if (obj_malloc(ctx, &s->h, (void**)&s->d_s, (size_t)np * lw * 4) != cudaSuccess || tmp.alloc(lw * 8) != cudaSuccess) {
    ckks_free(s);
    return fail(ctx, CKKS_ENOMEM, "secret allocation failed");
  }
  int rc = cuda_check(ctx, cudaMemcpyAsync(tmp.p, coeffs, lw * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) {
    IdMap ids = id_ext(ctx->dp.L, ctx->dp.L, ctx->dp.alpha);
    launch_small_to_res(ctx->dp, tmp.as<int64_t>(), s->d_s, np, ids, ctx->stream);
    launch_ntt(ctx->dp, s->d_s, np, ids, false, ctx->stream);
    rc = launched(ctx, "secret NTT");
  }
  if (!rc) rc = sync_check(ctx, "secret");
  if (rc) {
    ckks_free(s);
    return rc;
  }
  *out = s;
  return CKKS_OK;
}

int ckks_sk_import(ckks_ctx* ctx, const int64_t* coeffs, ckks_sk** out) {
  if (!ctx || !coeffs || !out) return CKKS_EINVAL;
  for (int i = 0; i < ctx->N; ++i)
    if (coeffs[i] < -1 || coeffs[i] > 1) return fail(ctx, CKKS_EINVAL, "secret coefficient %d not ternary", i);
  return sk_from_coeffs(ctx, coeffs, out);
}

int ckks_keygen_secret(ckks_ctx* ctx, uint64_t seed, ckks_sk** out) {
  if (!ctx || !out) return CKKS_EINVAL;
  std::vector<int64_t> s(ctx->N);
  Sampler smp(seed ^ 0x5EC2E7ull);
  smp.ternary(s.data(), ctx->N, ctx->secret_hw);
  return sk_from_coeffs(ctx, s.data(), out);
}

// Key-switching key from s_from (NTT domain, all primes, device) to s.
static int keygen_ks(ckks_ctx* ctx, const ckks_sk* sk, const uint32_t* s_from, uint32_t galois, uint64_t seed,
                     ckks_evk** out) {
  const DevParams& dp = ctx->dp;
  const int L = dp.L, np = L + dp.alpha, dnum = dp.dnum;
  const size_t lw = limb_words(ctx), poly = (size_t)np * lw;
  ckks_evk* e = new_obj<ckks_evk>(ctx, K_EVK);
  if (!e) return CKKS_ENOMEM;
  e->galois = galois;
  if (obj_malloc(ctx, &e->h, (void**)&e->d, (size_t)dnum * 2 * poly * 4) != cudaSuccess) {
    delete e;
    return fail(ctx, CKKS_ENOMEM, "evk allocation failed");
  }
  Sampler smp(seed ^ 0xE7C0DEull);
  std::vector<uint32_t> a(poly);
  std::vector<int64_t> err(lw);
  std::vector<uint2> g(np);
  DevBuf d_err, d_e, d_g;
  int rc = CKKS_OK;
  if (d_err.alloc(lw * 8) || d_e.alloc(poly * 4) || d_g.alloc(np * sizeof(uint2))) rc = fail(ctx, CKKS_ENOMEM, "keygen scratch");
  IdMap ids = id_ext(L, L, dp.alpha);
  for (int j = 0; j < dnum && !rc; ++j) {
    for (int i = 0; i < np; ++i) {
      const uint32_t q = ctx->pc_host[i].q;
      for (size_t c = 0; c < lw; ++c) a[(size_t)i * lw + c] = smp.uniform(q);
    }
    for (size_t c = 0; c < lw; ++c) err[c] = smp.gaussian(ctx->sigma, 20);
    for (int i = 0; i < np; ++i) g[i] = (i < L && i / dp.alpha == j) ? ctx->gadget_p[i] : make_uint2(0, 0);
    uint32_t* b_j = e->d + (size_t)(2 * j) * poly;
    uint32_t* a_j = e->d + (size_t)(2 * j + 1) * poly;
    rc = cuda_check(ctx, cudaMemcpyAsync(a_j, a.data(), poly * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
    if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(d_err.p, err.data(), lw * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
    if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(d_g.p, g.data(), np * sizeof(uint2), cudaMemcpyHostToDevice, ctx->stream), "upload");
    if (rc) break;
    launch_small_to_res(dp, d_err.as<int64_t>(), d_e.as<uint32_t>(), np, ids, ctx->stream);
    launch_ntt(dp, d_e.as<uint32_t>(), np, ids, false, ctx->stream);
    // b_j = -a_j s + e_j + g_j s_from
    launch_lincomb(dp, a_j, sk->d_s, -1, d_e.as<uint32_t>(), nullptr, b_j, np, ids, ctx->stream);
    launch_add_scaled(dp, s_from, d_g.as<uint2>(), b_j, b_j, np, ids, ctx->stream);
    rc = launched(ctx, "keygen");
    if (!rc) rc = sync_check(ctx, "keygen");
  }
  if (!rc) {
    launch_to_mont(dp, e->d, 2 * dnum * np, ids, ctx->stream);
    rc = launched(ctx, "keygen");
    if (!rc) rc = sync_check(ctx, "keygen");
  }
  if (rc) {
    ckks_free(e);
    return rc;
  }
  *out = e;
  return CKKS_OK;
}

int ckks_keygen_relin(ckks_ctx* ctx, const ckks_sk* sk, uint64_t seed, ckks_evk** out) {
  if (!ctx || !sk || !out) return CKKS_EINVAL;
  const int np = ctx->dp.L + ctx->dp.alpha;
  DevBuf s2;
  if (s2.alloc((size_t)np * ctx->N * 4)) return fail(ctx, CKKS_ENOMEM, "keygen scratch");
  IdMap ids = id_ext(ctx->dp.L, ctx->dp.L, ctx->dp.alpha);
  launch_lincomb(ctx->dp, sk->d_s, sk->d_s, 1, nullptr, nullptr, s2.as<uint32_t>(), np, ids, ctx->stream);
  int rc = launched(ctx, "keygen");
  if (rc) return rc;
  return keygen_ks(ctx, sk, s2.as<uint32_t>(), 0, seed, out);
}

static int keygen_auto(ckks_ctx* ctx, const ckks_sk* sk, uint32_t galois, uint64_t seed, ckks_evk** out) {
  const int np = ctx->dp.L + ctx->dp.alpha;
  DevBuf sf;
  if (sf.alloc((size_t)np * ctx->N * 4)) return fail(ctx, CKKS_ENOMEM, "keygen scratch");
  launch_automorph(ctx->dp, sk->d_s, sf.as<uint32_t>(), np, galois, ctx->stream);
  int rc = launched(ctx, "keygen");
  if (rc) return rc;
  return keygen_ks(ctx, sk, sf.as<uint32_t>(), galois, seed, out);
}

int ckks_keygen_rot(ckks_ctx* ctx, const ckks_sk* sk, int r, uint64_t seed, ckks_evk** out) {
  if (!ctx || !sk || !out) return CKKS_EINVAL;
  return keygen_auto(ctx, sk, galois_rot(r, ctx->dp.log_n), seed, out);
}

int ckks_keygen_conj(ckks_ctx* ctx, const ckks_sk* sk, uint64_t seed, ckks_evk** out) {
  if (!ctx || !sk || !out) return CKKS_EINVAL;
  return keygen_auto(ctx, sk, (2u << ctx->dp.log_n) - 1, seed, out);
}

int ckks_evk_import(ckks_ctx* ctx, const uint32_t* host, uint32_t galois, ckks_evk** out) {
  if (!ctx || !host || !out) return CKKS_EINVAL;
  if (galois && (galois % 2 == 0 || galois >= (2u << ctx->dp.log_n)))
    return fail(ctx, CKKS_EINVAL, "galois element %u is not odd below 2N", galois);
  const DevParams& dp = ctx->dp;
  const int np = dp.L + dp.alpha;
  const size_t lw = limb_words(ctx), words = (size_t)dp.dnum * 2 * np * lw;
  ckks_evk* e = new_obj<ckks_evk>(ctx, K_EVK);
  if (!e) return CKKS_ENOMEM;
  e->galois = galois;
  DevBuf stage;
  if (obj_malloc(ctx, &e->h, (void**)&e->d, words * 4) != cudaSuccess || stage.alloc(words * 4)) {
    ckks_free(e);
    return fail(ctx, CKKS_ENOMEM, "evk allocation failed");
  }
  int rc = cuda_check(ctx, cudaMemcpyAsync(stage.p, host, words * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) {
    launch_permute(dp, stage.as<uint32_t>(), e->d, 2 * dp.dnum * np, true, ctx->stream);
    // checked mode: the imported key in [dnum][2][L + alpha] before its Montgomery form
    if (dp.checked) launch_check_range(dp, e->d, (size_t)np << dp.log_n, 2 * dp.dnum, dp.L, dp.alpha, 0, ctx->stream);
    launch_to_mont(dp, e->d, 2 * dp.dnum * np, id_ext(dp.L, dp.L, dp.alpha), ctx->stream);
    rc = launched(ctx, "evk import");
  }
  if (!rc) rc = sync_check(ctx, "evk import");
  if (rc) {
    ckks_free(e);
    return rc;
  }
  *out = e;
  return CKKS_OK;
}

// ---------------------------------------------------------------------------
// encoding and encryption
// ---------------------------------------------------------------------------

int ckks_encode(ckks_ctx* ctx, const double* re_im, int level, double scale, ckks_pt** out) {
  if (!ctx || !re_im || !out) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  std::vector<int64_t> m;
  host_encode(re_im, ctx->dp.log_n, scale, m);
  int rc = pt_alloc(ctx, level, scale, out);
  if (rc) return rc;
  DevBuf tmp;
  const int n = ctx->lvl_n(level), base = ctx->lvl_base(level);
  rc = tmp.alloc(m.size() * 8) ? fail(ctx, CKKS_ENOMEM, "encode scratch") : CKKS_OK;
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(tmp.p, m.data(), m.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) {
    launch_small_to_res(ctx->dp, tmp.as<int64_t>(), (*out)->d, n, id_ct(n, ctx->dp.L, base), ctx->stream);
    launch_ntt(ctx->dp, (*out)->d, n, id_ct(n, ctx->dp.L, base), false, ctx->stream);
    rc = launched(ctx, "encode");
  }
  if (!rc) rc = sync_check(ctx, "encode");
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

int ckks_encode_ext(ckks_ctx* ctx, const double* re_im, int level, double scale, ckks_pt** out) {
  if (!ctx || !re_im || !out) return CKKS_EINVAL;
  if (level < 0 || level >= ctx->n_levels()) return fail(ctx, CKKS_ELEVEL, "level %d out of range", level);
  std::vector<int64_t> m;
  host_encode(re_im, ctx->dp.log_n, scale, m);
  const int alpha = ctx->dp.alpha, n = ctx->lvl_n(level), base = ctx->lvl_base(level);
  int rc = pt_alloc(ctx, level, scale, out, alpha);
  if (rc) return rc;
  DevBuf tmp;
  rc = tmp.alloc(m.size() * 8) ? fail(ctx, CKKS_ENOMEM, "encode scratch") : CKKS_OK;
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(tmp.p, m.data(), m.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) {
    const IdMap ids = id_ext(n, ctx->dp.L, alpha, base);
    launch_small_to_res(ctx->dp, tmp.as<int64_t>(), (*out)->d, n + alpha, ids, ctx->stream);
    launch_ntt(ctx->dp, (*out)->d, n + alpha, ids, false, ctx->stream);
    rc = launched(ctx, "encode");
  }
  if (!rc) rc = sync_check(ctx, "encode");
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

int ckks_decode(ckks_ctx* ctx, const ckks_pt* pt, double* re_im_out) {
  if (!ctx || !pt || !re_im_out) return CKKS_EINVAL;
  const int n = ctx->lvl_n(pt->level), base = ctx->lvl_base(pt->level);
  const size_t lw = limb_words(ctx);
  DevBuf tmp;
  if (tmp.alloc((size_t)n * lw * 4)) return fail(ctx, CKKS_ENOMEM, "decode scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(tmp.p, pt->d, (size_t)n * lw * 4, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
  if (rc) return rc;
  launch_ntt(ctx->dp, tmp.as<uint32_t>(), n, id_ct(n, ctx->dp.L, base), true, ctx->stream);
  rc = launched(ctx, "decode");
  if (rc) return rc;
  std::vector<uint32_t> res((size_t)n * lw);
  rc = cuda_check(ctx, cudaMemcpyAsync(res.data(), tmp.p, res.size() * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  if (!rc) rc = sync_check(ctx, "decode");
  if (rc) return rc;
  host_decode(res.data(), n, ctx->q.data() + base, ctx->dp.log_n, pt->scale, re_im_out);
  return CKKS_OK;
}

int ckks_encrypt(ckks_ctx* ctx, const ckks_sk* sk, const ckks_pt* pt, uint64_t seed, ckks_ct** out) {
  if (!ctx || !sk || !pt || !out) return CKKS_EINVAL;
  const int n = ctx->lvl_n(pt->level), base = ctx->lvl_base(pt->level);
  const size_t lw = limb_words(ctx);
  int rc = ckks_ct_create(ctx, pt->level, out);
  if (rc) return rc;
  ckks_ct* c = *out;
  c->scale = pt->scale;
  Sampler smp(seed ^ 0xC1F3E7ull);
  std::vector<uint32_t> a((size_t)n * lw);
  for (int i = 0; i < n; ++i)
    for (size_t k = 0; k < lw; ++k) a[(size_t)i * lw + k] = smp.uniform(ctx->pc_host[base + i].q);
  std::vector<int64_t> e(lw);
  for (size_t k = 0; k < lw; ++k) e[k] = smp.gaussian(ctx->sigma, 20);
  DevBuf d_e, d_en;
  if (d_e.alloc(lw * 8) || d_en.alloc((size_t)n * lw * 4)) rc = fail(ctx, CKKS_ENOMEM, "encrypt scratch");
  uint32_t* b = c->d;
  uint32_t* ad = c->d + c->poly_stride();
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(ad, a.data(), a.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(d_e.p, e.data(), lw * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) {
    IdMap ids = id_ct(n, ctx->dp.L, base);
    launch_small_to_res(ctx->dp, d_e.as<int64_t>(), d_en.as<uint32_t>(), n, ids, ctx->stream);
    launch_ntt(ctx->dp, d_en.as<uint32_t>(), n, ids, false, ctx->stream);
    launch_lincomb(ctx->dp, ad, sk->d_s + ((size_t)base << ctx->dp.log_n), -1, pt->d, d_en.as<uint32_t>(), b, n, ids,
                   ctx->stream);
    rc = launched(ctx, "encrypt");
  }
  if (!rc) rc = sync_check(ctx, "encrypt");
  if (rc) {
    ckks_free(c);
    *out = nullptr;
  }
  return rc;
}

int ckks_decrypt(ckks_ctx* ctx, const ckks_sk* sk, const ckks_ct* c, ckks_pt** out) {
  if (!ctx || !sk || !c || !out) return CKKS_EINVAL;
  const int n = ctx->lvl_n(c->level), base = ctx->lvl_base(c->level);
  int rc = pt_alloc(ctx, c->level, c->scale, out);
  if (rc) return rc;
  launch_lincomb(ctx->dp, c->d + c->poly_stride(), sk->d_s + ((size_t)base << ctx->dp.log_n), 1, c->d, nullptr,
                 (*out)->d, n, id_ct(n, ctx->dp.L, base), ctx->stream);
  rc = launched(ctx, "decrypt");
  if (rc) {
    ckks_free(*out);
    *out = nullptr;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// homomorphic operations
// ---------------------------------------------------------------------------

int ckks_hadd(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out) {
  if (!ctx || !a || !b || !out) return CKKS_EINVAL;
  if (a->level != b->level) return fail(ctx, CKKS_ELEVEL, "hadd: levels %d and %d differ", a->level, b->level);
  if (!scales_match(a->scale, b->scale)) return fail(ctx, CKKS_ESCALE, "hadd: scales differ");
  if (out->cap_level < a->level) return fail(ctx, CKKS_ELEVEL, "hadd: output capacity too small");
  check_ct(ctx, a);
  check_ct(ctx, b);
  launch_hadd(ctx->dp, a->d, b->d, out->d, ctx->lvl_n(a->level), ctx->lvl_base(a->level), a->poly_stride(),
              b->poly_stride(), out->poly_stride(),
              ctx->stream);
  out->level = a->level;
  out->scale = a->scale;
  check_ct(ctx, out);
  return launched(ctx, "hadd");
}

int ckks_pmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_pt* pt, ckks_ct* out) {
  if (!ctx || !a || !pt || !out) return CKKS_EINVAL;
  if (pt->level < a->level) return fail(ctx, CKKS_ELEVEL, "pmult: plaintext level %d below %d", pt->level, a->level);
  if (out->cap_level < a->level) return fail(ctx, CKKS_ELEVEL, "pmult: output capacity too small");
  if (ctx->windowed && pt->level != a->level)
    return fail(ctx, CKKS_ELEVEL, "pmult: plaintext level %d differs from %d (level windows)", pt->level, a->level);
  check_ct(ctx, a);
  check_pt(ctx, pt);
  launch_pmult(ctx->dp, a->d, pt->d, out->d, ctx->lvl_n(a->level), ctx->lvl_base(a->level), a->poly_stride(),
               out->poly_stride(), ctx->stream);
  out->level = a->level;
  out->scale = a->scale * pt->scale;
  check_ct(ctx, out);
  return launched(ctx, "pmult");
}

int ckks_padd(ckks_ctx* ctx, const ckks_ct* a, const ckks_pt* pt, ckks_ct* out) {
  if (!ctx || !a || !pt || !out) return CKKS_EINVAL;
  if (pt->level < a->level) return fail(ctx, CKKS_ELEVEL, "padd: plaintext level %d below %d", pt->level, a->level);
  if (!scales_match(a->scale, pt->scale)) return fail(ctx, CKKS_ESCALE, "padd: scales differ");
  if (out->cap_level < a->level) return fail(ctx, CKKS_ELEVEL, "padd: output capacity too small");
  if (ctx->windowed && pt->level != a->level)
    return fail(ctx, CKKS_ELEVEL, "padd: plaintext level %d differs from %d (level windows)", pt->level, a->level);
  check_ct(ctx, a);
  check_pt(ctx, pt);
  launch_padd(ctx->dp, a->d, pt->d, out->d, ctx->lvl_n(a->level), ctx->lvl_base(a->level), a->poly_stride(),
              out->poly_stride(), ctx->stream);
  out->level = a->level;
  out->scale = a->scale;
  check_ct(ctx, out);
  return launched(ctx, "padd");
}

// Scale factor of the rescaling from `level`: 1 / q_level (single), or
// T_add / T_drop between the level windows (rational).
static double rescale_factor(const ckks_ctx* ctx, int level) {
  if (!ctx->windowed) return 1.0 / (double)ctx->q[level];
  const int s0 = ctx->lvl_first[level], n0 = ctx->lvl_count[level];
  const int s1 = ctx->lvl_first[level - 1], n1 = ctx->lvl_count[level - 1];
  double f = 1.0;
  for (int g = s0; g < s0 + n0; ++g)
    if (g < s1 || g >= s1 + n1) f /= (double)ctx->q[g];
  for (int g = s1; g < s1 + n1; ++g)
    if (g < s0 || g >= s0 + n0) f *= (double)ctx->q[g];
  return f;
}

// Rescale of [2][limbs] at `in` (poly stride sin) from `level` into out.
static void rescale_into(ckks_ctx* ctx, int level, const uint32_t* in, size_t sin, uint32_t* out, size_t sout) {
  if (ctx->windowed) launch_rational_rescale(ctx->dp, ctx->sc, ctx->rr[level], in, sin, out, sout, ctx->stream);
  else launch_rescale(ctx->dp, ctx->sc, in, sin, level + 1, out, sout, ctx->stream);
}

int ckks_rescale(ckks_ctx* ctx, const ckks_ct* in, ckks_ct* out) {
  if (!ctx || !in || !out) return CKKS_EINVAL;
  if (in->level < 1) return fail(ctx, CKKS_ELEVEL, "rescale at level 0");
  if (out == in || out->d == in->d) return fail(ctx, CKKS_EINVAL, "rescale: output aliases input");
  if (out->cap_level < in->level - 1) return fail(ctx, CKKS_ELEVEL, "rescale: output capacity too small");
  check_ct(ctx, in);
  rescale_into(ctx, in->level, in->d, in->poly_stride(), out->d, out->poly_stride());
  out->level = in->level - 1;
  out->scale = in->scale * rescale_factor(ctx, in->level);
  check_ct(ctx, out);
  return launched(ctx, "rescale");
}

}  // extern "C"

// Validation and key-switch arguments of HMult (Sec. 2.1: tensor, then
// relinearization by key switching, then optionally rescaling): fills k,
// sets out's level and scale; staged = a windowed context's rational
// rescale still has to follow the key switch (from the scratch U).
int prepare_hmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, const ckks_evk* evk, int flags, ckks_ct* out,
                  KsArgs& k, bool& staged) {
  if (!ctx || !a || !b || !evk || !out) return CKKS_EINVAL;
  if (flags & ~(CKKS_RESCALE | CKKS_RESCALE_MERGED)) return fail(ctx, CKKS_EINVAL, "hmult: unknown flags %d", flags);
  if (evk->galois != 0) return fail(ctx, CKKS_ENOKEY, "hmult needs a relinearization key");
  if (a->level != b->level) return fail(ctx, CKKS_ELEVEL, "hmult: levels %d and %d differ", a->level, b->level);
  if (out == a || out == b) return fail(ctx, CKKS_EINVAL, "hmult: output aliases an input");
  const bool merged = flags & CKKS_RESCALE_MERGED;
  const bool rs = (flags & CKKS_RESCALE) || merged;
  if (rs && a->level < 1) return fail(ctx, CKKS_ELEVEL, "hmult: cannot rescale at level 0");
  if (out->cap_level < a->level - (rs ? 1 : 0)) return fail(ctx, CKKS_ELEVEL, "hmult: output capacity too small");
  const size_t lw = limb_words(ctx);
  k = KsArgs{};
  ctx->set_level(k, a->level);
  k.mode = KS_TENSOR;
  k.x0 = a->d;
  k.x1 = b->d;
  k.poly_stride0 = a->poly_stride();
  k.poly_stride1 = b->poly_stride();
  k.evk = evk->d;
  k.extra = 1;
  // single rescaling is fused into ModDown; a rational one follows the key
  // switch (its ciphertext-size intermediate lives in the scratch U); the
  // merged form divides by P T_drop at once in either system
  const bool fused = rs && (!ctx->windowed || merged);
  k.rescale = fused ? 1 : 0;
  k.mm = merged ? &ctx->mm[a->level] : nullptr;
  staged = rs && ctx->windowed && !merged;
  k.out = staged ? ctx->sc.U : out->d;
  k.out_stride = staged ? (size_t)ctx->lvl_n(a->level) * lw : out->poly_stride();
  const int level = a->level;
  out->scale = a->scale * b->scale * (rs ? rescale_factor(ctx, level) : 1.0);
  out->level = rs ? level - 1 : level;
  return CKKS_OK;
}

// Validation and key-switch arguments of an automorphism (HRot, HConj;
// Eq. 4 then key switching), with out's level and scale set.
int prepare_hauto(ckks_ctx* ctx, const ckks_ct* c, uint32_t galois, const ckks_evk* evk, ckks_ct* out, KsArgs& k) {
  if (evk->galois != galois) return fail(ctx, CKKS_ENOKEY, "key is for galois element %u, need %u", evk->galois, galois);
  if (out == c) return fail(ctx, CKKS_EINVAL, "output aliases the input");
  if (out->cap_level < c->level) return fail(ctx, CKKS_ELEVEL, "output capacity too small");
  k = KsArgs{};
  ctx->set_level(k, c->level);
  k.mode = KS_AUTO;
  k.x0 = c->d;
  k.poly_stride0 = c->poly_stride();
  k.galois = galois;
  k.evk = evk->d;
  k.out = out->d;
  k.out_stride = out->poly_stride();
  k.extra = 2;
  out->level = c->level;
  out->scale = c->scale;
  return CKKS_OK;
}

uint32_t galois_of_rotation(int r, int log_n) { return galois_rot(r, log_n); }

extern "C" {

// Key switch of an operation in the unfused form (its scratch is allocated
// on the first use).
static int keyswitch_unfused(ckks_ctx* ctx, const KsArgs& k, const char* what) {
  if (k.mm) return fail(ctx, CKKS_EINVAL, "%s: the unfused form has no merged ModDown + rescale", what);
  if (ctx->dp.alpha > 64) return fail(ctx, CKKS_EINVAL, "%s: the unfused form converts at most 64 sources", what);
  if (!ctx->d_unfused && cudaMalloc(&ctx->d_unfused, unfused_scratch_words(ctx->dp) * sizeof(uint32_t)) != cudaSuccess)
    return fail(ctx, CKKS_ENOMEM, "%s: unfused scratch allocation failed", what);
  launch_keyswitch_unfused(ctx->dp, k, ctx->d_unfused, ctx->stream);
  return launched(ctx, what);
}

int ckks_hmult(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, const ckks_evk* evk, int flags, ckks_ct* out) {
  KsArgs k;
  bool staged = false;
  const int level = a ? a->level : 0;
  if (ctx && a && b && out) {
    check_ct(ctx, a);
    check_ct(ctx, b);
  }
  const int rc = prepare_hmult(ctx, a, b, evk, flags, out, k, staged);
  if (rc != CKKS_OK) return rc;
  if (ctx->dp.unfused) {
    const int ru = keyswitch_unfused(ctx, k, "hmult");
    check_ct(ctx, out);
    return ru;
  }
  launch_keyswitch(ctx->dp, ctx->sc, k, KM_KEYSWITCH, nullptr, ctx->stream);
  if (staged) rescale_into(ctx, level, ctx->sc.U, k.out_stride, out->d, out->poly_stride());
  check_ct(ctx, out);
  return launched(ctx, "hmult");
}

static int hauto(ckks_ctx* ctx, const ckks_ct* c, uint32_t galois, const ckks_evk* evk, ckks_ct* out) {
  KsArgs k;
  if (out) check_ct(ctx, c);
  const int rc = prepare_hauto(ctx, c, galois, evk, out, k);
  if (rc != CKKS_OK) return rc;
  if (ctx->dp.unfused) {
    const int ru = keyswitch_unfused(ctx, k, "hrot");
    check_ct(ctx, out);
    return ru;
  }
  launch_keyswitch(ctx->dp, ctx->sc, k, KM_KEYSWITCH, nullptr, ctx->stream);
  check_ct(ctx, out);
  return launched(ctx, "hrot");
}

int ckks_hrot(ckks_ctx* ctx, const ckks_ct* c, int r, const ckks_evk* evk, ckks_ct* out) {
  if (!ctx || !c || !evk || !out) return CKKS_EINVAL;
  return hauto(ctx, c, galois_rot(r, ctx->dp.log_n), evk, out);
}

int ckks_hconj(ckks_ctx* ctx, const ckks_ct* c, const ckks_evk* evk, ckks_ct* out) {
  if (!ctx || !c || !evk || !out) return CKKS_EINVAL;
  return hauto(ctx, c, (2u << ctx->dp.log_n) - 1, evk, out);
}

int ckks_hrot_hoisted(ckks_ctx* ctx, const ckks_ct* c, int count, const int* r, const ckks_evk* const* evks,
                      ckks_ct* const* outs) {
  if (!ctx || !c || count < 0 || (count > 0 && (!r || !evks || !outs))) return CKKS_EINVAL;
  if (count == 0) return CKKS_OK;
  std::vector<KsArgs> ks((size_t)count);
  for (int i = 0; i < count; ++i) {
    const ckks_evk* evk = evks[i];
    ckks_ct* out = outs[i];
    if (!evk || !out) return fail(ctx, CKKS_EINVAL, "hoisted rotation %d: missing key or output", i);
    const uint32_t galois = galois_rot(r[i], ctx->dp.log_n);
    if (evk->galois != galois)
      return fail(ctx, CKKS_ENOKEY, "hoisted rotation %d: key is for galois element %u, need %u", i, evk->galois,
                  galois);
    if (out == c || out->d == c->d) return fail(ctx, CKKS_EINVAL, "hoisted rotation %d: output aliases the input", i);
    if (out->cap_level < c->level) return fail(ctx, CKKS_ELEVEL, "hoisted rotation %d: output capacity too small", i);
    for (int j = 0; j < i; ++j)
      if (outs[j]->d == out->d) return fail(ctx, CKKS_EINVAL, "hoisted rotations %d and %d share an output", j, i);
    KsArgs& k = ks[(size_t)i];
    ctx->set_level(k, c->level);
    k.mode = KS_AUTO;
    k.x0 = c->d;
    k.poly_stride0 = c->poly_stride();
    k.galois = galois;
    k.evk = evk->d;
    k.out = out->d;
    k.out_stride = out->poly_stride();
    k.extra = 2;
    k.hoisted = 1;
  }
  check_ct(ctx, c);
  launch_hoisted_rotations(ctx->dp, ctx->sc, ks.data(), count, ctx->stream);
  for (int i = 0; i < count; ++i) {
    outs[i]->level = c->level;
    outs[i]->scale = c->scale;
    check_ct(ctx, outs[i]);
  }
  return launched(ctx, "hrot_hoisted");
}

int ckks_linear_transform(ckks_ctx* ctx, const ckks_ct* c, int count, const int* r, const ckks_evk* const* evks,
                          const ckks_pt* const* pts, ckks_ct* out) {
  if (!ctx || !c || !out || count < 1 || !r || !pts || !evks) return CKKS_EINVAL;
  if (count > ckks::kLtMax) return fail(ctx, CKKS_EINVAL, "linear transform: at most %d terms", ckks::kLtMax);
  if (out == c || out->d == c->d) return fail(ctx, CKKS_EINVAL, "linear transform: output aliases the input");
  if (out->cap_level < c->level) return fail(ctx, CKKS_ELEVEL, "linear transform: output capacity too small");
  ckks::LtArgs lt{};
  lt.count = count;
  const double pscale = pts[0] ? pts[0]->scale : 0.0;
  for (int i = 0; i < count; ++i) {
    const ckks_pt* pt = pts[i];
    if (!pt) return fail(ctx, CKKS_EINVAL, "linear transform: term %d has no plaintext", i);
    if (pt->ext != ctx->dp.alpha)
      return fail(ctx, CKKS_EINVAL, "linear transform: term %d needs an extended plaintext (ckks_encode_ext)", i);
    if (pt->level < c->level || (ctx->windowed && pt->level != c->level))
      return fail(ctx, CKKS_ELEVEL, "linear transform: term %d plaintext level does not match", i);
    if (std::fabs(pt->scale - pscale) > 1e-9 * pscale)
      return fail(ctx, CKKS_ESCALE, "linear transform: term %d plaintext scale differs", i);
    lt.pt[i] = pt->d;
    lt.pt_p[i] = ctx->lvl_n(pt->level);
    const uint32_t galois = galois_rot(r[i], ctx->dp.log_n);
    if (galois == 1) {
      lt.galois[i] = 1;
      lt.evk[i] = nullptr;
      continue;
    }
    const ckks_evk* evk = evks[i];
    if (!evk) return fail(ctx, CKKS_ENOKEY, "linear transform: term %d has no key", i);
    if (evk->galois != galois)
      return fail(ctx, CKKS_ENOKEY, "linear transform: term %d key is for galois element %u, need %u", i,
                  evk->galois, galois);
    lt.galois[i] = galois;
    lt.evk[i] = evk->d;
    ++lt.rotated;
  }
  KsArgs k{};
  ctx->set_level(k, c->level);
  k.x0 = c->d;
  k.poly_stride0 = c->poly_stride();
  k.out = out->d;
  k.out_stride = out->poly_stride();
  check_ct(ctx, c);
  for (int i = 0; i < count; ++i) check_pt(ctx, pts[i]);
  launch_linear_transform(ctx->dp, ctx->sc, k, lt, ctx->stream);
  out->level = c->level;
  out->scale = c->scale * pscale;
  check_ct(ctx, out);
  return launched(ctx, "linear_transform");
}

// ---------------------------------------------------------------------------
// step-level entry points (host buffers, canonical layout, synchronous)
// ---------------------------------------------------------------------------

static int check_ids(ckks_ctx* ctx, const int* ids, int count) {
  for (int i = 0; i < count; ++i)
    if (ids[i] < 0 || ids[i] >= ctx->dp.L + ctx->dp.alpha) return fail(ctx, CKKS_EINVAL, "prime id %d out of range", ids[i]);
  return CKKS_OK;
}

static int finish(ckks_ctx* ctx, const char* what) {
  int rc = launched(ctx, what);
  if (rc) return rc;
  return sync_check(ctx, what);
}

int ckks_step_smr(ckks_ctx* ctx, const int64_t* x, int n, int prime_id, int32_t* y) {
  if (!ctx || !x || !y || n < 0) return CKKS_EINVAL;
  if (check_ids(ctx, &prime_id, 1)) return CKKS_EINVAL;
  DevBuf dx, dy;
  if (dx.alloc((size_t)n * 8) || dy.alloc((size_t)n * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(dx.p, x, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  launch_smr(ctx->dp, dx.as<int64_t>(), dy.as<int32_t>(), n, prime_id, ctx->stream);
  rc = cuda_check(ctx, cudaMemcpyAsync(y, dy.p, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "smr");
}

int ckks_step_ntt(ckks_ctx* ctx, uint32_t* data, int limbs, const int* prime_ids, int inverse) {
  if (!ctx || !data || !prime_ids || limbs < 0) return CKKS_EINVAL;
  if (check_ids(ctx, prime_ids, limbs)) return CKKS_EINVAL;
  const size_t lw = limb_words(ctx), words = (size_t)limbs * lw;
  DevBuf d, t, ids;
  if (d.alloc(words * 4) || t.alloc(words * 4) || ids.alloc((size_t)limbs * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(d.p, data, words * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(ids.p, prime_ids, (size_t)limbs * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  IdMap m = id_arr(ids.as<int>());
  if (!inverse) {
    launch_ntt(ctx->dp, d.as<uint32_t>(), limbs, m, false, ctx->stream);
    launch_permute(ctx->dp, d.as<uint32_t>(), t.as<uint32_t>(), limbs, false, ctx->stream);
  } else {
    launch_permute(ctx->dp, d.as<uint32_t>(), t.as<uint32_t>(), limbs, true, ctx->stream);
    launch_ntt(ctx->dp, t.as<uint32_t>(), limbs, m, true, ctx->stream);
  }
  rc = cuda_check(ctx, cudaMemcpyAsync(data, t.p, words * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "ntt");
}

int ckks_step_bconv(ckks_ctx* ctx, const uint32_t* in, int k, const int* src_ids, uint32_t* out, int m,
                    const int* dst_ids, int variant) {
  if (!ctx || !in || !out || !src_ids || !dst_ids || k < 1 || m < 1) return CKKS_EINVAL;
  if (k > 64) return fail(ctx, CKKS_EINVAL, "bconv: at most 64 source limbs");
  if (check_ids(ctx, src_ids, k) || check_ids(ctx, dst_ids, m)) return CKKS_EINVAL;
  if (variant != 0 && variant != 1) return fail(ctx, CKKS_EINVAL, "bconv: unknown variant %d", variant);
  // constants of Eq. 2 for this source basis
  std::vector<uint2> cin(k);
  std::vector<int32_t> mat((size_t)m * k);
  const int mp = (7 * m + 15) / 16 * 16, kp = (4 * (k + 1) + 31) / 32 * 32;
  std::vector<uint8_t> ab((size_t)mp * kp, 0);
  auto mulm = [](uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)((uint64_t)a * b % q); };
  auto powm = [&](uint32_t b, uint32_t e, uint32_t q) {
    uint32_t r = 1;
    for (; e; e >>= 1, b = mulm(b, b, q))
      if (e & 1) r = mulm(r, b, q);
    return r;
  };
  auto put = [&](int t, int kk, uint32_t v) {  // byte planes of one matrix entry
    for (int s = 0; s < 7; ++s)
      for (int a = 0; a < 4; ++a)
        if (s - a >= 0 && s - a <= 3) ab[(size_t)(7 * t + s) * kp + 4 * kk + a] = (uint8_t)(v >> (8 * (s - a)));
  };
  for (int i = 0; i < k; ++i) {
    const uint32_t qi = ctx->pc_host[src_ids[i]].q;
    uint32_t hat = 1;
    for (int i2 = 0; i2 < k; ++i2)
      if (i2 != i) hat = mulm(hat, ctx->pc_host[src_ids[i2]].q % qi, qi);
    const uint32_t inv = powm(hat, qi - 2, qi);
    cin[i] = make_uint2(inv, (uint32_t)(((uint64_t)inv << 32) / qi));
    for (int t = 0; t < m; ++t) {
      const PrimeConst& P = ctx->pc_host[dst_ids[t]];
      uint32_t h = 1;
      for (int i2 = 0; i2 < k; ++i2)
        if (i2 != i) h = mulm(h, ctx->pc_host[src_ids[i2]].q % P.q, P.q);
      const uint32_t v = mulm(h, P.mont, P.q);
      mat[(size_t)t * k + i] = v > P.q / 2 ? (int32_t)((int64_t)v - P.q) : (int32_t)v;
      const uint32_t r2 = mulm(P.mont, P.mont, P.q);
      put(t, i, mulm(h, r2, P.q));
    }
  }
  for (int t = 0; t < m; ++t) {  // count limb: [-Qs 2^64]_p
    const PrimeConst& P = ctx->pc_host[dst_ids[t]];
    uint32_t Q = 1;
    for (int i2 = 0; i2 < k; ++i2) Q = mulm(Q, ctx->pc_host[src_ids[i2]].q % P.q, P.q);
    put(t, k, mulm((P.q - Q) % P.q, mulm(P.mont, P.mont, P.q), P.q));
  }
  const size_t lw = limb_words(ctx);
  DevBuf din, dout, dsrc, ddst, dcin, dmat, dab;
  if (din.alloc((size_t)k * lw * 4) || dout.alloc((size_t)m * lw * 4) || dsrc.alloc(k * 4) || ddst.alloc(m * 4) ||
      dcin.alloc(k * sizeof(uint2)) || dmat.alloc(mat.size() * 4) || dab.alloc(ab.size()))
    return fail(ctx, CKKS_ENOMEM, "scratch");
  cudaStream_t st = ctx->stream;
  int rc = cuda_check(ctx, cudaMemcpyAsync(din.p, in, (size_t)k * lw * 4, cudaMemcpyHostToDevice, st), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(dsrc.p, src_ids, k * 4, cudaMemcpyHostToDevice, st), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(ddst.p, dst_ids, m * 4, cudaMemcpyHostToDevice, st), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(dcin.p, cin.data(), k * sizeof(uint2), cudaMemcpyHostToDevice, st), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(dmat.p, mat.data(), mat.size() * 4, cudaMemcpyHostToDevice, st), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(dab.p, ab.data(), ab.size(), cudaMemcpyHostToDevice, st), "upload");
  if (rc) return rc;
  launch_bconv(ctx->dp, din.as<uint32_t>(), k, dsrc.as<int>(), dcin.as<uint2>(), dmat.as<int32_t>(),
               dout.as<uint32_t>(), m, ddst.as<int>(), variant, dab.as<uint8_t>(), mp, kp, st);
  rc = cuda_check(ctx, cudaMemcpyAsync(out, dout.p, (size_t)m * lw * 4, cudaMemcpyDeviceToHost, st), "download");
  return rc ? rc : finish(ctx, "bconv");
}

int ckks_step_tensor(ckks_ctx* ctx, const uint32_t* ct1, const uint32_t* ct2, int n_q, uint32_t* out) {
  if (!ctx || !ct1 || !ct2 || !out) return CKKS_EINVAL;
  if (n_q < 1 || n_q > ctx->dp.L) return fail(ctx, CKKS_ELEVEL, "tensor: %d limbs", n_q);
  const size_t w = (size_t)n_q * limb_words(ctx);
  DevBuf a, b, o;
  if (a.alloc(2 * w * 4) || b.alloc(2 * w * 4) || o.alloc(3 * w * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(a.p, ct1, 2 * w * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(b.p, ct2, 2 * w * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  launch_tensor(ctx->dp, a.as<uint32_t>(), b.as<uint32_t>(), o.as<uint32_t>(), n_q, ctx->stream);
  rc = cuda_check(ctx, cudaMemcpyAsync(out, o.p, 3 * w * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "tensor");
}

int ckks_step_automorph(ckks_ctx* ctx, const uint32_t* in, int limbs, uint32_t galois, uint32_t* out) {
  if (!ctx || !in || !out || limbs < 0) return CKKS_EINVAL;
  if (galois % 2 == 0 || galois >= (2u << ctx->dp.log_n)) return fail(ctx, CKKS_EINVAL, "bad galois element");
  const size_t w = (size_t)limbs * limb_words(ctx);
  DevBuf a, b;
  if (a.alloc(w * 4) || b.alloc(w * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(a.p, in, w * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  launch_permute(ctx->dp, a.as<uint32_t>(), b.as<uint32_t>(), limbs, true, ctx->stream);
  launch_automorph(ctx->dp, b.as<uint32_t>(), a.as<uint32_t>(), limbs, galois, ctx->stream);
  launch_permute(ctx->dp, a.as<uint32_t>(), b.as<uint32_t>(), limbs, false, ctx->stream);
  rc = cuda_check(ctx, cudaMemcpyAsync(out, b.p, w * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "automorph");
}

static int step_ks(ckks_ctx* ctx, const uint32_t* d, int n_q, const ckks_evk* evk, int km, uint32_t* out,
                   size_t out_limbs) {
  if (n_q < 1 || n_q > ctx->dp.L) return fail(ctx, CKKS_ELEVEL, "%d limbs out of range", n_q);
  if (ctx->windowed) return fail(ctx, CKKS_EINVAL, "step entries need single-rescaling levels");
  const size_t lw = limb_words(ctx), w = (size_t)n_q * lw;
  DevBuf din, dcan, dout;
  if (din.alloc(w * 4) || dcan.alloc(w * 4) || dout.alloc(out_limbs * lw * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(dcan.p, d, w * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  launch_permute(ctx->dp, dcan.as<uint32_t>(), din.as<uint32_t>(), n_q, true, ctx->stream);
  KsArgs k{};
  ctx->set_level(k, n_q - 1);  // step entries: single-rescaling levels only
  k.mode = KS_PLAIN;
  k.x0 = din.as<uint32_t>();
  k.evk = evk ? evk->d : nullptr;
  k.extra = 0;
  launch_keyswitch(ctx->dp, ctx->sc, k, km, dout.as<uint32_t>(), ctx->stream);
  DevBuf canon;
  if (canon.alloc(out_limbs * lw * 4)) return fail(ctx, CKKS_ENOMEM, "scratch");
  launch_permute(ctx->dp, dout.as<uint32_t>(), canon.as<uint32_t>(), (int)out_limbs, false, ctx->stream);
  rc = cuda_check(ctx, cudaMemcpyAsync(out, canon.p, out_limbs * lw * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "keyswitch step");
}

int ckks_step_modup(ckks_ctx* ctx, const uint32_t* d, int n_q, uint32_t* out) {
  if (!ctx || !d || !out) return CKKS_EINVAL;
  const int digits = (n_q + ctx->dp.alpha - 1) / ctx->dp.alpha;
  return step_ks(ctx, d, n_q, nullptr, KM_MODUP, out, (size_t)digits * (n_q + ctx->dp.alpha));
}

int ckks_step_keyswitch_acc(ckks_ctx* ctx, const uint32_t* d, int n_q, const ckks_evk* evk, uint32_t* acc) {
  if (!ctx || !d || !evk || !acc) return CKKS_EINVAL;
  return step_ks(ctx, d, n_q, evk, KM_ACC_ALL, acc, 2 * (size_t)(n_q + ctx->dp.alpha));
}

int ckks_step_moddown(ckks_ctx* ctx, const uint32_t* acc, int n_q, uint32_t* out) {
  if (!ctx || !acc || !out) return CKKS_EINVAL;
  if (n_q < 1 || n_q > ctx->dp.L) return fail(ctx, CKKS_ELEVEL, "%d limbs out of range", n_q);
  const size_t lw = limb_words(ctx);
  const size_t in_limbs = 2 * (size_t)(n_q + ctx->dp.alpha), out_limbs = 2 * (size_t)n_q;
  DevBuf dcan, din, dout, dres;
  if (dcan.alloc(in_limbs * lw * 4) || din.alloc(in_limbs * lw * 4) || dout.alloc(out_limbs * lw * 4) ||
      dres.alloc(out_limbs * lw * 4))
    return fail(ctx, CKKS_ENOMEM, "scratch");
  int rc = cuda_check(ctx, cudaMemcpyAsync(dcan.p, acc, in_limbs * lw * 4, cudaMemcpyHostToDevice, ctx->stream), "upload");
  if (rc) return rc;
  launch_permute(ctx->dp, dcan.as<uint32_t>(), din.as<uint32_t>(), (int)in_limbs, true, ctx->stream);
  launch_moddown(ctx->dp, ctx->sc, din.as<uint32_t>(), n_q, dout.as<uint32_t>(), ctx->stream);
  launch_permute(ctx->dp, dout.as<uint32_t>(), dres.as<uint32_t>(), (int)out_limbs, false, ctx->stream);
  rc = cuda_check(ctx, cudaMemcpyAsync(out, dres.p, out_limbs * lw * 4, cudaMemcpyDeviceToHost, ctx->stream), "download");
  return rc ? rc : finish(ctx, "moddown step");
}

}  // extern "C"
