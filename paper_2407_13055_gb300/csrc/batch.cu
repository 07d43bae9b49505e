// Batched form: a list of independent operations at mixed levels issued
// across execution lanes, optionally captured once into a CUDA graph so that
// the whole list is one launch (declarations in include/ckks.h).
//
// Stage-major persistent form (CKKS_BATCH_PERSISTENT): every key-switching
// operation runs its ModUp on its lane into a ModUp / accumulator region of
// its own, the lanes join, one persistent kernel runs the KeyMult + MAC of
// all of them and every element-wise operation from a device work queue
// (limb-major, so each evaluation-key limb is read once per batch and reused
// from L2), the lanes fork again for the ModDown tails, and join. Rescale
// operations (and a windowed context's HMult with rational rescaling) run
// whole on their lanes before the join.
#include <algorithm>
#include <atomic>
#include <vector>

#include "internal.h"

struct ckks_batch {
  ckks_ctx* ctx;
  std::vector<ckks_op> ops;
  std::vector<ckks_ctx*> lanes;        // direct: lane 0 is ctx itself; graph: all lanes are clones
  std::vector<cudaStream_t> streams;   // streams created for the clone lanes
  bool owns_lane0 = false;
  std::vector<cudaEvent_t> events;     // fork/join events, one per lane
  std::vector<cudaEvent_t> events2;    // second fork/join of the persistent form
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches_per_run = 0;
  // persistent form
  bool persistent = false;
  std::vector<int> role;               // per operation: 0 whole on its lane, 1 key switch, 2 element-wise
  std::vector<ckks::KsArgs> ks;        // role 1: key-switch arguments
  std::vector<size_t> t_off, a_off;    // role 1: ModUp limbs and accumulators in the arena (words)
  uint32_t* arena = nullptr;
  ckks::PersOp* d_ops = nullptr;
  int2* d_items = nullptr;
  int* d_q = nullptr;                  // [head, abort]
  int n_items = 0;
  int blocks = 0;
  int* h_admitted = nullptr;           // host-mapped admitted-operation count
  int* d_admitted = nullptr;
};

namespace {

int issue_one(ckks_ctx* lane, const ckks_op& o) {
  switch (o.op) {
    case CKKS_OP_HMULT:
      return ckks_hmult(lane, o.a, o.b, o.evk, o.flags, o.out);
    case CKKS_OP_HROT:
      return ckks_hrot(lane, o.a, o.r, o.evk, o.out);
    case CKKS_OP_HCONJ:
      return ckks_hconj(lane, o.a, o.evk, o.out);
    case CKKS_OP_PMULT:
      return ckks_pmult(lane, o.a, o.pt, o.out);
    case CKKS_OP_RESCALE:
      return ckks_rescale(lane, o.a, o.out);
    case CKKS_OP_HADD:
      return ckks_hadd(lane, o.a, o.b, o.out);
    case CKKS_OP_PADD:
      return ckks_padd(lane, o.a, o.pt, o.out);
    default:
      return CKKS_EINVAL;
  }
}

int cuda_fail(ckks_ctx* ctx, cudaError_t e, const char* what) {
  ctx->err = std::string("batch: ") + what + ": " + cudaGetErrorString(e);
  return CKKS_ECUDA;
}

// Issue the whole list: lane l takes operations i = l mod lanes; lanes 1..
// fork from and join back into lane 0's stream.
int issue_all(ckks_batch* b) {
  ckks_ctx* ctx = b->ctx;
  const size_t nl = b->lanes.size();
  cudaStream_t main = b->lanes[0]->stream;
  cudaError_t e = cudaEventRecord(b->events[0], main);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fork");
  for (size_t l = 1; l < nl; ++l)
    if ((e = cudaStreamWaitEvent(b->lanes[l]->stream, b->events[0], 0)) != cudaSuccess) return cuda_fail(ctx, e, "fork");
  for (size_t i = 0; i < b->ops.size(); ++i) {
    ckks_ctx* lane = b->lanes[i % nl];
    const int rc = issue_one(lane, b->ops[i]);
    if (rc != CKKS_OK) {
      if (lane != ctx) ctx->err = lane->err;
      return rc;
    }
  }
  for (size_t l = 1; l < nl; ++l) {
    if ((e = cudaEventRecord(b->events[l], b->lanes[l]->stream)) != cudaSuccess) return cuda_fail(ctx, e, "join");
    if ((e = cudaStreamWaitEvent(main, b->events[l], 0)) != cudaSuccess) return cuda_fail(ctx, e, "join");
  }
  return CKKS_OK;
}

// Fork lanes 1.. from lane 0's stream (ev[0]) or join them back (ev[l]).
int fork_lanes(ckks_batch* b, std::vector<cudaEvent_t>& ev) {
  cudaStream_t main = b->lanes[0]->stream;
  cudaError_t e = cudaEventRecord(ev[0], main);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "fork");
  for (size_t l = 1; l < b->lanes.size(); ++l)
    if ((e = cudaStreamWaitEvent(b->lanes[l]->stream, ev[0], 0)) != cudaSuccess) return cuda_fail(b->ctx, e, "fork");
  return CKKS_OK;
}

int join_lanes(ckks_batch* b, std::vector<cudaEvent_t>& ev) {
  cudaStream_t main = b->lanes[0]->stream;
  cudaError_t e;
  for (size_t l = 1; l < b->lanes.size(); ++l) {
    if ((e = cudaEventRecord(ev[l], b->lanes[l]->stream)) != cudaSuccess) return cuda_fail(b->ctx, e, "join");
    if ((e = cudaStreamWaitEvent(main, ev[l], 0)) != cudaSuccess) return cuda_fail(b->ctx, e, "join");
  }
  return CKKS_OK;
}

// The stage-major schedule of the persistent form (see the top of the file).
int issue_persistent(ckks_batch* b) {
  const size_t nl = b->lanes.size();
  const size_t limb = (size_t)1 << b->ctx->dp.log_n;
  int rc = fork_lanes(b, b->events);
  for (size_t i = 0; i < b->ops.size() && rc == CKKS_OK; ++i) {
    ckks_ctx* lane = b->lanes[i % nl];
    if (b->role[i] == 0) {
      rc = issue_one(lane, b->ops[i]);
      if (rc != CKKS_OK && lane != b->ctx) b->ctx->err = lane->err;
    } else if (b->role[i] == 1) {
      ckks::Scratch sc = lane->sc;
      sc.T = b->arena + b->t_off[i];
      ckks::launch_ks_modup(lane->dp, sc, b->ks[i], lane->stream);
    }
  }
  if (rc == CKKS_OK) rc = join_lanes(b, b->events);
  if (rc != CKKS_OK) return rc;
  ckks_ctx* l0 = b->lanes[0];
  cudaError_t e = cudaMemsetAsync(b->d_q, 0, 2 * sizeof(int), l0->stream);
  if (e != cudaSuccess) return cuda_fail(b->ctx, e, "queue reset");
  ckks::launch_persistent(l0->dp, b->d_ops, b->d_items, b->n_items, b->d_q, b->d_admitted, b->blocks, l0->stream);
  rc = fork_lanes(b, b->events2);
  for (size_t i = 0; i < b->ops.size() && rc == CKKS_OK; ++i) {
    if (b->role[i] != 1) continue;
    ckks_ctx* lane = b->lanes[i % nl];
    const ckks::KsArgs& k = b->ks[i];
    ckks::launch_ks_tail(lane->dp, lane->sc, k, b->arena + b->a_off[i], (size_t)(k.n + lane->dp.alpha) * limb,
                         lane->stream);
  }
  if (rc == CKKS_OK) rc = join_lanes(b, b->events2);
  if (rc == CKKS_OK && (e = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(b->ctx, e, "launch");
  return rc;
}

// Roles, key-switch arguments, arena, work items and the queue of the
// persistent form. Runs after the validation run (levels and scales set).
int build_persistent(ckks_batch* b) {
  const size_t nl = b->lanes.size();
  const int n_ops = (int)b->ops.size();
  const ckks::DevParams& dp = b->ctx->dp;
  const size_t limb = (size_t)1 << dp.log_n;
  b->role.assign(n_ops, 0);
  b->ks.assign(n_ops, ckks::KsArgs{});
  b->t_off.assign(n_ops, 0);
  b->a_off.assign(n_ops, 0);
  std::vector<ckks::PersOp> ops(n_ops);
  size_t words = 0;
  int max_ext = 0;
  for (int i = 0; i < n_ops; ++i) {
    const ckks_op& o = b->ops[i];
    ckks_ctx* lane = b->lanes[i % nl];
    ckks::PersOp& p = ops[i];
    p = ckks::PersOp{};
    if (o.op == CKKS_OP_HMULT || o.op == CKKS_OP_HROT || o.op == CKKS_OP_HCONJ) {
      // the validation run left out's level and scale as the operation sets
      // them; preparing again sets the same values
      const int lvl = o.out->level;
      const double scl = o.out->scale;
      bool staged = false;
      int rc;
      if (o.op == CKKS_OP_HMULT) {
        rc = prepare_hmult(lane, o.a, o.b, o.evk, o.flags, o.out, b->ks[i], staged);
      } else {
        const uint32_t g = o.op == CKKS_OP_HROT ? galois_of_rotation(o.r, dp.log_n) : (2u << dp.log_n) - 1;
        rc = prepare_hauto(lane, o.a, g, o.evk, o.out, b->ks[i]);
      }
      o.out->level = lvl;
      o.out->scale = scl;
      if (rc != CKKS_OK) {
        if (lane != b->ctx) b->ctx->err = lane->err;
        return rc;
      }
      if (staged) continue;  // whole on its lane
      const ckks::KsArgs& k = b->ks[i];
      const int ext = k.n + dp.alpha;
      const int digits = (k.base + k.n - 1) / dp.alpha - k.base / dp.alpha + 1;
      b->role[i] = 1;
      b->t_off[i] = words;
      words += (size_t)digits * ext * limb;
      b->a_off[i] = words;
      words += 2 * (size_t)ext * limb;
      p.kind = ckks::PK_KEYMULT;
      p.digits = digits;
      p.ks = k;
      max_ext = std::max(max_ext, ext);
    } else if (o.op == CKKS_OP_HADD || o.op == CKKS_OP_PADD || o.op == CKKS_OP_PMULT) {
      b->role[i] = 2;
      p.kind = o.op == CKKS_OP_HADD ? ckks::PK_HADD : (o.op == CKKS_OP_PADD ? ckks::PK_PADD : ckks::PK_PMULT);
      p.x = o.a->d;
      p.sx = o.a->poly_stride();
      p.y = o.op == CKKS_OP_HADD ? o.b->d : o.pt->d;
      p.sy = o.op == CKKS_OP_HADD ? o.b->poly_stride() : 0;
      p.out = o.out->d;
      p.so = o.out->poly_stride();
      p.n = b->ctx->lvl_n(o.a->level);
      p.base = b->ctx->lvl_base(o.a->level);
    }
  }
  std::vector<int2> items;
  for (int t = 0; t < max_ext; ++t)
    for (int i = 0; i < n_ops; ++i)
      if (b->role[i] == 1 && t < b->ks[i].n + dp.alpha) items.push_back(make_int2(i, t));
  for (int i = 0; i < n_ops; ++i)
    if (b->role[i] == 2)
      for (int y = 0; y < 2 * ops[i].n; ++y) items.push_back(make_int2(i, y));
  b->n_items = (int)items.size();
  if (words && cudaMalloc(&b->arena, words * sizeof(uint32_t)) != cudaSuccess) {
    b->ctx->err = "batch: persistent arena allocation failed";
    return CKKS_ENOMEM;
  }
  for (int i = 0; i < n_ops; ++i)
    if (b->role[i] == 1) {
      ops[i].T = b->arena + b->t_off[i];
      ops[i].A = b->arena + b->a_off[i];
    }
  cudaError_t e = cudaMalloc(&b->d_ops, std::max<size_t>(1, ops.size()) * sizeof(ckks::PersOp));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_q, 2 * sizeof(int));
  if (e != cudaSuccess) {
    b->ctx->err = "batch: persistent queue allocation failed";
    return CKKS_ENOMEM;
  }
  if ((e = cudaMemcpy(b->d_ops, ops.data(), ops.size() * sizeof(ckks::PersOp), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (!items.empty() &&
       (e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
           cudaSuccess))
    return cuda_fail(b->ctx, e, "persistent tables");
  void* h = nullptr;
  if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    b->ctx->err = "batch: admission counter allocation failed";
    return CKKS_ENOMEM;
  }
  b->h_admitted = static_cast<int*>(h);
  *static_cast<volatile int*>(h) = 0;
  void* d = nullptr;
  if ((e = cudaHostGetDevicePointer(&d, h, 0)) != cudaSuccess) return cuda_fail(b->ctx, e, "admission counter");
  b->d_admitted = static_cast<int*>(d);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx->device);
  b->blocks = 2 * std::max(1, sms);
  return CKKS_OK;
}

// Sets the admitted-operation count seen by the persistent kernel.
void set_admitted(ckks_batch* b, int v) {
  std::atomic_thread_fence(std::memory_order_seq_cst);
  *static_cast<volatile int*>(b->h_admitted) = v;
  std::atomic_thread_fence(std::memory_order_seq_cst);
}

bool aliases(const ckks_ct* x, const ckks_ct* y) { return x && y && x->d == y->d; }

void destroy(ckks_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (size_t l = b->owns_lane0 ? 0 : 1; l < b->lanes.size(); ++l) ckks_ctx_destroy(b->lanes[l]);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaEvent_t e : b->events2) cudaEventDestroy(e);
  if (b->arena) cudaFree(b->arena);
  if (b->d_ops) cudaFree(b->d_ops);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_q) cudaFree(b->d_q);
  if (b->h_admitted) cudaFreeHost(b->h_admitted);
  delete b;
}

}  // namespace

extern "C" int ckks_batch_create(ckks_ctx* ctx, const ckks_op* ops, int count, int lanes, int use_graph,
                                 ckks_batch** out) {
  if (!ctx || !ops || count < 1 || lanes < 1 || lanes > 64 || !out) return CKKS_EINVAL;
  if (use_graph & ~(CKKS_BATCH_GRAPH | CKKS_BATCH_PERSISTENT)) {
    ctx->err = "batch: unknown mode flags";
    return CKKS_EINVAL;
  }
  *out = nullptr;
  const bool graph = (use_graph & CKKS_BATCH_GRAPH) != 0, persistent = (use_graph & CKKS_BATCH_PERSISTENT) != 0;
  // The operations must be independent: no output may be another operation's
  // input or output.
  for (int i = 0; i < count; ++i) {
    if (!ops[i].out || !ops[i].a) {
      ctx->err = "batch: operation without input or output";
      return CKKS_EINVAL;
    }
    for (int j = 0; j < count; ++j) {
      if (aliases(ops[i].out, ops[j].a) || aliases(ops[i].out, ops[j].b) ||
          (i != j && aliases(ops[i].out, ops[j].out))) {
        ctx->err = "batch: operation outputs must not alias any input or output of the batch";
        return CKKS_EINVAL;
      }
    }
  }
  ckks_batch* b = new (std::nothrow) ckks_batch();
  if (!b) return CKKS_ENOMEM;
  b->ctx = ctx;
  b->ops.assign(ops, ops + count);
  b->persistent = persistent;
  // Direct mode: lane 0 is the context itself. Graph mode: every lane is a
  // clone on a private non-blocking stream (stream capture is not possible
  // on the legacy default stream), and the graph is launched into the
  // context stream.
  b->owns_lane0 = graph;
  if (!graph) b->lanes.push_back(ctx);
  int rc = CKKS_OK;
  for (int l = 0; l < lanes && rc == CKKS_OK; ++l) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = CKKS_ECUDA;
    else b->events.push_back(e);
    if (rc == CKKS_OK && persistent) {
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = CKKS_ECUDA;
      else b->events2.push_back(e);
    }
    if ((l == 0 && !graph) || rc != CKKS_OK) continue;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      rc = CKKS_ECUDA;
      break;
    }
    b->streams.push_back(s);
    ckks_ctx* c = nullptr;
    rc = ckks_ctx_clone(ctx, s, &c);
    if (rc == CKKS_OK) b->lanes.push_back(c);
  }
  // One direct run validates every operation and sets output levels/scales;
  // in graph mode it first waits for the work already queued on the context
  // stream (the graph itself is launched into that stream).
  if (rc == CKKS_OK && graph) {
    cudaError_t e = cudaEventRecord(b->events[0], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->lanes[0]->stream, b->events[0], 0);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "order after context stream");
  }
  if (rc == CKKS_OK) rc = issue_all(b);
  if (rc == CKKS_OK) {
    const cudaError_t e = cudaStreamSynchronize(b->lanes[0]->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "validation run");
  }
  if (rc == CKKS_OK && persistent) {
    rc = build_persistent(b);
    if (rc == CKKS_OK) set_admitted(b, count);
  }
  if (rc == CKKS_OK && graph) {
    const uint64_t l0 = ckks::launch_count();
    cudaStream_t cs = b->lanes[0]->stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "begin capture");
    if (rc == CKKS_OK) {
      const int irc = persistent ? issue_persistent(b) : issue_all(b);
      e = cudaStreamEndCapture(cs, &b->graph);
      rc = irc != CKKS_OK ? irc : (e != cudaSuccess ? cuda_fail(ctx, e, "end capture") : CKKS_OK);
    }
    if (rc == CKKS_OK && (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
      rc = cuda_fail(ctx, e, "instantiate");
    b->launches_per_run = ckks::launch_count() - l0;
  }
  if (rc != CKKS_OK) {
    if (ctx->err.empty()) ctx->err = "batch: creation failed";
    cudaGetLastError();
    destroy(b);
    return rc;
  }
  *out = b;
  return CKKS_OK;
}

static int batch_launch(ckks_batch* b) {
  if (b->exec) {
    const cudaError_t e = cudaGraphLaunch(b->exec, b->ctx->stream);
    if (e != cudaSuccess) {
      b->ctx->err = std::string("batch: graph launch: ") + cudaGetErrorString(e);
      return CKKS_ECUDA;
    }
    ckks::count_launch((int)b->launches_per_run);
    return CKKS_OK;
  }
  return b->persistent ? issue_persistent(b) : issue_all(b);
}

extern "C" int ckks_batch_run(ckks_batch* b) {
  if (!b) return CKKS_EINVAL;
  if (b->persistent) return ckks_batch_run_admit(b, (int)b->ops.size());
  return batch_launch(b);
}

extern "C" int ckks_batch_run_admit(ckks_batch* b, int admitted) {
  if (!b) return CKKS_EINVAL;
  if (!b->persistent || admitted < 0 || admitted > (int)b->ops.size()) {
    b->ctx->err = "batch: admission needs a persistent batch and 0 <= admitted <= count";
    return CKKS_EINVAL;
  }
  // a lower count must not reach a kernel of an earlier run still in flight
  if (admitted < *static_cast<volatile int*>(b->h_admitted)) {
    const cudaError_t e = cudaStreamSynchronize(b->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "admission");
  }
  set_admitted(b, admitted);
  return batch_launch(b);
}

extern "C" int ckks_batch_admit(ckks_batch* b, int admitted) {
  if (!b) return CKKS_EINVAL;
  if (!b->persistent || admitted < *static_cast<volatile int*>(b->h_admitted) || admitted > (int)b->ops.size()) {
    b->ctx->err = "batch: admission can only grow, up to the operation count, on a persistent batch";
    return CKKS_EINVAL;
  }
  set_admitted(b, admitted);
  return CKKS_OK;
}

extern "C" void ckks_batch_destroy(ckks_batch* b) {
  if (b) {
    cudaStreamSynchronize(b->ctx->stream);
    for (ckks_ctx* l : b->lanes) cudaStreamSynchronize(l->stream);
  }
  destroy(b);
}
