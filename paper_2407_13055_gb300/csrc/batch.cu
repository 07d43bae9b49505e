// Batched form: a list of independent operations at mixed levels issued
// across execution lanes, optionally captured once into a CUDA graph so that
// the whole list is one launch (declarations in include/ckks.h).
#include <vector>

#include "internal.h"

struct ckks_batch {
  ckks_ctx* ctx;
  std::vector<ckks_op> ops;
  std::vector<ckks_ctx*> lanes;        // direct: lane 0 is ctx itself; graph: all lanes are clones
  std::vector<cudaStream_t> streams;   // streams created for the clone lanes
  bool owns_lane0 = false;
  std::vector<cudaEvent_t> events;     // fork/join events, one per lane
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches_per_run = 0;
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

bool aliases(const ckks_ct* x, const ckks_ct* y) { return x && y && x->d == y->d; }

void destroy(ckks_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (size_t l = b->owns_lane0 ? 0 : 1; l < b->lanes.size(); ++l) ckks_ctx_destroy(b->lanes[l]);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  delete b;
}

}  // namespace

extern "C" int ckks_batch_create(ckks_ctx* ctx, const ckks_op* ops, int count, int lanes, int use_graph,
                                 ckks_batch** out) {
  if (!ctx || !ops || count < 1 || lanes < 1 || lanes > 64 || !out) return CKKS_EINVAL;
  *out = nullptr;
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
  // Direct mode: lane 0 is the context itself. Graph mode: every lane is a
  // clone on a private non-blocking stream (stream capture is not possible
  // on the legacy default stream), and the graph is launched into the
  // context stream.
  b->owns_lane0 = use_graph != 0;
  if (!use_graph) b->lanes.push_back(ctx);
  int rc = CKKS_OK;
  for (int l = 0; l < lanes && rc == CKKS_OK; ++l) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = CKKS_ECUDA;
    else b->events.push_back(e);
    if ((l == 0 && !use_graph) || rc != CKKS_OK) continue;
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
  if (rc == CKKS_OK && use_graph) {
    cudaError_t e = cudaEventRecord(b->events[0], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->lanes[0]->stream, b->events[0], 0);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "order after context stream");
  }
  if (rc == CKKS_OK) rc = issue_all(b);
  if (rc == CKKS_OK) {
    const cudaError_t e = cudaStreamSynchronize(b->lanes[0]->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "validation run");
  }
  if (rc == CKKS_OK && use_graph) {
    const uint64_t l0 = ckks::launch_count();
    cudaStream_t cs = b->lanes[0]->stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "begin capture");
    if (rc == CKKS_OK) {
      const int irc = issue_all(b);
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

extern "C" int ckks_batch_run(ckks_batch* b) {
  if (!b) return CKKS_EINVAL;
  if (b->exec) {
    const cudaError_t e = cudaGraphLaunch(b->exec, b->ctx->stream);
    if (e != cudaSuccess) {
      b->ctx->err = std::string("batch: graph launch: ") + cudaGetErrorString(e);
      return CKKS_ECUDA;
    }
    ckks::count_launch((int)b->launches_per_run);
    return CKKS_OK;
  }
  return issue_all(b);
}

extern "C" void ckks_batch_destroy(ckks_batch* b) {
  if (b) {
    cudaStreamSynchronize(b->ctx->stream);
    for (ckks_ctx* l : b->lanes) cudaStreamSynchronize(l->stream);
  }
  destroy(b);
}
