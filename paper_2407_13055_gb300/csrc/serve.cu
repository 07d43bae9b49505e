// Served form: continuous batching of single HMult / HRot requests over
// execution lanes, with admission by device footprint (the paper runs one
// operation at a time; its Sec. 5.2 names multi-query batching as another
// model). The scheduler is a host loop on the calling thread: it admits
// requests in arrival order as lanes and pool bytes free up, enqueues each on
// its lane's stream followed by a CUDA event, and polls the events of the
// running requests. Nothing here allocates device memory.
#include <chrono>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// The library's own issue: the operation on the lane, then the lane's event.
int issue_own(ckks_ctx* lane, const ckks_request& r, ckks_ct* lane_out, cudaEvent_t ev) {
  ckks_ct* out = r.out ? r.out : lane_out;
  const int rc = r.op == CKKS_OP_HMULT ? ckks_hmult(lane, r.a, r.b, r.evk, CKKS_RESCALE, out)
                                       : ckks_hrot(lane, r.a, r.r, r.evk, out);
  if (rc != CKKS_OK) return rc;
  const cudaError_t e = cudaEventRecord(ev, lane->stream);
  if (e != cudaSuccess) {
    lane->err = std::string("serve: event record: ") + cudaGetErrorString(e);
    return CKKS_ECUDA;
  }
  return CKKS_OK;
}

// 1: the lane's request has completed, 0: still running, < 0: failure.
int query_own(ckks_ctx* lane, cudaEvent_t ev) {
  const cudaError_t e = cudaEventQuery(ev);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  lane->err = std::string("serve: ") + cudaGetErrorString(e);
  return CKKS_ECUDA;
}

}  // namespace

extern "C" int ckks_serve_run(ckks_ctx* const* lanes, int n_lanes, ckks_pool* pool, const ckks_request* reqs, int n,
                              ckks_ct* const* lane_outs, const ckks_serve_hooks* hooks, ckks_request_done* done,
                              int* order) {
  if (n_lanes < 1 || n_lanes > 64 || !pool || n < 0 || (n > 0 && (!reqs || !done))) return CKKS_EINVAL;
  const bool own = hooks == nullptr;
  if (!own && (!hooks->issue || !hooks->query)) return CKKS_EINVAL;
  if (own) {
    if (!lanes) return CKKS_EINVAL;
    for (int l = 0; l < n_lanes; ++l)
      if (!lanes[l]) return CKKS_EINVAL;
  }
  ckks_ctx* ectx = own ? lanes[0] : nullptr;  // where error messages go
  auto reject = [&](const std::string& msg) {
    if (ectx) ectx->err = msg;
    return CKKS_EINVAL;
  };
  // The bytes the pool already holds (resident keys) stay held for the run,
  // so a request larger than the rest of the budget could never start.
  const size_t held = pool->used.load();
  const size_t room = pool->budget > held ? pool->budget - held : 0;
  for (int i = 0; i < n; ++i) {
    const ckks_request& r = reqs[i];
    if (r.op != CKKS_OP_HMULT && r.op != CKKS_OP_HROT)
      return reject("serve: request " + std::to_string(i) + ": op must be CKKS_OP_HMULT or CKKS_OP_HROT");
    if (i > 0 && r.arrival_s < reqs[i - 1].arrival_s)
      return reject("serve: requests must be sorted by arrival time");
    if (r.bytes > room)
      return reject("serve: request " + std::to_string(i) + " needs " + std::to_string(r.bytes) +
                    " bytes, more than the pool can grant (" + std::to_string(room) + " free of " +
                    std::to_string(pool->budget) + ")");
    if (own && (!r.a || !r.evk || (r.op == CKKS_OP_HMULT && !r.b) || (!r.out && !lane_outs)))
      return reject("serve: request " + std::to_string(i) + " lacks an input, key or output");
  }
  for (int i = 0; i < n; ++i) done[i] = ckks_request_done{-1.0, -1.0, -1};
  if (n == 0) return CKKS_OK;

  std::vector<cudaEvent_t> ev(own ? n_lanes : 0, nullptr);
  for (size_t l = 0; l < ev.size(); ++l) {
    const cudaError_t e = cudaEventCreateWithFlags(&ev[l], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (size_t k = 0; k < l; ++k) cudaEventDestroy(ev[k]);
      ectx->err = std::string("serve: event create: ") + cudaGetErrorString(e);
      return CKKS_ECUDA;
    }
  }

  using Clock = std::chrono::steady_clock;
  const Clock::time_point t0 = Clock::now();
  auto now = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  std::vector<int> running(n_lanes, -1);  // request on each lane, -1 when idle
  int next = 0, completed = 0, busy = 0, rc = CKKS_OK;
  while (busy > 0 || (rc == CKKS_OK && next < n)) {
    // completions: release the bytes, free the lane
    for (int l = 0; l < n_lanes && busy > 0; ++l) {
      const int i = running[l];
      if (i < 0) continue;
      const int st = own ? query_own(lanes[l], ev[l]) : hooks->query(hooks->user, l);
      if (st == 0) continue;
      if (st < 0 && rc == CKKS_OK) {
        rc = st;
        if (own && l != 0) ectx->err = lanes[l]->err;
      }
      done[i].end_s = now();
      ckks_pool_release(pool, reqs[i].bytes);
      if (order) order[completed] = i;
      ++completed;
      running[l] = -1;
      --busy;
    }
    // admissions, in arrival order: an idle lane and the request's bytes
    while (rc == CKKS_OK && next < n && reqs[next].arrival_s <= now()) {
      int l = 0;
      while (l < n_lanes && running[l] >= 0) ++l;
      if (l == n_lanes || ckks_pool_acquire(pool, reqs[next].bytes) != CKKS_OK) break;
      done[next].start_s = now();
      const int irc = own ? issue_own(lanes[l], reqs[next], lane_outs ? lane_outs[l] : nullptr, ev[l])
                          : hooks->issue(hooks->user, next, l);
      if (irc != CKKS_OK) {
        if (own && l != 0) ectx->err = lanes[l]->err;
        ckks_pool_release(pool, reqs[next].bytes);
        done[next].start_s = -1.0;
        rc = irc;
        break;
      }
      done[next].lane = l;
      running[l] = next++;
      ++busy;
    }
  }
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  return rc;
}
