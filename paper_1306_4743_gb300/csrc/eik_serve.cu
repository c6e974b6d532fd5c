// eik_serve.cu -- serving entry points (eik_submit / eik_poll / eik_cancel):
// continuous batching over a few execution slots.
//
// A submitted request waits in arrival order.  Whenever a slot is free, the
// waiting requests at the front (same tolerance, up to kMaxBatch requests
// and opts.serve_batch_nodes grid nodes) are launched together as one batch -- one persistent cell kernel over all
// their cells -- on that slot's own stream, as long as the device memory of
// all busy slots plus the new batch fits the context's budget.  Batches on
// different slots run concurrently on the device, so requests that arrive
// while others are solving start as soon as a slot and memory free up.
// Each poll retires finished batches (copying results to the callers'
// buffers) and admits more requests; nothing runs on a background thread.
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "eik_serve.h"

namespace eik {

constexpr int kSlots = 3;
constexpr int kMaxBatch = 64;

struct Request {
  int64_t dims[3];
  double h, tol;
  const float* F;  // the caller's buffers, read until the ticket completes
  const uint8_t* mask;
  const double* q;
  double* u_out;
  double* staging;  // where the batch writes; u_out unless cancelled
  int state;        // 0 waiting, 1 on the device, 2 done
  bool cancelled;
  int status;
  eik_stats stats;
};

struct Slot {
  Exec ex;
  bool ready = false;
  bool busy = false;
  Launch L;
  std::vector<uint64_t> tickets;
  std::vector<double*> sinks;  // result buffers of requests cancelled mid-flight
};

struct ServeState {
  uint64_t next_ticket = 1;
  std::map<uint64_t, Request*> req;
  std::deque<uint64_t> waiting;
  Slot slots[kSlots];
};

void serve_destroy(ServeState* s) {
  if (!s) return;
  for (Slot& sl : s->slots) {
    if (sl.ready) exec_free(sl.ex);  // waits for its stream first
    for (double* p : sl.sinks) delete[] p;
  }
  for (auto& kv : s->req) delete kv.second;
  delete s;
}

}  // namespace eik

eik::ServeState*& eik_serve_slot(eik_ctx* ctx);


namespace {

using eik::Request;
using eik::ServeState;
using eik::Slot;
using eik::kMaxBatch;

// The same rule as the synchronous calls: each edge in [1, 2^24], at most
// 2^34 nodes, bounded before the product is formed.
bool dims_ok(const int64_t* d) {
  for (int a = 0; a < 3; ++a)
    if (d[a] < 1 || d[a] > (1 << 24)) return false;
  return (long long)d[0] * d[1] <= (1ll << 34) / d[2];
}

void release_inputs(Request* r) {
  r->F = nullptr;
  r->mask = nullptr;
  r->q = nullptr;
}

// Retire every batch whose stream has finished.
void retire(eik_ctx* ctx, ServeState* s) {
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaStreamQuery(sl.ex.stream);
    if (q == cudaErrorNotReady) continue;
    int rc;
    eik_stats st;
    memset(&st, 0, sizeof(st));
    if (q != cudaSuccess) {
      cudaGetLastError();
      rc = EIK_ECUDA;
    } else {
      rc = eik_finish_batch(ctx, sl.ex, sl.L, &st);
    }
    for (uint64_t id : sl.tickets) {
      auto it = s->req.find(id);
      if (it == s->req.end()) continue;
      Request* r = it->second;
      r->state = 2;
      r->status = rc;
      r->stats = st;
      release_inputs(r);
      if (r->cancelled) {  // nobody waits for it any more
        delete r;
        s->req.erase(it);
      }
    }
    sl.busy = false;
    sl.tickets.clear();
    for (double* p : sl.sinks) delete[] p;
    sl.sinks.clear();
  }
}

// Launch waiting requests on free slots while memory allows.
void admit(eik_ctx* ctx, ServeState* s) {
  const size_t budget = eik_ctx_budget(ctx);
  while (!s->waiting.empty()) {
    Slot* free_slot = nullptr;
    size_t used = 0;
    for (Slot& sl : s->slots) {
      if (sl.busy) used += sl.ex.arena_size;
      else if (!free_slot) free_slot = &sl;
    }
    if (!free_slot) return;
    if (!free_slot->ready) {
      if (eik::exec_init(free_slot->ex, true) != EIK_OK) return;
      free_slot->ready = true;
    }
    // the batch: front requests with the front request's tolerance
    std::vector<uint64_t> ids;
    std::vector<int64_t> dims;
    std::vector<double> hs;
    const double tol = s->req[s->waiting.front()]->tol;
    const unsigned long long cap_nodes = eik_ctx_batch_nodes(ctx);
    unsigned long long batch_nodes = 0;
    size_t bytes = 0;
    for (auto it = s->waiting.begin(); it != s->waiting.end() && (int)ids.size() < kMaxBatch &&
                                           (ids.empty() || batch_nodes < cap_nodes);
         ++it) {
      Request* r = s->req[*it];
      if (r->tol != tol) continue;
      dims.insert(dims.end(), r->dims, r->dims + 3);
      hs.push_back(r->h);
      const size_t b = eik_plan_bytes(ctx, (int)hs.size(), dims.data(), hs.data(), true);
      const size_t need = std::max(b, free_slot->ex.arena_size);
      if (budget && used + need > budget) {
        dims.resize(dims.size() - 3);
        hs.pop_back();
        break;
      }
      bytes = b;
      ids.push_back(*it);
      batch_nodes += (unsigned long long)(r->dims[0] * r->dims[1] * r->dims[2]);
    }
    if (ids.empty()) {
      const uint64_t id = s->waiting.front();
      Request* r = s->req[id];
      int64_t d[3] = {r->dims[0], r->dims[1], r->dims[2]};
      const size_t alone = eik_plan_bytes(ctx, 1, d, &r->h, true);
      if (budget && alone > budget) {  // can never fit
        s->waiting.pop_front();
        r->state = 2;
        r->status = EIK_EBUDGET;
        release_inputs(r);
        continue;
      }
      return;  // wait for memory to free up
    }
    (void)bytes;
    std::vector<const float*> F;
    std::vector<const uint8_t*> M;
    std::vector<const double*> Q;
    std::vector<double*> U;
    for (uint64_t id : ids) {
      Request* r = s->req[id];
      F.push_back(r->F);
      M.push_back(r->mask);
      Q.push_back(r->q);
      U.push_back(r->staging);
      r->state = 1;
    }
    for (uint64_t id : ids)
      s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), id));
    const int rc = eik_launch_batch(ctx, free_slot->ex, (int)ids.size(), dims.data(), hs.data(),
                                    F.data(), M.data(), Q.data(), tol, U.data(), true,
                                    free_slot->ex.stream, true, free_slot->L, 0, 0);
    if (rc != EIK_OK) {
      cudaStreamSynchronize(free_slot->ex.stream);
      cudaGetLastError();
      for (uint64_t id : ids) {
        Request* r = s->req[id];
        r->state = 2;
        r->status = rc;
        release_inputs(r);
      }
      continue;
    }
    free_slot->busy = true;
    free_slot->tickets = ids;
  }
}

}  // namespace

extern "C" {

int eik_submit(eik_ctx* ctx, const int64_t dims[3], double h, const float* F,
               const uint8_t* src_mask, const double* q, double tol, double* u_out,
               uint64_t* ticket) {
  if (!ctx || !dims || !F || !src_mask || !q || !u_out || !ticket) return EIK_EINVAL;
  if (!dims_ok(dims) || !(h > 0.0) || !(tol >= 0.0)) return EIK_EINVAL;
  ServeState*& s = eik_serve_slot(ctx);
  if (!s) {
    s = new (std::nothrow) ServeState();
    if (!s) return EIK_ENOMEM;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) return EIK_ENOMEM;
  memcpy(r->dims, dims, sizeof(r->dims));
  r->h = h;
  r->tol = tol;
  r->F = F;
  r->mask = src_mask;
  r->q = q;
  r->u_out = u_out;
  r->staging = u_out;
  r->state = 0;
  r->cancelled = false;
  r->status = EIK_OK;
  memset(&r->stats, 0, sizeof(r->stats));
  const uint64_t id = s->next_ticket++;
  s->req[id] = r;
  s->waiting.push_back(id);
  admit(ctx, s);  // start at once if a slot is free
  *ticket = id;
  return EIK_OK;
}

int eik_poll(eik_ctx* ctx, uint64_t ticket, int* done, eik_stats* stats) {
  if (!ctx || !done) return EIK_EINVAL;
  *done = 0;
  ServeState* s = eik_serve_slot(ctx);
  if (!s) return EIK_ENOTFOUND;
  retire(ctx, s);
  admit(ctx, s);
  auto it = s->req.find(ticket);
  if (it == s->req.end() || it->second->cancelled) return EIK_ENOTFOUND;
  Request* r = it->second;
  if (r->state != 2) return EIK_OK;
  *done = 1;
  const int rc = r->status;
  if (stats) *stats = r->stats;
  delete r;
  s->req.erase(it);
  return rc;
}

int eik_cancel(eik_ctx* ctx, uint64_t ticket) {
  if (!ctx) return EIK_EINVAL;
  ServeState* s = eik_serve_slot(ctx);
  if (!s) return EIK_ENOTFOUND;
  auto it = s->req.find(ticket);
  if (it == s->req.end() || it->second->cancelled) return EIK_ENOTFOUND;
  Request* r = it->second;
  if (r->state == 1) {
    // on the device: let the batch finish, but write its result into a
    // private sink so the caller may free u_out now; a result written in
    // place (page-locked u_out) cannot be redirected, so wait for the batch
    const size_t nodes = (size_t)r->dims[0] * r->dims[1] * r->dims[2];
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      for (int t = 0; t < (int)sl.tickets.size(); ++t) {
        if (sl.tickets[t] != ticket) continue;
        if (sl.L.direct[t]) {
          cudaStreamSynchronize(sl.ex.stream);
          continue;
        }
        double* sink = new (std::nothrow) double[nodes];
        if (!sink) return EIK_ENOMEM;
        sl.L.outs[t] = sink;  // the finish copies here; freed on retire
        sl.sinks.push_back(sink);
      }
    }
    r->cancelled = true;
    return EIK_OK;
  }
  for (auto p = s->waiting.begin(); p != s->waiting.end(); ++p)
    if (*p == ticket) {
      s->waiting.erase(p);
      break;
    }
  delete r;
  s->req.erase(it);
  return EIK_OK;
}

}  // extern "C"
