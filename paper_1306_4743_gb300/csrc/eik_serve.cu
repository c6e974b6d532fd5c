// eik_serve.cu -- request queue of the serving entry points.
#include <string.h>

#include <deque>
#include <map>
#include <new>
#include <vector>

#include "eik_serve.h"

namespace eik {

struct Request {
  int64_t dims[3];
  double h, tol;
  std::vector<float> F;
  std::vector<uint8_t> mask;
  std::vector<double> q;
  double* u_out;
  int state;   // 0 pending, 1 done
  int status;
  eik_stats stats;
};

struct ServeState {
  uint64_t next_ticket = 1;
  std::map<uint64_t, Request*> req;
  std::deque<uint64_t> pending;
};

void serve_destroy(ServeState* s) {
  if (!s) return;
  for (auto& kv : s->req) delete kv.second;
  delete s;
}

}  // namespace eik

eik::ServeState*& eik_serve_slot(eik_ctx* ctx);

namespace {

bool dims_ok(const int64_t* d) {
  for (int a = 0; a < 3; ++a)
    if (d[a] < 1 || d[a] > (1 << 24)) return false;
  return true;
}

// Run every pending request in one batched launch.
int run_pending(eik_ctx* ctx, eik::ServeState* s) {
  if (s->pending.empty()) return EIK_OK;
  std::vector<uint64_t> ids(s->pending.begin(), s->pending.end());
  s->pending.clear();
  // one launch per tolerance value (a batch shares its tolerance)
  std::map<double, std::vector<uint64_t>> by_tol;
  for (uint64_t id : ids) by_tol[s->req[id]->tol].push_back(id);
  for (auto& kv : by_tol) {
    const std::vector<uint64_t>& g = kv.second;
    const int count = (int)g.size();
    std::vector<int64_t> dims(3 * count);
    std::vector<double> h(count);
    std::vector<const float*> F(count);
    std::vector<const uint8_t*> M(count);
    std::vector<const double*> Q(count);
    std::vector<double*> U(count);
    for (int t = 0; t < count; ++t) {
      eik::Request* r = s->req[g[t]];
      memcpy(&dims[3 * t], r->dims, sizeof(r->dims));
      h[t] = r->h;
      F[t] = r->F.data();
      M[t] = r->mask.data();
      Q[t] = r->q.data();
      U[t] = r->u_out;
    }
    eik_stats st;
    const int rc = eik_run_batch(ctx, count, dims.data(), h.data(), F.data(), M.data(), Q.data(),
                                 kv.first, U.data(), true, nullptr, &st, 0);
    for (int t = 0; t < count; ++t) {
      eik::Request* r = s->req[g[t]];
      r->state = 1;
      r->status = rc;
      r->stats = st;
      r->F.clear();
      r->F.shrink_to_fit();
      r->mask.clear();
      r->mask.shrink_to_fit();
      r->q.clear();
      r->q.shrink_to_fit();
    }
  }
  return EIK_OK;
}

}  // namespace

extern "C" {

int eik_submit(eik_ctx* ctx, const int64_t dims[3], double h, const float* F,
               const uint8_t* src_mask, const double* q, double tol, double* u_out,
               uint64_t* ticket) {
  if (!ctx || !dims || !F || !src_mask || !q || !u_out || !ticket) return EIK_EINVAL;
  if (!dims_ok(dims) || !(h > 0.0) || !(tol >= 0.0)) return EIK_EINVAL;
  eik::ServeState*& s = eik_serve_slot(ctx);
  if (!s) {
    s = new (std::nothrow) eik::ServeState();
    if (!s) return EIK_ENOMEM;
  }
  eik::Request* r = new (std::nothrow) eik::Request();
  if (!r) return EIK_ENOMEM;
  const size_t nodes = (size_t)dims[0] * dims[1] * dims[2];
  memcpy(r->dims, dims, sizeof(r->dims));
  r->h = h;
  r->tol = tol;
  r->F.assign(F, F + nodes);
  r->mask.assign(src_mask, src_mask + nodes);
  r->q.assign(q, q + nodes);
  r->u_out = u_out;
  r->state = 0;
  r->status = EIK_OK;
  memset(&r->stats, 0, sizeof(r->stats));
  const uint64_t id = s->next_ticket++;
  s->req[id] = r;
  s->pending.push_back(id);
  *ticket = id;
  return EIK_OK;
}

int eik_poll(eik_ctx* ctx, uint64_t ticket, int* done, eik_stats* stats) {
  if (!ctx || !done) return EIK_EINVAL;
  *done = 0;
  eik::ServeState* s = eik_serve_slot(ctx);
  if (!s) return EIK_ENOTFOUND;
  auto it = s->req.find(ticket);
  if (it == s->req.end()) return EIK_ENOTFOUND;
  if (it->second->state == 0) run_pending(ctx, s);
  eik::Request* r = it->second;
  if (r->state != 1) return EIK_OK;
  *done = 1;
  const int rc = r->status;
  if (stats) *stats = r->stats;
  delete r;
  s->req.erase(it);
  return rc;
}

int eik_cancel(eik_ctx* ctx, uint64_t ticket) {
  if (!ctx) return EIK_EINVAL;
  eik::ServeState* s = eik_serve_slot(ctx);
  if (!s) return EIK_ENOTFOUND;
  auto it = s->req.find(ticket);
  if (it == s->req.end()) return EIK_ENOTFOUND;
  for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
    if (*p == ticket) {
      s->pending.erase(p);
      break;
    }
  delete it->second;
  s->req.erase(it);
  return EIK_OK;
}

}  // extern "C"
