// eik_serve.h -- execution slots and the launch / finish split of a batched
// solve (internal to libeik.so): a synchronous call launches and finishes on
// the context's own slot; the serving queue keeps several slots in flight.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "eik.h"
#include "eik_internal.h"

namespace eik {

struct Launch;

// Device and pinned host memory, stream and events of one batch in flight.
struct Exec {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* arena = nullptr;  // device arena (grow-only)
  size_t arena_size = 0;
  char* h_small = nullptr;  // pinned: tables to the device, control block back
  size_t h_small_size = 0;
  char* h_out = nullptr;  // pinned: results of an asynchronous host-buffer batch
  size_t h_out_size = 0;
  char* h_ctl = nullptr;  // pinned: read-back of the control block
  size_t h_ctl_size = 0;
  cudaEvent_t ev[6] = {};
  // captured launch sequence of the last device-buffer batch, replayed while
  // its arguments (and so its arena layout and tensor maps) are unchanged
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned long long> graph_key;
  Launch* graph_launch = nullptr;
};

// A launched batch, until eik_finish_batch has read it back.
struct Launch {
  int count = 0, n = 0, grid = 0;
  int launches = 0;  // kernels this batch enqueued
  int wpc = 1;       // warps per worker of the min-mode cell kernels
  bool polish = false, host_io = false, async_out = false;
  long long nodes_total = 0;
  Control* hres = nullptr;  // pinned copy of the control block
  std::vector<double*> outs;
  std::vector<size_t> out_off;  // offsets in h_out (asynchronous host outputs)
  std::vector<long long> out_nodes;
  std::vector<char> direct;     // 1: the result is written in place (page-locked u_out)
};

int exec_init(Exec& e, bool own_stream);
void exec_free(Exec& e);

struct ServeState;
void serve_destroy(ServeState* s);

}  // namespace eik

// Device bytes a batch needs (the arena of its slot).
size_t eik_plan_bytes(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                      bool host_io);
size_t eik_ctx_budget(eik_ctx* ctx);
unsigned long long eik_ctx_batch_nodes(eik_ctx* ctx);

// Enqueue a batch on `ex` / `st`.  With async_out, host outputs are staged in
// pinned memory and copied to the caller's buffers by eik_finish_batch.
int eik_launch_batch(eik_ctx* ctx, eik::Exec& ex, int count, const int64_t* dims,
                     const double* h, const float* const* F, const uint8_t* const* mask,
                     const double* const* q, double tol, double* const* u_out, bool host_io,
                     cudaStream_t st, bool async_out, eik::Launch& L, size_t arena_limit,
                     int n_override);
// Read back a batch whose stream work has completed.
int eik_finish_batch(eik_ctx* ctx, eik::Exec& ex, eik::Launch& L, eik_stats* stats);

// Launch and finish on the context's own slot (synchronous).
int eik_run_batch(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                  const float* const* F, const uint8_t* const* mask, const double* const* q,
                  double tol, double* const* u_out, bool host_io, cudaStream_t st,
                  eik_stats* stats, int n_override);
