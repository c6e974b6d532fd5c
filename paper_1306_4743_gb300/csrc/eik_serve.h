// eik_serve.h -- serving state of a context (eik_submit / eik_poll /
// eik_cancel), internal to libeik.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eik.h"

namespace eik {
struct ServeState;
void serve_destroy(ServeState* s);
}  // namespace eik

// The batched solve of eik_api.cu.
int eik_run_batch(eik_ctx* ctx, int count, const int64_t* dims, const double* h,
                  const float* const* F, const uint8_t* const* mask, const double* const* q,
                  double tol, double* const* u_out, bool host_io, cudaStream_t st,
                  eik_stats* stats, int n_override);
