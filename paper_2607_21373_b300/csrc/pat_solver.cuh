// Host-side drivers of the forward map, its transpose and the batched CGLS (RTO).
#pragma once

#include <cuda_runtime.h>

#include "pat_internal.h"

namespace pat {

// Workspace layout of one RTO solve with K stacked samples (byte offsets,
// 256-aligned).  Fields: x, d, r_d, q_d, r_p, s, state (a0, w0, a1, w1),
// per-sample scalars, reduction partials, status word.
struct RtoLayout {
  size_t x, d, r_d, q_d, r_p, s, state, gamma, alpha, beta, sigma, partial, status, total;
  int n_part;  // reduction blocks per partial slot
};

size_t state_bytes(const DeviceMesh& m, int K);   // 4 N K real
RtoLayout rto_layout(const DeviceMesh& m, int K);

pat_status forward(const DeviceMesh& m, const void* p0, int K, void* Y, double scale, void* ws,
                   cudaStream_t st);
pat_status adjoint(const DeviceMesh& m, const void* Yhat, int K, void* out, double scale, void* ws,
                   cudaStream_t st);

pat_status cgls_begin(const DeviceMesh& m, const void* y_obs, double sigma, int K, const void* eta,
                      const void* xi, uint64_t seed, char* ws, cudaStream_t st);
pat_status cgls_iterate(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                        cudaStream_t st);
pat_status cgls_finish(const DeviceMesh& m, int K, double* samples, double* mean, double* stdev, char* ws,
                       cudaStream_t st);
pat_status residual_norms(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st);

// Counter-based N(0,1) draws (SplitMix64 output function + Box-Muller).
pat_status draw_normals(uint64_t seed, int stream_id, int64_t n_elem, int K, double* out, cudaStream_t st);

int sm_count();
pat_status cuda_check(cudaError_t e, const char* what);

}  // namespace pat
