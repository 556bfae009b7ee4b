// Host-side drivers of the forward map, its transpose and the batched CGLS (RTO).
#pragma once

#include <cuda_runtime.h>

#include <initializer_list>
#include <vector>

#include "pat_internal.h"

// Return the status of `expr` from the enclosing function unless it is PAT_OK.
#define PAT_TRY(expr)            \
  do {                           \
    pat_status _s = (expr);      \
    if (_s != PAT_OK) return _s; \
  } while (0)

namespace pat {

// Workspace layout of one RTO solve with K stacked samples (byte offsets,
// 256-aligned).  Fields: x, d, r_d, q_d, r_p, s, state (a0, w0, a1, w1),
// per-sample scalars, reduction partials, status word; w and the LSQR
// scalars lsq [kLsq][K] are used by the LSQR driver only.
struct RtoLayout {
  size_t x, d, r_d, q_d, r_p, s, state, gamma, alpha, beta, sigma, partial, status, w, lsq, total;
  int n_part;  // reduction blocks per partial slot
};
constexpr int kLsq = 12;

size_t state_bytes(const DeviceMesh& m, int K);   // 4 N K real
RtoLayout rto_layout(const DeviceMesh& m, int K);

pat_status forward(const DeviceMesh& m, const void* p0, int K, void* Y, double scale, void* ws,
                   cudaStream_t st);
pat_status adjoint(const DeviceMesh& m, const void* Yhat, int K, void* out, double scale, void* ws,
                   cudaStream_t st);

pat_status cgls_begin(const DeviceMesh& m, const void* y_obs, double sigma, int K, const void* eta,
                      const void* xi, uint64_t seed, char* ws, cudaStream_t st, bool zero_draws = false);
pat_status cgls_iterate(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                        cudaStream_t st, bool blocks);
pat_status cgls_finish(const DeviceMesh& m, int K, double* samples, double* mean, double* stdev, char* ws,
                       cudaStream_t st);
pat_status residual_norms(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st, bool blocks);
// One wave solve of the CGLS loop on an RTO workspace (dir 0: q_d = G d / sigma
// from the d field; dir 1: s = G^T r_d / sigma), replayed from a CUDA graph.
pat_status cgls_solve(const DeviceMesh& m, int dir, int K, double sigma, char* ws, cudaStream_t st);
// Pooled-statistics passes over the CGLS / LSQR iterate x held in ws (moments_kernel)
// and their in-place finish (moments_finish_kernel).
pat_status rto_moments(const DeviceMesh& m, int K, const double* center, double* out, char* ws, cudaStream_t st);
pat_status moments_finish(int64_t N, double n, int which, double* v, cudaStream_t st);

// LSQR (Paige & Saunders) on the same extended system and workspace; the
// iterate x sits where CGLS keeps it, so cgls_finish also finishes LSQR.
pat_status lsqr_begin(const DeviceMesh& m, const void* y_obs, double sigma, int K, const void* eta,
                      const void* xi, uint64_t seed, bool zero_draws, char* ws, cudaStream_t st);
pat_status lsqr_iterate(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                        cudaStream_t st);
pat_status lsqr_residual(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st);
pat_status whitened_misfit(const DeviceMesh& m, const double* x, const void* y_obs, double sigma, int K,
                           double* out, char* ws, cudaStream_t st);

// Building blocks of the grouped (multi-mesh) driver, pat_multi.cu.
template <typename T>
struct Step3Args;
template <typename T>
Step3Args<T> fwd3_args(const DeviceMesh& m, int K, int V, const T* p0, T* Y, T scale, T* const b[3], int i,
                       int64_t* threads);
template <typename T>
Step3Args<T> adj3_args(const DeviceMesh& m, int K, int V, const T* Yhat, T scale, T* const b[3], int i,
                       int64_t* threads);
template <typename T>
pat_status begin_pre(const DeviceMesh& m, const T* y_obs, double sigma, int K, const T* eta, const T* xi,
                     uint64_t seed, char* ws, cudaStream_t st, bool zero_draws = false);
template <typename T>
pat_status begin_post(const DeviceMesh& m, int K, char* ws, cudaStream_t st);
template <typename T>
pat_status iter_mid(const DeviceMesh& m, int K, char* ws, cudaStream_t st);
template <typename T>
pat_status iter_post(const DeviceMesh& m, int K, char* ws, cudaStream_t st);
int vec_width(const DeviceMesh& m, int K, std::initializer_list<const void*> ptrs);
int stage_span(const DeviceMesh& m, bool adj, int KV);
pat_status autotune(const DeviceMesh& m, int K, char* ws, int n_probe, pat_tune_entry* table, int* n_entries,
                    cudaStream_t st);

// Grouped RTO over several meshes (pat_multi.cu): one RTO problem per job.
struct Job {
  const DeviceMesh* m;
  int K;
  const void* y_obs;
  double sigma;
  const void* eta;
  const void* xi;
  uint64_t seed;
  double *samples, *mean, *stdev;
  char* ws;
};

pat_status rto_multi(const std::vector<Job>& jobs, int n_iter, cudaStream_t st);

// One three-level step launch with the mesh's variant for (direction, K) and
// V samples per thread (a width the variant and the buffers allow: V <=
// tuned_vec(m, dir, K), K % V == 0, buffers aligned to V elements).
template <typename T>
void step_tuned(const DeviceMesh& m, bool adj, int V, const Step3Args<T>& A, int64_t threads, cudaStream_t st);
int tuned_vec(const DeviceMesh& m, int dir, int K);

// Misfit gradient with respect to per-element c^2 (pat_grad.cu).
size_t grad_workspace_bytes(const DeviceMesh& m, int K);
pat_status grad_c2(const DeviceMesh& m, const void* p0, const void* Yhat, int K, double* g, void* p0_grad, char* ws,
                   cudaStream_t st);

// Counter-based N(0,1) draws (SplitMix64 output function + Box-Muller).
pat_status draw_normals(uint64_t seed, int stream_id, int64_t n_elem, int K, double* out, cudaStream_t st);

int sm_count();
pat_status cuda_check(cudaError_t e, const char* what);

}  // namespace pat
