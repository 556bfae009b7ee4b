// Uneven batches: several meshes (sizes, time-step counts, sensor sets, noise
// levels and sample counts K) solved together.  Each time-step launch covers
// the rows of every job that still has a step to take at that index, so small
// meshes ride along with large ones instead of leaving the GPU half empty; the
// per-sample CGLS vector work stays per job.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pat_kernels.cuh"
#include "pat_solver.cuh"

namespace pat {

template <typename T, int V, bool SPLIT, bool ADJ>
static void launch_group(const std::vector<const DeviceMesh*>& ms, const std::vector<Step3Args<T>>& a,
                         const std::vector<int64_t>& thr, cudaStream_t st) {
  for (size_t base = 0; base < a.size(); base += kMaxGroup) {
    Step3Group<T> G{};
    G.n = (int)std::min<size_t>(kMaxGroup, a.size() - base);
    int64_t off = 0;
    int cap = 0;
    bool stage = true;
    for (int g = 0; g < G.n; ++g) {
      G.block_off[g] = off;
      G.a[g] = a[base + g];
      const int KV = G.a[g].K / V;
      const int span = KV >= 2 ? stage_span(*ms[base + g], ADJ, KV) : 0;
      G.a[g].stage_cap = span;
      cap = std::max(cap, span);
      stage = stage && KV >= 2;
      off += (thr[base + g] + 255) / 256;
    }
    G.block_off[G.n] = off;
    for (int g = G.n + 1; g <= kMaxGroup; ++g) G.block_off[g] = off;
    const size_t smem = stage_bytes<T, SPLIT>(cap);
    if (off == 0) continue;
    if constexpr (sizeof(T) == 4 && SPLIT && (V == 4 || V == 8)) {
      // packed f32x2 kernel (the default variant of the single-mesh launches)
      for (int g = 0; g < G.n; ++g) G.a[g].hl = ADJ ? ms[base + g]->adj3.hl : ms[base + g]->fwd.hl;
      step3f_group_kernel<V, 4, ADJ><<<(unsigned)off, 256, 0, st>>>(G);
      continue;
    }
    if (stage && smem <= 48 * 1024) {
      // every member addresses the block's shared memory with the common capacity
      for (int g = 0; g < G.n; ++g) G.a[g].stage_cap = cap;
      step3_group_kernel<T, V, SPLIT, ADJ, true><<<(unsigned)off, 256, smem, st>>>(G);
    } else {
      step3_group_kernel<T, V, SPLIT, ADJ, false><<<(unsigned)off, 256, 0, st>>>(G);
    }
  }
}

template <typename T>
static T* state_buf(const Job& j, int q) {
  const RtoLayout L = rto_layout(*j.m, j.K);
  return (T*)(j.ws + L.state) + (size_t)q * j.m->N * j.K;
}

// q_d = G d / sigma for every job, one launch per time index
template <typename T, int V, bool SPLIT>
static void grouped_forward(const std::vector<Job>& jobs, int max_nt, cudaStream_t st) {
  for (int i = 0; i <= max_nt; ++i) {
    std::vector<Step3Args<T>> a;
    std::vector<int64_t> thr;
    std::vector<const DeviceMesh*> ms;
    for (const Job& j : jobs) {
      if (i > j.m->n_steps) continue;
      const RtoLayout L = rto_layout(*j.m, j.K);
      T* const b[3] = {state_buf<T>(j, 0), state_buf<T>(j, 1), state_buf<T>(j, 2)};
      int64_t t = 0;
      ms.push_back(j.m);
      a.push_back(fwd3_args<T>(*j.m, j.K, V, (const T*)(j.ws + L.d), (T*)(j.ws + L.q_d), (T)(1.0 / j.sigma), b, i,
                               &t));
      thr.push_back(t);
    }
    launch_group<T, V, SPLIT, false>(ms, a, thr, st);
  }
}

// s = G^T r_d / sigma for every job
template <typename T, int V, bool SPLIT>
static void grouped_adjoint(const std::vector<Job>& jobs, int max_nt, cudaStream_t st) {
  for (int i = 0; i <= max_nt; ++i) {
    std::vector<Step3Args<T>> a;
    std::vector<int64_t> thr;
    std::vector<const DeviceMesh*> ms;
    for (const Job& j : jobs) {
      if (i > j.m->n_steps) continue;
      const RtoLayout L = rto_layout(*j.m, j.K);
      T* const b[3] = {state_buf<T>(j, 0), state_buf<T>(j, 1), state_buf<T>(j, 2)};
      int64_t t = 0;
      ms.push_back(j.m);
      a.push_back(adj3_args<T>(*j.m, j.K, V, (const T*)(j.ws + L.r_d), (T)(1.0 / j.sigma), b, i, &t));
      thr.push_back(t);
    }
    launch_group<T, V, SPLIT, true>(ms, a, thr, st);
  }
  for (const Job& j : jobs) {
    const DeviceMesh& m = *j.m;
    const RtoLayout L = rto_layout(m, j.K);
    const int NT = m.n_steps;
    const int64_t rt = m.N * (int64_t)j.K / V;
    adj3_finish_kernel<T, V, SPLIT><<<(unsigned)((rt + 255) / 256), 256, 0, st>>>(
        rt, j.K, m.fwd.ptr, m.fwd.col, static_cast<const T*>(m.fwd.hi), m.fwd.lo, m.ml, state_buf<T>(j, NT % 3),
        state_buf<T>(j, (NT - 1) % 3), (T*)(j.ws + L.s));
  }
}

template <typename T, int V, bool SPLIT>
static pat_status multi_t(const std::vector<Job>& jobs, int n_iter, cudaStream_t st) {
  int max_nt = 0;
  for (const Job& j : jobs) max_nt = std::max(max_nt, j.m->n_steps);
  for (const Job& j : jobs) {
    pat_status s = begin_pre<T>(*j.m, (const T*)j.y_obs, j.sigma, j.K, (const T*)j.eta, (const T*)j.xi, j.seed, j.ws,
                                st);
    if (s) return s;
  }
  grouped_adjoint<T, V, SPLIT>(jobs, max_nt, st);
  for (const Job& j : jobs) {
    pat_status s = begin_post<T>(*j.m, j.K, j.ws, st);
    if (s) return s;
  }
  for (int it = 0; it < n_iter; ++it) {
    grouped_forward<T, V, SPLIT>(jobs, max_nt, st);
    for (const Job& j : jobs) {
      pat_status s = iter_mid<T>(*j.m, j.K, j.ws, st);
      if (s) return s;
    }
    grouped_adjoint<T, V, SPLIT>(jobs, max_nt, st);
    for (const Job& j : jobs) {
      pat_status s = iter_post<T>(*j.m, j.K, j.ws, st);
      if (s) return s;
    }
  }
  for (const Job& j : jobs) {
    pat_status s = cgls_finish(*j.m, j.K, j.samples, j.mean, j.stdev, j.ws, st);
    if (s) return s;
  }
  return cuda_check(cudaGetLastError(), "pat_rto_sample_multi launch");
}

pat_status rto_multi(const std::vector<Job>& jobs, int n_iter, cudaStream_t st) {
  const DeviceMesh& m0 = *jobs[0].m;
  int V = 4;
  for (const Job& j : jobs) {
    const RtoLayout L = rto_layout(*j.m, j.K);
    V = std::min(V, vec_width(*j.m, j.K, {j.ws, j.ws + L.d, j.ws + L.q_d, j.ws + L.r_d, j.ws + L.s}));
  }
  if (m0.prec == PAT_F64) {
    if (V >= 2) return multi_t<double, 2, false>(jobs, n_iter, st);
    return multi_t<double, 1, false>(jobs, n_iter, st);
  }
  if (m0.split) {
    if (V == 4) return multi_t<float, 4, true>(jobs, n_iter, st);
    if (V == 2) return multi_t<float, 2, true>(jobs, n_iter, st);
    return multi_t<float, 1, true>(jobs, n_iter, st);
  }
  if (V == 4) return multi_t<float, 4, false>(jobs, n_iter, st);
  if (V == 2) return multi_t<float, 2, false>(jobs, n_iter, st);
  return multi_t<float, 1, false>(jobs, n_iter, st);
}

}  // namespace pat
