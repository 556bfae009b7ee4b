// Uneven batches: several meshes (sizes, time-step counts, sensor sets, noise
// levels and sample counts K) solved together.  Each time-step launch covers
// the rows of every job that still has a step to take at that index, so small
// meshes ride along with large ones instead of leaving the GPU half empty; the
// per-sample CGLS vector work stays per job.  With FP32 split coefficients and
// K a multiple of 8 for every job, a step launch is one persistent grid of the
// fixed-width kernels over all jobs' rows (16 slots when every mesh has them,
// else 8), launched as a programmatic dependent of the previous step, and each
// grouped wave solve (all of its step launches) is captured once per call into
// a CUDA graph that the CGLS loop replays.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "pat_kernels.cuh"
#include "pat_solver.cuh"
#include "pat_wide.cuh"

namespace pat {

// Which fixed-width layout a grouped launch can use: 2 = 16 slots, 1 = 8 slots,
// 0 = none (some job lacks FP32 split fixed-width rows).
static int group_layout(const std::vector<const DeviceMesh*>& ms) {
  bool w16 = true, ell = true;
  for (const DeviceMesh* m : ms) {
    const bool f32s = m->prec == PAT_F32 && m->split;
    w16 = w16 && f32s && m->fwd.w16_col && m->adj3.w16_col;
    ell = ell && f32s && m->fwd.ell_col && m->adj3.ell_col;
  }
  return w16 ? 2 : ell ? 1 : 0;
}

// One persistent grouped launch of the fixed-width kernels (V = 8).
template <bool ADJ>
static void launch_group_fixed(const std::vector<const DeviceMesh*>& ms, const std::vector<Step3Args<float>>& a,
                               const std::vector<int64_t>& thr, int layout, cudaStream_t st) {
  for (size_t base = 0; base < a.size(); base += kMaxGroup) {
    Step3Group<float> G{};
    G.n = (int)std::min<size_t>(kMaxGroup, a.size() - base);
    int64_t off = 0;
    for (int g = 0; g < G.n; ++g) {
      const DeviceMesh& m = *ms[base + g];
      const DevCSR& E = ADJ ? m.adj3 : m.fwd;
      G.block_off[g] = off;  // in 32-thread chunks
      G.a[g] = a[base + g];
      G.a[g].ell_desc = E.ell_desc;
      G.a[g].ell_col = layout == 2 ? E.w16_col : E.ell_col;  // quad-interleaved 16-slot copy
      G.a[g].ell_hl = layout == 2 ? E.w16_hl : E.ell_hl;
      G.a[g].ovf_ptr = layout == 2 ? E.w16_ovf_ptr : E.ovf_ptr;
      G.a[g].ovf_col = layout == 2 ? E.w16_ovf_col : E.ovf_col;
      G.a[g].ovf_hl = layout == 2 ? E.w16_ovf_hl : E.ovf_hl;
      G.a[g].order = nullptr;
      G.a[g].pf_rows = 0;
      off += (thr[base + g] + 31) / 32;
    }
    for (int g = G.n; g <= kMaxGroup; ++g) G.block_off[g] = off;
    if (off == 0) continue;
    void (*kern)(const Step3Group<float>, int64_t) =
        layout == 2 ? step3g_persist_kernel<ADJ, true> : step3g_persist_kernel<ADJ, false>;
    static int per_sm[2][2] = {{0, 0}, {0, 0}};
    static std::once_flag once;
    std::call_once(once, [] {
      const void* fns[2][2] = {{(const void*)step3g_persist_kernel<false, false>,
                                (const void*)step3g_persist_kernel<false, true>},
                               {(const void*)step3g_persist_kernel<true, false>,
                                (const void*)step3g_persist_kernel<true, true>}};
      for (int d = 0; d < 2; ++d)
        for (int w = 0; w < 2; ++w)
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[d][w], fns[d][w], 256, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm[d][w] = 1;
          }
    });
    const int resident = std::max(1, per_sm[ADJ ? 1 : 0][layout == 2 ? 1 : 0]);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)resident * sm_count(), (off + 7) / 8));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(256u);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, G, off) != cudaSuccess) {
      cudaGetLastError();  // attribute refused: plain launch
      kern<<<(unsigned)grid, 256u, 0, st>>>(G, off);
    }
  }
}

template <typename T, int V, bool SPLIT, bool ADJ>
static void launch_group(const std::vector<const DeviceMesh*>& ms, const std::vector<Step3Args<T>>& a,
                         const std::vector<int64_t>& thr, cudaStream_t st) {
  if constexpr (sizeof(T) == 4 && SPLIT && V == 8) {
    const int layout = group_layout(ms);
    if (layout) {
      launch_group_fixed<ADJ>(ms, a, thr, layout, st);
      return;
    }
  }
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
      a.back().inj_cur = nullptr;  // the grouped kernels compute the sensor terms in the row
      a.back().inj_next = nullptr;
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

// The two grouped wave solves of this call, each captured once into a CUDA
// graph on the first job's private capture stream and replayed on st (direct
// launches when st is being captured by the caller, or the capture fails).
template <typename T, int V, bool SPLIT>
struct GroupedSolves {
  const std::vector<Job>& jobs;
  int max_nt;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};

  GroupedSolves(const std::vector<Job>& j, int nt) : jobs(j), max_nt(nt) {}
  ~GroupedSolves() {
    for (cudaGraphExec_t e : exec)
      if (e) cudaGraphExecDestroy(e);
  }
  void direct(int dir, cudaStream_t st) {
    if (dir == 0)
      grouped_forward<T, V, SPLIT>(jobs, max_nt, st);
    else
      grouped_adjoint<T, V, SPLIT>(jobs, max_nt, st);
  }
  pat_status run(int dir, cudaStream_t st) {
    const DeviceMesh& m0 = *jobs[0].m;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((m0.flags & PAT_MESH_NO_GRAPHS) || !m0.capture_stream || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      direct(dir, st);
      return cuda_check(cudaGetLastError(), "grouped solve launch");
    }
    if (!exec[dir]) {
      std::lock_guard<std::mutex> lock(m0.graph_mutex);
      cudaStream_t cap = (cudaStream_t)m0.capture_stream;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaGetLastError();
        direct(dir, st);
        return cuda_check(cudaGetLastError(), "grouped solve launch");
      }
      direct(dir, cap);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cap, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_check(e, "grouped solve capture");
      }
      e = cudaGraphInstantiate(&exec[dir], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        exec[dir] = nullptr;
        return cuda_check(e, "grouped solve instantiate");
      }
    }
    return cuda_check(cudaGraphLaunch(exec[dir], st), "grouped solve graph launch");
  }
};

template <typename T, int V, bool SPLIT>
static pat_status multi_t(const std::vector<Job>& jobs, int n_iter, cudaStream_t st) {
  int max_nt = 0;
  for (const Job& j : jobs) max_nt = std::max(max_nt, j.m->n_steps);
  GroupedSolves<T, V, SPLIT> solves(jobs, max_nt);
  for (const Job& j : jobs) {
    pat_status s = begin_pre<T>(*j.m, (const T*)j.y_obs, j.sigma, j.K, (const T*)j.eta, (const T*)j.xi, j.seed, j.ws,
                                st);
    if (s) return s;
  }
  PAT_TRY(solves.run(1, st));
  for (const Job& j : jobs) {
    pat_status s = begin_post<T>(*j.m, j.K, j.ws, st);
    if (s) return s;
  }
  for (int it = 0; it < n_iter; ++it) {
    PAT_RANGE("grouped CGLS iteration");
    PAT_TRY(solves.run(0, st));
    for (const Job& j : jobs) {
      pat_status s = iter_mid<T>(*j.m, j.K, j.ws, st);
      if (s) return s;
    }
    PAT_TRY(solves.run(1, st));
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
  int V = (m0.prec == PAT_F32 && m0.split) ? 8 : 4;
  for (const Job& j : jobs) {
    const RtoLayout L = rto_layout(*j.m, j.K);
    V = std::min(V, vec_width(*j.m, j.K, {j.ws, j.ws + L.d, j.ws + L.q_d, j.ws + L.r_d, j.ws + L.s}));
  }
  if (m0.prec == PAT_F64) {
    if (V >= 2) return multi_t<double, 2, false>(jobs, n_iter, st);
    return multi_t<double, 1, false>(jobs, n_iter, st);
  }
  if (m0.split) {
    if (V == 8) return multi_t<float, 8, true>(jobs, n_iter, st);
    if (V == 4) return multi_t<float, 4, true>(jobs, n_iter, st);
    if (V == 2) return multi_t<float, 2, true>(jobs, n_iter, st);
    return multi_t<float, 1, true>(jobs, n_iter, st);
  }
  if (V == 4) return multi_t<float, 4, false>(jobs, n_iter, st);
  if (V == 2) return multi_t<float, 2, false>(jobs, n_iter, st);
  return multi_t<float, 1, false>(jobs, n_iter, st);
}

}  // namespace pat
