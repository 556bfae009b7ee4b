// Gradient of a data misfit with respect to the per-element squared sound
// speed, by the discrete adjoint with checkpointed recomputation of the
// forward trajectory.
//
// With K(theta) = sum_e theta_e K_e^0 the step x_{s+1} = x_s + w_s - Kt x_s - Bt w_s
// (Kt = dt^2 M^{-1} K) depends on theta only through Kt x_s.  The cotangent
// of x_{s+1}, pulled back through that term, is the transposed variable u
// of the three-level transposed recursion (the same u as in
// eq. adjoint-verlet's M qhat = vhat, scaled by dt), so
//     dL/dtheta_e = -dt^2 sum_{m=1}^{N_T} u_m|_e^T K_e^0 x_{m-1}|_e,
// summed over the K stacked samples.  The forward states x_0..x_{N_T-1} are
// needed in reverse order; every L-th pair (x_s, x_{s-1}) is kept
// (L = ceil(sqrt(N_T))) and each segment is recomputed before its reverse sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "pat_kernels.cuh"
#include "pat_solver.cuh"

namespace pat {

// One checkpoint segment's element passes, all at once:
//   g[e] += scale * sum_{q < nq} sum_k u_{s0+1+q}[t_a, k] K0_ab x_{s0+q}[t_b, k]
// (FP64 accumulation per element).  x_{s0+q} = xseg + q NK; u_m sits in slot
// m % R of the ring urings (R slots of NK).  Each element's coefficients are
// read and its g updated once per segment instead of once per step.
template <typename T>
__global__ void __launch_bounds__(256) grad_c2_seg_kernel(int64_t E, int K, int64_t NK, const int32_t* __restrict__ tets,
                                                          const T* __restrict__ k0, const T* __restrict__ uring,
                                                          int R, int s0, const T* __restrict__ xseg, int nq,
                                                          double scale, double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int4 t = *reinterpret_cast<const int4*>(tets + 4 * e);
  const int64_t n[4] = {(int64_t)t.x * K, (int64_t)t.y * K, (int64_t)t.z * K, (int64_t)t.w * K};
  T km[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) km[q] = k0[10 * e + q];
  // symmetric 4x4 from the upper triangle (00 01 02 03 11 12 13 22 23 33)
  const T Km[4][4] = {{km[0], km[1], km[2], km[3]},
                      {km[1], km[4], km[5], km[6]},
                      {km[2], km[5], km[7], km[8]},
                      {km[3], km[6], km[8], km[9]}};
  double acc = 0.0;
  for (int q = nq - 1; q >= 0; --q) {
    const T* u = uring + (int64_t)((s0 + 1 + q) % R) * NK;
    const T* x = xseg + (int64_t)q * NK;
    for (int k = 0; k < K; ++k) {
      T uu[4], xx[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uu[a] = u[n[a] + k];
        xx[a] = x[n[a] + k];
      }
      T s = T(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T r = T(0);
#pragma unroll
        for (int b = 0; b < 4; ++b) r = fma(Km[a][b], xx[b], r);
        s = fma(uu[a], r, s);
      }
      acc += (double)s;
    }
  }
  g[e] += scale * acc;
}

// Workspace: checkpoints (x_{jL}, x_{jL-1}) of every segment, the segment's
// recomputed states x_{s0} .. x_{s0+L-1}, the ring of transposed states
// (L + 2 slots: a segment's passes need u_{s0+1} .. u_{s1}, its steps also
// u_{s0} and u_{s1+1}), four state buffers (the first sweep's rotation, then
// the transposed launches' chunk counters and sensor terms in the fourth),
// the segment recomputation's two chunk counters, and g.
struct GradLayout {
  size_t ck, seg, ring, rot, ctr, g, total;
  int L, n_ck, R;
};

static inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

GradLayout grad_layout(const DeviceMesh& m, int K) {
  GradLayout G{};
  const size_t rs = m.prec == PAT_F64 ? 8 : 4;
  const size_t NK = (size_t)m.N * K;
  G.L = (int)std::ceil(std::sqrt((double)m.n_steps));
  G.n_ck = (m.n_steps + G.L - 1) / G.L;
  G.R = G.L + 2;
  size_t o = 0;
  G.ck = o; o = al256(o + (size_t)G.n_ck * 2 * NK * rs);
  G.seg = o; o = al256(o + (size_t)G.L * NK * rs);
  G.ring = o; o = al256(o + (size_t)G.R * NK * rs);
  G.rot = o; o = al256(o + 4 * NK * rs);
  G.ctr = o; o = al256(o + 2 * sizeof(unsigned int));
  G.g = o; o = al256(o + (size_t)m.E * 8);
  G.total = o;
  return G;
}

// One step launch: the mesh's tuned variant (three-level form), else the
// generic three-level kernel with one sample per thread.
template <typename T>
static void launch_one(const DeviceMesh& m, bool adj, int V, Step3Args<T> A, int64_t threads, cudaStream_t st) {
  if (m.three_level) {
    step_tuned<T>(m, adj, V, A, threads, st);
    return;
  }
  A.stage_cap = 0;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  // split (hi, lo) coefficients exist for FP32 meshes only
  if (sizeof(T) == 4 && m.split) {
    if (adj)
      step3_kernel<T, 1, sizeof(T) == 4, true, false><<<blocks, 256, 0, st>>>(A);
    else
      step3_kernel<T, 1, sizeof(T) == 4, false, false><<<blocks, 256, 0, st>>>(A);
  } else {
    if (adj)
      step3_kernel<T, 1, false, true, false><<<blocks, 256, 0, st>>>(A);
    else
      step3_kernel<T, 1, false, false, false><<<blocks, 256, 0, st>>>(A);
  }
}

template <typename T, int V, bool SPLIT>
static void finish_as(const DeviceMesh& m, int K, const T* u_last, const T* u_prev, T* out, cudaStream_t st) {
  const int64_t rt = m.N * (int64_t)K / V;
  adj3_finish_kernel<T, V, SPLIT><<<(unsigned)((rt + 255) / 256), 256, 0, st>>>(
      rt, K, m.fwd.ptr, m.fwd.col, static_cast<const T*>(m.fwd.hi), m.fwd.lo, m.ml, u_last, u_prev, out);
}

template <typename T>
static void finish(const DeviceMesh& m, int V, int K, const T* u_last, const T* u_prev, T* out, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (m.split) {
      if (V == 8) return finish_as<T, 8, true>(m, K, u_last, u_prev, out, st);
      if (V == 4) return finish_as<T, 4, true>(m, K, u_last, u_prev, out, st);
      if (V == 2) return finish_as<T, 2, true>(m, K, u_last, u_prev, out, st);
      return finish_as<T, 1, true>(m, K, u_last, u_prev, out, st);
    }
    if (V == 8) return finish_as<T, 8, false>(m, K, u_last, u_prev, out, st);
    if (V == 4) return finish_as<T, 4, false>(m, K, u_last, u_prev, out, st);
    if (V == 2) return finish_as<T, 2, false>(m, K, u_last, u_prev, out, st);
    return finish_as<T, 1, false>(m, K, u_last, u_prev, out, st);
  } else {
    if (V == 2) return finish_as<T, 2, false>(m, K, u_last, u_prev, out, st);
    return finish_as<T, 1, false>(m, K, u_last, u_prev, out, st);
  }
}

// Every launch of one gradient evaluation on stream st.  Vf / Va: samples per
// thread of the forward / transposed step launches.
template <typename T>
static pat_status grad_body(const DeviceMesh& m, const T* p0, const T* Yhat, int K, double* g_out, T* p0_grad,
                            char* ws, int Vf, int Va, cudaStream_t st) {
  const GradLayout G = grad_layout(m, K);
  const int64_t NK = m.N * (int64_t)K;
  const size_t fb = (size_t)NK * sizeof(T);
  T* ck = (T*)(ws + G.ck);
  T* seg = (T*)(ws + G.seg);
  T* ring = (T*)(ws + G.ring);
  T* const b[3] = {(T*)(ws + G.rot), (T*)(ws + G.rot) + NK, (T*)(ws + G.rot) + 2 * NK};
  unsigned int* fctr = (unsigned int*)(ws + G.ctr);
  double* g = (double*)(ws + G.g);
  const int NT = m.n_steps, L = G.L, R = G.R;
  auto slot = [&](int mstep) { return ring + (int64_t)(mstep % R) * NK; };
  PAT_TRY(cuda_check(cudaMemsetAsync(g, 0, (size_t)m.E * 8, st), "grad memset"));
  PAT_TRY(cuda_check(cudaMemsetAsync(fctr, 0, 2 * sizeof(unsigned int), st), "grad counters"));
  PAT_TRY(cuda_check(cudaMemsetAsync(b[2] + NK, 0, 2 * sizeof(unsigned int), st), "grad counters"));
  // 1. forward sweep (launch i: x_{i+1} into b[i % 3]) keeping (x_{jL}, x_{jL-1}), x_{-1} = x_0
  {
    PAT_RANGE("gradient: forward sweep");
    for (int i = 0; i < NT; ++i) {
      if (i % L == 0) {
        const T* cur = i == 0 ? p0 : b[(i - 1) % 3];
        const T* prev = i <= 1 ? p0 : b[(i - 2) % 3];
        T* c = ck + (size_t)(i / L) * 2 * NK;
        PAT_TRY(cuda_check(cudaMemcpyAsync(c, cur, fb, cudaMemcpyDeviceToDevice, st), "checkpoint"));
        PAT_TRY(cuda_check(cudaMemcpyAsync(c + NK, prev, fb, cudaMemcpyDeviceToDevice, st), "checkpoint"));
      }
      if (i == NT - 1) break;  // x_{N_T} is not needed
      int64_t thr = 0;
      Step3Args<T> A = fwd3_args<T>(m, K, Vf, p0, ck, T(0), b, i, &thr);
      A.y_out = nullptr;  // no observations
      launch_one<T>(m, false, Vf, A, A.row_threads, st);
    }
  }
  // 2. reverse sweep: the transposed launches i = 0 .. N_T of a transposed
  // solve (launch i >= 1 takes u_{m-1} from u_m, u_{m+1}, m = N_T - i + 1),
  // their states in the ring; each segment's forward states recomputed first
  // and its element passes run once its u's exist
  PAT_TRY(cuda_check(cudaMemsetAsync(b[2] + NK, 0, 2 * sizeof(unsigned int), st), "grad counters"));
  PAT_RANGE("gradient: reverse sweep");
  int64_t thr = 0;
  {
    Step3Args<T> A = adj3_args<T>(m, K, Va, Yhat, T(1), b, 0, &thr);
    A.xn = slot(NT);
    launch_one<T>(m, true, Va, A, thr, st);
  }
  int i = 1, li = 0;
  const int64_t eblocks = (m.E + 255) / 256;
  for (int j = G.n_ck - 1; j >= 0; --j) {
    const int s0 = j * L;
    const int s1 = std::min(NT, s0 + L);  // states x_{s0} .. x_{s1-1} are needed
    const T* c0 = ck + (size_t)j * 2 * NK;
    PAT_TRY(cuda_check(cudaMemcpyAsync(seg, c0, fb, cudaMemcpyDeviceToDevice, st), "segment start"));
    for (int q = 1; q < s1 - s0; ++q) {  // seg[q] = x_{s0+q}
      Step3Args<T> A = fwd3_args<T>(m, K, Vf, p0, ck, T(0), b, 1, &thr);
      A.x = seg + (size_t)(q - 1) * NK;
      const bool first = s0 == 0 && q == 1;  // x_{-1} = x_0
      A.xp = first ? nullptr : (q == 1 ? c0 + NK : seg + (size_t)(q - 2) * NK);
      A.prev_mode = first ? 1 : 0;
      A.xn = seg + (size_t)q * NK;
      A.y_out = nullptr;
      A.dyn_ctr = fctr + (li & 1);
      A.dyn_next = fctr + ((li + 1) & 1);
      ++li;
      launch_one<T>(m, false, Vf, A, A.row_threads, st);
    }
    // transposed launches down to u_{s0}: m = s1 .. s0 + 1
    for (int mstep = s1; mstep > s0; --mstep, ++i) {
      Step3Args<T> A = adj3_args<T>(m, K, Va, Yhat, T(1), b, i, &thr);
      A.x = slot(mstep);
      A.xp = i == 1 ? nullptr : slot(mstep + 1);
      A.xn = slot(mstep - 1);
      launch_one<T>(m, true, Va, A, thr, st);
    }
    // dL/dtheta += -dt^2 sum_{m = s0+1}^{s1} u_m^T K0 x_{m-1}
    grad_c2_seg_kernel<T><<<(unsigned)eblocks, 256, 0, st>>>(m.E, K, NK, m.etets, static_cast<const T*>(m.eK0), ring,
                                                             R, s0, seg, s1 - s0, -m.dt * m.dt, g);
  }
  if (p0_grad) finish<T>(m, Va, K, slot(0), slot(1), p0_grad, st);
  PAT_TRY(cuda_check(cudaMemcpyAsync(g_out, g, (size_t)m.E * 8, cudaMemcpyDeviceToDevice, st), "grad copy"));
  return cuda_check(cudaGetLastError(), "grad launch");
}

// The whole evaluation is captured once per (K, buffers) into a CUDA graph and
// replayed (direct launches when graphs are off or st is being captured).
template <typename T>
static pat_status grad_t(const DeviceMesh& m, const T* p0, const T* Yhat, int K, double* g_out, T* p0_grad,
                         char* ws, cudaStream_t st) {
  const int Vb = vec_width(m, K, {p0, Yhat, p0_grad, ws});
  const int Vf = m.three_level ? std::min(Vb, tuned_vec(m, 0, K)) : 1;
  const int Va = m.three_level ? std::min(Vb, tuned_vec(m, 1, K)) : 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((m.flags & PAT_MESH_NO_GRAPHS) || !m.capture_stream || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return grad_body<T>(m, p0, Yhat, K, g_out, p0_grad, ws, Vf, Va, st);
  }
  const std::array<uintptr_t, 6> key = {(uintptr_t)p0, (uintptr_t)Yhat, (uintptr_t)g_out, (uintptr_t)p0_grad, (uintptr_t)ws,
                       (uintptr_t)K};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    auto it = m.grad_graphs.find(key);
    if (it != m.grad_graphs.end()) exec = (cudaGraphExec_t)it->second;
  }
  if (!exec) {
    cudaStream_t cap = (cudaStream_t)m.capture_stream;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return grad_body<T>(m, p0, Yhat, K, g_out, p0_grad, ws, Vf, Va, st);
    }
    const pat_status s = grad_body<T>(m, p0, Yhat, K, g_out, p0_grad, ws, Vf, Va, cap);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(cap, &gr);
    if (s != PAT_OK || e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      return s != PAT_OK ? s : cuda_check(e, "gradient capture");
    }
    e = cudaGraphInstantiate(&exec, gr, 0);
    cudaGraphDestroy(gr);
    PAT_TRY(cuda_check(e, "gradient graph instantiate"));
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    m.grad_graphs[key] = (void*)exec;
  }
  return cuda_check(cudaGraphLaunch(exec, st), "gradient graph launch");
}

size_t grad_workspace_bytes(const DeviceMesh& m, int K) { return grad_layout(m, K).total; }

pat_status grad_c2(const DeviceMesh& m, const void* p0, const void* Yhat, int K, double* g, void* p0_grad, char* ws,
                   cudaStream_t st) {
  if (m.prec == PAT_F64)
    return grad_t<double>(m, (const double*)p0, (const double*)Yhat, K, g, (double*)p0_grad, ws, st);
  return grad_t<float>(m, (const float*)p0, (const float*)Yhat, K, g, (float*)p0_grad, ws, st);
}

}  // namespace pat
