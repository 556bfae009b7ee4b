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

#include "pat_kernels.cuh"
#include "pat_solver.cuh"

namespace pat {

// g[e] += scale * sum_k u[t_a, k] K0_ab x[t_b, k]   (FP64 accumulation per element)
template <typename T>
__global__ void __launch_bounds__(256) grad_c2_kernel(int64_t E, int K, const int32_t* __restrict__ tets,
                                                      const T* __restrict__ k0, const T* __restrict__ u,
                                                      const T* __restrict__ x, double scale, double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int4 t = *reinterpret_cast<const int4*>(tets + 4 * e);
  const int64_t n[4] = {t.x, t.y, t.z, t.w};
  T km[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) km[q] = k0[10 * e + q];
  // symmetric 4x4 from the upper triangle (00 01 02 03 11 12 13 22 23 33)
  const T Km[4][4] = {{km[0], km[1], km[2], km[3]},
                      {km[1], km[4], km[5], km[6]},
                      {km[2], km[5], km[7], km[8]},
                      {km[3], km[6], km[8], km[9]}};
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    T uu[4], xx[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      uu[a] = u[n[a] * K + k];
      xx[a] = x[n[a] * K + k];
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
  g[e] += scale * acc;
}

struct GradLayout {
  size_t ck, seg, adj, g, total;
  int L, n_ck;
};

static inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

GradLayout grad_layout(const DeviceMesh& m, int K) {
  GradLayout G{};
  const size_t rs = m.prec == PAT_F64 ? 8 : 4;
  const size_t NK = (size_t)m.N * K;
  G.L = (int)std::ceil(std::sqrt((double)m.n_steps));
  G.n_ck = (m.n_steps + G.L - 1) / G.L;
  size_t o = 0;
  G.ck = o; o = al256(o + (size_t)G.n_ck * 2 * NK * rs);
  G.seg = o; o = al256(o + (size_t)std::max(G.L + 1, 3) * NK * rs);  // also the rotation of the first sweep
  G.adj = o; o = al256(o + 3 * NK * rs);
  G.g = o; o = al256(o + (size_t)m.E * 8);
  G.total = o;
  return G;
}

template <typename T, int V, bool SPLIT>
static void step(const DeviceMesh& m, const DevCSR& csr, int K, const T* x, const T* xp, int prev_mode, T* xn,
                 const T* ya, const T* yb, T inj_scale, cudaStream_t st) {
  Step3Args<T> A{};
  A.N = m.N;
  A.K = K;
  A.n_obs = m.n_obs;
  A.row_threads = m.N * (int64_t)K / V;
  A.prev_mode = prev_mode;
  A.ptr = csr.ptr;
  A.col = csr.col;
  A.hi = static_cast<const T*>(csr.hi);
  A.lo = csr.lo;
  A.nb = m.row_nb;
  A.ninj = m.row_ninj;
  A.x = x;
  A.xp = xp;
  A.xn = xn;
  A.ya = ya;
  A.yb = yb;
  A.inj_scale = inj_scale;
  const unsigned blocks = (unsigned)((A.row_threads + 255) / 256);
  A.stage_cap = 0;  // V = 1, K small: one thread per row, no staging
  if (&csr == &m.adj3)
    step3_kernel<T, V, SPLIT, true, false><<<blocks, 256, 0, st>>>(A);
  else
    step3_kernel<T, V, SPLIT, false, false><<<blocks, 256, 0, st>>>(A);
}

template <typename T, int V, bool SPLIT>
static pat_status grad_t(const DeviceMesh& m, const T* p0, const T* Yhat, int K, double* g_out, T* p0_grad,
                         char* ws, cudaStream_t st) {
  const GradLayout G = grad_layout(m, K);
  const int64_t NK = m.N * (int64_t)K;
  const size_t fb = (size_t)NK * sizeof(T);
  T* ck = (T*)(ws + G.ck);
  T* seg = (T*)(ws + G.seg);
  T* ub[3] = {(T*)(ws + G.adj), (T*)(ws + G.adj) + NK, (T*)(ws + G.adj) + 2 * NK};
  double* g = (double*)(ws + G.g);
  const int NT = m.n_steps, L = G.L;
  pat_status s = cuda_check(cudaMemsetAsync(g, 0, (size_t)m.E * 8, st), "grad memset");
  if (s) return s;
  // 1. forward sweep keeping (x_{jL}, x_{jL-1}) for every segment j (x_{-1} = x_0)
  {
    T* rot[3] = {seg, seg + NK, seg + 2 * NK};
    const T* cur = p0;
    const T* prev = p0;
    for (int st_i = 0; st_i < NT; ++st_i) {
      if (st_i % L == 0) {
        T* slot = ck + (size_t)(st_i / L) * 2 * NK;
        cudaMemcpyAsync(slot, cur, fb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(slot + NK, prev, fb, cudaMemcpyDeviceToDevice, st);
      }
      T* out = rot[st_i % 3];
      step<T, V, SPLIT>(m, m.fwd, K, cur, st_i == 0 ? nullptr : prev, st_i == 0 ? 1 : 0, out, nullptr, nullptr,
                        T(0), st);
      prev = cur;
      cur = out;
    }
  }
  // 2. reverse sweep: transposed three-level recursion, segment by segment
  const int64_t ystride = (int64_t)m.n_obs * K;
  // u_{N_T} = M^{-1} I_{N_T} / 2
  step<T, V, SPLIT>(m, m.adj3, K, nullptr, nullptr, 2, ub[0], Yhat + (int64_t)(NT - 1) * ystride, nullptr, T(1),
                    st);
  const T* ucur = ub[0];
  const T* uprev = nullptr;
  int nb = 1;
  const int64_t eblocks = (m.E + 255) / 256;
  for (int j = G.n_ck - 1; j >= 0; --j) {
    const int s0 = j * L;
    const int s1 = std::min(NT, s0 + L);  // states x_{s0} .. x_{s1-1} are needed
    // recompute the segment: seg[i] = x_{s0+i}
    const T* c0 = ck + (size_t)j * 2 * NK;
    cudaMemcpyAsync(seg, c0, fb, cudaMemcpyDeviceToDevice, st);
    for (int i = 1; i < s1 - s0; ++i) {
      const T* xprev = (i == 1) ? c0 + NK : seg + (size_t)(i - 2) * NK;
      step<T, V, SPLIT>(m, m.fwd, K, seg + (size_t)(i - 1) * NK, (s0 == 0 && i == 1) ? nullptr : xprev,
                        (s0 == 0 && i == 1) ? 1 : 0, seg + (size_t)i * NK, nullptr, nullptr, T(0), st);
    }
    for (int mstep = s1; mstep > s0; --mstep) {
      // dL/dtheta += -dt^2 u_m^T K0 x_{m-1}
      grad_c2_kernel<T><<<(unsigned)eblocks, 256, 0, st>>>(m.E, K, m.etets, static_cast<const T*>(m.eK0), ucur,
                                                           seg + (size_t)(mstep - 1 - s0) * NK, -m.dt * m.dt, g);
      T* out = ub[nb % 3];
      step<T, V, SPLIT>(m, m.adj3, K, ucur, uprev, uprev ? 0 : 2, out, Yhat + (int64_t)(mstep - 1) * ystride,
                        mstep >= 2 ? Yhat + (int64_t)(mstep - 2) * ystride : nullptr, T(1), st);
      uprev = ucur;
      ucur = out;
      ++nb;
    }
  }
  if (p0_grad) {
    const int64_t rt = NK / V;
    adj3_finish_kernel<T, V, SPLIT><<<(unsigned)((rt + 255) / 256), 256, 0, st>>>(
        rt, K, m.fwd.ptr, m.fwd.col, static_cast<const T*>(m.fwd.hi), m.fwd.lo, m.ml, ucur, uprev, p0_grad);
  }
  s = cuda_check(cudaMemcpyAsync(g_out, g, (size_t)m.E * 8, cudaMemcpyDeviceToDevice, st), "grad copy");
  if (s) return s;
  return cuda_check(cudaGetLastError(), "grad launch");
}

size_t grad_workspace_bytes(const DeviceMesh& m, int K) { return grad_layout(m, K).total; }

pat_status grad_c2(const DeviceMesh& m, const void* p0, const void* Yhat, int K, double* g, void* p0_grad, char* ws,
                   cudaStream_t st) {
  if (m.prec == PAT_F64) return grad_t<double, 1, false>(m, (const double*)p0, (const double*)Yhat, K, g,
                                                          (double*)p0_grad, ws, st);
  if (m.split)
    return grad_t<float, 1, true>(m, (const float*)p0, (const float*)Yhat, K, g, (float*)p0_grad, ws, st);
  return grad_t<float, 1, false>(m, (const float*)p0, (const float*)Yhat, K, g, (float*)p0_grad, ws, st);
}

}  // namespace pat
