// Device kernels of the RTO hot path (sm_103a).  Launchers are in pat_kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pat_internal.h"

namespace pat {

// V consecutive samples of one node, moved as one 4/8/16-byte access.
template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
  T v[V];
};

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld(const T* __restrict__ p) {
  return *reinterpret_cast<const Pack<T, V>*>(p);
}
template <typename T, int V>
__device__ __forceinline__ void st(T* __restrict__ p, const Pack<T, V>& x) {
  *reinterpret_cast<Pack<T, V>*>(p) = x;
}

// ---------------------------------------------------------------------------
// Forward step in scaled Stoermer-Verlet variables.
//
// With a^n = p^{n+1/2} and w^n = dt v^n, one step of eq. fully-discrete (M -> M_L)
// is  w^{n+1} = w^n - dt^2 M^{-1} K a^n - dt M^{-1} B w^n,  a^{n+1} = a^n + w^{n+1},
// and the observed pressure p^{n} = a^n - w^n / 2.  a^0 = p0, w^0 = 0.
// Row blocks update all nodes x samples; the trailing blocks gather the
// observation of the *input* state (sensors read p = a - w/2 of three nodes).
// ---------------------------------------------------------------------------
template <typename T>
struct FwdArgs {
  int64_t N;
  int32_t K;
  int32_t n_obs;
  int64_t row_threads;  // N * K / V
  const int32_t* __restrict__ ptr;
  const uint32_t* __restrict__ col;
  const T* __restrict__ hi;
  const float* __restrict__ lo;
  const T* __restrict__ a_in;
  const T* __restrict__ w_in;  // nullptr: w = 0 (first step)
  T* __restrict__ a_out;
  T* __restrict__ w_out;
  const int32_t* __restrict__ det_node;
  const T* __restrict__ det_w;
  T* __restrict__ y_out;  // nullptr: no observation in this launch
  T scale;
};

template <typename T, int V, bool SPLIT>
__global__ void __launch_bounds__(256) fwd_step_kernel(const FwdArgs<T> A) {
  const int KV = A.K / V;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.row_threads) {
    if (A.a_out == nullptr) return;
    const int64_t row = t / KV;
    const int kv = (int)(t - row * KV);
    const int64_t off = row * A.K + (int64_t)kv * V;
    T acc[V], accl[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = accl[q] = T(0);
    const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
    for (int e = e0; e < e1; ++e) {
      const uint32_t c = A.col[e];
      const T* src = (c & kTagB) ? A.w_in : A.a_in;
      if (src == nullptr) continue;
      const Pack<T, V> x = ld<T, V>(src + (int64_t)(c & kIdxMask) * A.K + (int64_t)kv * V);
      const T h = A.hi[e];
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = fma(h, x.v[q], acc[q]);
      if constexpr (SPLIT) {
        const T l = A.lo[e];
#pragma unroll
        for (int q = 0; q < V; ++q) accl[q] = fma(l, x.v[q], accl[q]);
      }
    }
    const Pack<T, V> a = ld<T, V>(A.a_in + off);
    Pack<T, V> w;
    if (A.w_in) {
      w = ld<T, V>(A.w_in + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) w.v[q] = T(0);
    }
    Pack<T, V> an, wn;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      wn.v[q] = w.v[q] - (acc[q] + accl[q]);
      an.v[q] = a.v[q] + wn.v[q];
    }
    st<T, V>(A.w_out + off, wn);
    st<T, V>(A.a_out + off, an);
    return;
  }
  if (A.y_out == nullptr) return;
  const int64_t g = t - A.row_threads;
  if (g >= (int64_t)A.n_obs * KV) return;
  const int d = (int)(g / KV);
  const int kv = (int)(g - (int64_t)d * KV);
  T acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = T(0);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int64_t node = A.det_node[3 * d + s];
    const T wt = A.det_w[3 * d + s];
    const Pack<T, V> a = ld<T, V>(A.a_in + node * A.K + (int64_t)kv * V);
    if (A.w_in) {
      const Pack<T, V> w = ld<T, V>(A.w_in + node * A.K + (int64_t)kv * V);
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = fma(wt, a.v[q] - T(0.5) * w.v[q], acc[q]);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = fma(wt, a.v[q], acc[q]);
    }
  }
  Pack<T, V> y;
#pragma unroll
  for (int q = 0; q < V; ++q) y.v[q] = A.scale * acc[q];
  st<T, V>(A.y_out + (int64_t)d * A.K + (int64_t)kv * V, y);
}

// ---------------------------------------------------------------------------
// Transposed step (Section 5.1, eq. adjoint-verlet, in the scaled variables).
//
// The forward step maps (a, w) -> (a + w', w') with w' = w - Kt a - Bt w,
// Kt = dt^2 M^{-1} K, Bt = dt M^{-1} B.  Carrying the cotangent as (ah, u) with
// u = M^{-1}(what + ah), one transposed step is
//     ah' = ah - dt^2 K u,      u' = u - dt M^{-1} B u + M^{-1} ah'
// (K, B symmetric), and the sensor injection of the next (earlier) time adds
// Pi^T yhat to ah' and M^{-1} Pi^T yhat / 2 to u'.  ah = G^T yhat at the end.
// Null inputs stand for a zero state (the first launch only injects).
// ---------------------------------------------------------------------------
template <typename T>
struct AdjArgs {
  int64_t N;
  int32_t K;
  int64_t row_threads;
  const int32_t* __restrict__ ptr;
  const uint32_t* __restrict__ col;
  const T* __restrict__ hi;
  const float* __restrict__ lo;
  const T* __restrict__ minv_hi;
  const float* __restrict__ minv_lo;
  const T* __restrict__ ah_in;
  const T* __restrict__ u_in;
  T* __restrict__ ah_out;
  T* __restrict__ u_out;
  const T* __restrict__ yhat;  // [n_obs][K] of the injected time, or nullptr
  T inj_scale;
};

template <typename T, int V, bool SPLIT>
__global__ void __launch_bounds__(256) adj_step_kernel(const AdjArgs<T> A) {
  const int KV = A.K / V;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.row_threads) return;
  const int64_t row = t / KV;
  const int kv = (int)(t - row * KV);
  const int64_t off = row * A.K + (int64_t)kv * V;
  T ak[V], akl[V], bq[V], bql[V], inj[V];
#pragma unroll
  for (int q = 0; q < V; ++q) ak[q] = akl[q] = bq[q] = bql[q] = inj[q] = T(0);
  const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
  for (int e = e0; e < e1; ++e) {
    const uint32_t c = A.col[e];
    const int64_t j = (int64_t)(c & kIdxMask);
    const T h = A.hi[e];
    if (c & kTagInj) {
      if (A.yhat) {
        const Pack<T, V> y = ld<T, V>(A.yhat + j * A.K + (int64_t)kv * V);
#pragma unroll
        for (int q = 0; q < V; ++q) inj[q] = fma(h, y.v[q], inj[q]);
      }
      continue;
    }
    if (A.u_in == nullptr) continue;
    const Pack<T, V> x = ld<T, V>(A.u_in + j * A.K + (int64_t)kv * V);
    if (c & kTagB) {
#pragma unroll
      for (int q = 0; q < V; ++q) bq[q] = fma(h, x.v[q], bq[q]);
      if constexpr (SPLIT) {
        const T l = A.lo[e];
#pragma unroll
        for (int q = 0; q < V; ++q) bql[q] = fma(l, x.v[q], bql[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) ak[q] = fma(h, x.v[q], ak[q]);
      if constexpr (SPLIT) {
        const T l = A.lo[e];
#pragma unroll
        for (int q = 0; q < V; ++q) akl[q] = fma(l, x.v[q], akl[q]);
      }
    }
  }
  Pack<T, V> ah, u;
  if (A.ah_in) {
    ah = ld<T, V>(A.ah_in + off);
    u = ld<T, V>(A.u_in + off);
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) ah.v[q] = u.v[q] = T(0);
  }
  const T mh = A.minv_hi[row];
  T ml = T(0);
  if constexpr (SPLIT) ml = A.minv_lo[row];
  Pack<T, V> ahn, un;
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const T an = ah.v[q] - (ak[q] + akl[q]);
    const T I = A.inj_scale * inj[q];
    const T z = an + T(0.5) * I;  // M^{-1} multiplies ah' (before injection) + I/2
    un.v[q] = u.v[q] - (bq[q] + bql[q]) + (mh * z + ml * z);
    ahn.v[q] = an + I;
  }
  st<T, V>(A.ah_out + off, ahn);
  st<T, V>(A.u_out + off, un);
}

}  // namespace pat

namespace pat {

// ---------------------------------------------------------------------------
// Three-level form of the same propagator (12 bytes per node and sample).
//
// With x_s = a_s = p^{s+1/2} the scaled Stoermer-Verlet step of fwd_step_kernel
// reads, after eliminating w_s = x_s - x_{s-1},
//     x_{s+1} = x_s + w_s - Kt x_s - Bt w_s,   Kt = dt^2 M^{-1} K,  Bt = dt M^{-1} B,
// and the observation is p^s = x_s - w_s/2 = (x_s + x_{s-1}) / 2.  Forward start:
// x_0 = p0, x_{-1} = x_0 (v^0 = 0).
//
// The transposed step of Section 5.1 has the same three-level form in the
// variable u = M^{-1}(what + ah) (K, B symmetric):
//     u_{m-1} = u_m + w - Kt u_m - Bt w + M^{-1}(I_m + I_{m-1}) / 2,   w = u_m - u_{m+1},
// where I_m = Pi^T yhat^m; it starts from u_{N_T+1} = 0, u_{N_T} = M^{-1} I_{N_T} / 2
// and ends with G^T yhat = M (u_1 - u_2) + M Bt u_2 (adj3_finish_kernel).
// The difference x_s - x_{s-1} of two consecutive FP32 states is exact whenever
// they are within a factor of two (Sterbenz), so nothing is lost against
// carrying w.
// ---------------------------------------------------------------------------
template <typename T>
struct Step3Args {
  int64_t N;
  int32_t K;
  int32_t n_obs;
  int64_t row_threads;
  int32_t prev_mode;  // 0: xp is a buffer; 1: xp equals x (zero velocity); 2: xp is zero
  const int32_t* __restrict__ ptr;
  const uint32_t* __restrict__ col;
  const T* __restrict__ hi;
  const float* __restrict__ lo;
  const T* __restrict__ x;   // nullptr: zero state (adjoint start)
  const T* __restrict__ xp;
  T* __restrict__ xn;
  // adjoint source: kTagInj entries carry w_d / (2 M_i) and read ya + yb
  const T* __restrict__ ya;
  const T* __restrict__ yb;
  T inj_scale;
  // forward observation of the current state, scale * Pi (x + xp) / 2
  const int32_t* __restrict__ det_node;
  const T* __restrict__ det_w;
  T* __restrict__ y_out;
  T scale;
};

// Rows are walked in chunks of CH entries: the chunk's columns and
// coefficients are loaded first, then all CH neighbour vectors, then the FMAs,
// so each thread keeps CH independent 16-byte loads in flight instead of one
// dependent index->value chain per entry.
constexpr int kChunk = 8;

template <typename T, int V, bool SPLIT, bool ADJ>
__device__ __forceinline__ void step3_body(const Step3Args<T>& A, const int64_t t) {
  const int KV = A.K / V;
  if (t < A.row_threads) {
    const int64_t row = t / KV;
    const int kv = (int)(t - row * KV);
    const int64_t off = row * A.K + (int64_t)kv * V;
    T acc[V], accl[V], src[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = accl[q] = src[q] = T(0);
    const bool have_x = A.x != nullptr;
    const bool xp_buf = A.prev_mode == 0;
    const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
    if (have_x) {
      for (int e = e0; e < e1; e += kChunk) {
        uint32_t c[kChunk];
        T h[kChunk];
        float l[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
          const bool in = e + q < e1;
          c[q] = in ? A.col[e + q] : kTagInj;
          h[q] = in ? A.hi[e + q] : T(0);
          if constexpr (SPLIT) l[q] = in ? A.lo[e + q] : 0.0f;
        }
        Pack<T, V> xv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
          if (!(c[q] & kTagInj)) {
            xv[q] = ld<T, V>(A.x + (int64_t)(c[q] & kIdxMask) * A.K + (int64_t)kv * V);
          } else {
#pragma unroll
            for (int r = 0; r < V; ++r) xv[q].v[r] = T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
          if ((c[q] & (kTagB | kTagInj)) == kTagB) {
            // the boundary term acts on w_j = x_j - xp_j
            if (xp_buf) {
              const Pack<T, V> pj = ld<T, V>(A.xp + (int64_t)(c[q] & kIdxMask) * A.K + (int64_t)kv * V);
#pragma unroll
              for (int r = 0; r < V; ++r) xv[q].v[r] -= pj.v[r];
            } else if (A.prev_mode == 1) {
#pragma unroll
              for (int r = 0; r < V; ++r) xv[q].v[r] = T(0);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
#pragma unroll
          for (int r = 0; r < V; ++r) acc[r] = fma(h[q], xv[q].v[r], acc[r]);
          if constexpr (SPLIT) {
#pragma unroll
            for (int r = 0; r < V; ++r) accl[r] = fma((T)l[q], xv[q].v[r], accl[r]);
          }
        }
      }
    }
    if constexpr (ADJ) {
      // sensor entries sit at the end of the row
      for (int e = e1 - 1; e >= e0; --e) {
        const uint32_t c = A.col[e];
        if (!(c & kTagInj)) break;
        const int64_t j = (int64_t)(c & kIdxMask);
        const T h = A.hi[e];
        Pack<T, V> ys;
#pragma unroll
        for (int q = 0; q < V; ++q) ys.v[q] = T(0);
        if (A.ya) {
          const Pack<T, V> y = ld<T, V>(A.ya + j * A.K + (int64_t)kv * V);
#pragma unroll
          for (int q = 0; q < V; ++q) ys.v[q] += y.v[q];
        }
        if (A.yb) {
          const Pack<T, V> y = ld<T, V>(A.yb + j * A.K + (int64_t)kv * V);
#pragma unroll
          for (int q = 0; q < V; ++q) ys.v[q] += y.v[q];
        }
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fma(h, ys.v[q], src[q]);
      }
    }
    Pack<T, V> xi, xpi, xo;
    if (have_x) {
      xi = ld<T, V>(A.x + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) xi.v[q] = T(0);
    }
    if (xp_buf) {
      xpi = ld<T, V>(A.xp + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) xpi.v[q] = (A.prev_mode == 1) ? xi.v[q] : T(0);
    }
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const T w = xi.v[q] - xpi.v[q];
      const T wn = w - (acc[q] + accl[q]) + A.inj_scale * src[q];
      xo.v[q] = xi.v[q] + wn;
    }
    st<T, V>(A.xn + off, xo);
    return;
  }
  if (A.y_out == nullptr) return;
  const int64_t g = t - A.row_threads;
  if (g >= (int64_t)A.n_obs * KV) return;
  const int d = (int)(g / KV);
  const int kv = (int)(g - (int64_t)d * KV);
  T acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = T(0);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int64_t node = A.det_node[3 * d + s];
    const T wt = A.det_w[3 * d + s];
    const Pack<T, V> a = ld<T, V>(A.x + node * A.K + (int64_t)kv * V);
    if (A.prev_mode == 0) {
      const Pack<T, V> b = ld<T, V>(A.xp + node * A.K + (int64_t)kv * V);
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = fma(wt, T(0.5) * (a.v[q] + b.v[q]), acc[q]);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] = fma(wt, a.v[q], acc[q]);
    }
  }
  Pack<T, V> y;
#pragma unroll
  for (int q = 0; q < V; ++q) y.v[q] = A.scale * acc[q];
  st<T, V>(A.y_out + (int64_t)d * A.K + (int64_t)kv * V, y);
}

template <typename T, int V, bool SPLIT, bool ADJ>
__global__ void __launch_bounds__(256) step3_kernel(const Step3Args<T> A) {
  step3_body<T, V, SPLIT, ADJ>(A, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Several meshes advanced by one launch: block b belongs to the group member g
// with block_off[g] <= b < block_off[g+1] (uneven batches of meshes and K).
constexpr int kMaxGroup = 8;
template <typename T>
struct Step3Group {
  int32_t n;
  int64_t block_off[kMaxGroup + 1];
  Step3Args<T> a[kMaxGroup];
};

template <typename T, int V, bool SPLIT, bool ADJ>
__global__ void __launch_bounds__(256) step3_group_kernel(const __grid_constant__ Step3Group<T> G) {
  int g = 0;
  while (g + 1 < G.n && (int64_t)blockIdx.x >= G.block_off[g + 1]) ++g;
  const int64_t t = ((int64_t)blockIdx.x - G.block_off[g]) * blockDim.x + threadIdx.x;
  step3_body<T, V, SPLIT, ADJ>(G.a[g], t);
}

// G^T yhat = M (u_1 - u_2) + M Bt u_2 from the last two transposed states
// (B entries of the forward rows carry Bt = dt B_ij / M_i).
template <typename T, int V, bool SPLIT>
__global__ void __launch_bounds__(256) adj3_finish_kernel(int64_t row_threads, int K, const int32_t* __restrict__ ptr,
                                                          const uint32_t* __restrict__ col, const T* __restrict__ hi,
                                                          const float* __restrict__ lo, const double* __restrict__ ml,
                                                          const T* __restrict__ u1, const T* __restrict__ u2,
                                                          T* __restrict__ out) {
  const int KV = K / V;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= row_threads) return;
  const int64_t row = t / KV;
  const int kv = (int)(t - row * KV);
  const int64_t off = row * K + (int64_t)kv * V;
  T acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = T(0);
  for (int e = ptr[row]; e < ptr[row + 1]; ++e) {
    const uint32_t c = col[e];
    if (!(c & kTagB)) continue;
    const Pack<T, V> x = ld<T, V>(u2 + (int64_t)(c & kIdxMask) * K + (int64_t)kv * V);
    T h = hi[e];
    if constexpr (SPLIT) h += (T)lo[e];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = fma(h, x.v[q], acc[q]);
  }
  const Pack<T, V> a = ld<T, V>(u1 + off), b = ld<T, V>(u2 + off);
  const T m = (T)ml[row];
  Pack<T, V> o;
#pragma unroll
  for (int q = 0; q < V; ++q) o.v[q] = m * ((a.v[q] - b.v[q]) + acc[q]);
  st<T, V>(out + off, o);
}

}  // namespace pat
