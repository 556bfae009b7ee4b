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
// q = t / KV for the thread-to-row mapping without a 64-bit division (which
// the GPU emulates in software): a shift when KV is a power of two, else a
// 32-bit division while t fits.  Exact for t >= 0, KV >= 1.
__device__ __forceinline__ int64_t div_kv(int64_t t, int KV) {
  if ((KV & (KV - 1)) == 0) return t >> (__ffs(KV) - 1);
  if (t <= 0xffffffffll) return (int64_t)((uint32_t)t / (uint32_t)KV);
  return t / KV;
}

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
    const int64_t row = div_kv(t, KV);
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
  const int d = (int)div_kv(g, KV);
  const int kv = (int)(g - (int64_t)d * KV);
  T acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = T(0);
#pragma unroll
  for (int s = 0; s < kDetPts; ++s) {
    const int64_t node = A.det_node[kDetPts * d + s];
    const T wt = A.det_w[kDetPts * d + s];
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
  const int64_t row = div_kv(t, KV);
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
  int32_t stage_cap;  // shared-memory entries per block (STAGE kernels)
  int64_t pf_rows;    // > 0: prefetch into L2 the streamed data of the rows this many rows ahead
  const float2* __restrict__ hl;     // (hi, lo) pairs of FP32 split coefficients
  const int32_t* __restrict__ order; // processing order of the rows (nullptr: 0, 1, 2, ...)
  // row pairs (pair kernel): union columns and both rows' (hi, lo) pairs per slot
  const uint32_t* __restrict__ pair_col;
  const float4* __restrict__ pair_cf;
  const uint8_t* __restrict__ pair_n;
  // row quads (quad kernel): see DevCSR
  const int32_t* __restrict__ quad_ptr;
  const uint32_t* __restrict__ quad_n;
  const uint32_t* __restrict__ quad_col;
  const float4* __restrict__ quad_cf;
  // fixed-width copy of the rows (ELL kernel)
  const uint32_t* __restrict__ ell_col;
  const float2* __restrict__ ell_hl;
  const uint32_t* __restrict__ ell_desc;
  const int32_t* __restrict__ ovf_ptr;
  const uint32_t* __restrict__ ovf_col;
  const float2* __restrict__ ovf_hl;
  const uint8_t* __restrict__ nb;    // [N] boundary entries per row
  const uint8_t* __restrict__ ninj;  // [N] sensor entries per row (adjoint rows)
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
  // bounded waits of the kernels that stage rows by bulk copies: the status
  // word that gets PAT_ETIMEOUT and the SM cycles a warp waits before it gives up
  int32_t* status;
  long long wait_cycles;
  // dynamic chunk hand-out (persistent kernels): this launch's chunk counter
  // and the next launch's, which this launch zeroes (both in the unused
  // fourth state buffer of the three-level form)
  unsigned int* dyn_ctr;
  unsigned int* dyn_next;
  // transposed 16-slot kernels: the sensor rows' terms sum_e c_e (ya + yb)[col_e]
  // of this launch, prepared by the previous launch (inj_cur; null: computed
  // in the row), and the next launch's, which this launch's extra threads
  // prepare from that launch's data slices ya_next, yb_next (inj_next; null:
  // none); a row's term at its first overflow entry, [overflow entries][K],
  // in the fourth state buffer
  const T* __restrict__ inj_cur;
  T* __restrict__ inj_next;
  const T* __restrict__ ya_next;
  const T* __restrict__ yb_next;
  const int32_t* __restrict__ inj_rows;
  int64_t n_inj;
};

// Row metadata staging.  With STAGE, the block first copies the column /
// coefficient entries of all rows it covers (a contiguous CSR range) into
// shared memory with coalesced loads, so the K/V threads of a row read them
// from shared memory instead of each issuing its own global loads.  The host
// guarantees that the staged range fits A.stage_cap entries.
//
// Every row lists its stiffness entries, then its boundary entries (count
// nb[row]), then (adjoint rows) its sensor entries (count ninj[row]).  All
// stiffness and boundary entries multiply x_j; the boundary entries, which act
// on w_j = x_j - xp_j, then get the xp_j part subtracted in a short second
// loop over the boundary rows only.  The main loop has no per-entry branches.
template <typename T, bool SPLIT>
struct CoefT;
template <>
struct CoefT<float, true> {
  using type = float2;
};
template <>
struct CoefT<float, false> {
  using type = float;
};
template <>
struct CoefT<double, false> {
  using type = double;
};

template <typename T, bool SPLIT>
__device__ __forceinline__ typename CoefT<T, SPLIT>::type coef_ld(const T* hi, const float* lo, int64_t e) {
  if constexpr (SPLIT) {
    return make_float2(hi[e], lo[e]);
  } else {
    return hi[e];
  }
}

template <typename T, int V, bool SPLIT>
__device__ __forceinline__ void coef_fma(const typename CoefT<T, SPLIT>::type c, const Pack<T, V>& x, T (&acc)[V],
                                         T (&accl)[V]) {
  if constexpr (SPLIT) {
#pragma unroll
    for (int r = 0; r < V; ++r) {
      acc[r] = fma(c.x, x.v[r], acc[r]);
      accl[r] = fma(c.y, x.v[r], accl[r]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < V; ++r) acc[r] = fma(c, x.v[r], acc[r]);
  }
}

template <typename T, int V, bool SPLIT, bool ADJ, bool STAGE>
__device__ __forceinline__ void step3_body(const Step3Args<T>& A, const int64_t tb0, unsigned char* smem) {
  using C = typename CoefT<T, SPLIT>::type;
  const int KV = A.K / V;
  const int64_t t = tb0 + threadIdx.x;
  const uint32_t* mcol = A.col;
  const C* mval = nullptr;  // staged coefficients
  int64_t base = 0;
  if constexpr (STAGE) {
    if (tb0 < A.row_threads) {  // uniform over the block
      C* s_val = reinterpret_cast<C*>(smem);
      uint32_t* s_col = reinterpret_cast<uint32_t*>(smem + ((size_t)A.stage_cap * sizeof(C) + 15) / 16 * 16);
      const int64_t r0 = div_kv(tb0, KV);
      const int64_t tl = (tb0 + (int64_t)blockDim.x < A.row_threads ? tb0 + (int64_t)blockDim.x : A.row_threads) - 1;
      const int64_t r1 = div_kv(tl, KV);
      base = A.ptr[r0];
      const int n = (int)(A.ptr[r1 + 1] - base);
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
        s_col[q] = A.col[base + q];
        s_val[q] = coef_ld<T, SPLIT>(A.hi, A.lo, base + q);
      }
      __syncthreads();
      mcol = s_col;
      mval = s_val;
    }
  }
  if (t < A.row_threads) {
    const int64_t row = div_kv(t, KV);
    const int kv = (int)(t - row * KV);
    const int64_t off = row * A.K + (int64_t)kv * V;
    T acc[V], accl[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = accl[q] = T(0);
    const int e0 = (int)(A.ptr[row] - base), e1 = (int)(A.ptr[row + 1] - base);
    const int ni = ADJ ? (int)A.ninj[row] : 0;
    const int eA = e1 - ni;             // end of the stiffness + boundary entries
    const int eB = eA - (int)A.nb[row];  // first boundary entry
    const uint32_t Ku = (uint32_t)A.K;
    auto coef = [&](int e) -> C {
      if constexpr (STAGE) {
        return mval[e];
      } else {
        return coef_ld<T, SPLIT>(A.hi, A.lo, e);
      }
    };
    if (A.x) {
      const T* xk = A.x + (int64_t)kv * V;
#pragma unroll 4
      for (int e = e0; e < eA; ++e) {
        const uint32_t j = mcol[e] & kIdxMask;
        const Pack<T, V> xj = ld<T, V>(xk + (size_t)j * Ku);
        coef_fma<T, V, SPLIT>(coef(e), xj, acc, accl);
      }
      if (eB < eA && A.prev_mode != 2) {
        // boundary entries act on w_j = x_j - xp_j: remove their xp_j part
        // (same accumulation order as the packed kernel, so variants agree bitwise)
        const T* pk = (A.prev_mode == 0 ? A.xp : A.x) + (int64_t)kv * V;
        for (int e = eB; e < eA; ++e) {
          const uint32_t j = mcol[e] & kIdxMask;
          const Pack<T, V> pj = ld<T, V>(pk + (size_t)j * Ku);
          Pack<T, V> neg;
#pragma unroll
          for (int q = 0; q < V; ++q) neg.v[q] = -pj.v[q];
          coef_fma<T, V, SPLIT>(coef(e), neg, acc, accl);
        }
      }
    }
    T src[V];
#pragma unroll
    for (int q = 0; q < V; ++q) src[q] = T(0);
    if constexpr (ADJ) {
      for (int e = eA; e < e1; ++e) {
        const uint32_t j = mcol[e] & kIdxMask;
        T h;
        if constexpr (STAGE) {
          if constexpr (SPLIT) {
            h = mval[e].x;
          } else {
            h = mval[e];
          }
        } else {
          h = A.hi[e];
        }
        // same accumulation order as the packed kernels (variants agree bitwise)
        if (A.ya) {
          const Pack<T, V> y = ld<T, V>(A.ya + (int64_t)j * A.K + (int64_t)kv * V);
#pragma unroll
          for (int q = 0; q < V; ++q) src[q] = fma(h, y.v[q], src[q]);
        }
        if (A.yb) {
          const Pack<T, V> y = ld<T, V>(A.yb + (int64_t)j * A.K + (int64_t)kv * V);
#pragma unroll
          for (int q = 0; q < V; ++q) src[q] = fma(h, y.v[q], src[q]);
        }
      }
    }
    Pack<T, V> xi, xpi, xo;
    if (A.x) {
      xi = ld<T, V>(A.x + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) xi.v[q] = T(0);
    }
    if (A.prev_mode == 0) {
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
  const int d = (int)div_kv(g, KV);
  const int kv = (int)(g - (int64_t)d * KV);
  T acc[V];
#pragma unroll
  for (int q = 0; q < V; ++q) acc[q] = T(0);
#pragma unroll
  for (int s = 0; s < kDetPts; ++s) {
    const int64_t node = A.det_node[kDetPts * d + s];
    const T wt = A.det_w[kDetPts * d + s];
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

// bytes of dynamic shared memory for stage_cap entries
template <typename T, bool SPLIT>
__host__ __device__ constexpr size_t stage_bytes(int cap) {
  return ((size_t)cap * (SPLIT ? 8 : sizeof(T)) + 15) / 16 * 16 + (size_t)cap * 4;
}

template <typename T, int V, bool SPLIT, bool ADJ, bool STAGE>
__global__ void __launch_bounds__(256) step3_kernel(const Step3Args<T> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  step3_body<T, V, SPLIT, ADJ, STAGE>(A, (int64_t)blockIdx.x * blockDim.x, smem);
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

template <typename T, int V, bool SPLIT, bool ADJ, bool STAGE>
__global__ void __launch_bounds__(256) step3_group_kernel(const __grid_constant__ Step3Group<T> G) {
  extern __shared__ __align__(16) unsigned char smem[];
  int g = 0;
  while (g + 1 < G.n && (int64_t)blockIdx.x >= G.block_off[g + 1]) ++g;
  step3_body<T, V, SPLIT, ADJ, STAGE>(G.a[g], ((int64_t)blockIdx.x - G.block_off[g]) * blockDim.x, smem);
}

// ---------------------------------------------------------------------------
// Packed fast path of the three-level step for FP32 fields with hi+lo
// coefficients: V = 4 or 8 samples per thread held as float pairs, every
// product-accumulate a packed fma.rn.f32x2 (two samples per instruction), the
// row walked in predicated chunks so that a row's neighbour loads are issued
// together, the (hi, lo) coefficient pair read as one 8-byte load.
// ---------------------------------------------------------------------------
// Counter-based N(0,1) draws (SplitMix64, Steele, Lea and Flood 2014, and the
// Box-Muller cosine branch): the draw keyed by (seed, stream, sample k,
// element e) uses outputs 2c+1 and 2c+2 of SplitMix64 seeded with `seed`,
// c = ((k << 1 | stream) << 40) | e, as the uniforms u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t i) {
  uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double normal_draw(uint64_t seed, int stream, uint64_t k, uint64_t e) {
  const uint64_t c = (((k << 1) | (uint64_t)stream) << 40) | e;
  const uint64_t h1 = splitmix_out(seed, 2 * c + 1);
  const uint64_t h2 = splitmix_out(seed, 2 * c + 2);
  const double u1 = ((double)(h1 >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(h2 >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}


typedef unsigned long long u64;

__device__ __forceinline__ u64 dup2(float c) {
  u64 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(c));
  return r;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float2 unpack2(u64 v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}
template <int P>
__device__ __forceinline__ void ld_pairs(const float* p, u64 (&out)[P]) {
  if constexpr (P == 2) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    out[0] = v.x;
    out[1] = v.y;
  } else {
    const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(p + 4);
    out[0] = v0.x;
    out[1] = v0.y;
    out[2] = v1.x;
    out[3] = v1.y;
  }
}

// Bulk prefetch into L2 (a hint: no data reaches the SM).  Both the address and
// the size are rounded to the 16-byte granularity the instruction requires.
__device__ __forceinline__ void l2_prefetch(const void* p, int64_t bytes) {
  const uintptr_t a = (uintptr_t)p, a16 = (a + 15) & ~(uintptr_t)15;
  bytes -= (int64_t)(a16 - a);
  if (bytes < 16) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a16), "r"((uint32_t)(bytes & ~(int64_t)15))
               : "memory");
}

// Called by one thread: prefetch into L2 the data that the rows [r0, r1) will
// stream (their own state rows x_s and x_{s-1} and their row metadata), so that
// the threads which take those rows later find them in L2 instead of waiting
// on DRAM.  Rows in natural order only.
template <bool ELL>
__device__ __noinline__ void prefetch_ahead(const Step3Args<float>& A, int64_t r0, int64_t r1) {
  r1 = min(r1, A.N);
  if (r0 >= r1) return;
  const int64_t n = r1 - r0, rb = (int64_t)A.K * 4;
  if (A.x) l2_prefetch(A.x + r0 * A.K, n * rb);
  if (A.prev_mode == 0) l2_prefetch(A.xp + r0 * A.K, n * rb);
  if constexpr (ELL) {
    l2_prefetch(A.ell_desc + r0, n * 4);
    l2_prefetch(A.ell_col + r0 * 8, n * 32);
    l2_prefetch(A.ell_hl + r0 * 8, n * 64);
  } else {
    const int64_t e0 = A.ptr[r0], e1 = A.ptr[r1];
    l2_prefetch(A.ptr + r0, n * 4);
    l2_prefetch(A.col + e0, (e1 - e0) * 4);
    l2_prefetch(A.hl + e0, (e1 - e0) * 8);
  }
}

template <int V, int CH, bool ADJ, bool EARLY>
__device__ __forceinline__ void step3f_body(const Step3Args<float>& A, const int64_t tb0) {
  constexpr int P = V / 2;  // CH = entries per chunk
  const int KV = A.K / V;
  const int64_t t = tb0 + threadIdx.x;
  if (A.pf_rows > 0 && threadIdx.x == 0 && tb0 < A.row_threads)
    prefetch_ahead<false>(A, div_kv(tb0, KV) + A.pf_rows,
                          div_kv(min(tb0 + (int64_t)blockDim.x, A.row_threads), KV) + 1 + A.pf_rows);
  if (t >= A.row_threads) {
    // sensor gather of the input state (forward launches only)
    if (A.y_out == nullptr) return;
    const int64_t g = t - A.row_threads;
    if (g >= (int64_t)A.n_obs * KV) return;
    const int d = (int)div_kv(g, KV);
    const int kv = (int)(g - (int64_t)d * KV);
    float acc[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = 0.0f;
#pragma unroll
    for (int s = 0; s < kDetPts; ++s) {
      const int64_t node = A.det_node[kDetPts * d + s];
      const float wt = A.det_w[kDetPts * d + s];
      const Pack<float, V> a = ld<float, V>(A.x + node * A.K + (int64_t)kv * V);
      if (A.prev_mode == 0) {
        const Pack<float, V> b = ld<float, V>(A.xp + node * A.K + (int64_t)kv * V);
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = fmaf(wt, 0.5f * (a.v[q] + b.v[q]), acc[q]);
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = fmaf(wt, a.v[q], acc[q]);
      }
    }
    Pack<float, V> y;
#pragma unroll
    for (int q = 0; q < V; ++q) y.v[q] = A.scale * acc[q];
    st<float, V>(A.y_out + (int64_t)d * A.K + (int64_t)kv * V, y);
    return;
  }
  const int64_t rowi = div_kv(t, KV);
  const int kv = (int)(t - rowi * KV);
  // rows are independent within a step, so they may be processed in any order;
  // a spatially local order (Z-order of the nodes) keeps a block's neighbour
  // rows in its SM's L1
  const int64_t row = A.order ? (int64_t)A.order[rowi] : rowi;
  const int64_t off = row * A.K + (int64_t)kv * V;
  // EARLY: the node's own x and xp are loaded before the row walk so that their
  // latency overlaps the neighbour loads (more registers held across the walk)
  Pack<float, V> xi, xpi;
  auto load_own = [&]() {
    if (A.x) {
      xi = ld<float, V>(A.x + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) xi.v[q] = 0.0f;
    }
    if (A.prev_mode == 0) {
      xpi = ld<float, V>(A.xp + off);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) xpi.v[q] = (A.prev_mode == 1) ? xi.v[q] : 0.0f;
    }
  };
  if constexpr (EARLY) load_own();
  const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
  const int ni = ADJ ? (int)A.ninj[row] : 0;
  const int eA = e1 - ni;
  const int eB = eA - (int)A.nb[row];
  const uint32_t Ku = (uint32_t)A.K;
  u64 acc[P], accl[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
  if (A.x) {
    const float* xk = A.x + (int64_t)kv * V;
    // software pipeline: the next chunk's columns and coefficients are loaded
    // while the current chunk's neighbour loads are in flight
    uint32_t j[CH];
    float2 c[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const bool in = e0 + q < eA;
      j[q] = in ? (A.col[e0 + q] & kIdxMask) : 0u;
      c[q] = in ? A.hl[e0 + q] : make_float2(0.0f, 0.0f);
    }
    for (int e = e0; e < eA; e += CH) {
      u64 x[CH][P];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        if (e + q < eA) {
          ld_pairs<P>(xk + (size_t)j[q] * Ku, x[q]);
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) x[q][p] = 0ull;
        }
      }
      float2 cc[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        cc[q] = c[q];
        const int en = e + CH + q;
        const bool in = en < eA;
        j[q] = in ? (A.col[en] & kIdxMask) : 0u;
        c[q] = in ? A.hl[en] : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const u64 ch = dup2(cc[q].x), cl = dup2(cc[q].y);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          acc[p] = ffma2(ch, x[q][p], acc[p]);
          accl[p] = ffma2(cl, x[q][p], accl[p]);
        }
      }
    }
    if (eB < eA && A.prev_mode != 2) {
      // boundary entries act on w_j = x_j - xp_j: remove their xp_j part
      const float* pk = (A.prev_mode == 0 ? A.xp : A.x) + (int64_t)kv * V;
      for (int e = eB; e < eA; ++e) {
        const float2 c = A.hl[e];
        u64 x[P];
        ld_pairs<P>(pk + (size_t)(A.col[e] & kIdxMask) * Ku, x);
        const u64 ch = dup2(-c.x), cl = dup2(-c.y);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          acc[p] = ffma2(ch, x[p], acc[p]);
          accl[p] = ffma2(cl, x[p], accl[p]);
        }
      }
    }
  }
  float src[V];
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  if constexpr (ADJ) {
    for (int e = eA; e < e1; ++e) {
      const int64_t j = (int64_t)(A.col[e] & kIdxMask);
      const float h = A.hl[e].x;
      if (A.ya) {
        const Pack<float, V> y = ld<float, V>(A.ya + j * A.K + (int64_t)kv * V);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(h, y.v[q], src[q]);
      }
      if (A.yb) {
        const Pack<float, V> y = ld<float, V>(A.yb + j * A.K + (int64_t)kv * V);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(h, y.v[q], src[q]);
      }
    }
  }
  if constexpr (!EARLY) load_own();
  Pack<float, V> xo;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const float2 a = unpack2(acc[p]), al = unpack2(accl[p]);
    const float w0 = xi.v[2 * p] - xpi.v[2 * p], w1 = xi.v[2 * p + 1] - xpi.v[2 * p + 1];
    xo.v[2 * p] = xi.v[2 * p] + (w0 - (a.x + al.x) + A.inj_scale * src[2 * p]);
    xo.v[2 * p + 1] = xi.v[2 * p + 1] + (w1 - (a.y + al.y) + A.inj_scale * src[2 * p + 1]);
  }
  st<float, V>(A.xn + off, xo);
}

template <int V, int CH, bool ADJ, bool EARLY>
__global__ void __launch_bounds__(256) step3f_kernel(const Step3Args<float> A) {
  step3f_body<V, CH, ADJ, EARLY>(A, (int64_t)blockIdx.x * blockDim.x);
}

// the same with at least 6 resident blocks per SM asked of the compiler (<= 40 registers)
template <int V, int CH, bool ADJ>
__global__ void __launch_bounds__(1024) step3f_big_kernel(const Step3Args<float> A) {
  step3f_body<V, CH, ADJ, false>(A, (int64_t)blockIdx.x * blockDim.x);
}

template <int V, int CH, bool ADJ>
__global__ void __launch_bounds__(256, 6) step3f_occ_kernel(const Step3Args<float> A) {
  step3f_body<V, CH, ADJ, false>(A, (int64_t)blockIdx.x * blockDim.x);
}

template <int V, int CH, bool ADJ>
__global__ void __launch_bounds__(256) step3f_group_kernel(const __grid_constant__ Step3Group<float> G) {
  int g = 0;
  while (g + 1 < G.n && (int64_t)blockIdx.x >= G.block_off[g + 1]) ++g;
  step3f_body<V, CH, ADJ, false>(G.a[g], ((int64_t)blockIdx.x - G.block_off[g]) * blockDim.x);
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
  const int64_t row = div_kv(t, KV);
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

// The rpb row lanes' sums of each sample column k of a block into
// partial[block][k], in a fixed order: with K dividing 32 the 32/K row lanes
// of a warp first combine by warp shuffles (a fixed tree), then the block's
// warps are added in order; otherwise the rpb row lanes are added in order
// through shared memory.  Every thread of the block calls it.
__device__ __forceinline__ void block_partial(double acc, int K, int rpb, double* sh, double* __restrict__ partial) {
  const int k = threadIdx.x % K;
  if (K < 32 && (32 % K) == 0) {  // blockDim.x = 256: whole warps
    for (int off = 16; off >= K; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < K) sh[warp * K + lane] = acc;
    __syncthreads();
    if (threadIdx.x < K) {
      double t = 0.0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += sh[j * K + k];
      partial[(int64_t)blockIdx.x * K + k] = t;
    }
    return;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int j = 0; j < rpb; ++j) t += sh[j * K + k];
    partial[(int64_t)blockIdx.x * K + k] = t;
  }
}

// Column k of the [na][K] block partials summed by the 32 lanes of a warp:
// lane j adds blocks j, j + 32, ... in order, then a butterfly of warp
// shuffles; every lane ends with the same bits (each level adds the same two
// values in either order).
__device__ __forceinline__ double warp_colsum(const double* __restrict__ pa, int na, int K, int k) {
  double s = 0.0;
  for (int b = (int)(threadIdx.x & 31); b < na; b += 32) s += pa[(int64_t)b * K + k];
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

}  // namespace pat
