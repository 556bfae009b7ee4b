// Whittle-Matern prior on the GPU (Section 4.1.2, eq. matern-cov-op; Section
// 6.4): a Gaussian field on a periodic box grid, T z = F^{-1} diag(sqrt(S)) F z
// with z ~ N(0, I), S(k) = (1/l^2 + |2 pi k|^2)^{-(s + d/2)} normalised to the
// marginal variance sigma^2, carried to the finite element nodes by trilinear
// interpolation P; RTO then runs in the latent space of z (Section 6.4: the
// optimisation is carried out in the latent Gaussian parameter space), on the
// extended system A = [G P T / sigma_n ; I], b = (y_obs / sigma_n + eta, xi).
//
// Kernels:
//   - T as five passes over the K-stacked grid field [G][K] (G = n_g^3, grid
//     point (ix, iy, iz) at (ix n_g + iy) n_g + iz): forward FFTs along x and y,
//     then one pass doing the forward FFT along z, the multiplication by
//     sqrt(S) and the inverse FFT along z, then inverse FFTs along y and x.
//     A line's transform for a chunk of KC samples is split in the four-step
//     way over n_g / 16 threads per sample, each holding 16 values in
//     registers, with one exchange through shared memory per transform; every
//     global access reads or writes KC contiguous floats of one grid point.
//   - P (nodes <- grid) gathers 8 grid values per node; P^T (grid <- nodes)
//     gathers through a host-built grid -> node CSR of the same FP32 weights
//     (no atomics; exactly P's transpose).
//   - With K even, T runs on K / 2 complex fields z_k + i z_{k+1}: T is
//     complex-linear and maps real fields to real fields (sqrt(S) is real and
//     even in the frequency), so the real and imaginary parts of the result
//     are T z_k and T z_{k+1}; the real [G][K] array read as complex [G][K/2]
//     is exactly that packing, and every pass moves half the bytes.
//   - Latent CGLS: the wave solves are the mesh's (graph-replayed) forward and
//     transposed solves on an RTO workspace; the latent iterate x is FP64, d,
//     r, s are FP32 and updated in FP32, and every inner product, norm and
//     scalar is accumulated and kept in FP64 (squares summed in FP32 over runs
//     of 8 rows, the runs in FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pat_internal.h"
#include "pat_kernels.cuh"
#include "pat_solver.cuh"

namespace pat {

struct MaternGrid {
  int ng = 0, log2ng = 0;
  int64_t G = 0, N = 0;
  double lo[3] = {0, 0, 0}, len = 0, ell = 0, s = 0, sigma = 0;
  int device = -1;
  float* filt = nullptr;     // [G] sqrt(S)
  float2* twid = nullptr;    // [ng] exp(-2 pi i j / ng)
  int32_t* p_idx = nullptr;  // [N][8] grid points of each node
  float* p_w = nullptr;      // [N][8] trilinear weights
  int32_t* pt_ptr = nullptr; // [G + 1] grid -> node CSR
  int32_t* pt_node = nullptr;
  float* pt_w = nullptr;
};

}  // namespace pat

struct pat_matern {
  pat::MaternGrid g;
};

namespace pat {
namespace {

inline unsigned nblk(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }
inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Samples per FFT block: the largest of 32, 16, ..., 1 that divides K.
int fft_kc(int K) {
  int kc = 32;
  while (K % kc) kc /= 2;
  return kc;
}

// ---------------------------------------------------------------------------
// FFT passes.  MODE 0: forward, real input -> complex output (axis x).
// MODE 1: forward complex -> complex.  MODE 2: forward, times filt, inverse
// (axis z).  MODE 3: inverse complex -> complex.  MODE 4: inverse, complex ->
// real output scale * Re + (addend or 0) (axis x).  MODE 5: inverse, complex
// -> the pair (scale Re, scale Im) + (addend pair or 0) (axis x; two samples
// packed in one complex field).
// axis: 0 = x (stride n_g^2), 1 = y (stride n_g), 2 = z (stride 1) in grid points.
//
// A line of length NG = N1 N2 (N1 = min(16, NG)) is split in the four-step
// (Cooley-Tukey) way: with n = N2 n1 + n2 and j = k1 + N1 k2,
//   X_j = sum_{n2} W_NG^{n2 k1} W_N2^{n2 k2} [sum_{n1} x_n W_N1^{n1 k1}],
// W_M = exp(-2 pi i / M).  A line is worked by N2 threads per sample: thread
// n2 loads x_{N2 n1 + n2} (n1 = 0 .. N1-1) into registers, transforms them in
// registers (length N1), multiplies by W_NG^{n2 k1}, and one exchange through
// shared memory hands it the values of N1 / N2 frequencies k1 for every n2, on
// which it runs the length-N2 transforms in registers.  Shared memory is read
// and written once per element per split (a radix-2 sweep through shared
// memory touches it log2(NG) times).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a times w (CONJ: times conj(w))
template <bool CONJ>
__device__ __forceinline__ float2 cmul_c(float2 a, float2 w) {
  return CONJ ? make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : cmul(a, w);
}

// cos and sin of 2 pi q / 16, q = 0 .. 7 (cos(pi/8) = sqrt(2 + sqrt 2) / 2,
// sin(pi/8) = sqrt(2 - sqrt 2) / 2, cos(pi/4) = sqrt(2) / 2)
__host__ __device__ constexpr float cos16(int q) {
  return q == 0 ? 1.0f
       : q == 1 ? 0.92387953251128674f
       : q == 2 ? 0.70710678118654752f
       : q == 3 ? 0.38268343236508977f
       : q == 4 ? 0.0f
       : q == 5 ? -0.38268343236508977f
       : q == 6 ? -0.70710678118654752f
                : -0.92387953251128674f;
}
// sin(2 pi q / 16) = cos(2 pi (q - 4) / 16)
__host__ __device__ constexpr float sin16(int q) { return cos16(q >= 4 ? q - 4 : 4 - q); }

// b times W_16^q (CONJ: times W_16^{-q}); q is a constant once the callers'
// loops are unrolled, so the branches fold away
template <bool CONJ>
__device__ __forceinline__ float2 mul_w16(float2 b, int q) {
  if (q == 0) return b;
  if (q == 4) return CONJ ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
  const float c = cos16(q), s = sin16(q);
  return CONJ ? make_float2(b.x * c - b.y * s, b.y * c + b.x * s) : make_float2(b.x * c + b.y * s, b.y * c - b.x * s);
}

__host__ __device__ constexpr int brev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2_c(int m) { return m <= 1 ? 0 : 1 + ilog2_c(m / 2); }

// In-register DFT of length M (a power of two <= 16): v_k <- sum_n v_n W_M^{nk}
// (CONJ: W_M^{-nk}), natural order in and out; radix-2 decimation in time on
// the bit-reversed copy, butterflies of span 2h with the roots W_{2h}^p = W_16^{8p/h}.
// (Template recursion keeps every index a compile-time constant, so v stays in
// registers.)
template <int M, int I>
__device__ __forceinline__ void brev_perm(float2* v) {
  if constexpr (I < M) {
    constexpr int r = brev_c(I, ilog2_c(M));
    if constexpr (r > I) {
      const float2 t = v[I];
      v[I] = v[r];
      v[r] = t;
    }
    brev_perm<M, I + 1>(v);
  }
}
template <int M, bool CONJ, int H>
__device__ __forceinline__ void dft_stages(float2* v) {
  if constexpr (H < M) {
#pragma unroll
    for (int i0 = 0; i0 < M; i0 += 2 * H)
#pragma unroll
      for (int p = 0; p < H; ++p) {
        const float2 a = v[i0 + p];
        const float2 b = mul_w16<CONJ>(v[i0 + p + H], p * (8 / H));
        v[i0 + p] = make_float2(a.x + b.x, a.y + b.y);
        v[i0 + p + H] = make_float2(a.x - b.x, a.y - b.y);
      }
    dft_stages<M, CONJ, 2 * H>(v);
  }
}
template <int M, bool CONJ>
__device__ __forceinline__ void dft_reg(float2* v) {
  brev_perm<M, 0>(v);
  dft_stages<M, CONJ, 1>(v);
}

// Forward split: thread n2 = t2 of the line holds v[n1] = x_{N2 n1 + t2}; on
// return v[i N2 + k2] = X_{(t2 + N2 i) + N1 k2}, i < N1 / N2.  su is the line's
// [NG][KC] exchange buffer (element (e, k) at (e << lkc) + k); tw the NG roots
// W_NG^e.  Every thread of the block calls it (two block barriers).
template <int N1, int N2, bool CONJ>
__device__ __forceinline__ void fft_split_fwd(float2* v, float2* su, int t2, int k, int lkc,
                                              const float2* __restrict__ tw) {
  dft_reg<N1, CONJ>(v);
  if constexpr (N2 > 1) {
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul_c<CONJ>(v[k1], __ldg(tw + t2 * k1));
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) su[((t2 * N1 + k1) << lkc) + k] = v[k1];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N1 / N2; ++i)
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[i * N2 + n2] = su[((n2 * N1 + t2 + N2 * i) << lkc) + k];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N1 / N2; ++i) dft_reg<N2, CONJ>(v + i * N2);
  }
}

// The transposed split: from v[i N2 + k2] = X_{(t2 + N2 i) + N1 k2} to
// v[n1] = x_{N2 n1 + t2}, x_n = sum_j X_j W_NG^{nj} (CONJ: W_NG^{-nj}).
template <int N1, int N2, bool CONJ>
__device__ __forceinline__ void fft_split_bwd(float2* v, float2* su, int t2, int k, int lkc,
                                              const float2* __restrict__ tw) {
  if constexpr (N2 > 1) {
#pragma unroll
    for (int i = 0; i < N1 / N2; ++i) {
      dft_reg<N2, CONJ>(v + i * N2);
#pragma unroll
      for (int n2 = 1; n2 < N2; ++n2)
        v[i * N2 + n2] = cmul_c<CONJ>(v[i * N2 + n2], __ldg(tw + (t2 + N2 * i) * n2));
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) su[((n2 * N1 + t2 + N2 * i) << lkc) + k] = v[i * N2 + n2];
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = su[((t2 * N1 + k1) << lkc) + k];
    __syncthreads();
  }
  dft_reg<N1, CONJ>(v);
}

// Launch geometry of a pass: N2 KC threads per (line, sample chunk) unit,
// blocks of max(256, N2 KC) threads, blockDim * N1 float2 of shared memory.
template <int LOG2NG>
struct FftGeom {
  static constexpr int NG = 1 << LOG2NG, L1 = LOG2NG < 4 ? LOG2NG : 4, N1 = 1 << L1, L2 = LOG2NG - L1,
                       N2 = 1 << L2;
};

template <int LOG2NG, int MODE>
// (in and out may be the same buffer: a unit's threads load all of its values
// before the first barrier and store after the last one, and units are disjoint.)
__global__ void __launch_bounds__(512) fft_pass_kernel(const void* in, void* out, const float* __restrict__ addend,
                                                       int K, int KC, int axis, int64_t units,
                                                       const float2* __restrict__ tw, const float* __restrict__ filt,
                                                       float scale) {
  using Gm = FftGeom<LOG2NG>;
  constexpr int NG = Gm::NG, N1 = Gm::N1, N2 = Gm::N2;
  extern __shared__ float2 sh[];
  const int lkc = __ffs(KC) - 1;
  const int k = threadIdx.x & (KC - 1);
  const int t2 = (threadIdx.x >> lkc) & (N2 - 1);
  const int ul = threadIdx.x >> (lkc + Gm::L2);
  const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> (lkc + Gm::L2)) + ul;
  const bool live = u < units;
  float2* su = sh + ((size_t)ul << (LOG2NG + lkc));
  const int chunks = K >> lkc;
  const int64_t line = live ? u / chunks : 0;
  const int kc0 = live ? (int)(u - line * chunks) * KC : 0;
  // the two fixed coordinates of this line, and its first grid point and stride
  const int a = (int)(line >> LOG2NG), b = (int)(line & (NG - 1));
  int64_t g0, stride;
  if (axis == 0) {
    g0 = (int64_t)a * NG + b;  // (0, a, b)
    stride = (int64_t)NG * NG;
  } else if (axis == 1) {
    g0 = (int64_t)a * NG * NG + b;  // (a, 0, b)
    stride = NG;
  } else {
    g0 = ((int64_t)a * NG + b) * NG;  // (a, b, 0)
    stride = 1;
  }
  const int64_t base = g0 * K + kc0 + k, jstep = stride * K;
  float2 v[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    const int64_t off = base + (int64_t)(N2 * n1 + t2) * jstep;
    if (!live) {
      v[n1] = make_float2(0.0f, 0.0f);
    } else if constexpr (MODE == 0) {
      v[n1] = make_float2(__ldg(static_cast<const float*>(in) + off), 0.0f);
    } else {
      v[n1] = static_cast<const float2*>(in)[off];
    }
  }
  fft_split_fwd<N1, N2, (MODE >= 3)>(v, su, t2, k, lkc, tw);
  if constexpr (MODE == 2) {
    // multiply by sqrt(S) at (a, b, j), then the inverse along z, which lands
    // each value back where this thread loaded it
#pragma unroll
    for (int i = 0; i < N1 / N2; ++i)
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const float f = __ldg(filt + g0 + (t2 + N2 * i) + N1 * k2);
        v[i * N2 + k2] = make_float2(f * v[i * N2 + k2].x, f * v[i * N2 + k2].y);
      }
    fft_split_bwd<N1, N2, true>(v, su, t2, k, lkc, tw);
    if (live) {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) static_cast<float2*>(out)[base + (int64_t)(N2 * n1 + t2) * jstep] = v[n1];
    }
  } else if (live) {
#pragma unroll
    for (int i = 0; i < N1 / N2; ++i)
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int64_t off = base + (int64_t)((t2 + N2 * i) + N1 * k2) * jstep;
        const float2 w = v[i * N2 + k2];
        if constexpr (MODE == 4) {
          static_cast<float*>(out)[off] = scale * w.x + (addend ? __ldg(addend + off) : 0.0f);
        } else if constexpr (MODE == 5) {
          float2 o = make_float2(scale * w.x, scale * w.y);
          if (addend) {
            const float2 ad = __ldg(reinterpret_cast<const float2*>(addend) + off);
            o.x += ad.x;
            o.y += ad.y;
          }
          static_cast<float2*>(out)[off] = o;
        } else {
          static_cast<float2*>(out)[off] = w;
        }
      }
  }
}

// Sample index of element e of a [rows][K] array: lk = log2(K) when K is a
// power of two (a mask), else -1 (a division).
__device__ __forceinline__ int kof(int64_t e, int K, int lk) {
  return lk >= 0 ? (int)(e & (K - 1)) : (int)(e % K);
}

// ---------------------------------------------------------------------------
// Interpolation and its transpose; one thread per (point, sample), so a warp's
// accesses to one grid point's or node's samples are contiguous.
// ---------------------------------------------------------------------------
__global__ void interp_kernel(int64_t N, int K, int lk, const int32_t* __restrict__ idx, const float* __restrict__ w,
                              const float* __restrict__ grid, float* __restrict__ nodes) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  const int k = kof(t, K, lk);
  const int64_t i = lk >= 0 ? t >> lk : t / K;
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc = fmaf(w[i * 8 + c], grid[(int64_t)idx[i * 8 + c] * K + k], acc);
  nodes[t] = acc;
}

__global__ void interp_t_kernel(int64_t G, int K, int lk, const int32_t* __restrict__ ptr,
                                const int32_t* __restrict__ node, const float* __restrict__ w,
                                const float* __restrict__ vals, float* __restrict__ grid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G * K) return;
  const int k = kof(t, K, lk);
  const int64_t g = lk >= 0 ? t >> lk : t / K;
  float acc = 0.0f;
  for (int e = ptr[g]; e < ptr[g + 1]; ++e) acc = fmaf(w[e], vals[(int64_t)node[e] * K + k], acc);
  grid[t] = acc;
}

// ---------------------------------------------------------------------------
// Latent CGLS vector work (FP64 scalars per sample)
// ---------------------------------------------------------------------------
// part[b][k] = sum of X[r][k]^2 over the rows r = b R + l + j gridDim.x R
// (l < R = 256 / min(K, 256) row lanes of block b; samples over blockIdx.y
// when K > 256).  A lane adds runs of 8 of its rows in FP32 (non-negative
// terms: a run's relative error is at most 8 units of FP32 rounding) and the
// runs in FP64, and the R lanes are added in a fixed order (warp shuffles,
// then the warps in order, when K divides 32): the sums are deterministic.  (B300 issues FP64 arithmetic at a small
// fraction of its FP32 rate; a double operation per element would bound
// these passes by the FP64 pipe, not by memory.)
__global__ void __launch_bounds__(256) sq_partial_kernel(const float* __restrict__ X, int64_t rows, int K,
                                                         double* __restrict__ part) {
  __shared__ double red[256];
  const int KB = K < 256 ? K : 256, R = 256 / KB;
  const int kl = threadIdx.x % KB, l = threadIdx.x / KB;
  const int k = blockIdx.y * KB + kl;
  const int64_t step = (int64_t)gridDim.x * R;
  double acc = 0.0;
  if (l < R && k < K) {
    int64_t r = (int64_t)blockIdx.x * R + l;
    for (; r + 7 * step < rows; r += 8 * step) {
      float run = 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float v = X[(r + q * step) * K + k];
        run = fmaf(v, v, run);
      }
      acc += (double)run;
    }
    float run = 0.0f;
    for (; r < rows; r += step) {
      const float v = X[r * K + k];
      run = fmaf(v, v, run);
    }
    acc += (double)run;
  }
  if (KB < 32 && (32 % KB) == 0) {
    // the 32 / KB row lanes of a warp by warp shuffles (a fixed tree), then the warps in order
    for (int off = 16; off >= KB; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < KB) red[warp * KB + lane] = acc;
    __syncthreads();
    if (threadIdx.x < KB && k < K) {
      double sum = 0.0;
      for (int j = 0; j < 8; ++j) sum += red[j * KB + kl];
      part[(int64_t)blockIdx.x * K + k] = sum;
    }
    return;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (l == 0 && k < K) {
    double sum = 0.0;
    for (int j = 0; j < R; ++j) sum += red[j * KB + kl];
    part[(int64_t)blockIdx.x * K + k] = sum;
  }
}

__device__ __forceinline__ bool bad(double v) { return !(v > 0.0) || !isfinite(v); }

// The scalar kernels run one warp per sample (128-thread blocks); the warp
// sums the sample's block partials by warp_colsum and its first lane finishes.
#define LAT_WARP_K()                                                   \
  const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); \
  if (k >= K) return;                                                  \
  const bool lead = (threadIdx.x & 31) == 0

// gamma = ||s||^2 (begin)
__global__ void gamma0_kernel(const double* part, int nb, int K, double* gamma, int* status) {
  LAT_WARP_K();
  const double g = warp_colsum(part, nb, K, k);
  if (!lead) return;
  if (!isfinite(g)) atomicExch(status, (int)PAT_ENUMERIC);
  gamma[k] = g;
}

// alpha = gamma / (||q_d||^2 + ||d||^2), and alpha rounded to FP32 for the
// FP32 residual updates
__global__ void alpha_kernel(const double* pq, const double* pd, int nb, int K, const double* gamma, double* alpha,
                             float* alphaf, int* status) {
  LAT_WARP_K();
  const double qq = warp_colsum(pq, nb, K, k) + warp_colsum(pd, nb, K, k);
  if (!lead) return;
  double a = 0.0;
  if (gamma[k] > 0.0) {
    if (bad(qq)) atomicExch(status, (int)PAT_ENUMERIC);
    else a = gamma[k] / qq;
  }
  alpha[k] = a;
  alphaf[k] = (float)a;
}

// beta = ||s||^2 / gamma (and rounded to FP32); gamma = ||s||^2
__global__ void beta_kernel(const double* part, int nb, int K, double* gamma, float* betaf, int* status) {
  LAT_WARP_K();
  const double g = warp_colsum(part, nb, K, k);
  if (!lead) return;
  double b = 0.0;
  if (!isfinite(g)) atomicExch(status, (int)PAT_ENUMERIC);
  else if (gamma[k] > 0.0) b = g / gamma[k];
  betaf[k] = (float)b;
  gamma[k] = g;
}

// Four consecutive elements per thread; with K a multiple of 4 they are
// samples k .. k+3 of one row and move as vectors.
// x += alpha d (the FP64 iterate: one conversion and one FP64 FMA per
// element); r_p -= alpha d in FP32 (q_p = d for the identity prior block)
__global__ void lat_update_x_kernel(int64_t n, int K, int lk, const double* __restrict__ alpha,
                                    const float* __restrict__ alphaf, const float* __restrict__ d,
                                    double* __restrict__ x, float* __restrict__ rp) {
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (e0 >= n) return;
  if ((K & 3) == 0) {
    const int k = kof(e0, K, lk);
    const float4 dv = *reinterpret_cast<const float4*>(d + e0);
    const float4 af = *reinterpret_cast<const float4*>(alphaf + k);
    const double2 a01 = *reinterpret_cast<const double2*>(alpha + k),
                  a23 = *reinterpret_cast<const double2*>(alpha + k + 2);
    double2 x01 = *reinterpret_cast<double2*>(x + e0), x23 = *reinterpret_cast<double2*>(x + e0 + 2);
    x01.x = fma(a01.x, (double)dv.x, x01.x);
    x01.y = fma(a01.y, (double)dv.y, x01.y);
    x23.x = fma(a23.x, (double)dv.z, x23.x);
    x23.y = fma(a23.y, (double)dv.w, x23.y);
    *reinterpret_cast<double2*>(x + e0) = x01;
    *reinterpret_cast<double2*>(x + e0 + 2) = x23;
    float4 r = *reinterpret_cast<float4*>(rp + e0);
    r.x = fmaf(-af.x, dv.x, r.x);
    r.y = fmaf(-af.y, dv.y, r.y);
    r.z = fmaf(-af.z, dv.z, r.z);
    r.w = fmaf(-af.w, dv.w, r.w);
    *reinterpret_cast<float4*>(rp + e0) = r;
  } else {
    for (int64_t e = e0; e < e0 + 4 && e < n; ++e) {
      const int k = kof(e, K, lk);
      const float dv = d[e];
      x[e] = fma(alpha[k], (double)dv, x[e]);
      rp[e] = fmaf(-alphaf[k], dv, rp[e]);
    }
  }
}

// y = y + c w in FP32 (r_d -= alpha q_d with c = -alpha; d = s + beta d with
// w = d, y = s written to d): out[e] = fmaf(sgn * c[k], w[e], y[e])
// (out may alias w or y: each element is read before it is written, by one thread)
__global__ void lat_axpy_kernel(int64_t n, int K, int lk, const float* __restrict__ c, float sgn, const float* w,
                                const float* y, float* out) {
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (e0 >= n) return;
  if ((K & 3) == 0) {
    const int k = kof(e0, K, lk);
    const float4 cv = *reinterpret_cast<const float4*>(c + k);
    const float4 wv = *reinterpret_cast<const float4*>(w + e0);
    float4 yv = *reinterpret_cast<const float4*>(y + e0);
    yv.x = fmaf(sgn * cv.x, wv.x, yv.x);
    yv.y = fmaf(sgn * cv.y, wv.y, yv.y);
    yv.z = fmaf(sgn * cv.z, wv.z, yv.z);
    yv.w = fmaf(sgn * cv.w, wv.w, yv.w);
    *reinterpret_cast<float4*>(out + e0) = yv;
  } else {
    for (int64_t e = e0; e < e0 + 4 && e < n; ++e) out[e] = fmaf(sgn * c[kof(e, K, lk)], w[e], y[e]);
  }
}

// latent prior draws: r_p[g][k] = xi (given) or the library draw of stream 1
// (the prior-draw stream) at element g for sample first + k; x = 0
__global__ void lat_begin_kernel(int64_t rows, int K, int lk, const float* __restrict__ xi, uint64_t seed,
                                 uint64_t first, float* __restrict__ rp, double* __restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * K) return;
  const int kk = kof(t, K, lk);
  const int64_t g = lk >= 0 ? t >> lk : t / K;
  const uint64_t k = first + (uint64_t)kk;
  rp[t] = xi ? xi[t] : (float)normal_draw(seed, 1, k, (uint64_t)g);
  x[t] = 0.0;
}

__global__ void f64_to_f32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}
__global__ void f32_to_f64_kernel(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (double)a[t];
}

template <typename T>
pat_status upload_vec(const std::vector<T>& h, T** d) {
  if (cudaMalloc((void**)d, std::max<size_t>(1, h.size()) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    set_error("pat_matern_create: out of device memory");
    return PAT_ENOMEM;
  }
  if (!h.empty()) return cuda_check(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return PAT_OK;
}

void free_grid(MaternGrid& g) {
  void* ps[] = {g.filt, g.twid, g.p_idx, g.p_w, g.pt_ptr, g.pt_node, g.pt_w};
  for (void* p : ps)
    if (p) cudaFree(p);
  g.filt = nullptr, g.twid = nullptr, g.p_idx = nullptr, g.p_w = nullptr;
  g.pt_ptr = nullptr, g.pt_node = nullptr, g.pt_w = nullptr;
}

// Layout of the latent workspace after the mesh's RTO workspace.
struct LatLayout {
  size_t rto, x, d, r, s, tmp, cbuf, gamma, alpha, alphaf, betaf, part, total;
  int nb;
};
LatLayout lat_layout(const DeviceMesh& m, const MaternGrid& g, int K) {
  LatLayout L{};
  L.nb = 148 * 4;  // blocks of the sum-of-squares passes (partial sums per block and sample)
  size_t o = a256(rto_layout(m, K).total);
  L.rto = 0;
  const size_t GK = (size_t)g.G * K;
  L.x = o; o = a256(o + GK * 8);
  L.d = o; o = a256(o + GK * 4);
  L.r = o; o = a256(o + GK * 4);
  L.s = o; o = a256(o + GK * 4);
  L.tmp = o; o = a256(o + GK * 4);
  L.cbuf = o; o = a256(o + GK * 8);
  L.gamma = o; o = a256(o + K * 8);
  L.alpha = o; o = a256(o + K * 8);
  L.alphaf = o; o = a256(o + K * 4);
  L.betaf = o; o = a256(o + K * 4);
  L.part = o; o = a256(o + (size_t)2 * L.nb * K * 8);
  L.total = o;
  return L;
}

template <int LOG2NG>
void fft_passes(const MaternGrid& g, const float* in, int K, float* out, const float* addend, float2* cbuf,
                cudaStream_t st) {
  using Gm = FftGeom<LOG2NG>;
  const float scale = (float)(1.0 / (double)g.G);
  auto al8 = [](const void* p) { return ((uintptr_t)p & 7) == 0; };
  if (K % 2 == 0 && al8(in) && al8(out) && al8(addend)) {
    // two samples per complex field
    const int Kc = K / 2, KC = fft_kc(Kc);
    const int tpu = Gm::N2 * KC, bs = std::max(256, tpu);
    const int64_t units = (int64_t)g.ng * g.ng * (Kc / KC);
    const unsigned blocks = (unsigned)((units + bs / tpu - 1) / (bs / tpu));
    const size_t smem = (size_t)bs * Gm::N1 * sizeof(float2);
    fft_pass_kernel<LOG2NG, 1><<<blocks, bs, smem, st>>>(in, cbuf, nullptr, Kc, KC, 0, units, g.twid, g.filt, 1.0f);
    fft_pass_kernel<LOG2NG, 1><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, Kc, KC, 1, units, g.twid, g.filt, 1.0f);
    fft_pass_kernel<LOG2NG, 2><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, Kc, KC, 2, units, g.twid, g.filt, 1.0f);
    fft_pass_kernel<LOG2NG, 3><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, Kc, KC, 1, units, g.twid, g.filt, 1.0f);
    fft_pass_kernel<LOG2NG, 5><<<blocks, bs, smem, st>>>(cbuf, out, addend, Kc, KC, 0, units, g.twid, g.filt, scale);
    return;
  }
  const int KC = fft_kc(K);
  const int tpu = Gm::N2 * KC, bs = std::max(256, tpu);
  const int64_t units = (int64_t)g.ng * g.ng * (K / KC);
  const unsigned blocks = (unsigned)((units + bs / tpu - 1) / (bs / tpu));
  const size_t smem = (size_t)bs * Gm::N1 * sizeof(float2);
  fft_pass_kernel<LOG2NG, 0><<<blocks, bs, smem, st>>>(in, cbuf, nullptr, K, KC, 0, units, g.twid, g.filt, 1.0f);
  fft_pass_kernel<LOG2NG, 1><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, K, KC, 1, units, g.twid, g.filt, 1.0f);
  fft_pass_kernel<LOG2NG, 2><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, K, KC, 2, units, g.twid, g.filt, 1.0f);
  fft_pass_kernel<LOG2NG, 3><<<blocks, bs, smem, st>>>(cbuf, cbuf, nullptr, K, KC, 1, units, g.twid, g.filt, 1.0f);
  fft_pass_kernel<LOG2NG, 4><<<blocks, bs, smem, st>>>(cbuf, out, addend, K, KC, 0, units, g.twid, g.filt, scale);
}

// The passes of the largest grid use more than the default 48 KB of dynamic
// shared memory (512-thread blocks x 16 values x 8 bytes).
void fft_allow_smem() {
  const int smem = 512 * 16 * (int)sizeof(float2);
  const void* fns[6] = {(const void*)fft_pass_kernel<8, 0>, (const void*)fft_pass_kernel<8, 1>,
                        (const void*)fft_pass_kernel<8, 2>, (const void*)fft_pass_kernel<8, 3>,
                        (const void*)fft_pass_kernel<8, 4>, (const void*)fft_pass_kernel<8, 5>};
  for (const void* f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// out = T in (in, out real [G][K]); out may alias addend; cbuf complex [G][K]
pat_status apply_T(const MaternGrid& g, const float* in, int K, float* out, const float* addend, float2* cbuf,
                   cudaStream_t st) {
  switch (g.log2ng) {
    case 3: fft_passes<3>(g, in, K, out, addend, cbuf, st); break;
    case 4: fft_passes<4>(g, in, K, out, addend, cbuf, st); break;
    case 5: fft_passes<5>(g, in, K, out, addend, cbuf, st); break;
    case 6: fft_passes<6>(g, in, K, out, addend, cbuf, st); break;
    case 7: fft_passes<7>(g, in, K, out, addend, cbuf, st); break;
    default: fft_passes<8>(g, in, K, out, addend, cbuf, st); break;
  }
  return cuda_check(cudaGetLastError(), "Matern T launch");
}

// log2(K) for a power of two, else -1 (the kernels' index split)
int log2_or_neg(int K) {
  if (K & (K - 1)) return -1;
  int l = 0;
  while ((1 << l) < K) ++l;
  return l;
}

pat_status interp(const MaternGrid& g, const float* grid, int K, float* nodes, cudaStream_t st) {
  interp_kernel<<<nblk(g.N * K), 256, 0, st>>>(g.N, K, log2_or_neg(K), g.p_idx, g.p_w, grid, nodes);
  return cuda_check(cudaGetLastError(), "Matern P launch");
}

pat_status interp_t(const MaternGrid& g, const float* nodes, int K, float* grid, cudaStream_t st) {
  interp_t_kernel<<<nblk(g.G * K), 256, 0, st>>>(g.G, K, log2_or_neg(K), g.pt_ptr, g.pt_node, g.pt_w, nodes, grid);
  return cuda_check(cudaGetLastError(), "Matern P^T launch");
}

pat_status sq_partials(const float* X, int64_t rows, int K, int nb, double* part, cudaStream_t st) {
  sq_partial_kernel<<<dim3((unsigned)nb, (unsigned)((K + 255) / 256)), 256, 0, st>>>(X, rows, K, part);
  return cuda_check(cudaGetLastError(), "Matern reduction launch");
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_matern_create(const pat_mesh* mesh, int32_t n_grid, const double* box_lo, double box_len, double ell,
                             double s, double sigma, pat_matern** out) {
  clear_error();
  if (!mesh || !box_lo || !out) {
    set_error("pat_matern_create: NULL argument");
    return PAT_EINVAL;
  }
  if (!check_device(mesh, "pat_matern_create")) return PAT_EINVAL;
  if (mesh->d.prec != PAT_F32) {
    set_error("pat_matern_create: the latent-space sampler runs on FP32 meshes");
    return PAT_EUNSUPPORTED;
  }
  int log2ng = 0;
  while ((1 << log2ng) < n_grid) ++log2ng;
  if (n_grid < 8 || n_grid > 256 || (1 << log2ng) != n_grid) {
    set_error("pat_matern_create: n_grid = %d must be a power of two in [8, 256]", n_grid);
    return PAT_EINVAL;
  }
  if (!(box_len > 0.0) || !(ell > 0.0) || !(s > 0.0) || !(sigma > 0.0)) {
    set_error("pat_matern_create: box_len, ell, s and sigma must be > 0");
    return PAT_EINVAL;
  }
  const HostMesh& hm = mesh->d.host;
  const int64_t N = hm.N, ng = n_grid, G = ng * ng * ng;
  const double h = box_len / (double)ng;
  MaternGrid g;
  g.ng = n_grid, g.log2ng = log2ng, g.G = G, g.N = N, g.len = box_len, g.ell = ell, g.s = s, g.sigma = sigma;
  for (int c = 0; c < 3; ++c) g.lo[c] = box_lo[c];
  cudaGetDevice(&g.device);
  // sqrt(S) at the DFT frequencies k_j = j / L (j < ng/2), (j - ng) / L above,
  // normalised so that mean(S) = sigma^2 (the discrete marginal variance)
  std::vector<double> kf(ng);
  for (int64_t j = 0; j < ng; ++j) kf[j] = (double)(j < (ng + 1) / 2 ? j : j - ng) / box_len;
  std::vector<double> S(G);
  double mean = 0.0;
  const double ex = -(s + 1.5);
  for (int64_t a = 0; a < ng; ++a)
    for (int64_t b = 0; b < ng; ++b)
      for (int64_t c = 0; c < ng; ++c) {
        const double k2 = kf[a] * kf[a] + kf[b] * kf[b] + kf[c] * kf[c];
        const double v = std::pow(1.0 / (ell * ell) + 4.0 * M_PI * M_PI * k2, ex);
        S[(a * ng + b) * ng + c] = v;
        mean += v;
      }
  mean /= (double)G;
  std::vector<float> filt(G);
  for (int64_t q = 0; q < G; ++q) filt[q] = (float)std::sqrt(S[q] * sigma * sigma / mean);
  std::vector<float2> tw(ng);
  for (int64_t j = 0; j < ng; ++j) {
    const double ang = -2.0 * M_PI * (double)j / (double)ng;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  // trilinear interpolation of the nodes (inside [lo, lo + L) on every axis;
  // periodic wrap for the upper neighbours)
  std::vector<int32_t> pidx(N * 8);
  std::vector<float> pw(N * 8);
  for (int64_t i = 0; i < N; ++i) {
    int64_t i0[3];
    double f[3];
    for (int c = 0; c < 3; ++c) {
      const double u = (hm.xyz[3 * i + c] - box_lo[c]) / h;
      i0[c] = (int64_t)std::floor(u);
      if (i0[c] < 0 || i0[c] > ng - 1) {
        set_error("pat_matern_create: node %lld lies outside the box", (long long)i);
        return PAT_EINVAL;
      }
      f[c] = u - (double)i0[c];
    }
    int q = 0;
    for (int dx = 0; dx < 2; ++dx)
      for (int dy = 0; dy < 2; ++dy)
        for (int dz = 0; dz < 2; ++dz, ++q) {
          const int64_t ix = (i0[0] + dx) % ng, iy = (i0[1] + dy) % ng, iz = (i0[2] + dz) % ng;
          pidx[i * 8 + q] = (int32_t)((ix * ng + iy) * ng + iz);
          pw[i * 8 + q] = (float)((dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]));
        }
  }
  // the grid -> node CSR of the same weights (P^T as a gather)
  std::vector<int32_t> ptr(G + 1, 0);
  for (int64_t e = 0; e < N * 8; ++e) ++ptr[pidx[e] + 1];
  for (int64_t q = 0; q < G; ++q) ptr[q + 1] += ptr[q];
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1), node(N * 8);
  std::vector<float> wt(N * 8);
  for (int64_t e = 0; e < N * 8; ++e) {
    const int32_t q = pidx[e];
    node[fill[q]] = (int32_t)(e / 8);
    wt[fill[q]] = pw[e];
    ++fill[q];
  }
  pat_status st = upload_vec(filt, &g.filt);
  if (!st) st = upload_vec(tw, &g.twid);
  if (!st) st = upload_vec(pidx, &g.p_idx);
  if (!st) st = upload_vec(pw, &g.p_w);
  if (!st) st = upload_vec(ptr, &g.pt_ptr);
  if (!st) st = upload_vec(node, &g.pt_node);
  if (!st) st = upload_vec(wt, &g.pt_w);
  if (st) {
    free_grid(g);
    return st;
  }
  if (log2ng == 8) fft_allow_smem();
  pat_matern* m = new (std::nothrow) pat_matern;
  if (!m) {
    free_grid(g);
    set_error("pat_matern_create: out of host memory");
    return PAT_ENOMEM;
  }
  m->g = g;
  *out = m;
  return PAT_OK;
}

pat_status pat_matern_destroy(pat_matern* m) {
  clear_error();
  if (!m) return PAT_OK;
  free_grid(m->g);
  delete m;
  return PAT_OK;
}

pat_status pat_matern_workspace_bytes(const pat_mesh* mesh, const pat_matern* m, int32_t K, size_t* bytes) {
  clear_error();
  if (!mesh || !m || !bytes) {
    set_error("pat_matern_workspace_bytes: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_matern_workspace_bytes")) return PAT_EINVAL;
  *bytes = lat_layout(mesh->d, m->g, K).total;
  return PAT_OK;
}

static pat_status matern_ws_check(const pat_mesh* mesh, const pat_matern* m, int K, const void* ws, size_t bytes,
                                  const char* fn) {
  if (!mesh || !m) {
    set_error("%s: NULL mesh or prior", fn);
    return PAT_EINVAL;
  }
  if (bad_K(K, fn) || !check_device(mesh, fn)) return PAT_EINVAL;
  if (m->g.N != mesh->d.N) {
    set_error("%s: the prior was built for another mesh", fn);
    return PAT_EINVAL;
  }
  const size_t need = lat_layout(mesh->d, m->g, K).total;
  if (!ws || bytes < need || reinterpret_cast<uintptr_t>(ws) % 256) {
    set_error("%s: workspace %p of %zu bytes must be 256-byte aligned and hold %zu", fn, ws, bytes, need);
    return PAT_EINVAL;
  }
  return PAT_OK;
}

pat_status pat_matern_apply(const pat_mesh* mesh, const pat_matern* m, int32_t op, const float* in, int32_t K,
                            float* out, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  pat_status s = matern_ws_check(mesh, m, K, ws, ws_bytes, "pat_matern_apply");
  if (s) return s;
  if (!in || !out || op < 0 || op > 3) {
    set_error("pat_matern_apply: NULL field or op not in 0..3");
    return PAT_EINVAL;
  }
  const LatLayout L = lat_layout(mesh->d, m->g, K);
  char* w = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  switch (op) {
    case 0:
      return apply_T(m->g, in, K, out, nullptr, (float2*)(w + L.cbuf), st);
    case 1:
      return interp(m->g, in, K, out, st);
    case 2:
      return interp_t(m->g, in, K, out, st);
    default:  // P T
      s = apply_T(m->g, in, K, (float*)(w + L.tmp), nullptr, (float2*)(w + L.cbuf), st);
      if (s) return s;
      return interp(m->g, (const float*)(w + L.tmp), K, out, st);
  }
}

pat_status pat_matern_layout(const pat_mesh* mesh, const pat_matern* m, int32_t K, size_t* off) {
  clear_error();
  if (!mesh || !m || !off) {
    set_error("pat_matern_layout: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_matern_layout")) return PAT_EINVAL;
  const LatLayout L = lat_layout(mesh->d, m->g, K);
  const RtoLayout R = rto_layout(mesh->d, K);
  off[0] = L.x;
  off[1] = L.d;
  off[2] = L.r;
  off[3] = L.s;
  off[4] = L.gamma;
  off[5] = R.r_d;
  off[6] = R.status;
  return PAT_OK;
}

pat_status pat_rto_sample_matern(const pat_mesh* mesh, const pat_matern* m, const void* y_obs, double sigma, int32_t K,
                                 int32_t n_iter, const void* eta, const float* xi, uint64_t seed, double* z_samples,
                                 double* p_samples, double* mean, double* stdev, void* ws, size_t ws_bytes,
                                 void* stream) {
  PAT_RANGE("pat_rto_sample_matern");
  clear_error();
  pat_status s = matern_ws_check(mesh, m, K, ws, ws_bytes, "pat_rto_sample_matern");
  if (s) return s;
  if (!y_obs || n_iter < 0 || !(sigma > 0.0) || !std::isfinite(sigma)) {
    set_error("pat_rto_sample_matern: NULL y_obs, n_iter < 0 or sigma not finite and > 0");
    return PAT_EINVAL;
  }
  if (stdev && K < 2) {
    set_error("pat_rto_sample_matern: the std estimator needs K >= 2");
    return PAT_EINVAL;
  }
  const DeviceMesh& dm = mesh->d;
  const MaternGrid& g = m->g;
  const LatLayout L = lat_layout(dm, g, K);
  const RtoLayout R = rto_layout(dm, K);
  char* w = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t G = g.G, ndata = (int64_t)dm.n_steps * dm.n_obs;
  float *dz = (float*)(w + L.d), *rz = (float*)(w + L.r), *sz = (float*)(w + L.s), *tmp = (float*)(w + L.tmp);
  float2* cbuf = (float2*)(w + L.cbuf);
  double *x = (double*)(w + L.x), *gamma = (double*)(w + L.gamma), *alpha = (double*)(w + L.alpha),
         *pa = (double*)(w + L.part), *pb = pa + (size_t)L.nb * K;
  float *alphaf = (float*)(w + L.alphaf), *betaf = (float*)(w + L.betaf);
  const int lk = log2_or_neg(K);
  const unsigned vb = nblk((G * K + 3) / 4), vbd = nblk((ndata * K + 3) / 4);
  int* status = (int*)(w + R.status);
  float *node_in = (float*)(w + R.d), *node_out = (float*)(w + R.s), *q_d = (float*)(w + R.q_d),
        *r_d = (float*)(w + R.r_d);
  // r_d = y / sigma + eta (draws of stream 0 when eta is NULL), status, sigma
  PAT_TRY(begin_pre<float>(dm, (const float*)y_obs, sigma, K, (const float*)eta, nullptr, seed, w, st));
  lat_begin_kernel<<<nblk(G * K), 256, 0, st>>>(G, K, lk, xi, seed, (uint64_t)dm.first_sample, rz, x);
  // s = T P^T G^T r_d / sigma + r_p; d = s; gamma = ||s||^2
  auto transpose_into_s = [&]() -> pat_status {
    PAT_TRY(cgls_solve(dm, 1, K, sigma, w, st));
    PAT_TRY(interp_t(g, node_out, K, tmp, st));
    return apply_T(g, tmp, K, sz, rz, cbuf, st);
  };
  PAT_TRY(transpose_into_s());
  PAT_TRY(cuda_check(cudaMemcpyAsync(dz, sz, (size_t)G * K * 4, cudaMemcpyDeviceToDevice, st), "latent copy"));
  PAT_TRY(sq_partials(sz, G, K, L.nb, pa, st));
  gamma0_kernel<<<nblk((int64_t)K * 32, 128), 128, 0, st>>>(pa, L.nb, K, gamma, status);
  for (int it = 0; it < n_iter; ++it) {
    PAT_RANGE("latent CGLS iteration");
    // q_d = G P T d / sigma
    PAT_TRY(apply_T(g, dz, K, tmp, nullptr, cbuf, st));
    PAT_TRY(interp(g, tmp, K, node_in, st));
    PAT_TRY(cgls_solve(dm, 0, K, sigma, w, st));
    PAT_TRY(sq_partials(q_d, ndata, K, L.nb, pa, st));
    PAT_TRY(sq_partials(dz, G, K, L.nb, pb, st));
    alpha_kernel<<<nblk((int64_t)K * 32, 128), 128, 0, st>>>(pa, pb, L.nb, K, gamma, alpha, alphaf, status);
    lat_update_x_kernel<<<vb, 256, 0, st>>>(G * K, K, lk, alpha, alphaf, dz, x, rz);
    lat_axpy_kernel<<<vbd, 256, 0, st>>>(ndata * K, K, lk, alphaf, -1.0f, q_d, r_d, r_d);  // r_d -= alpha q_d
    PAT_TRY(transpose_into_s());
    PAT_TRY(sq_partials(sz, G, K, L.nb, pa, st));
    beta_kernel<<<nblk((int64_t)K * 32, 128), 128, 0, st>>>(pa, L.nb, K, gamma, betaf, status);
    lat_axpy_kernel<<<vb, 256, 0, st>>>(G * K, K, lk, betaf, 1.0f, dz, sz, dz);  // d = s + beta d
  }
  PAT_TRY(cuda_check(cudaGetLastError(), "pat_rto_sample_matern launch"));
  if (z_samples)
    PAT_TRY(cuda_check(cudaMemcpyAsync(z_samples, x, (size_t)G * K * 8, cudaMemcpyDeviceToDevice, st), "z copy"));
  if (p_samples || mean || stdev) {
    // nodal samples p = P T z (FP32 transform of the FP64 iterate) into the RTO
    // workspace's x field, from which the statistics kernel reads
    f64_to_f32_kernel<<<nblk(G * K), 256, 0, st>>>(G * K, x, sz);
    PAT_TRY(apply_T(g, sz, K, tmp, nullptr, cbuf, st));
    PAT_TRY(interp(g, tmp, K, node_in, st));
    f32_to_f64_kernel<<<nblk(g.N * K), 256, 0, st>>>(g.N * K, node_in, (double*)(w + R.x));
    PAT_TRY(cgls_finish(dm, K, p_samples, mean, stdev, w, st));
  }
  return cuda_check(cudaGetLastError(), "pat_rto_sample_matern launch");
}

}  // extern "C"
