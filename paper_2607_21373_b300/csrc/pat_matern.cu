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
//     Each block owns one grid line and a chunk of KC samples: the line's
//     n_g x KC complex values sit in shared memory (n_g = 128, KC = 32: 32 KB),
//     bit-reversed on load, then log2(n_g) radix-2 butterfly stages with a
//     twiddle table; every global access reads or writes KC contiguous floats of
//     one grid point.
//   - P (nodes <- grid) gathers 8 grid values per node; P^T (grid <- nodes)
//     gathers through a host-built grid -> node CSR of the same FP32 weights
//     (no atomics; exactly P's transpose).
//   - Latent CGLS: the wave solves are the mesh's (graph-replayed) forward and
//     transposed solves on an RTO workspace; the latent vectors x (FP64), d, r,
//     s (FP32) and every inner product, norm and scalar (FP64) are per sample.
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
  float2* twid = nullptr;    // [ng / 2] exp(-2 pi i j / ng)
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
// real output scale * Re + (addend or 0) (axis x).
// axis: 0 = x (stride n_g^2), 1 = y (stride n_g), 2 = z (stride 1) in grid points.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 FFT of the KC = 2^lkc lines in sh[ng][KC] (already
// bit-reversed); inverse uses the conjugate twiddles.  Index arithmetic by
// shifts and masks (n_g and KC are powers of two).
__device__ __forceinline__ void fft_stages(float2* sh, const float2* tw, int log2ng, int lkc, bool inverse) {
  const int nb = 1 << (log2ng - 1 + lkc);  // butterflies per stage
  const int kmask = (1 << lkc) - 1;
  for (int st = 1; st <= log2ng; ++st) {
    const int hmask = (1 << (st - 1)) - 1;
    const int tshift = log2ng - st;  // twiddle index stride n_g / 2^st
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int k = b & kmask;
      const int j = b >> lkc;  // butterfly index within the line, 0 .. ng/2-1
      const int pos = j & hmask;
      const int i0 = ((j >> (st - 1)) << st) + pos, i1 = i0 + hmask + 1;
      float2 w = tw[pos << tshift];
      if (inverse) w.y = -w.y;
      const float2 a = sh[(i0 << lkc) + k];
      const float2 c = cmul(w, sh[(i1 << lkc) + k]);
      sh[(i0 << lkc) + k] = make_float2(a.x + c.x, a.y + c.y);
      sh[(i1 << lkc) + k] = make_float2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int j, int bits) { return (int)(__brev((unsigned)j) >> (32 - bits)); }

template <int MODE>
// (in and out may be the same buffer: a block reads all of its line before it
// writes any of it, and no other block touches that line.)
__global__ void __launch_bounds__(256) fft_pass_kernel(const void* in, void* out,
                                                       const float* __restrict__ addend, int ng, int log2ng, int K,
                                                       int KC, int axis, const float2* __restrict__ tw,
                                                       const float* __restrict__ filt, float scale) {
  extern __shared__ float2 sh[];
  const int lkc = __ffs(KC) - 1, kmask = KC - 1;
  const int chunks = K / KC;
  const int64_t line = blockIdx.x / chunks;
  const int kc0 = (int)(blockIdx.x - line * chunks) * KC;
  // the two fixed coordinates of this line, and its first grid point and stride
  const int a = (int)(line / ng), b = (int)(line - (int64_t)a * ng);
  int64_t g0, stride;
  if (axis == 0) {
    g0 = (int64_t)a * ng + b;  // (0, a, b)
    stride = (int64_t)ng * ng;
  } else if (axis == 1) {
    g0 = (int64_t)a * ng * ng + b;  // (a, 0, b)
    stride = ng;
  } else {
    g0 = ((int64_t)a * ng + b) * ng;  // (a, b, 0)
    stride = 1;
  }
  const int n = ng * KC;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int j = e >> lkc, k = e & kmask;
    const int64_t off = (g0 + (int64_t)j * stride) * K + kc0 + k;
    float2 v;
    if constexpr (MODE == 0) {
      v = make_float2(static_cast<const float*>(in)[off], 0.0f);
    } else {
      v = static_cast<const float2*>(in)[off];
    }
    sh[(bitrev(j, log2ng) << lkc) + k] = v;
  }
  __syncthreads();
  fft_stages(sh, tw, log2ng, lkc, MODE >= 3);
  if constexpr (MODE == 2) {
    // multiply by sqrt(S) at (a, b, j), then inverse along z
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int j = e >> lkc, k = e & kmask;
      const float f = filt[g0 + j];
      const float2 v = sh[(j << lkc) + k];
      sh[(j << lkc) + k] = make_float2(f * v.x, f * v.y);
    }
    __syncthreads();
    // bit-reverse the filtered line for the inverse transform (in place, pairwise swaps)
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int j = e >> lkc, k = e & kmask;
      const int r = bitrev(j, log2ng);
      if (r > j) {
        const float2 t = sh[(j << lkc) + k];
        sh[(j << lkc) + k] = sh[(r << lkc) + k];
        sh[(r << lkc) + k] = t;
      }
    }
    __syncthreads();
    fft_stages(sh, tw, log2ng, lkc, true);
  }
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int j = e >> lkc, k = e & kmask;
    const int64_t off = (g0 + (int64_t)j * stride) * K + kc0 + k;
    const float2 v = sh[(j << lkc) + k];
    if constexpr (MODE == 4) {
      static_cast<float*>(out)[off] = scale * v.x + (addend ? addend[off] : 0.0f);
    } else {
      static_cast<float2*>(out)[off] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Interpolation and its transpose; one thread per (point, sample), so a warp's
// accesses to one grid point's or node's samples are contiguous.
// ---------------------------------------------------------------------------
__global__ void interp_kernel(int64_t N, int K, const int32_t* __restrict__ idx, const float* __restrict__ w,
                              const float* __restrict__ grid, float* __restrict__ nodes) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  const int64_t i = t / K;
  const int k = (int)(t - i * K);
  float acc = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc = fmaf(w[i * 8 + c], grid[(int64_t)idx[i * 8 + c] * K + k], acc);
  nodes[t] = acc;
}

__global__ void interp_t_kernel(int64_t G, int K, const int32_t* __restrict__ ptr, const int32_t* __restrict__ node,
                                const float* __restrict__ w, const float* __restrict__ vals,
                                float* __restrict__ grid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G * K) return;
  const int64_t g = t / K;
  const int k = (int)(t - g * K);
  float acc = 0.0f;
  for (int e = ptr[g]; e < ptr[g + 1]; ++e) acc = fmaf(w[e], vals[(int64_t)node[e] * K + k], acc);
  grid[t] = acc;
}

// ---------------------------------------------------------------------------
// Latent CGLS vector work (FP64 scalars per sample)
// ---------------------------------------------------------------------------
// partial[b][k] = sum over rows r = b, b + nb, b + 2 nb, ... of X[r][k]^2, in
// that order (deterministic); one thread per (block, sample), rows strided.
template <typename T>
__global__ void sq_partial_kernel(const T* __restrict__ X, int64_t rows, int K, int nb, double* __restrict__ part) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * K) return;
  const int b = (int)(t / K);
  const int k = (int)(t - (int64_t)b * K);
  double s = 0.0;
  for (int64_t r = b; r < rows; r += nb) {
    const double v = (double)X[r * K + k];
    s += v * v;
  }
  part[t] = s;
}

__device__ __forceinline__ double colsum(const double* part, int nb, int K, int k) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * K + k];
  return s;
}

__device__ __forceinline__ bool bad(double v) { return !(v > 0.0) || !isfinite(v); }

// gamma = ||s||^2 (begin)
__global__ void gamma0_kernel(const double* part, int nb, int K, double* gamma, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double g = colsum(part, nb, K, k);
  if (!isfinite(g)) atomicExch(status, (int)PAT_ENUMERIC);
  gamma[k] = g;
}

// alpha = gamma / (||q_d||^2 + ||d||^2)
__global__ void alpha_kernel(const double* pq, const double* pd, int nb, int K, const double* gamma, double* alpha,
                             int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double qq = colsum(pq, nb, K, k) + colsum(pd, nb, K, k);
  double a = 0.0;
  if (gamma[k] > 0.0) {
    if (bad(qq)) atomicExch(status, (int)PAT_ENUMERIC);
    else a = gamma[k] / qq;
  }
  alpha[k] = a;
}

// beta = ||s||^2 / gamma; gamma = ||s||^2
__global__ void beta_kernel(const double* part, int nb, int K, double* gamma, double* beta, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double g = colsum(part, nb, K, k);
  double b = 0.0;
  if (!isfinite(g)) atomicExch(status, (int)PAT_ENUMERIC);
  else if (gamma[k] > 0.0) b = g / gamma[k];
  beta[k] = b;
  gamma[k] = g;
}

// x += alpha d (FP64); r_p -= alpha d  (q_p = d for the identity prior block)
__global__ void lat_update_x_kernel(int64_t rows, int K, const double* __restrict__ alpha, const float* __restrict__ d,
                                    double* __restrict__ x, float* __restrict__ rp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * K) return;
  const double a = alpha[t % K];
  const double dv = (double)d[t];
  x[t] += a * dv;
  rp[t] = (float)((double)rp[t] - a * dv);
}

// r_d -= alpha q_d
__global__ void lat_update_rd_kernel(int64_t rows, int K, const double* __restrict__ alpha,
                                     const float* __restrict__ q, float* __restrict__ r) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * K) return;
  r[t] = (float)((double)r[t] - alpha[t % K] * (double)q[t]);
}

// d = s + beta d
__global__ void lat_update_d_kernel(int64_t rows, int K, const double* __restrict__ beta, const float* __restrict__ s,
                                    float* __restrict__ d) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * K) return;
  d[t] = (float)((double)s[t] + beta[t % K] * (double)d[t]);
}

// latent prior draws: r_p[g][k] = xi (given) or the library draw of stream 1
// (the prior-draw stream) at element g for sample first + k; x = 0
__global__ void lat_begin_kernel(int64_t rows, int K, const float* __restrict__ xi, uint64_t seed, uint64_t first,
                                 float* __restrict__ rp, double* __restrict__ x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * K) return;
  const int64_t g = t / K;
  const uint64_t k = first + (uint64_t)(t - g * K);
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
  size_t rto, x, d, r, s, tmp, cbuf, gamma, alpha, beta, part, total;
  int nb;
};
LatLayout lat_layout(const DeviceMesh& m, const MaternGrid& g, int K) {
  LatLayout L{};
  L.nb = std::min<int64_t>(1024, std::max<int64_t>(1, g.G / 64));
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
  L.beta = o; o = a256(o + K * 8);
  L.part = o; o = a256(o + (size_t)2 * L.nb * K * 8);
  L.total = o;
  return L;
}

// out = T in (in, out real [G][K]); out may alias addend; cbuf complex [G][K]
pat_status apply_T(const MaternGrid& g, const float* in, int K, float* out, const float* addend, float2* cbuf,
                   cudaStream_t st) {
  const int KC = fft_kc(K);
  const int64_t lines = (int64_t)g.ng * g.ng;
  const unsigned blocks = (unsigned)(lines * (K / KC));
  const size_t smem = (size_t)g.ng * KC * sizeof(float2);
  const float scale = (float)(1.0 / (double)g.G);
  fft_pass_kernel<0><<<blocks, 256, smem, st>>>(in, cbuf, nullptr, g.ng, g.log2ng, K, KC, 0, g.twid, g.filt, 1.0f);
  fft_pass_kernel<1><<<blocks, 256, smem, st>>>(cbuf, cbuf, nullptr, g.ng, g.log2ng, K, KC, 1, g.twid, g.filt, 1.0f);
  fft_pass_kernel<2><<<blocks, 256, smem, st>>>(cbuf, cbuf, nullptr, g.ng, g.log2ng, K, KC, 2, g.twid, g.filt, 1.0f);
  fft_pass_kernel<3><<<blocks, 256, smem, st>>>(cbuf, cbuf, nullptr, g.ng, g.log2ng, K, KC, 1, g.twid, g.filt, 1.0f);
  fft_pass_kernel<4><<<blocks, 256, smem, st>>>(cbuf, out, addend, g.ng, g.log2ng, K, KC, 0, g.twid, g.filt, scale);
  return cuda_check(cudaGetLastError(), "Matern T launch");
}

pat_status interp(const MaternGrid& g, const float* grid, int K, float* nodes, cudaStream_t st) {
  interp_kernel<<<nblk(g.N * K), 256, 0, st>>>(g.N, K, g.p_idx, g.p_w, grid, nodes);
  return cuda_check(cudaGetLastError(), "Matern P launch");
}

pat_status interp_t(const MaternGrid& g, const float* nodes, int K, float* grid, cudaStream_t st) {
  interp_t_kernel<<<nblk(g.G * K), 256, 0, st>>>(g.G, K, g.pt_ptr, g.pt_node, g.pt_w, nodes, grid);
  return cuda_check(cudaGetLastError(), "Matern P^T launch");
}

pat_status sq_partials(const float* X, int64_t rows, int K, int nb, double* part, cudaStream_t st) {
  sq_partial_kernel<float><<<nblk((int64_t)nb * K), 256, 0, st>>>(X, rows, K, nb, part);
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
  std::vector<float2> tw(ng / 2);
  for (int64_t j = 0; j < ng / 2; ++j) {
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
  const size_t smem = (size_t)ng * 32 * sizeof(float2);
  if (smem > 48 * 1024) {
    const void* fns[5] = {(const void*)fft_pass_kernel<0>, (const void*)fft_pass_kernel<1>,
                          (const void*)fft_pass_kernel<2>, (const void*)fft_pass_kernel<3>,
                          (const void*)fft_pass_kernel<4>};
    for (const void* f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
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

pat_status pat_rto_sample_matern(const pat_mesh* mesh, const pat_matern* m, const void* y_obs, double sigma, int32_t K,
                                 int32_t n_iter, const void* eta, const float* xi, uint64_t seed, double* z_samples,
                                 double* p_samples, double* mean, double* stdev, void* ws, size_t ws_bytes,
                                 void* stream) {
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
         *beta = (double*)(w + L.beta), *pa = (double*)(w + L.part), *pb = pa + (size_t)L.nb * K;
  int* status = (int*)(w + R.status);
  float *node_in = (float*)(w + R.d), *node_out = (float*)(w + R.s), *q_d = (float*)(w + R.q_d),
        *r_d = (float*)(w + R.r_d);
  // r_d = y / sigma + eta (draws of stream 0 when eta is NULL), status, sigma
  PAT_TRY(begin_pre<float>(dm, (const float*)y_obs, sigma, K, (const float*)eta, nullptr, seed, w, st));
  lat_begin_kernel<<<nblk(G * K), 256, 0, st>>>(G, K, xi, seed, (uint64_t)dm.first_sample, rz, x);
  // s = T P^T G^T r_d / sigma + r_p; d = s; gamma = ||s||^2
  auto transpose_into_s = [&]() -> pat_status {
    PAT_TRY(cgls_solve(dm, 1, K, sigma, w, st));
    PAT_TRY(interp_t(g, node_out, K, tmp, st));
    return apply_T(g, tmp, K, sz, rz, cbuf, st);
  };
  PAT_TRY(transpose_into_s());
  PAT_TRY(cuda_check(cudaMemcpyAsync(dz, sz, (size_t)G * K * 4, cudaMemcpyDeviceToDevice, st), "latent copy"));
  PAT_TRY(sq_partials(sz, G, K, L.nb, pa, st));
  gamma0_kernel<<<nblk(K, 128), 128, 0, st>>>(pa, L.nb, K, gamma, status);
  for (int it = 0; it < n_iter; ++it) {
    // q_d = G P T d / sigma
    PAT_TRY(apply_T(g, dz, K, tmp, nullptr, cbuf, st));
    PAT_TRY(interp(g, tmp, K, node_in, st));
    PAT_TRY(cgls_solve(dm, 0, K, sigma, w, st));
    PAT_TRY(sq_partials(q_d, ndata, K, L.nb, pa, st));
    PAT_TRY(sq_partials(dz, G, K, L.nb, pb, st));
    alpha_kernel<<<nblk(K, 128), 128, 0, st>>>(pa, pb, L.nb, K, gamma, alpha, status);
    lat_update_x_kernel<<<nblk(G * K), 256, 0, st>>>(G, K, alpha, dz, x, rz);
    lat_update_rd_kernel<<<nblk(ndata * K), 256, 0, st>>>(ndata, K, alpha, q_d, r_d);
    PAT_TRY(transpose_into_s());
    PAT_TRY(sq_partials(sz, G, K, L.nb, pa, st));
    beta_kernel<<<nblk(K, 128), 128, 0, st>>>(pa, L.nb, K, gamma, beta, status);
    lat_update_d_kernel<<<nblk(G * K), 256, 0, st>>>(G, K, beta, sz, dz);
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
