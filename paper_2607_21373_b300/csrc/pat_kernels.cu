// Launchers of the time-step kernels and the batched CGLS driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "pat_kernels.cuh"
#include "pat_tile.cuh"
#include "pat_wide.cuh"
#include "pat_solver.cuh"

namespace pat {

pat_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PAT_OK;
  set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
  return PAT_ECUDA;
}


int sm_count() {
  int dev = 0, n = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

// Profiling hooks (no-ops unless pat_profile_enable was called on the mesh).
static void* prof_event(const DeviceMesh& m, size_t idx) {
  Profiler& P = m.prof;
  while (P.events.size() <= idx) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    P.events.push_back((void*)e);
  }
  return P.events[idx];
}
static size_t prof_begin(const DeviceMesh& m, int kind, cudaStream_t st) {
  Profiler& P = m.prof;
  if (!P.on) return (size_t)-1;
  const size_t pair = P.used++;
  void* e = prof_event(m, 2 * pair);
  prof_event(m, 2 * pair + 1);
  if (P.kind.size() <= pair) P.kind.resize(pair + 1);
  P.kind[pair] = kind;
  if (e) cudaEventRecord((cudaEvent_t)e, st);
  return pair;
}
static void prof_end(const DeviceMesh& m, size_t pair, int64_t launches, cudaStream_t st) {
  Profiler& P = m.prof;
  if (!P.on || pair == (size_t)-1) return;
  void* e = prof_event(m, 2 * pair + 1);
  if (e) cudaEventRecord((cudaEvent_t)e, st);
  (P.kind[pair] == 0 ? P.fwd_launches : P.adj_launches) += launches;
  P.total_launches += launches;
}
static inline void count(const DeviceMesh& m, int64_t n) {
  if (m.prof.on) m.prof.total_launches += n;
}

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
static inline size_t real_size(const DeviceMesh& m) { return m.prec == PAT_F64 ? 8 : 4; }

size_t state_bytes(const DeviceMesh& m, int K) { return align256(4 * (size_t)m.N * K * real_size(m)); }

// Widest per-thread vector that divides K and keeps every access aligned.
template <typename T>
static int pick_vec(int K, std::initializer_list<const void*> ptrs) {
  int V = (sizeof(T) == 4) ? 8 : 2;
  while (V > 1) {
    bool ok = (K % V) == 0;
    for (const void* p : ptrs)
      if (p && (reinterpret_cast<uintptr_t>(p) % (V * sizeof(T))) != 0) ok = false;
    if (ok) break;
    V /= 2;
  }
  return V;
}

template <typename T, int V, bool SPLIT>
static void launch_fwd(const FwdArgs<T>& a, int64_t threads, cudaStream_t st) {
  const int64_t blocks = (threads + 255) / 256;
  fwd_step_kernel<T, V, SPLIT><<<(unsigned)blocks, 256, 0, st>>>(a);
}
template <typename T, int V, bool SPLIT>
static void launch_adj(const AdjArgs<T>& a, cudaStream_t st) {
  const int64_t blocks = (a.row_threads + 255) / 256;
  adj_step_kernel<T, V, SPLIT><<<(unsigned)blocks, 256, 0, st>>>(a);
}

template <typename T, int V, bool SPLIT>
static pat_status forward_t(const DeviceMesh& m, const T* p0, int K, T* Y, T scale, T* ws, cudaStream_t st) {
  const int64_t NK = m.N * (int64_t)K;
  T* a[2] = {ws, ws + 2 * NK};
  T* w[2] = {ws + NK, ws + 3 * NK};
  FwdArgs<T> A{};
  A.N = m.N;
  A.K = K;
  A.n_obs = m.n_obs;
  A.row_threads = NK / V;
  A.ptr = m.fwd.ptr;
  A.col = m.fwd.col;
  A.hi = static_cast<const T*>(m.fwd.hi);
  A.lo = m.fwd.lo;
  A.det_node = m.det_node;
  A.det_w = static_cast<const T*>(m.det_w);
  A.scale = scale;
  const int64_t obs_threads = (int64_t)m.n_obs * K / V;
  const int64_t ystride = (int64_t)m.n_obs * K;
  const size_t pp = prof_begin(m, 0, st);
  for (int s = 0; s < m.n_steps; ++s) {
    A.a_in = (s == 0) ? p0 : a[(s - 1) & 1];
    A.w_in = (s == 0) ? nullptr : w[(s - 1) & 1];
    A.a_out = a[s & 1];
    A.w_out = w[s & 1];
    A.y_out = (s == 0) ? nullptr : Y + (int64_t)(s - 1) * ystride;  // observation of state s
    launch_fwd<T, V, SPLIT>(A, A.row_threads + (s == 0 ? 0 : obs_threads), st);
  }
  // observation of the final state N_T
  A.a_in = a[(m.n_steps - 1) & 1];
  A.w_in = w[(m.n_steps - 1) & 1];
  A.a_out = nullptr;
  A.w_out = nullptr;
  A.y_out = Y + (int64_t)(m.n_steps - 1) * ystride;
  FwdArgs<T> G = A;
  G.row_threads = 0;
  launch_fwd<T, V, SPLIT>(G, obs_threads, st);
  prof_end(m, pp, m.n_steps + 1, st);
  return cuda_check(cudaGetLastError(), "forward step launch");
}

template <typename T, int V, bool SPLIT>
static pat_status adjoint_t(const DeviceMesh& m, const T* Yhat, int K, T* out, T scale, T* ws, cudaStream_t st) {
  const int64_t NK = m.N * (int64_t)K;
  T* ah[2] = {ws, ws + 2 * NK};
  T* u[2] = {ws + NK, ws + 3 * NK};
  AdjArgs<T> A{};
  A.N = m.N;
  A.K = K;
  A.row_threads = NK / V;
  A.ptr = m.adj.ptr;
  A.col = m.adj.col;
  A.hi = static_cast<const T*>(m.adj.hi);
  A.lo = m.adj.lo;
  A.minv_hi = static_cast<const T*>(m.minv_hi);
  A.minv_lo = m.minv_lo;
  A.inj_scale = scale;
  const int64_t ystride = (int64_t)m.n_obs * K;
  const int NT = m.n_steps;
  // zero state + injection of the last observation time
  const size_t pp = prof_begin(m, 1, st);
  A.ah_in = nullptr;
  A.u_in = nullptr;
  A.ah_out = ah[0];
  A.u_out = u[0];
  A.yhat = Yhat + (int64_t)(NT - 1) * ystride;
  launch_adj<T, V, SPLIT>(A, st);
  int cur = 0;
  for (int mstep = NT; mstep >= 1; --mstep) {
    A.ah_in = ah[cur];
    A.u_in = u[cur];
    A.ah_out = (mstep == 1 && out) ? out : ah[cur ^ 1];
    A.u_out = u[cur ^ 1];
    A.yhat = (mstep >= 2) ? Yhat + (int64_t)(mstep - 2) * ystride : nullptr;
    launch_adj<T, V, SPLIT>(A, st);
    cur ^= 1;
  }
  prof_end(m, pp, NT + 1, st);
  return cuda_check(cudaGetLastError(), "adjoint step launch");
}

// Largest CSR range covered by one 256-thread block of a row phase with KV
// threads per row (cached per mesh, direction and KV).
int stage_span(const DeviceMesh& m, bool adj, int KV) {
  std::lock_guard<std::mutex> lock(m.stage_mutex);
  auto key = std::make_pair(adj ? 1 : 0, KV);
  auto it = m.stage_span.find(key);
  if (it != m.stage_span.end()) return it->second;
  const std::vector<int32_t>& ptr = adj ? m.adj3_ptr_h : m.fwd_ptr_h;
  const int64_t rows_threads = m.N * (int64_t)KV;
  int span = 0;
  for (int64_t tb0 = 0; tb0 < rows_threads; tb0 += 256) {
    const int64_t r0 = tb0 / KV;
    const int64_t r1 = (std::min(tb0 + 256, rows_threads) - 1) / KV;
    span = std::max(span, ptr[r1 + 1] - ptr[r0]);
  }
  m.stage_span[key] = span;
  return span;
}

// Shared-memory staging pays when several threads share a row and the block's
// rows fit in 48 KB.
template <typename T, bool SPLIT>
static int stage_cap_for(const DeviceMesh& m, bool adj, int K, int V) {
  const int KV = K / V;
  if (KV < 2) return 0;
  const int span = stage_span(m, adj, KV);
  return stage_bytes<T, SPLIT>(span) <= 48 * 1024 ? span : 0;
}

// Variant selection: a forced variant (autotuning probes) wins, then the
// autotuned one for (direction, K), then the default (widest vector, staged).
namespace {
thread_local bool g_force_on = false;
thread_local TuneCfg g_force;
}  // namespace

static bool variant(const DeviceMesh& m, int dir, int K, TuneCfg* out) {
  if (g_force_on) {
    *out = g_force;
    return true;
  }
  std::lock_guard<std::mutex> lock(m.tune_mutex);
  auto it = m.tuned.find(std::make_pair(dir, K));
  if (it == m.tuned.end()) return false;
  *out = it->second;
  return true;
}

// Tile-staged launch (variant packed == 2): one block per 32-row tile plus
// gather blocks; its shared memory holds the tile's staged source rows.
template <bool ADJ>
static bool launch_tiled(const DeviceMesh& m, const Step3Args<float>& a, cudaStream_t st) {
  // the tiles update every row: launches without rows to update (the final
  // observation-only launch of a forward solve) and the zero-state adjoint start
  // go to the packed kernel
  if (a.x == nullptr || a.xn == nullptr || a.row_threads == 0 || a.K % 8 || a.K > 8 * 1024 / kTileRows ||
      !m.fwd.hl || m.n_tiles == 0 || !m.row_order)
    return false;
  const size_t smem = 128 + (size_t)m.tile_max_slots * a.K * 4;
  if (smem > 200 * 1024) return false;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(step3t_kernel<8, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  TileArgs Tl{m.tile_range_ptr, m.tile_range_src, m.tile_range_cnt, m.tile_range_slot, m.tile_slots,
              ADJ ? m.tile_slot_adj : m.tile_slot_fwd, m.d_status, m.n_tiles, m.row_order, m.tile_wait_cycles};
  Step3Args<float> A = a;
  A.hl = ADJ ? m.adj3.hl : m.fwd.hl;
  const int bdim = kTileRows * (a.K / 8);
  const int64_t gather_threads = (!ADJ && a.y_out) ? (int64_t)a.n_obs * (a.K / 8) : 0;
  const int64_t blocks = m.n_tiles + (gather_threads + bdim - 1) / bdim;
  step3t_kernel<8, ADJ><<<(unsigned)blocks, bdim, smem, st>>>(A, Tl);
  return true;
}

// Persistent double-buffered tile launch (variant packed == 4): enough blocks
// to fill every SM, each walking a strided subset of the tiles.
template <bool ADJ>
static bool launch_pipelined(const DeviceMesh& m, const Step3Args<float>& a, cudaStream_t st) {
  if (a.x == nullptr || a.xn == nullptr || a.row_threads == 0 || a.K % 8 || a.K > 8 * 512 / kTileRows ||
      !m.fwd.hl || m.n_tiles == 0 || !m.row_order)
    return false;
  const size_t smem = 128 + 2 * (size_t)m.tile_max_slots * a.K * 4;
  if (smem > 220 * 1024) return false;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(step3p_kernel<ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const int bdim = kTileRows * (a.K / 8);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step3p_kernel<ADJ>, bdim, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  TileArgs Tl{m.tile_range_ptr, m.tile_range_src, m.tile_range_cnt, m.tile_range_slot, m.tile_slots,
              ADJ ? m.tile_slot_adj : m.tile_slot_fwd, m.d_status, m.n_tiles, m.row_order, m.tile_wait_cycles};
  Step3Args<float> A = a;
  A.hl = ADJ ? m.adj3.hl : m.fwd.hl;
  const int blocks = std::min(m.n_tiles, per_sm * sm_count());
  step3p_kernel<ADJ><<<(unsigned)blocks, bdim, smem, st>>>(A, Tl, m.tile_max_slots);
  return true;
}

// Resident blocks per SM of kernel `fn` with `bdim`-thread blocks (cached).
static int resident_blocks(const void* fn, int bdim) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({fn, bdim});
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bdim, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  // The step kernels live on L1 hits of the neighbour gathers: ask for the
  // smallest shared-memory carveout that still holds the static shared memory
  // of the blocks found resident (the default may reserve far more, e.g. a
  // 132 KB carveout for 68 KB of blocks), so the rest of the SM's 256 KB stays
  // L1; kept only if the occupancy does not change.
  cudaFuncAttributes fa{};
  int dev = 0, smem_sm = 0, reserved = 0;
  if (per_sm > 0 && cudaFuncGetAttributes(&fa, fn) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
      smem_sm > 0) {
    const int64_t need = (int64_t)per_sm * ((int64_t)fa.sharedSizeBytes + reserved);
    const int pct = (int)std::min<int64_t>(100, (need * 100 + smem_sm - 1) / smem_sm);
    int after = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&after, fn, bdim, 0) != cudaSuccess || after < per_sm)
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutDefault);
  }
  cudaGetLastError();
  cache[{fn, bdim}] = per_sm;
  return per_sm;
}

// Rows covered by one resident wave of kernel `fn` launched with `bdim`-thread
// blocks, KV threads per row (the L2 prefetch distance of one wave).
static int64_t wave_rows(const void* fn, int bdim, int KV) {
  return (int64_t)resident_blocks(fn, bdim) * sm_count() * bdim / std::max(KV, 1);
}

// Persistent fixed-width launch: one resident wave of blocks (c.persist 1:
// grid-stride chunks; 2: one contiguous slab of chunks per block; 3: grid-stride
// with staged row metadata), optionally
// as a programmatic dependent of the previous kernel on the stream.
template <int V, bool ADJ, bool W>
static void launch_persist(Step3Args<float> a, const TuneCfg& c, int64_t threads, cudaStream_t st) {
  const int64_t n_chunks = (threads + 31) / 32;
  const int bs = (c.big && c.persist == 1) ? 1024 : 256;
  void (*kern)(const Step3Args<float>, int64_t) =
      c.persist == 2 ? step3e_slab_kernel<V, ADJ, W>
      : bs == 1024   ? step3e_persist_kernel<V, ADJ, W, 1024>
                     : step3e_persist_kernel<V, ADJ, W, 256>;
  if constexpr (V == 8 && !W) {
    if (c.hint && c.persist == 1 && bs == 256) kern = step3e_persist_kernel<V, ADJ, false, 256, true>;
    // metadata staged through shared memory: at most kStageRows rows per 32-thread chunk
    if (c.persist == 3 && a.K / V >= 4 && !a.order) kern = step3e_stage_kernel<ADJ>;
    if (c.batch && c.persist == 1 && bs == 256 && !c.hint) {
      if (c.batch == 8)
        kern = step3e_persist_kernel<V, ADJ, false, 256, false, 8, 2>;
      else if (c.batch == 2 && c.minb == 6)
        kern = step3e_persist_kernel<V, ADJ, false, 256, false, 2, 6>;
      else if (c.batch == 2)
        kern = step3e_persist_kernel<V, ADJ, false, 256, false, 2, 5>;
      else if (c.batch == 4 && c.minb == 5)
        kern = step3e_persist_kernel<V, ADJ, false, 256, false, 4, 5, true>;
      else if (c.batch == 4)
        kern = step3e_persist_kernel<V, ADJ, false, 256, false, 4, 4, true>;
    }
  }
  const int per_sm = std::max(1, resident_blocks((const void*)kern, bs));
  const int64_t grid =
      std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sm_count(), (n_chunks + bs / 32 - 1) / (bs / 32)));
  a.pf_rows = (c.pf && !a.order) ? c.pf : 0;
  if (c.pdl) {  // overlap this grid's start with the previous step's drain
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)bs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, a, n_chunks) == cudaSuccess) return;
    cudaGetLastError();  // attribute refused: plain launch
  }
  kern<<<(unsigned)grid, (unsigned)bs, 0, st>>>(a, n_chunks);
}

// 16-slot fixed-width launch (variant packed == 5): persistent grid-stride
// blocks as a programmatic dependent of the previous step.  c.batch: source
// rows per gather round (4 or 8); c.early: each round's columns loaded with
// it; c.big: 1024-thread blocks; c.minb: 3 asks for 3 resident blocks of 256.
template <bool ADJ, bool QUAD>
static void (*pick_wide(const TuneCfg& c, int* bs))(const Step3Args<float>, int64_t) {
  *bs = 256;
  if (c.big) {
    *bs = 1024;
    return step3w_persist_kernel<ADJ, 4, true, 1024, 1, 2, QUAD>;
  }
  if (c.batch == 8) {
    return c.minb == 3 ? step3w_persist_kernel<ADJ, 8, true, 256, 3, 2, QUAD>
           : c.early   ? step3w_persist_kernel<ADJ, 8, true, 256, 2, 2, QUAD>
                       : step3w_persist_kernel<ADJ, 8, false, 256, 2, 2, QUAD>;
  }
  if constexpr (QUAD) {
    if (c.pfm) {  // the quad's coefficient lines prefetched into L1; serial tail
      if (c.own)
        return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, true, 1, true>
                       : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, true, 1, true>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, true, 0, true>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, true, 0, true>;
    }
  }
  if constexpr (!QUAD) {
    if (c.pfm) {
      if (c.own) return step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, 1, true>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, false, true>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, false, true>;
    }
  }
  if constexpr (!QUAD) {
    if (c.own == 2) {
      if (c.tail)
        return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 2>
                       : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, 2>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, false, 2>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 2, false, 2>;
    }
  }
  if constexpr (!QUAD) {
    if (c.dyn) {  // chunks handed out by an atomic counter (own rows by cp.async, serial tail)
      if (c.own)
        return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 1, false, true>
                       : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, 1, false, true>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 0, false, true>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, 0, false, true>;
    }
  }
  if constexpr (!QUAD) {
    if (c.own == 3) {  // own x_{s-1} rows only by cp.async
      if (c.tail)
        return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 3>
                       : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, false, 3>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, false, 3>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 2, false, 3>;
    }
    if (c.minb == 3 && c.own == 1) {  // 3 blocks of 256 per SM: up to 85 registers a thread
      if (c.tail)
        return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 3, 1, false, 1>
                       : step3w_persist_kernel<ADJ, 4, false, 256, 3, 1, false, 1>;
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 3, 2, false, 1>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 3, 2, false, 1>;
    }
    if (c.wide && c.early) {  // 256-bit metadata loads (own rows by cp.async when c.own)
      if (c.own)
        return c.tail ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 1, false, false, true>
                      : step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, false, 1, false, false, true>;
      return c.tail ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, false, 0, false, false, true>
                    : step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, false, 0, false, false, true>;
    }
  }
  if (c.own) {
    if (c.tail)
      return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, QUAD, 1>
                     : step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, QUAD, 1>;
    return c.early ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, QUAD, 1>
                   : step3w_persist_kernel<ADJ, 4, false, 256, 4, 2, QUAD, 1>;
  }
  if (c.early)
    return c.tail ? step3w_persist_kernel<ADJ, 4, true, 256, 4, 1, QUAD> : step3w_persist_kernel<ADJ, 4, true, 256, 4, 2, QUAD>;
  return c.tail ? step3w_persist_kernel<ADJ, 4, false, 256, 4, 1, QUAD> : step3w_persist_kernel<ADJ, 4, false, 256, 4, 2, QUAD>;
}

template <bool ADJ>
static void launch_wide(Step3Args<float> a, const TuneCfg& c, int64_t threads, cudaStream_t st) {
  const int64_t n_chunks = (threads + 31) / 32;
  int bs = 256;
  void (*kern)(const Step3Args<float>, int64_t) =
      c.packed == 6 ? pick_wide<ADJ, false>(c, &bs) : pick_wide<ADJ, true>(c, &bs);
  const int per_sm = std::max(1, resident_blocks((const void*)kern, bs));
  const int64_t grid =
      std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sm_count(), (n_chunks + bs / 32 - 1) / (bs / 32)));
  a.pf_rows = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.pdl ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kern, a, n_chunks) == cudaSuccess) return;
  cudaGetLastError();  // attribute refused: plain launch
  kern<<<(unsigned)grid, (unsigned)bs, 0, st>>>(a, n_chunks);
}

// Row-pair launch (variant packed == 7): persistent grid-stride blocks over the
// pairs' chunks, as a programmatic dependent of the previous step.
template <bool ADJ>
static void launch_pairs(Step3Args<float> a, const TuneCfg& c, int64_t threads, cudaStream_t st) {
  const int KV = a.K / 8;
  const int64_t gather = threads - a.row_threads;  // sensor-gather threads
  a.row_threads = a.row_threads > 0 ? (a.N + 1) / 2 * KV : 0;
  const int64_t n_chunks = (a.row_threads + gather + 31) / 32;
  const int bs = 256;
  void (*kern)(const Step3Args<float>, int64_t) =
      c.minb == 3 ? step3u_persist_kernel<ADJ, 256, 3> : step3u_persist_kernel<ADJ, 256, 2>;
  const int per_sm = std::max(1, resident_blocks((const void*)kern, bs));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sm_count(), (n_chunks + 7) / 8));
  a.pf_rows = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.pdl ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kern, a, n_chunks) == cudaSuccess) return;
  cudaGetLastError();
  kern<<<(unsigned)grid, (unsigned)bs, 0, st>>>(a, n_chunks);
}

// Row-quad launch (variant packed == 8, K = 64): persistent grid-stride blocks
// over the quads' chunks (then the sensor-gather chunks), as a programmatic
// dependent of the previous step.  c.own: the rows' own values by cp.async.
template <bool ADJ>
static void launch_quads(Step3Args<float> a, const TuneCfg& c, int64_t threads, cudaStream_t st) {
  const int64_t n_chunks = (threads + 31) / 32;
  const int bs = 256;
  void (*kern)(const Step3Args<float>, int64_t) =
      c.own ? step3q_persist_kernel<ADJ, true> : step3q_persist_kernel<ADJ, false>;
  const int per_sm = std::max(1, resident_blocks((const void*)kern, bs));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sm_count(), (n_chunks + 7) / 8));
  a.pf_rows = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.pdl ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, kern, a, n_chunks) == cudaSuccess) return;
  cudaGetLastError();
  kern<<<(unsigned)grid, (unsigned)bs, 0, st>>>(a, n_chunks);
}

template <typename T, int V, bool SPLIT, bool ADJ>
static void launch_step3(const DeviceMesh& m, Step3Args<T> a, int64_t threads, cudaStream_t st) {
  const int64_t blocks = (threads + 255) / 256;
  TuneCfg c;  // defaults: packed, unstaged
  variant(m, ADJ ? 1 : 0, a.K, &c);
  if constexpr (sizeof(T) == 4 && SPLIT && V == 8) {
    if (c.packed == 2 && launch_tiled<ADJ>(m, a, st)) return;
    if (c.packed == 4 && launch_pipelined<ADJ>(m, a, st)) return;
  }
  if constexpr (sizeof(T) == 4 && SPLIT && (V == 1 || V == 8)) {
    const DevCSR& E = ADJ ? m.adj3 : m.fwd;
    if constexpr (V == 8) {
      if (c.packed == 8 && E.quad_col && E.w16r_col && a.K == 64) {  // row quads
        a.quad_ptr = E.quad_ptr;
        a.quad_n = E.quad_n;
        a.quad_col = E.quad_col;
        a.quad_cf = E.quad_cf;
        a.ell_desc = E.ell_desc;
        a.ovf_ptr = E.w16_ovf_ptr;
        a.ovf_col = E.w16_ovf_col;
        a.ovf_hl = E.w16_ovf_hl;
        launch_quads<ADJ>(a, c, threads, st);
        return;
      }
      if (c.packed == 7 && E.pair_col && E.w16r_col) {  // row pairs
        a.pair_col = E.pair_col;
        a.pair_cf = E.pair_cf;
        a.pair_n = E.pair_n;
        a.ell_col = E.w16r_col;
        a.ell_hl = E.w16r_hl;
        a.ell_desc = E.ell_desc;
        a.ovf_ptr = E.w16_ovf_ptr;
        a.ovf_col = E.w16_ovf_col;
        a.ovf_hl = E.w16_ovf_hl;
        launch_pairs<ADJ>(a, c, threads, st);
        return;
      }
    }
    if ((c.packed == 5 || (c.packed == 6 && V == 8)) && E.w16_col && (V == 8 || a.K == 1)) {  // 16-slot rows
      a.ell_col = c.packed == 6 ? E.w16r_col : E.w16_col;
      a.ell_hl = c.packed == 6 ? E.w16r_hl : E.w16_hl;
      a.ell_desc = E.ell_desc;
      a.ovf_ptr = E.w16_ovf_ptr;
      a.ovf_col = E.w16_ovf_col;
      a.ovf_hl = E.w16_ovf_hl;
      a.status = m.d_status;
      a.wait_cycles = m.tile_wait_cycles;
      if constexpr (V == 1) {
        if (c.minb == 6)
          step3w1_kernel<ADJ, 6><<<(unsigned)blocks, 256, 0, st>>>(a);
        else
          step3w1_kernel<ADJ><<<(unsigned)blocks, 256, 0, st>>>(a);
      } else {
        // the transposed kernel's extra threads prepare the next launch's sensor terms
        const int64_t prep = (ADJ && a.inj_next) ? a.n_inj * (a.K / 8) : 0;
        launch_wide<ADJ>(a, c, threads + prep, st);
      }
      return;
    }
  }
  if constexpr (sizeof(T) == 4 && SPLIT && V == 1) {
    const DevCSR& E = ADJ ? m.adj3 : m.fwd;
    if (c.packed == 3 && E.ell_col && a.K == 1) {  // fixed-width rows, one sample
      a.ell_col = E.ell_col;
      a.ell_hl = E.ell_hl;
      a.ell_desc = E.ell_desc;
      a.ovf_ptr = E.ovf_ptr;
      a.ovf_col = E.ovf_col;
      a.ovf_hl = E.ovf_hl;
      if (c.minb == 6)
        step3e1_kernel<ADJ, 6><<<(unsigned)blocks, 256, 0, st>>>(a);
      else
        step3e1_kernel<ADJ><<<(unsigned)blocks, 256, 0, st>>>(a);
      return;
    }
  }
  if constexpr (sizeof(T) == 4 && SPLIT && (V == 4 || V == 8)) {
    const DevCSR& E = ADJ ? m.adj3 : m.fwd;
    if (c.packed == 3 && E.ell_col) {  // fixed-width rows
      a.ell_col = E.ell_col;
      a.ell_hl = E.ell_hl;
      a.ell_desc = E.ell_desc;
      a.ovf_ptr = E.ovf_ptr;
      a.ovf_col = E.ovf_col;
      a.ovf_hl = E.ovf_hl;
      a.order = c.order ? m.row_order : nullptr;
      if (c.persist) {
        if constexpr (V == 8) {
          if (c.wide) {
            launch_persist<V, ADJ, true>(a, c, threads, st);
            return;
          }
        }
        launch_persist<V, ADJ, false>(a, c, threads, st);
      } else if (c.big) {
        const int64_t bb = (threads + 1023) / 1024;
        step3e_big_kernel<V, ADJ><<<(unsigned)bb, 1024, 0, st>>>(a);
      } else if (c.minb == 6 && V == 4) {
        if constexpr (V == 4) {
          if (c.pf && !a.order)
            a.pf_rows = c.pf * wave_rows((const void*)step3e_occ_kernel<V, ADJ, 6>, 256, a.K / V);
          step3e_occ_kernel<V, ADJ, 6><<<(unsigned)blocks, 256, 0, st>>>(a);
        }
      } else {
        if (c.pf && !a.order) a.pf_rows = c.pf * wave_rows((const void*)step3e_kernel<V, ADJ>, 256, a.K / V);
        step3e_kernel<V, ADJ><<<(unsigned)blocks, 256, 0, st>>>(a);
      }
      return;
    }
  }
  if constexpr (sizeof(T) == 4 && SPLIT && (V == 4 || V == 8)) {
    if (c.packed) {
      a.hl = (ADJ ? m.adj3.hl : m.fwd.hl);
      a.order = c.order ? m.row_order : nullptr;
      const unsigned nb = (unsigned)blocks;
      if (c.big) {
        const unsigned bb = (unsigned)((threads + 1023) / 1024);
        if (c.chunk == 2)
          step3f_big_kernel<V, 2, ADJ><<<bb, 1024, 0, st>>>(a);
        else
          step3f_big_kernel<V, 4, ADJ><<<bb, 1024, 0, st>>>(a);
      } else if (c.minb == 6) {
        if (c.chunk == 2)
          step3f_occ_kernel<V, 2, ADJ><<<nb, 256, 0, st>>>(a);
        else
          step3f_occ_kernel<V, 4, ADJ><<<nb, 256, 0, st>>>(a);
      } else if (c.early) {
        if (c.chunk == 2)
          step3f_kernel<V, 2, ADJ, true><<<nb, 256, 0, st>>>(a);
        else
          step3f_kernel<V, 4, ADJ, true><<<nb, 256, 0, st>>>(a);
      } else {
        if (c.pf && !a.order)
          a.pf_rows = c.pf * wave_rows(c.chunk == 2 ? (const void*)step3f_kernel<V, 2, ADJ, false>
                                                    : (const void*)step3f_kernel<V, 4, ADJ, false>,
                                       256, a.K / V);
        if (c.chunk == 2)
          step3f_kernel<V, 2, ADJ, false><<<nb, 256, 0, st>>>(a);
        else if (c.chunk == 8 && V == 4)
          step3f_kernel<V, 8, ADJ, false><<<nb, 256, 0, st>>>(a);
        else
          step3f_kernel<V, 4, ADJ, false><<<nb, 256, 0, st>>>(a);
      }
      return;
    }
  }
  const bool allow = c.stage != 0;
  a.stage_cap = allow ? stage_cap_for<T, SPLIT>(m, ADJ, a.K, V) : 0;
  if (a.stage_cap > 0)
    step3_kernel<T, V, SPLIT, ADJ, true><<<(unsigned)blocks, 256, stage_bytes<T, SPLIT>(a.stage_cap), st>>>(a);
  else
    step3_kernel<T, V, SPLIT, ADJ, false><<<(unsigned)blocks, 256, 0, st>>>(a);
}

// Launch i (0 <= i <= N_T) of a three-level forward solve: steps 0..N_T-1, then
// the observation of state N_T.  Step s reads x_s (p0 for s = 0) and x_{s-1}
// and writes x_{s+1} into b[s % 3]; it observes state s (s >= 1).
// The chunk counters of the dynamic hand-out: two words at the start of the
// fourth state buffer (unused by the three-level form); launch i counts on
// word i % 2 and zeroes word (i + 1) % 2 for launch i + 1.  A solve zeroes
// both before its first launch (zero_dyn_counters).
template <typename T>
void dyn_counters(Step3Args<T>& A, T* const b[3], int64_t NK, int i) {
  unsigned int* w = reinterpret_cast<unsigned int*>(b[2] + NK);
  A.dyn_ctr = w + (i & 1);
  A.dyn_next = w + ((i + 1) & 1);
}
template <typename T>
pat_status zero_dyn_counters(T* const b[3], int64_t NK, cudaStream_t st) {
  return cuda_check(cudaMemsetAsync(b[2] + NK, 0, 2 * sizeof(unsigned int), st), "chunk counter reset");
}

template <typename T>
Step3Args<T> fwd3_args(const DeviceMesh& m, int K, int V, const T* p0, T* Y, T scale, T* const b[3], int i,
                       int64_t* threads) {
  Step3Args<T> A{};
  dyn_counters(A, b, m.N * (int64_t)K, i);
  A.N = m.N;
  A.K = K;
  A.n_obs = m.n_obs;
  A.ptr = m.fwd.ptr;
  A.col = m.fwd.col;
  A.hi = static_cast<const T*>(m.fwd.hi);
  A.lo = m.fwd.lo;
  A.nb = m.row_nb;
  A.ninj = m.row_ninj;
  A.det_node = m.det_node;
  A.det_w = static_cast<const T*>(m.det_w);
  A.scale = scale;
  A.inj_scale = T(0);
  const int NT = m.n_steps;
  const int64_t rows = m.N * (int64_t)K / V;
  const int64_t obs = (int64_t)m.n_obs * K / V;
  const int64_t ystride = (int64_t)m.n_obs * K;
  const int s = std::min(i, NT);
  A.x = (s == 0) ? p0 : b[(s - 1) % 3];
  A.xp = (s == 0) ? nullptr : (s == 1 ? p0 : b[(s - 2) % 3]);
  A.prev_mode = (s == 0) ? 1 : 0;  // x_{-1} = x_0: zero initial velocity
  if (i < NT) {
    A.xn = b[i % 3];
    A.row_threads = rows;
    A.y_out = (i == 0) ? nullptr : Y + (int64_t)(i - 1) * ystride;
    *threads = rows + (i == 0 ? 0 : obs);
  } else {
    A.xn = nullptr;
    A.row_threads = 0;
    A.y_out = Y + (int64_t)(NT - 1) * ystride;
    *threads = obs;
  }
  return A;
}

// Launch i (0 <= i <= N_T) of a three-level transposed solve: i = 0 forms
// u_{N_T} = M^{-1} I_{N_T} / 2 from the zero state into b[0]; launch i >= 1 is the
// transposed step m = N_T - i + 1, reading b[(i-1) % 3] (and b[(i-2) % 3]) and
// injecting yhat^m and yhat^{m-1}.  The last two states end in b[N_T % 3] and
// b[(N_T-1) % 3] (adj3_finish_kernel).
template <typename T>
Step3Args<T> adj3_args(const DeviceMesh& m, int K, int V, const T* Yhat, T scale, T* const b[3], int i,
                       int64_t* threads) {
  Step3Args<T> A{};
  dyn_counters(A, b, m.N * (int64_t)K, i);
  A.N = m.N;
  A.K = K;
  A.n_obs = m.n_obs;
  A.ptr = m.adj3.ptr;
  A.col = m.adj3.col;
  A.hi = static_cast<const T*>(m.adj3.hi);
  A.lo = m.adj3.lo;
  A.nb = m.row_nb;
  A.ninj = m.row_ninj;
  A.inj_scale = scale;
  A.scale = T(0);
  A.row_threads = m.N * (int64_t)K / V;
  *threads = A.row_threads;
  const int NT = m.n_steps;
  const int64_t ystride = (int64_t)m.n_obs * K;
  A.xn = b[i % 3];
  if (i == 0) {
    A.x = nullptr;
    A.xp = nullptr;
    A.prev_mode = 2;
    A.ya = Yhat + (int64_t)(NT - 1) * ystride;
    A.yb = nullptr;
  } else {
    const int mstep = NT - i + 1;
    A.x = b[(i - 1) % 3];
    A.xp = (i == 1) ? nullptr : b[(i - 2) % 3];
    A.prev_mode = (i == 1) ? 2 : 0;  // u_{N_T+1} = 0
    A.ya = Yhat + (int64_t)(mstep - 1) * ystride;                          // yhat^m
    A.yb = (mstep >= 2) ? Yhat + (int64_t)(mstep - 2) * ystride : nullptr;  // yhat^{m-1}
  }
  // sensor terms one launch ahead: two [overflow entries][K] buffers after
  // the chunk counters in the fourth state buffer (launch i reads buffer
  // i % 2, which launch i - 1 wrote, and writes buffer (i + 1) % 2 for launch
  // i + 1); a sensor row's term sits at its first overflow entry
  const int64_t NK = m.N * (int64_t)K;
  const int64_t n_ovf = m.adj3.w16_ovf_n;
  if (m.n_inj > 0 && n_ovf > 0 && 2 * n_ovf * K + 64 <= NK) {
    T* const S0 = b[2] + NK + 64;
    T* const S[2] = {S0, S0 + n_ovf * K};
    A.inj_rows = m.inj_rows;
    A.n_inj = m.n_inj;
    A.inj_cur = i >= 1 ? S[i & 1] : nullptr;
    if (i + 1 <= NT) {
      const int mn = NT - i;  // the step of launch i + 1
      A.inj_next = S[(i + 1) & 1];
      A.ya_next = Yhat + (int64_t)(mn - 1) * ystride;
      A.yb_next = (mn >= 2) ? Yhat + (int64_t)(mn - 2) * ystride : nullptr;
    }
  }
  return A;
}

template <typename T, int V, bool SPLIT>
static pat_status forward3_t(const DeviceMesh& m, const T* p0, int K, T* Y, T scale, T* ws, cudaStream_t st) {
  const int64_t NK = m.N * (int64_t)K;
  PAT_RANGE("forward solve");
  T* const b[3] = {ws, ws + NK, ws + 2 * NK};
  PAT_TRY(zero_dyn_counters(b, NK, st));
  const size_t pp = prof_begin(m, 0, st);
  for (int i = 0; i <= m.n_steps; ++i) {
    int64_t threads = 0;
    const Step3Args<T> A = fwd3_args<T>(m, K, V, p0, Y, scale, b, i, &threads);
    launch_step3<T, V, SPLIT, false>(m, A, threads, st);
  }
  prof_end(m, pp, m.n_steps + 1, st);
  return cuda_check(cudaGetLastError(), "forward step launch");
}

template <typename T, int V, bool SPLIT>
static pat_status adjoint3_t(const DeviceMesh& m, const T* Yhat, int K, T* out, T scale, T* ws, cudaStream_t st) {
  const int64_t NK = m.N * (int64_t)K;
  PAT_RANGE("transposed solve");
  T* const b[3] = {ws, ws + NK, ws + 2 * NK};
  PAT_TRY(zero_dyn_counters(b, NK, st));
  const int NT = m.n_steps;
  const size_t pp = prof_begin(m, 1, st);
  for (int i = 0; i <= NT; ++i) {
    int64_t threads = 0;
    const Step3Args<T> A = adj3_args<T>(m, K, V, Yhat, scale, b, i, &threads);
    launch_step3<T, V, SPLIT, true>(m, A, threads, st);
  }
  // G^T yhat = M (u_0 - u_1) + M Bt u_1 from the last two transposed states
  const int64_t rt = NK / V;
  adj3_finish_kernel<T, V, SPLIT><<<(unsigned)((rt + 255) / 256), 256, 0, st>>>(
      rt, K, m.fwd.ptr, m.fwd.col, static_cast<const T*>(m.fwd.hi), m.fwd.lo, m.ml, b[NT % 3], b[(NT - 1) % 3], out);
  prof_end(m, pp, NT + 2, st);
  return cuda_check(cudaGetLastError(), "adjoint step launch");
}

template <typename T>
static pat_status forward_disp(const DeviceMesh& m, const T* p0, int K, T* Y, T scale, T* ws, cudaStream_t st) {
  int V = pick_vec<T>(K, {p0, Y, ws});
  const bool sp = m.split;
  TuneCfg cfg;
  variant(m, 0, K, &cfg);
  V = std::min(V, m.three_level ? cfg.V : 4);
  if (m.three_level) {
    if constexpr (sizeof(T) == 4) {
      if (V == 8) return sp ? forward3_t<T, 8, true>(m, p0, K, Y, scale, ws, st) : forward3_t<T, 8, false>(m, p0, K, Y, scale, ws, st);
      if (V == 4) return sp ? forward3_t<T, 4, true>(m, p0, K, Y, scale, ws, st) : forward3_t<T, 4, false>(m, p0, K, Y, scale, ws, st);
      if (V == 2) return sp ? forward3_t<T, 2, true>(m, p0, K, Y, scale, ws, st) : forward3_t<T, 2, false>(m, p0, K, Y, scale, ws, st);
      return sp ? forward3_t<T, 1, true>(m, p0, K, Y, scale, ws, st) : forward3_t<T, 1, false>(m, p0, K, Y, scale, ws, st);
    } else {
      if (V == 2) return forward3_t<T, 2, false>(m, p0, K, Y, scale, ws, st);
      return forward3_t<T, 1, false>(m, p0, K, Y, scale, ws, st);
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (V == 4) return sp ? forward_t<T, 4, true>(m, p0, K, Y, scale, ws, st) : forward_t<T, 4, false>(m, p0, K, Y, scale, ws, st);
    if (V == 2) return sp ? forward_t<T, 2, true>(m, p0, K, Y, scale, ws, st) : forward_t<T, 2, false>(m, p0, K, Y, scale, ws, st);
    return sp ? forward_t<T, 1, true>(m, p0, K, Y, scale, ws, st) : forward_t<T, 1, false>(m, p0, K, Y, scale, ws, st);
  } else {
    if (V == 2) return forward_t<T, 2, false>(m, p0, K, Y, scale, ws, st);
    return forward_t<T, 1, false>(m, p0, K, Y, scale, ws, st);
  }
}

template <typename T>
static pat_status adjoint_disp(const DeviceMesh& m, const T* Yh, int K, T* out, T scale, T* ws, cudaStream_t st) {
  int V = pick_vec<T>(K, {Yh, out, ws});
  const bool sp = m.split;
  TuneCfg cfg;
  variant(m, 1, K, &cfg);
  V = std::min(V, m.three_level ? cfg.V : 4);
  if (m.three_level) {
    if constexpr (sizeof(T) == 4) {
      if (V == 8) return sp ? adjoint3_t<T, 8, true>(m, Yh, K, out, scale, ws, st) : adjoint3_t<T, 8, false>(m, Yh, K, out, scale, ws, st);
      if (V == 4) return sp ? adjoint3_t<T, 4, true>(m, Yh, K, out, scale, ws, st) : adjoint3_t<T, 4, false>(m, Yh, K, out, scale, ws, st);
      if (V == 2) return sp ? adjoint3_t<T, 2, true>(m, Yh, K, out, scale, ws, st) : adjoint3_t<T, 2, false>(m, Yh, K, out, scale, ws, st);
      return sp ? adjoint3_t<T, 1, true>(m, Yh, K, out, scale, ws, st) : adjoint3_t<T, 1, false>(m, Yh, K, out, scale, ws, st);
    } else {
      if (V == 2) return adjoint3_t<T, 2, false>(m, Yh, K, out, scale, ws, st);
      return adjoint3_t<T, 1, false>(m, Yh, K, out, scale, ws, st);
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (V == 4) return sp ? adjoint_t<T, 4, true>(m, Yh, K, out, scale, ws, st) : adjoint_t<T, 4, false>(m, Yh, K, out, scale, ws, st);
    if (V == 2) return sp ? adjoint_t<T, 2, true>(m, Yh, K, out, scale, ws, st) : adjoint_t<T, 2, false>(m, Yh, K, out, scale, ws, st);
    return sp ? adjoint_t<T, 1, true>(m, Yh, K, out, scale, ws, st) : adjoint_t<T, 1, false>(m, Yh, K, out, scale, ws, st);
  } else {
    if (V == 2) return adjoint_t<T, 2, false>(m, Yh, K, out, scale, ws, st);
    return adjoint_t<T, 1, false>(m, Yh, K, out, scale, ws, st);
  }
}

// One three-level step launch with the mesh's variant for (direction, K), for
// drivers that place the states themselves (the gradient's checkpointed sweeps).
template <typename T, bool ADJ>
static void step_tuned_dir(const DeviceMesh& m, int V, const Step3Args<T>& A, int64_t thr, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (m.split) {
      if (V == 8) return launch_step3<T, 8, true, ADJ>(m, A, thr, st);
      if (V == 4) return launch_step3<T, 4, true, ADJ>(m, A, thr, st);
      if (V == 2) return launch_step3<T, 2, true, ADJ>(m, A, thr, st);
      return launch_step3<T, 1, true, ADJ>(m, A, thr, st);
    }
    if (V == 8) return launch_step3<T, 8, false, ADJ>(m, A, thr, st);
    if (V == 4) return launch_step3<T, 4, false, ADJ>(m, A, thr, st);
    if (V == 2) return launch_step3<T, 2, false, ADJ>(m, A, thr, st);
    return launch_step3<T, 1, false, ADJ>(m, A, thr, st);
  } else {
    if (V == 2) return launch_step3<T, 2, false, ADJ>(m, A, thr, st);
    return launch_step3<T, 1, false, ADJ>(m, A, thr, st);
  }
}

template <typename T>
void step_tuned(const DeviceMesh& m, bool adj, int V, const Step3Args<T>& A, int64_t threads, cudaStream_t st) {
  if (adj)
    step_tuned_dir<T, true>(m, V, A, threads, st);
  else
    step_tuned_dir<T, false>(m, V, A, threads, st);
}
template void step_tuned<float>(const DeviceMesh&, bool, int, const Step3Args<float>&, int64_t, cudaStream_t);
template void step_tuned<double>(const DeviceMesh&, bool, int, const Step3Args<double>&, int64_t, cudaStream_t);

int tuned_vec(const DeviceMesh& m, int dir, int K) {
  TuneCfg c;  // untuned: the default variant's width
  variant(m, dir, K, &c);
  return c.V;
}

pat_status forward(const DeviceMesh& m, const void* p0, int K, void* Y, double scale, void* ws, cudaStream_t st) {
  if (m.prec == PAT_F64)
    return forward_disp<double>(m, (const double*)p0, K, (double*)Y, scale, (double*)ws, st);
  return forward_disp<float>(m, (const float*)p0, K, (float*)Y, (float)scale, (float*)ws, st);
}

pat_status adjoint(const DeviceMesh& m, const void* Yh, int K, void* out, double scale, void* ws, cudaStream_t st) {
  if (m.prec == PAT_F64)
    return adjoint_disp<double>(m, (const double*)Yh, K, (double*)out, scale, (double*)ws, st);
  return adjoint_disp<float>(m, (const float*)Yh, K, (float*)out, (float)scale, (float*)ws, st);
}

// ===========================================================================
// Batched CGLS (textbook CGLS on the extended system, eq. extended-matrices;
// per-sample scalars and the iterate x in FP64)
// ===========================================================================

// Counter-based normal draws.  SplitMix64 (Steele, Lea, Flood 2014): the i-th
// output of a generator seeded with s is mix(s + i * 0x9E3779B97F4A7C15).  A
// draw keyed by (seed, stream, sample k, element e) uses outputs 2c+1 and 2c+2
// with c = ((k << 1 | stream) << 40) | e as two uniforms for Box-Muller
// (cosine branch): z = sqrt(-2 ln u1) cos(2 pi u2), u1 in (0, 1].
__global__ void draw_normals_kernel(uint64_t seed, int stream, int64_t n_elem, int K, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_elem * K) return;
  const int64_t e = t / K;
  const int k = (int)(t - e * K);
  out[t] = normal_draw(seed, stream, (uint64_t)k, (uint64_t)e);
}

// r_d = y_obs / sigma + eta, r_p = xi  (b of eq. extended-matrices with C = M_L^{-1})
// With zero_draws (the MAP problem, eq. MAP) eta = 0 and xi = 0.
// Library draws of sample k use the draw index first + k.
template <typename T>
__global__ void rhs_kernel(int64_t n_data, int64_t N, int K, const T* __restrict__ y_obs, const T* __restrict__ eta,
                           const T* __restrict__ xi, uint64_t seed, double inv_sigma, T* __restrict__ r_d,
                           T* __restrict__ r_p, int zero_draws, uint64_t first) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nd = n_data * K;
  if (t < nd) {
    const int64_t e = t / K;
    const int k = (int)(t - e * K);
    const double et = zero_draws ? 0.0 : eta ? (double)eta[t] : normal_draw(seed, 0, first + k, (uint64_t)e);
    r_d[t] = (T)((double)y_obs[e] * inv_sigma + et);
  } else if (t < nd + N * K) {
    const int64_t u = t - nd;
    const int64_t i = u / K;
    const int k = (int)(u - i * K);
    r_p[u] = zero_draws ? T(0) : xi ? xi[u] : (T)normal_draw(seed, 1, first + k, (uint64_t)i);
  }
}

// Deterministic per-sample reductions: block b sums rows b*rpb + r0 + j*grid*rpb
// for its sample column k = tid % K, then the rpb partial sums of a block are
// combined in a fixed order (warp shuffles first when K divides 32,
// block_partial); partial[b][k].  A finishing kernel then sums the blocks'
// partials of a sample with one warp (warp_colsum).  Mode 0: sum x^2; mode 1:
// sum w_r x^2.
struct RedShape {
  int rpb, bdim, grid;
};
static RedShape red_shape(int K, int64_t rows, int n_part) {
  RedShape r;
  r.rpb = std::max(1, 256 / K);
  r.bdim = r.rpb * K;
  r.grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_part, (rows + r.rpb - 1) / r.rpb));
  return r;
}

// Finishing kernels: one warp per sample column (128-thread blocks).
inline unsigned fin_blocks(int K) { return (unsigned)(((int64_t)K * 32 + 127) / 128); }
#define PAT_FIN_K()                                                    \
  const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); \
  if (k >= K) return;                                                  \
  const bool lead = (threadIdx.x & 31) == 0

template <typename T, bool WEIGHTED>
__global__ void sumsq_kernel(const T* __restrict__ X, const double* __restrict__ w, int64_t rows, int K, int rpb,
                             double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int k = threadIdx.x % K;
  const int r0 = threadIdx.x / K;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpb + r0; r < rows; r += (int64_t)gridDim.x * rpb) {
    const double x = (double)X[r * K + k];
    acc += WEIGHTED ? w[r] * x * x : x * x;
  }
  block_partial(acc, K, rpb, sh, partial);
}

// s = ah + sqrt(M_L) r_p (eq. lsqr-transpose-action), optionally d = s, and sum s^2.
template <typename T>
__global__ void combine_s_kernel(const T* ah, const T* __restrict__ r_p, const double* __restrict__ sqml,
                                 int64_t rows, int K, int rpb, T* s_out, T* __restrict__ d_out,
                                 double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int k = threadIdx.x % K;
  const int r0 = threadIdx.x / K;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpb + r0; r < rows; r += (int64_t)gridDim.x * rpb) {
    const int64_t i = r * K + k;
    const T s = (T)((double)ah[i] + sqml[r] * (double)r_p[i]);
    s_out[i] = s;
    if (d_out) d_out[i] = s;
    acc += (double)s * (double)s;
  }
  block_partial(acc, K, rpb, sh, partial);
}

__global__ void set_double_kernel(double* p, double v) { *p = v; }

__device__ __forceinline__ void flag(int* status, int code) { atomicCAS(status, 0, code); }

// gamma = sum of partial slot A (first CGLS scalar)
__global__ void finalize_gamma0_kernel(const double* pa, int na, int K, double* gamma, int* status) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k);
  if (!lead) return;
  if (!isfinite(s)) flag(status, PAT_ENUMERIC);
  gamma[k] = s;
}

// alpha = gamma / ||q||^2, ||q||^2 = ||q_d||^2 + ||M^{1/2} d||^2
__global__ void finalize_alpha_kernel(const double* pa, int na, const double* pb, int nb, int K, const double* gamma,
                                      double* alpha, int* status) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k) + warp_colsum(pb, nb, K, k);
  if (!lead) return;
  double a = 0.0;
  if (gamma[k] == 0.0) {
    a = 0.0;  // converged exactly: keep the iterate
  } else if (!(s > 0.0) || !isfinite(s) || !isfinite(gamma[k])) {
    flag(status, PAT_ENUMERIC);
  } else {
    a = gamma[k] / s;
  }
  alpha[k] = a;
}

// gamma' = ||s||^2, beta = gamma'/gamma, gamma = gamma'
__global__ void finalize_beta_kernel(const double* pa, int na, int K, double* gamma, double* beta, int* status) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k);
  if (!lead) return;
  double bt = 0.0;
  if (gamma[k] > 0.0 && isfinite(s)) {
    bt = s / gamma[k];
  } else if (gamma[k] != 0.0 || !isfinite(s)) {
    flag(status, PAT_ENUMERIC);
  }
  beta[k] = bt;
  gamma[k] = s;
}

// out[2k] = sum of the data-block partials, out[2k+1] = sum of the prior-block
// partials of sample k (the two blocks of ||r||^2 separately)
__global__ void finalize_blocks_kernel(const double* pa, int na, const double* pb, int nb, int K, double* out) {
  PAT_FIN_K();
  const double sa = warp_colsum(pa, na, K, k), sb = warp_colsum(pb, nb, K, k);
  if (!lead) return;
  out[2 * k] = sa;
  out[2 * k + 1] = sb;
}

__global__ void finalize_sum2_kernel(const double* pa, int na, const double* pb, int nb, int K, double* out) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k) + warp_colsum(pb, nb, K, k);
  if (lead) out[k] = s;
}

// x += alpha d (FP64), r_p -= alpha sqrt(M_L) d
template <typename T>
__global__ void update_x_rp_kernel(int64_t N, int K, const double* __restrict__ alpha, const T* __restrict__ d,
                                   const double* __restrict__ sqml, double* __restrict__ x, T* __restrict__ r_p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  const int64_t i = t / K;
  const int k = (int)(t - i * K);
  const double a = alpha[k];
  const double dv = (double)d[t];
  x[t] += a * dv;
  r_p[t] = (T)((double)r_p[t] - a * sqml[i] * dv);
}

// r_d -= alpha q_d
template <typename T>
__global__ void update_rd_kernel(int64_t n, int K, const double* __restrict__ alpha, const T* __restrict__ q,
                                 T* __restrict__ r) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int k = (int)(t % K);
  r[t] = (T)((double)r[t] - alpha[k] * (double)q[t]);
}

// d = s + beta d
template <typename T>
__global__ void update_d_kernel(int64_t N, int K, const double* __restrict__ beta, const T* __restrict__ s,
                                T* __restrict__ d) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * K) return;
  const int k = (int)(t % K);
  d[t] = (T)((double)s[t] + beta[k] * (double)d[t]);
}

// eq. ergodic: mean and std with 1/(K-1), per node, two passes in FP64
__global__ void mean_std_kernel(int64_t N, int K, const double* __restrict__ x, double* __restrict__ mean,
                                double* __restrict__ stdev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* r = x + i * K;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += r[k];
  const double m = s / K;
  if (mean) mean[i] = m;
  if (stdev) {
    double v = 0.0;
    for (int k = 0; k < K; ++k) v += (r[k] - m) * (r[k] - m);
    stdev[i] = K > 1 ? sqrt(v / (K - 1)) : 0.0;
  }
}

// Pooled statistics of eq. ergodic over samples held by several processes, in
// two passes so that no variance is formed by cancellation: pass 0 writes
// out[i] = sum_k x_ik, pass 1 writes out[i] = sum_k (x_ik - center_i)^2; the
// caller sums out over the processes between the passes and after pass 1.
__global__ void moments_kernel(int64_t N, int K, const double* __restrict__ x, const double* __restrict__ center,
                               double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* r = x + i * K;
  double s = 0.0;
  if (center == nullptr) {
    for (int k = 0; k < K; ++k) s += r[k];
  } else {
    const double c = center[i];
    for (int k = 0; k < K; ++k) s += (r[k] - c) * (r[k] - c);
  }
  out[i] = s;
}

// In place: which 0, v = v / n (the mean from the pooled sum); which 1,
// v = sqrt(v / (n - 1)) (the std from the pooled squared deviations).
__global__ void moments_finish_kernel(int64_t N, double n, int which, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  v[i] = which == 0 ? v[i] / n : sqrt(v[i] / (n - 1.0));
}

RtoLayout rto_layout(const DeviceMesh& m, int K) {
  RtoLayout L{};
  const size_t rs = real_size(m);
  const size_t NK = (size_t)m.N * K;
  const size_t DK = (size_t)m.n_steps * m.n_obs * K;
  L.n_part = std::min(1024, 2 * sm_count());
  size_t o = 0;
  L.x = o; o = align256(o + NK * 8);
  L.d = o; o = align256(o + NK * rs);
  L.r_d = o; o = align256(o + DK * rs);
  L.q_d = o; o = align256(o + DK * rs);
  L.r_p = o; o = align256(o + NK * rs);
  L.s = o; o = align256(o + NK * rs);
  L.state = o; o = align256(o + 4 * NK * rs);
  L.gamma = o; o = align256(o + K * 8);
  L.alpha = o; o = align256(o + K * 8);
  L.beta = o; o = align256(o + K * 8);
  L.sigma = o; o = align256(o + 8);
  L.partial = o; o = align256(o + (size_t)4 * L.n_part * K * 8);
  L.status = o; o = align256(o + 4);
  L.w = o; o = align256(o + NK * rs);
  L.lsq = o; o = align256(o + (size_t)kLsq * K * 8);
  L.total = o;
  return L;
}

static inline unsigned nblocks(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// One forward (dir 0: d -> q_d) or transposed (dir 1: r_d -> s) solve of the
// CGLS loop, replayed from a CUDA graph captured on first use (N_T + 1 or
// N_T + 2 launches become one graph launch).  Falls back to direct launches
// when the stream is already being captured or graphs are disabled.
pat_status cgls_solve(const DeviceMesh& m, int dir, int K, double sigma, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  auto direct = [&](cudaStream_t s) {
    return dir == 0 ? forward(m, ws + L.d, K, ws + L.q_d, 1.0 / sigma, ws + L.state, s)
                    : adjoint(m, ws + L.r_d, K, ws + L.s, 1.0 / sigma, ws + L.state, s);
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((m.flags & PAT_MESH_NO_GRAPHS) || !m.capture_stream || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return direct(st);
  }
  uint64_t sbits;
  std::memcpy(&sbits, &sigma, 8);
  const auto key = std::make_tuple(dir, (const void*)ws, K, sbits);
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    auto it = m.graphs.find(key);
    if (it != m.graphs.end()) exec = (cudaGraphExec_t)it->second;
  }
  if (!exec) {
    // capture on the mesh's private stream (the caller's may be the legacy
    // default stream, which cannot be captured); the graph then runs on st
    cudaStream_t cap = (cudaStream_t)m.capture_stream;
    const bool prof_on = m.prof.on;
    m.prof.on = false;  // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      m.prof.on = prof_on;
      cudaGetLastError();
      return direct(st);
    }
    const pat_status s = direct(cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    m.prof.on = prof_on;
    if (s != PAT_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s != PAT_OK ? s : cuda_check(e, "graph end capture");
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    PAT_TRY(cuda_check(e, "graph instantiate"));
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    m.graphs[key] = (void*)exec;
  }
  const size_t pp = prof_begin(m, dir, st);
  PAT_TRY(cuda_check(cudaGraphLaunch(exec, st), "graph launch"));
  prof_end(m, pp, dir == 0 ? m.n_steps + 1 : m.n_steps + (m.three_level ? 2 : 1), st);
  return PAT_OK;
}

// CGLS phases around the two wave solves of an iteration (also driven per job
// by the grouped multi-mesh driver).
template <typename T>
pat_status begin_pre(const DeviceMesh& m, const T* y_obs, double sigma, int K, const T* eta, const T* xi,
                     uint64_t seed, char* ws, cudaStream_t st, bool zero_draws) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.status, 0, 4, st), "cgls_begin memset"));
  set_double_kernel<<<1, 1, 0, st>>>((double*)(ws + L.sigma), sigma);
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.x, 0, (size_t)m.N * K * 8, st), "cgls_begin memset x"));
  rhs_kernel<T><<<nblocks((ndata + m.N) * K), 256, 0, st>>>(ndata, m.N, K, y_obs, eta, xi, seed, 1.0 / sigma,
                                                            (T*)(ws + L.r_d), (T*)(ws + L.r_p), zero_draws ? 1 : 0,
                                                            (uint64_t)m.first_sample);
  count(m, 2);
  return cuda_check(cudaGetLastError(), "cgls_begin launch");
}

// after s = G^T r_d / sigma landed in s: s += M^{1/2} r_p, d = s, gamma = ||s||^2
template <typename T>
pat_status begin_post(const DeviceMesh& m, int K, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  double* part = (double*)(ws + L.partial);
  combine_s_kernel<T><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(
      (T*)(ws + L.s), (T*)(ws + L.r_p), m.sqrt_ml, m.N, K, rsN.rpb, (T*)(ws + L.s), (T*)(ws + L.d), part);
  finalize_gamma0_kernel<<<fin_blocks(K), 128, 0, st>>>(part, rsN.grid, K, (double*)(ws + L.gamma),
                                                           (int*)(ws + L.status));
  count(m, 2);
  return cuda_check(cudaGetLastError(), "cgls_begin launch");
}

// after q_d = G d / sigma: alpha = gamma / (||q_d||^2 + ||M^{1/2} d||^2); x += alpha d;
// r_p -= alpha M^{1/2} d; r_d -= alpha q_d
template <typename T>
pat_status iter_mid(const DeviceMesh& m, int K, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  T* d = (T*)(ws + L.d);
  double* part = (double*)(ws + L.partial);
  double* pa = part;
  double* pb = part + (size_t)L.n_part * K;
  const RedShape rsD = red_shape(K, ndata, L.n_part);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  double* alpha = (double*)(ws + L.alpha);
  sumsq_kernel<T, false><<<rsD.grid, rsD.bdim, rsD.bdim * sizeof(double), st>>>((T*)(ws + L.q_d), nullptr, ndata, K,
                                                                                 rsD.rpb, pa);
  sumsq_kernel<T, true><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(d, m.ml, m.N, K, rsN.rpb, pb);
  finalize_alpha_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, pb, rsN.grid, K, (double*)(ws + L.gamma),
                                                          alpha, (int*)(ws + L.status));
  update_x_rp_kernel<T><<<nblocks(m.N * K), 256, 0, st>>>(m.N, K, alpha, d, m.sqrt_ml, (double*)(ws + L.x),
                                                          (T*)(ws + L.r_p));
  update_rd_kernel<T><<<nblocks(ndata * K), 256, 0, st>>>(ndata, K, alpha, (T*)(ws + L.q_d), (T*)(ws + L.r_d));
  count(m, 5);
  return cuda_check(cudaGetLastError(), "cgls_iterate launch");
}

// after s = G^T r_d / sigma landed in s: s += M^{1/2} r_p; beta = ||s||^2 / gamma; d = s + beta d
template <typename T>
pat_status iter_post(const DeviceMesh& m, int K, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  double* pa = (double*)(ws + L.partial);
  T* s = (T*)(ws + L.s);
  double* beta = (double*)(ws + L.beta);
  combine_s_kernel<T><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(s, (T*)(ws + L.r_p), m.sqrt_ml, m.N, K,
                                                                             rsN.rpb, s, nullptr, pa);
  finalize_beta_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsN.grid, K, (double*)(ws + L.gamma), beta,
                                                         (int*)(ws + L.status));
  update_d_kernel<T><<<nblocks(m.N * K), 256, 0, st>>>(m.N, K, beta, s, (T*)(ws + L.d));
  count(m, 3);
  return cuda_check(cudaGetLastError(), "cgls_iterate launch");
}

template <typename T>
static pat_status begin_t(const DeviceMesh& m, const T* y_obs, double sigma, int K, const T* eta, const T* xi,
                          uint64_t seed, char* ws, cudaStream_t st, bool zero_draws) {
  PAT_TRY(begin_pre<T>(m, y_obs, sigma, K, eta, xi, seed, ws, st, zero_draws));
  // s = A^T r, d = s, gamma = ||s||^2 (the transpose lands in s, combined in place)
  PAT_TRY(cgls_solve(m, 1, K, sigma, ws, st));
  return begin_post<T>(m, K, ws, st);
}

// ||r||^2 per sample of the current CGLS residual (blocks = false: out[K]), or
// its data and prior blocks separately (blocks = true: out[K][2])
template <typename T>
static pat_status residual_t(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st, bool blocks) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  double* part = (double*)(ws + L.partial);
  double* pa = part + 2 * (size_t)L.n_part * K;
  double* pb = part + 3 * (size_t)L.n_part * K;
  const RedShape rsD = red_shape(K, ndata, L.n_part);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  sumsq_kernel<T, false><<<rsD.grid, rsD.bdim, rsD.bdim * sizeof(double), st>>>((T*)(ws + L.r_d), nullptr, ndata, K,
                                                                                 rsD.rpb, pa);
  sumsq_kernel<T, false><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>((T*)(ws + L.r_p), nullptr, m.N, K,
                                                                                 rsN.rpb, pb);
  if (blocks)
    finalize_blocks_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, pb, rsN.grid, K, out);
  else
    finalize_sum2_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, pb, rsN.grid, K, out);
  count(m, 3);
  return cuda_check(cudaGetLastError(), "residual launch");
}

template <typename T>
static pat_status iterate_t(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                            cudaStream_t st, bool blocks) {
  const RtoLayout L = rto_layout(m, K);
  if (!(sigma > 0.0)) {
    set_error("pat_cgls_iterate: sigma must be > 0 (got %g)", sigma);
    return PAT_EINVAL;
  }
  for (int it = 0; it < n_iter; ++it) {
    PAT_RANGE("CGLS iteration");
    // q = A d: q_d = G d / sigma (forward), q_p = M^{1/2} d (implicit)
    PAT_TRY(cgls_solve(m, 0, K, sigma, ws, st));
    PAT_TRY(iter_mid<T>(m, K, ws, st));
    // s = A^T r = G^T r_d / sigma + M^{1/2} r_p
    PAT_TRY(cgls_solve(m, 1, K, sigma, ws, st));
    PAT_TRY(iter_post<T>(m, K, ws, st));
    if (resid) PAT_TRY(residual_t<T>(m, K, resid + (int64_t)it * (blocks ? 2 : 1) * K, ws, st, blocks));
  }
  return PAT_OK;
}

pat_status cgls_begin(const DeviceMesh& m, const void* y_obs, double sigma, int K, const void* eta, const void* xi,
                      uint64_t seed, char* ws, cudaStream_t st, bool zero_draws) {
  if (m.prec == PAT_F64)
    return begin_t<double>(m, (const double*)y_obs, sigma, K, (const double*)eta, (const double*)xi, seed, ws, st,
                           zero_draws);
  return begin_t<float>(m, (const float*)y_obs, sigma, K, (const float*)eta, (const float*)xi, seed, ws, st,
                        zero_draws);
}

pat_status cgls_iterate(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                        cudaStream_t st, bool blocks) {
  if (m.prec == PAT_F64) return iterate_t<double>(m, sigma, K, n_iter, resid, ws, st, blocks);
  return iterate_t<float>(m, sigma, K, n_iter, resid, ws, st, blocks);
}

pat_status residual_norms(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st, bool blocks) {
  if (m.prec == PAT_F64) return residual_t<double>(m, K, out, ws, st, blocks);
  return residual_t<float>(m, K, out, ws, st, blocks);
}

pat_status rto_moments(const DeviceMesh& m, int K, const double* center, double* out, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  moments_kernel<<<nblocks(m.N), 256, 0, st>>>(m.N, K, (const double*)(ws + L.x), center, out);
  count(m, 1);
  return cuda_check(cudaGetLastError(), "rto_moments launch");
}

pat_status moments_finish(int64_t N, double n, int which, double* v, cudaStream_t st) {
  moments_finish_kernel<<<nblocks(N), 256, 0, st>>>(N, n, which, v);
  return cuda_check(cudaGetLastError(), "moments_finish launch");
}

pat_status cgls_finish(const DeviceMesh& m, int K, double* samples, double* mean, double* stdev, char* ws,
                       cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const double* x = (const double*)(ws + L.x);
  if (samples)
    PAT_TRY(cuda_check(cudaMemcpyAsync(samples, x, (size_t)m.N * K * 8, cudaMemcpyDeviceToDevice, st),
                       "cgls_finish copy"));
  if (mean || stdev) {
    mean_std_kernel<<<nblocks(m.N), 256, 0, st>>>(m.N, K, x, mean, stdev);
    count(m, 1);
  }
  return cuda_check(cudaGetLastError(), "cgls_finish launch");
}

// ---------------------------------------------------------------------------
// LSQR (Paige & Saunders 1982, the paper's solver) on the extended system.
// The left Golub-Kahan vectors are kept unnormalised, ub_i = beta_i u_i, so no
// pass over the data-space fields is spent on normalising them:
//   ub_{i+1} = A v_i - (alpha_i / beta_i) ub_i,        beta_{i+1} = ||ub_{i+1}||,
//   t = A^T ub_{i+1} / beta_{i+1} - beta_{i+1} v_i,    alpha_{i+1} = ||t||, v_{i+1} = t / alpha_{i+1},
// then the plane rotation and the x, w updates of the published algorithm.
// Fields: ub = (r_d, r_p), v = d, A v data block = q_d, A^T ub data part = s,
// w = w, x = x (FP64); per-sample FP64 scalars in lsq [kLsq][K].
// ---------------------------------------------------------------------------
enum LsqSlot { kAlpha = 0, kBeta, kRhoBar, kPhiBar, kC, kS, kRho, kPhi, kFx, kFw, kIa, kIb };

// ub = A v - c ub on one block with c = alpha / beta per sample (P: prior block,
// A v = sqrt(M_L) v; else data block, A v = q), and the partial sums of ub^2.
template <typename T, bool P>
__global__ void lsqr_u_kernel(const T* __restrict__ q, const double* __restrict__ sqml, T* ub, int64_t rows, int K,
                              int rpb, const double* __restrict__ lsq, double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int k = threadIdx.x % K;
  const int r0 = threadIdx.x / K;
  const double b = lsq[kBeta * K + k];
  const double c = b != 0.0 ? lsq[kAlpha * K + k] / b : 0.0;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpb + r0; r < rows; r += (int64_t)gridDim.x * rpb) {
    const int64_t i = r * K + k;
    const double av = P ? sqml[r] * (double)q[i] : (double)q[i];
    const T u = (T)(av - c * (double)ub[i]);
    ub[i] = u;
    acc += (double)u * (double)u;
  }
  block_partial(acc, K, rpb, sh, partial);
}

// t = (ah + sqrt(M_L) ub_p) / beta - beta v (v NULL at the start) into out, and sum t^2
template <typename T>
__global__ void lsqr_t_kernel(const T* ah, const T* __restrict__ ub_p, const double* __restrict__ sqml,
                              const T* __restrict__ v, int64_t rows, int K, int rpb, const double* __restrict__ lsq,
                              T* out, double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int k = threadIdx.x % K;
  const int r0 = threadIdx.x / K;
  const double b = lsq[kBeta * K + k], ib = lsq[kIb * K + k];
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpb + r0; r < rows; r += (int64_t)gridDim.x * rpb) {
    const int64_t i = r * K + k;
    double t = ((double)ah[i] + sqml[r] * (double)ub_p[i]) * ib;
    if (v) t -= b * (double)v[i];
    const T tv = (T)t;
    out[i] = tv;
    acc += (double)tv * (double)tv;
  }
  block_partial(acc, K, rpb, sh, partial);
}

__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// beta_1 = ||b||: phibar = beta, 1 / beta
__global__ void lsqr_beta0_kernel(const double* pa, int na, const double* pb, int nb, int K, double* lsq,
                                  int* status) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k) + warp_colsum(pb, nb, K, k);
  if (!lead) return;
  if (!isfinite(s)) flag(status, PAT_ENUMERIC);
  const double beta = sqrt(s);
  lsq[kBeta * K + k] = beta;
  lsq[kPhiBar * K + k] = beta;
  lsq[kIb * K + k] = safe_div(1.0, beta);
}

// alpha_1 = ||A^T u_1||: rhobar = alpha, 1 / alpha
__global__ void lsqr_alpha0_kernel(const double* pa, int na, int K, double* lsq, int* status) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k);
  if (!lead) return;
  if (!isfinite(s)) flag(status, PAT_ENUMERIC);
  const double alpha = sqrt(s);
  lsq[kAlpha * K + k] = alpha;
  lsq[kRhoBar * K + k] = alpha;
  lsq[kIa * K + k] = safe_div(1.0, alpha);
}

// beta_{i+1} = ||ub_{i+1}||, then the rotation quantities that need it:
// rho = (rhobar^2 + beta^2)^{1/2}, c = rhobar / rho, s = beta / rho, phi = c phibar, phibar = s phibar
__global__ void lsqr_beta_kernel(const double* pa, int na, const double* pb, int nb, int K, double* lsq,
                                 int* status) {
  PAT_FIN_K();
  const double s2 = warp_colsum(pa, na, K, k) + warp_colsum(pb, nb, K, k);
  if (!lead) return;
  if (!isfinite(s2)) flag(status, PAT_ENUMERIC);
  const double beta = sqrt(s2), rhobar = lsq[kRhoBar * K + k], phibar = lsq[kPhiBar * K + k];
  const double rho = sqrt(rhobar * rhobar + beta * beta);
  const double c = safe_div(rhobar, rho), s = safe_div(beta, rho);
  lsq[kBeta * K + k] = beta;
  lsq[kIb * K + k] = safe_div(1.0, beta);
  lsq[kRho * K + k] = rho;
  lsq[kC * K + k] = c;
  lsq[kS * K + k] = s;
  lsq[kPhi * K + k] = c * phibar;
  lsq[kPhiBar * K + k] = s * phibar;
}

// alpha_{i+1} = ||t||, theta = s alpha, rhobar = -c alpha, x / w coefficients phi / rho, theta / rho
__global__ void lsqr_alpha_kernel(const double* pa, int na, int K, double* lsq, int* status) {
  PAT_FIN_K();
  const double s2 = warp_colsum(pa, na, K, k);
  if (!lead) return;
  if (!isfinite(s2)) flag(status, PAT_ENUMERIC);
  const double alpha = sqrt(s2), rho = lsq[kRho * K + k];
  const double theta = lsq[kS * K + k] * alpha;
  lsq[kAlpha * K + k] = alpha;
  lsq[kIa * K + k] = safe_div(1.0, alpha);
  lsq[kRhoBar * K + k] = -lsq[kC * K + k] * alpha;
  lsq[kFx * K + k] = safe_div(lsq[kPhi * K + k], rho);
  lsq[kFw * K + k] = safe_div(theta, rho);
}

// v = t / alpha; with W: x += (phi / rho) w, w = v - (theta / rho) w; else (start) w = v
template <typename T, bool W>
__global__ void lsqr_vxw_kernel(int64_t N, int K, const T* __restrict__ t, const double* __restrict__ lsq, T* v,
                                T* w, double* x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const int k = (int)(i % K);
  const T vn = (T)((double)t[i] * lsq[kIa * K + k]);
  v[i] = vn;
  if constexpr (W) {
    const double wo = (double)w[i];
    x[i] += lsq[kFx * K + k] * wo;
    w[i] = (T)((double)vn - lsq[kFw * K + k] * wo);
  } else {
    w[i] = vn;
  }
}

// out[k] = phibar^2 (the squared residual norm of the current iterate)
__global__ void lsqr_resid_kernel(int K, const double* __restrict__ lsq, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double p = lsq[kPhiBar * K + k];
  out[k] = p * p;
}

template <typename T>
static pat_status lsqr_begin_t(const DeviceMesh& m, const T* y_obs, double sigma, int K, const T* eta, const T* xi,
                               uint64_t seed, bool zero_draws, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  // ub_1 = b (r_d, r_p), x = 0
  PAT_TRY(begin_pre<T>(m, y_obs, sigma, K, eta, xi, seed, ws, st, zero_draws));
  double* lsq = (double*)(ws + L.lsq);
  double* pa = (double*)(ws + L.partial);
  double* pb = pa + (size_t)L.n_part * K;
  const RedShape rsD = red_shape(K, ndata, L.n_part);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  int* status = (int*)(ws + L.status);
  sumsq_kernel<T, false><<<rsD.grid, rsD.bdim, rsD.bdim * sizeof(double), st>>>((T*)(ws + L.r_d), nullptr, ndata, K,
                                                                                 rsD.rpb, pa);
  sumsq_kernel<T, false><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>((T*)(ws + L.r_p), nullptr, m.N, K,
                                                                                 rsN.rpb, pb);
  lsqr_beta0_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, pb, rsN.grid, K, lsq, status);
  // t = A^T ub_1 / beta_1; alpha_1 = ||t||; v_1 = t / alpha_1; w_1 = v_1
  PAT_TRY(cgls_solve(m, 1, K, sigma, ws, st));
  T* s = (T*)(ws + L.s);
  lsqr_t_kernel<T><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(
      s, (T*)(ws + L.r_p), m.sqrt_ml, nullptr, m.N, K, rsN.rpb, lsq, s, pa);
  lsqr_alpha0_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsN.grid, K, lsq, status);
  lsqr_vxw_kernel<T, false><<<nblocks(m.N * K), 256, 0, st>>>(m.N, K, s, lsq, (T*)(ws + L.d), (T*)(ws + L.w),
                                                              (double*)(ws + L.x));
  count(m, 6);
  return cuda_check(cudaGetLastError(), "lsqr_begin launch");
}

template <typename T>
static pat_status lsqr_iterate_t(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                                 cudaStream_t st) {
  if (!(sigma > 0.0)) {
    set_error("pat_lsqr_iterate: sigma must be > 0 (got %g)", sigma);
    return PAT_EINVAL;
  }
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  double* lsq = (double*)(ws + L.lsq);
  double* pa = (double*)(ws + L.partial);
  double* pb = pa + (size_t)L.n_part * K;
  const RedShape rsD = red_shape(K, ndata, L.n_part);
  const RedShape rsN = red_shape(K, m.N, L.n_part);
  int* status = (int*)(ws + L.status);
  T* v = (T*)(ws + L.d);
  T* s = (T*)(ws + L.s);
  for (int it = 0; it < n_iter; ++it) {
    PAT_RANGE("LSQR iteration");
    // ub = A v - (alpha / beta) ub: data block from q_d = G v / sigma, prior block sqrt(M_L) v
    PAT_TRY(cgls_solve(m, 0, K, sigma, ws, st));
    lsqr_u_kernel<T, false><<<rsD.grid, rsD.bdim, rsD.bdim * sizeof(double), st>>>(
        (T*)(ws + L.q_d), nullptr, (T*)(ws + L.r_d), ndata, K, rsD.rpb, lsq, pa);
    lsqr_u_kernel<T, true><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(
        v, m.sqrt_ml, (T*)(ws + L.r_p), m.N, K, rsN.rpb, lsq, pb);
    lsqr_beta_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, pb, rsN.grid, K, lsq, status);
    // t = A^T ub / beta - beta v, alpha = ||t||, v = t / alpha, x and w updates
    PAT_TRY(cgls_solve(m, 1, K, sigma, ws, st));
    lsqr_t_kernel<T><<<rsN.grid, rsN.bdim, rsN.bdim * sizeof(double), st>>>(
        s, (T*)(ws + L.r_p), m.sqrt_ml, v, m.N, K, rsN.rpb, lsq, s, pa);
    lsqr_alpha_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsN.grid, K, lsq, status);
    lsqr_vxw_kernel<T, true><<<nblocks(m.N * K), 256, 0, st>>>(m.N, K, s, lsq, v, (T*)(ws + L.w),
                                                               (double*)(ws + L.x));
    count(m, 6);
    if (resid) {
      lsqr_resid_kernel<<<nblocks(K, 128), 128, 0, st>>>(K, lsq, resid + (int64_t)it * K);
      count(m, 1);
    }
  }
  return cuda_check(cudaGetLastError(), "lsqr_iterate launch");
}

pat_status lsqr_begin(const DeviceMesh& m, const void* y_obs, double sigma, int K, const void* eta, const void* xi,
                      uint64_t seed, bool zero_draws, char* ws, cudaStream_t st) {
  if (m.prec == PAT_F64)
    return lsqr_begin_t<double>(m, (const double*)y_obs, sigma, K, (const double*)eta, (const double*)xi, seed,
                                zero_draws, ws, st);
  return lsqr_begin_t<float>(m, (const float*)y_obs, sigma, K, (const float*)eta, (const float*)xi, seed, zero_draws,
                             ws, st);
}

pat_status lsqr_iterate(const DeviceMesh& m, double sigma, int K, int n_iter, double* resid, char* ws,
                        cudaStream_t st) {
  if (m.prec == PAT_F64) return lsqr_iterate_t<double>(m, sigma, K, n_iter, resid, ws, st);
  return lsqr_iterate_t<float>(m, sigma, K, n_iter, resid, ws, st);
}

pat_status lsqr_residual(const DeviceMesh& m, int K, double* out, char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  lsqr_resid_kernel<<<nblocks(K, 128), 128, 0, st>>>(K, (const double*)(ws + L.lsq), out);
  count(m, 1);
  return cuda_check(cudaGetLastError(), "lsqr residual launch");
}

// ---------------------------------------------------------------------------
// Discrepancy diagnostic (Section 6.1): ||G x_k - y_obs|| / (sigma sqrt(N_T N_obs))
// for each sample column of the FP64 iterate x [N][K].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void to_real_kernel(int64_t n, const double* __restrict__ x, T* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)x[i];
}

template <typename T>
__global__ void misfit_kernel(const T* __restrict__ Y, const T* __restrict__ y_obs, int64_t rows, int K, int rpb,
                              double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int k = threadIdx.x % K;
  const int r0 = threadIdx.x / K;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * rpb + r0; r < rows; r += (int64_t)gridDim.x * rpb) {
    const double d = (double)Y[r * K + k] - (double)y_obs[r];
    acc += d * d;
  }
  block_partial(acc, K, rpb, sh, partial);
}

__global__ void misfit_finish_kernel(const double* pa, int na, int K, double scale, double* out) {
  PAT_FIN_K();
  const double s = warp_colsum(pa, na, K, k);
  if (lead) out[k] = sqrt(s) * scale;
}

template <typename T>
static pat_status misfit_t(const DeviceMesh& m, const double* x, const T* y_obs, double sigma, int K, double* out,
                           char* ws, cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t ndata = (int64_t)m.n_steps * m.n_obs;
  T* xr = (T*)(ws + L.d);
  T* Y = (T*)(ws + L.q_d);
  to_real_kernel<T><<<nblocks(m.N * K), 256, 0, st>>>(m.N * K, x, xr);
  count(m, 1);
  PAT_TRY(cuda_check(cudaGetLastError(), "misfit launch"));
  PAT_TRY(forward(m, xr, K, Y, 1.0, ws + L.state, st));
  double* pa = (double*)(ws + L.partial);
  const RedShape rsD = red_shape(K, ndata, L.n_part);
  misfit_kernel<T><<<rsD.grid, rsD.bdim, rsD.bdim * sizeof(double), st>>>(Y, y_obs, ndata, K, rsD.rpb, pa);
  misfit_finish_kernel<<<fin_blocks(K), 128, 0, st>>>(pa, rsD.grid, K, 1.0 / (sigma * std::sqrt((double)ndata)),
                                                         out);
  count(m, 2);
  return cuda_check(cudaGetLastError(), "misfit launch");
}

pat_status whitened_misfit(const DeviceMesh& m, const double* x, const void* y_obs, double sigma, int K,
                           double* out, char* ws, cudaStream_t st) {
  if (m.prec == PAT_F64) return misfit_t<double>(m, x, (const double*)y_obs, sigma, K, out, ws, st);
  return misfit_t<float>(m, x, (const float*)y_obs, sigma, K, out, ws, st);
}

template Step3Args<float> fwd3_args<float>(const DeviceMesh&, int, int, const float*, float*, float, float* const[3],
                                           int, int64_t*);
template Step3Args<double> fwd3_args<double>(const DeviceMesh&, int, int, const double*, double*, double,
                                             double* const[3], int, int64_t*);
template Step3Args<float> adj3_args<float>(const DeviceMesh&, int, int, const float*, float, float* const[3], int,
                                           int64_t*);
template Step3Args<double> adj3_args<double>(const DeviceMesh&, int, int, const double*, double, double* const[3],
                                             int, int64_t*);
template pat_status begin_pre<float>(const DeviceMesh&, const float*, double, int, const float*, const float*, uint64_t,
                                     char*, cudaStream_t, bool);
template pat_status begin_pre<double>(const DeviceMesh&, const double*, double, int, const double*, const double*,
                                      uint64_t, char*, cudaStream_t, bool);
template pat_status begin_post<float>(const DeviceMesh&, int, char*, cudaStream_t);
template pat_status begin_post<double>(const DeviceMesh&, int, char*, cudaStream_t);
template pat_status iter_mid<float>(const DeviceMesh&, int, char*, cudaStream_t);
template pat_status iter_mid<double>(const DeviceMesh&, int, char*, cudaStream_t);
template pat_status iter_post<float>(const DeviceMesh&, int, char*, cudaStream_t);
template pat_status iter_post<double>(const DeviceMesh&, int, char*, cudaStream_t);

int vec_width(const DeviceMesh& m, int K, std::initializer_list<const void*> ptrs) {
  return m.prec == PAT_F64 ? pick_vec<double>(K, ptrs) : pick_vec<float>(K, ptrs);
}

// Autotuning of the three-level step: every variant (V samples per thread,
// row staging on/off) runs n_probe forward and n_probe transposed steps on
// zeroed buffers of an RTO workspace, timed with CUDA events; the fastest per
// direction is kept for (mesh, K).
template <typename T>
static pat_status probe_t(const DeviceMesh& m, int K, char* ws, int n_probe, int dir, cudaStream_t st, float* us) {
  const RtoLayout L = rto_layout(m, K);
  const int64_t NK = m.N * (int64_t)K;
  T* const b[3] = {(T*)(ws + L.state), (T*)(ws + L.state) + NK, (T*)(ws + L.state) + 2 * NK};
  cudaEvent_t e0, e1;
  PAT_TRY(cuda_check(cudaEventCreate(&e0), "autotune event"));
  PAT_TRY(cuda_check(cudaEventCreate(&e1), "autotune event"));
  const int V = std::min(g_force.V, pick_vec<T>(K, {ws + L.d, ws + L.q_d, ws + L.r_d, ws + L.state}));
  // the first two launches of a solve start from the zero state (x_{s-1} or
  // x_s absent) and run faster than the steady state: untimed
  const int skip = m.n_steps >= 4 ? 2 : 0;
  auto run = [&](bool timed) {
    zero_dyn_counters(b, NK, st);
    for (int i = 0; i < skip + n_probe; ++i) {
      if (timed && i == skip) cudaEventRecord(e0, st);
      int64_t thr = 0;
      if (dir == 0) {
        const Step3Args<T> A = fwd3_args<T>(m, K, V, (const T*)(ws + L.d), (T*)(ws + L.q_d), T(1), b, i, &thr);
        if constexpr (sizeof(T) == 4) {
          if (m.split) {
            if (V == 8) launch_step3<T, 8, true, false>(m, A, thr, st);
            else if (V == 4) launch_step3<T, 4, true, false>(m, A, thr, st);
            else if (V == 2) launch_step3<T, 2, true, false>(m, A, thr, st);
            else launch_step3<T, 1, true, false>(m, A, thr, st);
          } else {
            if (V == 4) launch_step3<T, 4, false, false>(m, A, thr, st);
            else if (V == 2) launch_step3<T, 2, false, false>(m, A, thr, st);
            else launch_step3<T, 1, false, false>(m, A, thr, st);
          }
        } else {
          if (V == 2) launch_step3<T, 2, false, false>(m, A, thr, st);
          else launch_step3<T, 1, false, false>(m, A, thr, st);
        }
      } else {
        const Step3Args<T> A = adj3_args<T>(m, K, V, (const T*)(ws + L.r_d), T(1), b, i, &thr);
        if constexpr (sizeof(T) == 4) {
          if (m.split) {
            if (V == 8) launch_step3<T, 8, true, true>(m, A, thr, st);
            else if (V == 4) launch_step3<T, 4, true, true>(m, A, thr, st);
            else if (V == 2) launch_step3<T, 2, true, true>(m, A, thr, st);
            else launch_step3<T, 1, true, true>(m, A, thr, st);
          } else {
            if (V == 4) launch_step3<T, 4, false, true>(m, A, thr, st);
            else if (V == 2) launch_step3<T, 2, false, true>(m, A, thr, st);
            else launch_step3<T, 1, false, true>(m, A, thr, st);
          }
        } else {
          if (V == 2) launch_step3<T, 2, false, true>(m, A, thr, st);
          else launch_step3<T, 1, false, true>(m, A, thr, st);
        }
      }
    }
    if (timed) cudaEventRecord(e1, st);
  };
  run(false);
  run(true);
  pat_status s = cuda_check(cudaEventSynchronize(e1), "autotune sync");
  float ms = 0.0f;
  if (!s) s = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "autotune elapsed");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *us = 1e3f * ms / n_probe;
  return s;
}

// Step-kernel variants timed by pat_autotune (fields as in TuneCfg; only_v: the
// one V a variant is written for, 0 = any).  The packed f32x2 CSR, generic,
// tile-staged and fixed-width (ELL) families and their options; the persistent
// fixed-width ones are the fastest on large meshes.
constexpr int kTuneTableMax = 256;  // entries pat_autotune writes at most

struct TuneVariant {
  int packed, stage, chunk, zorder, big, pf, persist, pdl, wide, hint, batch, minb, early, only_v, own = 0,
      pfm = 0, dyn = 0;
};
static const TuneVariant kTuneVariants[] = {
    // packed, stage, chunk, zorder, big, pf, persist, pdl, wide, hint, batch, minb, early, only_v
    {1, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  0 packed f32x2, chunks of 2
    {1, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  1 packed, chunks of 4
    {1, 0, 8, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  2 packed, chunks of 8
    {1, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0},  //  3 packed, chunks of 2, own values first
    {1, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0},  //  4 packed, chunks of 4, own values first
    {1, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 6, 0, 0},  //  5 packed, chunks of 2, >= 6 blocks/SM
    {1, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 6, 0, 0},  //  6 packed, chunks of 4, >= 6 blocks/SM
    {0, 1, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  7 generic, metadata staged in shared memory
    {0, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  8 generic
    {2, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  //  9 tile-staged (bulk copies of 32-row tiles' source rows)
    {1, 0, 2, 1, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 10 packed, chunks of 2, Z-order rows
    {1, 0, 4, 1, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 11 packed, chunks of 4, Z-order rows
    {3, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 12 fixed-width (ELL)
    {3, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 6, 0, 1},  // 98 fixed-width, one sample, 6 blocks/SM (40 registers)
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 6, 0, 1},  // 99 16 slots, one sample, 6 blocks/SM (40 registers)
    {4, 0, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 13 persistent double-buffered tiles
    {1, 0, 2, 1, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 14 packed, chunks of 2, 1024-thread blocks, Z-order
    {3, 0, 4, 1, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 15 fixed-width, 1024-thread blocks, Z-order
    {1, 0, 2, 0, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 16 packed, chunks of 2, 1024-thread blocks
    {3, 0, 4, 0, 1, 0, 0, 0, 0, 0, 0, 1, 0, 0},  // 17 fixed-width, 1024-thread blocks
    {3, 0, 4, 0, 0, 1, 0, 0, 0, 0, 0, 1, 0, 0},  // 18 fixed-width, L2 prefetch 1 wave
    {3, 0, 4, 0, 0, 2, 0, 0, 0, 0, 0, 1, 0, 0},  // 19 fixed-width, L2 prefetch 2 waves
    {1, 0, 2, 0, 0, 1, 0, 0, 0, 0, 0, 1, 0, 0},  // 20 packed, chunks of 2, L2 prefetch 1 wave
    {1, 0, 4, 0, 0, 1, 0, 0, 0, 0, 0, 1, 0, 0},  // 21 packed, chunks of 4, L2 prefetch 1 wave
    {3, 0, 4, 0, 0, 1, 0, 0, 0, 0, 0, 6, 0, 4},  // 22 fixed-width, >= 6 blocks/SM, L2 prefetch (V = 4)
    {3, 0, 4, 0, 0, 1, 1, 0, 0, 0, 0, 1, 0, 0},  // 23 persistent, prefetch 1 stride
    {3, 0, 4, 0, 0, 2, 1, 0, 0, 0, 0, 1, 0, 0},  // 24 persistent, prefetch 2 strides
    {3, 0, 4, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0},  // 25 persistent
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 0, 1, 0, 0},  // 26 persistent, PDL
    {3, 0, 4, 0, 0, 1, 1, 1, 0, 0, 0, 1, 0, 0},  // 27 persistent, PDL, prefetch 1
    {3, 0, 4, 0, 0, 0, 1, 1, 1, 0, 0, 1, 0, 0},  // 28 persistent, PDL, 256-bit loads
    {3, 0, 4, 0, 0, 1, 1, 1, 1, 0, 0, 1, 0, 0},  // 29 persistent, PDL, 256-bit loads, prefetch 1
    {3, 0, 4, 0, 0, 0, 2, 1, 1, 0, 0, 1, 0, 0},  // 30 slabs, PDL, 256-bit loads
    {3, 0, 4, 0, 0, 1, 2, 1, 1, 0, 0, 1, 0, 0},  // 31 slabs, PDL, 256-bit loads, prefetch 1
    {3, 0, 4, 0, 0, 0, 2, 1, 0, 0, 0, 1, 0, 0},  // 32 slabs, PDL
    {3, 0, 4, 0, 0, 1, 2, 1, 0, 0, 0, 1, 0, 0},  // 33 slabs, PDL, prefetch 1
    {3, 0, 4, 0, 1, 0, 1, 1, 1, 0, 0, 1, 0, 0},  // 34 persistent, PDL, 1024-thread blocks, 256-bit loads
    {3, 0, 4, 0, 1, 0, 1, 1, 0, 0, 0, 1, 0, 0},  // 35 persistent, PDL, 1024-thread blocks
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 1, 0, 1, 0, 0},  // 36 persistent, PDL, L2 eviction hints
    {3, 0, 4, 0, 0, 1, 1, 1, 0, 1, 0, 1, 0, 0},  // 37 persistent, PDL, L2 eviction hints, prefetch 1
    {3, 0, 4, 0, 0, 0, 3, 1, 0, 0, 0, 1, 0, 0},  // 38 persistent, staged metadata, PDL
    {3, 0, 4, 0, 0, 1, 3, 1, 0, 0, 0, 1, 0, 0},  // 39 persistent, staged metadata, PDL, prefetch 1
    {3, 0, 4, 0, 0, 0, 3, 0, 0, 0, 0, 1, 0, 0},  // 40 persistent, staged metadata
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 8, 1, 0, 0},  // 41 persistent, PDL, batches of 8 source rows
    {3, 0, 4, 0, 0, 1, 1, 1, 0, 0, 8, 1, 0, 0},  // 42 persistent, PDL, batches of 8, prefetch 1
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 2, 1, 0, 0},  // 43 persistent, PDL, batches of 2
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 2, 6, 0, 0},  // 44 persistent, PDL, batches of 2, >= 6 blocks/SM
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 0},  // 45 persistent, PDL, batches of 4, metadata per batch
    {3, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 5, 0, 0},  // 46 the same, >= 5 blocks/SM
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 0},  // 47 16 slots, persistent, PDL, rounds of 4
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 1, 0},  // 48 16 slots, rounds of 4, columns per round
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 8, 1, 0, 0},  // 49 16 slots, rounds of 8 (2 blocks/SM)
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 8, 1, 1, 0},  // 50 16 slots, rounds of 8, columns per round
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 0, 8, 3, 1, 0},  // 51 the same, 3 blocks/SM
    {5, 0, 4, 0, 1, 0, 1, 1, 0, 0, 4, 1, 1, 0},  // 52 16 slots, 1024-thread blocks, rounds of 4
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 0},  // 53 16 slots, rounds of 4, tail walked one entry at a time
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 0},  // 54 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8},  // 55 16 slots row-major, rounds of 4
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 1, 8},  // 56 16 slots row-major, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8},  // 57 16 slots row-major, serial tail
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8},  // 58 16 slots row-major, columns per round, serial tail
    {6, 0, 4, 0, 1, 0, 1, 1, 0, 0, 4, 1, 1, 8},  // 59 16 slots row-major, 1024-thread blocks
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 1},  // 60 16 slots row-major, serial tail, own rows by cp.async
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 1},  // 61 the same, columns per round
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 1},  // 62 16 slots quad, columns per round, serial tail, own async
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 1, 1},  // 65 row-major, serial tail, own async, next metadata to L1
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 0, 1},  // 66 row-major, serial tail, next metadata to L1
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 0, 1},  // 67 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 2},  // 68 row-major, serial tail, own rows by bulk copies per warp
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 2},  // 69 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8, 2},  // 70 row-major, paired tail, own rows by bulk copies
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 1, 8, 2},  // 71 the same, columns per round
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 1, 1},  // 74 quad slots, serial tail, own async, quad's pairs to L1
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 1, 1},  // 75 the same, columns per round
    {5, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 0, 1},  // 76 quad slots, serial tail, quad's pairs to L1
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 3},  // 89 row-major, own x_{s-1} async, serial tail, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8, 3},  // 90 row-major, own x_{s-1} async, paired tail
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 1, 8, 3},  // 91 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 3},  // 92 row-major, own x_{s-1} async, serial tail
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 3, 1, 8, 1},  // 85 row-major, own async, serial tail, 3 blocks/SM
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 3, 0, 8, 1},  // 86 row-major, own async, paired tail, 3 blocks/SM
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 3, 0, 8, 1},  // 87 row-major, own async, serial tail, 3 blocks/SM, no early
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 3, 1, 8, 1},  // 88 row-major, own async, paired tail, 3 blocks/SM, early
    {6, 0, 4, 0, 0, 0, 1, 1, 1, 1, 4, 1, 1, 8, 1},  // 82 row-major, 256-bit metadata, serial tail, own async
    {6, 0, 4, 0, 0, 0, 1, 1, 1, 0, 4, 1, 1, 8, 1},  // 83 the same, paired tail
    {6, 0, 4, 0, 0, 0, 1, 1, 1, 1, 4, 1, 1, 8, 0},  // 84 row-major, 256-bit metadata, serial tail
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8, 1},  // 80 row-major, paired tail, own rows by cp.async
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 1, 8, 1},  // 81 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 0, 8, 1, 0, 1},  // 77 row-major, serial tail, own async, chunks by counter
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 1, 0, 1},  // 78 the same, columns per round
    {6, 0, 4, 0, 0, 0, 1, 1, 0, 1, 4, 1, 1, 8, 0, 0, 1},  // 79 row-major, serial tail, columns per round, by counter
    {8, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8, 0},  // 72 row quads (union of four rows' sources), K = 64
    {8, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8, 1},  // 73 row quads, own rows by cp.async
    {7, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 1, 0, 8},     // 63 row pairs (union of two rows' sources), 2 blocks/SM
    {7, 0, 4, 0, 0, 0, 1, 1, 0, 0, 4, 3, 0, 8},     // 64 row pairs, 3 blocks/SM
};

// Whether variant t exists for V samples per thread and K samples on mesh m.
static bool tune_applicable(const TuneVariant& t, const DeviceMesh& m, int V, int K) {
  if (t.only_v && V != t.only_v) return false;
  if (t.packed == 6)
    return m.prec == PAT_F32 && m.split && m.fwd.w16r_col && V == 8 && (!t.dyn || m.three_level) &&
           (t.own != 2 || (K >= 8 && K <= 256 && 32 % (K / 8) == 0 && m.d_status != nullptr));  // whole rows per chunk
  if (t.packed == 7)
    return m.prec == PAT_F32 && m.split && m.fwd.pair_col && m.adj3.pair_col && m.fwd.w16r_col && V == 8;
  if (t.packed == 8)
    return m.prec == PAT_F32 && m.split && m.fwd.quad_col && m.adj3.quad_col && m.fwd.w16r_col && V == 8 &&
           K == 64;
  if (t.packed == 5)  // 16-slot rows: V = 8 persistent, or one thread per row for K = 1
    return m.prec == PAT_F32 && m.split && m.fwd.w16_col && (!t.pfm || K == 64) &&
           (V == 8 || (V == 1 && K == 1 && t.batch == 4 && !t.early && !t.big && !t.hint));
  if ((t.batch || t.hint || t.wide || t.big) && V != 8) return false;
  if (t.persist == 3 && (V != 8 || K / V < 4)) return false;  // staged metadata: <= kStageRows rows per chunk
  if ((t.pf || t.persist) && V == 1) return false;
  if (t.minb > 1 && V == 8 && t.batch == 0) return false;  // would spill
  const bool f32s = m.prec == PAT_F32 && m.split;
  switch (t.packed) {
    case 1:
      if (!(f32s && (V == 4 || V == 8)) || (t.chunk == 8 && V == 8)) return false;
      break;
    case 2:
      if (!(f32s && V == 8 && K <= 8 * 1024 / kTileRows && m.n_tiles > 0)) return false;
      break;
    case 3:
      if (!(f32s && (V == 4 || V == 8 || (V == 1 && K == 1)) && m.fwd.ell_col)) return false;
      break;
    case 4:
      if (!(f32s && V == 8 && K <= 8 * 512 / kTileRows && m.n_tiles > 0)) return false;
      break;
    default:
      if (V == 8) return false;
  }
  return !(t.stage && K / V < 2);
}

pat_status autotune(const DeviceMesh& m, int K, char* ws, int n_probe, pat_tune_entry* table, int* n_entries,
                    cudaStream_t st) {
  const RtoLayout L = rto_layout(m, K);
  n_probe = std::max(2, std::min(n_probe, m.n_steps >= 4 ? m.n_steps - 2 : m.n_steps));  // + 2 untimed launches
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.d, 0, L.q_d - L.d, st), "autotune memset"));
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.q_d, 0, L.r_p - L.q_d, st), "autotune memset"));
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.r_d, 0, L.q_d - L.r_d, st), "autotune memset"));
  PAT_TRY(cuda_check(cudaMemsetAsync(ws + L.state, 0, L.gamma - L.state, st), "autotune memset"));
  const int vmax = m.prec == PAT_F64 ? 2 : 8;
  int n = 0;
  for (int dir = 0; dir < 2; ++dir) {
    TuneCfg best;
    float best_us = 1e30f;
    for (int V = vmax; V >= 1; V /= 2) {
      if (K % V) continue;
      for (const TuneVariant& t : kTuneVariants) {
        if (!tune_applicable(t, m, V, K)) continue;
        g_force_on = true;
        g_force.V = V;
        g_force.stage = t.stage;
        g_force.packed = t.packed;
        g_force.chunk = t.chunk;
        g_force.minb = t.minb;
        g_force.early = t.early;
        g_force.order = t.zorder;
        g_force.big = t.big;
        g_force.pf = t.pf;
        g_force.persist = t.persist;
        g_force.pdl = t.pdl;
        g_force.wide = t.wide;
        g_force.hint = t.hint;
        g_force.batch = t.batch;
        g_force.tail = t.packed >= 5 ? t.hint : 0;
        g_force.own = t.packed >= 5 ? t.own : 0;
        g_force.pfm = (t.packed == 5 || t.packed == 6) ? t.pfm : 0;
        g_force.dyn = t.packed == 6 ? t.dyn : 0;
        float us = 0.0f;
        pat_status s = m.prec == PAT_F64 ? probe_t<double>(m, K, ws, n_probe, dir, st, &us)
                                         : probe_t<float>(m, K, ws, n_probe, dir, st, &us);
        g_force_on = false;
        if (s) return s;
        if (table && n < kTuneTableMax)
          table[n] = pat_tune_entry{dir,    V,       t.stage, t.packed, t.packed ? t.chunk : 0,
                                    t.minb, t.early, t.zorder, t.big, t.pf, t.persist, t.pdl,
                                    t.wide, t.packed >= 5 ? 0 : t.hint, t.batch,
                                    t.packed >= 5 ? t.hint : 0, t.own, t.pfm, t.dyn, (double)us};
        ++n;
        if (us < best_us) {
          best_us = us;
          best = g_force;
        }
      }
    }
    std::lock_guard<std::mutex> lock(m.tune_mutex);
    m.tuned[std::make_pair(dir, K)] = best;
  }
  {
    // captured solves still hold the previous variant
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    drop_graphs_locked(m);
  }
  if (n_entries) *n_entries = n;
  return PAT_OK;
}

pat_status draw_normals(uint64_t seed, int stream_id, int64_t n_elem, int K, double* out, cudaStream_t st) {
  draw_normals_kernel<<<nblocks(n_elem * K), 256, 0, st>>>(seed, stream_id, n_elem, K, out);
  return cuda_check(cudaGetLastError(), "draw_normals launch");
}

}  // namespace pat
