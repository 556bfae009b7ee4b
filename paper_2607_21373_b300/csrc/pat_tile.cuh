// Tile-staged three-level step for K-stacked FP32 fields (K a multiple of 8).
//
// A block owns a tile of R = 64 rows that are consecutive in the Z-order of the
// node coordinates (a compact brick of the mesh).  Before it computes, the rows
// of x_s that its stiffness/boundary entries read -- the union of the tile's
// neighbourhoods, precomputed on the host as a few contiguous row ranges --
// are copied global -> shared memory by asynchronous bulk copies
// (cp.async.bulk with mbarrier completion), so the many neighbour reads of
// the tile hit shared memory and the memory system sees a handful of large
// contiguous transfers per tile instead of one 16-32 byte load per thread
// per entry.  Column indices are replaced by 16-bit shared-memory slots.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pat_kernels.cuh"

namespace pat {

constexpr int kTileRows = 64;

struct TileArgs {
  const int32_t* __restrict__ range_ptr;  // [T+1] into the range arrays
  const int32_t* __restrict__ range_src;  // first source row of a range
  const int32_t* __restrict__ range_cnt;  // rows in a range
  const int32_t* __restrict__ range_slot; // first shared-memory slot of a range
  const int32_t* __restrict__ tile_slots; // [T] staged rows per tile
  const uint16_t* __restrict__ slot;      // per CSR entry: shared-memory slot of its source row
  int32_t* status;                        // device status word (PAT_ETIMEOUT on a stuck copy)
  int32_t n_tiles;                        // blocks beyond the tiles gather the sensor observations
  const int32_t* __restrict__ order;      // rows of tile t: order[t*R .. t*R+R)
  long long wait_cycles;                  // SM cycles a block waits for its copies before it reports
                                          // PAT_ETIMEOUT and gives up on the tile
};

// Cycles a block that gave up still waits for its copies in flight to land
// before it exits (its shared memory must outlive them): about two seconds at
// 2 GHz, far beyond any copy.
constexpr long long kDrainWait = 4000000000ll;

// observation of the input state by thread g of the gather blocks
template <int V>
__device__ __forceinline__ void gather_obs(const Step3Args<float>& A, int64_t g) {
  const int KV = A.K / V;
  if (A.y_out == nullptr || g >= (int64_t)A.n_obs * KV) return;
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
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait for phase 0 of an mbarrier: false once `cycles` SM clock cycles
// have passed without completion.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int V, bool ADJ>
__global__ void __launch_bounds__(1024) step3t_kernel(const Step3Args<float> A, const TileArgs Tl) {
  static_assert(V == 8, "tile kernel handles 8 samples per thread");
  constexpr int P = V / 2;
  extern __shared__ __align__(128) unsigned char tile_smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(tile_smem);
  float* rows = reinterpret_cast<float*>(tile_smem + 128);
  const int KV = A.K / V;
  const int tile = blockIdx.x;
  if (tile >= Tl.n_tiles) {
    gather_obs<V>(A, (int64_t)(tile - Tl.n_tiles) * blockDim.x + threadIdx.x);
    return;
  }
  if (A.xn == nullptr || A.row_threads == 0) return;  // no rows to update (the host never launches this)
  const int64_t r0 = (int64_t)tile * kTileRows;
  const uint32_t bar_s = smem_u32(bar);
  const size_t row_bytes = (size_t)A.K * 4;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // warp 0: lane 0 announces the tile's bytes, then the lanes issue the
    // range copies in parallel
    const int q0 = Tl.range_ptr[tile], q1 = Tl.range_ptr[tile + 1];
    if (threadIdx.x == 0) {
      const uint32_t bytes = (uint32_t)((size_t)Tl.tile_slots[tile] * row_bytes);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes) : "memory");
    }
    __syncwarp();
    for (int q = q0 + (int)threadIdx.x; q < q1; q += 32) {
      const float* src = A.x + (int64_t)Tl.range_src[q] * A.K;
      const uint32_t dst = smem_u32(rows + (size_t)Tl.range_slot[q] * A.K);
      const uint32_t n = (uint32_t)((size_t)Tl.range_cnt[q] * row_bytes);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
          "l"(src), "r"(n), "r"(bar_s)
          : "memory");
    }
  }
  const int lr = threadIdx.x / KV;  // row within the tile
  const int kv = threadIdx.x - lr * KV;
  const bool active = r0 + lr < A.N;
  const int64_t row = active ? (int64_t)Tl.order[r0 + lr] : 0;
  const int64_t off = row * A.K + (int64_t)kv * V;
  // the node's previous value comes from global memory while the copies run
  Pack<float, V> xpi;
  if (active && A.prev_mode == 0) xpi = ld<float, V>(A.xp + off);
  if (!mbar_wait(bar_s, Tl.wait_cycles)) {
    atomicExch(Tl.status, (int)PAT_ETIMEOUT);
    mbar_wait(bar_s, kDrainWait);  // let the copies land before the block's memory is released
    return;
  }
  if (!active) return;
  const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
  const int ni = ADJ ? (int)A.ninj[row] : 0;
  const int eA = e1 - ni;
  const int eB = eA - (int)A.nb[row];
  u64 acc[P], accl[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
  const float* sk = rows + kv * V;
#pragma unroll 4
  for (int e = e0; e < eA; ++e) {
    const float2 c = A.hl[e];
    const float* sp = sk + (size_t)Tl.slot[e] * A.K;
    const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sp);
    const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sp + 4);
    const u64 ch = dup2(c.x), cl = dup2(c.y);
    acc[0] = ffma2(ch, v0.x, acc[0]);
    accl[0] = ffma2(cl, v0.x, accl[0]);
    acc[1] = ffma2(ch, v0.y, acc[1]);
    accl[1] = ffma2(cl, v0.y, accl[1]);
    acc[2] = ffma2(ch, v1.x, acc[2]);
    accl[2] = ffma2(cl, v1.x, accl[2]);
    acc[3] = ffma2(ch, v1.y, acc[3]);
    accl[3] = ffma2(cl, v1.y, accl[3]);
  }
  const uint32_t Ku = (uint32_t)A.K;
  if (eB < eA && A.prev_mode != 2) {
    // boundary entries act on w_j = x_j - xp_j: remove their xp_j part
    for (int e = eB; e < eA; ++e) {
      const float2 c = A.hl[e];
      u64 x[P];
      if (A.prev_mode == 0) {
        ld_pairs<P>(A.xp + (int64_t)kv * V + (size_t)(A.col[e] & kIdxMask) * Ku, x);
      } else {
        const float* sp = sk + (size_t)Tl.slot[e] * A.K;  // xp = x
        const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sp);
        const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sp + 4);
        x[0] = v0.x;
        x[1] = v0.y;
        x[2] = v1.x;
        x[3] = v1.y;
      }
      const u64 ch = dup2(-c.x), cl = dup2(-c.y);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        acc[p] = ffma2(ch, x[p], acc[p]);
        accl[p] = ffma2(cl, x[p], accl[p]);
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
  // own x from the staged rows (the row itself is one of its entries' sources)
  const Pack<float, V> xi = ld<float, V>(A.x + off);
  if (A.prev_mode != 0) {
#pragma unroll
    for (int q = 0; q < V; ++q) xpi.v[q] = (A.prev_mode == 1) ? xi.v[q] : 0.0f;
  }
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

// ---------------------------------------------------------------------------
// Fixed-width (ELL) packed kernel: a row's first 8 entries sit at [row][8], so
// their columns and coefficients arrive in one round of broadcast loads with no
// row-pointer load in front (padding slots read the row itself with a zero
// coefficient); longer rows continue in an overflow CSR.  Entries 0..7 are
// then processed as two chunks of 4 neighbour rows.
// ---------------------------------------------------------------------------
// Stiffness / boundary entry e (< the row's count eA) of a fixed-width row:
// slots 0..7, then the row's overflow list.
template <int V>
__device__ __forceinline__ void ell_entry(const Step3Args<float>& A, int64_t row, int e, uint32_t* col, float2* c) {
  if (e < 8) {
    *col = A.ell_col[row * 8 + e];
    *c = A.ell_hl[row * 8 + e];
  } else {
    const int64_t o = A.ovf_ptr[row] + (e - 8);
    *col = A.ovf_col[o];
    *c = A.ovf_hl[o];
  }
}

// One-sample row tail: entries e0 <= e < e1 fetched by entry(e, &col, &c),
// their sources gathered from xs and accumulated with sign sg (+1 or -1, so
// sg * c is exact) in entry order: the same products in the same order as a
// walk one entry at a time, with 4 entries' loads in flight per round instead
// of two dependent loads per entry.
template <typename Entry>
__device__ __forceinline__ void tail1(int e0, int e1, const float* __restrict__ xs, float sg, Entry entry,
                                      float& acc, float& accl) {
  for (int e = e0; e < e1; e += 4) {
    uint32_t col[4];
    float2 c[4];
    float x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e + j < e1) entry(e + j, &col[j], &c[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (e + j < e1) ? xs[col[j]] : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e + j < e1) {
        acc = fmaf(sg * c[j].x, x[j], acc);
        accl = fmaf(sg * c[j].y, x[j], accl);
      }
  }
}

// One-sample sensor term: src = sum over the row's sensor entries j < ni (in
// order, ya then yb, either may be absent) of c_j (ya + yb)[col_j], 4 entries'
// loads in flight per round (the same products in the same order).
template <typename Entry>
__device__ __forceinline__ float inj1(int ni, const float* __restrict__ ya, const float* __restrict__ yb, Entry entry) {
  float src = 0.0f;
  for (int e = 0; e < ni; e += 4) {
    uint32_t col[4];
    float2 c[4];
    float a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e + j < ni) entry(e + j, &col[j], &c[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = (ya && e + j < ni) ? ya[col[j]] : 0.0f;
      b[j] = (yb && e + j < ni) ? yb[col[j]] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (e + j < ni) {
        if (ya) src = fmaf(c[j].x, a[j], src);
        if (yb) src = fmaf(c[j].x, b[j], src);
      }
  }
  return src;
}

// Sensor (injection) entry j of a fixed-width row with eA stiffness / boundary
// entries: always in the overflow list, after the stiffness entries beyond 8.
__device__ __forceinline__ void inj_entry(const Step3Args<float>& A, int64_t row, int j, int eA, uint32_t* col,
                                          float2* c) {
  const int64_t o = A.ovf_ptr[row] + max(eA - 8, 0) + j;
  *col = A.ovf_col[o];
  *c = A.ovf_hl[o];
}

// Four consecutive fixed-width slots of a row (columns c, (hi, lo) pairs in
// ha, hb; padding slots carry a zero coefficient): gather the V samples of
// each source row, then accumulate hi and lo products in slot order.
template <int P>
__device__ __forceinline__ void ell_half(const float* xk, uint32_t Ku, uint4 c, float4 ha, float4 hb,
                                         u64 (&acc)[P], u64 (&accl)[P]) {
  const uint32_t cols[4] = {c.x, c.y, c.z, c.w};
  const float2 cf[4] = {make_float2(ha.x, ha.y), make_float2(ha.z, ha.w), make_float2(hb.x, hb.y),
                        make_float2(hb.z, hb.w)};
  u64 x[4][P];
#pragma unroll
  for (int q = 0; q < 4; ++q) ld_pairs<P>(xk + (size_t)cols[q] * Ku, x[q]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 cc = cf[q];
    const u64 ch = dup2(cc.x), cl = dup2(cc.y);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      acc[p] = ffma2(ch, x[q][p], acc[p]);
      accl[p] = ffma2(cl, x[q][p], accl[p]);
    }
  }
}

// Row metadata of one 32-thread chunk (at most kStageRows rows, so K / V >= 4),
// staged in shared memory by the warp that will process it.
constexpr int kStageRows = 9;
struct alignas(16) EllStage {
  uint32_t desc[12];
  uint4 col[2 * kStageRows];
  float4 hl[4 * kStageRows];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// L2 eviction-priority hints (H variants of the fixed-width kernel): the new
// state x_{s+1} and the row metadata are kept (evict_last), since the next
// steps read them again; the own rows of x_{s-1}, read for the last time,
// leave first (evict_first).
__device__ __forceinline__ uint64_t l2_policy_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_hint_f4(const float* p, uint64_t pol) {
  float4 v;
  asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_hint_u4(const void* p, uint64_t pol) {
  uint4 v;
  asm("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint_f4(float* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}

// Sample layout of the fixed-width kernel's threads.  With W (256-bit loads,
// V = 8) a thread's 8 samples are contiguous, kv*8 .. kv*8+7, read and written
// by one 32-byte access.  Otherwise, with V = 8 a thread's
// samples are two runs of 4: kv*4 .. kv*4+3 and K/2 + kv*4 .. K/2 + kv*4+3, so
// that one 16-byte load per lane covers, across the 8 lanes of a row, one
// contiguous 128-byte span of a source row (instead of every other 16 bytes of
// 256); with V = 4 a thread's 4 samples are one run.  Only the assignment of
// samples to threads changes: every sample's arithmetic is the same.
template <int V, bool W = false>
__device__ __forceinline__ void ld_runs(const float* p, int64_t hs, u64 (&out)[V / 2]) {
  if constexpr (W) {  // one 256-bit load of 8 contiguous samples
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(out[0]), "=l"(out[1]), "=l"(out[2]), "=l"(out[3])
                 : "l"(p));
    return;
  }
  const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(p);
  out[0] = v0.x;
  out[1] = v0.y;
  if constexpr (V == 8) {
    const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(p + hs);
    out[2] = v1.x;
    out[3] = v1.y;
  }
}

template <int V, bool W = false>
__device__ __forceinline__ Pack<float, V> ld_run_pack(const float* p, int64_t hs) {
  Pack<float, V> r;
  if constexpr (W) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
                   "=f"(r.v[6]), "=f"(r.v[7])
                 : "l"(p));
    return r;
  }
  const float4 v0 = *reinterpret_cast<const float4*>(p);
  r.v[0] = v0.x, r.v[1] = v0.y, r.v[2] = v0.z, r.v[3] = v0.w;
  if constexpr (V == 8) {
    const float4 v1 = *reinterpret_cast<const float4*>(p + hs);
    r.v[4] = v1.x, r.v[5] = v1.y, r.v[6] = v1.z, r.v[7] = v1.w;
  }
  return r;
}

template <int V, bool W = false>
__device__ __forceinline__ void st_run_pack(float* p, int64_t hs, const Pack<float, V>& x) {
  if constexpr (W) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(x.v[0]), "f"(x.v[1]),
                 "f"(x.v[2]), "f"(x.v[3]), "f"(x.v[4]), "f"(x.v[5]), "f"(x.v[6]), "f"(x.v[7])
                 : "memory");
    return;
  }
  *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
  if constexpr (V == 8) *reinterpret_cast<float4*>(p + hs) = make_float4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

// The tail of a fixed-width row of WD slots: its stiffness / boundary entries
// beyond the slots (acting on x, coefficient c) and the xp parts of its
// boundary entries (the last nb of its eA entries, acting on pk with -c).  The
// entries are taken in pairs whose two gathers are in flight together (more
// would spill at the register budget of the persistent kernels), and their
// products are accumulated in entry order, exactly as a one-entry-at-a-time
// walk would: the boundary rows of a cube carry up to 18 entries and 7
// corrections, and a serial walk makes them several times slower than an
// interior row and holds up the warp that has one.
// Positions of slot e of a fixed-width row of WD slots: row-major, or (QUAD,
// 16 slots) interleaved by quads of rows (see the 16-slot layout in pat_wide.cuh).
template <int WD, bool QUAD>
__device__ __forceinline__ int64_t slot_col_at(int64_t row, int e) {
  if constexpr (QUAD) return (row >> 2) * (4 * WD) + (e >> 2) * 16 + (row & 3) * 4 + (e & 3);
  return row * WD + e;
}
template <int WD, bool QUAD>
__device__ __forceinline__ int64_t slot_hl_at(int64_t row, int e) {
  if constexpr (QUAD) return (row >> 2) * (4 * WD) + (e >> 1) * 8 + (row & 3) * 2 + (e & 1);
  return row * WD + e;
}

// Slots the V = 8 eight-slot rows gather in their rounds: an interior row of
// the pruned Kuhn lattice has 7 entries, so the eighth slot would only read the
// row itself with a zero coefficient; entry 7 onward goes to the tail.
constexpr int kMain8 = 7;

// CORR_ONLY: only the xp parts of the boundary entries (the caller has
// accumulated every entry's x part already).
// T0: the first entry the tail takes (the caller's slot loop covered entries
// 0 .. T0-1; entries T0 .. WD-1 are read from their slots, the rest from the
// overflow list).
template <int V, bool W, int WD, int TB = 2, bool QUAD = false, bool CORR_ONLY = false, int T0 = WD>
__device__ __forceinline__ void fixed_row_tail(const Step3Args<float>& A, int64_t row, int eA, int nb,
                                               const float* xk, const float* pk, int64_t hs, uint32_t Ku,
                                               u64 (&acc)[V / 2], u64 (&accl)[V / 2]) {
  constexpr int P = V / 2;
  if ((CORR_ONLY || eA <= T0) && (nb == 0 || pk == nullptr)) return;
  const int64_t o0 = (int64_t)A.ovf_ptr[row] - WD;  // overflow index of entry e >= WD: o0 + e
  auto fetch = [&](int e, uint32_t* col, float2* c) {
    if (e < WD) {
      *col = A.ell_col[slot_col_at<WD, QUAD>(row, e)];
      *c = A.ell_hl[slot_hl_at<WD, QUAD>(row, e)];
    } else {
      *col = A.ovf_col[o0 + e];
      *c = A.ovf_hl[o0 + e];
    }
  };
  auto batch = [&](int e0, int e1, const float* src, float sign) {
    for (; e0 < e1; e0 += TB) {
      uint32_t cq[TB];
      float2 cf[TB];
      u64 x[TB][P];
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        cq[q] = 0u;
        cf[q] = make_float2(0.0f, 0.0f);
        if (e0 + q < e1) fetch(e0 + q, &cq[q], &cf[q]);
      }
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        if (e0 + q < e1) {
          ld_runs<V, W>(src + (size_t)cq[q] * Ku, hs, x[q]);
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) x[q][p] = 0ull;
        }
      }
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        if (e0 + q < e1) {
          const u64 ch = dup2(sign * cf[q].x), cl = dup2(sign * cf[q].y);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc[p] = ffma2(ch, x[q][p], acc[p]);
            accl[p] = ffma2(cl, x[q][p], accl[p]);
          }
        }
      }
    }
  };
  if constexpr (TB == 1) {
    if constexpr (!CORR_ONLY) batch(T0, eA, xk, 1.0f);
    if (nb > 0 && pk != nullptr) batch(eA - nb, eA, pk, -1.0f);
  } else {
    // the tail's x entries and the corrections as one sequence, so a batch can
    // hold the last x entry and the first correction (one round trip fewer
    // when the x entries are odd in number); the products keep their order
    const int nx = CORR_ONLY ? 0 : max(eA - T0, 0);
    const int nc = (nb > 0 && pk != nullptr) ? nb : 0;
    const int c0 = eA - nb;  // first boundary entry
    for (int v0 = 0; v0 < nx + nc; v0 += TB) {
      uint32_t cq[TB];
      float2 cf[TB];
      u64 x[TB][P];
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        const int v = v0 + q;
        cq[q] = 0u;
        cf[q] = make_float2(0.0f, 0.0f);
        if (v < nx + nc) fetch(v < nx ? T0 + v : c0 + (v - nx), &cq[q], &cf[q]);
      }
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        const int v = v0 + q;
        if (v < nx + nc) {
          ld_runs<V, W>((v < nx ? xk : pk) + (size_t)cq[q] * Ku, hs, x[q]);
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) x[q][p] = 0ull;
        }
      }
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        const int v = v0 + q;
        if (v < nx + nc) {
          const float sign = v < nx ? 1.0f : -1.0f;
          const u64 ch = dup2(sign * cf[q].x), cl = dup2(sign * cf[q].y);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc[p] = ffma2(ch, x[q][p], acc[p]);
            accl[p] = ffma2(cl, x[q][p], accl[p]);
          }
        }
      }
    }
  }
}

template <int V, bool ADJ, bool W = false, bool H = false, bool SMD = false, int NB = 4, bool PB = (NB == 2)>
__device__ __forceinline__ void step3e_row(const Step3Args<float>& A, const int64_t t,
                                           const EllStage* sm = nullptr, int64_t r0 = 0) {
  static_assert(!H || (V == 8 && !W), "cache-hint variant: V = 8, 128-bit loads");
  static_assert(!SMD || (V == 8 && !W && !H), "staged-metadata variant: V = 8, 128-bit loads");
  constexpr int P = V / 2;
  const int KV = A.K / V;
  if (t >= A.row_threads) {
    gather_obs<V>(A, t - A.row_threads);
    return;
  }
  const int64_t rowi = div_kv(t, KV);
  const int kv = (int)(t - rowi * KV);
  const int64_t row = A.order ? (int64_t)A.order[rowi] : rowi;
  static_assert(V == 4 || V == 8, "fixed-width kernel: V = 4 or 8");
  static_assert(!W || V == 8, "256-bit loads: V = 8");
  const int64_t hs = (V == 8 && !W) ? A.K / 2 : 0;  // offset of a thread's second run of samples
  const int64_t base = (int64_t)kv * (W ? 8 : 4);   // offset of its first run
  const int64_t off = row * A.K + base;
  const int lr = SMD ? (int)(row - r0) : 0;  // row within the staged chunk
  const uint32_t desc = SMD ? sm->desc[lr] : A.ell_desc[row];
  const int n = (int)(desc & 255u), nb = (int)((desc >> 8) & 255u), ni = (int)((desc >> 16) & 255u);
  const int eA = n - ni;  // stiffness + boundary entries
  // V = 8: all 8 columns and coefficient pairs loaded up front; V = 4: per
  // half of the row, which needs fewer registers (same arithmetic order)
  uint4 c0 = make_uint4(0u, 0u, 0u, 0u), c1 = c0;
  float4 h01 = make_float4(0.f, 0.f, 0.f, 0.f), h23 = h01, h45 = h01, h67 = h01;
  if constexpr (W) {
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(c0.x), "=r"(c0.y), "=r"(c0.z), "=r"(c0.w), "=r"(c1.x), "=r"(c1.y), "=r"(c1.z), "=r"(c1.w)
                 : "l"(A.ell_col + row * 8));
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(h01.x), "=f"(h01.y), "=f"(h01.z), "=f"(h01.w), "=f"(h23.x), "=f"(h23.y), "=f"(h23.z),
                   "=f"(h23.w)
                 : "l"(A.ell_hl + row * 8));
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(h45.x), "=f"(h45.y), "=f"(h45.z), "=f"(h45.w), "=f"(h67.x), "=f"(h67.y), "=f"(h67.z),
                   "=f"(h67.w)
                 : "l"(A.ell_hl + row * 8 + 4));
  } else if constexpr (SMD) {
    c0 = sm->col[2 * lr];
    c1 = sm->col[2 * lr + 1];
    h01 = sm->hl[4 * lr];
    h23 = sm->hl[4 * lr + 1];
    h45 = sm->hl[4 * lr + 2];
    h67 = sm->hl[4 * lr + 3];
  } else if constexpr (H) {
    const uint64_t keep = l2_policy_last();
    c0 = ld_hint_u4(A.ell_col + row * 8, keep);
    c1 = ld_hint_u4(A.ell_col + row * 8 + 4, keep);
    h01 = ld_hint_f4(reinterpret_cast<const float*>(A.ell_hl + row * 8), keep);
    h23 = ld_hint_f4(reinterpret_cast<const float*>(A.ell_hl + row * 8 + 2), keep);
    h45 = ld_hint_f4(reinterpret_cast<const float*>(A.ell_hl + row * 8 + 4), keep);
    h67 = ld_hint_f4(reinterpret_cast<const float*>(A.ell_hl + row * 8 + 6), keep);
  } else if constexpr (V == 8 && !PB) {
    c0 = *reinterpret_cast<const uint4*>(A.ell_col + row * 8);
    c1 = *reinterpret_cast<const uint4*>(A.ell_col + row * 8 + 4);
    h01 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8);
    h23 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 2);
    h45 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 4);
    h67 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 6);
  }
  const uint32_t Ku = (uint32_t)A.K;
  u64 acc[P], accl[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
  if (A.x) {
    const float* xk = A.x + base;
    if constexpr (V == 8 && PB) {
      // batches of NB (2 or 4) source rows, each batch's columns and
      // coefficient pairs loaded with it (L1 hits after the first): fewer live
      // registers than loading all 8 up front
      static_assert(NB == 2 || NB == 4, "per-batch metadata: batches of 2 or 4");
#pragma unroll
      for (int h = 0; h < 8 / NB; ++h) {
        uint32_t cq[NB];
        if constexpr (NB == 2) {
          const uint2 c = *reinterpret_cast<const uint2*>(A.ell_col + row * 8 + 2 * h);
          cq[0] = c.x, cq[1] = c.y;
        } else {
          const uint4 c = *reinterpret_cast<const uint4*>(A.ell_col + row * 8 + 4 * h);
          cq[0] = c.x, cq[1] = c.y, cq[2] = c.z, cq[3] = c.w;
        }
        u64 x[NB][P];
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (NB * h + q < kMain8) ld_runs<V, W>(xk + (size_t)cq[q] * Ku, hs, x[q]);
        float2 cf[NB];
#pragma unroll
        for (int q = 0; q < NB; q += 2) {
          const float4 hq = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + NB * h + q);
          cf[q] = make_float2(hq.x, hq.y);
          cf[q + 1] = make_float2(hq.z, hq.w);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (NB * h + q >= kMain8) continue;
          const u64 ch = dup2(cf[q].x), cl = dup2(cf[q].y);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc[p] = ffma2(ch, x[q][p], acc[p]);
            accl[p] = ffma2(cl, x[q][p], accl[p]);
          }
        }
      }
    } else if constexpr (V == 8) {
      const uint32_t cols[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      const float2 cf[8] = {make_float2(h01.x, h01.y), make_float2(h01.z, h01.w), make_float2(h23.x, h23.y),
                            make_float2(h23.z, h23.w), make_float2(h45.x, h45.y), make_float2(h45.z, h45.w),
                            make_float2(h67.x, h67.y), make_float2(h67.z, h67.w)};
      // NB source rows in flight per batch: 8 (one gather latency per row,
      // more registers), 4 (default) or 2 (fewer registers, more warps)
      static_assert(NB == 2 || NB == 4 || NB == 8, "batch of 2, 4 or 8 source rows");
#pragma unroll
      for (int h = 0; h < 8 / NB; ++h) {
        u64 x[NB][P];
        // the 8 slots hold only stiffness / boundary entries and padding (the
        // row itself with a zero coefficient): no per-entry test
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (NB * h + q < kMain8) ld_runs<V, W>(xk + (size_t)cols[NB * h + q] * Ku, hs, x[q]);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          if (NB * h + q >= kMain8) continue;
          const float2 c = cf[NB * h + q];
          const u64 ch = dup2(c.x), cl = dup2(c.y);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc[p] = ffma2(ch, x[q][p], acc[p]);
            accl[p] = ffma2(cl, x[q][p], accl[p]);
          }
        }
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 cq = *reinterpret_cast<const uint4*>(A.ell_col + row * 8 + 4 * h);
        const float4 ha = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 4 * h);
        const float4 hb = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 4 * h + 2);
        ell_half<P>(xk, Ku, cq, ha, hb, acc, accl);
      }
    }
    // entries beyond the 8 slots, then the xp parts of the boundary entries
    // (boundary entries act on w_j = x_j - xp_j)
    const float* pk = A.prev_mode == 2 ? nullptr : (A.prev_mode == 0 ? A.xp : A.x) + base;
    // (V = 8: the rounds covered slots 0 .. 6, the tail starts at entry 7)
    fixed_row_tail<V, W, 8, 2, false, false, (V == 8 ? kMain8 : 8)>(A, row, eA, nb, xk, pk, hs, Ku, acc, accl);
  }
  float src[V];
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  if constexpr (ADJ) {
    for (int e = 0; e < ni; ++e) {
      uint32_t col;
      float2 c;
      inj_entry(A, row, e, eA, &col, &c);
      const int64_t j = (int64_t)col;
      if (A.ya) {
        const Pack<float, V> y = ld_run_pack<V, W>(A.ya + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
      }
      if (A.yb) {
        const Pack<float, V> y = ld_run_pack<V, W>(A.yb + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
      }
    }
  }
  if constexpr (V == 8 && PB) {
    // the update one run of 4 samples at a time (fewer live registers)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t o = off + r * hs;
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 xv = A.x ? *reinterpret_cast<const float4*>(A.x + o) : z;
      const float4 pv = A.prev_mode == 0 ? *reinterpret_cast<const float4*>(A.xp + o) : (A.prev_mode == 1 ? xv : z);
      const float xs[4] = {xv.x, xv.y, xv.z, xv.w}, ps[4] = {pv.x, pv.y, pv.z, pv.w};
      float out[4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const float2 a = unpack2(acc[2 * r + p]), al = unpack2(accl[2 * r + p]);
        const float w0 = xs[2 * p] - ps[2 * p], w1 = xs[2 * p + 1] - ps[2 * p + 1];
        out[2 * p] = xs[2 * p] + (w0 - (a.x + al.x) + A.inj_scale * src[4 * r + 2 * p]);
        out[2 * p + 1] = xs[2 * p + 1] + (w1 - (a.y + al.y) + A.inj_scale * src[4 * r + 2 * p + 1]);
      }
      *reinterpret_cast<float4*>(A.xn + o) = make_float4(out[0], out[1], out[2], out[3]);
    }
    return;
  }
  Pack<float, V> xi, xpi, xo;
  if (A.x) {
    xi = ld_run_pack<V, W>(A.x + off, hs);
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) xi.v[q] = 0.0f;
  }
  if (A.prev_mode == 0) {
    if constexpr (H) {
      const uint64_t leave = l2_policy_first();
      const float4 a = ld_hint_f4(A.xp + off, leave), b = ld_hint_f4(A.xp + off + hs, leave);
      xpi.v[0] = a.x, xpi.v[1] = a.y, xpi.v[2] = a.z, xpi.v[3] = a.w;
      xpi.v[4] = b.x, xpi.v[5] = b.y, xpi.v[6] = b.z, xpi.v[7] = b.w;
    } else {
      xpi = ld_run_pack<V, W>(A.xp + off, hs);
    }
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) xpi.v[q] = (A.prev_mode == 1) ? xi.v[q] : 0.0f;
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const float2 a = unpack2(acc[p]), al = unpack2(accl[p]);
    const float w0 = xi.v[2 * p] - xpi.v[2 * p], w1 = xi.v[2 * p + 1] - xpi.v[2 * p + 1];
    xo.v[2 * p] = xi.v[2 * p] + (w0 - (a.x + al.x) + A.inj_scale * src[2 * p]);
    xo.v[2 * p + 1] = xi.v[2 * p + 1] + (w1 - (a.y + al.y) + A.inj_scale * src[2 * p + 1]);
  }
  if constexpr (H) {
    const uint64_t keep = l2_policy_last();
    st_hint_f4(A.xn + off, make_float4(xo.v[0], xo.v[1], xo.v[2], xo.v[3]), keep);
    st_hint_f4(A.xn + off + hs, make_float4(xo.v[4], xo.v[5], xo.v[6], xo.v[7]), keep);
  } else {
    st_run_pack<V, W>(A.xn + off, hs, xo);
  }
}

template <int V, bool ADJ>
__device__ __forceinline__ void step3e_body(const Step3Args<float>& A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (A.pf_rows > 0 && threadIdx.x == 0 && t < A.row_threads) {
    const int KV = A.K / V;
    prefetch_ahead<true>(A, div_kv(t, KV) + A.pf_rows,
                         div_kv(min(t + (int64_t)blockDim.x, A.row_threads), KV) + 1 + A.pf_rows);
  }
  step3e_row<V, ADJ>(A, t);
}

template <int V, bool ADJ>
__global__ void __launch_bounds__(256, V == 8 ? 4 : 5) step3e_kernel(const Step3Args<float> A) {
  step3e_body<V, ADJ>(A);
}

// Persistent form: a grid of resident blocks whose warps each walk 32-thread
// chunks c, c + S, c + 2S, ... (S = warps in the grid).  A warp takes its next
// chunk as soon as it is done, instead of idling until every warp of its block
// has finished.  With A.pf_rows = d > 0, thread 0 asks L2 (bulk prefetch) for
// the rows of the block's chunks d strides ahead, once per stride.
// Launched as a programmatic dependent of the previous step, the grid's blocks
// may become resident while that step drains; griddepcontrol.wait holds them
// until it has completed and its writes are visible (a no-op otherwise).
template <int V, bool ADJ, bool W, int BS = 256, bool H = false, int NB = 4,
          int MINB = (BS == 256 ? (V == 8 ? 4 : 5) : 1), bool PB = (NB == 2)>
__global__ void __launch_bounds__(BS, MINB) step3e_persist_kernel(const Step3Args<float> A, int64_t n_chunks) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int KV = A.K / V;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t S = (int64_t)gridDim.x * wpb;
  for (int64_t cb = (int64_t)blockIdx.x * wpb; cb < n_chunks; cb += S) {
    if (A.pf_rows > 0 && threadIdx.x == 0) {
      const int64_t t0 = (cb + A.pf_rows * S) * 32;
      if (t0 < A.row_threads)
        prefetch_ahead<true>(A, div_kv(t0, KV), div_kv(min(t0 + 32 * (int64_t)wpb, A.row_threads) - 1, KV) + 1);
    }
    const int64_t c = cb + (threadIdx.x >> 5);
    if (c < n_chunks) step3e_row<V, ADJ, W, H, false, NB, PB>(A, c * 32 + lane);
  }
}

// Persistent grid-stride kernel with the row metadata software-pipelined
// through shared memory: while a warp processes chunk c, its lanes have
// cp.async copies of chunk c + S's descriptors, columns and coefficient pairs
// in flight into the warp's other stage buffer, so a chunk's critical path
// starts with shared-memory reads instead of an L2 round trip before the
// neighbour gather.  V = 8, K / V >= 4 (at most kStageRows rows per chunk),
// rows in natural order.  Optional L2 bulk prefetch as in the persistent kernel.
template <bool ADJ>
__global__ void __launch_bounds__(256, 4) step3e_stage_kernel(const Step3Args<float> A, int64_t n_chunks) {
  constexpr int V = 8, WPB = 8;
  __shared__ EllStage stage[WPB][2];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int KV = A.K / V;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t S = (int64_t)gridDim.x * WPB;
  // copies of chunk c's metadata into dst: per row one 4-byte descriptor,
  // two 16-byte column pieces, four 16-byte coefficient pieces
  auto issue = [&](int64_t c, EllStage* dst) {
    const int64_t t0 = c * 32;
    if (t0 < A.row_threads) {
      const int64_t q0 = div_kv(t0, KV), q1 = div_kv(min(t0 + 32, A.row_threads) - 1, KV);
      const int total = (int)(q1 - q0 + 1) * 7;
      for (int i = lane; i < total; i += 32) {
        const int r = i / 7, part = i - 7 * r;
        const int64_t row = q0 + r;
        if (part == 0)
          cp_async4(&dst->desc[r], A.ell_desc + row);
        else if (part < 3)
          cp_async16(&dst->col[2 * r + part - 1], A.ell_col + row * 8 + 4 * (part - 1));
        else
          cp_async16(&dst->hl[4 * r + part - 3], A.ell_hl + row * 8 + 2 * (part - 3));
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int64_t c = (int64_t)blockIdx.x * WPB + w;
  int s = 0;
  issue(c, &stage[w][0]);
  for (; c < n_chunks; c += S) {
    if (A.pf_rows > 0 && threadIdx.x == 0) {
      const int64_t cb = c - w, t0 = (cb + A.pf_rows * S) * 32;
      if (t0 < A.row_threads)
        prefetch_ahead<true>(A, div_kv(t0, KV), div_kv(min(t0 + 32 * (int64_t)WPB, A.row_threads) - 1, KV) + 1);
    }
    issue(c + S, &stage[w][s ^ 1]);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
    const int64_t t0 = c * 32;
    const int64_t r0 = t0 < A.row_threads ? div_kv(t0, KV) : 0;
    step3e_row<V, ADJ, false, false, true>(A, t0 + lane, &stage[w][s], r0);
    __syncwarp();
    s ^= 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Persistent slab form: block b owns the contiguous chunk range
// [b L, (b + 1) L) (L = ceil(chunks / blocks)) and its warps walk it in order,
// w, w + 8, w + 16, ...  Rows then advance slowly through the block's SM, so
// the source rows one grid line away (+-(n_x + 1) in a lexicographic node
// order) are fetched from L2 once and reused from L1 by the rows that follow,
// instead of once per 32-row group.  Thread 0 bulk-prefetches into L2 the rows
// of the block's chunks A.pf_rows block-iterations ahead.
template <int V, bool ADJ, bool W>
__global__ void __launch_bounds__(256, V == 8 ? 4 : 5) step3e_slab_kernel(const Step3Args<float> A,
                                                                          int64_t n_chunks) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int KV = A.K / V;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t L = (n_chunks + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * L, c1 = min(c0 + L, n_chunks);
  for (int64_t cb = c0; cb < c1; cb += wpb) {
    if (A.pf_rows > 0 && threadIdx.x == 0) {
      const int64_t t0 = (cb + A.pf_rows * wpb) * 32;
      const int64_t t1 = min(min(t0 + 32 * (int64_t)wpb, c1 * 32), A.row_threads);
      if (t0 < t1) prefetch_ahead<true>(A, div_kv(t0, KV), div_kv(t1 - 1, KV) + 1);
    }
    const int64_t c = cb + (threadIdx.x >> 5);
    if (c < c1) step3e_row<V, ADJ, W>(A, c * 32 + lane);
  }
}

// the same with at least MINB resident 256-thread blocks per SM asked of the
// compiler: more warps, hence more loads in flight, at the cost of registers
template <int V, bool ADJ, int MINB>
__global__ void __launch_bounds__(256, MINB) step3e_occ_kernel(const Step3Args<float> A) {
  step3e_body<V, ADJ>(A);
}

// the same with 1024-thread blocks: with rows in Z-order a block is a compact
// brick of the mesh whose neighbour rows stay in its SM's L1
template <int V, bool ADJ>
__global__ void __launch_bounds__(1024) step3e_big_kernel(const Step3Args<float> A) {
  step3e_body<V, ADJ>(A);
}

// Wait for the given phase parity of an mbarrier, bounded by `cycles`.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Persistent, double-buffered tile-staged kernel: each block walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; while it computes one tile from one
// shared-memory buffer, the bulk copies of its next tile fill the other, so
// the copy latency hides behind compute instead of serialising with it.
template <bool ADJ>
__global__ void __launch_bounds__(512) step3p_kernel(const Step3Args<float> A, const TileArgs Tl, int slots_cap) {
  constexpr int V = 8, P = 4;
  extern __shared__ __align__(128) unsigned char ptile_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(ptile_smem);
  float* bufs[2] = {reinterpret_cast<float*>(ptile_smem + 128),
                    reinterpret_cast<float*>(ptile_smem + 128) + (size_t)slots_cap * A.K};
  const uint32_t bar_s[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
  const int KV = A.K / V;
  const size_t row_bytes = (size_t)A.K * 4;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s[1]) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile, int b) {  // by warp 0
    const int q0 = Tl.range_ptr[tile], q1 = Tl.range_ptr[tile + 1];
    if (threadIdx.x == 0) {
      const uint32_t bytes = (uint32_t)((size_t)Tl.tile_slots[tile] * row_bytes);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s[b]), "r"(bytes) : "memory");
    }
    __syncwarp();
    for (int q = q0 + (int)threadIdx.x; q < q1; q += 32) {
      const float* src = A.x + (int64_t)Tl.range_src[q] * A.K;
      const uint32_t dst = smem_u32(bufs[b] + (size_t)Tl.range_slot[q] * A.K);
      const uint32_t n = (uint32_t)((size_t)Tl.range_cnt[q] * row_bytes);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
          "l"(src), "r"(n), "r"(bar_s[b])
          : "memory");
    }
  };
  const int lr = threadIdx.x / KV;
  const int kv = threadIdx.x - lr * KV;
  const uint32_t Ku = (uint32_t)A.K;
  int tile = blockIdx.x;
  if (tile < Tl.n_tiles && threadIdx.x < 32) issue(tile, 0);
  for (int it = 0; tile < Tl.n_tiles; ++it, tile += gridDim.x) {
    const int b = it & 1;
    const int next = tile + gridDim.x;
    if (next < Tl.n_tiles && threadIdx.x < 32) issue(next, b ^ 1);
    const bool ok = mbar_wait_parity(bar_s[b], (uint32_t)((it >> 1) & 1), Tl.wait_cycles);
    if (__syncthreads_or(!ok)) {
      // a copy did not complete in time: report, let in-flight copies land, stop
      if (threadIdx.x == 0) atomicExch(Tl.status, (int)PAT_ETIMEOUT);
      mbar_wait_parity(bar_s[b], (uint32_t)((it >> 1) & 1), kDrainWait);
      if (next < Tl.n_tiles) mbar_wait_parity(bar_s[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1), kDrainWait);
      return;
    }
    const int64_t r0 = (int64_t)tile * kTileRows;
    if (r0 + lr < A.N) {
      const int64_t row = Tl.order[r0 + lr];
      const int64_t off = row * A.K + (int64_t)kv * V;
      const int e0 = A.ptr[row], e1 = A.ptr[row + 1];
      const int ni = ADJ ? (int)A.ninj[row] : 0;
      const int eA = e1 - ni;
      const int eB = eA - (int)A.nb[row];
      Pack<float, V> xpi;
      if (A.prev_mode == 0) xpi = ld<float, V>(A.xp + off);
      u64 acc[P], accl[P];
#pragma unroll
      for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
      const float* sk = bufs[b] + kv * V;
#pragma unroll 4
      for (int e = e0; e < eA; ++e) {
        const float2 c = A.hl[e];
        const float* sp = sk + (size_t)Tl.slot[e] * A.K;
        const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sp);
        const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sp + 4);
        const u64 ch = dup2(c.x), cl = dup2(c.y);
        acc[0] = ffma2(ch, v0.x, acc[0]);
        accl[0] = ffma2(cl, v0.x, accl[0]);
        acc[1] = ffma2(ch, v0.y, acc[1]);
        accl[1] = ffma2(cl, v0.y, accl[1]);
        acc[2] = ffma2(ch, v1.x, acc[2]);
        accl[2] = ffma2(cl, v1.x, accl[2]);
        acc[3] = ffma2(ch, v1.y, acc[3]);
        accl[3] = ffma2(cl, v1.y, accl[3]);
      }
      if (eB < eA && A.prev_mode != 2) {
        for (int e = eB; e < eA; ++e) {
          const float2 c = A.hl[e];
          u64 x[P];
          if (A.prev_mode == 0) {
            ld_pairs<P>(A.xp + (int64_t)kv * V + (size_t)(A.col[e] & kIdxMask) * Ku, x);
          } else {
            const float* sp = sk + (size_t)Tl.slot[e] * A.K;  // xp = x
            const ulonglong2 v0 = *reinterpret_cast<const ulonglong2*>(sp);
            const ulonglong2 v1 = *reinterpret_cast<const ulonglong2*>(sp + 4);
            x[0] = v0.x;
            x[1] = v0.y;
            x[2] = v1.x;
            x[3] = v1.y;
          }
          const u64 ch = dup2(-c.x), cl = dup2(-c.y);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            acc[p] = ffma2(ch, x[p], acc[p]);
            accl[p] = ffma2(cl, x[p], accl[p]);
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
      const Pack<float, V> xi = ld<float, V>(A.x + off);
      if (A.prev_mode != 0) {
#pragma unroll
        for (int q = 0; q < V; ++q) xpi.v[q] = (A.prev_mode == 1) ? xi.v[q] : 0.0f;
      }
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
    __syncthreads();  // buffer b is refilled by the copies issued in iteration it + 1
  }
  // sensor observations of the input state
  if (!ADJ && A.y_out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)A.n_obs * KV;
         g += (int64_t)gridDim.x * blockDim.x)
      gather_obs<V>(A, g);
  }
}

// Fixed-width kernel for one sample (K = 1): one thread per row, the row's 8
// fixed slots (columns and coefficient pairs: six 16-byte loads) arrive in one
// round and its 8 neighbour values in the next, instead of the row-pointer ->
// column -> value chain of the CSR walk.
template <bool ADJ, int MINB = 1>  // MINB 6: at most 40 registers, 6 blocks of 256 per SM
__global__ void __launch_bounds__(256, MINB) step3e1_kernel(const Step3Args<float> A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.row_threads) {
    gather_obs<1>(A, t - A.row_threads);
    return;
  }
  const int64_t row = t;
  const uint32_t desc = A.ell_desc[row];
  const int n = (int)(desc & 255u), nb = (int)((desc >> 8) & 255u), ni = (int)((desc >> 16) & 255u);
  const int eA = n - ni;
  const uint4 c0 = *reinterpret_cast<const uint4*>(A.ell_col + row * 8);
  const uint4 c1 = *reinterpret_cast<const uint4*>(A.ell_col + row * 8 + 4);
  const float4 h01 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8);
  const float4 h23 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 2);
  const float4 h45 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 4);
  const float4 h67 = *reinterpret_cast<const float4*>(A.ell_hl + row * 8 + 6);
  const uint32_t cols[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  const float hs[8] = {h01.x, h01.z, h23.x, h23.z, h45.x, h45.z, h67.x, h67.z};
  const float ls[8] = {h01.y, h01.w, h23.y, h23.w, h45.y, h45.w, h67.y, h67.w};
  float acc = 0.0f, accl = 0.0f;
  if (A.x) {
    // padded slots: the row itself with zero coefficients
    float xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) xv[q] = A.x[cols[q]];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      acc = fmaf(hs[q], xv[q], acc);
      accl = fmaf(ls[q], xv[q], accl);
    }
    auto entry = [&](int e, uint32_t* col, float2* c) { ell_entry<1>(A, row, e, col, c); };
    tail1(8, eA, A.x, 1.0f, entry, acc, accl);
    if (nb > 0 && A.prev_mode != 2) tail1(eA - nb, eA, A.prev_mode == 0 ? A.xp : A.x, -1.0f, entry, acc, accl);
  }
  float src = 0.0f;
  if constexpr (ADJ)
    src = inj1(ni, A.ya, A.yb, [&](int e, uint32_t* col, float2* c) { inj_entry(A, row, e, eA, col, c); });
  const float xi = A.x ? A.x[row] : 0.0f;
  const float xpi = A.prev_mode == 0 ? A.xp[row] : (A.prev_mode == 1 ? xi : 0.0f);
  const float w = xi - xpi;
  A.xn[row] = xi + (w - (acc + accl) + A.inj_scale * src);
}

}  // namespace pat
