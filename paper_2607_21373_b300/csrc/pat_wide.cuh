// Sixteen-slot fixed-width rows: the three-level step (Section 3, eq.
// fully-discrete in the scaled three-level form) for meshes whose rows carry
// more than 8 stiffness / boundary entries.  A P1 tetrahedral mesh couples a
// node to every node it shares a tetrahedron with: 15 entries per interior row
// of the Kuhn cube's full graph (its diagonal edges assemble to exact zeros,
// which this layout keeps), about 15 on an unstructured mesh.  With 8 slots
// the remaining entries went through the overflow list one dependent load at
// a time; here the first 16 sit at fixed positions, so a row's columns and
// coefficient pairs arrive in one round of broadcast loads and its source rows
// in two to four rounds of independent gathers.
//
// Layout (per direction): 16 columns (uint32) and 16 (hi, lo) coefficient
// pairs (float2) per row, interleaved by quads of consecutive rows: the
// 16-byte chunk q (columns 4q..4q+3, or pairs 2q, 2q+1) of the quad's 4 rows
// lies in 64 contiguous bytes, so a warp holding 4 consecutive rows (K = 64:
// 8 lanes per row) fetches one chunk of all 4 with one 64-byte access instead
// of 4 scattered ones; the descriptor word of the 8-slot layout; an overflow
// CSR holding the stiffness / boundary entries beyond 16 followed by every
// sensor entry.  A slot past the row's count holds the row itself with a zero
// coefficient.
// Entries are visited in the row's CSR order, hi and lo products accumulated
// separately, so every variant gives the same bits as the 8-slot and CSR
// kernels.
#pragma once

#include "pat_tile.cuh"

namespace pat {

constexpr int kWide = 16;
constexpr int kMainSlots = 15;  // slots the 16-slot kernels' round loop gathers (the rest: the tail)

// Stiffness / boundary entry e (< the row's count eA) of a quad-interleaved 16-slot row.
__device__ __forceinline__ void wide_entry(const Step3Args<float>& A, int64_t row, int e, uint32_t* col,
                                           float2* c) {
  if (e < kWide) {
    *col = A.ell_col[slot_col_at<kWide, true>(row, e)];
    *c = A.ell_hl[slot_hl_at<kWide, true>(row, e)];
  } else {
    const int64_t o = A.ovf_ptr[row] + (e - kWide);
    *col = A.ovf_col[o];
    *c = A.ovf_hl[o];
  }
}

// Sensor entry j of a 16-slot row with eA stiffness / boundary entries.
__device__ __forceinline__ void wide_inj(const Step3Args<float>& A, int64_t row, int j, int eA, uint32_t* col,
                                         float2* c) {
  const int64_t o = A.ovf_ptr[row] + max(eA - kWide, 0) + j;
  *col = A.ovf_col[o];
  *c = A.ovf_hl[o];
}

// The sensor term of row `row` for 8 samples (two runs of 4 at base, base + hs):
// src = sum over the row's sensor entries e of c_e (ya + yb)[col_e], in entry
// order, ya then yb (either may be absent).  One routine for the term computed
// in the row and for the term prepared a launch ahead, so both give the same bits.
__device__ __forceinline__ void sensor_term(const Step3Args<float>& A, int64_t row, int ni, int eA,
                                            const float* ya, const float* yb, int64_t base, int64_t hs,
                                            float (&src)[8]) {
  constexpr int V = 8;
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  for (int e = 0; e < ni; ++e) {
    uint32_t col;
    float2 c;
    wide_inj(A, row, e, eA, &col, &c);
    const int64_t j = (int64_t)col;
    if (ya) {
      const Pack<float, V> y = ld_run_pack<V>(ya + j * A.K + base, hs);
#pragma unroll
      for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
    }
    if (yb) {
      const Pack<float, V> y = ld_run_pack<V>(yb + j * A.K + base, hs);
#pragma unroll
      for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
    }
  }
}

// Extra thread g of a transposed launch: the next launch's sensor term of
// sensor row g / (K/8), samples of thread g % (K/8), into A.inj_next at the
// row's first overflow entry.
__device__ __forceinline__ void sensor_prep(const Step3Args<float>& A, int64_t g) {
  constexpr int V = 8;
  const int KV = A.K / V;
  const int64_t slot = div_kv(g, KV);
  if (slot >= A.n_inj) return;
  const int kv = (int)(g - slot * KV);
  const int64_t row = A.inj_rows[slot];
  const uint32_t desc = A.ell_desc[row];
  const int n = (int)(desc & 255u), ni = (int)((desc >> 16) & 255u);
  const int64_t hs = A.K / 2, base = (int64_t)kv * 4;
  float src[V];
  sensor_term(A, row, ni, n - ni, A.ya_next, A.yb_next, base, hs, src);
  Pack<float, V> o;
#pragma unroll
  for (int q = 0; q < V; ++q) o.v[q] = src[q];
  st_run_pack<V>(A.inj_next + (int64_t)A.ovf_ptr[row] * A.K + base, hs, o);
}

// Thread t of the row threads: 8 samples of one row (two runs of 4, as in the
// 8-slot kernel), NB source rows gathered per round.  PB: each round's columns
// and coefficient pairs are loaded with it (fewer live registers); otherwise
// all 16 columns arrive up front and the coefficient pairs per round.
//
// OA: the row's own values of x_s and x_{s-1} (the last loads the update
// needs) are copied global -> shared memory while the gathers run, instead of
// costing one more round trip after them.  OA = 1: by cp.async, each thread
// its own 4 x 16 bytes (`own`: 4 float4 at a stride of `own_stride` float4).
// OA = 2: by two bulk copies per warp chunk (its rows of x_s and x_{s-1}, 1 KB
// each) that one lane issued before the call, completing on the warp's
// mbarrier `bar` in phase `phase`; `ob` points at this thread's first value in
// the chunk's x_s copy (x_{s-1} 256 floats further).  `staged` says whether
// the copies were issued (the warp's rows exist and x is not the zero state).
// A wait that runs past A.wait_cycles reports PAT_ETIMEOUT, lets the copies
// land (bounded again) and carries on with whatever arrived.
//
// WL (row-major slots, rounds of 4): the row's metadata in 256-bit loads — a
// round's four coefficient pairs in one, two rounds' columns in one — so the
// 4 rows of a warp fetch 32 bytes per row and line instead of 16 (half the L1
// wavefronts for the metadata).
template <bool ADJ, int NB, bool PB, int TB = 2, bool QUAD = true, int OA = 0, bool WL = false>
__device__ __forceinline__ void step3w_row(const Step3Args<float>& A, const int64_t t, float4* own = nullptr,
                                           int own_stride = 0, const float* ob = nullptr, uint32_t bar = 0,
                                           uint32_t phase = 0, bool staged = false) {
  constexpr int V = 8, P = 4;
  static_assert(NB == 4 || NB == 8, "rounds of 4 or 8 source rows");
  static_assert(!WL || (!QUAD && NB == 4 && PB), "256-bit metadata loads: row-major slots, rounds of 4 with their columns");
  const int KV = A.K / V;
  if (t >= A.row_threads) {
    if constexpr (ADJ) {
      if (A.inj_next) sensor_prep(A, t - A.row_threads);
    } else {
      gather_obs<V>(A, t - A.row_threads);
    }
    return;
  }
  const int64_t row = div_kv(t, KV);
  const int kv = (int)(t - row * KV);
  const int64_t hs = A.K / 2;
  const int64_t base = (int64_t)kv * 4;
  const int64_t off = row * A.K + base;
  if constexpr (OA == 1) {
    if (A.x) {
      cp_async16(own, A.x + off);
      cp_async16(own + own_stride, A.x + off + hs);
    }
    if (A.prev_mode == 0) {
      cp_async16_cg(own + 2 * own_stride, A.xp + off);
      cp_async16_cg(own + 3 * own_stride, A.xp + off + hs);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  if constexpr (OA == 3) {  // x_{s-1} only (own: 2 float4); x_s is read at the update, an L1 hit after
                            // the row's own diagonal gather
    if (A.prev_mode == 0) {
      cp_async16_cg(own, A.xp + off);
      cp_async16_cg(own + own_stride, A.xp + off + hs);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const uint32_t desc = A.ell_desc[row];
  const int n = (int)(desc & 255u), nb = (int)((desc >> 8) & 255u), ni = (int)((desc >> 16) & 255u);
  const int eA = n - ni;
  const uint32_t Ku = (uint32_t)A.K;
  // chunk q of this row: cp[CS q] (4 columns), hp[CS q] (2 coefficient pairs)
  constexpr int CS = QUAD ? 4 : 1;
  const uint4* cp = reinterpret_cast<const uint4*>(A.ell_col) + (QUAD ? (row >> 2) * 16 + (row & 3) : row * 4);
  const float4* hp = reinterpret_cast<const float4*>(A.ell_hl) + (QUAD ? (row >> 2) * 32 + (row & 3) : row * 8);
  u64 acc[P], accl[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
  if (A.x) {
    const float* xk = A.x + base;
    uint32_t cols[kWide];
    if constexpr (!PB) {
#pragma unroll
      for (int q = 0; q < kWide / 4; ++q) {
        const uint4 c = cp[CS * q];
        cols[4 * q] = c.x, cols[4 * q + 1] = c.y, cols[4 * q + 2] = c.z, cols[4 * q + 3] = c.w;
      }
    }
#pragma unroll
    for (int h = 0; h < kWide / NB; ++h) {
      if constexpr (WL) {
        if (h % 2 == 0) {  // columns of rounds h and h + 1
          uint32_t* cq = cols + 4 * h;
          asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
              : "=r"(cq[0]), "=r"(cq[1]), "=r"(cq[2]), "=r"(cq[3]), "=r"(cq[4]), "=r"(cq[5]), "=r"(cq[6]),
                "=r"(cq[7])
              : "l"(cp + h));
        }
      } else if constexpr (PB) {
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
          const uint4 c = cp[CS * (h * (NB / 4) + q)];
          cols[NB * h + 4 * q] = c.x, cols[NB * h + 4 * q + 1] = c.y;
          cols[NB * h + 4 * q + 2] = c.z, cols[NB * h + 4 * q + 3] = c.w;
        }
      }
      // slots past the row's count read the row itself with a zero coefficient:
      // no per-slot test, the gathers of a round issue back to back.  The last
      // slot (kMainSlots = 15: an interior row of a P1 mesh has about 15
      // entries, and the Kuhn cube's exactly 15) is left to the tail, which
      // reads it only for rows that use it.
      u64 x[NB][P];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (NB * h + q < kMainSlots) ld_runs<V>(xk + (size_t)cols[NB * h + q] * Ku, hs, x[q]);
      float2 cf[NB];
      if constexpr (WL) {
        float f[8];
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]), "=f"(f[7])
            : "l"(hp + 2 * h));
#pragma unroll
        for (int q = 0; q < NB; ++q) cf[q] = make_float2(f[2 * q], f[2 * q + 1]);
      } else {
#pragma unroll
        for (int q = 0; q < NB; q += 2) {
          const float4 hq = hp[CS * ((NB * h + q) / 2)];
          cf[q] = make_float2(hq.x, hq.y);
          cf[q + 1] = make_float2(hq.z, hq.w);
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (NB * h + q >= kMainSlots) continue;
        const u64 ch = dup2(cf[q].x), cl = dup2(cf[q].y);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          acc[p] = ffma2(ch, x[q][p], acc[p]);
          accl[p] = ffma2(cl, x[q][p], accl[p]);
        }
      }
    }
    // entries 15 and beyond (slot 15, then the overflow list), then the xp
    // parts of the boundary entries (boundary entries act on w_j = x_j - xp_j)
    const float* pk = A.prev_mode == 2 ? nullptr : (A.prev_mode == 0 ? A.xp : A.x) + base;
    fixed_row_tail<V, false, kWide, TB, QUAD, false, kMainSlots>(A, row, eA, nb, xk, pk, hs, Ku, acc, accl);
  }
  float src[V];
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  if constexpr (ADJ) {
    if (ni > 0) {
      if (A.inj_cur) {  // prepared by the previous launch: one contiguous read
        const Pack<float, V> y = ld_run_pack<V>(A.inj_cur + (int64_t)A.ovf_ptr[row] * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = y.v[q];
      } else {
        sensor_term(A, row, ni, eA, A.ya, A.yb, base, hs, src);
      }
    }
  }
  Pack<float, V> xi, xpi, xo;
  if constexpr (OA == 1 || OA == 3) asm volatile("cp.async.wait_group 0;" ::: "memory");
  if constexpr (OA == 2) {
    if (staged && !mbar_wait_parity(bar, phase, A.wait_cycles)) {
      atomicExch(A.status, (int)PAT_ETIMEOUT);
      mbar_wait_parity(bar, phase, kDrainWait);
    }
  }
  auto unpack4 = [](float4 a, float4 b, Pack<float, V>& o) {
    o.v[0] = a.x, o.v[1] = a.y, o.v[2] = a.z, o.v[3] = a.w;
    o.v[4] = b.x, o.v[5] = b.y, o.v[6] = b.z, o.v[7] = b.w;
  };
  if (A.x) {
    if (OA == 2 && staged)
      unpack4(*reinterpret_cast<const float4*>(ob), *reinterpret_cast<const float4*>(ob + hs), xi);
    else if constexpr (OA == 1)
      unpack4(own[0], own[own_stride], xi);
    else
      xi = ld_run_pack<V>(A.x + off, hs);
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) xi.v[q] = 0.0f;
  }
  if (A.prev_mode == 0) {
    if (OA == 2 && staged)
      unpack4(*reinterpret_cast<const float4*>(ob + 256), *reinterpret_cast<const float4*>(ob + 256 + hs), xpi);
    else if constexpr (OA == 1)
      unpack4(own[2 * own_stride], own[3 * own_stride], xpi);
    else if constexpr (OA == 3)
      unpack4(own[0], own[own_stride], xpi);
    else
      xpi = ld_run_pack<V>(A.xp + off, hs);
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
  st_run_pack<V>(A.xn + off, hs, xo);
}

// Persistent grid-stride form (as the 8-slot persistent kernel): a resident
// wave of blocks whose warps walk 32-thread chunks with the grid's stride,
// launched as a programmatic dependent of the previous step.
// PFM: before a warp works on a chunk it asks L1 to prefetch the row metadata
// (descriptor, columns, coefficient pairs; row-major slots) of its next chunk,
// so that chunk starts with L1 hits instead of a round trip to L2.  With the
// quad-interleaved slots (K = 64: a chunk is one quad) it instead prefetches
// the current quad's four 128-byte lines of coefficient pairs: each round of
// 4 sources reads a new line of them, which would otherwise cost every round
// its own L2 round trip.
//
// OA = 2 (K / 8 divides 32, so a 32-thread chunk covers whole rows: 32 / (K/8)
// rows, 1 KB of each state array): each warp owns a 2 KB shared-memory copy of its
// chunk's x_s and x_{s-1} rows and an mbarrier; lane 0 issues the chunk's two
// bulk copies once every lane is done with the previous chunk's copy.
//
// DYN: chunks are handed out by an atomic counter instead of the grid stride:
// a warp that is done takes the next chunk in row order, so warps whose
// chunks hold slow rows (boundary rows with long tails, sensor rows) no longer
// set the end of the step.  Lane 0 asks for the following chunk when it
// starts one, so the counter's round trip hides behind the chunk's work.
template <bool ADJ, int NB, bool PB, int BS, int MINB, int TB = 2, bool QUAD = true, int OA = 0,
          bool PFM = false, bool DYN = false, bool WL = false>
__global__ void __launch_bounds__(BS, MINB) step3w_persist_kernel(const Step3Args<float> A, int64_t n_chunks) {
  // per-thread slots of the own-row copies, slot q of thread i at [q][i]
  // (consecutive threads contiguous: conflict-free 16-byte accesses)
  __shared__ float4 own_buf[OA == 1 ? 4 * BS : OA == 3 ? 2 * BS : 1];
  __shared__ __align__(128) float own_rows[OA == 2 ? (BS / 32) * 512 : 1];
  __shared__ __align__(8) uint64_t own_bar[OA == 2 ? BS / 32 : 1];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint32_t bar = 0, phase = 0;
  float* ow = own_rows + (OA == 2 ? warp * 512 : 0);
  if constexpr (OA == 2) {
    bar = smem_u32(&own_bar[warp]);
    if (lane == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int wpb = BS >> 5;
  const int64_t S = (int64_t)gridDim.x * wpb;
  const int KV = A.K / 8;
  unsigned int c_next = 0;
  if constexpr (DYN) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.dyn_next = 0u;  // the next launch starts from chunk 0
    if (lane == 0) c_next = atomicAdd(A.dyn_ctr, 1u);
    c_next = __shfl_sync(0xffffffffu, c_next, 0);
  }
  for (int64_t c = DYN ? (int64_t)c_next : (int64_t)blockIdx.x * wpb + warp; c < n_chunks;) {
    if constexpr (DYN) {
      if (lane == 0) c_next = atomicAdd(A.dyn_ctr, 1u);  // used at the end of this chunk
    }
    bool staged = false;
    const float* ob = nullptr;
    if constexpr (OA == 2) {
      const int64_t t0 = c * 32;
      const int64_t row0 = t0 / KV;
      const int64_t nr = (A.x && t0 < A.row_threads) ? min((int64_t)(32 / KV), A.N - row0) : 0;
      staged = nr > 0;
      if (staged) {
        __syncwarp();  // every lane is done with the previous chunk's copy
        if (lane == 0) {
          const uint32_t bytes = (uint32_t)(nr * A.K * 4);
          const uint32_t total = A.prev_mode == 0 ? 2 * bytes : bytes;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total) : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(ow)),
              "l"(A.x + row0 * A.K), "r"(bytes), "r"(bar)
              : "memory");
          if (A.prev_mode == 0)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(ow + 256)),
                "l"(A.xp + row0 * A.K), "r"(bytes), "r"(bar)
                : "memory");
        }
        const int64_t t = t0 + lane;
        const int64_t row = t / KV;
        ob = ow + (row - row0) * A.K + (t - row * KV) * 4;
      }
    }
    if constexpr (PFM && QUAD) {
      const int64_t t0 = c * 32;
      if (lane < 4 && t0 < A.row_threads && KV == 8)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(A.ell_hl + (t0 / 32) * 64 + lane * 16));
    }
    if constexpr (PFM && !QUAD) {
      const int64_t tn = (c + S) * 32 + lane;
      if (tn < A.row_threads) {
        const int64_t rn = div_kv(tn, KV);
        const int kv = (int)(tn - rn * KV);
        // lanes 0, 1, 2 of a row: columns (64 B), coefficient pairs (128 B), descriptor
        const void* p = kv == 0 ? (const void*)(A.ell_col + rn * kWide)
                        : kv == 1 ? (const void*)(A.ell_hl + rn * kWide)
                                  : (const void*)(A.ell_desc + rn);
        if (kv < 3) asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
      }
    }
    step3w_row<ADJ, NB, PB, TB, QUAD, OA, WL>(A, c * 32 + lane, own_buf + ((OA == 1 || OA == 3) ? threadIdx.x : 0),
                                              BS, ob, bar, phase, staged);
    if (staged) phase ^= 1u;
    if constexpr (DYN)
      c = (int64_t)__shfl_sync(0xffffffffu, c_next, 0);
    else
      c += S;
  }
}

// Row pairs: each of the K / 8 threads of a pair (K = 64: 8 threads, four
// pairs per warp) holds 8 samples of both rows 2p and 2p+1.  Every source row of the pair's union (the
// two rows' stiffness entries merged by column, then their boundary entries)
// is gathered once and multiplied into both rows' accumulators, with a zero
// coefficient where a row has no such entry: consecutive rows of a lattice or a
// bandwidth-reduced mesh share most of their neighbours (22 sources for 30
// entries in the interior of the Kuhn cube's full graph), so the gathers per
// row drop by about a quarter.  Each row visits its entries in its CSR order
// (zero products interleaved), so the results equal the per-row kernels'.  The
// boundary entries' x_{s-1} corrections, the sensor entries and the update
// then run per row from the row-major 16-slot copy (ell_* arguments).
template <bool ADJ>
__device__ __forceinline__ void row_finish(const Step3Args<float>& A, int64_t row, int64_t hs, int64_t base,
                                           u64 (&acc)[4], u64 (&accl)[4]) {
  constexpr int V = 8, P = 4;
  const int64_t off = row * A.K + base;
  const uint32_t desc = A.ell_desc[row];
  const int n = (int)(desc & 255u), nb = (int)((desc >> 8) & 255u), ni = (int)((desc >> 16) & 255u);
  const int eA = n - ni;
  if (A.x) {
    const float* pk = A.prev_mode == 2 ? nullptr : (A.prev_mode == 0 ? A.xp : A.x) + base;
    fixed_row_tail<V, false, kWide, 1, false, true>(A, row, eA, nb, A.x + base, pk, hs, (uint32_t)A.K, acc, accl);
  }
  float src[V];
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  if constexpr (ADJ) {
    for (int e = 0; e < ni; ++e) {
      uint32_t col;
      float2 c;
      wide_inj(A, row, e, eA, &col, &c);
      const int64_t j = (int64_t)col;
      if (A.ya) {
        const Pack<float, V> y = ld_run_pack<V>(A.ya + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
      }
      if (A.yb) {
        const Pack<float, V> y = ld_run_pack<V>(A.yb + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(c.x, y.v[q], src[q]);
      }
    }
  }
  Pack<float, V> xi, xpi, xo;
  if (A.x) {
    xi = ld_run_pack<V>(A.x + off, hs);
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) xi.v[q] = 0.0f;
  }
  if (A.prev_mode == 0) {
    xpi = ld_run_pack<V>(A.xp + off, hs);
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
  st_run_pack<V>(A.xn + off, hs, xo);
}

template <bool ADJ>
__device__ __forceinline__ void step3u_pair(const Step3Args<float>& A, const int64_t t) {
  constexpr int V = 8, P = 4;
  const int KV = A.K / V;
  if (t >= A.row_threads) {  // A.row_threads counts pair threads here
    gather_obs<V>(A, t - A.row_threads);
    return;
  }
  const int64_t pr = div_kv(t, KV);
  const int kv = (int)(t - pr * KV);
  const int64_t ra = 2 * pr, rb = ra + 1;
  const int64_t hs = A.K / 2, base = (int64_t)kv * 4;
  u64 accA[P], acclA[P], accB[P], acclB[P];
#pragma unroll
  for (int p = 0; p < P; ++p) accA[p] = acclA[p] = accB[p] = acclB[p] = 0ull;
  if (A.x) {
    const float* xk = A.x + base;
    const uint32_t Ku = (uint32_t)A.K;
    const int used = A.pair_n[pr];
    const uint4* cp = reinterpret_cast<const uint4*>(A.pair_col + pr * kPairSlots);
    const float4* fp = A.pair_cf + pr * kPairSlots;
    for (int s0 = 0; s0 < used; s0 += 4) {
      const uint4 c = cp[s0 >> 2];
      const uint32_t cols[4] = {c.x, c.y, c.z, c.w};
      u64 x[4][P];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_runs<V>(xk + (size_t)cols[q] * Ku, hs, x[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 f = fp[s0 + q];
        const u64 ha = dup2(f.x), la = dup2(f.y), hb = dup2(f.z), lb = dup2(f.w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          accA[p] = ffma2(ha, x[q][p], accA[p]);
          acclA[p] = ffma2(la, x[q][p], acclA[p]);
          accB[p] = ffma2(hb, x[q][p], accB[p]);
          acclB[p] = ffma2(lb, x[q][p], acclB[p]);
        }
      }
    }
  }
  row_finish<ADJ>(A, ra, hs, base, accA, acclA);
  if (rb < A.N) row_finish<ADJ>(A, rb, hs, base, accB, acclB);
}

template <bool ADJ, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) step3u_persist_kernel(const Step3Args<float> A, int64_t n_chunks) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int wpb = BS >> 5;
  const int64_t S = (int64_t)gridDim.x * wpb;
  for (int64_t c = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < n_chunks; c += S)
    step3u_pair<ADJ>(A, c * 32 + lane);
}

// Row quads (K = 64: a warp's 32 threads are the 8 threads x 8 samples of each
// of the 4 rows 4q .. 4q+3).  Every entry of the quad's union is one source row
// that all four rows' threads gather together: the four 8-thread groups read
// the same addresses, so one warp access fetches the source row once for the
// whole quad, and consecutive rows of a lattice-like numbering share most of
// their neighbours (about 36 sources for the 60 entries of four interior rows
// of the Kuhn cube's full graph).  Each group multiplies with its own row's
// coefficient pair (zero where the row has no such entry), in its CSR order,
// so every row accumulates the per-row kernels' products in their order.
// One round: the 4 entries' columns in one broadcast load, their source rows
// gathered together, each group's coefficient pairs for the 4 entries in two
// 16-byte loads (the quad's 4 rows side by side: 64 contiguous bytes).
template <int V, int P>
__device__ __forceinline__ void quad_list(const Step3Args<float>& A, int32_t e, int n, const float* src, int g,
                                          int64_t hs, uint32_t Ku, u64 (&acc)[P], u64 (&accl)[P]) {
  for (int h = 0; h < n; h += 4, e += 4) {
    const uint4 c = *reinterpret_cast<const uint4*>(A.quad_col + e);
    const uint32_t cols[4] = {c.x, c.y, c.z, c.w};
    u64 x[4][P];
#pragma unroll
    for (int q = 0; q < 4; ++q) ld_runs<V>(src + (size_t)cols[q] * Ku, hs, x[q]);
    const float4 f01 = A.quad_cf[(e >> 1) * 4 + g], f23 = A.quad_cf[((e >> 1) + 1) * 4 + g];
    const float2 cf[4] = {make_float2(f01.x, f01.y), make_float2(f01.z, f01.w), make_float2(f23.x, f23.y),
                          make_float2(f23.z, f23.w)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u64 ch = dup2(cf[q].x), cl = dup2(cf[q].y);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        acc[p] = ffma2(ch, x[q][p], acc[p]);
        accl[p] = ffma2(cl, x[q][p], accl[p]);
      }
    }
  }
}

// Chunk c of the quad kernel: quad c's rows, or (past the quads) 32 sensor-gather
// threads.  OA: the rows' own x_s, x_{s-1} copied to shared memory by cp.async
// while the union is gathered (`own`: this thread's 4 float4 at a stride of
// `own_stride`).  The sensor entries (transposed step) and the update then run
// per row from the row-major 16-slot copy's descriptor and overflow lists.
template <bool ADJ, bool OA>
__device__ __forceinline__ void step3q_chunk(const Step3Args<float>& A, int64_t c, int lane, float4* own,
                                             int own_stride) {
  constexpr int V = 8, P = 4;
  const int64_t t = c * 32 + lane;
  const int64_t rows = A.row_threads >> 3;  // 0 on a launch that only observes
  const int64_t nq = (rows + 3) >> 2;
  if (c >= nq) {
    gather_obs<V>(A, t - A.row_threads);
    return;
  }
  const int g = lane >> 3, kv = lane & 7;
  const int64_t row = 4 * c + g;
  const bool is_row = row < rows;  // else a sensor-gather thread of the last chunk
  const int64_t hs = A.K / 2, base = (int64_t)kv * 4;
  const int64_t off = row * A.K + base;
  if constexpr (OA) {
    if (is_row) {
      if (A.x) {
        cp_async16(own, A.x + off);
        cp_async16(own + own_stride, A.x + off + hs);
      }
      if (A.prev_mode == 0) {
        cp_async16_cg(own + 2 * own_stride, A.xp + off);
        cp_async16_cg(own + 3 * own_stride, A.xp + off + hs);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  u64 acc[P], accl[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = accl[p] = 0ull;
  if (A.x) {
    const uint32_t Ku = (uint32_t)A.K;
    const int32_t e0 = A.quad_ptr[c];
    const uint32_t qn = A.quad_n[c];
    const int nx = (int)(qn & 0xffffu), np = (int)(qn >> 16);
    quad_list<V, P>(A, e0, nx, A.x + base, g, hs, Ku, acc, accl);
    if (A.prev_mode != 2 && np > 0)
      quad_list<V, P>(A, e0 + nx, np, (A.prev_mode == 0 ? A.xp : A.x) + base, g, hs, Ku, acc, accl);
  }
  if (!is_row) {
    if constexpr (OA) asm volatile("cp.async.wait_group 0;" ::: "memory");
    gather_obs<V>(A, t - A.row_threads);
    return;
  }
  float src[V];
#pragma unroll
  for (int q = 0; q < V; ++q) src[q] = 0.0f;
  if constexpr (ADJ) {
    const uint32_t desc = A.ell_desc[row];
    const int n = (int)(desc & 255u), ni = (int)((desc >> 16) & 255u);
    const int eA = n - ni;
    for (int e = 0; e < ni; ++e) {
      uint32_t col;
      float2 cf;
      wide_inj(A, row, e, eA, &col, &cf);
      const int64_t j = (int64_t)col;
      if (A.ya) {
        const Pack<float, V> y = ld_run_pack<V>(A.ya + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(cf.x, y.v[q], src[q]);
      }
      if (A.yb) {
        const Pack<float, V> y = ld_run_pack<V>(A.yb + j * A.K + base, hs);
#pragma unroll
        for (int q = 0; q < V; ++q) src[q] = fmaf(cf.x, y.v[q], src[q]);
      }
    }
  }
  auto unpack4 = [](float4 a, float4 b, Pack<float, V>& o) {
    o.v[0] = a.x, o.v[1] = a.y, o.v[2] = a.z, o.v[3] = a.w;
    o.v[4] = b.x, o.v[5] = b.y, o.v[6] = b.z, o.v[7] = b.w;
  };
  if constexpr (OA) asm volatile("cp.async.wait_group 0;" ::: "memory");
  Pack<float, V> xi, xpi, xo;
  if (A.x) {
    if constexpr (OA)
      unpack4(own[0], own[own_stride], xi);
    else
      xi = ld_run_pack<V>(A.x + off, hs);
  } else {
#pragma unroll
    for (int q = 0; q < V; ++q) xi.v[q] = 0.0f;
  }
  if (A.prev_mode == 0) {
    if constexpr (OA)
      unpack4(own[2 * own_stride], own[3 * own_stride], xpi);
    else
      xpi = ld_run_pack<V>(A.xp + off, hs);
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
  st_run_pack<V>(A.xn + off, hs, xo);
}

template <bool ADJ, bool OA>
__global__ void __launch_bounds__(256, 4) step3q_persist_kernel(const Step3Args<float> A, int64_t n_chunks) {
  __shared__ float4 own_buf[OA ? 4 * 256 : 1];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int64_t S = (int64_t)gridDim.x * 8;
  for (int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); c < n_chunks; c += S)
    step3q_chunk<ADJ, OA>(A, c, lane, own_buf + (OA ? threadIdx.x : 0), 256);
}

// Uneven batch: one persistent grid over the 32-thread chunks of several jobs
// (meshes with their own sizes, sensor sets, time-step counts and K).  Job g
// owns chunks block_off[g] <= c < block_off[g + 1] (each job's row threads and
// sensor-gather threads rounded up to whole chunks), so a warp never mixes
// jobs; a warp's chunks increase, so its job index only moves forward.  Every
// job's rows run the single-mesh fixed-width row code (16 slots with WIDE,
// else 8) on that job's arguments.
template <bool ADJ, bool WIDE>
__global__ void __launch_bounds__(256, 4) step3g_persist_kernel(const __grid_constant__ Step3Group<float> G,
                                                                 int64_t n_chunks) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int64_t S = (int64_t)gridDim.x * 8;
  int g = 0;
  for (int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); c < n_chunks; c += S) {
    while (g + 1 < G.n && c >= G.block_off[g + 1]) ++g;
    const int64_t t = (c - G.block_off[g]) * 32 + lane;
    if constexpr (WIDE)
      step3w_row<ADJ, 4, true>(G.a[g], t);  // quad-interleaved slots (faster than row-major on this mix of K)
    else
      step3e_row<8, ADJ>(G.a[g], t);
  }
}

// One sample (K = 1): one thread per row, 16 fixed slots.
template <bool ADJ, int MINB = 1>  // MINB 6: at most 40 registers, 6 blocks of 256 per SM
__global__ void __launch_bounds__(256, MINB) step3w1_kernel(const Step3Args<float> A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.row_threads) {
    gather_obs<1>(A, t - A.row_threads);
    return;
  }
  const int64_t row = t;
  const uint32_t desc = A.ell_desc[row];
  const int n = (int)(desc & 255u), nb = (int)((desc >> 8) & 255u), ni = (int)((desc >> 16) & 255u);
  const int eA = n - ni;
  const uint4* cp = reinterpret_cast<const uint4*>(A.ell_col) + (row >> 2) * 16 + (row & 3);
  const float4* hp = reinterpret_cast<const float4*>(A.ell_hl) + (row >> 2) * 32 + (row & 3);
  float acc = 0.0f, accl = 0.0f;
  if (A.x) {
    uint32_t cols[kWide];
#pragma unroll
    for (int q = 0; q < kWide / 4; ++q) {
      const uint4 c = cp[4 * q];
      cols[4 * q] = c.x, cols[4 * q + 1] = c.y, cols[4 * q + 2] = c.z, cols[4 * q + 3] = c.w;
    }
    float xv[kWide];
#pragma unroll
    for (int q = 0; q < kWide; ++q) xv[q] = q < eA ? A.x[cols[q]] : 0.0f;
#pragma unroll
    for (int q = 0; q < kWide; q += 2) {
      const float4 h = hp[4 * (q / 2)];
      acc = fmaf(h.x, xv[q], acc);
      accl = fmaf(h.y, xv[q], accl);
      acc = fmaf(h.z, xv[q + 1], acc);
      accl = fmaf(h.w, xv[q + 1], accl);
    }
    auto entry = [&](int e, uint32_t* col, float2* c) { wide_entry(A, row, e, col, c); };
    tail1(kWide, eA, A.x, 1.0f, entry, acc, accl);
    if (nb > 0 && A.prev_mode != 2) tail1(eA - nb, eA, A.prev_mode == 0 ? A.xp : A.x, -1.0f, entry, acc, accl);
  }
  float src = 0.0f;
  if constexpr (ADJ)
    src = inj1(ni, A.ya, A.yb, [&](int e, uint32_t* col, float2* c) { wide_inj(A, row, e, eA, col, c); });
  const float xi = A.x ? A.x[row] : 0.0f;
  const float xpi = A.prev_mode == 0 ? A.xp[row] : (A.prev_mode == 1 ? xi : 0.0f);
  const float w = xi - xpi;
  A.xn[row] = xi + (w - (acc + accl) + A.inj_scale * src);
}

}  // namespace pat
