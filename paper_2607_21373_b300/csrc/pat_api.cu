// C ABI of libpat (declarations and contracts in include/pat.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pat_internal.h"
#include "pat_solver.cuh"
#include "pat_tile.cuh"

using namespace pat;

void pat::drop_graphs_locked(const DeviceMesh& m) {
  for (auto& kv : m.graphs)
    if (kv.second) cudaGraphExecDestroy((cudaGraphExec_t)kv.second);
  m.graphs.clear();
  for (auto& kv : m.grad_graphs)
    if (kv.second) cudaGraphExecDestroy((cudaGraphExec_t)kv.second);
  m.grad_graphs.clear();
}

namespace {

template <typename T>
pat_status upload(const std::vector<T>& h, T** d) {
  *d = nullptr;
  if (h.empty()) return PAT_OK;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e != cudaSuccess) {
    set_error("pat_mesh_create: cudaMalloc of %zu bytes failed (%s)", h.size() * sizeof(T), cudaGetErrorString(e));
    *d = nullptr;
    return e == cudaErrorMemoryAllocation ? PAT_ENOMEM : PAT_ECUDA;
  }
  e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_check(e, "pat_mesh_create upload");
  return PAT_OK;
}

void free_device(DeviceMesh& m) {
  if (m.capture_stream) {
    cudaStreamDestroy((cudaStream_t)m.capture_stream);
    m.capture_stream = nullptr;
  }
  {
    std::lock_guard<std::mutex> lock(m.graph_mutex);
    drop_graphs_locked(m);
  }
  for (void* e : m.prof.events)
    if (e) cudaEventDestroy((cudaEvent_t)e);
  m.prof.events.clear();
  m.prof.used = 0;
  void** ps[] = {(void**)&m.fwd.ptr, (void**)&m.fwd.col, &m.fwd.hi, (void**)&m.fwd.lo,
                 (void**)&m.adj.ptr, (void**)&m.adj.col, &m.adj.hi, (void**)&m.adj.lo,
                 (void**)&m.adj3.ptr, (void**)&m.adj3.col, &m.adj3.hi, (void**)&m.adj3.lo,
                 (void**)&m.fwd.hl, (void**)&m.adj.hl, (void**)&m.adj3.hl,
                 (void**)&m.fwd.ell_col, (void**)&m.fwd.ell_hl, (void**)&m.fwd.ell_desc, (void**)&m.fwd.ovf_ptr,
                 (void**)&m.fwd.ovf_col, (void**)&m.fwd.ovf_hl, (void**)&m.adj3.ell_col, (void**)&m.adj3.ell_hl,
                 (void**)&m.adj3.ell_desc, (void**)&m.adj3.ovf_ptr, (void**)&m.adj3.ovf_col, (void**)&m.adj3.ovf_hl,
                 (void**)&m.fwd.w16_col, (void**)&m.fwd.w16_hl, (void**)&m.fwd.w16_ovf_ptr,
                 (void**)&m.fwd.w16_ovf_col, (void**)&m.fwd.w16_ovf_hl, (void**)&m.adj3.w16_col,
                 (void**)&m.adj3.w16_hl, (void**)&m.adj3.w16_ovf_ptr, (void**)&m.adj3.w16_ovf_col,
                 (void**)&m.adj3.w16_ovf_hl, (void**)&m.fwd.w16r_col, (void**)&m.fwd.w16r_hl,
                 (void**)&m.adj3.w16r_col, (void**)&m.adj3.w16r_hl, (void**)&m.fwd.pair_col,
                 (void**)&m.fwd.pair_cf, (void**)&m.fwd.pair_n, (void**)&m.adj3.pair_col, (void**)&m.adj3.pair_cf,
                 (void**)&m.adj3.pair_n, (void**)&m.fwd.quad_ptr, (void**)&m.fwd.quad_n, (void**)&m.fwd.quad_col,
                 (void**)&m.fwd.quad_cf, (void**)&m.adj3.quad_ptr, (void**)&m.adj3.quad_n, (void**)&m.adj3.quad_col,
                 (void**)&m.adj3.quad_cf,
                 &m.minv_hi, (void**)&m.minv_lo, (void**)&m.ml, (void**)&m.sqrt_ml, (void**)&m.det_node,
                 &m.det_w, (void**)&m.etets, &m.eK0, (void**)&m.row_nb, (void**)&m.row_ninj,
                 (void**)&m.tile_range_ptr, (void**)&m.tile_range_src, (void**)&m.tile_range_cnt,
                 (void**)&m.tile_range_slot, (void**)&m.tile_slots, (void**)&m.tile_slot_fwd,
                 (void**)&m.tile_slot_adj, (void**)&m.d_status, (void**)&m.row_order, (void**)&m.inj_rows};
  for (void** p : ps) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

// Tagged device CSR of one direction, values in double before rounding.
struct HostRows {
  std::vector<int32_t> ptr;
  std::vector<uint32_t> col;
  std::vector<double> val;
};

template <typename T>
pat_status upload_rows(const HostRows& r, bool split, DevCSR& d) {
  d.nnz = (int64_t)r.col.size();
  pat_status s = upload(r.ptr, &d.ptr);
  if (s) return s;
  s = upload(r.col, &d.col);
  if (s) return s;
  std::vector<T> hi(r.val.size());
  for (size_t e = 0; e < hi.size(); ++e) hi[e] = (T)r.val[e];
  T* dh = nullptr;
  s = upload(hi, &dh);
  d.hi = dh;
  if (s) return s;
  if (split) {
    std::vector<float> lo(r.val.size());
    for (size_t e = 0; e < lo.size(); ++e) lo[e] = (float)(r.val[e] - (double)hi[e]);
    s = upload(lo, &d.lo);
    if (s) return s;
    std::vector<float2> hl(r.val.size());
    for (size_t e = 0; e < hl.size(); ++e) hl[e] = make_float2((float)hi[e], lo[e]);
    s = upload(hl, &d.hl);
    if (s) return s;
  }
  return PAT_OK;
}

}  // namespace

namespace pat {

bool check_device(const pat_mesh* mesh, const char* fn) {
  if (mesh->d.host_only) {
    set_error("%s: the mesh was created with PAT_MESH_HOST_ONLY", fn);
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != mesh->d.device) {
    set_error("%s: current device %d is not the mesh's device %d", fn, dev, mesh->d.device);
    return false;
  }
  return true;
}

pat_status check_ws(const pat_mesh* mesh, int op, int K, const void* ws, size_t bytes, const char* fn) {
  size_t need = 0;
  pat_status s = pat_workspace_bytes(mesh, op, K, &need);
  if (s) return s;
  if (!ws || bytes < need) {
    set_error("%s: workspace of %zu bytes at %p is too small (need %zu)", fn, bytes, ws, need);
    return PAT_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("%s: workspace must be 256-byte aligned", fn);
    return PAT_EINVAL;
  }
  return PAT_OK;
}

bool bad_K(int32_t K, const char* fn) {
  if (K < 1 || K > 1024) {
    set_error("%s: K = %d must be in [1, 1024]", fn, K);
    return true;
  }
  return false;
}

}  // namespace pat

namespace {

// Tiles of kTileRows consecutive rows: the union of the source rows of their
// stiffness / boundary entries as contiguous ranges (gaps of up to 4 rows are
// bridged), each entry's slot in the tile's staged rows, and the largest tile.
pat_status build_tiles(DeviceMesh& m, const HostRows& F, const HostRows& A3, const std::vector<uint8_t>& ninj,
                       const std::vector<int32_t>& order, bool upload_tables) {
  constexpr int R = kTileRows;  // rows order[t*R .. t*R+R) form tile t (a compact Z-order brick)
  const int64_t N = m.N;
  const int32_t T = (int32_t)((N + R - 1) / R);
  std::vector<int32_t> rptr(1, 0), rsrc, rcnt, rslot, tslots(T);
  std::vector<uint16_t> sf(F.col.size(), 0), sa(A3.col.size(), 0);
  std::vector<int32_t> srcs;
  int32_t max_slots = 0;
  for (int32_t t = 0; t < T; ++t) {
    const int64_t a = (int64_t)t * R, b = std::min<int64_t>(N, a + R);
    srcs.clear();
    for (int64_t ii = a; ii < b; ++ii) {
      const int64_t i = order[ii];
      for (int32_t e = F.ptr[i]; e < F.ptr[i + 1]; ++e) srcs.push_back((int32_t)(F.col[e] & kIdxMask));
    }
    std::sort(srcs.begin(), srcs.end());
    srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
    // ranges with small gaps bridged; slot of every source row
    std::vector<std::pair<int32_t, int32_t>> ranges;  // (start, count)
    for (int32_t j : srcs) {
      if (!ranges.empty() && j - (ranges.back().first + ranges.back().second) <= 2)
        ranges.back().second = j - ranges.back().first + 1;
      else
        ranges.push_back({j, 1});
    }
    int32_t slot = 0;
    for (auto& rg : ranges) {
      rsrc.push_back(rg.first);
      rcnt.push_back(rg.second);
      rslot.push_back(slot);
      slot += rg.second;
    }
    if (slot > 65535) {
      set_error("pat_mesh_create: a tile reads %d distinct rows (more than 65535)", slot);
      return PAT_EUNSUPPORTED;
    }
    rptr.push_back((int32_t)rsrc.size());
    tslots[t] = slot;
    max_slots = std::max(max_slots, slot);
    auto slot_of = [&](int32_t j) {
      // the range holding j (ranges are sorted by start)
      int lo = rptr[t], hi = (int)rsrc.size() - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (rsrc[mid] <= j) lo = mid; else hi = mid - 1;
      }
      return (uint16_t)(rslot[lo] + (j - rsrc[lo]));
    };
    // every slot must map back to its entry's source row (checked here, on the host,
    // because the kernel trusts these tables for its shared-memory reads)
    auto src_of = [&](uint16_t sl) {
      int q = rptr[t];
      while (q + 1 < (int)rsrc.size() && rslot[q + 1] <= sl) ++q;
      return rsrc[q] + (sl - rslot[q]);
    };
    for (int64_t ii = a; ii < b; ++ii) {
      const int64_t i = order[ii];
      for (int32_t e = F.ptr[i]; e < F.ptr[i + 1]; ++e) {
        const int32_t j = (int32_t)(F.col[e] & kIdxMask);
        sf[e] = slot_of(j);
        if (sf[e] >= slot || src_of(sf[e]) != j) {
          set_error("pat_mesh_create: internal error building the shared-memory tiles (row %lld)", (long long)i);
          return PAT_EUNSUPPORTED;
        }
      }
      const int32_t eA = A3.ptr[i + 1] - ninj[i];
      for (int32_t e = A3.ptr[i]; e < eA; ++e) {
        const int32_t j = (int32_t)(A3.col[e] & kIdxMask);
        sa[e] = slot_of(j);
        if (sa[e] >= slot || src_of(sa[e]) != j) {
          set_error("pat_mesh_create: internal error building the shared-memory tiles (row %lld)", (long long)i);
          return PAT_EUNSUPPORTED;
        }
      }
    }
  }
  m.n_tiles = T;
  m.tile_max_slots = max_slots;
  m.info.tile_rows = R;
  m.info.tile_max_staged = max_slots;
  {
    double tot = 0.0;
    for (int32_t t = 0; t < T; ++t) tot += tslots[t];
    m.info.tile_mean_staged = T ? tot / T : 0.0;
  }
  if (!upload_tables) return PAT_OK;
  pat_status s = upload(rptr, &m.tile_range_ptr);
  if (!s) s = upload(rsrc, &m.tile_range_src);
  if (!s) s = upload(rcnt, &m.tile_range_cnt);
  if (!s) s = upload(rslot, &m.tile_range_slot);
  if (!s) s = upload(tslots, &m.tile_slots);
  if (!s) s = upload(sf, &m.tile_slot_fwd);
  if (!s) s = upload(sa, &m.tile_slot_adj);
  if (!s) {
    std::vector<int32_t> z(1, 0);
    s = upload(z, &m.d_status);
  }
  return s;
}

// Fixed-width copy of a three-level CSR for the ELL kernels (FP32 split only):
// W = 8 or 16 slots per row.  The descriptor word is written with the 8-slot
// copy and shared by both.  The 8-slot copy is row-major ([row][slot]); the
// 16-slot copy interleaves each quad of consecutive rows so that one 16-byte
// chunk of 4 columns (or of 2 coefficient pairs) of the quad's 4 rows is 64
// contiguous bytes: column e of row i at (i/4)*64 + (e/4)*16 + (i%4)*4 + e%4,
// pair e at (i/4)*64 + (e/2)*8 + (i%4)*2 + e%2 (rows padded to a multiple of 4).
static int64_t ell_col_index(int64_t i, int e, int W) {
  return W == 8 ? i * 8 + e : (i / 4) * 64 + (e / 4) * 16 + (i % 4) * 4 + e % 4;
}
static int64_t ell_hl_index(int64_t i, int e, int W) {
  return W == 8 ? i * 8 + e : (i / 4) * 64 + (e / 2) * 8 + (i % 4) * 2 + e % 2;
}

pat_status build_ell(const HostRows& R, const std::vector<uint8_t>& nb, const std::vector<uint8_t>& ninj,
                     DevCSR& d, int W) {
  const int64_t N = (int64_t)R.ptr.size() - 1;
  const int64_t Np = W == 8 ? N : (N + 3) / 4 * 4;
  std::vector<uint32_t> col(Np * W, 0u), desc(N);
  std::vector<float2> hl(Np * W, make_float2(0.0f, 0.0f));
  std::vector<int32_t> optr(N + 1, 0);
  std::vector<uint32_t> ocol;
  std::vector<float2> ohl;
  auto pair = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  for (int64_t i = 0; i < N; ++i) {
    const int32_t e0 = R.ptr[i], n = R.ptr[i + 1] - e0;
    if (n > 255) {
      set_error("pat_mesh_create: row %lld has %d entries (more than 255)", (long long)i, n);
      return PAT_EUNSUPPORTED;
    }
    desc[i] = (uint32_t)n | ((uint32_t)nb[i] << 8) | ((uint32_t)ninj[i] << 16);
    // slots 0..W-1: the first stiffness / boundary entries, padded with the row
    // itself and a zero coefficient; overflow: the remaining stiffness / boundary
    // entries, then every sensor (injection) entry.  The kernels then walk the
    // W slots without a per-entry test.
    const int nA = n - (int)ninj[i];
    for (int q = 0; q < W; ++q) {
      if (q < nA) {
        col[ell_col_index(i, q, W)] = R.col[e0 + q] & kIdxMask;
        hl[ell_hl_index(i, q, W)] = pair(R.val[e0 + q]);
      } else {
        col[ell_col_index(i, q, W)] = (uint32_t)i;  // padding reads the row itself with a zero coefficient
        hl[ell_hl_index(i, q, W)] = make_float2(0.0f, 0.0f);
      }
    }
    for (int q = std::min(nA, W); q < n; ++q) {
      ocol.push_back(R.col[e0 + q] & kIdxMask);
      ohl.push_back(pair(R.val[e0 + q]));
    }
    optr[i + 1] = (int32_t)ocol.size();
  }
  if (ocol.empty()) {  // keep valid (unused) device arrays
    ocol.push_back(0);
    ohl.push_back(make_float2(0.0f, 0.0f));
  }
  pat_status s = PAT_OK;
  if (W == 8) {
    s = upload(col, &d.ell_col);
    if (!s) s = upload(hl, &d.ell_hl);
    if (!s) s = upload(desc, &d.ell_desc);
    if (!s) s = upload(optr, &d.ovf_ptr);
    if (!s) s = upload(ocol, &d.ovf_col);
    if (!s) s = upload(ohl, &d.ovf_hl);
  } else {
    s = upload(col, &d.w16_col);
    if (!s) s = upload(hl, &d.w16_hl);
    // the row-major copy of the same slots (the quad layout's alternative)
    std::vector<uint32_t> colr(N * W);
    std::vector<float2> hlr(N * W);
    for (int64_t i = 0; i < N; ++i)
      for (int q = 0; q < W; ++q) {
        colr[i * W + q] = col[ell_col_index(i, q, W)];
        hlr[i * W + q] = hl[ell_hl_index(i, q, W)];
      }
    if (!s) s = upload(colr, &d.w16r_col);
    if (!s) s = upload(hlr, &d.w16r_hl);
    if (!s) s = upload(optr, &d.w16_ovf_ptr);
    d.w16_ovf_n = optr.back();
    if (!s) s = upload(ocol, &d.w16_ovf_col);
    if (!s) s = upload(ohl, &d.w16_ovf_hl);
  }
  return s;
}

// Row pairs of a three-level CSR (see DevCSR): per pair the merge of the two
// rows' stiffness entries by column, then of their boundary entries, with both
// rows' coefficient pairs per slot.  Returns PAT_OK without building anything
// when some pair needs more than kPairSlots slots (the pair kernel is then not
// offered for the mesh).
pat_status build_pairs(const HostRows& R, const std::vector<uint8_t>& nb, const std::vector<uint8_t>& ninj,
                       DevCSR& d) {
  const int64_t N = (int64_t)R.ptr.size() - 1, P = (N + 1) / 2, U = kPairSlots;
  std::vector<uint32_t> col(P * U);
  std::vector<float4> cf(P * U);
  std::vector<uint8_t> cnt(P);
  auto split = [](double v) {
    const float h = (float)v;
    return std::make_pair(h, (float)(v - (double)h));
  };
  struct Slot {
    uint32_t col;
    double a, b;
  };
  std::vector<Slot> part, all;
  for (int64_t p = 0; p < P; ++p) {
    const int64_t ra = 2 * p, rb = 2 * p + 1;
    auto range = [&](int64_t r, bool boundary, int32_t* lo, int32_t* hi) {
      if (r >= N) {
        *lo = *hi = 0;
        return;
      }
      const int32_t e0 = R.ptr[r], eA = R.ptr[r + 1] - (int32_t)ninj[r];
      *lo = boundary ? eA - (int32_t)nb[r] : e0;
      *hi = boundary ? eA : eA - (int32_t)nb[r];
    };
    all.clear();
    for (int boundary = 0; boundary < 2; ++boundary) {
      int32_t a0, a1, b0, b1;
      range(ra, boundary != 0, &a0, &a1);
      range(rb, boundary != 0, &b0, &b1);
      part.clear();
      while (a0 < a1 || b0 < b1) {
        const uint32_t ca = a0 < a1 ? (R.col[a0] & kIdxMask) : 0xffffffffu;
        const uint32_t cb = b0 < b1 ? (R.col[b0] & kIdxMask) : 0xffffffffu;
        Slot sl{std::min(ca, cb), 0.0, 0.0};
        if (ca <= cb) sl.a = R.val[a0++];
        if (cb <= ca) sl.b = R.val[b0++];
        part.push_back(sl);
      }
      all.insert(all.end(), part.begin(), part.end());
    }
    if ((int64_t)all.size() > U) return PAT_OK;  // does not fit: no pair copy
    const int64_t used = ((int64_t)all.size() + 3) / 4 * 4;
    cnt[p] = (uint8_t)used;
    for (int64_t q = 0; q < U; ++q) {
      if (q < (int64_t)all.size()) {
        const auto ha = split(all[q].a), hb = split(all[q].b);
        col[p * U + q] = all[q].col;
        cf[p * U + q] = make_float4(ha.first, ha.second, hb.first, hb.second);
      } else {
        col[p * U + q] = (uint32_t)ra;  // padding reads row 2p with zero coefficients
        cf[p * U + q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
  }
  pat_status s = upload(col, &d.pair_col);
  if (!s) s = upload(cf, &d.pair_cf);
  if (!s) s = upload(cnt, &d.pair_n);
  return s;
}

// Row quads of a three-level CSR (see DevCSR): per quad of rows the merge of
// the four rows' stiffness entries by column, then of their boundary entries
// (both acting on x_s), then the boundary entries again with negated
// coefficients (acting on x_{s-1}).  A merge takes the smallest column among
// the rows' next entries and consumes that column from every row whose next
// entry it is, so each row meets its own entries in its CSR order and the
// products it accumulates are the per-row kernels' (zero products between).
pat_status build_quads(const HostRows& R, const std::vector<uint8_t>& nb, const std::vector<uint8_t>& ninj,
                       DevCSR& d) {
  const int64_t N = (int64_t)R.ptr.size() - 1, Q = (N + 3) / 4;
  std::vector<int32_t> qptr(Q + 1, 0);
  std::vector<uint32_t> qn(Q), qcol;
  std::vector<float4> qcf;
  auto split = [](double v) {
    const float h = (float)v;
    return std::make_pair(h, (float)(v - (double)h));
  };
  struct Entry {
    uint32_t col;
    double c[4];
  };
  std::vector<Entry> list;
  auto merge = [&](int64_t q, int part, double sign) {
    int32_t lo[4], hi[4];
    for (int g = 0; g < 4; ++g) {
      const int64_t r = 4 * q + g;
      if (r >= N) {
        lo[g] = hi[g] = 0;
        continue;
      }
      const int32_t e0 = R.ptr[r], eA = R.ptr[r + 1] - (int32_t)ninj[r], eB = eA - (int32_t)nb[r];
      lo[g] = part == 0 ? e0 : eB;
      hi[g] = part == 0 ? eB : eA;
    }
    for (;;) {
      uint32_t cmin = 0xffffffffu;
      for (int g = 0; g < 4; ++g)
        if (lo[g] < hi[g]) cmin = std::min(cmin, R.col[lo[g]] & kIdxMask);
      if (cmin == 0xffffffffu) break;
      Entry en{cmin, {0.0, 0.0, 0.0, 0.0}};
      for (int g = 0; g < 4; ++g)
        if (lo[g] < hi[g] && (R.col[lo[g]] & kIdxMask) == cmin) en.c[g] = sign * R.val[lo[g]++];
      list.push_back(en);
    }
  };
  auto flush = [&](int64_t q, size_t from) {  // pad the list from `from` to a multiple of 4 and append it
    while ((list.size() - from) % 4) list.push_back(Entry{(uint32_t)(4 * q), {0.0, 0.0, 0.0, 0.0}});
    const size_t n = list.size() - from;
    for (size_t e = from; e < list.size(); e += 2) {
      for (int g = 0; g < 4; ++g) {
        const auto a = split(list[e].c[g]), b = split(list[e + 1].c[g]);
        qcf.push_back(make_float4(a.first, a.second, b.first, b.second));
      }
      qcol.push_back(list[e].col);
      qcol.push_back(list[e + 1].col);
    }
    return n;
  };
  for (int64_t q = 0; q < Q; ++q) {
    list.clear();
    merge(q, 0, 1.0);
    merge(q, 1, 1.0);
    const size_t nx = flush(q, 0);
    const size_t from = list.size();
    merge(q, 1, -1.0);
    const size_t np = flush(q, from);
    if (nx > 0xffff || np > 0xffff) {
      set_error("pat_mesh_create: a row quad has more than 65535 entries");
      return PAT_EUNSUPPORTED;
    }
    qn[q] = (uint32_t)nx | ((uint32_t)np << 16);
    qptr[q + 1] = (int32_t)qcol.size();
  }
  if (qcol.empty()) {
    qcol.push_back(0);
    for (int g = 0; g < 4; ++g) qcf.push_back(make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  }
  pat_status s = upload(qptr, &d.quad_ptr);
  if (!s) s = upload(qn, &d.quad_n);
  if (!s) s = upload(qcol, &d.quad_col);
  if (!s) s = upload(qcf, &d.quad_cf);
  return s;
}

// Most stiffness / boundary entries of any row of a three-level CSR.
static int widest_row(const HostRows& R, const std::vector<uint8_t>& ninj) {
  int w = 0;
  for (size_t i = 0; i + 1 < R.ptr.size(); ++i) w = std::max(w, R.ptr[i + 1] - R.ptr[i] - (int)ninj[i]);
  return w;
}

// Device copies of the operators from the host assembly (also used after
// pat_mesh_set_c2, since exact-zero pruning can change the sparsity).
pat_status build_device(pat_mesh* mesh, uint32_t flags) {
  DeviceMesh& m = mesh->d;
  HostMesh& h = m.host;
  const int32_t n_obs = h.n_obs, n_steps = h.n_steps;
  const double dt = h.dt;
  const pat_prec prec = m.prec;
  pat_status s = PAT_OK;
  m.N = h.N;
  m.E = h.E;
  m.n_obs = n_obs;
  m.n_steps = n_steps;
  m.dt = dt;
  m.split = (prec == PAT_F32) && !(flags & PAT_MESH_SINGLE_COEF);
  const bool keep_zeros = (flags & PAT_MESH_KEEP_ZEROS) != 0;
  const int64_t N = h.N;
  m.host_only = (flags & PAT_MESH_HOST_ONLY) != 0;
  m.device = -1;
  if (!m.host_only) cudaGetDevice(&m.device);

  // sensor lists per node (for the adjoint's injection entries)
  std::vector<std::vector<std::pair<int32_t, double>>> inj(N);
  for (int32_t d = 0; d < n_obs; ++d)
    for (int a = 0; a < kDetPts; ++a)
      if (h.det_w[kDetPts * d + a] != 0.0) inj[h.det_node[kDetPts * d + a]].push_back({d, h.det_w[kDetPts * d + a]});

  m.three_level = !(flags & PAT_MESH_TWO_LEVEL);
  HostRows F, A, A3;
  std::vector<uint8_t> row_nb(N, 0), row_ninj(N, 0);
  F.ptr.assign(N + 1, 0);
  A.ptr.assign(N + 1, 0);
  A3.ptr.assign(N + 1, 0);
  int64_t nnz_k = 0;
  for (int64_t i = 0; i < N; ++i) {
    const double mi = h.ml[i];
    for (int64_t e = h.k_ptr[i]; e < h.k_ptr[i + 1]; ++e) {
      const double kv = h.k_val[e];
      if (kv == 0.0 && !keep_zeros) continue;  // an exact zero adds exactly nothing
      F.col.push_back((uint32_t)h.k_col[e]);
      F.val.push_back(dt * dt * kv / mi);
      A.col.push_back((uint32_t)h.k_col[e]);
      A.val.push_back(dt * dt * kv);
      ++nnz_k;
    }
    if (h.b_ptr[i + 1] - h.b_ptr[i] > 255 || inj[i].size() > 255) {
      set_error("pat_mesh_create: node %lld has more than 255 boundary or sensor entries", (long long)i);
      return PAT_EUNSUPPORTED;
    }
    row_nb[i] = (uint8_t)(h.b_ptr[i + 1] - h.b_ptr[i]);
    row_ninj[i] = (uint8_t)inj[i].size();
    for (int64_t e = h.b_ptr[i]; e < h.b_ptr[i + 1]; ++e) {
      F.col.push_back((uint32_t)h.b_col[e] | kTagB);
      F.val.push_back(dt * h.b_val[e] / mi);
      A.col.push_back((uint32_t)h.b_col[e] | kTagB);
      A.val.push_back(dt * h.b_val[e] / mi);
    }
    // three-level transposed rows: the forward row plus w_d / (2 M_i) per sensor at node i
    A3.col.insert(A3.col.end(), F.col.begin() + F.ptr[i], F.col.end());
    A3.val.insert(A3.val.end(), F.val.begin() + F.ptr[i], F.val.end());
    for (const auto& pr : inj[i]) {
      const double wr = prec == PAT_F32 ? (double)(float)pr.second : pr.second;
      A3.col.push_back((uint32_t)pr.first | kTagInj);
      A3.val.push_back(0.5 * wr / mi);
    }
    A3.ptr[i + 1] = (int32_t)A3.col.size();
    for (const auto& pr : inj[i]) {
      A.col.push_back((uint32_t)pr.first | kTagInj);
      // the same rounded weight as the forward gather, so Pi^T is Pi's exact transpose
      A.val.push_back(prec == PAT_F32 ? (double)(float)pr.second : pr.second);
    }
    if (F.col.size() > 0x7fffffffu || A.col.size() > 0x7fffffffu) {
      set_error("pat_mesh_create: operator too large for 32-bit row offsets");
      return PAT_EINVAL;
    }
    F.ptr[i + 1] = (int32_t)F.col.size();
    A.ptr[i + 1] = (int32_t)A.col.size();
  }
  // injection values are already rounded to the state precision, so their low part is 0
  std::vector<double> ml(h.ml), sqml(N), minv(N);
  for (int64_t i = 0; i < N; ++i) {
    sqml[i] = std::sqrt(h.ml[i]);
    minv[i] = 1.0 / h.ml[i];
  }
  std::vector<int32_t> det_node(h.det_node);
  m.fwd_ptr_h = F.ptr;
  m.adj3_ptr_h = A3.ptr;
  {
    std::lock_guard<std::mutex> lock(m.stage_mutex);
    m.stage_span.clear();
  }
  if (m.host_only) {
    m.fwd.nnz = (int64_t)F.col.size();
    m.adj.nnz = (int64_t)A.col.size();
    m.adj3.nnz = (int64_t)A3.col.size();
  } else if (prec == PAT_F64) {
    s = upload_rows<double>(F, false, m.fwd);
    if (!s) s = upload_rows<double>(A, false, m.adj);
    if (!s) s = upload_rows<double>(A3, false, m.adj3);
    double* p = nullptr;
    if (!s) s = upload(minv, &p);
    m.minv_hi = p;
    double* w = nullptr;
    if (!s) s = upload(h.det_w, &w);
    m.det_w = w;
  } else {
    s = upload_rows<float>(F, m.split, m.fwd);
    if (!s) s = upload_rows<float>(A, m.split, m.adj);
    if (!s) s = upload_rows<float>(A3, m.split, m.adj3);
    std::vector<float> mh(N), mlo(N), dw(h.det_w.size());
    for (int64_t i = 0; i < N; ++i) {
      mh[i] = (float)minv[i];
      mlo[i] = (float)(minv[i] - (double)mh[i]);
    }
    for (size_t e = 0; e < dw.size(); ++e) dw[e] = (float)h.det_w[e];
    float* p = nullptr;
    if (!s) s = upload(mh, &p);
    m.minv_hi = p;
    if (!s && m.split) s = upload(mlo, &m.minv_lo);
    float* w = nullptr;
    if (!s) s = upload(dw, &w);
    m.det_w = w;
  }
  if (!s && !m.host_only) s = upload(ml, &m.ml);
  if (!s && !m.host_only) s = upload(sqml, &m.sqrt_ml);
  if (!s && !m.host_only) s = upload(det_node, &m.det_node);
  std::vector<int32_t> order(N);
  {
    // Z-order (Morton) of the node coordinates quantised to 2^10 cells per axis
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], h.xyz[3 * i + c]);
        hi[c] = std::max(hi[c], h.xyz[3 * i + c]);
      }
    auto spread = [](uint64_t v) {  // insert two zero bits between the 10 bits of v
      uint64_t r = 0;
      for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1ull) << (3 * b);
      return r;
    };
    std::vector<std::pair<uint64_t, int32_t>> key(N);
    for (int64_t i = 0; i < N; ++i) {
      uint64_t q[3];
      for (int c = 0; c < 3; ++c) {
        const double u = hi[c] > lo[c] ? (h.xyz[3 * i + c] - lo[c]) / (hi[c] - lo[c]) : 0.0;
        q[c] = (uint64_t)std::min(1023.0, std::floor(u * 1024.0));
      }
      key[i] = {(spread(q[0]) << 2) | (spread(q[1]) << 1) | spread(q[2]), (int32_t)i};
    }
    std::sort(key.begin(), key.end());
    for (int64_t i = 0; i < N; ++i) order[i] = key[i].second;
  }
  if (!s && !m.host_only) s = upload(order, &m.row_order);
  if (!s) s = build_tiles(m, F, A3, row_ninj, order, !m.host_only);
  if (!s && !m.host_only && prec == PAT_F32 && m.split) {
    std::vector<uint8_t> no_inj(N, 0);
    s = build_ell(F, row_nb, no_inj, m.fwd, 8);
    if (!s) s = build_ell(A3, row_nb, row_ninj, m.adj3, 8);
    // 16-slot copies where some row spills out of 8 slots (the full P1 graph)
    if (!s && widest_row(F, no_inj) > 8) s = build_ell(F, row_nb, no_inj, m.fwd, kEllWide);
    if (!s && widest_row(A3, row_ninj) > 8) s = build_ell(A3, row_nb, row_ninj, m.adj3, kEllWide);
    // row pairs for the pair kernel (which finishes boundary rows from the 16-slot copy)
    if (!s && m.fwd.w16_col) s = build_pairs(F, row_nb, no_inj, m.fwd);
    if (!s && m.adj3.w16_col) s = build_pairs(A3, row_nb, row_ninj, m.adj3);
    // row quads for the quad-union kernel (which finishes rows from the 16-slot copy)
    if (!s && m.fwd.w16_col) s = build_quads(F, row_nb, no_inj, m.fwd);
    if (!s && m.adj3.w16_col) s = build_quads(A3, row_nb, row_ninj, m.adj3);
    // the status word of the kernels with bounded waits (16-slot rows with bulk-copied own rows)
    if (!s && m.fwd.w16_col && !m.d_status) {
      std::vector<int32_t> z(1, 0);
      s = upload(z, &m.d_status);
    }
  }
  if (!s && !m.host_only) {
    cudaStream_t cs = nullptr;
    s = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "pat_mesh_create capture stream");
    m.capture_stream = cs;
  }
  if (!s && !m.host_only) s = upload(row_nb, &m.row_nb);
  if (!s && !m.host_only) s = upload(row_ninj, &m.row_ninj);
  if (!s && !m.host_only) {
    // the sensor rows, for the transposed 16-slot kernels' one-launch-ahead sensor terms
    std::vector<int32_t> rows;
    for (int64_t i = 0; i < N; ++i)
      if (row_ninj[i]) rows.push_back((int32_t)i);
    m.n_inj = (int64_t)rows.size();
    if (rows.empty()) rows.push_back(0);
    s = upload(rows, &m.inj_rows);
  }
  if (!s && !m.host_only) {
    // element data of the c^2 gradient: vertices and K_e^0 (upper triangle, c = 1)
    std::vector<int32_t> et(h.tets);
    std::vector<double> k0(10 * (size_t)h.E);
    for (int64_t e = 0; e < h.E; ++e) {
      const double* g = &h.grads[e * 12];
      int q = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b)
          k0[10 * e + q++] = h.vol[e] * (g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2]);
    }
    s = upload(et, &m.etets);
    if (!s) {
      if (prec == PAT_F64) {
        double* p = nullptr;
        s = upload(k0, &p);
        m.eK0 = p;
      } else {
        std::vector<float> kf(k0.begin(), k0.end());
        float* p = nullptr;
        s = upload(kf, &p);
        m.eK0 = p;
      }
    }
  }
  if (s) {
    free_device(m);
    return s;
  }
  pat_mesh_info& I = m.info;
  I.n_nodes = N;
  I.n_tets = h.E;
  I.n_boundary_faces = (int64_t)h.bfaces.size() / 3;
  I.n_boundary_nodes = h.n_boundary_nodes;
  I.nnz_K = nnz_k;
  I.nnz_K_graph = (int64_t)h.k_col.size();
  I.nnz_B = (int64_t)h.b_col.size();
  I.n_obs = n_obs;
  I.n_steps = n_steps;
  I.prec = prec;
  I.dt = dt;
  const double vb = prec == PAT_F64 ? 8.0 : (m.split ? 8.0 : 4.0);
  I.operator_bytes = (double)(N + 1) * 4.0 + (double)m.fwd.nnz * (4.0 + vb);
  cudaError_t e = m.host_only ? cudaSuccess : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cuda_check(e, "pat_mesh_create");
    free_device(m);
    return PAT_ECUDA;
  }
  return PAT_OK;
}

}  // namespace

extern "C" {

const char* pat_last_error(void) { return pat::last_error(); }
const char* pat_version(void) { return "pat-b300 0.1 (sm_103a)"; }

pat_status pat_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                           const double* c2_elem, const double* det_xyz, int32_t n_obs, double dt, int32_t n_steps,
                           pat_prec prec, uint32_t flags, pat_mesh** out) {
  PAT_RANGE("pat_mesh_create");
  clear_error();
  if (!out || !xyz || !tets || (!det_xyz && n_obs > 0)) {
    set_error("pat_mesh_create: NULL argument");
    return PAT_EINVAL;
  }
  *out = nullptr;
  if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 1 || n_obs < 1 || (prec != PAT_F32 && prec != PAT_F64)) {
    set_error("pat_mesh_create: need dt > 0, n_steps >= 1, n_obs >= 1 and a valid precision "
              "(dt=%g n_steps=%d n_obs=%d prec=%d)", dt, n_steps, n_obs, (int)prec);
    return PAT_EINVAL;
  }
  pat_mesh* mesh = new (std::nothrow) pat_mesh();
  if (!mesh) {
    set_error("pat_mesh_create: out of host memory");
    return PAT_ENOMEM;
  }
  DeviceMesh& m = mesh->d;
  HostMesh& h = m.host;
  pat_status s;
  try {
    s = assemble_host(xyz, n_nodes, tets, n_tets, c2_elem, h);
    if (s == PAT_OK) s = locate_sensors(det_xyz, n_obs, h);
    h.dt = dt;
    h.n_steps = n_steps;
    if (s == PAT_OK && !(flags & PAT_MESH_SKIP_STABILITY)) s = check_stability(h, nullptr);
  } catch (const std::bad_alloc&) {
    set_error("pat_mesh_create: out of host memory");
    s = PAT_ENOMEM;
  }
  if (s != PAT_OK) {
    delete mesh;
    return s;
  }
  m.prec = prec;
  m.flags = flags;
  s = build_device(mesh, flags);
  if (s != PAT_OK) {
    delete mesh;
    return s;
  }
  *out = mesh;
  return PAT_OK;
}

pat_status pat_mesh_set_c2(pat_mesh* mesh, const double* c2_elem) {
  clear_error();
  if (!mesh || !c2_elem) {
    set_error("pat_mesh_set_c2: NULL argument");
    return PAT_EINVAL;
  }
  DeviceMesh& m = mesh->d;
  HostMesh& h = m.host;
  for (int64_t e = 0; e < h.E; ++e) {
    if (!(c2_elem[e] > 0.0) || !std::isfinite(c2_elem[e])) {
      set_error("pat_mesh_set_c2: c2 of tetrahedron %lld is %g (must be finite and > 0)", (long long)e, c2_elem[e]);
      return PAT_EINVAL;
    }
  }
  std::vector<double> old(h.c2);
  h.c2.assign(c2_elem, c2_elem + h.E);
  assemble_stiffness(h);
  pat_status s = PAT_OK;
  if (!(m.flags & PAT_MESH_SKIP_STABILITY)) s = check_stability(h, nullptr);
  if (s != PAT_OK) {  // keep the previous, stable operator
    h.c2 = old;
    assemble_stiffness(h);
    return s;
  }
  if (!m.host_only) {
    s = cuda_check(cudaDeviceSynchronize(), "pat_mesh_set_c2");
    if (s) return s;
  }
  free_device(m);
  return build_device(mesh, m.flags);
}

pat_status pat_mesh_destroy(pat_mesh* mesh) {
  clear_error();
  if (!mesh) return PAT_OK;
  free_device(mesh->d);
  delete mesh;
  return PAT_OK;
}

pat_status pat_mesh_query(const pat_mesh* mesh, pat_mesh_info* info) {
  clear_error();
  if (!mesh || !info) {
    set_error("pat_mesh_query: NULL argument");
    return PAT_EINVAL;
  }
  *info = mesh->d.info;
  return PAT_OK;
}

pat_status pat_mesh_export(const pat_mesh* mesh, double* lumped_mass, int32_t* det_nodes, double* det_w,
                           int32_t* boundary_faces) {
  clear_error();
  if (!mesh) {
    set_error("pat_mesh_export: NULL mesh");
    return PAT_EINVAL;
  }
  const HostMesh& h = mesh->d.host;
  if (lumped_mass) std::memcpy(lumped_mass, h.ml.data(), h.ml.size() * sizeof(double));
  if (det_nodes) std::memcpy(det_nodes, h.det_node.data(), h.det_node.size() * sizeof(int32_t));
  if (det_w) std::memcpy(det_w, h.det_w.data(), h.det_w.size() * sizeof(double));
  if (boundary_faces) std::memcpy(boundary_faces, h.bfaces.data(), h.bfaces.size() * sizeof(int32_t));
  return PAT_OK;
}

pat_status pat_mesh_export_csr(const pat_mesh* mesh, int32_t which, int64_t* nnz, int64_t* row_ptr, int32_t* col,
                               double* val) {
  clear_error();
  if (!mesh || (which != 0 && which != 1)) {
    set_error("pat_mesh_export_csr: NULL mesh or which not in {0, 1}");
    return PAT_EINVAL;
  }
  const HostMesh& h = mesh->d.host;
  const auto& P = which == 0 ? h.k_ptr : h.b_ptr;
  const auto& C = which == 0 ? h.k_col : h.b_col;
  const auto& Vv = which == 0 ? h.k_val : h.b_val;
  if (nnz) *nnz = (int64_t)C.size();
  if (row_ptr) std::memcpy(row_ptr, P.data(), P.size() * sizeof(int64_t));
  if (col) std::memcpy(col, C.data(), C.size() * sizeof(int32_t));
  if (val) std::memcpy(val, Vv.data(), Vv.size() * sizeof(double));
  return PAT_OK;
}

pat_status pat_workspace_bytes(const pat_mesh* mesh, int32_t op, int32_t K, size_t* bytes) {
  clear_error();
  if (!mesh || !bytes || op < 0 || op > 3) {
    set_error("pat_workspace_bytes: NULL argument or op not in {0, 1, 2, 3}");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_workspace_bytes")) return PAT_EINVAL;
  *bytes = (op == 3) ? grad_workspace_bytes(mesh->d, K)
                     : (op == 2) ? rto_layout(mesh->d, K).total : state_bytes(mesh->d, K);
  return PAT_OK;
}

pat_status pat_forward(const pat_mesh* mesh, const void* p0, int32_t K, void* Y, double scale, void* ws,
                       size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_forward");
  clear_error();
  if (!mesh || !p0 || !Y) {
    set_error("pat_forward: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_forward") || !check_device(mesh, "pat_forward")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 0, K, ws, ws_bytes, "pat_forward");
  if (s) return s;
  return forward(mesh->d, p0, K, Y, scale, ws, (cudaStream_t)stream);
}

pat_status pat_adjoint(const pat_mesh* mesh, const void* Yhat, int32_t K, void* p_hat, double scale, void* ws,
                       size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_adjoint");
  clear_error();
  if (!mesh || !Yhat || !p_hat) {
    set_error("pat_adjoint: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_adjoint") || !check_device(mesh, "pat_adjoint")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 1, K, ws, ws_bytes, "pat_adjoint");
  if (s) return s;
  return adjoint(mesh->d, Yhat, K, p_hat, scale, ws, (cudaStream_t)stream);
}

pat_status pat_cgls_layout(const pat_mesh* mesh, int32_t K, size_t* off) {
  clear_error();
  if (!mesh || !off) {
    set_error("pat_cgls_layout: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_cgls_layout")) return PAT_EINVAL;
  const RtoLayout L = rto_layout(mesh->d, K);
  off[0] = L.x;
  off[1] = L.d;
  off[2] = L.r_d;
  off[3] = L.r_p;
  off[4] = L.s;
  off[5] = L.gamma;
  off[6] = L.status;
  return PAT_OK;
}

pat_status pat_lsqr_layout(const pat_mesh* mesh, int32_t K, size_t* off) {
  clear_error();
  if (!mesh || !off) {
    set_error("pat_lsqr_layout: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_lsqr_layout")) return PAT_EINVAL;
  const RtoLayout L = rto_layout(mesh->d, K);
  off[0] = L.x;
  off[1] = L.r_d;
  off[2] = L.r_p;
  off[3] = L.d;
  off[4] = L.w;
  off[5] = L.lsq;
  off[6] = L.status;
  return PAT_OK;
}

pat_status pat_cgls_begin(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K, const void* eta,
                          const void* xi, uint64_t seed, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (!mesh || !y_obs) {
    set_error("pat_cgls_begin: NULL argument");
    return PAT_EINVAL;
  }
  if (!(sigma > 0.0) || !std::isfinite(sigma)) {
    set_error("pat_cgls_begin: sigma must be finite and > 0 (got %g)", sigma);
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_cgls_begin") || !check_device(mesh, "pat_cgls_begin")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_cgls_begin");
  if (s) return s;
  return cgls_begin(mesh->d, y_obs, sigma, K, eta, xi, seed, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_cgls_iterate(const pat_mesh* mesh, double sigma, int32_t K, int32_t n_iter, double* resid, void* ws,
                            size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_cgls_iterate");
  clear_error();
  if (!mesh || n_iter < 0) {
    set_error("pat_cgls_iterate: NULL mesh or n_iter < 0");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_cgls_iterate") || !check_device(mesh, "pat_cgls_iterate")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_cgls_iterate");
  if (s) return s;
  return cgls_iterate(mesh->d, sigma, K, n_iter, resid, (char*)ws, (cudaStream_t)stream, true);
}

pat_status pat_cgls_finish(const pat_mesh* mesh, int32_t K, double* samples, double* mean, double* stdev, void* ws,
                           size_t ws_bytes, void* stream) {
  clear_error();
  if (!mesh) {
    set_error("pat_cgls_finish: NULL mesh");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_cgls_finish") || !check_device(mesh, "pat_cgls_finish")) return PAT_EINVAL;
  if (stdev && K < 2) {
    set_error("pat_cgls_finish: the std estimator needs K >= 2");
    return PAT_EINVAL;
  }
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_cgls_finish");
  if (s) return s;
  return cgls_finish(mesh->d, K, samples, mean, stdev, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_rto_sample(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K, int32_t n_iter,
                          const void* eta, const void* xi, uint64_t seed, double* samples, double* mean,
                          double* stdev, double* resid, void* ws, size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_rto_sample");
  pat_status s = pat_cgls_begin(mesh, y_obs, sigma, K, eta, xi, seed, ws, ws_bytes, stream);
  if (s) return s;
  if (resid) {
    s = residual_norms(mesh->d, K, resid, (char*)ws, (cudaStream_t)stream, true);
    if (s) return s;
  }
  s = pat_cgls_iterate(mesh, sigma, K, n_iter, resid ? resid + 2 * (int64_t)K : nullptr, ws, ws_bytes, stream);
  if (s) return s;
  return pat_cgls_finish(mesh, K, samples, mean, stdev, ws, ws_bytes, stream);
}

static pat_status lsqr_begin_checked(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K,
                                     const void* eta, const void* xi, uint64_t seed, bool zero_draws, void* ws,
                                     size_t ws_bytes, void* stream, const char* fn) {
  if (!mesh || !y_obs) {
    set_error("%s: NULL argument", fn);
    return PAT_EINVAL;
  }
  if (!(sigma > 0.0) || !std::isfinite(sigma)) {
    set_error("%s: sigma must be finite and > 0 (got %g)", fn, sigma);
    return PAT_EINVAL;
  }
  if (bad_K(K, fn) || !check_device(mesh, fn)) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, fn);
  if (s) return s;
  return lsqr_begin(mesh->d, y_obs, sigma, K, eta, xi, seed, zero_draws, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_lsqr_begin(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K, const void* eta,
                          const void* xi, uint64_t seed, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  return lsqr_begin_checked(mesh, y_obs, sigma, K, eta, xi, seed, false, ws, ws_bytes, stream, "pat_lsqr_begin");
}

pat_status pat_lsqr_iterate(const pat_mesh* mesh, double sigma, int32_t K, int32_t n_iter, double* resid, void* ws,
                            size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_lsqr_iterate");
  clear_error();
  if (!mesh || n_iter < 0) {
    set_error("pat_lsqr_iterate: NULL mesh or n_iter < 0");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_lsqr_iterate") || !check_device(mesh, "pat_lsqr_iterate")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_lsqr_iterate");
  if (s) return s;
  return lsqr_iterate(mesh->d, sigma, K, n_iter, resid, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_rto_sample_lsqr(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K, int32_t n_iter,
                               const void* eta, const void* xi, uint64_t seed, double* samples, double* mean,
                               double* stdev, double* resid, void* ws, size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_rto_sample_lsqr");
  clear_error();
  if (n_iter < 0 || (stdev && K < 2)) {
    set_error("pat_rto_sample_lsqr: n_iter < 0, or stdev asked with K < 2");
    return PAT_EINVAL;
  }
  pat_status s =
      lsqr_begin_checked(mesh, y_obs, sigma, K, eta, xi, seed, false, ws, ws_bytes, stream, "pat_rto_sample_lsqr");
  if (s) return s;
  if (resid) {
    s = lsqr_residual(mesh->d, K, resid, (char*)ws, (cudaStream_t)stream);
    if (s) return s;
  }
  s = lsqr_iterate(mesh->d, sigma, K, n_iter, resid ? resid + K : nullptr, (char*)ws, (cudaStream_t)stream);
  if (s) return s;
  return cgls_finish(mesh->d, K, samples, mean, stdev, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_map_estimate(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t n_iter, int32_t solver,
                            double* x_map, double* resid, void* ws, size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_map_estimate");
  clear_error();
  if (n_iter < 0 || (solver != 0 && solver != 1) || !x_map) {
    set_error("pat_map_estimate: n_iter < 0, solver not 0 (CGLS) or 1 (LSQR), or NULL x_map");
    return PAT_EINVAL;
  }
  const char* fn = "pat_map_estimate";
  cudaStream_t st = (cudaStream_t)stream;
  pat_status s;
  if (solver == 1) {
    s = lsqr_begin_checked(mesh, y_obs, sigma, 1, nullptr, nullptr, 0, true, ws, ws_bytes, stream, fn);
    if (s) return s;
    if (resid) {
      s = lsqr_residual(mesh->d, 1, resid, (char*)ws, st);
      if (s) return s;
    }
    s = lsqr_iterate(mesh->d, sigma, 1, n_iter, resid ? resid + 1 : nullptr, (char*)ws, st);
  } else {
    if (!mesh || !y_obs || !(sigma > 0.0) || !std::isfinite(sigma)) {
      set_error("%s: NULL argument or sigma not finite and > 0", fn);
      return PAT_EINVAL;
    }
    if (!check_device(mesh, fn)) return PAT_EINVAL;
    s = check_ws(mesh, 2, 1, ws, ws_bytes, fn);
    if (s) return s;
    s = cgls_begin(mesh->d, y_obs, sigma, 1, nullptr, nullptr, 0, (char*)ws, st, true);
    if (s) return s;
    if (resid) {
      s = residual_norms(mesh->d, 1, resid, (char*)ws, st, false);
      if (s) return s;
    }
    s = cgls_iterate(mesh->d, sigma, 1, n_iter, resid ? resid + 1 : nullptr, (char*)ws, st, false);
  }
  if (s) return s;
  return cgls_finish(mesh->d, 1, x_map, nullptr, nullptr, (char*)ws, st);
}

pat_status pat_whitened_misfit(const pat_mesh* mesh, const double* x, const void* y_obs, double sigma, int32_t K,
                               double* out, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (!mesh || !x || !y_obs || !out || !(sigma > 0.0) || !std::isfinite(sigma)) {
    set_error("pat_whitened_misfit: NULL argument or sigma not finite and > 0");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_whitened_misfit") || !check_device(mesh, "pat_whitened_misfit")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_whitened_misfit");
  if (s) return s;
  return whitened_misfit(mesh->d, x, y_obs, sigma, K, out, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_rto_sample_multi(int32_t n_jobs, const pat_rto_job* jobs, int32_t n_iter, void* stream) {
  PAT_RANGE("pat_rto_sample_multi");
  clear_error();
  if (n_jobs < 1 || !jobs || n_iter < 0) {
    set_error("pat_rto_sample_multi: need n_jobs >= 1, jobs and n_iter >= 0");
    return PAT_EINVAL;
  }
  std::vector<Job> J;
  for (int32_t g = 0; g < n_jobs; ++g) {
    const pat_rto_job& q = jobs[g];
    if (!q.mesh || !q.y_obs) {
      set_error("pat_rto_sample_multi: job %d has a NULL mesh or y_obs", g);
      return PAT_EINVAL;
    }
    if (!(q.sigma > 0.0) || !std::isfinite(q.sigma)) {
      set_error("pat_rto_sample_multi: job %d: sigma must be finite and > 0", g);
      return PAT_EINVAL;
    }
    if (bad_K(q.K, "pat_rto_sample_multi") || !check_device(q.mesh, "pat_rto_sample_multi")) return PAT_EINVAL;
    if (q.stdev && q.K < 2) {
      set_error("pat_rto_sample_multi: job %d: the std estimator needs K >= 2", g);
      return PAT_EINVAL;
    }
    pat_status s = check_ws(q.mesh, 2, q.K, q.workspace, q.workspace_bytes, "pat_rto_sample_multi");
    if (s) return s;
    const DeviceMesh& m = q.mesh->d;
    const DeviceMesh& m0 = jobs[0].mesh->d;
    if (m.prec != m0.prec || m.split != m0.split || !m.three_level || !m0.three_level) {
      set_error("pat_rto_sample_multi: all meshes must share precision and coefficient storage and use the "
                "three-level form");
      return PAT_EUNSUPPORTED;
    }
    for (int32_t h = 0; h < g; ++h)
      if (jobs[h].workspace == q.workspace) {
        set_error("pat_rto_sample_multi: jobs %d and %d share a workspace", h, g);
        return PAT_EINVAL;
      }
    J.push_back(Job{&m, q.K, q.y_obs, q.sigma, q.eta, q.xi, q.seed, q.samples, q.mean, q.stdev, (char*)q.workspace});
  }
  return rto_multi(J, n_iter, (cudaStream_t)stream);
}

pat_status pat_rto_status(const pat_mesh* mesh, int32_t K, const void* ws, void* stream) {
  clear_error();
  if (!mesh || !ws) {
    set_error("pat_rto_status: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_rto_status")) return PAT_EINVAL;
  const RtoLayout L = rto_layout(mesh->d, K);
  int word = 0;
  pat_status s = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "pat_rto_status sync");
  if (s) return s;
  s = cuda_check(cudaMemcpy(&word, (const char*)ws + L.status, 4, cudaMemcpyDeviceToHost), "pat_rto_status read");
  if (s) return s;
  if (word != 0) {
    set_error("CGLS produced a non-finite or non-positive scalar (status %d)", word);
    return (pat_status)word;
  }
  if (mesh->d.d_status) {
    s = cuda_check(cudaMemcpy(&word, mesh->d.d_status, 4, cudaMemcpyDeviceToHost), "pat_rto_status read");
    if (s) return s;
    if (word != 0) {
      set_error("a time-step kernel gave up waiting for its shared-memory copies (status %d)", word);
      // reported once: clear the word so that later calls on the mesh start clean
      s = cuda_check(cudaMemset(mesh->d.d_status, 0, 4), "pat_rto_status clear");
      if (s) return s;
      return (pat_status)word;
    }
  }
  return PAT_OK;
}

pat_status pat_mesh_set_first_sample(pat_mesh* mesh, int64_t first_sample) {
  clear_error();
  // with K <= 1024 the largest draw index first_sample + K - 1 stays below 2^23
  if (!mesh || first_sample < 0 || first_sample > kMaxDrawSample - 1024) {
    set_error("pat_mesh_set_first_sample: NULL mesh or first_sample outside [0, %lld]",
              (long long)(kMaxDrawSample - 1024));
    return PAT_EINVAL;
  }
  mesh->d.first_sample = first_sample;
  return PAT_OK;
}

pat_status pat_rto_moments(const pat_mesh* mesh, int32_t K, const double* center, double* out, void* ws,
                           size_t ws_bytes, void* stream) {
  clear_error();
  if (!mesh || !out) {
    set_error("pat_rto_moments: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_rto_moments") || !check_device(mesh, "pat_rto_moments")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_rto_moments");
  if (s) return s;
  return rto_moments(mesh->d, K, center, out, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_moments_finish(int64_t n_nodes, double n_samples, int32_t which, double* v, void* stream) {
  clear_error();
  if (!v || n_nodes < 1 || (which != 0 && which != 1) || !(n_samples >= (which == 0 ? 1.0 : 2.0))) {
    set_error("pat_moments_finish: NULL buffer, n_nodes < 1, which not 0 or 1, or too few samples (%g)", n_samples);
    return PAT_EINVAL;
  }
  return moments_finish(n_nodes, n_samples, which, v, (cudaStream_t)stream);
}

pat_status pat_mesh_set_wait_cycles(pat_mesh* mesh, int64_t cycles) {
  clear_error();
  if (!mesh) {
    set_error("pat_mesh_set_wait_cycles: NULL mesh");
    return PAT_EINVAL;
  }
  mesh->d.tile_wait_cycles = cycles > 0 ? (long long)cycles : 4000000000ll;
  // captured solves carry the previous budget in their kernel arguments
  std::lock_guard<std::mutex> lock(mesh->d.graph_mutex);
  drop_graphs_locked(mesh->d);
  return PAT_OK;
}

pat_status pat_grad_c2(const pat_mesh* mesh, const void* p0, const void* Yhat, int32_t K, double* g_c2,
                       void* p0_grad, void* ws, size_t ws_bytes, void* stream) {
  PAT_RANGE("pat_grad_c2");
  clear_error();
  if (!mesh || !p0 || !Yhat || !g_c2) {
    set_error("pat_grad_c2: NULL argument");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_grad_c2") || !check_device(mesh, "pat_grad_c2")) return PAT_EINVAL;
  pat_status s = check_ws(mesh, 3, K, ws, ws_bytes, "pat_grad_c2");
  if (s) return s;
  return grad_c2(mesh->d, p0, Yhat, K, g_c2, p0_grad, (char*)ws, (cudaStream_t)stream);
}

pat_status pat_select_variant(pat_mesh* mesh, int32_t K, int32_t direction, const pat_tune_entry* v) {
  clear_error();
  if (!mesh || !v || direction < 0 || direction > 1) {
    set_error("pat_select_variant: NULL argument or direction not in {0, 1}");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_select_variant")) return PAT_EINVAL;
  const bool f32s = mesh->d.prec == PAT_F32 && mesh->d.split;
  if (v->packed == 7) {  // row pairs
    if (!(f32s && mesh->d.fwd.pair_col && mesh->d.adj3.pair_col && v->V == 8 && K % 8 == 0) ||
        (v->min_blocks != 1 && v->min_blocks != 3)) {
      set_error("pat_select_variant: the row-pair kernel needs FP32 split coefficients, pair tables (rows wider "
                "than 8 slots, every pair within %d union slots), V = 8 and min_blocks 1 or 3", kPairSlots);
      return PAT_EINVAL;
    }
    TuneCfg c;
    c.V = 8;
    c.packed = 7;
    c.persist = 1;
    c.pdl = v->pdl;
    c.minb = v->min_blocks;
    std::lock_guard<std::mutex> lock(mesh->d.tune_mutex);
    mesh->d.tuned[std::make_pair((int)direction, (int)K)] = c;
    std::lock_guard<std::mutex> lock2(mesh->d.graph_mutex);
    drop_graphs_locked(mesh->d);
    return PAT_OK;
  }
  if (v->packed == 8) {  // row quads
    if (!(f32s && mesh->d.fwd.quad_col && mesh->d.adj3.quad_col && mesh->d.fwd.w16r_col && v->V == 8 &&
          K == 64) || v->own_async == 2) {
      set_error("pat_select_variant: the row-quad kernel needs FP32 split coefficients, the 16-slot copy (rows "
                "wider than 8 slots), V = 8, K = 64 and own_async 0 or 1");
      return PAT_EINVAL;
    }
    TuneCfg c;
    c.V = 8;
    c.packed = 8;
    c.persist = 1;
    c.pdl = v->pdl;
    c.own = v->own_async ? 1 : 0;
    std::lock_guard<std::mutex> lock(mesh->d.tune_mutex);
    mesh->d.tuned[std::make_pair((int)direction, (int)K)] = c;
    std::lock_guard<std::mutex> lock2(mesh->d.graph_mutex);
    drop_graphs_locked(mesh->d);
    return PAT_OK;
  }
  if (v->packed == 5 || v->packed == 6) {  // 16-slot fixed-width rows (quad-interleaved / row-major)
    const bool ok = f32s && mesh->d.fwd.w16_col && K % 8 == 0
                        ? v->V == 8
                        : (f32s && mesh->d.fwd.w16_col && K == 1 && v->V == 1 && v->packed == 5);
    const int nb = v->gather_batch ? v->gather_batch : 4;
    if (!ok || (nb != 4 && nb != 8) ||
        (v->min_blocks != 1 && !(v->min_blocks == 3 && (nb == 8 || (v->packed == 6 && v->own_async == 1))) &&
         !(v->min_blocks == 6 && v->V == 1))) {
      set_error("pat_select_variant: 16-slot variant V=%d gather_batch=%d min_blocks=%d is not available for K=%d on "
                "this mesh (it needs rows wider than 8 slots, FP32 split coefficients, V = 8 or K = V = 1)",
                v->V, v->gather_batch, v->min_blocks, K);
      return PAT_EINVAL;
    }
    TuneCfg c;
    c.V = v->V;
    c.packed = v->packed;
    c.persist = 1;
    c.pdl = v->pdl;
    c.batch = nb;
    c.early = v->early;
    c.big = v->big_blocks && nb == 4;
    c.minb = v->min_blocks;
    if (v->own_async == 2 && (v->packed != 6 || K > 256 || K % 8 || 32 % (K / 8) || !mesh->d.d_status ||
                              nb != 4 || c.big || v->prefetch_meta)) {
      set_error("pat_select_variant: own rows by bulk copies (own_async = 2) need the row-major 16-slot rows "
                "(packed 6), rounds of 4, 256-thread blocks, no metadata prefetch and K in {8, 16, ..., 256}");
      return PAT_EINVAL;
    }
    if (v->own_async == 3 && (v->packed != 6 || nb != 4 || c.big || v->prefetch_meta || v->dyn_chunks ||
                              v->wide_loads || v->min_blocks != 1)) {
      set_error("pat_select_variant: own x_{s-1} rows only (own_async = 3) need the row-major 16-slot rows "
                "(packed 6), rounds of 4, 256-thread blocks and no other option");
      return PAT_EINVAL;
    }
    c.own = v->own_async == 2 ? 2 : v->own_async == 3 ? 3 : (v->own_async && nb == 4 && !c.big ? 1 : 0);
    c.tail = v->tail_serial && nb == 4 && !c.big;
    c.pfm = v->prefetch_meta && (v->packed == 6 || (v->packed == 5 && K == 64)) && nb == 4 && !c.big;
    if (c.pfm) c.tail = 1;
    if (v->dyn_chunks && (v->packed != 6 || nb != 4 || c.big || c.pfm || c.own == 2 || !mesh->d.three_level)) {
      set_error("pat_select_variant: chunks handed out by a counter (dyn_chunks) need the row-major 16-slot rows "
                "(packed 6) of the three-level form, rounds of 4, 256-thread blocks, no metadata prefetch and "
                "own_async 0 or 1");
      return PAT_EINVAL;
    }
    c.dyn = v->dyn_chunks ? 1 : 0;
    if (c.dyn) c.tail = 1;
    // 256-bit metadata loads: row-major slots, each round's columns with it
    c.wide = v->wide_loads && v->packed == 6 && c.early && nb == 4 && !c.big && !c.pfm && !c.dyn && c.own != 2;
    std::lock_guard<std::mutex> lock(mesh->d.tune_mutex);
    mesh->d.tuned[std::make_pair((int)direction, (int)K)] = c;
    std::lock_guard<std::mutex> lock2(mesh->d.graph_mutex);
    drop_graphs_locked(mesh->d);
    return PAT_OK;
  }
  const bool ok_v = (v->V == 1 || v->V == 2 || v->V == 4 || v->V == 8) && K % v->V == 0 &&
                    (mesh->d.prec == PAT_F32 || v->V <= 2);
  const bool ok_p = v->packed == 0 ? v->V != 8 && !(v->V == 1 && v->packed)
                    : v->packed == 1 ? f32s && (v->V == 4 || v->V == 8) && (v->chunk == 2 || v->chunk == 4 ||
                                                                             (v->chunk == 8 && v->V == 4))
                    : v->packed == 2 ? f32s && v->V == 8 && K <= 8 * 1024 / kTileRows
                    : v->packed == 3 ? f32s && (v->V == 4 || v->V == 8 || (v->V == 1 && K == 1))
                    : v->packed == 4 ? f32s && v->V == 8 && K <= 8 * 512 / kTileRows
                                     : false;
  const bool ok_pf = v->prefetch == 0 || (v->prefetch >= 1 && v->prefetch <= 4 && (v->packed == 1 || v->packed == 3) &&
                                          v->V != 1);
  // min_blocks 5 or 6 with V = 8 only for the persistent kernels whose source rows and
  // metadata come per batch (2 or 4 rows); otherwise they would spill
  const bool batched8 = v->packed == 3 && v->persistent == 1 && (v->gather_batch == 2 || v->gather_batch == 4);
  if (!ok_v || !ok_p || !ok_pf || (v->staged && K / v->V < 2) ||
      (v->min_blocks != 1 && v->min_blocks != 6 && !(v->min_blocks == 5 && batched8)) ||
      (v->min_blocks > 1 && v->V == 8 && !batched8)) {
    set_error("pat_select_variant: variant V=%d packed=%d chunk=%d staged=%d is not available for K=%d on this mesh",
              v->V, v->packed, v->chunk, v->staged, K);
    return PAT_EINVAL;
  }
  TuneCfg c;
  c.V = v->V;
  c.stage = v->staged;
  c.packed = v->packed;
  c.chunk = v->chunk ? v->chunk : 4;
  c.minb = v->min_blocks;
  c.early = v->early;
  c.order = v->zorder;
  c.big = v->big_blocks && v->V == 8 && (v->packed == 1 || v->packed == 3) && v->persistent != 2;
  c.pf = v->prefetch;
  c.persist = (v->packed == 3 && v->V != 1) ? std::min(std::max(v->persistent, 0), 3) : 0;
  if (c.persist == 3 && (v->V != 8 || K / v->V < 4)) c.persist = 1;
  c.pdl = c.persist && v->pdl;
  c.wide = c.persist && v->wide_loads && v->V == 8;
  c.hint = c.persist == 1 && !c.wide && !c.big && v->l2_hints && v->V == 8;
  c.batch = (c.persist == 1 && !c.wide && !c.big && !c.hint && v->V == 8 &&
             (v->gather_batch == 2 || v->gather_batch == 4 || v->gather_batch == 8))
                ? v->gather_batch
                : 0;
  {
    std::lock_guard<std::mutex> lock(mesh->d.tune_mutex);
    mesh->d.tuned[std::make_pair((int)direction, (int)K)] = c;
  }
  std::lock_guard<std::mutex> lock(mesh->d.graph_mutex);
  drop_graphs_locked(mesh->d);
  return PAT_OK;
}

pat_status pat_autotune(pat_mesh* mesh, int32_t K, void* ws, size_t ws_bytes, int32_t n_probe, pat_tune_entry* table,
                        int32_t* n_entries, void* stream) {
  PAT_RANGE("pat_autotune");
  clear_error();
  if (!mesh || n_probe < 1) {
    set_error("pat_autotune: NULL mesh or n_probe < 1");
    return PAT_EINVAL;
  }
  if (bad_K(K, "pat_autotune") || !check_device(mesh, "pat_autotune")) return PAT_EINVAL;
  if (!mesh->d.three_level) {
    set_error("pat_autotune: only the three-level form has tunable variants");
    return PAT_EUNSUPPORTED;
  }
  pat_status s = check_ws(mesh, 2, K, ws, ws_bytes, "pat_autotune");
  if (s) return s;
  int n = 0;
  s = autotune(mesh->d, K, (char*)ws, n_probe, table, &n, (cudaStream_t)stream);
  if (n_entries) *n_entries = n;
  return s;
}

pat_status pat_profile_enable(pat_mesh* mesh, int32_t enable) {
  clear_error();
  if (!mesh) {
    set_error("pat_profile_enable: NULL mesh");
    return PAT_EINVAL;
  }
  Profiler& P = mesh->d.prof;
  P.on = enable != 0;
  P.used = 0;
  P.fwd_launches = P.adj_launches = P.total_launches = 0;
  return PAT_OK;
}

pat_status pat_profile_read(pat_mesh* mesh, pat_profile* out) {
  clear_error();
  if (!mesh || !out) {
    set_error("pat_profile_read: NULL argument");
    return PAT_EINVAL;
  }
  Profiler& P = mesh->d.prof;
  pat_status s = cuda_check(cudaDeviceSynchronize(), "pat_profile_read sync");
  if (s) return s;
  std::memset(out, 0, sizeof(*out));
  for (size_t i = 0; i < P.used; ++i) {
    float ms = 0.0f;
    s = cuda_check(cudaEventElapsedTime(&ms, (cudaEvent_t)P.events[2 * i], (cudaEvent_t)P.events[2 * i + 1]),
                   "pat_profile_read elapsed");
    if (s) return s;
    if (P.kind[i] == 0) {
      out->fwd_ms += ms;
      out->fwd_loops++;
    } else {
      out->adj_ms += ms;
      out->adj_loops++;
    }
  }
  out->fwd_launches = P.fwd_launches;
  out->adj_launches = P.adj_launches;
  out->total_launches = P.total_launches;
  return PAT_OK;
}

pat_status pat_draw_normals(uint64_t seed, int32_t stream_id, int64_t n_elem, int32_t K, double* out, void* stream) {
  clear_error();
  if (!out || n_elem < 0 || K < 1 || (stream_id != 0 && stream_id != 1)) {
    set_error("pat_draw_normals: bad argument");
    return PAT_EINVAL;
  }
  return draw_normals(seed, stream_id, n_elem, K, out, (cudaStream_t)stream);
}

}  // extern "C"
