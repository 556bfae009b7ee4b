// Internal declarations shared by the host assembly, the kernels and the C ABI.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <array>
#include <cstdint>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/pat.h"

namespace pat {

// NVTX ranges around the library's calls, solves and solver iterations, so a
// timeline tool (Nsight Systems, or ncu's range filters) shows where a run's
// time goes; without an attached tool each range costs a couple of function
// calls.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define PAT_RANGE_CAT2(a, b) a##b
#define PAT_RANGE_CAT(a, b) PAT_RANGE_CAT2(a, b)
#define PAT_RANGE(name) ::pat::NvtxRange PAT_RANGE_CAT(pat_nvtx_range_, __LINE__)(name)


// Thread-local error message behind pat_last_error().
void set_error(const char* fmt, ...);
void clear_error();
const char* last_error();

// Column tags of the device CSR rows (see DeviceMesh).
constexpr uint32_t kTagB = 0x80000000u;    // entry acts on the velocity-like field
constexpr uint32_t kTagInj = 0x40000000u;  // entry injects a sensor value (adjoint)
constexpr uint32_t kIdxMask = 0x3FFFFFFFu;

// FP64 assembly on the host (Section 3).
struct HostMesh {
  int64_t N = 0, E = 0;
  int32_t n_obs = 0, n_steps = 0;
  double dt = 0.0;
  std::vector<double> xyz;          // [N][3]
  std::vector<int32_t> tets;        // [E][4]
  std::vector<double> c2;           // [E]
  std::vector<double> vol;          // [E]
  std::vector<double> grads;        // [E][4][3] barycentric gradients
  std::vector<double> ml;           // [N] lumped mass
  // stiffness on the full P1 graph (sorted columns, exact zeros kept)
  std::vector<int64_t> k_ptr;
  std::vector<int32_t> k_col;
  std::vector<double> k_val;
  // boundary mass
  std::vector<int32_t> bfaces;      // [F][3] sorted triples, lexicographic
  std::vector<int64_t> b_ptr;
  std::vector<int32_t> b_col;
  std::vector<double> b_val;
  int64_t n_boundary_nodes = 0;
  // sensors
  std::vector<int32_t> det_node;    // [n_obs][3]
  std::vector<double> det_w;        // [n_obs][3]
};

// Re-assembles the stiffness values for the current m.c2 (same graph).
void assemble_stiffness(HostMesh& m);
// Fills everything but the sensors; returns PAT_OK or an error (message set).
pat_status assemble_host(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
                         const double* c2, HostMesh& m);
// Locates sensors on boundary triangles.
// Nodes and P1 weights per sensor: a node-coincident sensor uses 1, one on a
// boundary triangle 3, one inside a tetrahedron 4 (unused points weigh 0).
constexpr int kDetPts = 4;
pat_status locate_sensors(const double* det_xyz, int32_t n_obs, HostMesh& m);
// Growth check of the propagator (FP64, host).  Returns PAT_OK or PAT_EUNSTABLE.
pat_status check_stability(const HostMesh& m, double* growth_out);

// Device copies.  One CSR per direction, each row holding tagged entries:
//   forward row i:  K entries  (col j, value dt^2 K_ij / M_i)       acting on a
//                   B entries  (col j | kTagB, value dt B_ij / M_i)   acting on w
//   adjoint row i:  K entries  (col j, value dt^2 K_ij)               acting on u
//                   B entries  (col j | kTagB, value dt B_ij / M_i)   acting on u
//                   sensor entries (col d | kTagInj, value w_di)      reading yhat
// Values are split hi + lo (two floats) for FP32 meshes unless single-coefficient
// storage was requested; FP64 meshes store one double.
struct DevCSR {
  int32_t* ptr = nullptr;
  uint32_t* col = nullptr;
  void* hi = nullptr;   // float or double
  float* lo = nullptr;  // FP32 split meshes only
  float2* hl = nullptr; // FP32 split meshes: (hi, lo) interleaved
  int64_t nnz = 0;
  // fixed-width copy (FP32 split meshes): the first 8 entries of every row at
  // [row][8] (padding: column = the row, coefficient 0), the rest of a longer
  // row in an overflow CSR; desc[row] = entries | boundary << 8 | sensors << 16
  uint32_t* ell_col = nullptr;
  float2* ell_hl = nullptr;
  uint32_t* ell_desc = nullptr;
  int32_t* ovf_ptr = nullptr;
  uint32_t* ovf_col = nullptr;
  float2* ovf_hl = nullptr;
  // the same with 16 fixed slots per row (built when some row has more than 8
  // stiffness / boundary entries: the full P1 graph, unstructured meshes)
  uint32_t* w16_col = nullptr;   // quad-interleaved
  float2* w16_hl = nullptr;
  uint32_t* w16r_col = nullptr;  // the same slots row-major ([row][16])
  float2* w16r_hl = nullptr;
  // row pairs (2p, 2p+1): the union of the two rows' stiffness entries, then
  // of their boundary entries, kPairSlots slots per pair ([pair][slot]); per
  // slot the column and both rows' (hi, lo) pairs (zero where a row has no
  // such entry); pair_n = slots used, a multiple of 4 (padding: column 2p,
  // zero coefficients).  Built when every pair fits.
  uint32_t* pair_col = nullptr;
  float4* pair_cf = nullptr;
  uint8_t* pair_n = nullptr;
  // row quads (4q .. 4q+3): the union of the four rows' stiffness entries,
  // then of their boundary entries (the x list), then of their boundary
  // entries again with negated coefficients (the x_{s-1} list), each list
  // merged by column in every row's own order and padded to a multiple of 4
  // (column 4q, zero coefficients).  quad_ptr[q]: first entry of quad q;
  // quad_n[q] = x-list length | x_{s-1}-list length << 16; quad_col[e]: the
  // entry's source row; quad_cf[(e/2)*4 + g] = (hi, lo) of entries e, e+1 for
  // row 4q+g (zero where the row has no such entry).
  int32_t* quad_ptr = nullptr;
  uint32_t* quad_n = nullptr;
  uint32_t* quad_col = nullptr;
  float4* quad_cf = nullptr;
  int32_t* w16_ovf_ptr = nullptr;
  uint32_t* w16_ovf_col = nullptr;
  float2* w16_ovf_hl = nullptr;
  int64_t w16_ovf_n = 0;  // overflow entries of the 16-slot copy (a sensor row owns at least one)
};

constexpr int kEllWide = 16;  // slots of the wide fixed-width copy
constexpr int kPairSlots = 40;  // union slots of a row pair

// The draw counter c = ((k << 1 | stream) << 40) | e leaves 23 bits for the
// sample index k: first_sample + K must stay below 2^23.
constexpr int64_t kMaxDrawSample = int64_t(1) << 23;

// Event-based loop timing and launch counting (pat_profile_*).
struct Profiler {
  bool on = false;
  std::vector<void*> events;  // cudaEvent_t pool, pairs (start, stop)
  std::vector<int> kind;      // per pair: 0 forward, 1 adjoint
  size_t used = 0;            // pairs in use
  int64_t fwd_launches = 0, adj_launches = 0, total_launches = 0;
};

// Kernel variant of the three-level step: samples per thread and row staging.
struct TuneCfg {
  int V = 4;
  int stage = 0;   // row metadata staged in shared memory (generic kernel)
  int packed = 1;  // packed f32x2 kernel (FP32 split coefficients, V = 4 or 8)
  int chunk = 4;   // packed kernel: row entries per pipelined chunk (2, 4 or 8)
  int minb = 1;    // packed kernel: minimum resident blocks per SM asked of the compiler
  int early = 0;   // packed kernel: load the node's own values before the row walk
  int order = 0;   // packed kernel: process rows in Z-order of the node coordinates
  int big = 0;     // packed kernels: 1024-thread blocks
  int pf = 0;      // packed kernels: L2 prefetch distance in resident waves (0: off)
  int persist = 0; // fixed-width kernel: persistent warps walking 32-thread chunks (1: grid-stride, 2: slabs,
                   // 3: grid-stride with the row metadata staged through shared memory)
  int pdl = 0;     // persistent kernel: programmatic dependent launch
  int wide = 0;    // persistent kernel, V = 8: 256-bit loads of 8 contiguous samples
  int hint = 0;    // persistent kernel, V = 8: L2 eviction-priority hints
  int batch = 0;   // persistent kernel, V = 8: source rows in flight per batch (0: 4 with the row's
                   // metadata loaded up front; 8; 2 or 4 with each batch's metadata loaded with it)
  int tail = 0;    // 16-slot kernel: 1 walks a row's tail entries one at a time (0: in pairs)
  int own = 0;     // 16-slot kernel: 1 copies the row's own x_s, x_{s-1} to shared memory by cp.async
  int pfm = 0;     // 16-slot row-major kernel: 1 prefetches the next chunk's row metadata into L1
  int dyn = 0;     // 16-slot row-major kernel: 1 hands the chunks out by an atomic counter
};

struct DeviceMesh {
  int64_t N = 0, E = 0;
  int32_t n_obs = 0, n_steps = 0;
  double dt = 0.0;
  pat_prec prec = PAT_F32;
  bool split = true;
  bool host_only = false;
  int device = 0;
  DevCSR fwd, adj;          // adj: transposed rows of the two-level form
  DevCSR adj3;              // forward rows + sensor entries w_d / (2 M_i) (three-level form)
  bool three_level = true;
  uint32_t flags = 0;
  uint8_t* row_nb = nullptr;    // [N] boundary entries per forward / three-level adjoint row
  uint8_t* row_ninj = nullptr;  // [N] sensor entries per three-level adjoint row
  // rows with sensor entries (ascending): the transposed 16-slot kernels prepare
  // these rows' sensor terms one launch ahead, each at its row's first overflow
  // entry (every sensor row has one: its sensor entries live there)
  int32_t* inj_rows = nullptr;
  int64_t n_inj = 0;
  // tiles of 32 rows for the tile-staged kernel: per tile, contiguous source-row
  // ranges to stage in shared memory, and per CSR entry its 16-bit slot
  int32_t n_tiles = 0, tile_max_slots = 0;
  int32_t *tile_range_ptr = nullptr, *tile_range_src = nullptr, *tile_range_cnt = nullptr,
          *tile_range_slot = nullptr, *tile_slots = nullptr;
  uint16_t *tile_slot_fwd = nullptr, *tile_slot_adj = nullptr;
  int32_t* d_status = nullptr;  // device status word of the tile kernels (PAT_ETIMEOUT)
  long long tile_wait_cycles = 4000000000ll;  // copy-wait budget of the tile kernels (pat_mesh_set_wait_cycles)
  int64_t first_sample = 0;  // draw index of sample 0 of library-drawn perturbations (pat_mesh_set_first_sample)
  int32_t* row_order = nullptr;  // [N] rows sorted by the Z-order (Morton) key of their coordinates
  int32_t* etets = nullptr;  // [E][4] element vertices (c^2 gradient)
  void* eK0 = nullptr;       // [E][10] real: upper triangle of V grad(l_a).grad(l_b) (c = 1)
  void* minv_hi = nullptr;   // [N] real: 1 / M_i
  float* minv_lo = nullptr;  // [N]
  double* ml = nullptr;      // [N] double
  double* sqrt_ml = nullptr; // [N] double
  int32_t* det_node = nullptr;  // [n_obs][3]
  void* det_w = nullptr;        // [n_obs][3] real
  pat_mesh_info info{};
  HostMesh host;             // kept for export / checks
  mutable Profiler prof;
  // host copies of the forward / three-level adjoint row pointers, and the
  // largest CSR range a 256-thread block covers for a given threads-per-row
  std::vector<int32_t> fwd_ptr_h, adj3_ptr_h;
  mutable std::map<std::pair<int, int>, int> stage_span;
  mutable std::mutex stage_mutex;
  // CUDA graphs of whole forward / transposed solves inside the CGLS loop,
  // keyed by (direction, workspace, K, scale bits); cudaGraphExec_t handles
  mutable std::map<std::tuple<int, const void*, int, uint64_t>, void*> graphs;
  // CUDA graphs of whole gradient evaluations (pat_grad_c2), keyed by
  // (p0, Yhat, g_c2, p0_grad, workspace, K)
  mutable std::map<std::array<uintptr_t, 6>, void*> grad_graphs;
  void* capture_stream = nullptr;  // private cudaStream_t the graphs are captured on
  mutable std::mutex graph_mutex;
  // variants picked by pat_autotune per (direction 0 fwd / 1 adj, K)
  mutable std::map<std::pair<int, int>, TuneCfg> tuned;
  mutable std::mutex tune_mutex;
};

// Destroys every captured graph of the mesh (solves and gradients); the
// caller holds m.graph_mutex.  Called whenever what a graph captured (kernel
// variants, wait budget, operators) changes.
void drop_graphs_locked(const DeviceMesh& m);

// Argument checks shared by the entry points (pat_api.cu): the mesh has device
// copies on the current device; K is in range; a workspace for op (as in
// pat_workspace_bytes) is large enough and 256-byte aligned.  Each sets the
// error message and reports failure.
bool check_device(const pat_mesh* mesh, const char* fn);
bool bad_K(int32_t K, const char* fn);
pat_status check_ws(const pat_mesh* mesh, int op, int K, const void* ws, size_t bytes, const char* fn);

}  // namespace pat

struct pat_mesh {
  pat::DeviceMesh d;
};
