/*
 * pat.h -- C ABI of the B300 photoacoustic RTO library (libpat.so).
 *
 * The library computes, on one CUDA device, the hot path of the matrix-free
 * randomize-then-optimize (RTO) posterior sampler for 3D photoacoustic
 * tomography of arXiv 2607.21373:
 *   - the P1 tetrahedral finite-element forward map G: initial pressure p0 ->
 *     sensor time series Y (Section 3: eq. semi-discrete with lumped mass,
 *     Stoermer-Verlet time stepping eq. fully-discrete, first-order absorbing
 *     boundary eq. boundary, sensor interpolation eq. lagrange);
 *   - its exact algebraic transpose G^T (Section 5.1: eq. backward-recursion
 *     with the transposed step eq. adjoint-verlet);
 *   - batched least-squares solves of the extended RTO system
 *     (eq. extended-matrices, eq. normal-equations, Algorithm 1) by CGLS or
 *     LSQR, K posterior samples at a time, and their pointwise mean / std
 *     (eq. ergodic); the MAP estimate (eq. MAP) and the discrepancy-principle
 *     diagnostic (Section 6.1).
 * Meshes are any tetrahedral meshes; sensors may sit at nodes, on boundary
 * triangles or inside tetrahedra (P1 interpolation, eq. lagrange).
 *
 * Conventions (all entry points):
 *   - Every call returns a pat_status; PAT_OK == 0.  On failure,
 *     pat_last_error() returns a thread-local, NUL-terminated message that stays
 *     valid until the next call on the same thread.  No call prints or aborts.
 *   - "host" pointers are ordinary CPU memory read during the call.  "device"
 *     pointers are CUDA device memory on the device that was current when the
 *     mesh was created; the caller owns them.  The library never allocates
 *     device memory inside a compute call: it uses the caller's workspace.
 *   - Compute calls are asynchronous and stream-ordered on `stream` (a
 *     cudaStream_t, NULL = legacy default stream).  Argument errors are
 *     returned synchronously; a kernel-detected numerical problem is recorded
 *     on the device and reported by the next call that reads it back
 *     (pat_rto_status).
 *   - Stacked samples: a field with K samples is stored node-major, samples
 *     contiguous: element (i, k) of an [N][K] array is at i*K + k.  Time
 *     series are [N_T][N_obs][K]: element (n, d, k) at (n*N_obs + d)*K + k,
 *     n = 0..N_T-1 holding the observation at t = (n+1) dt.
 *   - "real" is float for PAT_F32 meshes and double for PAT_F64 meshes.
 *   - Calls on different meshes may run concurrently; calls that share a
 *     workspace must not overlap on the GPU.
 */
#ifndef PAT_H
#define PAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pat_mesh pat_mesh; /* opaque; owns the device copies of the operators */

typedef enum {
  PAT_OK = 0,
  PAT_EINVAL = 1,       /* bad argument, shape, mesh or sensor placement        */
  PAT_ENOMEM = 2,       /* host or device allocation failed (mesh creation only)*/
  PAT_ECUDA = 3,        /* a CUDA runtime call failed                           */
  PAT_EUNSTABLE = 4,    /* the time step makes the propagator grow (create)     */
  PAT_ENUMERIC = 5,     /* non-finite or non-positive CGLS scalar               */
  PAT_ETIMEOUT = 6,     /* a bounded device wait ran out                        */
  PAT_EUNSUPPORTED = 7  /* valid request the library does not handle           */
} pat_status;

typedef enum { PAT_F32 = 0, PAT_F64 = 1 } pat_prec;

/* pat_mesh_create flags */
#define PAT_MESH_SKIP_STABILITY 0x1u /* do not run the growth check of the time step */
#define PAT_MESH_KEEP_ZEROS     0x2u /* keep graph entries that assemble to exactly 0.0 */
#define PAT_MESH_SINGLE_COEF    0x4u /* PAT_F32: one float per coefficient (no hi+lo split) */
#define PAT_MESH_TWO_LEVEL      0x10u /* step (p^{n+1/2}, dt v) pairs: 16 B per node and sample
                                         instead of the default three-level form's 12 B */
#define PAT_MESH_NO_GRAPHS      0x20u /* launch the CGLS loop's time steps one by one instead of
                                         replaying each wave solve from a CUDA graph */
#define PAT_MESH_HOST_ONLY      0x8u /* assemble on the host only (no device copy); compute
                                        calls on such a mesh return PAT_EINVAL, exports work */

/*
 * Assemble the operators of a P1 tetrahedral mesh and copy them to the current
 * device (Section 3, eq. semi-discrete and the mass-lumping paragraph).
 *
 *   xyz      host, [n_nodes][3] double: node coordinates.
 *   tets     host, [n_tets][4] int32: vertex indices, 0-based, any orientation.
 *   c2_elem  host, [n_tets] double: squared sound speed per tetrahedron, or NULL
 *            for c = 1.  It scales the element stiffness only; the absorbing
 *            boundary matrix is assembled at c = 1 (the paper's nondimensional
 *            setting).
 *   det_xyz  host, [n_obs][3] double: sensor positions, read by P1
 *            interpolation (the general Pi of Section 5.1): a position within
 *            1e-12 of the mesh extent of a node reads that node; one on a
 *            boundary triangle (a tetrahedron face not shared with another
 *            tetrahedron, within 1e-9 of the mesh size) interpolates in that
 *            triangle; any other position inside the mesh interpolates in the
 *            tetrahedron that holds it.
 *   dt       time step; n_steps = N_T observation times t_n = n dt, n = 1..N_T.
 *   prec     state precision of all compute calls on this mesh.
 *   flags    PAT_MESH_* bits.
 *   out      receives the new mesh.
 *
 * Matrices: K_e = c_e^2 V_e grad(l_a).grad(l_b); lumped mass M_L,i = sum of V_e/4
 * over the tetrahedra at node i; B_f = (A_f/12)(1 + delta_ab) on every boundary
 * triangle.  Unless PAT_MESH_SKIP_STABILITY is given, the call runs the
 * propagator for 300 steps in FP64 on the host from a seeded random state and
 * returns PAT_EUNSTABLE when the last 100 steps grow faster than 1e-3 per step.
 * Errors: PAT_EINVAL (index out of range, degenerate tetrahedron, sensor outside
 * the mesh, dt <= 0, n_steps < 1), PAT_EUNSTABLE, PAT_ENOMEM, PAT_ECUDA.
 */
pat_status pat_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                           const double* c2_elem, const double* det_xyz, int32_t n_obs, double dt,
                           int32_t n_steps, pat_prec prec, uint32_t flags, pat_mesh** out);

/*
 * Replace the squared sound speed per tetrahedron (host [n_tets] double) and
 * rebuild the device operators (same mesh, sensors, dt).  The growth check runs
 * again unless the mesh was created with PAT_MESH_SKIP_STABILITY; on
 * PAT_EUNSTABLE the previous c^2 stays in force.  Synchronises the device.
 */
pat_status pat_mesh_set_c2(pat_mesh* mesh, const double* c2_elem);

/* Release a mesh and its device memory.  NULL is accepted. */
pat_status pat_mesh_destroy(pat_mesh* mesh);

/* Sizes of a mesh (host outputs; any pointer may be NULL). */
typedef struct {
  int64_t n_nodes, n_tets, n_boundary_faces, n_boundary_nodes;
  int64_t nnz_K;        /* stored stiffness entries (after dropping exact zeros) */
  int64_t nnz_K_graph;  /* entries of the full P1 graph, zeros included          */
  int64_t nnz_B;
  int32_t n_obs, n_steps, prec;
  double dt;
  double operator_bytes; /* bytes of the forward-step operator read per step   */
  int32_t tile_rows;     /* rows per tile of the tile-staged kernel             */
  int32_t tile_max_staged; /* most source rows any tile stages in shared memory */
  double tile_mean_staged; /* mean source rows staged per tile                   */
} pat_mesh_info;
pat_status pat_mesh_query(const pat_mesh* mesh, pat_mesh_info* info);

/*
 * Copy assembly results to host buffers (each may be NULL):
 *   lumped_mass [N] double; det_nodes [n_obs][4] int32 and det_w [n_obs][4]
 *   double (the nodes and P1 weights of each sensor, weights >= 0: one node
 *   for a node-coincident sensor, a boundary triangle's three, a
 *   tetrahedron's four; unused entries repeat a node with weight 0);
 *   boundary_faces [F][3] int32 (sorted vertex triples, lexicographic order).
 */
pat_status pat_mesh_export(const pat_mesh* mesh, double* lumped_mass, int32_t* det_nodes,
                           double* det_w, int32_t* boundary_faces);

/*
 * Stiffness and boundary matrices as host CSR in FP64 (for checking): row_ptr
 * [N+1] int64, col [nnz] int32, val [nnz] double.  Pass NULL arrays to query
 * nnz only.  which = 0: K (full graph, exact zeros kept); 1: B.
 */
pat_status pat_mesh_export_csr(const pat_mesh* mesh, int32_t which, int64_t* nnz, int64_t* row_ptr,
                               int32_t* col, double* val);

/* Device workspace (bytes) needed by a compute call with K stacked samples.
 * op: 0 = pat_forward, 1 = pat_adjoint, 2 = pat_rto_* (CGLS state included),
 * 3 = pat_grad_c2 (checkpoints included). */
pat_status pat_workspace_bytes(const pat_mesh* mesh, int32_t op, int32_t K, size_t* bytes);

/*
 * Y = scale * G p0 for K stacked initial pressures (Section 3, eq. fully-discrete
 * and eq. discrete-wave-matrix; z0 = (p0, 0)).
 *   p0 device [N][K] real; Y device [N_T][N_obs][K] real (written).
 *   workspace device, >= pat_workspace_bytes(mesh, 0, K) bytes, 256-byte aligned.
 */
pat_status pat_forward(const pat_mesh* mesh, const void* p0, int32_t K, void* Y, double scale,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * pat_forward without a workspace, for callers that cannot allocate device
 * memory where they call it (plug-ins whose host framework owns every device
 * buffer and passes only inputs and outputs; real-time loops that must not
 * allocate).  The paper has no counterpart: this is a deployment variant of
 * pat_forward with the same arguments minus the workspace, and the same result.
 *   - The time-stepping state lives in a fixed 8 MiB device array inside the
 *     library (one per device that loads the library, held until the process
 *     exits), so N*K must not exceed 524,288 for PAT_F32 meshes or 262,144 for
 *     PAT_F64 meshes; larger requests return PAT_EINVAL with a message naming
 *     the limit.  The call never allocates or frees device memory.
 *   - The first call on a device looks up that array's device address (with the
 *     device current) and caches it for the rest of the process; make that first
 *     call before any stream capture.  The cached address does not survive
 *     cudaDeviceReset (the library's module is reloaded and the array may
 *     move): do not call this entry point after resetting the device.
 *   - All calls on a device share the one array: calls that overlap on the GPU
 *     (other streams, other host threads) race and corrupt each other's
 *     results; serialise them.  A call never reads what an earlier call left
 *     in the array.
 */
pat_status pat_forward_noalloc(const pat_mesh* mesh, const void* p0, int32_t K, void* Y, double scale,
                               void* stream);

/*
 * p_hat = scale * G^T Yhat (Section 5.1, eq. backward-recursion and
 * eq. adjoint-verlet): the exact transpose of pat_forward's map, up to rounding.
 *   Yhat device [N_T][N_obs][K] real; p_hat device [N][K] real (written).
 *   workspace >= pat_workspace_bytes(mesh, 1, K).
 */
pat_status pat_adjoint(const pat_mesh* mesh, const void* Yhat, int32_t K, void* p_hat, double scale,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * RTO: K posterior samples by CGLS on the extended system (eq. extended-matrices
 * with the independent Gaussian prior C = M_L^{-1} of eq. iid-prior, so the prior
 * block of b is xi), x0 = 0, exactly n_iter iterations (Algorithm 1; the paper
 * stops at fixed iteration limits).  FP32 meshes keep fields in FP32 and every
 * inner product, norm, CGLS scalar and the iterate x in FP64.
 *   y_obs   device [N_T][N_obs] real: observed data.
 *   sigma   noise standard deviation (> 0).
 *   eta     device [N_T][N_obs][K] real, N(0,1) data perturbations, or NULL to
 *           draw them on the device from `seed` (counter-based generator).
 *   xi      device [N][K] real, N(0,1) prior draws, or NULL (drawn from `seed`).
 *   samples device [N][K] double or NULL; mean, stdev device [N] double or NULL
 *           (stdev needs K >= 2; estimator of eq. ergodic with 1/(K-1)).
 *   resid   device [n_iter+1][K][2] double or NULL: the squared norms of the
 *           data block and the prior block of the residual r_j = b - A x_j of
 *           each iterate, ||r_d||^2 and ||r_p||^2 (the data misfit and prior
 *           terms of the convergence diagnostics of Section 6.1; their sum is
 *           ||r_j||^2).
 *   workspace >= pat_workspace_bytes(mesh, 2, K).
 * Each wave solve of the CGLS loop is captured once into a CUDA graph (per
 * workspace, K and sigma, cached on the mesh) and replayed, unless the stream
 * is already being captured or the mesh has PAT_MESH_NO_GRAPHS.
 * Errors: PAT_EINVAL; PAT_ENUMERIC is reported by pat_rto_status.
 */
pat_status pat_rto_sample(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K,
                          int32_t n_iter, const void* eta, const void* xi, uint64_t seed,
                          double* samples, double* mean, double* stdev, double* resid,
                          void* workspace, size_t workspace_bytes, void* stream);

/*
 * Uneven batch: several RTO problems -- meshes of different sizes, time-step
 * counts and sensor sets, each with its own data, noise level and number of
 * samples K -- solved together with n_iter CGLS iterations each.  Every
 * time-step launch covers the rows of all jobs that still have a step at that
 * index (one launch per step index for the whole batch), the per-sample CGLS
 * work stays per job.  Each job's fields follow pat_rto_sample (device pointers,
 * eta/xi NULL = drawn from seed, samples/mean/stdev may be NULL) and its
 * workspace must hold pat_workspace_bytes(mesh, 2, K).  All meshes must share
 * precision and coefficient storage and use the three-level form
 * (PAT_EUNSUPPORTED otherwise).  Results equal separate pat_rto_sample calls.
 */
typedef struct {
  const pat_mesh* mesh;
  const void* y_obs;
  double sigma;
  int32_t K;
  const void* eta;
  const void* xi;
  uint64_t seed;
  double* samples;
  double* mean;
  double* stdev;
  void* workspace;
  size_t workspace_bytes;
} pat_rto_job;
pat_status pat_rto_sample_multi(int32_t n_jobs, const pat_rto_job* jobs, int32_t n_iter, void* stream);

/*
 * The same solve in pieces, for callers that inspect or resume the CGLS state
 * held in the workspace:
 *   pat_cgls_begin    r = b, s = A^T r, d = s, gamma = ||s||^2, x = 0;
 *   pat_cgls_iterate  n_iter CGLS iterations (q = A d, alpha, x, r, s, beta, d);
 *                     resid (device [n_iter][K][2] double, or NULL) receives
 *                     the data and prior blocks of ||r||^2 of each new iterate;
 *   pat_cgls_finish   copy x to samples and form mean / stdev.
 * pat_cgls_layout returns byte offsets into the workspace of the state fields:
 *   off[0] x [N][K] double, off[1] d [N][K] real, off[2] r_d [N_T][N_obs][K] real,
 *   off[3] r_p [N][K] real, off[4] s [N][K] real, off[5] gamma [K] double,
 *   off[6] status word (int32; 0 = ok, else a pat_status).
 */
pat_status pat_cgls_begin(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K,
                          const void* eta, const void* xi, uint64_t seed, void* workspace,
                          size_t workspace_bytes, void* stream);
pat_status pat_cgls_iterate(const pat_mesh* mesh, double sigma, int32_t K, int32_t n_iter,
                            double* resid, void* workspace, size_t workspace_bytes, void* stream);
pat_status pat_cgls_finish(const pat_mesh* mesh, int32_t K, double* samples, double* mean,
                           double* stdev, void* workspace, size_t workspace_bytes, void* stream);
pat_status pat_cgls_layout(const pat_mesh* mesh, int32_t K, size_t* offsets /* [7] */);

/*
 * LSQR (Paige & Saunders, ACM TOMS 8, 1982; the solver the paper uses,
 * Section 5.1 and Algorithm 1) on the same extended system, workspace and
 * precision rules as the CGLS calls: the Golub-Kahan bidiagonalisation of
 * G_ext, one plane rotation per iteration and the x, w updates, every scalar
 * and x in FP64.  In exact arithmetic its iterates equal CGLS's; it is the
 * more robust of the two in finite precision.  The left vectors are kept
 * unnormalised (beta_i u_i) in the r_d / r_p fields, v in d, w in an extra
 * field; x sits where CGLS keeps it, so pat_cgls_finish (or
 * pat_whitened_misfit) also serves an LSQR solve.
 *   pat_lsqr_begin    beta_1 u_1 = b, alpha_1 v_1 = A^T u_1, w_1 = v_1, x = 0;
 *   pat_lsqr_iterate  n_iter iterations; resid (device [n_iter][K] double, or
 *                     NULL) receives phibar^2 = ||b - A x||^2 of each new
 *                     iterate (the residual identity of the algorithm).
 * Same arguments and errors as pat_cgls_begin / pat_cgls_iterate.
 */
pat_status pat_lsqr_begin(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K,
                          const void* eta, const void* xi, uint64_t seed, void* workspace,
                          size_t workspace_bytes, void* stream);
pat_status pat_lsqr_iterate(const pat_mesh* mesh, double sigma, int32_t K, int32_t n_iter,
                            double* resid, void* workspace, size_t workspace_bytes, void* stream);
/* Byte offsets of the LSQR state in the workspace: off[0] x [N][K] double,
 * off[1] beta u data block [N_T][N_obs][K] real, off[2] beta u prior block
 * [N][K] real, off[3] v [N][K] real, off[4] w [N][K] real, off[5] per-sample
 * scalars [12][K] double (rows: alpha, beta, rhobar, phibar, then temporaries
 * of the last iteration), off[6] status word. */
pat_status pat_lsqr_layout(const pat_mesh* mesh, int32_t K, size_t* offsets /* [7] */);

/* pat_rto_sample with LSQR instead of CGLS (Algorithm 1 as the paper states it);
 * resid [n_iter+1][K] receives ||r_j||^2 of each iterate, starting with ||b||^2. */
pat_status pat_rto_sample_lsqr(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t K,
                               int32_t n_iter, const void* eta, const void* xi, uint64_t seed,
                               double* samples, double* mean, double* stdev, double* resid,
                               void* workspace, size_t workspace_bytes, void* stream);

/*
 * MAP estimate (eq. MAP): the extended least-squares problem with zero
 * perturbations, b = (y_obs / sigma, 0), from x = 0 with n_iter iterations of
 * CGLS (solver 0) or LSQR (solver 1).  x_map device [N] double; resid device
 * [n_iter+1] double or NULL (||r_j||^2).  Workspace >= pat_workspace_bytes(mesh, 2, 1).
 */
pat_status pat_map_estimate(const pat_mesh* mesh, const void* y_obs, double sigma, int32_t n_iter,
                            int32_t solver, double* x_map, double* resid, void* workspace,
                            size_t workspace_bytes, void* stream);

/*
 * Discrepancy-principle diagnostic (Section 6.1): out[k] = ||G x_k - y_obs|| /
 * (sigma sqrt(N_T N_obs)) for each column of x (device [N][K] double), about 1
 * when the data are fitted to the noise level.  Euclidean data norm, as sigma
 * scales the noise vector (eq. noise-model).  out device [K] double.  Runs one
 * forward solve in the solver's workspace (>= pat_workspace_bytes(mesh, 2, K)):
 * it overwrites the d, q_d and time-stepping fields, so call it between solves,
 * not between the iterations of one.
 */
pat_status pat_whitened_misfit(const pat_mesh* mesh, const double* x, const void* y_obs, double sigma,
                               int32_t K, double* out, void* workspace, size_t workspace_bytes,
                               void* stream);

/* Synchronise `stream` and read the workspace's status word (PAT_OK, PAT_ENUMERIC ...),
 * then the mesh's time-step status word: PAT_ETIMEOUT when a tile-staged step
 * kernel gave up waiting for its shared-memory copies (the rows of that tile
 * were then not updated).  The mesh's word is cleared once reported. */
pat_status pat_rto_status(const pat_mesh* mesh, int32_t K, const void* workspace, void* stream);

/*
 * Failure-detection hook: the number of SM clock cycles a block of the
 * tile-staged step kernels (variants packed 2 and 4) waits for its bulk copies
 * before it records PAT_ETIMEOUT in the mesh's status word and gives up on its
 * tile (it still waits for the copies in flight to land before it exits, so
 * no copy outlives its shared memory).  cycles <= 0 restores the default of
 * 4e9 cycles (about two seconds).  A tiny budget makes every wait run out: a
 * test of the timeout path that neither hangs nor faults the GPU.  Drops the
 * mesh's captured CUDA graphs (they hold the previous budget).
 */
pat_status pat_mesh_set_wait_cycles(pat_mesh* mesh, int64_t cycles);

/*
 * Sample parallelism across processes (Section 6.4 runs one sample per process;
 * the paper has no multi-GPU code).  Each process holds a mesh and solves its
 * own K samples; the only exchange is the pointwise posterior statistics of
 * eq. ergodic over all processes' samples, in two passes of sums that the
 * caller adds up across processes (e.g. an NCCL all-reduce of the [N] buffers):
 *
 *   pat_mesh_set_first_sample  library-drawn perturbations (eta, xi NULL) of
 *       sample k of later calls on this mesh use the draw index
 *       first_sample + k (default 0): with first_sample = rank * K the
 *       processes' draws are those of one K_total-sample run, disjoint by
 *       construction.  0 <= first_sample <= 2^23 - 1024, else PAT_EINVAL.
 *   pat_rto_moments  from the iterate x of the last CGLS / LSQR solve held in
 *       `workspace` (K samples): center NULL -> out[i] = sum_k x_ik; center
 *       (device [N] double) -> out[i] = sum_k (x_ik - center_i)^2.  out device
 *       [N] double.  Workspace as pat_rto_sample's.
 *   pat_moments_finish  in place on v (device [n_nodes] double), n_samples
 *       the total over all processes: which 0: v /= n_samples (the mean from
 *       the summed first pass); which 1: v = sqrt(v / (n_samples - 1)) (the
 *       std from the summed second pass, centred on that mean).
 *
 * Order: moments (center NULL) -> sum across processes -> finish 0 = mean ->
 * moments (center = mean) -> sum across processes -> finish 1 = std.
 */
pat_status pat_mesh_set_first_sample(pat_mesh* mesh, int64_t first_sample);
pat_status pat_rto_moments(const pat_mesh* mesh, int32_t K, const double* center, double* out, void* workspace,
                           size_t workspace_bytes, void* stream);
pat_status pat_moments_finish(int64_t n_nodes, double n_samples, int32_t which, double* v, void* stream);

/*
 * Counter-based N(0,1) draws used when pat_cgls_begin / pat_rto_sample get NULL
 * eta or xi: out[e*K + k] for e < n_elem, k < K (device, double).  stream_id 0
 * gives eta (e = flat index n*N_obs + d), 1 gives xi (e = node).  Definition:
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) output i of seed s is
 * mix(s + i * 0x9E3779B97F4A7C15); with c = ((k << 1 | stream_id) << 40) | e,
 * u1 = (out(2c+1) >> 11 + 1) 2^-53, u2 = (out(2c+2) >> 11) 2^-53 and
 * z = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, cosine branch).  A sample's
 * draws depend on its index k and the seed only, not on K.
 */
pat_status pat_draw_normals(uint64_t seed, int32_t stream_id, int64_t n_elem, int32_t K, double* out,
                            void* stream);

/*
 * Whittle-Matern prior (Section 4.1.2, eq. matern-cov-op; Section 6.4) for FP32
 * meshes: the prior field p0 = P T z with z ~ N(0, I) on a periodic box grid of
 * n_grid^3 points, T = F^{-1} diag(sqrt(S)) F (F the unitary 3D DFT),
 * S(k) = (1/ell^2 + |2 pi k|^2)^{-(s + 3/2)} at the DFT frequencies scaled so
 * that the grid field's marginal variance is sigma^2 (the normalisation Z), and
 * P trilinear interpolation from the grid to the mesh nodes.  The box is
 * [box_lo[c], box_lo[c] + box_len) on every axis c, grid point j at
 * box_lo + j box_len / n_grid; every node must lie inside.  The paper's
 * covariance operator is followed (its Section 6.4 SPDE applies the cubed
 * operator to p0, which would square it).  Grid fields are K-stacked [G][K],
 * G = n_grid^3, grid point (ix, iy, iz) at (ix n_grid + iy) n_grid + iz.
 *
 *   pat_matern_create   builds sqrt(S) (FP32), P (8 grid points and FP32
 *       weights per node) and P^T as a grid -> node list of the same weights.
 *       n_grid a power of two in [8, 256].  Errors: PAT_EINVAL (arguments, a
 *       node outside the box), PAT_EUNSUPPORTED (FP64 mesh), PAT_ENOMEM.
 *   pat_matern_workspace_bytes  device workspace of the calls below for K
 *       samples: an RTO workspace of the mesh followed by the latent fields.
 *   pat_matern_apply  op 0: out = T in (grid -> grid); 1: out = P in (grid ->
 *       nodes [N][K]); 2: out = P^T in (nodes -> grid); 3: out = P T in (grid ->
 *       nodes).  FP32 device fields.
 *   pat_rto_sample_matern  K RTO samples in the latent space (Section 6.4):
 *       n_iter CGLS iterations from z = 0 on min ||(G P T z - y_obs)/sigma -
 *       eta||^2 + ||z - xi||^2, every inner product, norm, scalar and the
 *       iterate z in FP64.  eta device [N_T][N_obs][K] float or NULL (library
 *       draws, stream 0); xi device [G][K] float or NULL (library draws of
 *       stream 1 at element = grid point); both keyed by the mesh's first
 *       sample index as in pat_rto_sample.  Outputs (device double, each may be
 *       NULL): z_samples [G][K]; p_samples [N][K] = P T z; mean, stdev [N] of
 *       the nodal samples (eq. ergodic).  PAT_ENUMERIC is reported by
 *       pat_rto_status(mesh, K, workspace, stream) as for the other solvers.
 *   pat_matern_layout  byte offsets into the workspace of the latent CGLS
 *       state after pat_rto_sample_matern: off[0] z [G][K] double, off[1]
 *       direction d [G][K] float, off[2] latent residual block [G][K] float,
 *       off[3] s = A^T r [G][K] float, off[4] gamma [K] double, off[5] data
 *       residual block [N_T][N_obs][K] float, off[6] status word.  s is
 *       overwritten when p_samples, mean or stdev was requested.
 */
typedef struct pat_matern pat_matern;
pat_status pat_matern_create(const pat_mesh* mesh, int32_t n_grid, const double* box_lo /* [3] */, double box_len,
                             double ell, double s, double sigma, pat_matern** out);
pat_status pat_matern_destroy(pat_matern* prior);
pat_status pat_matern_workspace_bytes(const pat_mesh* mesh, const pat_matern* prior, int32_t K, size_t* bytes);
pat_status pat_matern_apply(const pat_mesh* mesh, const pat_matern* prior, int32_t op, const float* in, int32_t K,
                            float* out, void* workspace, size_t workspace_bytes, void* stream);
pat_status pat_matern_layout(const pat_mesh* mesh, const pat_matern* prior, int32_t K, size_t* offsets /* [7] */);
pat_status pat_rto_sample_matern(const pat_mesh* mesh, const pat_matern* prior, const void* y_obs, double sigma,
                                 int32_t K, int32_t n_iter, const void* eta, const float* xi, uint64_t seed,
                                 double* z_samples, double* p_samples, double* mean, double* stdev, void* workspace,
                                 size_t workspace_bytes, void* stream);

/*
 * Derivatives of a data misfit L(p0, theta) whose cotangent with respect to
 * Y = G(theta) p0 is Yhat (e.g. Yhat = G p0 - y_obs for 1/2 ||G p0 - y_obs||^2),
 * with theta_e = c_e^2 the per-tetrahedron squared sound speed of the mesh:
 *   g_c2     device [n_tets] double: dL/dtheta_e summed over the K samples,
 *            -dt^2 sum_m u_m|_e^T K_e^0 x_{m-1}|_e with x the forward states and
 *            u the transposed states (Section 5.1 recursion; K_e^0 the c = 1
 *            element stiffness of Section 3);
 *   p0_grad  device [N][K] real or NULL: G^T Yhat (dL/dp0).
 * The forward trajectory is recomputed from L = ceil(sqrt(N_T)) checkpoints, so
 * the call costs about two forward sweeps, one transposed sweep (the mesh's
 * tuned step kernels for K) and one element pass per checkpoint segment.
 * p0 device [N][K] real; Yhat device [N_T][N_obs][K] real;
 * workspace >= pat_workspace_bytes(mesh, 3, K) (checkpoints, L + 2 transposed
 * states, L recomputed states, four state buffers, g).  The first call with a
 * given (p0, Yhat, g_c2, p0_grad, workspace, K) captures the whole evaluation
 * into a CUDA graph on the mesh's capture stream; later calls with the same
 * buffers replay it on `stream` (new contents, same addresses).  Graphs are
 * dropped when a variant, the wait budget or c^2 changes; with
 * PAT_MESH_NO_GRAPHS, or while `stream` is being captured, the kernels are
 * launched directly.  Calls on one mesh from several host threads at once are
 * not supported.
 */
pat_status pat_grad_c2(const pat_mesh* mesh, const void* p0, const void* Yhat, int32_t K, double* g_c2,
                       void* p0_grad, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Autotuning of the time-step kernels for K stacked samples on this mesh:
 * every variant (samples per thread V in {8, 4, 2, 1} that divides K; for FP32
 * split coefficients a packed kernel doing two samples per fma.rn.f32x2 with
 * row chunks of 2, 4 or 8 entries; a generic kernel with the row metadata
 * staged in shared memory or read directly) runs n_probe forward and
 * n_probe transposed steps on zeroed buffers of `workspace` (an RTO workspace,
 * >= pat_workspace_bytes(mesh, 2, K); its CGLS state is overwritten), timed
 * with CUDA events on `stream`.  The fastest variant per direction is used by
 * every later call with this K on this mesh.  table (host, may be NULL)
 * receives up to 256 entries {direction 0 fwd / 1 adj, V, staged, packed, chunk,
 * min_blocks (resident blocks per SM asked of the compiler), early (own values
 * loaded before the row walk), zorder (rows processed in Z-order of the node
 * coordinates), big_blocks (1024-thread blocks), prefetch (0: off; n: each block
 * first asks L2 to prefetch, by bulk prefetch, the state rows and row metadata
 * of the rows n resident waves ahead), persistent (fixed-width kernel only:
 * 1 = a grid of resident blocks whose warps each walk 32-thread chunks with a
 * stride of the grid's warps, prefetch then counting strides; 2 = each block
 * walks one contiguous slab of chunks in order, prefetch counting its
 * iterations; 3 = as 1, with each warp's next chunk's row metadata copied
 * into shared memory by cp.async while it processes the current one, V = 8
 * and K / V >= 4 only, else 1), pdl (persistent only:
 * launched as a programmatic dependent of the previous step), wide_loads
 * (persistent, V = 8: each thread's 8 samples read and written by one 256-bit
 * access), l2_hints (persistent grid-stride, V = 8, 128-bit: the new state
 * and the row metadata stored / loaded with L2 evict_last priority, the last
 * read of x_{s-1} with evict_first), gather_batch (persistent grid-stride,
 * V = 8, 128-bit: source rows loaded per batch before any is used; 0 = 4
 * with the row's metadata loaded up front; 8 runs at 2 blocks per SM; 2 or 4
 * load each batch's metadata with it, with min_blocks 1 (4 per SM), 5 or 6),
 * us per step};
 * *n_entries the number of variants timed.  Synchronises the stream.
 */
typedef struct {
  int32_t direction, V, staged, packed, chunk, min_blocks, early, zorder, big_blocks, prefetch, persistent, pdl,
      wide_loads, l2_hints, gather_batch, tail_serial, own_async, prefetch_meta, dyn_chunks;
  double us_per_step;
} pat_tune_entry;
pat_status pat_autotune(pat_mesh* mesh, int32_t K, void* workspace, size_t workspace_bytes, int32_t n_probe,
                        pat_tune_entry* table, int32_t* n_entries, void* stream);

/* Use the given variant (fields as in pat_tune_entry) for direction 0
 * (forward) or 1 (transposed) and K samples on this mesh.  PAT_EINVAL if the
 * variant does not exist for this K and precision.  Every variant gives
 * bit-identical results.  packed selects the kernel family:
 *   2  the tile-staged kernel: each 32-row tile's source rows staged in shared
 *      memory by bulk asynchronous copies (bounded mbarrier waits);
 *   3  the 8-slot fixed-width kernel (the rows' first 8 entries at fixed
 *      positions, the rest in an overflow list);
 *   5  the 16-slot fixed-width kernel for meshes with rows wider than 8 entries
 *      (the full P1 graph), quad-interleaved slots, persistent, V = 8 (or V = 1
 *      for K = 1); 6 the same reading a row-major copy of the slots (V = 8);
 *   7  row pairs (the union of two rows' sources gathered once);
 *   8  row quads (K = 64: the union of four rows' sources gathered once).
 * Fields of the 16-slot kernels: gather_batch 4 or 8 source rows per round;
 * early = each round's columns loaded with it; big_blocks = 1024-thread blocks;
 * min_blocks 3 with rounds of 8; tail_serial = a row's entries past the round
 * loop and its boundary corrections walked one at a time instead of in pairs;
 * own_async = the row's own x_s and x_{s-1} copied to shared memory while its
 * gathers run (1: by cp.async, each thread its own values; 2, packed 6 with
 * K / 8 dividing 32: by two bulk asynchronous copies per warp of its rows,
 * completing on an mbarrier whose wait is bounded by the mesh's wait budget,
 * pat_mesh_set_wait_cycles, PAT_ETIMEOUT through pat_rto_status when it runs
 * out; 3, packed 6 with rounds of 4 and no other option: x_{s-1} alone by
 * cp.async, x_s read from L1 after the row's diagonal gather); prefetch_meta = each warp asks L1 for its next chunk's row metadata
 * (packed 6) or for the quad's coefficient lines (packed 5, K = 64);
 * dyn_chunks (packed 6, three-level form) = the warps' 32-thread chunks handed
 * out in row order by an atomic counter (kept in the workspace's fourth state
 * buffer) instead of the grid stride; wide_loads (packed 6 with early) = the
 * row metadata in 256-bit loads (for packed 3: 8 contiguous samples per
 * 256-bit load). */
pat_status pat_select_variant(pat_mesh* mesh, int32_t K, int32_t direction, const pat_tune_entry* variant);

/*
 * Live timing of the hot kernels, for benchmarks.  While enabled on a mesh,
 * every forward and transposed time loop run by calls on that mesh (pat_forward,
 * pat_adjoint and the loops inside the CGLS calls) is bracketed by two CUDA
 * events recorded on the launching stream, and every kernel launch is counted.
 * pat_profile_enable(mesh, 1) resets the counters; pat_profile_read
 * synchronises the device and returns the sums.  fwd_ms / adj_ms are the
 * summed event times of the loops (launch gaps included); *_launches count the
 * step kernels inside them; total_launches counts every kernel of the library.
 * Not thread-safe across concurrent calls on one mesh.
 */
typedef struct {
  double fwd_ms, adj_ms;
  int64_t fwd_loops, adj_loops;
  int64_t fwd_launches, adj_launches;
  int64_t total_launches;
} pat_profile;
pat_status pat_profile_enable(pat_mesh* mesh, int32_t enable);
pat_status pat_profile_read(pat_mesh* mesh, pat_profile* out);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* pat_last_error(void);

/* Library version string. */
const char* pat_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PAT_H */
