/*
 * snsweep.h -- C ABI of a GB300 (sm_103a) library for the graph-based S_N transport sweep on
 * curved high-order meshes (Haut, Maginot, Tomov, Southworth, Brunner, Bailey, "An Efficient
 * Sweep-based Solver for the S_N Equations on High-Order Meshes").
 *
 * What it computes (paper sections in brackets):
 *   steady mono-energetic S_N equation with isotropic scattering and inflow boundary values
 *   [Sec. 2, eq. 1-2]; upwind DG of order p on Q_r curved quadrilaterals/hexahedra [Sec. 2,
 *   eqs. 3-16]; per-direction element dependency graph with unity / face / sigma-inverse-face
 *   edge weights, made acyclic by a minimum-weight feedback arc set (exact on small SCCs,
 *   Eades-Lin-Smyth on large ones) [Sec. 3]; lagged transport sweeps inside source iteration
 *   [Sec. 3, eqs. 17-21].
 *
 * Conventions for every call:
 *   - Every call returns sn_status; SN_OK = 0.  On failure sn_last_error(ctx) holds a message.
 *     No call throws or aborts.  A failed call leaves previously accepted state unchanged
 *     unless stated otherwise.
 *   - All arrays are caller-owned, dense, row-major (C order), element indices 64-bit where
 *     the type says so.  The library copies what it keeps; it never frees caller memory.
 *   - Data pointers may be host or device pointers (CUDA unified addressing decides, per
 *     pointer, via cudaPointerGetAttributes).  Host buffers are staged through the context's
 *     device buffers; device buffers are used in place.
 *   - All device work is ordered on the context's CUDA stream (given at creation).  Calls that
 *     return host-visible results synchronise that stream before returning.
 *   - One context = one problem on one GPU.  A context is not thread-safe.
 *
 * Mesh conventions (sn_set_mesh):
 *   reference element [0,1]^dim; control points of the Q_r map on the equispaced reference
 *   nodes a/r, local index m = a0 + (r+1) a1 (+ (r+1)^2 a2) [Sec. 2, eq. 1].
 *   Local face f = 2*axis + side (side 0: xi_axis = 0).  A face's coordinates (s0[, s1]) are
 *   the remaining reference axes in increasing order.  orient[e][f] maps e's face
 *   coordinates to the neighbour's: swap (bit 2) first, then s -> 1 - s on the first (bit 0)
 *   and second (bit 1) result.
 *   DG unknowns: tensor Gauss-Lobatto-Legendre nodes of order p, node index as above with p.
 *   Face node (i, j) of face f is the volume node with index i along s0, j along s1.
 *   Boundary faces are numbered in increasing (element, local face) order.
 */
#ifndef SNSWEEP_H
#define SNSWEEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_ctx sn_ctx;

typedef enum {
  SN_OK = 0,
  SN_EINVAL = 1,          /* bad argument (null pointer, size out of range, non-finite value)   */
  SN_ENOMEM = 2,          /* device or host allocation failed                                    */
  SN_ECUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error string)     */
  SN_ETIMEOUT = 4,        /* a bounded device wait gave up (device error word set)              */
  SN_ENOTCONVERGED = 5,   /* source iteration hit max_iter before reaching tol                  */
  SN_EMESH = 6,           /* invalid mesh: det J <= 0, inconsistent connectivity                */
  SN_ESTATE = 7           /* call out of order (e.g. sweep before build_graph)                  */
} sn_status;

enum { SN_WEIGHT_UNITY = 0, SN_WEIGHT_FACE = 1, SN_WEIGHT_SIGINVFACE = 2 };
enum { SN_PREC_FP64 = 0, SN_PREC_MIXED = 1, SN_PREC_MIXED_DS = 2, SN_PREC_FP64_INV = 3, SN_PREC_DS_INV = 4 };
enum { SN_LAUNCH_LEVELS = 0, SN_LAUNCH_DATAFLOW = 1 };

typedef struct {
  int64_t n_arcs;          /* arcs e' -> e over all directions                                 */
  int64_t n_removed;       /* arcs removed (lagged) over all directions                        */
  int64_t n_scc;           /* non-trivial SCCs over all directions                             */
  int32_t max_scc;         /* largest SCC size                                                 */
  int32_t max_level;       /* largest sweep level (levels are 0-based)                          */
  int64_t n_mixed_faces;   /* (face side, direction) pairs whose inflow region is partial      */
  double ms_geometry;      /* device time of the geometric-factor stage                        */
  double ms_weights;       /* device time of the edge-weight stage                              */
  double ms_fas;           /* host time of SCC + feedback-arc-set                               */
  double ms_levels;        /* device time of level scheduling + work lists                      */
} sn_graph_stats;

typedef struct {
  int32_t iters;           /* source iterations performed                                      */
  int32_t converged;       /* 1 if ||phi_{l+1}-phi_l||_inf / ||phi_{l+1}||_inf < tol was reached */
  double residual;         /* last relative scalar-flux change                                  */
  double ms_total;         /* wall time of the iteration loop (host clock)                     */
} sn_si_stats;

/* Create a context on CUDA device `device`, ordering all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the context. */
sn_status sn_create(sn_ctx** out, int device, void* cuda_stream);

/* Destroy a context and free its device memory.  Accepts NULL. */
void sn_destroy(sn_ctx* ctx);

/* Last error message of this context ("" if none).  Owned by the context. */
const char* sn_last_error(const sn_ctx* ctx);

/* Mesh [Sec. 2, 'Discrete representation of the HO mesh'].
 *   dim 2 or 3; geometry order r in 1..3; n_elem >= 1.
 *   ctrl      [n_elem][(r+1)^dim][dim] control points (x_{e,m} of eq. 1).
 *   face_nbr  [n_elem][2 dim] neighbour element or -1 on the domain boundary.
 *   nbr_face  [n_elem][2 dim] the neighbour's local face (ignored where face_nbr = -1).
 *   orient    [n_elem][2 dim] orientation code (see header comment; 0..1 in 2D, 0..7 in 3D).
 * Errors: SN_EINVAL (sizes, codes), SN_EMESH (neighbour relation not symmetric).
 * Resets everything computed from an earlier mesh. */
sn_status sn_set_mesh(sn_ctx* ctx, int dim, int64_t n_elem, int r, const double* ctrl,
                      const int64_t* face_nbr, const int32_t* nbr_face, const int32_t* orient);

/* Simplex mesh [Sec. 2: simplicial elements]: triangles (dim = 2, P_r geometry) or straight-sided
 * tetrahedra (dim = 3, r = 1 only; SN_EINVAL otherwise).
 * Triangles: as sn_set_mesh with three faces per element.  Reference triangle {xi, eta >= 0,
 * xi + eta <= 1}, vertices v0 = (0,0), v1 = (1,0), v2 = (0,1), counterclockwise faces f0 = v0 v1,
 * f1 = v1 v2, f2 = v2 v0, each with the coordinate s in [0,1] from its first vertex to its second.
 *   ctrl      [n_elem][(r+1)(r+2)/2][2] control points in the node order v0, v1, v2, the r - 1
 *             interior nodes of f0, f1, f2 (at s = a/r, increasing s), then (r = 3) the centroid.
 *   face_nbr, nbr_face, orient [n_elem][3]; orient 1 when the neighbour runs the shared face in
 *   the opposite direction (counterclockwise neighbours always do), 0 when in the same.
 * The DG basis is then P_p (sn_set_discretization, p = 1..3, (p+1)(p+2)/2 unknowns) on the same
 * node pattern with the face nodes at the Gauss-Lobatto-Legendre positions of order p; volume
 * integrals use the collapsed Gauss rule (xi = u, eta = v (1 - u)) with p + r points per
 * direction.
 * Tetrahedra: four faces per element.  Reference vertices v0 = (0,0,0), v1 = (1,0,0),
 * v2 = (0,1,0), v3 = (0,0,1); face f is opposite vertex f with the vertex triples (v1 v2 v3),
 * (v0 v3 v2), (v0 v1 v3), (v0 v2 v1) = (A, B, C), ordered so that (B - A) x (C - A) points out
 * of the element, and face coordinates (s, t) the barycentrics of B and C.
 *   ctrl      [n_elem][4][3] vertices (positive volume).
 *   face_nbr, nbr_face, orient [n_elem][4]; orient k in 0..5: our face vertex j is the
 *   neighbour's face vertex pi_k(j), pi = (0 1 2), (1 2 0), (2 0 1), (0 2 1), (2 1 0), (1 0 2).
 * The DG basis is P_1 (4 unknowns: the vertices) or P_2 (10: the vertices, then the midpoints of
 * the edges v0v1, v1v2, v2v0, v0v3, v1v3, v2v3); volume integrals use the collapsed Gauss rule
 * (x = u, y = v (1 - u), z = w (1 - u)(1 - v)) with p + 2 points per direction, face integrals
 * the collapsed triangle rule with p + 1.  A flat face is wholly inflow or wholly outflow for
 * every direction, so no face is split.
 * Simplex problems are swept by the stored-inverse forms (SN_PREC_FP64_INV, SN_PREC_DS_INV); the
 * other forms, diffusion acceleration, the flux predictor and batches return SN_EINVAL. */
sn_status sn_set_mesh_simplex(sn_ctx* ctx, int dim, int64_t n_elem, int r, const double* ctrl,
                              const int64_t* face_nbr, const int32_t* nbr_face, const int32_t* orient);

/* DG order p: 1..3 in 2D, 1..2 in 3D (N = (p+1)^dim <= 32 unknowns per element) and, for hexahedra,
 * the number K of sub-squares per face axis of the composite face rule (1..4; ignored in 2D and for
 * tetrahedra, whose flat faces need no composite rule).
 * Quadrature: volume n_v = p + ceil(dim r / 2) Gauss-Legendre points per axis, faces
 * n_f = p + r; 2D faces are split at the sign changes of Omega.n [Sec. 2, last paragraph].
 * Simplex meshes use the collapsed rules of sn_set_mesh_simplex.
 * Errors: SN_ESTATE before sn_set_mesh; SN_EINVAL for p or K out of range. */
sn_status sn_set_discretization(sn_ctx* ctx, int p, int face_subdiv);

/* Angular quadrature {(w_d, Omega_d)} [Sec. 2, after eq. 2]: omega [n_dir][3] unit vectors
 * (2D problems use the first two components), w [n_dir] > 0.  n_dir in 1..4096. */
sn_status sn_set_quadrature(sn_ctx* ctx, int n_dir, const double* omega, const double* w);

/* Level-symmetric S_N set [Sec. 2, after eq. 2: omega_d > 0, sum omega_d = 4 pi; the paper's
 * results use level-symmetric S2 / S4 sets].  Needs no context and no GPU.
 *   N in {2, 4, 6, 8, 12}; dim 3: all eight octants, N(N+2) directions, weights (pi/2) x the
 *   octant point weight; dim 2: the four octants with Omega_z > 0 (the problem does not depend
 *   on z, each direction stands for its mirror image), N(N+2)/2 directions, weights pi x the
 *   octant point weight.  Construction: mu_i^2 = mu_1^2 + (i-1) 2 (1 - 3 mu_1^2)/(N-2); octant
 *   points = level-index triples (i, j, k), i + j + k = N/2 + 2 (i fastest, then j, then k),
 *   weighted by the published 7-digit class weights normalised to sum 1 per octant; octants in
 *   sign order (+,+,+), (-,+,+), (+,-,+), (-,-,+), then the same with Omega_z < 0.
 *   *n_dir receives the number of directions.  omega [n_dir][3] and w [n_dir] are host arrays
 *   written when both are non-NULL (both NULL: size query only).
 * Errors: SN_EINVAL (N not tabulated, dim not 2 or 3, n_dir NULL, exactly one of omega / w NULL). */
sn_status sn_quadrature_level_symmetric(int N, int dim, int* n_dir, double* omega, double* w);

/* Materials and sources [Sec. 2, eqs. 1, 8].
 *   sigma_t, sigma_s [n_elem] element-constant cross sections (sigma_t > 0, sigma_s >= 0).
 *   q        [n_elem][N] nodal isotropic source, or NULL (= 0).
 *   q_dir    [n_dir][n_elem][N] nodal direction-dependent source added to q, or NULL.
 *   psi_inc  [n_dir][n_bdr_faces][N_f] nodal incident angular flux on boundary faces
 *            (face-node order of the owning element), or NULL (vacuum).
 * Requires mesh, discretization and quadrature. */
sn_status sn_set_materials(sn_ctx* ctx, const double* sigma_t, const double* sigma_s,
                           const double* q, const double* q_dir, const double* psi_inc);

/* Number of boundary faces (valid after sn_set_mesh). */
int64_t sn_num_boundary_faces(const sn_ctx* ctx);

/* Build the sweep graph [Sec. 3]: geometric factors, upwind arcs and weights, strongly connected
 * components and a minimum-weight feedback arc set per component (exact for components of at most
 * exact_max <= 16 vertices, Eades-Lin-Smyth above), sweep levels -- all on the device; the work
 * lists are assembled on the host from the levels.  ms_fas in the stats is the wall time of the
 * component and feedback-arc-set stage.
 * weighting: SN_WEIGHT_UNITY / _FACE / _SIGINVFACE.  stats may be NULL.
 * Errors: SN_ESTATE (missing inputs), SN_EMESH (det J <= 0 somewhere). */
sn_status sn_build_graph(sn_ctx* ctx, int weighting, int exact_max, sn_graph_stats* stats);

/* Sweep schedule (no counterpart in the paper, which sweeps serially; both schedules compute
 * the same result, since any topological order of the kept graph does [Sec. 3]).
 *   SN_LAUNCH_LEVELS  : one kernel launch per wavefront level, replayed from a CUDA graph.
 *   SN_LAUNCH_DATAFLOW: one persistent launch per sweep; warps take (element, direction) pairs
 *                       from a queue in level order and wait only for the completion flags of
 *                       their kept upwind neighbours (bounded polling: a wait that exceeds its
 *                       limit makes the sweep return SN_ETIMEOUT instead of hanging).
 *   blocks_per_sm: CTAs of 128 threads per SM for the dataflow grid (0 = occupancy limit).
 * May be called at any time; applies to later sweeps. */
sn_status sn_set_launch(sn_ctx* ctx, int mode, int blocks_per_sm);

/* Poll limit of one dependency wait of the dataflow schedule (no counterpart in the paper):
 * a warp that has polled an upwind completion flag `polls` times without seeing it set stops
 * waiting, sets the sweep's device error word and lets every other wait and the work queue stop
 * early; the kernel then returns normally and the sweep call reports SN_ETIMEOUT (its results
 * are not valid).  0 restores the default of 2^20 polls (~0.1-1 s); small values make a wait
 * give up on purpose, which is how the timeout path is tested.  Applies to later sweeps of the
 * context and of batches created afterwards.  Errors: SN_EINVAL (polls < 0). */
sn_status sn_set_spin_limit(sn_ctx* ctx, int64_t polls);

/* Autotuner (no counterpart in the paper): runs two warm-up source iterations and then five
 * timed ones of every candidate schedule -- per-level launches, or the dataflow launch with 1, 2,
 * 3, 4 or the maximum resident CTAs per SM -- keeps the one with the fastest sweep via
 * sn_set_launch and resets the iteration state (sn_si_begin(ctx, NULL)).  mode_out /
 * blocks_per_sm_out may be NULL. */
sn_status sn_autotune(sn_ctx* ctx, int precision, int* mode_out, int* blocks_per_sm_out);

/* Stored local inverses of the stored-inverse forms (no counterpart in the paper, which factors
 * during the sweep): the left-hand side of eq. 21 for direction d and element e, G + F_e + M_t,
 * is the same in every source iteration, so its inverse is formed once, by Gauss-Jordan
 * elimination with partial pivoting in FP64, for all (direction, element) pairs in one launch,
 * together with the pair's inflow face blocks (the coupling matrices of its upwind traces), and
 * kept in context-owned device buffers: n_dir * n_elem * N * N entries for the inverses and
 * Nf * Nf per inflow face for the blocks, 8 bytes each.  precision SN_PREC_FP64_INV stores them
 * as doubles, SN_PREC_DS_INV as (hi, lo) FP32 pairs of the same FP64 values.
 * sn_prepare_inverse (re)forms them now in the layout of `precision`; *ms (may be NULL) receives
 * the device time of that launch.  Otherwise the first sweep of a stored-inverse form forms them
 * (and a sweep of the other stored-inverse form forms them again).  Valid after sn_build_graph;
 * new materials or a new graph drop them.  sn_release_inverse frees the buffers.
 * Errors: SN_ESTATE (no graph), SN_EINVAL (precision not a stored-inverse form), SN_ENOMEM (the
 * buffers do not fit in device memory). */
sn_status sn_prepare_inverse(sn_ctx* ctx, int precision, float* ms);
sn_status sn_release_inverse(sn_ctx* ctx);

/* Copy the graph out (valid after sn_build_graph).
 *   *n_removed receives the number of removed arcs; if removed != NULL and cap >= that number,
 *   removed [k][3] receives (direction, e, e') rows sorted ascending: e depends on e' and the
 *   dependency is lagged.  levels [n_dir][n_elem] (may be NULL) receives the sweep level of
 *   every (direction, element).  Returns SN_EINVAL if cap is too small (n_removed still set). */
sn_status sn_get_graph(sn_ctx* ctx, int64_t* n_removed, int32_t* removed, int64_t cap,
                       int32_t* levels);

/* One lagged sweep over all directions [eq. 21]:
 *   for each direction, element by element in level order, solve
 *   (G + F_e + M_t) psi_e = M (q + q_dir + sigma_s phi_in / (4 pi)) + boundary inflow
 *                           + sum_{kept e'} Fbar psi_new,e' + sum_{removed e'} Fbar psi_old,e'.
 *   phi_in   [n_elem][N]          scalar flux of the previous iterate.
 *   psi_old  [n_dir][n_elem][N]   previous angular flux (read for removed arcs only).
 *   psi_new  [n_dir][n_elem][N]   output; must not alias psi_old.
 *   precision SN_PREC_FP64: all local algebra in FP64.  SN_PREC_MIXED: FP32 assembly and LU,
 *   one refinement step whose residual is formed in FP64.  SN_PREC_MIXED_DS: as SN_PREC_MIXED
 *   but the matrix row and the residual are formed in double-single arithmetic (pairs of FP32
 *   values with error-free products and sums, ~2^-48 relative) on the FP32 pipe; only the
 *   right-hand side and the final sum are FP64.  SN_PREC_FP64_INV: FP64; the inverse of every
 *   (direction, element) matrix G + F_e + M_t, which does not change between iterations, and
 *   its inflow face blocks are formed once (see sn_prepare_inverse) and kept in device memory;
 *   a sweep forms the right-hand side and applies the inverse.  SN_PREC_DS_INV: the same stored
 *   FP64 values kept as (hi, lo) FP32 pairs, right-hand side and application in double-single
 *   arithmetic on the FP32 pipe.
 * Synchronises the stream before returning when any pointer is a host pointer. */
sn_status sn_sweep(sn_ctx* ctx, const double* phi_in, const double* psi_old, double* psi_new,
                   int precision);

/* Scalar-flux moment [eq. 2] and relative change:
 *   phi_out = sum_d w_d psi_d;  *residual = ||phi_out - phi_prev||_inf / ||phi_out||_inf
 *   (phi_prev may be NULL: treated as 0).  Also refreshes the context's scattering source for
 *   the next sweep.  Synchronises the stream (the residual is a host value). */
sn_status sn_moment(sn_ctx* ctx, const double* psi, const double* phi_prev, double* phi_out,
                    double* residual);

/* Source iteration [eq. 18 with the lagged sweep of eq. 21] from phi0 (NULL = 0) and
 * psi = 0 until the relative scalar-flux change drops below tol or max_iter sweeps ran.
 *   phi_out [n_elem][N], psi_out [n_dir][n_elem][N] (either may be NULL).
 *   history [history_cap] receives the residual of each iteration (may be NULL).
 * Returns SN_ENOTCONVERGED (results still written) if tol was not reached. */
sn_status sn_source_iterate(sn_ctx* ctx, double tol, int max_iter, int precision,
                            const double* phi0, double* phi_out, double* psi_out,
                            sn_si_stats* stats, double* history, int history_cap);

/* Resident source iteration, one step at a time (the loop of sn_source_iterate, exposed so a
 * caller can time or interleave single iterations).
 *   sn_si_begin : phi <- phi0 (NULL = 0), psi <- 0, scattering source from phi.
 *   sn_si_step  : one lagged sweep over all directions [eq. 21] into the context's other psi
 *                 buffer, then the fused scalar-flux moment + scattering-source update +
 *                 residual [eqs. 2, 18].  *residual (may be NULL) receives
 *                 ||phi_{l+1} - phi_l||_inf / ||phi_{l+1}||_inf; *ms_sweep (may be NULL) the device
 *                 time of the sweep launches measured with CUDA events on the context's stream.
 *                 Synchronises the stream.
 *   sn_si_result: copy the current phi [n_elem][N] and psi [n_dir][n_elem][N] out (either may be
 *                 NULL; host or device pointers). */
sn_status sn_si_begin(sn_ctx* ctx, const double* phi0);
sn_status sn_si_step(sn_ctx* ctx, int precision, double* residual, float* ms_sweep);
sn_status sn_si_result(sn_ctx* ctx, double* phi_out, double* psi_out);

/* Volume quadrature points and L2 errors (for manufactured solutions; no counterpart in the
 * paper's solver, whose Sec. 4.1 reports such errors).  Valid after sn_set_discretization.
 *   sn_num_volume_points: Q, the number of volume quadrature points per element (0 before).
 *   sn_volume_points: xq [n_elem][Q][dim] receives their physical positions x_e(xi_q) [eq. 1].
 *   sn_l2_error: *err = sqrt(sum_e sum_q w_q |J_e(xi_q)| (sum_n u_n(xi_q) phi[e][n] - exact_q[e][q])^2),
 *     phi [n_elem][N] a nodal field (e.g. the scalar flux), exact_q [n_elem][Q] the reference
 *     field's values at the points of sn_volume_points.
 * Host or device pointers.  Errors: SN_ESTATE (no discretization), SN_EINVAL (null array). */
int32_t sn_num_volume_points(const sn_ctx* ctx);
sn_status sn_volume_points(sn_ctx* ctx, double* xq);
sn_status sn_l2_error(sn_ctx* ctx, const double* phi, const double* exact_q, double* err);

/* ---- Batches: many independent problems in one persistent launch (no counterpart in the
 * paper; each problem is the method above).  The problems are contexts of the same dimension
 * on the same device whose graphs are built; they may differ in mesh size, geometry order, DG
 * order, direction set and materials.  A batch step sweeps every problem in one launch
 * (dataflow schedule: warps take (problem, level, pairs) tasks from a queue ordered by level
 * across problems; or one launch per level), then one launch forms every problem's scalar flux,
 * scattering source and residual; the step is replayed from a CUDA graph.  The batch owns only
 * its tables; flux buffers stay in the contexts (sn_si_result on a context reads its state after
 * batch steps).  Do not interleave single-context steps of a member with batch steps. */
typedef struct sn_batch sn_batch;
sn_status sn_batch_create(sn_batch** out, int n_problems, sn_ctx* const* problems, void* cuda_stream);
void sn_batch_destroy(sn_batch* batch);
const char* sn_batch_last_error(const sn_batch* batch);
/* Element-direction updates of one sweep over all problems. */
int64_t sn_batch_updates_per_sweep(const sn_batch* batch);
/* Schedule of later steps, as sn_set_launch (default: dataflow, maximum resident CTAs). */
sn_status sn_batch_set_launch(sn_batch* batch, int mode, int blocks_per_sm);
/* Autotuner over the same candidates as sn_autotune; resets the iteration state. */
sn_status sn_batch_tune(sn_batch* batch, int precision, int* mode_out, int* blocks_per_sm_out);
/* psi <- 0 and phi <- phi0[k] (host or device [E_k][N_k]; phi0 or phi0[k] NULL = 0) in every
 * problem. */
sn_status sn_batch_si_begin(sn_batch* batch, const double* const* phi0);
/* One source iteration of every problem; residuals [n_problems] (may be NULL) receive each
 * problem's relative scalar-flux change; *ms_sweep (may be NULL) the device time of the step.
 * With SN_PREC_FP64_INV the first step forms every member's stored inverses that are missing
 * (sn_prepare_inverse) before it sweeps. */
sn_status sn_batch_si_step(sn_batch* batch, int precision, double* residuals, float* ms_sweep);
/* Steps until every problem's relative change is below tol; iters [n] receives the first
 * iteration at which each problem reached it (-1 if never), residuals [n] the last change.
 * SN_ENOTCONVERGED if some problem did not reach tol in max_iter steps. */
sn_status sn_batch_source_iterate(sn_batch* batch, double tol, int max_iter, int precision, int32_t* iters,
                                  double* residuals, double* ms_total);

/* ---- Learned flux predictor (this project's addition; the paper has none).  A per-element
 * MLP -- x -> tanh(x W1 + b1) -> tanh(. W2 + b2) -> . W3 + b3, width 64, BF16 weights, FP32
 * accumulation, trained by Adam on the device -- supplies the initial scalar flux of source
 * iteration and a post-sweep correction; plain source iteration is the fallback and the arbiter
 * of convergence.  Packed parameters: W1 [n_in][64], b1 [64], W2 [64][64], b2 [64],
 * W3 [64][n_out], b3 [n_out] (FP32 masters). */
#define SN_FEATURES 16
typedef struct sn_mlp sn_mlp;
/* n_in, n_out in 1..64; Glorot-uniform weights from a seeded mt19937_64, zero biases. */
sn_status sn_mlp_create(sn_mlp** out, int device, void* cuda_stream, int n_in, int n_out, uint64_t seed);
void sn_mlp_destroy(sn_mlp* mlp);
int64_t sn_mlp_num_params(const sn_mlp* mlp);
/* get (may be NULL) receives the FP32 parameters; set (may be NULL) replaces them (and resets
 * the Adam state).  Host or device pointers. */
sn_status sn_mlp_params(sn_mlp* mlp, float* get, const float* set);
/* y [rows][n_out] = MLP(x [rows][n_in]). */
sn_status sn_mlp_forward(sn_mlp* mlp, int64_t rows, const float* x, float* y);
/* loss = sum (y - t)^2 / (2 rows n_out) and its gradient grad [n_params] (may be NULL). */
sn_status sn_mlp_grad(sn_mlp* mlp, int64_t rows, const float* x, const float* target, float* loss, float* grad);
/* Adam (lr, 0.9, 0.999, 1e-8) over epochs x minibatches of batch_rows consecutive rows (the rows
 * are expected pre-shuffled; minibatch order is shuffled by seed).  *loss_out = mean loss of the
 * last epoch. */
sn_status sn_mlp_train(sn_mlp* mlp, int64_t rows, const float* x, const float* target, int epochs, int batch_rows,
                       float lr, uint64_t seed, float* loss_out);

/* Per-element predictor data of a context (graph built):
 *   sn_predictor_features: feat [n_elem][16] = sigma_t, sigma_s, sigma_a, c, mean q, mean control
 *     point (3), volume, size h, distance to the mesh bounding box, boundary faces, mean face-
 *     neighbour sigma_t, sigma_t h, log sigma_t, mean face-neighbour c; phi_ref [n_elem] (may be
 *     NULL) = 4 pi max(mean q, 1e-12) / max(sigma_a, 1e-3 sigma_t).
 *   sn_predictor_init_targets: target [n_elem][N] = phi / phi_ref (initial-guess model output).
 *   sn_predictor_corr_data: from iterates phi_a, phi_b, phi_c (l-1, l, l+1): inputs [n_elem][18] =
 *     features, |c-b|/|b-a| (clipped at 10), log10(|c-b|/|c|); with phi_inf, target [n_elem] =
 *     log1p(clip(<phi_inf - c, c - b> / |c - b|^2, 0, 500)) (correction model output). */
sn_status sn_predictor_features(sn_ctx* ctx, float* feat, double* phi_ref);
sn_status sn_predictor_init_targets(sn_ctx* ctx, const double* phi, float* target);
sn_status sn_predictor_corr_data(sn_ctx* ctx, const double* phi_a, const double* phi_b, const double* phi_c,
                                 const double* phi_inf, float* inputs, float* target);

typedef struct {
  float init_mean[SN_FEATURES], init_istd[SN_FEATURES];          /* feature normalisation */
  float corr_mean[SN_FEATURES + 2], corr_istd[SN_FEATURES + 2];  /* correction-input normalisation */
  int32_t corr_start, corr_every;                                /* correction schedule */
} sn_predictor_cfg;

/* Source iteration with the predictor: phi_0 = init_model(normalised features) * phi_ref (or 0
 * without init_model); from iteration corr_start, every corr_every plain steps, the correction
 * model's g per element gives phi <- phi + expm1(clip(g, 0, 6)) (phi - phi_prev) and the
 * scattering source is refreshed.  A correction is accepted if the next plain residual is below
 * the one before it; otherwise corrections stop (plain source iteration continues).
 * Convergence is declared only on a step whose input was not corrected.  n_accepted /
 * n_rejected may be NULL. */
/* phi0 [n_elem][N] = init_model(normalised features) * phi_ref: the predicted initial flux. */
sn_status sn_predictor_initial_phi(sn_ctx* ctx, sn_mlp* init_model, const sn_predictor_cfg* cfg, double* phi0);

sn_status sn_source_iterate_learned(sn_ctx* ctx, double tol, int max_iter, int precision, sn_mlp* init_model,
                                    sn_mlp* corr_model, const sn_predictor_cfg* cfg, double* phi_out,
                                    sn_si_stats* stats, int32_t* n_accepted, int32_t* n_rejected);

/* Scalar-flux moment and relative change WITHOUT a context and without allocating anything
 * (the paper has no counterpart: this is a deployment entry point).
 *
 * For callers that cannot allocate device memory: code that only holds raw device buffers
 * handed to it by a host framework which owns all device memory through its own allocator
 * (fixed budget, no side allocations), or that must not call cudaMalloc/cudaFree because they
 * synchronise the whole device.  Such callers cannot create an sn_ctx, which allocates.
 *
 * Computes, on `cuda_stream` of device `device`, the same values as sn_moment:
 *   phi_out[e][m] = sum_d w[d] psi[d][e][m]   (d ascending)
 *   *residual     = max |phi_out - phi_prev| / max |phi_out|   (phi_prev NULL = 0)
 * w [n_dir], psi [n_dir][n_elem][n_dofs], phi_prev / phi_out [n_elem][n_dofs]: caller-owned
 * pointers to memory of `device` or managed memory (SN_EINVAL for host pointers and for buffers
 * of another device).  residual: host pointer or NULL; when given, the call synchronises the
 * stream.  The calling thread's current device is the same on return as before the call.  No scattering source is produced (there is no context).
 * Limit: n_elem * n_dofs <= 4,194,304 (SN_EINVAL beyond): the reduction scratch is a fixed
 * 256 KiB file-scope device array that every GPU loading the library holds until exit.  Calls
 * share that array and it keeps the last call's contents (every call overwrites what it
 * reads, so nothing needs clearing); calls that overlap on the GPU (other streams, other
 * threads) race on it.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  Calls no
 * cudaMalloc, cudaFree or allocating library routine. */
sn_status sn_moment_noalloc(int device, void* cuda_stream, int n_dir, int64_t n_elem, int n_dofs,
                            const double* w, const double* psi, const double* phi_prev,
                            double* phi_out, double* residual);

/* ---- Diffusion synthetic acceleration (the paper names DSA as the follow-up for scattering-
 * dominated problems [Sec. 4 opening, conclusions]; the operator is this library's reading).
 * After each sweep, sn_si_step (and so sn_source_iterate and the learned iteration) replaces the
 * scalar flux phi_half = sum_d w_d psi_d by phi_half + dphi, where dphi solves on the same DG space
 *   a(dphi, v) = int sigma_s (phi_half - phi_prev) v,
 *   a(u, v) = sum_K int_K (D grad u . grad v + sigma_a u v) + interior faces
 *             int (kappa [[u]][[v]] - {{D grad u . n}}[[v]] - [[u]]{{D grad v . n}}) + boundary faces
 *             int (kappa u v - (D grad u . n) v / 2 - u (D grad v . n) / 2),
 * D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s, [[u]] = u_owner - u_other (owner = lower element id),
 * kappa = max(c (D_o/h_o + D_t/h_t)/2, 1/4) inside, max(c D/h, 1/4) on the boundary, c = 2 p (p+1),
 * h = element measure / face measure.  The system is solved by conjugate gradients preconditioned
 * with the inverses of the diagonal blocks, to a relative residual of rtol (or max_iter
 * iterations).  The correction vanishes at the fixed point, which is that of plain source
 * iteration.  The operator is assembled at the first use after sn_build_graph and kept.
 * sn_set_dsa: enable (1) or disable (0) the step; rtol in (0, 1); max_iter 1..100000. */
sn_status sn_set_dsa(sn_ctx* ctx, int enable, double rtol, int max_iter);
/* One DSA correction on its own: phi_out = phi_half + dphi (all [n_elem][N], host or device).  Uses
 * the context's iteration buffers as scratch: call sn_si_begin before further sn_si_step calls.
 * *cg_iters (may be NULL) receives the CG iterations.  Errors: SN_ESTATE (no graph), SN_EMESH (a
 * singular diagonal block). */
sn_status sn_dsa_correction(sn_ctx* ctx, const double* phi_half, const double* phi_prev, double* phi_out,
                            int* cg_iters);
/* CG iterations of the last DSA solve of this context. */
int32_t sn_dsa_last_iters(const sn_ctx* ctx);

/* Number of kernel launches this context has issued since creation (diagnostics). */
int64_t sn_kernel_launches(const sn_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SNSWEEP_H */
