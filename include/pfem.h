/*
 * pfem.h - C ABI of the GB300 P1 finite-element operator and its warm-started solvers.
 *
 * The library evaluates, matrix-free and element by element, the discrete energy, the
 * internal-force residual and the tangent-times-vector product of P1 triangles (plane
 * strain) and P1 tetrahedra for linear elasticity and compressible Neo-Hookean material,
 * and drives Jacobi-PCG and Newton-Krylov solves started from a caller-supplied guess.
 *
 * Paper: "Pretrained Finite Element Method" (PFEM, arXiv 2601.03086).
 *   - energy loss, linear:       Sec. "Linear elastic plate with arbitrary holes" (plate
 *                                loss, Psi = 1/2 sigma:eps)
 *   - energy loss, Neo-Hookean:  Sec. "Nonlinear hyperelasticity" (Psi = 1/2 lam ln^2 J
 *                                - mu ln J + 1/2 mu (I1 - d))
 *   - explicit FE derivatives:   App. A (shape-function differentiation)
 *   - f_int, f_ext, tangent:     App. B (principle of virtual power, total Lagrangian,
 *                                K = K_geo + K_mat, Newton-Raphson with load steps)
 *   - warm start + criterion:    Sec. "Warm-start" (U^(0) = U^NO, ||r|| < tol, skip test)
 *
 * Conventions shared by every entry point
 *   - Node vectors (u, v, y, r, ...) are device pointers, DOF-interleaved: entry
 *     node*dim + i. Their element type is float for PFEM_F32 and double for PFEM_F64.
 *     The caller owns them; the library never frees or retains them.
 *   - Every call is ordered on the stream given at pfem_mesh_create (a cudaStream_t
 *     passed as void*, NULL = legacy default stream). Calls returning host values
 *     synchronise that stream; the others only enqueue work.
 *   - Dirichlet DOFs (mask = 1) are eliminated: the linear operator on full-length vectors
 *     is A = P K P + (I - P), P = projector on free DOFs; residuals are zero there.
 *   - No call traps the GPU. Errors come back as pfem_status; pfem_last_error() returns a
 *     thread-local message for the last failure of the calling thread.
 *   - Results are bitwise reproducible run to run (fixed reduction orders, no float
 *     atomics) for the same mesh, inputs and device.
 */
#ifndef PFEM_H
#define PFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PFEM_OK = 0,
  PFEM_ERR_INVALID_ARG = 1,        /* bad pointer, size, index, material or option */
  PFEM_ERR_DEGENERATE_ELEMENT = 2, /* |det D| <= 1e-12 (max edge)^d in the reference mesh */
  PFEM_ERR_INVERTED = 3,           /* some element has J = det F <= 0 (Neo-Hookean) */
  PFEM_ERR_NONFINITE = 4,          /* NaN/Inf met in a reduction */
  PFEM_ERR_NOT_CONVERGED = 5,      /* iteration cap reached */
  PFEM_ERR_OUT_OF_MEMORY = 6,      /* device or host allocation failed */
  PFEM_ERR_OVER_BUDGET = 7,        /* request can never fit the server's HBM budget */
  PFEM_PENDING = 8,                /* serving: result not ready yet */
  PFEM_ERR_TIMEOUT = 9,            /* a bounded wait gave up */
  PFEM_ERR_CUDA = 10,              /* a CUDA runtime call failed (message has details) */
  PFEM_ERR_UNSUPPORTED = 11        /* combination not built (e.g. dim or dtype) */
} pfem_status;

typedef enum { PFEM_LINEAR = 0, PFEM_NEOHOOKEAN = 1 } pfem_material_kind;
/* Vector element type and element arithmetic: F32 = float vectors, FP32 arithmetic;
 * F64 = double vectors, FP64 arithmetic; F64_F32 = double vectors, FP32 element arithmetic
 * (the operator the FP32 solvers apply to their FP64 iterates). Sums of energies are FP64. */
typedef enum { PFEM_F32 = 0, PFEM_F64 = 1, PFEM_F64_F32 = 2 } pfem_dtype;

typedef struct pfem_mesh_s* pfem_mesh_t;
typedef struct pfem_batch_s* pfem_batch_t;
typedef struct pfem_server_s* pfem_server_t;

/* Problem description (the point-cloud inputs of Sec. "Input and output of neural
 * operators": geometry, material, boundary conditions). All pointers are HOST pointers, read during pfem_mesh_create only. */
typedef struct {
  int32_t dim;                     /* 2: P1 triangles, plane strain, unit thickness; 3: P1 tets */
  int64_t n_nodes;                 /* >= 1 */
  const double* coords;            /* n_nodes*dim reference coordinates X, node-major */
  int64_t n_elems;                 /* >= 0 */
  const int32_t* conn;             /* n_elems*(dim+1) node ids; either orientation accepted */
  int32_t kind;                    /* pfem_material_kind */
  const double* mat_a;             /* per element: E (linear, > 0) | mu (Neo-Hookean, > 0) */
  const double* mat_b;             /* per element: nu in (-1, 0.5) (linear) | lambda >= 0 (NH) */
  const uint8_t* dirichlet_mask;   /* n_nodes*dim, 1 = prescribed DOF; NULL = none */
  const double* dirichlet_values;  /* n_nodes*dim values at full load; NULL = all zero */
  int64_t n_facets;                /* traction facets (edges in 2-D, triangles in 3-D) */
  const int32_t* facets;           /* n_facets*dim node ids */
  const double* traction;          /* n_facets*dim constant traction per facet */
  const double* f_ext_extra;       /* n_nodes*dim extra nodal force (body force), may be NULL */
} pfem_mesh_desc;

/* Plan statistics of a mesh (host-side bookkeeping; useful for traffic accounting). */
typedef struct {
  int64_t n_nodes, n_elems, n_dofs, n_free_dofs;
  int64_t n_tiles;          /* element tiles (shared-memory work units) */
  int64_t n_local_nodes;    /* sum over tiles of nodes touched by the tile */
  int64_t n_halo_nodes;     /* nodes whose elements span more than one tile */
  int64_t n_partials;       /* (tile, halo node) pairs */
  int64_t device_bytes;     /* device memory held by the mesh */
  int32_t max_tile_elems, max_tile_nodes;
  int64_t n_fans;           /* element fans (chains of simplices around a hinge, one per thread) */
  int32_t max_tile_slots;   /* largest per-tile count of (fan, node) contribution slots */
  int32_t reserved;
} pfem_mesh_stats;

typedef struct {
  int32_t iterations;              /* PCG iterations (all inner PCG iterations for Newton) */
  int32_t newton_iterations;       /* tangent solves (Newton only) */
  int32_t replacements;            /* FP64 residual replacements performed */
  int32_t inverted_backtracks;     /* Newton step halvings caused by J <= 0 */
  double rel_residual_recursive;   /* ||r_k|| / ref as tracked by the iteration */
  double rel_residual_true_f64;    /* ||P(f_ext - f_int(u))|| / ref with the FP64 operator */
  double initial_rel_residual;     /* ||r(u0)|| / ref, the Sec. "Warm-start" skip-test quantity */
  double reference_norm;           /* ref = ||r(u_lift)||: zero free DOFs, prescribed values */
  pfem_status status;
  int64_t kernel_launches;         /* kernels this solve ran (graph replays included) */
  double queue_s;                  /* serving: submit -> admission (s) */
  double total_s;                  /* serving: submit -> result ready (s) */
  double apply_ms;                 /* kernel timing on, plain loop: summed PCG-fused apply time */
  double update_ms;                /* kernel timing on, plain loop: summed update-kernel time */
  int32_t timed_iterations;        /* iterations those sums cover (0 = not timed) */
  int32_t load_step_cuts;          /* Newton: load increments halved after a failed level */
} pfem_solve_info;

/* ---- mesh ------------------------------------------------------------------------ */

/* Validate, plan (Morton-ordered element tiles, tile-local node lists, halo lists) and
 * upload a mesh. The library owns the resulting device memory until pfem_mesh_destroy.
 * Errors: INVALID_ARG (sizes, ids, materials, non-finite input), DEGENERATE_ELEMENT,
 * OUT_OF_MEMORY, CUDA. On error *out is NULL. */
pfem_status pfem_mesh_create(const pfem_mesh_desc* desc, void* cuda_stream, pfem_mesh_t* out);
void pfem_mesh_destroy(pfem_mesh_t mesh);

/* Plane-strain quadrilateral mesh (Sec. "Nonlinear hyperelasticity": the Q4 beam and Q8 Cook
 * membrane): desc->dim = 2, desc->conn holds n_elems * npe node ids per element, npe = 4
 * (bilinear, corners counterclockwise; 2 x 2 Gauss points) or 8 (serendipity: corners
 * counterclockwise, then the mid-edge nodes of edges 0-1, 1-2, 2-3, 3-0; 3 x 3 Gauss points).
 * Traction facets are element edges of npe == 4 ? 2 : 3 node ids (a, b[, mid]) with constant
 * traction (consistent loads |e|/2 at each end, or |e| (1/6, 1/6, 2/3)). Materials, Dirichlet
 * data and ownership as pfem_mesh_create. The mesh works with pfem_energy, pfem_residual,
 * pfem_tangent_apply, pfem_jacobi_diag, the energy-gradient / Hessian entry points and the
 * single-mesh solvers (graph and plain loops); the multi-vector, batch, no-alloc, persistent
 * and serving paths are for simplex meshes (PFEM_ERR_UNSUPPORTED). Errors: INVALID_ARG,
 * DEGENERATE_ELEMENT (det J <= 0 at a Gauss point, e.g. clockwise nodes), OUT_OF_MEMORY. */
pfem_status pfem_mesh_create_quad(const pfem_mesh_desc* desc, int32_t npe, void* cuda_stream, pfem_mesh_t* out);

/* Host-only: validate and plan desc exactly as pfem_mesh_create does, then check the plan's
 * structural invariants (every element in one tile, every incidence in one slot, complete
 * nodes holding all their incidences, halo nodes with one partial per touching tile).
 * Touches no device; fills *out (may be NULL). Same error codes as pfem_mesh_create. */
pfem_status pfem_plan_check(const pfem_mesh_desc* desc, pfem_mesh_stats* out);
pfem_status pfem_mesh_stats_get(pfem_mesh_t mesh, pfem_mesh_stats* out);

/* Load step factor s (App. B load stepping): f_ext and the prescribed values are both
 * multiplied by s in every later call. Default 1. */
pfem_status pfem_mesh_set_load_scale(pfem_mesh_t mesh, double s);

/* ---- element operator (energies of Secs. "Linear elastic plate with arbitrary holes" and
 *      "Nonlinear hyperelasticity"; App. B forces and tangent) -------------------------- */

/* Pi(u) = sum_e V_e Psi_e(u) - s f_ext . u and the strain part sum_e V_e Psi_e(u).
 * u: n_dofs device vector (dtype). Results are written to HOST doubles (either may be
 * NULL); the call synchronises. Neo-Hookean elements with J <= 0 make both +inf and the
 * call returns PFEM_ERR_INVERTED. Arithmetic: element terms in dtype, sums in FP64. */
pfem_status pfem_energy(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, double* energy,
                        double* strain_energy);

/* r = P (f_int(u) - s f_ext): the gradient of Pi on free DOFs, zero on Dirichlet DOFs
 * (App. B: f_iI = int dN_I/dX_l F_ik S_kl dV; linear: f_int = K u). u, r: n_dofs device
 * vectors of dtype, r written. Asynchronous. */
pfem_status pfem_residual(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, void* r);

/* y = A(u) v = P K(u) P v + (I - P) v, K(u) = K_geo + K_mat (App. B); u is ignored for
 * linear material (may be NULL). Asynchronous. */
pfem_status pfem_tangent_apply(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, const void* v,
                               void* y);

/* y_j = A v_j for k vectors at once (several load cases on one mesh: the six unit strains of
 * Sec. "Three-dimensional solid mechanics homogenization", or independent solves sharing each
 * operator application). The element data is read once per group of six vectors instead of
 * once per vector, and pairs of vectors share one FP32x2 instruction stream. v, y: k vectors
 * of n_dofs each, vector j starting at element j * n_dofs (float for PFEM_F32, double for
 * PFEM_F64_F32; the element arithmetic is FP32 for both). Linear material only (u is ignored
 * and may be NULL); Neo-Hookean meshes and other dtypes return PFEM_ERR_UNSUPPORTED; k < 0 or
 * NULL vectors PFEM_ERR_INVALID_ARG; k = 0 does nothing. Dirichlet handling as in
 * pfem_tangent_apply. Uses the mesh's scratch: do not overlap with other calls on the mesh.
 * Asynchronous. */
pfem_status pfem_tangent_apply_multi(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, int32_t k, const void* v,
                                     void* y);

/* Same result as pfem_tangent_apply, for callers that cannot allocate device memory when
 * they apply the operator (a frozen or exhausted memory pool, code running inside allocator
 * callbacks, runtimes that only own memory handed to them up front). The paper has no
 * counterpart: this is a library convenience. The call allocates nothing; the per-call
 * scratch of the element-tile pass (halo partial sums) lives in a fixed 16 MiB device array.
 * The array is created on a device when the first mesh is created there (pfem_mesh_create
 * looks its address up, which loads its module), never by this call, and the device then
 * holds it until the process exits. Limits and behaviour:
 *   - meshes whose halo scratch (n_partials * 4 * 4 bytes for F32/F64_F32, * 4 * 8 for F64:
 *     at most 1,048,576 partials in FP32 arithmetic and 524,288 in FP64) exceeds 16 MiB are
 *     rejected with PFEM_ERR_INVALID_ARG;
 *   - the current device must be the mesh's device (else PFEM_ERR_INVALID_ARG);
 *   - every call shares the one array and it keeps the last call's contents (each call
 *     overwrites what it reads, so nothing needs clearing); calls that overlap on the GPU,
 *     on any stream, race on it and must be serialised by the caller.
 * Arguments, layouts and the other errors are those of pfem_tangent_apply. */
pfem_status pfem_tangent_apply_noalloc(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, const void* v,
                                       void* y);

/* Derivatives of the energy loss for reverse-mode differentiation (the backward pass of the
 * physics loss of Sec. "Pretraining"; App. A explicit derivatives), with the upstream
 * factor applied inside the kernel. scale: a device scalar of the vector type
 * (float for PFEM_F32, double otherwise), NULL = 1.
 *   pfem_energy_gradient:  g = scale * P (f_int(u) - s f_ext)   (dPi/du on free DOFs, 0 on
 *                          prescribed DOFs; the same values as pfem_residual when scale = 1)
 *   pfem_energy_hvp:       y = scale * P K(u) P v                (Hessian of Pi on the free DOFs
 *                          times v; rows and columns of prescribed DOFs are zero, unlike the
 *                          identity block of pfem_tangent_apply)
 * u, v, g, y: n_dofs device vectors of dtype. Asynchronous. */
pfem_status pfem_energy_gradient(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, const void* scale, void* g);
pfem_status pfem_energy_hvp(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, const void* v, const void* scale,
                            void* y);

/* out = a . b over the mesh's n_dofs entries (device vectors of dtype), summed in FP64 in a
 * fixed order and written to the device scalar out in the vector type (the chain-rule term of
 * the upstream factor in the energy loss's double backward). Asynchronous. */
pfem_status pfem_dot(pfem_mesh_t mesh, pfem_dtype dtype, const void* a, const void* b, void* out);

/* d = diag A(u): diag K(u) on free DOFs, 1 on Dirichlet DOFs (the Jacobi preconditioner).
 * u ignored for linear material. Asynchronous. */
pfem_status pfem_jacobi_diag(pfem_mesh_t mesh, pfem_dtype dtype, const void* u, void* d);

/* ---- warm-started solvers (Sec. "Warm-start"; App. B) ------------------------------ */

/* Linear elasticity K U = F by Jacobi-PCG started from u0 (NULL = zero). The prescribed
 * values overwrite u0 on Dirichlet DOFs. Stops when ||r_k|| / ref < tol with
 * ref = ||r(u_lift)|| (= ||f_ext,free|| when the prescribed values are zero); checked
 * before the first iteration (skip test). dtype selects the element arithmetic (F32: FP32
 * operator with FP64 vectors, dots and norms plus FP64 residual replacement; F64: FP64
 * throughout). u0, u_out: FP64 device vectors (may alias). info may be NULL.
 * Returns NOT_CONVERGED if max_iter is reached (u_out then holds the last iterate). */
pfem_status pfem_solve_linear(pfem_mesh_t mesh, pfem_dtype dtype, const double* u0, double tol,
                              int32_t max_iter, double* u_out, pfem_solve_info* info);

/* Neo-Hookean (or linear) equilibrium by Newton-Raphson with n_load_steps equal load steps
 * (App. B); a warm start passes u0 = U^NO and n_load_steps = 1, bypassing the earlier
 * steps. Residuals and updates in FP64; tangent applies in dtype; inner Jacobi-PCG to
 * inner_tol relative to the current residual. Step halving (<= 10) when a trial makes
 * J <= 0. A load level that still fails (every halving inverts an element, max_newton
 * iterations without convergence, or a non-finite residual) is retried from the last
 * converged state with half the load increment (at most 8 times per solve, reported in
 * info->load_step_cuts); then INVERTED / NOT_CONVERGED / NONFINITE. u0/u_out: FP64 device
 * vectors (may alias, u0 NULL = zero). */
pfem_status pfem_solve_newton(pfem_mesh_t mesh, pfem_dtype dtype, const double* u0, double tol,
                              int32_t n_load_steps, int32_t max_newton, double inner_tol,
                              double* u_out, pfem_solve_info* info);

/* k independent linear solves on one mesh that share every operator application (several
 * load cases: App. B K u = f per case; the six unit-strain cases of the homogenisation
 * appendix): solves P (K + S) P x_j = P b_j by Jacobi-PCG for j < k, where S is the mesh's
 * penalty-spring matrix (zero without springs), with x_j = 0 on prescribed DOFs. b, u0, u_out:
 * k vectors of n_dofs FP64 device values each, vector j at element j * n_dofs (u0 NULL = zero
 * start; u0 and u_out may alias). Per solve: stops when ||P (b_j - A x_j)|| / ||P b_j|| < tol
 * (checked before the first iteration, confirmed with the FP64 operator), at most max_iter
 * iterations. dtype: PFEM_F32 = FP32 element arithmetic in one multi-vector element pass per
 * iteration, FP64 vectors, dots and residual replacements; PFEM_F64 = FP64 element arithmetic.
 * infos: k entries (may be NULL). Linear material only. Returns the first failing status
 * (NOT_CONVERGED, NONFINITE) or PFEM_OK when every solve converged. */
pfem_status pfem_solve_linear_multi(pfem_mesh_t mesh, pfem_dtype dtype, int32_t k, const double* b,
                                    const double* u0, double tol, int32_t max_iter, double* u_out,
                                    pfem_solve_info* infos);

/* Effective elastic tensor of a periodic cell (appendix "Numerical homogenization theory",
 * with the TPMS cells of appendix "Generation of TPMS geometries" as typical input): for the
 * six unit strains eps0 (11, 22, 33, 12, 13, 23; shear cases with both off-diagonal entries
 * 1, as printed) the fluctuation X^v solves (K + S) X^v = K X^0 with X^0 = eps0 (X - X_min)
 * and S the mesh's penalty springs between opposite-face nodes (pfem_mesh_set_springs), by
 * six PCG solves sharing each operator pass; then E^H = X^T K X / |Omega| with X = X^0 - X^v
 * (the appendix's integral of (eps0 - eps^v) : E : (eps0 - eps^v)); |Omega| is the volume of
 * the coordinates' bounding box. The mesh must fix every DOF of one node at the cell's minimum
 * corner (the periodic coupling leaves rigid translations free) and have no other prescribed
 * DOFs. coords: HOST n_nodes*3 reference coordinates (those the mesh was built from). xv0:
 * optional warm start of the six fluctuations (device, 6 * n_dofs FP64, NULL = zero: the
 * Sec. "Warm-start" use). eh: HOST 36 doubles, row-major E^H. xv_out: optional device
 * 6 * n_dofs FP64 output of the fluctuations. infos: 6 entries (may be NULL). dtype selects the
 * element arithmetic of the solves (PFEM_F32 / PFEM_F64); loads and E^H use FP64. Returns
 * PFEM_ERR_NOT_CONVERGED (E^H still written) if a solve stopped at max_iter. Synchronises. */
pfem_status pfem_homogenize(pfem_mesh_t mesh, pfem_dtype dtype, const double* coords, const double* xv0, double tol,
                            int32_t max_iter, double* eh, double* xv_out, pfem_solve_info* infos);

/* Penalty springs between node pairs (the homogenisation appendix's "virtual elements" that
 * couple corresponding nodes of opposite faces of a periodic cell): energy 1/2 kappa
 * |u_a - u_b|^2 per pair. pairs: HOST array of n_pairs (a, b) node ids; stiffness kappa >= 0;
 * n_pairs = 0 removes them. Replaces any earlier set; synchronises the mesh stream. With
 * springs, pfem_tangent_apply(_multi), pfem_residual, pfem_jacobi_diag and the linear solvers
 * use K + S (pfem_solve_linear then needs zero prescribed values and load scale 1); the energy,
 * its autograd entry points, batches, the no-alloc apply and Newton return
 * PFEM_ERR_UNSUPPORTED. Errors: INVALID_ARG (ids out of range or equal, kappa < 0 or not
 * finite), OUT_OF_MEMORY / CUDA. */
pfem_status pfem_mesh_set_springs(pfem_mesh_t mesh, int64_t n_pairs, const int32_t* pairs, double stiffness);

/* Solver loop style for later solves (process-wide); every mode gives bitwise identical
 * iterates. 0: one persistent cooperative kernel runs PCG iterations until an FP64
 * residual replacement or termination (grid barriers with bounded waits: a barrier that
 * gives up ends the solve with PFEM_ERR_TIMEOUT); FP64 element arithmetic, or a device that
 * cannot hold the grid, uses mode 2 instead. 1: the two kernels of one iteration at a time
 * with a host-synchronised convergence check (the plain GPU loop used as the serving
 * baseline). 2 (default): the iteration captured as a CUDA graph with a device-side while
 * loop. Other values: PFEM_ERR_INVALID_ARG. */
pfem_status pfem_set_solver_mode(int32_t mode);

/* Failure-detection settings of the persistent solver mode (process-wide; the default is
 * spin_limit <= 0, absent_cta = -1). Every grid-barrier wait of the persistent PCG kernel polls
 * at most spin_limit times (each poll sleeps >= 32 ns; the default allows more than a second)
 * and then flags the barrier, so the solve ends with PFEM_ERR_TIMEOUT and the context stays
 * usable. absent_cta >= 0 makes that CTA of later persistent launches leave at its first grid
 * barrier without arriving, as a CTA that never arrives would, so that tests can make the
 * other CTAs' waits run out (host-side injection; nothing faults or hangs). absent_cta < -1:
 * PFEM_ERR_INVALID_ARG. The paper has no counterpart. */
pfem_status pfem_set_barrier_test(int64_t spin_limit, int32_t absent_cta);

/* Per-kernel timing of later solves (process-wide; 1 = on, 0 = off, the default; other
 * values PFEM_ERR_INVALID_ARG). While on, the plain loop (solver mode 1) brackets the two
 * kernels of every PCG iteration with CUDA events on the mesh's stream and reports their
 * summed durations in pfem_solve_info (apply_ms, update_ms, timed_iterations); the graph
 * and persistent loops are not timed. */
pfem_status pfem_set_kernel_timing(int32_t on);

/* ---- ragged batch: energy loss, gradient and Hessian-vector product in one launch --- */

/* The differentiable FE energy loss of Secs. "Linear elastic plate with arbitrary holes"
 * and "Nonlinear hyperelasticity" over several meshes at once (the
 * pretraining loss is summed over a batch of geometries). Groups 3-D meshes (one device;
 * materials may differ per mesh) for one-launch evaluation. The meshes must outlive the
 * batch; a batch evaluation uses the meshes' scratch, so it must not overlap on the GPU with
 * other calls on the same meshes. Batch vectors are the concatenation of the meshes' DOF
 * vectors in the order given (offsets from pfem_batch_offsets). */
pfem_status pfem_batch_create(const pfem_mesh_t* meshes, int32_t n_meshes, pfem_batch_t* out);
void pfem_batch_destroy(pfem_batch_t batch);
/* offsets[m] = first DOF of mesh m, offsets[n_meshes] = total DOFs (host array). */
pfem_status pfem_batch_offsets(pfem_batch_t batch, int64_t* offsets);

/* For every mesh m at once (FP32 element arithmetic, FP64 energy sums), with s_m =
 * mesh_scale[m] (device floats, NULL = 1):
 *   energy_dev[m] = Pi_m(u)                    if energy_dev != NULL (device doubles)
 *   grad          = s_m P (f_int(u) - f_ext)   if grad != NULL  (gradient of s_m Pi_m on free DOFs)
 *   hvp           = s_m P K(u) P v            if hvp != NULL   (Hessian of s_m Pi_m times v; zero
 *                                                                on prescribed DOFs)
 * u, v, grad, hvp: float device vectors over the batch's total DOFs. One element launch for
 * all meshes plus one small energy reduction. Asynchronous on the first mesh's stream.
 * inverted_dev (device int32, may be NULL) receives the number of elements with J <= 0. */
pfem_status pfem_batch_eval(pfem_batch_t batch, const float* u, const float* v, const float* mesh_scale,
                            double* energy_dev, float* grad, float* hvp, int32_t* inverted_dev);

/* ---- serving: continuous batching of warm-started solves -------------------------- */

typedef enum { PFEM_SOLVE_LINEAR = 0, PFEM_SOLVE_NEWTON = 1 } pfem_solve_kind;

/* A server owns planner threads, one worker thread and a CUDA stream on the device current
 * at creation (Sec. "Warm-start": problems arrive at a platform whose FE iterations refine each
 * warm start). Requests are planned on the host as they arrive, admitted in arrival order
 * while a slot is free and their device footprint (mesh plan + solver vectors) fits
 * hbm_budget_bytes, and then every resident solve advances in shared launches (one fused
 * element apply over all their tiles and one vector update per PCG step); finished solves
 * free their slot and memory while the others continue. 3-D meshes only. */
pfem_status pfem_serve_create(size_t hbm_budget_bytes, int32_t max_slots, pfem_server_t* out);

/* Copies the description and u0 (HOST, n_nodes*dim doubles, NULL = zero start) and queues
 * the request. kind: pfem_solve_kind (PFEM_SOLVE_LINEAR needs linear material); tol as in
 * pfem_solve_linear / pfem_solve_newton (inner PCG 1e-8); Newton runs n_load_steps (>= 1).
 * FP32 element operator, FP64 vectors. *ticket receives the request id. */
pfem_status pfem_serve_submit(pfem_server_t server, const pfem_mesh_desc* desc, int32_t kind,
                              const double* u0_host, double tol, int32_t n_load_steps,
                              uint64_t* ticket);

/* PFEM_PENDING until the request finished; then copies the solution to u_out_host
 * (n_nodes*dim doubles, may be NULL), fills info (may be NULL, with queue/total latency),
 * releases the ticket and returns the request's status (OVER_BUDGET if its footprint can
 * never fit the budget). */
pfem_status pfem_serve_poll(pfem_server_t server, uint64_t ticket, double* u_out_host,
                            pfem_solve_info* info);

/* Worker-thread accounting since creation, out[0..7]: seconds spent waiting for the device
 * after each chunk of shared steps, admitting requests (uploads, solve set-up), rebuilding
 * the device tables and capturing the chunk graph, and running the per-request state
 * machine; then the counts of chunks, table rebuilds and admitted requests; out[7] = 0.
 * Values are read without stopping the worker. */
pfem_status pfem_serve_stats(pfem_server_t server, double* out);

/* Waits (at most timeout_s) until every submitted request has finished; TIMEOUT otherwise. */
pfem_status pfem_serve_drain(pfem_server_t server, double timeout_s);

/* Stops the server; requests still running are abandoned. */
void pfem_serve_destroy(pfem_server_t server);

/* ---- physics attention (Sec. "Transolver") ------------------------------------------
 *
 * The physics-attention module of the Transolver backbone that produces the warm starts, for
 * N points with C feature channels X (N x C) and S physics-aware tokens:
 *   U = X W_U + b_U (N x C);  M = softmax over the S tokens of X W_M + b_M (N x S);
 *   Z_J = sum_I M_IJ U_I / sum_I M_IJ (S x C; a token whose weight sum is 0 is the zero row);
 *   Q, K, V = Z W_Q + b_Q, Z W_K + b_K, Z W_V + b_V; per head h (C/H channels each)
 *   Z^t_h = softmax(scale Q_h K_h^T) V_h (the section prints scale = 1);
 *   X^t = M Z^t (N x C).
 * Each "MLP" of the section is one affine map here. Weights are (in, out) matrices.
 *
 * Precision: X, X^t and M are bf16 in memory, the projections and sums run on the tensor
 * cores with FP32 accumulation, U and Z^t are rounded to bf16 before their products; the
 * tokens, Q/K/V and the attention are FP32. Results are bitwise reproducible. */
typedef struct pfem_attn_s* pfem_attn_t;

typedef struct {               /* HOST float arrays, read during pfem_attn_create only */
  const float *wu, *bu;        /* C x C (in, out) and C: the U map; rounded to bf16 */
  const float *wm, *bm;        /* C x S and S: the slice logits; wm rounded to bf16 */
  const float *wq, *bq;        /* C x C and C each: the token projections (FP32) */
  const float *wk, *bk;
  const float *wv, *bv;
} pfem_attn_weights;

/* Build a module on the current device with its weights resident. n_channels must be 128;
 * n_tokens a multiple of 16 in [16, 128]; n_heads 2, 4, 8 or 16 (64, 32, 16 or 8 channels
 * per head); calls run on cuda_stream (NULL = legacy default stream).
 * Errors: INVALID_ARG (NULL pointer, non-finite weight or scale), UNSUPPORTED (sizes),
 * OUT_OF_MEMORY / CUDA. On error *out is NULL. */
pfem_status pfem_attn_create(int32_t n_channels, int32_t n_tokens, int32_t n_heads, double scale,
                             const pfem_attn_weights* weights, void* cuda_stream, pfem_attn_t* out);

/* Enqueue the forward pass for n_points points (0 = nothing to do). Device pointers, 16-byte
 * aligned: x (bf16 [n_points][128], read), xt (bf16 [n_points][128], written), m (bf16
 * [n_points][S_pad] with S_pad = 64 for S <= 64 and 128 otherwise, written with the slice
 * weights and zero pad columns; NULL = a workspace of the handle, grown on demand with a
 * stream synchronisation), z and zt (float [S][128], the tokens Z and Z^t; NULL = not
 * copied out). Only enqueues work; pfem_attn_sync reports errors raised on the device.
 * Errors: INVALID_ARG (NULL or misaligned pointer, n_points < 0 or >= 2^31 - 128), CUDA. */
pfem_status pfem_attn_forward(pfem_attn_t attn, int64_t n_points, const void* x, void* xt, void* m,
                              float* z, float* zt);

/* Synchronise the module's stream. TIMEOUT if a bounded device wait of an earlier forward
 * expired (its outputs are then incomplete; the error word is cleared). */
pfem_status pfem_attn_sync(pfem_attn_t attn);

/* Synchronise the stream and free the module. NULL is ignored. */
void pfem_attn_destroy(pfem_attn_t attn);

/* Kernel timing of later forwards (on != 0): CUDA events on the module's stream around each
 * of its four kernels. pfem_attn_kernel_ms waits for the last timed forward and writes the
 * durations in ms of its slice, token-sum, token-attention and deslice kernels to ms[0..3].
 * INVALID_ARG when timing is off. */
pfem_status pfem_attn_set_timing(pfem_attn_t attn, int32_t on);
pfem_status pfem_attn_kernel_ms(pfem_attn_t attn, double* ms);

/* ---- bounds-checked build ------------------------------------------------------------
 * libpfem_checked.so is the same library compiled with PFEM_CHECKED: the element-tile
 * kernels check every global node index and halo-partial range they gather or scatter
 * through; an index out of range is replaced by 0 (a valid address) and flagged instead of
 * dereferenced. */

/* Checked build: synchronise the device, then *word = OR of the flags raised since the last
 * call (bit 0: node index out of range, bit 1: partial range out of range, bit 31: the flag
 * could not be read), and clear them. Regular build: *word = 0, UNSUPPORTED. */
pfem_status pfem_check_status(uint32_t* word);

/* Checked build, for tests of the checks: overwrite the global node id of tile-node record
 * local_node (0 <= local_node < stats.n_local_nodes) with node_id (< 2^28, any value,
 * in range or not). Synchronises the mesh's stream. Regular build: UNSUPPORTED, nothing
 * changed. */
pfem_status pfem_debug_set_node_id(pfem_mesh_t mesh, int64_t local_node, int64_t node_id);

/* ---- misc ------------------------------------------------------------------------- */

const char* pfem_last_error(void);
/* Library version string. */
const char* pfem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PFEM_H */
