/*
 * nbte.h -- C ABI of libnanobte: steady non-gray phonon BTE (relaxation-time
 * approximation) on one B300 GPU.
 *
 * What the library computes (paper: "NanoBTE", Sec. II and III):
 *   for every band l and discrete direction i the steady per-mode equation
 *   (Sec. II, Eq. (4))   v_l s_i . grad e + (e - e0_l)/tau_l = S_l,
 *   e0_l = C_l T / W (Eq. (11)), discretised with first-order upwind finite
 *   volumes; walls are thermalizing, diffuse, specular or partially specular
 *   (Sec. II, Sec. III A/B); the volumetric heat source is an equilibrium
 *   source, uniform over directions and split over bands by heat capacity
 *   (Sec. III B); the lattice temperature follows from the collision moment
 *   (Eq. (5)) -- the sequential scheme (Eq. (6)) -- or additionally from the
 *   diffusion-type correction of Eqs. (8)-(10) -- the synthetic scheme
 *   (Eq. (12)); the heat flux is the moment of Eq. (7).
 *
 * Conventions for every call:
 *   - SI units: metres, kelvin, J/(m^3 K), m/s, s, W/m^3.
 *   - Host arrays only.  The caller owns every array it passes; the library
 *     copies what it needs before returning and never keeps a caller pointer.
 *     Output arrays are caller-allocated and written in full on success.
 *   - Every call returns an int status: NBTE_OK (0) or a negative NBTE_ERR_*
 *     code; on error nothing observable has changed (for solves: the solver
 *     state is as after the last completed iteration) and nbte_last_error()
 *     describes the failure.  Argument checks (sizes, NaN, signs, mesh
 *     validity) happen before any device work.
 *   - Handles are not thread-safe: one handle must not be used by two host
 *     threads at once.  Different handles are independent.
 *   - Each solver runs on its own CUDA stream (or the one given with
 *     nbte_solver_set_stream) of the device current when it was created.
 */
#ifndef NBTE_H
#define NBTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbte_mesh nbte_mesh;
typedef struct nbte_solver nbte_solver;

enum {
  NBTE_OK = 0,
  NBTE_ERR_ARG = -1,            /* invalid argument (size, NaN, sign, range)        */
  NBTE_ERR_MESH = -2,           /* invalid mesh (degenerate cell, untagged face...) */
  NBTE_ERR_OOM = -3,            /* host or device allocation failed                 */
  NBTE_ERR_CUDA = -4,           /* a CUDA call failed                               */
  NBTE_ERR_NOT_CONVERGED = -5,  /* max_iter reached before tol (results are kept)  */
  NBTE_ERR_DIVERGED = -6,       /* residual grew without bound / non-finite values  */
  NBTE_ERR_DEVICE_TIMEOUT = -7, /* a bounded device-side wait gave up               */
  NBTE_ERR_STATE = -8           /* call out of order (e.g. solve before set_bands)  */
};

/* cell types: node counts and local orderings
 *   NBTE_TRI  (2D) 3 nodes;  NBTE_QUAD (2D) 4 nodes in cyclic order;
 *   NBTE_TET  (3D) 4 nodes;  NBTE_HEX  (3D) 8 nodes, bottom cycle 0-1-2-3 then
 *   top cycle 4-5-6-7 with node 4 above node 0 (faces planar).            */
enum { NBTE_TRI = 3, NBTE_QUAD = 4, NBTE_TET = 10, NBTE_HEX = 12 };

/* wall types (Sec. II; Sec. III A/B) */
enum { NBTE_THERMALIZING = 0, NBTE_DIFFUSE = 1, NBTE_SPECULAR = 2, NBTE_PARTIAL = 3 };

/* ------------------------------------------------------------------ mesh --
 * nbte_mesh_create: build the finite-volume mesh (faces, outward face
 * vectors, volumes, centroids) from nodes and cells.
 *   dim          2 or 3; must match cell_type.
 *   xyz          n_nodes*dim coordinates, node-major.
 *   cell_nodes   n_cells*nodes_per_cell node indices (0-based).
 *   bface_nodes  n_bfaces*nodes_per_face node indices of the exterior faces
 *                (2 per face in 2D, 3 for tet meshes, 4 for hex meshes), any
 *                order within a face; bface_tag[n_bfaces] their integer tags.
 * Every exterior face must appear exactly once in bface_nodes, and every
 * listed face must be exterior: otherwise NBTE_ERR_MESH.  Degenerate cells
 * (volume or face area ~0, non-convex) give NBTE_ERR_MESH.  Geometry:
 * centroids are vertex averages; a 3D quadrilateral face vector is half the
 * cross product of its diagonals; volumes come from the divergence theorem.
 * The library renumbers cells internally (space-filling-curve order); every
 * per-cell array of this API is in the caller's cell order.
 */
int nbte_mesh_create(int dim, int64_t n_nodes, const double* xyz, int cell_type,
                     int64_t n_cells, const int64_t* cell_nodes, int64_t n_bfaces,
                     const int64_t* bface_nodes, const int32_t* bface_tag, nbte_mesh** out);
int nbte_mesh_destroy(nbte_mesh* mesh);
/* n_cells of the mesh; total volume (m^3, or m^2 in 2D) */
int nbte_mesh_info(const nbte_mesh* mesh, int64_t* n_cells, double* volume);

/* ---------------------------------------------------------------- solver --
 * nbte_solver_create: a solver bound to `mesh` (the mesh must outlive it) and
 * the CUDA device current at this call.  T_ref: reference temperature (K)
 * around which deviations are carried (Sec. III A uses 300 K).            */
int nbte_solver_create(const nbte_mesh* mesh, double T_ref, nbte_solver** out);
int nbte_solver_destroy(nbte_solver* solver);
/* Use the caller's stream (a cudaStream_t passed as void*) for all device work
 * of this solver; NULL restores the solver's own stream.                 */
int nbte_solver_set_stream(nbte_solver* solver, void* cuda_stream);

/* Band table (Sec. II; Sec. III A/B): heat capacity C[l] > 0 (J/m^3K),
 * group velocity v[l] > 0 (m/s), relaxation time tau[l] > 0 (s).          */
int nbte_set_bands(nbte_solver* solver, int n_bands, const double* C, const double* v,
                   const double* tau);

/* Discrete-ordinates set (Sec. II, Eq. (11)): s[n_dirs*3] unit vectors
 * (|s| = 1 within 1e-9), w[n_dirs] > 0.  On a 2D mesh only (s_x, s_y) enter
 * the transport; s_z distinguishes out-of-plane directions of a 3D material
 * (Sec. III A, the cross-plane case).  W = sum w.                         */
int nbte_set_quadrature(nbte_solver* solver, int n_dirs, const double* s, const double* w);

/* One condition per boundary tag.  T_wall (K) is used by THERMALIZING walls;
 * specularity p in [0,1] by PARTIAL walls (incoming = p*specular +
 * (1-p)*diffuse).  Every tag present in the mesh must be covered and at least
 * one wall must be THERMALIZING (otherwise the steady problem has no unique
 * solution): NBTE_ERR_ARG.                                                */
typedef struct {
  int32_t tag;
  int32_t type;
  double T_wall;
  double specularity;
} nbte_boundary;
int nbte_set_boundaries(nbte_solver* solver, int n, const nbte_boundary* bcs);

/* Volumetric heat generation Qdot[n_cells] (W/m^3, finite; NULL = none).  */
int nbte_set_heat_source(nbte_solver* solver, const double* Qdot);

/* ------------------------------------------------------------------ solve --
 * scheme:    0 sequential (Eq. (6)); 1 synthetic, diffusion-synthetic form of
 *            Eqs. (8)-(10) (correction added to the kinetic temperature of
 *            the new distribution); 2 synthetic, literal form (correction
 *            added to the previous iterate).
 * precision: 0 FP64 throughout; 1 FP32 sweep (distributions and transport
 *            coefficients FP32; moments, temperature, residual, correction
 *            and energy balance FP64).
 * tol:       stop when |T^{n+1}-T^n|_inf / |T^{n+1}-T_ref|_inf < tol.  With
 *            the FP32 sweep the increment bottoms out at the rounding floor
 *            (about 1e-8..1e-7); the solve also stops, with NBTE_OK, once the
 *            increment is below 1e-5 and has not fallen by 10% over 200
 *            iterations (info.residual then reports that floor).
 * max_iter:  iteration cap (> 0).  n_iter > 0 instead runs exactly n_iter
 *            iterations with no convergence test.
 * T_init:    initial temperature field [n_cells] (K) or NULL (= T_ref).
 * warm:      1 = continue from the solver's current state (T and wall
 *            values) instead of T_init.
 * band_group: bands per work item: 1, 2, 4 or 8 with an FP32 sweep, 1, 2
 *            or 4 in FP64.  cta_threads: threads per sweep CTA, a multiple of
 *            32 in [64, 544]; one copy warp plus one consumer thread per
 *            position of a pipelined chunk.  threads_per_cell: 0 or 1 (one
 *            thread carries all bands of its group for a cell).  With
 *            band_group = cta_threads = 0 the first solve times every
 *            feasible layout once (a few sweeps on scratch state) and keeps
 *            the fastest for this plan, band table and precision.  None of
 *            them changes results beyond rounding order; an infeasible
 *            choice (two copy stages exceed shared memory) is NBTE_ERR_ARG.
 * ring:      where the sweep keeps the outgoing values of a direction's live
 *            cells: 0 = shared memory when it fits, else global memory;
 *            1 = shared memory (NBTE_ERR_ARG if it does not fit); 2 = global
 *            memory (one region per work item, L2-resident while it runs).
 *            Results are identical either way.
 * init:      starting temperature when not warm: 0 = T_init (or T_ref);
 *            1 = the diffusion-limit (Fourier) solution, L T' = Qdot V with
 *            the thermalizing walls' temperatures as Dirichlet data and no
 *            flux through other walls, L the synthetic correction's TPFA
 *            operator, solved by its CG to 1e-12 (excludes T_init).  Only
 *            the starting point changes, never the converged field.
 * order:     upwind order of the face values: 0 or 1 = first order (the
 *            default); 2 = second order on interior faces: the upwind cell's
 *            value plus its least-squares gradient (over its face
 *            neighbours) times the offset to the face centroid, the gradient
 *            taken from the previous iteration's distribution (a deferred
 *            correction added to the sweep's right-hand side; none in the
 *            first sweep).  Wall faces keep the cell value, so wall coupling
 *            and energy conservation are those of the first-order scheme;
 *            cells with fewer than dim + 1 face neighbours (wall triangles
 *            and tetrahedra, corner quadrilaterals and hexahedra) carry no
 *            gradient, which keeps the lagged correction contracting on
 *            unstructured meshes.  Holds one more distribution and one
 *            source per (work item, position) on the device.
 * deterministic: how the sweep sums the collision moment of Eq. (5) over
 *            work items.  0 (default) = by the layout's size: when one
 *            partial per (work item, cell) takes at most 256 MB, the sweep
 *            writes them and the update kernel sums each cell's in a fixed
 *            order (results reproducible bit for bit); above that, FP64
 *            atomic adds into one sum per cell, whose order, and so whose
 *            last bits, vary from run to run (about 1e-16 relative in FP64;
 *            an FP32 sweep may then round a temperature to the neighbouring
 *            FP32 value).  1 = always the fixed-order partials.
 * cg_tol, cg_max_iter: relative residual and cap of the conjugate-gradient
 *            solve of the synthetic correction (0 = defaults 1e-2, 5000); the
 *            correction only changes the rate of convergence, not the limit.
 *            Each solve starts from the previous correction scaled by its
 *            Galerkin factor.
 * use_graph: 1 = replay each iteration from a captured CUDA graph.
 * skip_outputs: 1 = do not compute the energy temperature, heat flux and wall
 *            heat of the last sweep (kind-0 and kind-2 temperatures remain
 *            readable); saves one extra sweep per call.
 * profile:   1 = time every sweep launch with CUDA events on the solver's
 *            stream (reported in nbte_solve_info); adds a host sync per
 *            iteration.
 * With n_iter > 0 (and profile 0) the iterations are enqueued back to back
 * and the host synchronises once at the end.
 */
typedef struct {
  int32_t scheme;
  int32_t precision;
  double tol;
  int32_t max_iter;
  int32_t n_iter;
  const double* T_init;
  int32_t warm;
  int32_t band_group;
  int32_t threads_per_cell;
  double cg_tol;
  int32_t cg_max_iter;
  int32_t use_graph;
  int32_t skip_outputs;
  int32_t profile;
  int32_t cta_threads;
  int32_t ring;
  int32_t init;
  int32_t order;
  int32_t deterministic;
} nbte_solve_opts;

/* Filled on return from nbte_solve_steady (also on NOT_CONVERGED):
 *   iterations        sweeps performed;
 *   residual          last relative increment (see tol);
 *   energy_imbalance  |net heat through thermalizing walls - integral of
 *                     Qdot| / max(integral |Qdot|, sum |wall heat|), FP64;
 *   lagged_faces      inflow faces whose upwind value is taken from the
 *                     previous iteration to break upwind-graph cycles;
 *   seconds           wall time of the iteration loop;
 *   cg_iterations     total CG iterations (synthetic schemes);
 *   sweep_seconds     summed device time of the sweep launches (profile=1);
 *   sweep_launches    sweep launches timed (profile=1);
 *   kernel_launches   kernels this call launched (graph replays counted by
 *                     their kernel nodes);
 *   status            this solve's own status (the call's return value for
 *                     nbte_solve_steady; per solver for nbte_solve_batch).  */
typedef struct {
  int32_t iterations;
  double residual;
  double energy_imbalance;
  int64_t lagged_faces;
  double seconds;
  int64_t cg_iterations;
  double sweep_seconds;
  int64_t sweep_launches;
  int64_t kernel_launches;
  int32_t status;
} nbte_solve_info;

/* Default options: sequential, FP64, tol 1e-10, max_iter 10000.           */
int nbte_default_opts(nbte_solve_opts* opts);

/* Run the iteration (Eq. (6) or Eq. (12)) until tol or for n_iter sweeps.
 * Returns NBTE_OK, NBTE_ERR_NOT_CONVERGED (results of the last iteration are
 * kept and readable), NBTE_ERR_DIVERGED or NBTE_ERR_DEVICE_TIMEOUT.       */
int nbte_solve_steady(nbte_solver* solver, const nbte_solve_opts* opts, nbte_solve_info* info);

/* Solve several independent problems together (Sec. II iteration for each,
 * one options record for all).  Every iteration runs all still-unconverged
 * solvers at once: their sweeps share fused launches (one per sweep variant),
 * their synthetic corrections one cooperative CG launch in which each solver
 * owns a share of the blocks, on solvers[0]'s stream.  A solver leaves the
 * batch when it converges, exactly as nbte_solve_steady would stop it, so
 * each result equals its solve alone (to the CG's rounding: its block share
 * differs).  infos[k] (may be NULL) gets solver k's record, status included.
 * Requirements: n in [1, 148] distinct solvers of one device; opts->T_init
 * NULL; opts->profile 0.  Returns NBTE_OK if every solver converged, else
 * the first failing solver's status; every solver's results stay readable. */
int nbte_solve_batch(nbte_solver* const* solvers, int32_t n, const nbte_solve_opts* opts,
                     nbte_solve_info* infos);

/* Results of the last solve, in the caller's cell order, written to the
 * caller's out[n_cells] (both calls return after out is written).  When out
 * is page-locked host memory (cudaHostAlloc, cudaHostRegister) the values
 * are copied into it by DMA directly, else through a pinned staging buffer.
 *   kind 0: lattice temperature T_L after the last update (K);
 *   kind 1: energy temperature sum_l sum_i w_i e / C_tot of the last sweep (K);
 *   kind 2: kinetic pseudo-temperature of the last sweep, Eq. (5), before any
 *           synthetic correction (K).                                      */
int nbte_get_temperature(const nbte_solver* solver, int kind, double* out);
/* Heat flux of the last sweep, Eq. (7): out[n_cells*dim] (W/m^2).          */
int nbte_get_heat_flux(const nbte_solver* solver, double* out);
/* Net outward heat flow through the walls of one tag after the last sweep
 * (W, or W/m in 2D): sum over its faces of sum_l sum_i w_i v_l (s_i.An) e~. */
int nbte_get_wall_heat(const nbte_solver* solver, int32_t tag, double* out);
/* The phonon energy density e'_{band,direction} of the last sweep, Eq. (4):
 * out[n_cells] (J/m^3 per unit solid angle), as the deviation from the
 * equilibrium at T_ref (e' = e - C T_ref / W), in the caller's cell order.
 * Recomputed on the device by re-running the last sweep for the work item
 * holding (direction, band), whose inputs are still resident; valid until
 * the next solve or setter call.  NBTE_ERR_STATE without a previous solve,
 * NBTE_ERR_ARG for an index out of range.                                  */
int nbte_get_distribution(nbte_solver* solver, int32_t direction, int32_t band, double* out);

/* Planner statistics of the current quadrature/mesh (for tuning and tests):
 * stats[0] total levels over all directions, [1] max levels of one
 * direction, [2] max ring slots of one direction, [3] lagged faces,
 * [4] work items, [5] bands per item, [6] value ring (1 shared memory,
 * 2 global memory), [7] device bytes
 * held by the solver, [8] inflow entries per cell record, [9] exported
 * (direction, cell) values, [10] imported wall/lag values, [11] threads per
 * sweep CTA.  With band_group = cta_threads = 0 and bands, quadrature and
 * boundaries set, this runs the layout autotuner first (see
 * nbte_solve_opts), so the layout reported is the one a solve will use.     */
int nbte_plan_stats(nbte_solver* solver, const nbte_solve_opts* opts, int64_t stats[12]);

/* ------------------------------------------------------------- serving ----
 * A request queue in front of the batched iteration (continuous batching).
 * Submitted solves are planned on host threads (n_planners), admitted to the
 * device in arrival order while their estimated device memory fits
 * budget_bytes (0 = 80% of the free device memory at creation; a solve larger
 * than the budget runs alone), and iterated together with every admitted
 * solve as in nbte_solve_batch, at most max_active (1..148) at a time.
 * Arrivals join and converged solves leave between iterations.  Every
 * request uses opts (T_init NULL, profile 0; band_group / cta_threads 0 take
 * the planner's heuristic layout, not the autotuner).  The device is the
 * caller's current device at creation.
 *
 * A submitted solver (mesh, bands, quadrature, boundaries, heat source set)
 * stays owned by the caller, who must not use or destroy it until the
 * request is done.  When done, its results are readable as after
 * nbte_solve_steady (temperature, flux, wall heat); the device memory the
 * iteration held is released (nbte_get_distribution then reports
 * NBTE_ERR_STATE until the solver is solved again).                         */
typedef struct nbte_server nbte_server;
int nbte_server_create(const nbte_solve_opts* opts, size_t budget_bytes, int32_t max_active, int32_t n_planners,
                       nbte_server** out);
/* Queue a solve; *request receives its id.  NBTE_ERR_STATE if the solver is
 * not fully set up or already queued.                                       */
int nbte_server_submit(nbte_server* server, nbte_solver* solver, int64_t* request);
/* *state: 0 queued, 1 planned, 2 running, 3 done.  When done, returns the
 * solve's status, fills info (may be NULL) and seconds[0] = submit-to-done,
 * seconds[1] = submit-to-admission (seconds may be NULL).                   */
int nbte_server_poll(nbte_server* server, int64_t request, int32_t* state, nbte_solve_info* info,
                     double* seconds);
/* Block until every submitted request is done (timeout_s <= 0: no limit;
 * NBTE_ERR_NOT_CONVERGED when the timeout passes first).                    */
int nbte_server_drain(nbte_server* server, double timeout_s);
/* stats[0] batched iterations run, [1] requests submitted, [2] done,
 * [3] estimated device bytes held by admitted requests.                     */
int nbte_server_stats(nbte_server* server, int64_t stats[4]);
/* Stops the threads; requests not yet done are abandoned.                   */
int nbte_server_destroy(nbte_server* server);

/* --------------------------------------------------- allocation-free solve --
 * nbte_laplacian_solve_noalloc: solve A x = rhs for a sparse symmetric
 * positive-definite A by Jacobi-preconditioned conjugate gradients, without
 * allocating any memory.  The paper has no counterpart; this call exists for
 * callers that cannot call cudaMalloc -- e.g. code running inside another
 * framework's memory pool or under a fixed device-memory budget, or a
 * real-time loop where an allocation may block or fail.  It is a one-level
 * variant of the CG kernel that solves the synthetic correction.
 *   n                 rows, 0 <= n <= 262144 (larger n: NBTE_ERR_ARG);
 *                     n = 0 only does the per-device set-up described below
 *                     (the other arguments are then ignored).
 *   row_ptr, col, val the matrix in CSR form, int32 indices, FP64 values,
 *                     DEVICE pointers owned by the caller; every row holds a
 *                     positive diagonal entry (else NBTE_ERR_ARG).
 *   rhs, x            DEVICE arrays of n doubles owned by the caller; x is
 *                     overwritten with the solution (start value 0).
 *   tol, max_iter     stop when |r|_2 <= tol |rhs|_2 (tested on the device
 *                     as r.r <= tol^2 rhs.rhs), at most max_iter steps.
 *   iterations, residual  host outputs (may be NULL); residual is
 *                     |r|_2 / |rhs|_2 of the last iterate.
 *   cuda_stream       cudaStream_t as void* (NULL = legacy default stream);
 *                     the call returns after the solve has finished on it.
 * Working vectors live in one fixed array of about 10 MB in the library's
 * device code.  With lazy module loading (the CUDA default) the driver
 * allocates that array on a device when the first call there loads that
 * code, not when the library is loaded: make a first call (n = 0 suffices)
 * on each device before a memory budget applies; calls after it allocate
 * nothing.  The array then stays allocated on that device until the process
 * exits.  The first call on each device also looks up the array's device
 * address with that device current; make it outside any CUDA stream
 * capture.  All calls on a device share the array and its contents, so calls
 * that overlap on the GPU (other streams, other host threads) race;
 * serialise them.
 * Returns NBTE_OK, NBTE_ERR_ARG, NBTE_ERR_NOT_CONVERGED (x holds the last
 * iterate), NBTE_ERR_DEVICE_TIMEOUT or NBTE_ERR_CUDA.                      */
int nbte_laplacian_solve_noalloc(int n, const int32_t* row_ptr, const int32_t* col, const double* val,
                                 const double* rhs, double* x, double tol, int max_iter, int32_t* iterations,
                                 double* residual, void* cuda_stream);

/* ------------------------------------------------------------ diagnostics --
 * nbte_test_timeouts: every device-side wait of the library is bounded (the
 * sweep's copy pipeline: about a second; the CG grid barriers; the
 * allocation-free solve's barrier); a wait that runs out sets an error word,
 * its kernel returns, and the call reports NBTE_ERR_DEVICE_TIMEOUT.  With
 * on != 0, every such wait of the launches made after this call (in the
 * whole process) runs out: the sweep's producer issues no copy, so its
 * consumers' waits run out on their bound, and the barrier waits give up
 * after one poll.  on = 0 restores normal operation.  For testing the
 * timeout paths.  After a timeout the solver's iterate is incomplete: the
 * next nbte_solve_steady starts again from its initial state even when warm
 * is set.  No paper counterpart.                                          */
int nbte_test_timeouts(int32_t on);

/* Message of the last failing call on this thread (library-owned string). */
const char* nbte_last_error(void);
/* Library version string. */
const char* nbte_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NBTE_H */
