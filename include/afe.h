/*
 * afe.h - C ABI of the GB300 (sm_103a) quadrature-free ADER-AFE-DG step on 3D polyhedral meshes.
 *
 * The operation is one explicit ADER step of the agglomerated-finite-element (AFE)
 * discontinuous Galerkin scheme of arXiv 2605.00619 over every polyhedral cell:
 *   - artificial-viscosity detector (Sec. 4.5, Eqs. divergence3D and beta3D),
 *   - CFL time step (Sec. 4.2, Eq. timestep),
 *   - element-local space-time Galerkin predictor, a fixed-point iteration on the
 *     cell's continuous nodal subgrid DOFs (Sec. 4.3, Eqs. ADER-localCauchy, ader4),
 *   - time-integrated predictor and fluxes (Eq. TAvectors),
 *   - Rusanov fluxes on the sub-triangles of each polygonal face (Sec. 4.4, Eq. 3.33),
 *   - corrector update M_i (u^{n+1} - u^n) = volume term - face term (Sec. 4.4).
 *
 * Conventions shared by every entry point
 *   - Every call returns an afe_status; outputs go through out-parameters.
 *   - On error a message is available from afe_last_error() (thread-local), and the
 *     mesh handle keeps its last valid state.
 *   - The library copies every input array; the caller owns all host buffers and the
 *     handle owns all device memory it allocates.  Device pointers passed in
 *     (afe_set_state_device, afe_get_state_device) stay owned by the caller.
 *   - Conserved variables are ordered (rho, rho*u, rho*v, rho*w, rho*E); states are
 *     node-major [n_nodes][5] FP64.  The node order is the library's own: contiguous per
 *     cell (cell i owns nodes node_ptr[i] .. node_ptr[i+1]-1); afe_get_node_coords gives
 *     their positions, so initial data is set by nodal interpolation there.
 *   - All GPU work of a handle runs on its stream (afe_mesh_create's cuda_stream, or
 *     afe_set_stream); entry points that return host data synchronise that stream.
 *   - There is no CPU fallback: without a usable CUDA device every call that needs the
 *     GPU returns AFE_ECUDA.
 */
#ifndef AFE_H
#define AFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AFE_OK = 0,
  AFE_EINVAL = 1,     /* bad argument (null pointer, size, unsupported option)           */
  AFE_EMESH = 2,      /* invalid mesh: degenerate sub-tet, non-conforming subgrid, a cell
                         whose subgrid is not a ball, an unmatched face on a periodic mesh */
  AFE_ENOMEM = 3,     /* device or host allocation failed                                  */
  AFE_ECUDA = 4,      /* CUDA runtime error (message names the call)                       */
  AFE_ENOCONV = 5,    /* the predictor hit picard_max in at least one cell (step applied)   */
  AFE_ENONFINITE = 6, /* NaN/Inf or non-positive density or pressure after the step        */
  AFE_ETIMEOUT = 7    /* a bounded wait on device progress gave up                          */
} afe_status;

typedef enum { AFE_EULER = 0, AFE_NAVIER_STOKES = 1 } afe_equations;
/* AFE_FP64: every step of the path in FP64.  AFE_FP32: predictor, face fluxes and the
 * corrector's inverse-mass apply in FP32, with FP64 master state, FP64 CFL reduction and
 * an FP64 correction of each cell's conserved totals. */
typedef enum { AFE_FP64 = 0, AFE_FP32 = 1 } afe_precision;
typedef enum { AFE_BC_PERIODIC = 0, AFE_BC_TRANSMISSIVE = 1 } afe_bc;

typedef struct {
  int order;          /* polynomial degree N in {1, 2, 3, 4} (Sec. 4.1, App. A); at N = 4 the
                         cells (about 1,100 nodes) exceed the FP32 shared-memory predictor and
                         both forms run the global-scratch kernels                            */
  int equations;      /* afe_equations; Euler ignores mu, Pr, kappa unless the limiter adds mu */
  int precision;      /* afe_precision                                                         */
  double gamma;       /* ratio of specific heats (Sec. 2)                                      */
  double R;           /* gas constant; c_v = R / (gamma - 1)                                  */
  double mu;          /* dynamic viscosity (Navier-Stokes)                                     */
  double Pr;          /* Prandtl number, used when kappa < 0                                   */
  double kappa;       /* heat conduction; < 0 selects kappa_i = mu_i * gamma * c_v / Pr        */
  double cfl;         /* CFL number of Eq. timestep                                            */
  int limiter;        /* 1: artificial-viscosity limiter of Sec. 4.5                            */
  double m1;          /* detector constant m_1 of Eq. beta3D (0.1 in the paper)                */
  double picard_tol;  /* stop when max|q^{r+1}-q^r| <= tol * max(1, max|q^r|), per cell       */
  int picard_max;     /* iteration cap; hitting it is reported as AFE_ENOCONV                  */
  double period[3];   /* domain period per axis; used for sub-tet vertices with image shifts   */
  int visc_dt_subtet; /* 0: the viscous term of Eq. timestep uses the cell length h_i, as printed;
                         1: it uses the cell's smallest sub-tet length min_k 6|T_k|/|dT_k|,
                         a stricter bound: the explicit step of the viscous terms scales
                         with the square of the smallest sub-tet size, and on subgrids with
                         thin sub-tets viscous or limited runs stay finite only with it       */
  int h_diameter;     /* 0: h_i = 6|P_i| / |dP_i| (insphere-equivalent diameter; Sec. 4.2 leaves the
                         length open); 1: h_i = the cell's diameter, the largest distance
                         between two of its vertices (the example Sec. 4.2 names).  h_i enters
                         the time step (Eq. timestep), the face penalty of Eq. 3.33 and the
                         artificial viscosity of Sec. 4.5                                    */
} afe_params;

typedef struct {
  double dt;            /* last time step                                        */
  double t;             /* accumulated simulation time                           */
  int64_t steps;        /* completed steps                                       */
  double picard_mean;   /* mean predictor iterations over cells, last step       */
  int32_t picard_max;   /* max predictor iterations over cells, last step        */
  int64_t nonconverged; /* cell-steps that hit picard_max since the last afe_step /
                           afe_sync (one step after afe_step)                     */
  int64_t troubled;     /* cell-steps with beta_i > 0, same span                  */
  double totals[5];     /* sum_i 1^T M_i u_i per conserved variable (FP64)       */
  int64_t kernel_launches; /* kernels launched by afe_step / afe_step_async so far */
} afe_stats;

typedef struct afe_mesh afe_mesh; /* opaque; owns all device memory of one simulation */

/* Fill *p with the paper's settings (Sec. 5: gamma 1.4, R 1, kappa 0, CFL 0.3, m_1 0.1,
 * tolerance 1e-12) for degree `order`, FP64, Euler, no limiter, picard_max 64. */
afe_status afe_default_params(afe_params* p, int order);

/* Build a mesh from polyhedra and their tetrahedral subgrid (Sec. 4.1) and run the FP64
 * set-up on the GPU: sub-tet Jacobians, cell mass matrices M_i (Sec. 4.4), their inverses
 * (stored per cell, Sec. 4.3), face matching, characteristic lengths.
 *   xyz             [n_vertices][3] vertex positions (host).
 *   cell_subtet_ptr [n_cells + 1] CSR offsets into the sub-tets (host); n_subtets = ptr[n_cells].
 *   subtet_vtx      [n_subtets][4] global vertex ids (host).
 *   subtet_shift    [n_subtets][4][3] periodic image of each sub-tet vertex, or NULL; a vertex
 *                   sits at xyz[id] + shift * period (host).
 *   boundary        afe_bc: periodic (every cell-boundary triangle must be matched) or
 *                   transmissive (unmatched triangles are domain boundary, outer state = inner).
 *   cuda_stream     cudaStream_t for all work of the handle (NULL = legacy default stream).
 * Sub-tets with negative orientation are reoriented; a zero-volume sub-tet, a non-conforming
 * subgrid or a cell that is not a topological ball returns AFE_EMESH. */
afe_status afe_mesh_create(const afe_params* p, int64_t n_vertices, const double* xyz,
                           int64_t n_cells, const int64_t* cell_subtet_ptr,
                           const int64_t* subtet_vtx, const int8_t* subtet_shift, int boundary,
                           void* cuda_stream, afe_mesh** out);

/* Host-only validation of the same inputs as afe_mesh_create (no GPU is touched): builds the
 * topology and returns AFE_OK, AFE_EINVAL or AFE_EMESH, with the number of AFE nodes and of
 * cell-boundary sub-triangles in *n_nodes / *n_face_tris (either may be NULL). */
afe_status afe_mesh_validate(const afe_params* p, int64_t n_vertices, const double* xyz,
                             int64_t n_cells, const int64_t* cell_subtet_ptr,
                             const int64_t* subtet_vtx, const int8_t* subtet_shift, int boundary,
                             int64_t* n_nodes, int64_t* n_face_tris);

/* Number of AFE nodes (DOF points) and, if node_ptr is not NULL, the per-cell offsets
 * [n_cells + 1] (host). */
afe_status afe_num_nodes(const afe_mesh* m, int64_t* n_nodes, int64_t* node_ptr);

/* Node positions [n_nodes][3] (host); nodes of cells touching a periodic boundary are given
 * in the frame of their own cell. */
afe_status afe_get_node_coords(const afe_mesh* m, double* xyz);

/* Replace the stream used by the handle. */
afe_status afe_set_stream(afe_mesh* m, void* cuda_stream);

/* Set the conserved state u^n from a host array [n_nodes][5] FP64 (synchronous copy). */
afe_status afe_set_state(afe_mesh* m, const double* q);

/* Set the state from a device array [n_nodes][5] FP64, ordered on `cuda_stream`
 * (NULL = the handle's stream); the copy is device-to-device and asynchronous. */
afe_status afe_set_state_device(afe_mesh* m, const double* dq, void* cuda_stream);

/* Copy the state to a host array [n_nodes][5] FP64 (synchronises the handle's stream). */
afe_status afe_get_state(const afe_mesh* m, double* q);

/* Copy the state to a device array [n_nodes][5] FP64 on the handle's stream (asynchronous). */
afe_status afe_get_state_device(const afe_mesh* m, double* dq);

/* CFL time step of Eq. timestep at the current state (FP64 reduction on the GPU; includes
 * the limiter's artificial viscosity when the limiter is on). */
afe_status afe_compute_dt(afe_mesh* m, double* dt);

/* One ADER-AFE-DG step.  dt > 0: use it; dt <= 0: the CFL time step, computed and kept on
 * the device.  Waits for the step and returns AFE_ENOCONV / AFE_ENONFINITE if a cell did
 * not converge or the new state is not admissible (the step is applied either way). */
afe_status afe_step(afe_mesh* m, double dt);

/* `nsteps` steps enqueued back to back on the handle's stream with no host synchronisation
 * between them (dt as in afe_step); returns after enqueueing.  Status flags accumulate over
 * the steps enqueued since the last afe_step / afe_sync and are reported by afe_get_stats /
 * afe_sync. */
afe_status afe_step_async(afe_mesh* m, double dt, int nsteps);

/* Wait for the handle's stream and return the accumulated status of afe_step_async calls
 * (AFE_OK, AFE_ENOCONV or AFE_ENONFINITE), clearing it. */
afe_status afe_sync(afe_mesh* m);

/* Statistics of the last step plus FP64 conserved totals of the current state. */
afe_status afe_get_stats(const afe_mesh* m, afe_stats* s);

/* Diagnostics of the last step (host arrays, NULL to skip): the time-integrated predictor
 * q_bar at every node [n_nodes][5] (Eq. TAvectors; recorded only after
 * afe_set_diagnostics(m, 1)), predictor iterations per cell [n_cells], beta_i and mu_i per
 * cell [n_cells]. */
afe_status afe_set_diagnostics(afe_mesh* m, int on);
afe_status afe_get_diagnostics(const afe_mesh* m, double* qbar, int32_t* iterations,
                               double* beta, double* mu);

/* Per-stage device timing.  With profiling on, every step records CUDA events on the
 * handle's stream around its stages; afe_stage_times adds up the elapsed milliseconds of all
 * steps since the last reset into ms[4] = {limiter + time step, predictor, face fluxes,
 * corrector} and the number of steps into *nsteps, synchronising the stream (reset != 0
 * clears the record). */
afe_status afe_set_profiling(afe_mesh* m, int on);
afe_status afe_stage_times(afe_mesh* m, double* ms, int64_t* nsteps, int reset);

/* How the handle's step runs (a host-side report; no GPU work).  The FP32 form keeps each
 * cell's fixed-point iteration in the shared memory of one predictor block when the cell fits
 * (fp32_shared = 1): the right-hand side of Eq. ader4 is formed in chunks of sub-tets (16 per
 * chunk at N = 2, 3 when the cell leaves room for them, else 8: a "narrow" cell) and M_i^-1
 * streams through a ring of stages of 32 rows (in the tensor-memory form 16 or 8 rows when a
 * large cell leaves less room; as many stages as fit, at most 8; a cell whose N_i is not a
 * multiple of the stage height ends with a partial, "masked" stage).  Meshes whose largest cell
 * does not fit that plan run the FP32 form with global-memory scratch on the CUDA cores
 * (fp32_shared = 0), as does, always, the FP64 form. */
typedef struct {
  int32_t fp32_shared;     /* 1: FP32 shared-memory predictor (M_i^-1 apply on the tensor cores)  */
  int32_t corrector_block; /* 1: FP32 corrector with one block per cell                           */
  int64_t smem_bytes;      /* dynamic shared memory of one predictor block (0 when not used)     */
  int32_t max_nodes;       /* largest N_i                                                          */
  int32_t max_subtets;     /* most sub-tets in one cell                                            */
  int32_t ring_min;        /* fewest M_i^-1 stages in the ring over the cells (the largest cell)   */
  int32_t ring_max;        /* most stages over the cells                                           */
  int64_t narrow_cells;    /* cells whose right-hand side takes the narrow chunks                  */
  int64_t masked_cells;    /* cells whose last M_i^-1 stage is partial                             */
  int32_t tcgen05;         /* 1: the M_i^-1 apply runs on the 5th-generation tensor cores with
                              tensor memory (tcgen05); 0: on the warp-level mma.sync path          */
  int32_t stage_rows_min;  /* shortest M_i^-1 ring stage over the cells (32, 16 or 8 rows)        */
} afe_plan;
afe_status afe_plan_info(const afe_mesh* m, afe_plan* out);

/* Which form of the FP32 predictor's M_i^-1 apply a handle uses: 0 (the default) the
 * warp-level mma.sync form; 1 the form on the 5th-generation tensor cores with tensor memory
 * (tcgen05), for meshes whose every cell fits its shared-memory plan (up to 640 nodes per cell;
 * else AFE_EINVAL).  Both compute the same 3xTF32 product (results agree to FP32 rounding, not
 * bit for bit); on the measured workloads the mma.sync form is the faster one.  A batch takes
 * the tensor-memory form only when every member asks for it.  Other values: AFE_EINVAL. */
afe_status afe_set_predictor_variant(afe_mesh* m, int32_t variant);

/* Poll limit of the first bounded wait the FP32 shared-memory predictor makes for every cell
 * (for the cell's sub-tet records to arrive in shared memory; default 1048576 polls, far
 * beyond the time the copy takes).  A wait that runs out makes the block wait, with the
 * default limit, for the copy it issued, leave the kernel, and the step report
 * AFE_ETIMEOUT; the state of the handle is then undefined.  polls = 0 gives up at once:
 * it exists to exercise that failure path.  Batches copy the setting when created.
 * polls < 0 returns AFE_EINVAL. */
afe_status afe_set_wait_limit(afe_mesh* m, int32_t polls);

/* How the FP32 shared-memory predictor schedules its work; the paper has no counterpart (it
 * concerns the launch, not the method).  Every setting leaves each cell's arithmetic unchanged
 * except `variant`, so results are bit for bit the same across cost_order, ring_cap and narrow.
 *   cost_order  1: the persistent predictor blocks take cells in decreasing order of their
 *               estimated cost per fixed-point iteration (S Nt Np (155 + 30 Np) + 10 Nt N_i^2
 *               flops; ties in index order), so that the last cells of a launch are cheap ones
 *               and the blocks finish together (the cells of a batch are bucketed by cost across
 *               its members); 0: index order.
 *   variant     0: mma.sync form of the M_i^-1 apply; 1: tcgen05 / tensor-memory form (only if
 *               every cell fits its plan; see afe_set_predictor_variant).
 *   ring_cap    most M_i^-1 stages in flight in the ring (0: as many as fit, at most 8).
 *   narrow      1: right-hand side in chunks of 8 sub-tets even where 16 fit.
 * Other values: AFE_EINVAL. */
typedef struct {
  int32_t cost_order;
  int32_t variant;
  int32_t ring_cap;
  int32_t narrow;
} afe_schedule;
afe_status afe_set_schedule(afe_mesh* m, const afe_schedule* s);
afe_status afe_get_schedule(const afe_mesh* m, afe_schedule* s);

/* Choose the schedule by measurement: with the time step of the current state computed on the
 * device, every candidate (cost_order 0/1; variant 0, and 1 where the cells fit; ring_cap 0 or
 * 2; narrow 0, and 1 where wide chunks are used) times `trials` launches of the predictor alone
 * (CUDA events on the handle's stream; the predictor writes only per-step intermediates, so
 * the state is unchanged), and the fastest is set.  *best receives it, *best_ms and
 * *default_ms (either may be NULL) the mean predictor time with it and with the default
 * schedule {0, 0, 0, 0}.  The choice is remembered per mesh signature (order, cells and their
 * node and sub-tet counts) for this process: a later call on an equal mesh only sets it.
 * Synchronises the stream.  FP32 handles with the shared-memory predictor only (else
 * AFE_EINVAL); trials in 1..64. */
afe_status afe_autotune(afe_mesh* m, int trials, afe_schedule* best, double* best_ms, double* default_ms);

/* The two reductions of the CFL time step (Sec. 4.2) over the first `n_cells` cells of the
 * handle, for stepping one mesh partitioned over several handles (ranks) with one global time
 * step: with the limiter's viscosity of the current state (Sec. 4.5), *bracket_max receives the
 * largest |lambda| + 2 |lambda^v| (2N+1)/h over the nodes of those cells and *h_min their
 * smallest characteristic length.  The caller combines them over the ranks (max, min) and
 * steps every rank with dt = cfl * h_min / ((2N+1) * bracket_max), the expression the library
 * evaluates itself for a single mesh.  Synchronises the handle's stream; 1 <= n_cells <= the
 * handle's cells, else AFE_EINVAL; an inadmissible state returns AFE_ENONFINITE. */
afe_status afe_cfl_pieces(afe_mesh* m, int64_t n_cells, double* bracket_max, double* h_min);

/* Conserved totals of a caller-provided device state, with no device memory allocated by the
 * call.  The paper has no counterpart: this serves callers that must not call cudaMalloc at
 * the point of use, e.g. code running inside a framework whose caching allocator owns all
 * device memory, or a loop that has to stay free of allocation and the implicit device
 * synchronisation cudaMalloc/cudaFree bring.
 *   m        handle created earlier (its node weights w_i = M_i 1 are read).
 *   dq       device array [n_nodes][5] FP64, the state to sum (caller-owned).
 *   dtotals  device array [5] FP64 receiving sum_i w_i . u_i per conserved variable.
 *   cuda_stream  stream to run on (NULL = the handle's stream); the call is asynchronous.
 * The partial sums live in a fixed device array inside the library (AFE_NOALLOC_MAX_PARTIALS
 * partials of AFE_NOALLOC_CHUNK nodes each, 160 KiB, held by every GPU that loads the library
 * until the process exits), so meshes with more than AFE_NOALLOC_MAX_NODES nodes are rejected
 * with AFE_EINVAL.  The first call on a device looks up that array's device address; make
 * that first call before any stream capture (a first call on a capturing stream returns
 * AFE_EINVAL and does nothing).  All calls share the one array: calls that
 * overlap on the GPU (different streams, no ordering between them) race and must not be
 * issued.  Nothing in the array needs to start at zero: each call writes every partial it
 * reads. */
#define AFE_NOALLOC_CHUNK 65536
#define AFE_NOALLOC_MAX_PARTIALS 4096
#define AFE_NOALLOC_MAX_NODES ((int64_t)AFE_NOALLOC_CHUNK * AFE_NOALLOC_MAX_PARTIALS)
afe_status afe_conserved_totals_noalloc(const afe_mesh* m, const double* dq, double* dtotals,
                                        void* cuda_stream);

/* ---- Several simulations advanced together ------------------------------------------
 * The paper advances one mesh; it has no counterpart for this.  A batch advances up to
 * AFE_MAX_BATCH independent handles -- each with its own mesh, state, parameters, dt and
 * time -- with one kernel launch per stage over all their cells, so that many small
 * simulations occupy the GPU the way one large mesh does.  Every kernel works per cell, per
 * polygonal face or per member, and the CFL maximum is an order-independent integer
 * atomicMax, so each member's result is bit-identical to stepping it alone.
 * Requirements (else AFE_EINVAL): every member AFE_FP32 with the same order N, on the
 * current device, with cells small enough for the shared-memory FP32 kernels, and the
 * members' largest cells fitting that shared-memory plan together.
 * Ownership: members keep owning their memory and must outlive the batch; the batch owns a
 * work counter, its CUDA graph and, when created with cuda_stream NULL, a non-blocking
 * stream of its own.  afe_batch_create waits for the members' streams; afterwards the batch
 * orders all its work on its stream, so a member must not be stepped on its own between
 * afe_batch_step_async and afe_batch_sync. */
#define AFE_MAX_BATCH 64
typedef struct afe_batch afe_batch;

afe_status afe_batch_create(afe_mesh* const* members, int n_members, void* cuda_stream,
                            afe_batch** out);

/* Enqueue `nsteps` steps of every member (dt <= 0: each member its own CFL step; dt > 0: that
 * step for all).  use_graph != 0: one step is captured into a CUDA graph on first use (again
 * when dt changes) and the graph is launched nsteps times; otherwise the kernels are
 * launched directly.  Returns after enqueueing; status flags accumulate until
 * afe_batch_sync. */
afe_status afe_batch_step_async(afe_batch* b, double dt, int nsteps, int use_graph);

/* Wait for the batch stream.  member_status[n_members] (NULL to skip) receives each member's
 * status over the steps since the last sync (AFE_OK, AFE_ENOCONV, AFE_ENONFINITE or
 * AFE_ETIMEOUT); the return value is the most severe of them.  Each member's time, step
 * count and last dt (afe_get_stats) are brought up to date. */
afe_status afe_batch_sync(afe_batch* b, int* member_status);

/* The schedule of a batch's predictor (see afe_schedule; the cost order runs over the cells of
 * all members together) and its measured choice (as afe_autotune, on the batch).  Setting a
 * schedule drops the batch's captured graph (it is captured again on the next step). */
afe_status afe_batch_set_schedule(afe_batch* b, const afe_schedule* s);
afe_status afe_batch_autotune(afe_batch* b, int trials, afe_schedule* best, double* best_ms,
                              double* default_ms);

/* Total cells and nodes of the members, kernels launched so far (counted one by one, also
 * when they ran inside graphs) and graph launches (NULL to skip any). */
afe_status afe_batch_info(const afe_batch* b, int64_t* n_cells, int64_t* n_nodes,
                          int64_t* launches, int64_t* graph_launches);

/* Wait for the batch stream and release the batch (not its members; NULL is ignored). */
void afe_batch_destroy(afe_batch* b);

/* Bytes of device memory held by the handle. */
afe_status afe_device_bytes(const afe_mesh* m, int64_t* bytes);

/* Message of the last failed call on this thread ("" if none). */
const char* afe_last_error(void);

/* Release the handle and all its device memory (NULL is ignored). */
void afe_mesh_destroy(afe_mesh* m);

#ifdef __cplusplus
}
#endif

#endif /* AFE_H */
