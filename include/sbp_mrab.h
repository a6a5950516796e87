/*
 * sbp_mrab.h -- C ABI of the GB300 library for multi-rate Adams-Bashforth time integration of
 * the SBP-SAT discretised compressible Euler / Navier-Stokes equations on two overset
 * structured meshes (arXiv 1805.06607, "Multi-Rate Time Integration on Overset Meshes").
 *
 * Conventions
 *  - Every call returns an sbp_status; nothing throws across the ABI. sbp_status_string()
 *    names a status; sbp_last_error_message() gives detail for the calling thread's last
 *    failure (a CUDA error string, the offending argument, ...).
 *  - Device memory for states, histories and right-hand sides is owned by the caller and
 *    passed as plain device pointers. The library owns the tables it derives at creation
 *    (class maps, metrics, SAT lists, donor stencils) and a small device error word; they
 *    are freed by sbp_system_destroy.
 *  - Fields are structure-of-arrays: variable v of point (i, j) sits at
 *    base[v * field_elems + j * pitch + i], i fastest, with pitch and field_elems from
 *    sbp_mesh_info. nvar = 4 in 2D: (rho, rho u, rho v, rho E). The element type is double
 *    for SBP_F64 systems and float for SBP_F32 systems, fixed at creation.
 *  - Streams are cudaStream_t values passed as void*; NULL means the legacy default stream.
 *    Calls that return host results (sbp_timestep, sbp_check) synchronise that stream.
 *  - A system is not thread-safe; use one system per host thread.
 */
#ifndef SBP_MRAB_H
#define SBP_MRAB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbp_system_s *sbp_system_t;

typedef enum {
  SBP_OK = 0,
  SBP_ERR_ARG = -1,       /* null pointer, bad enum or size */
  SBP_ERR_SHAPE = -2,     /* mesh too small, non-positive cell volume, inconsistent sizes */
  SBP_ERR_DTYPE = -3,     /* element type not supported for the requested call */
  SBP_ERR_CUDA = -4,      /* a CUDA runtime call failed (detail in the message) */
  SBP_ERR_NONFINITE = -5, /* a kernel met a non-finite or non-physical state */
  SBP_ERR_DONOR = -6,     /* no valid donor stencil for a receiver */
  SBP_ERR_TIMEOUT = -7,   /* a bounded device wait gave up */
  SBP_ERR_BOUNDS = -8,    /* a kernel index check failed */
  SBP_ERR_STATE = -9      /* call out of order (e.g. stepping before sbp_mrab_init) */
} sbp_status;

enum { SBP_BC_PERIODIC = 0, SBP_BC_INTERFACE = 1, SBP_BC_FARFIELD = 2, SBP_BC_WALL = 3 };
enum { SBP_EULER = 0, SBP_NS = 1 };
enum { SBP_F64 = 0, SBP_F32 = 1 };

/* One structured 2D mesh. Faces are ordered i-low, i-high, j-low, j-high. A periodic direction
 * must have SBP_BC_PERIODIC on both of its faces. Curvilinear meshes give host coordinate
 * arrays x, y of nj*ni points (i fastest; copied at creation). Cartesian meshes may leave x, y
 * NULL and give lo/h instead. shift is the coordinate jump across a periodic wrap:
 * (dx, dy) when i wraps, then (dx, dy) when j wraps (0 for a closed O-grid). */
typedef struct {
  int n[2];
  int periodic[2];
  int bc[4];
  int cartesian;
  double lo[2], h[2];
  const double *x, *y;
  double shift[4];
} sbp_mesh_desc;

/* Physics, penalties and integrator. Non-dimensionalisation: rho_inf = 1, c_inf = 1,
 * T = gamma p / rho; mu is the viscous coefficient (Mach/Re), constant, with Stokes' lambda =
 * -2/3 mu and heat conductivity mu / (Pr (gamma - 1)). qinf is the far-field state. The
 * integrator is MRAB of order `order` with `hist_len` >= order history values (extended
 * history when larger), step ratio H/h = step_ratio >= 1, mesh `fast_mesh` advancing at the
 * micro step. hole_cells: background points farther than hole_cells background spacings
 * inside the fine mesh's outer boundary are holes. */
typedef struct {
  int physics;
  int dtype;
  double gamma, mu, pr, twall;
  double omega_corner;           /* Omega of Sec. 4.2 eq. (penalty_interp) at corner receivers */
  double sigma_interface;        /* sigma^I of eq. (int); the paper uses 1/2 */
  double sigma_physical;         /* sigma^I of the far-field and wall penalties */
  double cfl;
  double qinf[4];
  int order, hist_len, step_ratio, fast_mesh;
  double hole_cells;             /* hole margin in background spacings (<= 0: 4) */
  int scheme;                    /* MRAB ordering, an sbp_mrab_scheme (0: the paper's) */
  /* Sponge layer at far-field faces (Sec. 5.1: sponge boundaries of a given depth in cells;
   * the form is cited, not printed). Within sponge_cells (0: off, at most 16) points of a
   * far-field face the right-hand side gains -sigma (q - qinf), sigma = sponge_strength
   * ((D - d) / D)^2 for the index distance d < D = sponge_cells to the nearest far-field face.
   * 2D systems and chains, 3D Cartesian systems (distance to the nearest of their far-field
   * faces) and the background of a 3D curvilinear pair. Forward paths only: the adjoint calls
   * reject a system with a sponge. */
  int sponge_cells;
  double sponge_strength;
} sbp_params;

/* The orderings of a macro step that Sec. 3.3 lists as design choices. The paper's runs use
 * fastest-first without re-extrapolation (the default): the fast micro steps take the slow
 * state from the slow extrapolant, and the slow right-hand side at t + H is evaluated with the
 * fast state reached at t + H. The slowest-first variants advance the slow state first and
 * evaluate the slow right-hand side at t + H with the fast state extrapolated over the macro
 * step (fast history ending at t); the fast micro steps then take the slow state from the
 * slow extrapolant of the history ending at t (SLOWEST_FIRST: the slow right-hand side runs
 * beside the fast micro steps) or re-extrapolated from the history ending at t + H
 * (SLOWEST_FIRST_REEXTRAPOLATE). All take one slow and step_ratio fast right-hand sides per
 * macro step. 3D systems, batches and the adjoint support fastest-first only. */
typedef enum {
  SBP_MRAB_FASTEST_FIRST = 0,
  SBP_MRAB_SLOWEST_FIRST = 1,
  SBP_MRAB_SLOWEST_FIRST_REEXTRAPOLATE = 2
} sbp_mrab_scheme;

typedef struct {
  int ni, nj, pitch;
  size_t field_elems;   /* elements of one variable plane: pitch * nj */
  size_t state_bytes;   /* nvar planes */
  size_t hist_bytes;    /* hist_len * state_bytes */
  int nvar, n_holes, n_receivers, n_sat_points;
  int elem_size;        /* 8 (F64) or 4 (F32) */
  int strip_width;      /* columns per CTA of the right-hand-side kernel */
  int rows_per_cta;     /* rows per CTA (chosen by the autotuner, see sbp_autotune) */
  int single_pass;      /* 1: the single-pass marching kernel (rows_per_cta = its chunk of rows);
                           0: the flux + derivative kernel pair */
  int rows_update;      /* kernel pair: rows per CTA of the derivative (update) kernel, 4..32 */
  /* The four fields above describe the kernels of the fused right-hand side + MRAB update
   * (sbp_mrab_step); these describe those of the right-hand side alone (sbp_rhs_eval,
   * sbp_rhs_eval_noalloc, Runge-Kutta stages), which the autotuner chooses separately. */
  int eval_strip_width, eval_rows_per_cta, eval_single_pass, eval_rows_update;
} sbp_mesh_info;

/* Create a two-mesh overset system (mesh 0 = background, mesh 1 = the overset fine mesh) and
 * run its setup (Sec. 2.2 and Sec. 4.1): hole cut, SBP segment classes, metrics (computed on
 * the device by the derivative operator), SAT lists, donor search and Lagrange weights, and
 * the Adams-Bashforth / MRAB coefficient plan (Sec. 3.1-3.3). Synchronous. Each mesh needs
 * 8..65535 points per direction (SBP_ERR_SHAPE otherwise: the closures need 8 points, and the
 * point tables pack (i, j) into 16 bits each). */
sbp_status sbp_system_create(const sbp_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                             sbp_system_t *out);
sbp_status sbp_system_destroy(sbp_system_t sys);
sbp_status sbp_mesh_info_get(sbp_system_t sys, int mesh, sbp_mesh_info *info);

/* The host part of sbp_system_create alone (no device calls, so it also runs on a machine
 * without a GPU): the same argument checks, hole cut, SBP segment classes, SAT lists, donor
 * search with Lagrange weights (Sec. 2.2) and the Adams-Bashforth / MRAB coefficient plan
 * (Sec. 3.1-3.3), for inspection and tests. Errors as sbp_system_create. */
typedef struct sbp_host_tables_s *sbp_host_tables_t;
sbp_status sbp_host_tables_create(const sbp_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                  sbp_host_tables_t *out);
sbp_status sbp_host_tables_destroy(sbp_host_tables_t tables);
/* iblank (ni*nj bytes), receivers, donor_base, donor_w as in sbp_get_tables; n_receivers
 * (host int) the receiver count. Any output pointer may be NULL. */
sbp_status sbp_host_tables_get(sbp_host_tables_t tables, int mesh, signed char *iblank, int *receivers,
                               int *donor_base, double *donor_w, int *n_receivers);
/* The coefficient plan on unit steps: ab (m doubles) the weights of one Adams-Bashforth step
 * over [0, 1] on the history nodes -(m-1)..0 (oldest first); ext (sr*m doubles, row j) the slow
 * extrapolant's weights integrated over [0, j/sr] on the same nodes (row 0 zero); m, sr (host
 * ints) the history length and step ratio. Any output pointer may be NULL. */
sbp_status sbp_host_tables_plan(sbp_host_tables_t tables, double *ab, double *ext, int *m, int *sr);

/* Setup tables copied to host memory, for inspection and tests.
 *  iblank: nj*ni bytes (1 active, 0 hole). metrics: 5*nj*ni doubles, planes
 *  (xi_x/J, xi_y/J, eta_x/J, eta_y/J, J). receivers: n_receivers point indices j*ni+i;
 *  donor_base: 2 ints per receiver (i0, j0) on the other mesh; donor_w: 8 doubles per receiver
 *  (4 Lagrange weights along i, then 4 along j). Any output pointer may be NULL. */
sbp_status sbp_get_tables(sbp_system_t sys, int mesh, signed char *iblank, double *metrics,
                          int *receivers, int *donor_base, double *donor_w);

/* Donor-cell Lagrange interpolation (Sec. 2.2; Sec. 3.3 step 2 for the extrapolated state):
 * for each receiver r of recv_mesh, qhat[v*n_receivers + r] = sum over the 4x4 donor stencil
 * of w_i w_j q_donor. With NS physics and fvhat != NULL also the six Cartesian viscous-flux
 * components (F^V_x then F^V_y; momentum x, momentum y, energy) interpolated the same way into
 * fvhat[c*n_receivers + r]. q_donor is a full state of the other mesh (device). qhat, fvhat:
 * device, caller-owned. */
sbp_status sbp_overset_interp(sbp_system_t sys, int recv_mesh, const void *q_donor, void *qhat,
                              void *fvhat, void *stream);

/* Right-hand side dq/dt of one mesh (Sec. 2.2 eq. (int)): metric-weighted inviscid and
 * viscous fluxes, SBP 4-2 derivatives with segment closures, physical and interface SAT
 * penalties, the interface values interpolated from q_other. rhs: device, caller-owned,
 * same layout as q_self; holes get 0. */
sbp_status sbp_rhs_eval(sbp_system_t sys, int mesh, const void *q_self, const void *q_other, void *rhs,
                        void *stream);

/* sbp_rhs_eval for callers that cannot have device memory allocated for them while they run:
 * a process whose device memory is all reserved up front by another allocator (a framework's
 * caching pool), or a latency-critical loop in which the device-wide synchronisation that
 * cudaMalloc and cudaFree imply is not acceptable. The paper has no counterpart; the result
 * equals sbp_rhs_eval's. The
 * receiver workspace (interpolated states and viscous fluxes) lives in one fixed device array
 * of SBP_NOALLOC_MAX_RECEIVERS * 10 doubles (640 KiB) that the library defines and that every
 * GPU loading the library keeps until the process exits; the call allocates and frees nothing.
 * Meshes with more receivers than SBP_NOALLOC_MAX_RECEIVERS get SBP_ERR_SHAPE. All calls share
 * the array and nothing in it needs to start at zero (the gather overwrites each entry it later
 * reads); calls that overlap on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller. The first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream capture. */
#define SBP_NOALLOC_MAX_RECEIVERS 8192
sbp_status sbp_rhs_eval_noalloc(sbp_system_t sys, int mesh, const void *q_self, const void *q_other, void *rhs,
                                void *stream);

/* Stable step estimate of Sec. 4.1 eqs. (ts_inv), (ts_visc), (ts_overall) on both meshes for
 * the given states, without the CFL factor (dt_mesh[2], host), and the macro step
 * H = min(cfl dt_slow, step_ratio cfl dt_fast) (host). Synchronises the stream. */
sbp_status sbp_timestep(sbp_system_t sys, const void *q_mesh0, const void *q_mesh1, double *dt_mesh,
                        double *H, void *stream);

/* Bind caller-owned device buffers for the time integrator: per mesh two state buffers (the
 * integrator alternates between them) and one history ring of hist_len states. */
sbp_status sbp_bind(sbp_system_t sys, int mesh, void *q_a, void *q_b, void *hist);
/* Device pointer of the bound buffer that holds mesh's current state. */
sbp_status sbp_current_state(sbp_system_t sys, int mesh, void **q);

/* Bootstrap (Sec. 3.1): Heun's third-order Runge-Kutta at the micro step h = H/step_ratio for
 * (hist_len-1)*step_ratio steps from the current bound states, recording the fast right-hand
 * side every micro step and the slow one every macro step. H <= 0 takes H from sbp_timestep
 * on the initial states. Allocates and frees its own stage buffers. */
sbp_status sbp_mrab_init(sbp_system_t sys, double H, void *stream);

/* n macro steps of the fastest-first MRAB scheme without re-extrapolation (Sec. 3.3, Steps
 * 1-7, any integer step ratio). Per macro step: interpolate the fast state to the slow
 * receivers; slow RHS fused with the slow state update; then step_ratio fused fast RHS +
 * fast updates, each fed by the slow extrapolant at its micro time. Asynchronous.
 * Slowest-first systems (sbp_params.scheme): the slow state update alone (its newest history
 * value exists), the fast state extrapolated to the slow receivers' donors after the first
 * micro step has pushed a_f(t), the slow RHS at t + H from them, and the fast micro steps
 * (beside the slow RHS without re-extrapolation, after it with). sbp_mrab_init ends with the
 * slow RHS at the bootstrap's end time for these. */
sbp_status sbp_mrab_step(sbp_system_t sys, int n, void *stream);

/* Change the macro step to H (> 0) for the following macro steps (Sec. 3.3 Step 1: H_i may
 * change from one macro step to the next, h_i = H_i / step_ratio). While the histories still
 * hold values at the old spacing (the next hist_len - 1 macro steps), every Adams-Bashforth
 * and extrapolation weight is solved on the history's node times (the moment conditions of
 * Sec. 3.1 with the nodes shifted to the start of the interval and scaled by its step) and the
 * steps are launched kernel by kernel; then CUDA-graph replay resumes with the plan's weights
 * times the new H. Fastest-first systems after sbp_mrab_init only (SBP_ERR_STATE). */
sbp_status sbp_mrab_set_step(sbp_system_t sys, double H);

/* Whether sbp_mrab_step replays CUDA graphs (default 1) or launches kernel by kernel (0).
 * With graphs, each macro step is one graph launch on the caller's stream: the graph is
 * captured once per ring/buffer phase (at most 4 hist_len^2 of them, on first use) and runs
 * the slow right-hand side and the first fast micro step on parallel branches, which both
 * depend only on the states at t; where the fast receivers' donor points cover at most a
 * quarter of the slow mesh (split kernels, no periodic wrap of that region), only the slow
 * mesh's tiles around them precede the fast micro steps, and the rest of the slow right-hand
 * side runs on a third, low-priority branch beside them. Results are identical in both modes. The phase timers
 * (sbp_profile_enable) force the kernel-by-kernel mode while they are on. */
sbp_status sbp_use_graphs(sbp_system_t sys, int enable);
/* Kernel launches in one macro step's CUDA graph: the kernel nodes of the graph that
 * sbp_mrab_step replayed last (host int; 0 before the first replay). A count of this library's
 * own launches per macro step, for reports; no counterpart in the paper. */
sbp_status sbp_graph_launches(sbp_system_t sys, int *kernels);

/* Autotuner of the right-hand side's kernel and block shape. Three kernel designs compute the
 * same bits: a pair (contravariant fluxes of a 32 x rows tile with a halo-3 primitive tile in
 * shared memory, then derivatives + SAT + update from a halo-3 flux tile; 4, 8, 16 or 32 rows per
 * CTA); a single pass that marches a strip of 58 columns up a chunk of 8, 16, 32, 64 or 128
 * rows, 4 rows per step, with 16-row ring buffers of state, metrics, class bytes (copied one
 * step ahead with cp.async, or, at chunks of 16 to 128 rows, the state and metrics by TMA
 * tensor copies), primitives and fluxes in shared memory (state, metrics and result cross HBM
 * once); and a column-marching single pass (one mesh column per thread, strips of 116 or 244
 * columns, chunks of 32 to 256 rows, one row per step, the j-direction stencil taps in
 * per-thread register windows and one shared-memory row per stage for the i-direction ones).
 * For each mesh the autotuner times every candidate on the bound state, as
 * the fused right-hand side + MRAB update of the next macro step (its outputs go to the state
 * buffer that step overwrites; the history is only read), and keeps the fastest (reported by
 * sbp_mesh_info_get). It runs at the end of sbp_mrab_init
 * while enabled (the default); enabling it on an initialised system runs it at once.
 * Synchronises the stream. */
sbp_status sbp_autotune(sbp_system_t sys, int enable, void *stream);

/* Choose the right-hand-side kernel of `mesh` by hand (the autotuner's choice otherwise): strip
 * = 0 selects the kernel pair with rows & 0xFF = 4, 8, 16 or 32 rows per CTA of the flux kernel
 * and rows >> 8 = 4, 8, 16 or 32 rows of the derivative kernel (0: the same); strip = 58 the
 * single-pass marching kernel with chunks of rows & 0xFFFF rows (1..65535), its state and metric
 * rows copied into the shared-memory rings by per-thread cp.async, or, with rows | SBP_STAGE_TMA,
 * by TMA tensor copies (one thread issues 72 x 4 boxes that complete on an mbarrier; a wait
 * that runs out after about a second records SBP_ERR_TIMEOUT for sbp_check); strip = 116 or 244 the
 * column-marching kernel (one column per thread, CTAs of 128 or 256 threads, the j-direction
 * stencils from per-thread register windows; meshes at least 128 or 256 points wide) with chunks
 * of `rows` rows. All give the same bits.
 * Later autotuner runs (sbp_mrab_init, sbp_autotune) override the choice; disable the
 * autotuner (sbp_autotune(sys, 0, stream)) to keep it. */
#define SBP_STAGE_TMA 0x10000
sbp_status sbp_set_rhs_shape(sbp_system_t sys, int mesh, int strip, int rows);

/* The integrator state of `mesh` between macro steps (after sbp_mrab_init): its current state
 * and the hist_len - 1 right-hand-side history entries the next macro step reads, oldest first
 * (the MRAB stepping vector of Sec. 3.3 / the step matrix of Sec. 4.3). set = 0 copies them to
 * the caller's device buffers q (state layout) and hist ((hist_len - 1) states, contiguous);
 * set = 1 copies them from those buffers into the integrator, so a run can be checkpointed and
 * resumed, or perturbed. Asynchronous on the stream. Fastest-first systems only
 * (SBP_ERR_STATE otherwise). */
sbp_status sbp_integrator_state(sbp_system_t sys, int mesh, void *q, void *hist, int set, void *stream);

/* Checkpoint and resume of the whole integrator between macro steps (after sbp_mrab_init):
 * both meshes' current states and history rings, the ring positions, the node times of the
 * history entries, H, the elapsed time and the variable-step counter, in one host blob.
 * sbp_checkpoint_save with blob NULL sets *size to the bytes needed; otherwise *size (in) is the
 * buffer's capacity (SBP_ERR_ARG if too small) and (out) the bytes written. Synchronises the
 * stream. sbp_checkpoint_load restores a blob into a system created with the same meshes and
 * parameters and with bound buffers (SBP_ERR_STATE otherwise); it need not have run
 * sbp_mrab_init. Macro steps after a load give the same bits as the steps after the save.
 * SBP_ERR_ARG for a blob that is not a checkpoint, is truncated, or comes from a system with
 * another element type, physics, scheme, history length or step ratio; SBP_ERR_SHAPE for other
 * mesh sizes. The blob is in the host's byte order. Synchronises the stream. */
sbp_status sbp_checkpoint_save(sbp_system_t sys, void *blob, size_t *size, void *stream);
sbp_status sbp_checkpoint_load(sbp_system_t sys, const void *blob, size_t size, void *stream);

/* n steps of the classical fourth-order Runge-Kutta method at step h on both meshes at one
 * rate, the single-rate baseline of Sec. 4.4 and 6.1 (eq. (perf_RK4): four right-hand sides
 * of every point per step). Each stage evaluates both meshes' right-hand sides with the overset
 * coupling to the other mesh's stage state (sbp_overset_interp + sbp_rhs_eval), then
 * y <- y + h/6 k1 + h/3 k2 + h/3 k3 + h/6 k4 with FP64 accumulation, in place in the current
 * state buffers (sbp_bind). Needs h > 0 (SBP_ERR_ARG) and bound buffers (SBP_ERR_STATE).
 * Allocates five states per mesh of stage storage on first use (kept with the system). A step
 * is one CUDA graph replay while graphs are on (sbp_use_graphs). Leaves the MRAB history
 * stale: sbp_mrab_init must run again before sbp_mrab_step. Asynchronous on the stream; the
 * elapsed time (sbp_mrab_time) advances by n h. */
sbp_status sbp_rk4_step(sbp_system_t sys, int n, double h, void *stream);

/* Macro step size H and elapsed time since the end of the bootstrap. */
sbp_status sbp_mrab_time(sbp_system_t sys, double *H, double *t);

/* Phase timers, the device-side counterpart of the paper's RHS / interpolation time split
 * (Sec. 6.2, Table perfthird). While enabled, sbp_mrab_step records a CUDA event pair on its
 * stream around every kernel launch and attributes the elapsed device time to one phase:
 * interpolation to the slow mesh's receivers, the slow fused RHS + update, interpolation to the
 * fast mesh's receivers (with the slow extrapolation), the fast fused RHS + update.
 * sbp_profile_read waits for the recorded events and returns, per phase, the accumulated
 * milliseconds and launch counts (arrays of SBP_PHASE_COUNT); reset != 0 clears them. */
enum { SBP_PHASE_INTERP_SLOW = 0, SBP_PHASE_RHS_SLOW = 1, SBP_PHASE_INTERP_FAST = 2, SBP_PHASE_RHS_FAST = 3,
       SBP_PHASE_COUNT = 4 };
sbp_status sbp_profile_enable(sbp_system_t sys, int enable);
sbp_status sbp_profile_read(sbp_system_t sys, double *ms, int *launches, int reset);

/* ---- Batches of overset systems --------------------------------------------------------------
 * Many independent two-mesh systems (for example many small problems of different sizes and
 * step ratios) advanced together: every MRAB micro step (Sec. 3.3) of every member is ONE
 * cooperative persistent launch with three phases separated by grid barriers: donor values of
 * all receiving meshes, contravariant fluxes of all tiles, then SBP derivatives + SAT + update
 * of all tiles. A macro step is max(step_ratio) such launches, replayed as a CUDA graph per
 * ring phase. The grid barrier's spin is bounded (about a second); on expiry the kernel records
 * SBP_ERR_TIMEOUT in the batch's error word (sbp_batch_check) and returns.
 * Members must be initialised (sbp_mrab_init), share element type, physics and fine-mesh kind
 * (all Cartesian or all curvilinear) and have a Cartesian slow mesh; they stay usable on their
 * own (their states and ring positions follow the batch). The results equal stepping each
 * member alone. Euler batches may instead run the single-pass right-hand side: the launch's
 * phases are then donor values, the SAT values of every boundary / receiver point, and 58-column
 * strips of 32 or 64 rows (the marching kernel's body), with the same bits. autotune != 0 picks
 * the work-item shape (tile pairs of 8 or 16 rows; for Euler also strips of 32 or 64 rows) by
 * timing two macro steps per candidate on a snapshot of every member's buffers (restored
 * afterwards). */
typedef struct sbp_batch_s *sbp_batch_t;
sbp_status sbp_batch_create(const sbp_system_t *systems, int n, int autotune, void *stream, sbp_batch_t *out);
sbp_status sbp_batch_destroy(sbp_batch_t batch);
/* n macro steps of every member (asynchronous). */
sbp_status sbp_batch_step(sbp_batch_t batch, int n, void *stream);
/* members, rows per work item (8, 16: tile pairs of 32 columns; 32, 64: single-pass strips of
 * 58 columns), cooperative grid size, number of ring phases (graphs). */
sbp_status sbp_batch_info(sbp_batch_t batch, int *members, int *rows_per_cta, int *grid, int *period);
/* Work-item shape (replaces the autotuner's choice; between steps): rows = 8 or 16 for tile
 * pairs, 32, 64 or 128 for single-pass strips (Euler batches only); SBP_ERR_ARG otherwise. */
sbp_status sbp_batch_set_shape(sbp_batch_t batch, int rows);
/* Synchronise the stream and report (then clear) the batch's device error word. */
sbp_status sbp_batch_check(sbp_batch_t batch, void *stream);

/* ---- Discrete adjoint (SBP_F64 systems only) --------------------------------------------------
 * Exact derivatives of the discrete operators above (not of the continuous equations): the
 * right-hand side of Sec. 2.2 eq. (int) with its SBP closures, SAT penalties and interface
 * values, the donor-cell interpolation of Sec. 2.2, the Runge-Kutta bootstrap of Sec. 3.1 and
 * the MRAB macro step of Sec. 3.3 (fastest-first, no re-extrapolation). The paper does not
 * derive an adjoint; these calls differentiate the method as implemented. Local Jacobians are
 * exact (forward-mode dual numbers on the same point-wise formulas); the derivative stencils
 * enter through their transposes, including the closure rows; every sum is a fixed-order
 * gather, so repeated calls give identical bits. Characteristic splittings (the sign of a
 * wave speed in K+/-) are differentiated on the branch the state selects. Buffers are device
 * memory in the state layout unless stated; the library allocates its FP64 workspace (about 17
 * planes per mesh plus 30 doubles per receiver) on the first call and keeps it until
 * sbp_system_destroy. All of these return SBP_ERR_DTYPE on SBP_F32 systems. */

/* Replace the far-field state qinf[4] (host) of the system (Sec. 4.1 far-field SAT target). */
sbp_status sbp_set_freestream(sbp_system_t sys, const double *qinf);

/* Vector-Jacobian product of sbp_rhs_eval(mesh, q_self, q_other): with R = dq/dt of `mesh`,
 * writes lq_self = (dR/dq_self)^T lam and lq_other = (dR/dq_other)^T lam (through the receivers'
 * interpolated states and viscous fluxes), and, when lqinf != NULL, lqinf[4] (host) =
 * (dR/dqinf)^T lam (synchronises the stream). lam has the layout of q_self; its values at holes
 * are ignored. Outputs are overwritten, pad columns included. */
sbp_status sbp_rhs_eval_vjp(sbp_system_t sys, int mesh, const void *q_self, const void *q_other, const void *lam,
                            void *lq_self, void *lq_other, double *lqinf, void *stream);

/* Jacobian-vector product of sbp_rhs_eval: drhs = (dR/dq_self) dq_self + (dR/dq_other) dq_other +
 * (dR/dqinf) dqinf (dqinf: host, 4 values, or NULL for zero). drhs is 0 at holes. */
sbp_status sbp_rhs_eval_jvp(sbp_system_t sys, int mesh, const void *q_self, const void *q_other,
                            const void *dq_self, const void *dq_other, const double *dqinf, void *drhs,
                            void *stream);

/* Vector-Jacobian product of sbp_overset_interp(recv_mesh, q_donor): lq_donor (state layout of the
 * donor mesh, overwritten) = adjoint of q_donor for receiver-value adjoints lqhat (4 x
 * n_receivers) and lfvhat (6 x n_receivers, NULL for zero; ignored for Euler). */
sbp_status sbp_overset_interp_vjp(sbp_system_t sys, int recv_mesh, const void *q_donor, const void *lqhat,
                                  const void *lfvhat, void *lq_donor, void *stream);

/* Probe-pressure objective of a whole run and its gradient. From the initial states q0 (device,
 * state layout) the run is the bootstrap of sbp_mrab_init followed by n_steps macro steps of
 * sbp_mrab_step, all with macro step H (the eager kernel sequence; identical results to the
 * graphs). The objective is
 *   J = H * sum over macro steps n = 1..n_steps of sum over probes p of p_p(t_n)^2,
 * with p_p the pressure interpolated at probe p from the background (mesh 0) state after step n
 * through the 4x4 Lagrange stencil of the interface interpolation (Sec. 2.2) on the
 * background's nodes. probe_xy: host, 2 per probe; every stencil point must be active.
 * Outputs (any may be NULL): J (host), probe_p (host, n_steps x n_probes pressures), the
 * gradients dJ/dq0 of both meshes (device, state layout; both or neither) and dJ/dqinf[4]
 * (host; the far-field state enters through the far-field SAT only; the viscous coefficient,
 * H and the initial states are held fixed), forward_steps (host: macro steps run, recomputation
 * included). Without gradient outputs only the forward runs.
 * The reverse sweep recomputes forward steps from checkpoints: n_snapshots device snapshots
 * (each a state and a history ring per mesh) besides the initial one, placed by binomial
 * checkpointing (Griewank): every macro step is recomputed at most r times, r the least integer
 * with C(n_snapshots + r, r) >= n_steps. n_snapshots >= n_steps - 1 stores every step (one
 * recomputation each). Workspace (snapshots, bootstrap stage states, adjoint rings) is allocated
 * for the call and freed before it returns; the system's bound buffers and ring positions are
 * left unchanged. Synchronises the stream. */
typedef struct {
  int n_steps;
  int n_snapshots;
  int n_probes;
  const double *probe_xy;
  double H;
} sbp_adjoint_desc;
sbp_status sbp_adjoint_probe(sbp_system_t sys, const sbp_adjoint_desc *desc, const void *q0_mesh0,
                             const void *q0_mesh1, double *J, double *probe_p, void *dJ_dq0_mesh0,
                             void *dJ_dq0_mesh1, double *dJ_dqinf, long *forward_steps, void *stream);

/* ---- 3D Cartesian systems ---------------------------------------------------------------------
 * Two overset uniform Cartesian 3D meshes (mesh 0 = background, mesh 1 = the fine box): the
 * compressible Navier-Stokes / Euler equations of App. C.1 in three directions,
 * dq/dt = -(D_x (F - F^V) + D_y (G - G^V) + D_z (H - H^V)) + SAT with D_x = D_xi / hx etc.
 * (SBP 4-2, Sec. 2.1), the interface and far-field SAT of Sec. 2.2 eq. (int) with the
 * characteristic matrices of the 3D flux Jacobian, 4 x 4 x 4 donor-cell Lagrange
 * interpolation (Sec. 2.2), and the same MRAB integrator (Sec. 3.1-3.3) as the 2D systems.
 * q = (rho, rho u, rho v, rho w, rho E): nvar = 5 planes; variable v of point (i, j, k) sits at
 * base[v * field_elems + (k * nj + j) * pitch + i]. Faces are ordered i-low, i-high, j-low,
 * j-high, k-low, k-high; a periodic direction has SBP_BC_PERIODIC on both faces; the walls of
 * the 2D systems are not offered in 3D. Hole cut: background points inside the fine box and
 * more than hole_cells background spacings from each of its non-periodic faces. The sbp_params
 * fields are read as for 2D systems (qinf takes its first four entries as (rho, rho u, rho v,
 * rho E) with rho w = 0: use sbp3_set_freestream for a full 5-component state). */
typedef struct sbp3_system_s *sbp3_system_t;
typedef struct {
  int n[3];
  int periodic[3];
  int bc[6];
  double lo[3], h[3];
} sbp3_mesh_desc;
typedef struct {
  int ni, nj, nk, pitch;
  size_t field_elems;   /* pitch * nj * nk */
  size_t state_bytes;   /* 5 planes */
  int nvar, n_holes, n_receivers, n_sat_points, elem_size;
} sbp3_mesh_info;

sbp_status sbp3_system_create(const sbp3_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                              sbp3_system_t *out);
sbp_status sbp3_system_destroy(sbp3_system_t sys);
sbp_status sbp3_mesh_info_get(sbp3_system_t sys, int mesh, sbp3_mesh_info *info);
/* qinf[5] (host): far-field state of the far-field SAT. */
sbp_status sbp3_set_freestream(sbp3_system_t sys, const double *qinf);
/* Setup tables (host, any pointer may be NULL): iblank ni*nj*nk bytes (1 active); receivers
 * n_receivers linear indices (k*nj + j)*ni + i; donor_base 3 ints and donor_w 12 doubles
 * (4 Lagrange weights along i, j, k) per receiver. */
sbp_status sbp3_get_tables(sbp3_system_t sys, int mesh, signed char *iblank, long long *receivers, int *donor_base,
                           double *donor_w);
/* The host part of sbp3_system_create alone (no device calls): argument checks, hole cut,
 * segment classes, SAT lists, donor search and weights; tables as sbp3_get_tables, n_receivers
 * (host int) the receiver count. Any output pointer may be NULL. */
typedef struct sbp3_host_tables_s *sbp3_host_tables_t;
sbp_status sbp3_host_tables_create(const sbp3_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                   sbp3_host_tables_t *out);
sbp_status sbp3_host_tables_destroy(sbp3_host_tables_t tables);
sbp_status sbp3_host_tables_get(sbp3_host_tables_t tables, int mesh, signed char *iblank, long long *receivers,
                                int *donor_base, double *donor_w, int *n_receivers);
/* Interpolation to recv_mesh's receivers from the other mesh's state (device): qhat 5 x
 * n_receivers, fvhat 12 x n_receivers (Cartesian viscous fluxes F^V_x, F^V_y, F^V_z, each
 * momentum x, y, z and energy; NS only, may be NULL). */
sbp_status sbp3_overset_interp(sbp3_system_t sys, int recv_mesh, const void *q_donor, void *qhat, void *fvhat,
                               void *stream);
/* Right-hand side of one mesh with its receivers fed from q_other; holes get 0. */
sbp_status sbp3_rhs_eval(sbp3_system_t sys, int mesh, const void *q_self, const void *q_other, void *rhs,
                         void *stream);
/* Time step of Sec. 4.1 per mesh (without the CFL factor) and the macro step H (host). */
sbp_status sbp3_timestep(sbp3_system_t sys, const void *q0, const void *q1, double *dt_mesh, double *H,
                         void *stream);
/* Integrator buffers, bootstrap and macro steps: as sbp_bind, sbp_mrab_init, sbp_mrab_step. */
sbp_status sbp3_bind(sbp3_system_t sys, int mesh, void *q_a, void *q_b, void *hist);
sbp_status sbp3_current_state(sbp3_system_t sys, int mesh, void **q);
sbp_status sbp3_mrab_init(sbp3_system_t sys, double H, void *stream);
sbp_status sbp3_mrab_step(sbp3_system_t sys, int n, void *stream);
sbp_status sbp3_check(sbp3_system_t sys, void *stream);
/* Right-hand-side kernels of one mesh (both give the same bits): kchunk > 0 marches along k
 * (Navier-Stokes: primitives in a shared-memory ring, flux tiles staged one plane ahead), each
 * CTA a 32 x 8 column tile and kchunk planes; kchunk = 0 (the default) takes the per-point
 * kernels (primitives, fluxes, derivatives one point per thread). SBP_ERR_ARG for a bad mesh or
 * kchunk outside 0..4096. */
sbp_status sbp3_set_rhs_kernel(sbp3_system_t sys, int mesh, int kchunk);

/* y[i] = x[i] widened from FP32 to FP64 (device buffers of n elements, asynchronous on stream),
 * by the integer re-encoding that the FP32 forms use for their FP64 accumulations (the MRAB
 * update and the slow-state extrapolation): exact, equal bit for bit to the hardware
 * conversion for every input, without issuing to the FP64 pipe. */
sbp_status sbp_f32_to_f64(const void *x, void *y, size_t n, void *stream);
/* ---- Chains of nested overset meshes, one rate per mesh --------------------------------------
 * Sec. 3.3: the multi-rate scheme extends to any number of rates (read as the two-rate
 * fastest-first recursion nested level by level); Sec. 2.2's overset coupling at every level.
 * meshes[0] is the outermost mesh; meshes[r] (r >= 1) lies inside meshes[r - 1] and cuts a hole
 * into it (points inside its outer boundary and more than hole_cells spacings of mesh r - 1 from
 * it). Mesh r's receivers are its interface faces, interpolated from mesh r - 1, and the segment
 * ends next to the hole mesh r + 1 cuts, interpolated from mesh r + 1 (4 x 4 Lagrange stencils,
 * interface SAT of eq. (int)). Every mesh but the innermost must be Cartesian; the outermost has
 * no interface faces. ratios[r] (n_meshes - 1 of them, 1..16, product <= 2^20) is the step of
 * mesh r over the step of mesh r + 1: with macro step H, mesh r steps H / (ratios[0] ...
 * ratios[r - 1]). params as for sbp_system_create (step_ratio and fast_mesh are not read; no
 * sponge layer). Host tables and device tables are owned by the chain. SBP_ERR_SHAPE for a
 * receiver next to both its outer face and a hole, or an interface face without an enclosing
 * mesh; SBP_ERR_DONOR for a receiver without a valid stencil. */
typedef struct sbp_chain_s *sbp_chain_t;
sbp_status sbp_chain_create(const sbp_mesh_desc *meshes, int n_meshes, const int *ratios, const sbp_params *params,
                            sbp_chain_t *out);
sbp_status sbp_chain_destroy(sbp_chain_t chain);
/* Sizes and layout of mesh r (as sbp_mesh_info_get; hist_bytes for hist_len states). */
sbp_status sbp_chain_mesh_info(sbp_chain_t chain, int mesh, sbp_mesh_info *info);
/* Host copies of mesh r's setup (any pointer may be NULL): iblank (ni*nj), receivers (point
 * index j*ni+i, ascending), donor_mesh (the mesh each receiver reads), donor_base (2 ints) and
 * donor_w (8 doubles) per receiver, as sbp_get_tables. */
sbp_status sbp_chain_tables(sbp_chain_t chain, int mesh, signed char *iblank, int *receivers, int *donor_mesh,
                            int *donor_base, double *donor_w);
/* dq/dt of mesh r (device, the state layout) with its receivers fed from the states q_all[0..n-1]
 * (one device state per mesh) as they are. Asynchronous on stream. */
sbp_status sbp_chain_rhs_eval(sbp_chain_t chain, int mesh, const void *const *q_all, void *rhs, void *stream);
/* Sec. 4.1's stable step of every mesh without the CFL factor (dt_mesh[n], host) and the macro
 * step H = min over r of cfl dt_r (ratios[0] ... ratios[r - 1]) (host): every mesh's own step
 * respects the CFL limit. Synchronises the stream. */
sbp_status sbp_chain_timestep(sbp_chain_t chain, const void *const *q_all, double *dt_mesh, double *H, void *stream);
/* Integrator buffers of mesh r (device, caller-owned): two states and a ring of hist_len states. */
sbp_status sbp_chain_bind(sbp_chain_t chain, int mesh, void *q_a, void *q_b, void *hist);
sbp_status sbp_chain_current_state(sbp_chain_t chain, int mesh, void **q);
/* Bootstrap (Heun's RK3 at the innermost step for (hist_len - 1) macro steps of mesh 0, recording
 * each mesh's right-hand side at its own step) with macro step H (<= 0: from sbp_chain_timestep).
 * Synchronises the stream. */
sbp_status sbp_chain_mrab_init(sbp_chain_t chain, double H, void *stream);
/* n macro steps: for mesh r at the start tau of each of its steps, the donor values (mesh r - 1
 * extrapolated to tau by the polynomial through its history from the start of its current
 * step, mesh r + 1 at tau), the right-hand side at tau fused with the Adams-Bashforth update
 * (FP64 accumulation), then mesh r + 1's steps over the same interval. Asynchronous. */
sbp_status sbp_chain_mrab_step(sbp_chain_t chain, int n, void *stream);
sbp_status sbp_chain_mrab_time(sbp_chain_t chain, double *H, double *t);
/* Synchronise the stream and report (then clear) the chain's device error word. */
sbp_status sbp_chain_check(sbp_chain_t chain, void *stream);

/* Measurement utility (the paper has no counterpart: it is the denominator of the FP64 roofline
 * that the benchmark reports). Launches one kernel of grid x block threads on stream in which
 * every thread runs 8 independent chains of iters FP64 fused multiply-adds and writes one double
 * to out (device, grid * block doubles, caller-owned); *flops (host, may be NULL) receives the
 * FP64 operations it performs (2 per FMA). Time it with events on the same stream. SBP_ERR_ARG
 * for a null out, non-positive sizes or a block that is not a multiple of 32 up to 1024. */
sbp_status sbp_fp64_rate_probe(void *out, int grid, int block, long iters, double *flops, void *stream);
/* Failure-detection self-test (the paper has no counterpart): the bounded wait of the grid
 * barrier that separates the phases of a batch launch (sbp_batch_step), run on `grid` CTAs of 32
 * threads that wait for `arrivals` arrivals with at most max_spins polls of 256 ns each. With
 * arrivals > grid no CTA can pass: each gives up after its poll limit, records SBP_ERR_TIMEOUT in
 * the launch's error word and returns, so the context stays usable. *status (host) receives
 * that error word (0 when the barrier opened), *passed (host) the CTAs that passed. Allocates a
 * 16-byte device word set and synchronises the stream. SBP_ERR_ARG for grid outside 1..8,
 * arrivals < 1 or max_spins outside 1..65536 (a limit of at most ~17 ms). */
sbp_status sbp_barrier_selftest(int grid, int arrivals, unsigned max_spins, int *status, int *passed,
                                void *stream);
/* ---- 3D curvilinear operator -------------------------------------------------------------------
 * The flux divergence of the 3D compressible Euler / Navier-Stokes equations (App. C.1) on one
 * curvilinear structured mesh of n[0] x n[1] x n[2] points (i fastest), non-periodic in every
 * direction, with the SBP 4-2 derivative (Sec. 2.1) and its closures at both ends of every line;
 * plus the optional far-field SAT (sbp3c_set_farfield) and, for overset coupling, the host hole
 * cut and donor search, the device gather and the interface SAT at given receivers:
 *   dq/dt = -J sum_m D_m (sum_j M[m][j] (F_j - F^V_j)),   M[m][j] = xi_m,x_j / J,
 * with the metric terms in the symmetric conservative form of Thomas and Lombard (the paper defers
 * the metrics to other work), M[m][j] = D_b((X_c)_a X_e) - D_a((X_c)_b X_e) over cyclic (m, a, b)
 * and (j, c, e), J = 1 / det(D_a X_c) (computed in FP64 on the device at creation, stored in the
 * element type); viscous gradients by d/dx_j = J sum_m M[m][j] D_m. A uniform state has zero
 * divergence to rounding. params: physics, dtype, gamma, mu, pr are read. x, y, z: host arrays of
 * n[0]*n[1]*n[2] doubles (copied). States and right-hand sides: 5 device planes of
 * n[0]*n[1]*n[2] elements, unpitched, q = (rho, rho u, rho v, rho w, rho E). SBP_ERR_SHAPE for a
 * direction outside 8..65535 points. */
typedef struct sbp3c_mesh_s *sbp3c_mesh_t;
sbp_status sbp3c_mesh_create(const int *n, const double *x, const double *y, const double *z,
                             const sbp_params *params, sbp3c_mesh_t *out);
sbp_status sbp3c_mesh_destroy(sbp3c_mesh_t mesh);
/* metrics (host): 10 planes of n[0]*n[1]*n[2] doubles, M[m][j] m-major, then J. Synchronous. */
sbp_status sbp3c_get_metrics(sbp3c_mesh_t mesh, double *metrics);
/* Far-field SAT (Sec. 5.1's characteristic penalty, Sec. 2.2 eq. (int) towards a free stream) on
 * all six faces: at a point on the low (side +1) or high (side -1) face of index direction m the
 * right-hand side gains -(sigma / p0) K^side_k (q - qinf) with k = grad xi_m = J M[m][:] and
 * p0 = 17/48, one term for each face the point lies on (edges and corners take two or three);
 * no viscous penalty. qinf (host, 5 values, copied): the free stream's conserved variables;
 * NULL turns the SAT off (the default at creation). SBP_ERR_ARG for sigma < 0 or a free stream
 * without positive density and pressure. */
sbp_status sbp3c_set_farfield(sbp3c_mesh_t mesh, const double *qinf, double sigma);
/* Donor search on a curvilinear mesh (Sec. 2.2: donor-receiver pairing; weights from the
 * Lagrange shape functions). Host only, no device calls. For each of the npts points
 * pts[3 t .. 3 t + 2] = (x, y, z): computational coordinates (s, r, t) (index units) with
 * X(s, r, t) = p, X the mesh map interpolated by the 4 x 4 x 4 Lagrange basis on the stencil
 * that starts at floor(.) - 1 clamped into the mesh, found by Newton's method from a nearby
 * node (the nearest of a coarse subset of nodes, refined locally by halving the stride; the
 * nearest of all nodes if the iteration from there fails to converge inside the index range)
 * until three consecutive steps stay below 1e-10; a point it converges to outside the index
 * range, or fails on more than a cell outside it, is outside the mesh.
 * Points outside the nodes' bounding box padded by the longest edge between neighbouring nodes
 * are outside the mesh without a search. Outputs (host, caller
 * owned): base 3 ints per point (i0, j0, k0), w 12 doubles per point (the 4 basis values along
 * i, then j, then k: the value at the point is sum wi[a] wj[b] wk[c] f(i0 + a, j0 + b, k0 + c)),
 * xi 3 doubles per point (NULL to skip). n, x, y, z as for sbp3c_mesh_create; iblank
 * (n[0]*n[1]*n[2] bytes, NULL: all active) marks active points. SBP_ERR_DONOR for the first
 * point with no valid stencil (outside the mesh, no convergence, or an inactive point in its
 * stencil), its index in *first_failed (NULL to skip; -1 when all succeed). */
sbp_status sbp3c_donor_search(const int *n, const double *x, const double *y, const double *z,
                              const signed char *iblank, int npts, const double *pts, int *base, double *w,
                              double *xi, int *first_failed);
/* Hole cut against a curvilinear mesh (Sec. 2.2 hole cutting; reading, as for the Cartesian 3D
 * systems in the overlapping mesh's index units). Host only, no device calls. For each of the
 * npts points pts[3 t ..] (e.g. another mesh's nodes) the inverse map of the mesh (as in
 * sbp3c_donor_search) is sought; a point found inside the mesh with every index coordinate more
 * than margin (>= 0) from the faces (margin < s < n[a] - 1 - margin) is a hole: iblank[t] = 0.
 * Other entries of iblank (host, npts bytes) are left as they are. */
sbp_status sbp3c_hole_cut(const int *n, const double *x, const double *y, const double *z, int npts,
                          const double *pts, double margin, signed char *iblank);
/* Overset gather on the mesh (Sec. 2.2 interpolation): out[v * nrecv + r] = sum over a, b, c in
 * 0..3 of w[12 r + a] w[12 r + 4 + b] w[12 r + 8 + c] q_v(base[3 r] + a, base[3 r + 1] + b,
 * base[3 r + 2] + c) for the 5 variables v. q: a state (5 device planes); base (3 ints per
 * receiver) and w (12 doubles per receiver) as sbp3c_donor_search writes them, copied to the
 * device by the caller; out: 5 planes of nrecv elements of the mesh's element type (device).
 * The weights are applied in the element type. A stencil that does not lie inside the mesh
 * (base outside 0 .. n[a] - 4 in some direction) gives zeros for that receiver and records
 * SBP_ERR_BOUNDS in the mesh's device error word (read by sbp3c_mesh_check), without reading out
 * of range. Asynchronous on stream. */
sbp_status sbp3c_interp(sbp3c_mesh_t mesh, const void *q, int nrecv, const int *base, const double *w, void *out,
                        void *stream);
/* Synchronise the stream and report (then clear) the mesh's device error word. */
sbp_status sbp3c_mesh_check(sbp3c_mesh_t mesh, void *stream);
/* Interface SAT terms at receiver points (Sec. 2.2 eq. (int), the normal of index direction m
 * being k = grad xi_m = J M[m][:]). sbp3c_set_interface stores nterms terms (host, copied):
 * terms[6 e ..] = (i, j, k, m, side, r): receiver point (i, j, k), normal direction m (0..2),
 * side +1 (the domain lies towards higher index) or -1, donor column r (0 <= r < nrecv); scale
 * (NULL: all 1) weights each term (corner weights); sigma is the interface penalty. Terms are
 * grouped by point and keep their order within a point. SBP_ERR_ARG for a point outside the
 * mesh, a bad direction, side or column, or sigma < 0. sbp3c_interface_sat adds, at each
 * receiver point, sum over its terms of
 *   scale * (-(1/p0) [(sigma K^side_k + sigma1 I)(q - qhat_r) - side/2 (F^V_k - F^V_k hat_r)])
 * to rhs (device, the mesh's element type), with sigma1 = mu |k|^2 / 2 and F^V_k =
 * sum_d k_d F^V_d (momentum and energy rows; Navier-Stokes only): the receiver's own viscous
 * fluxes come from chain-rule gradients of q. qhat: 5 x nrecv donor states (device, plane v at
 * qhat + v * nrecv); fvhat: 12 x nrecv donor viscous fluxes, the 4 components (momentum x, y,
 * z, energy) of F^V_x, then F^V_y, then F^V_z (Cartesian; required for Navier-Stokes, else
 * ignored). Deterministic (one thread per point). Asynchronous on stream. */
sbp_status sbp3c_set_interface(sbp3c_mesh_t mesh, int nterms, const int *terms, const double *scale, int nrecv,
                               double sigma);
sbp_status sbp3c_interface_sat(sbp3c_mesh_t mesh, const void *q, const void *qhat, const void *fvhat, void *rhs,
                               void *stream);
/* rhs = dq/dt (device, asynchronous on stream). */
sbp_status sbp3c_rhs_eval(sbp3c_mesh_t mesh, const void *q, void *rhs, void *stream);

/* ---- 3D curvilinear overset pairs ---------------------------------------------------------------
 * Two curvilinear meshes stepped together (Sec. 2.2 overset coupling, Sec. 3.1-3.3 MRAB): mesh 0,
 * the background, with the far-field SAT (sbp3c_set_farfield's form, sigma = sigma_physical) on
 * all six faces; mesh 1, the overset mesh, with interface SAT terms (eq. (int), sigma =
 * sigma_interface) on all six faces. Setup: the hole cut of the background by the overset mesh
 * (sbp3c_hole_cut with margin = params.hole_cells index units of the overset mesh; <= 0: 4),
 * every maximal active run along a line an SBP segment of at least 8 points (shorter runs
 * become holes), receivers at the overset mesh's faces and at the background's active points
 * next to a hole, one interface term per normal direction and side (corner weight Omega =
 * omega_corner where a point has several), donor stencils by sbp3c_donor_search (no hole in a
 * stencil; SBP_ERR_DONOR otherwise), the coefficient plan of the 2D systems. Right-hand sides:
 * the 3D curvilinear operator per active segment (metric terms on whole lines), 0 at holes; the
 * receivers' donor values are the other mesh's state and, for Navier-Stokes, its Cartesian
 * viscous fluxes, gathered with the stencils' weights; with sponge_cells > 0 the background's
 * right-hand side gains the sponge term of sbp_params after its SAT terms (the index distance to
 * the nearest of its six far-field faces; 0 at holes; the overset mesh has none). Time step (the 2D curvilinear form over
 * three directions): per active point 1 / (sum_m |u . k_m| + c |K| + 2 nu |K|^2), k_m = grad
 * xi_m, |K|^2 = sum_m |k_m|^2, nu = max(mu, gamma mu / Pr) / rho; H = min(cfl dt_slow, SR cfl
 * dt_fast). Integrator: fastest-first MRAB of order `order` with `hist_len` values and step
 * ratio `step_ratio`, mesh `fast_mesh` at the micro step, bootstrapped by Heun's RK3 at the
 * micro step, as sbp_mrab_init / sbp_mrab_step. States and right-hand sides: 5 device planes of
 * n[0]*n[1]*n[2] elements, unpitched, q = (rho, rho u, rho v, rho w, rho E); the element type
 * is params.dtype. x, y, z: host arrays of n[0]*n[1]*n[2] doubles, i fastest (copied). */
typedef struct {
  int n[3];
  const double *x, *y, *z;
} sbp3c_mesh_desc;
typedef struct sbp3c_system_s *sbp3c_system_t;
/* Synchronous. SBP_ERR_ARG, SBP_ERR_SHAPE, SBP_ERR_DTYPE for bad parameters or sizes (8..65535
 * points per direction), SBP_ERR_DONOR when a receiver has no valid stencil (message names it),
 * SBP_ERR_CUDA on a failed allocation. The far-field state starts as params.qinf (rho, rho u,
 * rho v, rho E) with rho w = 0; sbp3c_system_set_freestream sets all five. */
sbp_status sbp3c_system_create(const sbp3c_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                               sbp3c_system_t *out);
sbp_status sbp3c_system_destroy(sbp3c_system_t sys);
/* ni, nj, nk, pitch (= ni), field_elems, state_bytes, n_holes, n_receivers, n_sat_points (points
 * with SAT terms of any kind), elem_size of one mesh. */
sbp_status sbp3c_system_info(sbp3c_system_t sys, int mesh, sbp3_mesh_info *info);
/* qinf[5] (host): the far-field state. SBP_ERR_ARG without positive density and pressure. */
sbp_status sbp3c_system_set_freestream(sbp3c_system_t sys, const double *qinf);
/* Setup tables (host, any pointer may be NULL): iblank n[0]*n[1]*n[2] bytes (1 active, 0 hole,
 * after hole growth); receivers n_receivers linear indices (k n[1] + j) n[0] + i, sorted;
 * donor_base 3 ints (i0, j0, k0) and donor_w 12 doubles (Lagrange weights along i, j, k) per
 * receiver, on the other mesh. */
sbp_status sbp3c_system_tables(sbp3c_system_t sys, int mesh, signed char *iblank, long long *receivers,
                               int *donor_base, double *donor_w);
/* The host part of sbp3c_system_create alone (no device calls); errors as sbp3c_system_create,
 * tables as sbp3c_system_tables, n_receivers (host int) the receiver count. */
typedef struct sbp3c_host_tables_s *sbp3c_host_tables_t;
sbp_status sbp3c_host_tables_create(const sbp3c_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                    sbp3c_host_tables_t *out);
sbp_status sbp3c_host_tables_destroy(sbp3c_host_tables_t tables);
sbp_status sbp3c_host_tables_get(sbp3c_host_tables_t tables, int mesh, signed char *iblank, long long *receivers,
                                 int *donor_base, double *donor_w, int *n_receivers);
/* Donor values at recv_mesh's receivers from the other mesh's state q_donor (device): qhat 5 x
 * n_receivers, fvhat 12 x n_receivers (F^V_x, F^V_y, F^V_z, each momentum x, y, z and energy;
 * Navier-Stokes only, may be NULL). Asynchronous on stream. */
sbp_status sbp3c_system_interp(sbp3c_system_t sys, int recv_mesh, const void *q_donor, void *qhat, void *fvhat,
                               void *stream);
/* Right-hand side of one mesh with its receivers fed from q_other (device). Asynchronous. */
sbp_status sbp3c_system_rhs_eval(sbp3c_system_t sys, int mesh, const void *q_self, const void *q_other, void *rhs,
                                 void *stream);
/* Time step per mesh (without the CFL factor; dt_mesh: 2 doubles, may be NULL) and the macro step
 * H (host, may be NULL). Synchronises the stream. */
sbp_status sbp3c_system_timestep(sbp3c_system_t sys, const void *q0, const void *q1, double *dt_mesh, double *H,
                                 void *stream);
/* Integrator buffers (device, caller-owned): two states and hist_len right-hand sides per mesh,
 * as sbp_bind; the state to start from is q_a. */
sbp_status sbp3c_system_bind(sbp3c_system_t sys, int mesh, void *q_a, void *q_b, void *hist);
sbp_status sbp3c_system_current_state(sbp3c_system_t sys, int mesh, void **q);
/* Bootstrap with macro step H (H <= 0: from sbp3c_system_timestep at the bound states); allocates
 * and frees its stage buffers, synchronises the stream. SBP_ERR_STATE before sbp3c_system_bind. */
sbp_status sbp3c_system_mrab_init(sbp3c_system_t sys, double H, void *stream);
/* n macro steps, asynchronous on stream. SBP_ERR_STATE before sbp3c_system_mrab_init. */
sbp_status sbp3c_system_mrab_step(sbp3c_system_t sys, int n, void *stream);
/* The macro step and the time reached since sbp3c_system_mrab_init (host). */
sbp_status sbp3c_system_mrab_time(sbp3c_system_t sys, double *H, double *t);
/* Synchronise the stream and report (then clear) the device error word (SBP_ERR_NONFINITE: a
 * step produced a non-finite or non-positive-density state at an active point). */
sbp_status sbp3c_system_check(sbp3c_system_t sys, void *stream);

/* Synchronise the stream and report (then clear) the device error word. */
sbp_status sbp_check(sbp_system_t sys, void *stream);

/* Bounds checks. The gathers that follow tables built by the library's setup (donor indices into
 * the distinct donor points) check their indices in builds compiled with SBP_BOUNDS_CHECK
 * defined (paper_1805_06607_gb300/build.py: build(bounds_check=True), into _build_checked/): an
 * index out of range is replaced by a valid one and recorded as SBP_ERR_BOUNDS in the system's
 * device error word, read by the system's check call. Indices the caller supplies
 * (sbp3c_interp's stencil bases) are checked in every build. */

const char *sbp_status_string(sbp_status s);
const char *sbp_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* SBP_MRAB_H */
