/*
 * libdvbe: D2Q9 discrete-velocity Boltzmann finite-volume step on GB300.
 *
 * The method is the one compared by Zhu, Wang and Guo (arXiv 1511.00242):
 * the discrete unified gas-kinetic scheme (DUGKS, Sec 2.2) and the
 * Bardow-Karlin-Gusev characteristics-based off-lattice Boltzmann scheme
 * (BKG, Sec 2.3), both written as a cell-centred finite-volume update of the
 * transformed distribution f_tilde (Eqs. eq_update and lwfv) on a structured
 * tensor-product mesh, uniform or stretched.
 *
 * Conventions (all entry points):
 *   - Every call returns a dvbe_status; nothing throws or aborts across the
 *     ABI.  On failure dvbe_last_error() gives a thread-local message.
 *   - Host arrays are always float64, C order: a scalar field is [ny][nx]
 *     (x fastest), a distribution is [9][ny][nx].  The caller owns them; the
 *     library copies in or out and returns after the copy has finished.
 *   - The library owns handles and all device memory.  Device memory comes
 *     from cudaMalloc unless an allocator is installed (dvbe_set_allocator).
 *   - Velocity index alpha (Sec 2.1): 0 rest; 1..4 = c(cos, sin)((alpha-1) pi/2);
 *     5..8 = sqrt(2) c (cos, sin)((2 alpha - 9) pi/4), c = sqrt(3 RT).
 *   - Boundary sides are indexed W=0, E=1, S=2, N=3.
 */
#ifndef DVBE_H
#define DVBE_H

#include <stddef.h>

#if defined(__GNUC__)
#define DVBE_API __attribute__((visibility("default")))
#else
#define DVBE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DVBE_OK = 0,
  DVBE_ERR_INVALID_ARG = 1, /* a NULL pointer, a bad size, a bad enum value  */
  DVBE_ERR_CFL = 2,         /* CFL number >= 1 (Eq. eq:cfl) without override */
  DVBE_ERR_OOM = 3,         /* device or host allocation failed              */
  DVBE_ERR_CUDA = 4,        /* a CUDA runtime call failed                    */
  DVBE_ERR_DIVERGED = 5,    /* a non-finite or non-positive density was met  */
  DVBE_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out            */
  DVBE_ERR_UNSUPPORTED = 7  /* valid request this build does not provide     */
} dvbe_status;

/* DVBE_DUGKS: Sec 2.2.  DVBE_BKG: Sec 2.3.  The two collision-free face
 * values that Sec 2.4 contrasts with them (Eqs. cfd2, cfd1): the cell f^n
 * reconstructed at x_b - h xi (upwind) or at x_b (central) is the flux
 * distribution itself, with no collision term; the update starts from
 * f_tilde^+ as in the other schemes.  These two run on the single solver
 * only (dvbe_batch_create rejects them). */
typedef enum {
  DVBE_DUGKS = 0,
  DVBE_BKG = 1,
  DVBE_CFREE_UPWIND = 2,
  DVBE_CFREE_CENTRAL = 3
} dvbe_scheme;

/* Storage of f_tilde in device memory.  Arithmetic is FP64 for DVBE_F64 and
 * FP32 for every other mode.  *_DEV modes store d = (f_tilde - w_alpha rho0)/s_alpha;
 * s_alpha = 1 for DVBE_F32_DEV and, for the 16-bit modes, the power of two
 * nearest to dev_scale * w_alpha * rho0 (exact to apply and undo).  The FP32
 * modes, DVBE_F32 included, compute on deviations of f_tilde from a fixed
 * reference near w_alpha rho0, so rounding scales with the deviation;
 * DVBE_F32 still stores f_tilde itself, rounded to FP32 every step. */
typedef enum {
  DVBE_F64 = 0,
  DVBE_F32 = 1,
  DVBE_F32_DEV = 2,
  DVBE_F16_DEV = 3,
  DVBE_BF16_DEV = 4
} dvbe_precision;

/* Boundary conditions (Sec 2.5 and the flat-plate set-up of Sec 3.3). */
typedef enum {
  DVBE_BC_PERIODIC = 0,        /* must pair W with E or S with N, one segment   */
  DVBE_BC_WALL_BOUNCEBACK = 1, /* ghost extrapolation + half-way bounce-back    */
  DVBE_BC_WALL_DIFFUSE = 2,    /* ghost extrapolation + diffuse reflection      */
  DVBE_BC_INFLOW_EQ = 3,       /* free stream: ghosts f_eq(rho, ux, uy); at the
                                  face the entering distributions take it      */
  DVBE_BC_OUTFLOW_ZG = 4,      /* zero-gradient ghosts                          */
  DVBE_BC_SYMMETRY = 5,        /* mirrored ghosts                               */
  DVBE_BC_OUTFLOW_NEQ = 6      /* outflow at the segment's density rho: ghost =
                                  inner value + f_eq(rho, u_1) - f_eq(rho_1, u_1)
                                  (not in the paper; bounded at small dt/tau
                                  where the zero-gradient outflow may not be) */
} dvbe_bc_kind;

/* A segment of one side: faces whose centre coordinate along the side lies in
 * [s0, s1) take this condition.  (ux, uy) is the wall velocity U_w for walls;
 * (rho, ux, uy) the free-stream state for inflow. */
typedef struct {
  int kind; /* dvbe_bc_kind */
  double s0, s1;
  double rho, ux, uy;
} dvbe_bc_segment;

#define DVBE_MAX_SEGMENTS 8 /* per side */

typedef struct dvbe_mesh_ *dvbe_mesh;
typedef struct dvbe_solver_ *dvbe_solver;
typedef struct dvbe_batch_ *dvbe_batch;

/* The problem statement of Sec 2: mesh, velocity model (RT), relaxation time
 * tau (nu = tau RT, Eq. nu_tau), time step dt, scheme, boundary conditions. */
typedef struct {
  dvbe_mesh mesh;
  double RT, tau, dt;
  double rho0;      /* reference density of the deviation form (0 -> 1)         */
  int scheme;       /* dvbe_scheme                                               */
  int precision;    /* dvbe_precision                                            */
  const dvbe_bc_segment *bc[4];
  int nbc[4];
  int allow_cfl_ge_1; /* non-zero: accept CFL >= 1 (the paper's blow-up test)    */
  int bkg_fd;       /* BKG on a uniform mesh: use the finite-difference form of
                       Eqs. bkgfd / central_schemes (identical up to rounding)   */
  double dev_scale; /* s_alpha = power of two nearest dev_scale w_alpha rho0 for
                       F16_DEV / BF16_DEV (0 -> default: 1/256 for F16, 1 for
                       BF16); ignored otherwise (F32_DEV stores d unscaled)     */
  void *cuda_stream; /* cudaStream_t to run on (NULL: the library creates its own
                        non-blocking stream)                                    */
  int recon;        /* dvbe_recon: face reconstruction (0: linear)               */
  int path;         /* dvbe_path: 0 the fused step kernels where they apply,
                       1 the multi-pass step with face arrays                   */
} dvbe_params;

/* Reconstruction of the face value phi(x_b - h xi).  DVBE_RECON_LINEAR: the
 * linear interpolation between the two cells of the face (Eqs. eq_char,
 * f_left), the paper's.  DVBE_RECON_UPWIND_CELL: the reconstruction of the
 * traditional upwind FV schemes Sec 2.4 contrasts with it: the upwind cell
 * C's value carried to the foot point with C's central-difference gradient,
 * phi_C + (x_b - h xi - x_C) . grad phi_C; directions along a face, and faces
 * on non-periodic sides, keep the linear one.  It runs on the multi-pass
 * path (DVBE_F64 or DVBE_F32 storage), single solver only. */
typedef enum { DVBE_RECON_LINEAR = 0, DVBE_RECON_UPWIND_CELL = 1 } dvbe_recon;

/* Step implementation.  DVBE_PATH_FUSED: one fused kernel (two on meshes
 * with inner strips) per step, every precision.  DVBE_PATH_MULTIPASS: the
 * step as separate kernels with face arrays in device memory (cell stage,
 * ghost layers, x faces, y faces, update; about five times the memory traffic
 * of the fused step), in FP64 or FP32 storage with arithmetic of the same
 * precision (other storage modes: DVBE_ERR_UNSUPPORTED); it carries the
 * reconstruction variants and the quadrilateral meshes. */
typedef enum { DVBE_PATH_FUSED = 0, DVBE_PATH_MULTIPASS = 1 } dvbe_path;

/* ---- velocity set and mesh --------------------------------------------- */

/* Sec 2.1: xi[9][2] (row-major), w[9], opp[9] (xi_opp = -xi). */
DVBE_API dvbe_status dvbe_d2q9(double RT, double *xi, double *w, int *opp);

/* Face coordinates of a structured tensor mesh (Sec 2.2: cells V_k with faces
 * at x = xf[i], y = yf[j]).  xf has nx+1, yf ny+1 strictly increasing
 * entries; both are copied.  nx, ny >= 2. */
DVBE_API dvbe_status dvbe_mesh_create(int nx, int ny, const double *xf, const double *yf,
                             dvbe_mesh *out);
DVBE_API void dvbe_mesh_destroy(dvbe_mesh mesh);
/* Cell centres xc[nx], yc[ny] and volumes |V_k| vol[ny][nx] (any may be NULL)
 * of a tensor mesh; DVBE_ERR_UNSUPPORTED for a quadrilateral mesh. */
DVBE_API dvbe_status dvbe_mesh_geometry(dvbe_mesh mesh, double *xc, double *yc, double *vol);

/* Curvilinear structured mesh of general quadrilateral cells (the FV form of
 * Sec 2.2 holds for cells V_k with faces of any orientation).  X, Y are the
 * vertex coordinates [(ny+1)][(nx+1)], row-major, copied; cell (i, j) has the
 * vertices (i, j), (i+1, j), (i+1, j+1), (i, j+1), counter-clockwise.  Every
 * cell's area must be positive (else DVBE_ERR_INVALID_ARG); nx, ny >= 2.
 * On this mesh:
 *   - cell centre = mean of the four vertices, volume = area; face = the
 *     edge between two cells, with its midpoint x_b, unit normal n (towards
 *     increasing i on x-faces, increasing j on y-faces) and length A;
 *   - the face value phi(x_b - h xi) generalises the linear reconstruction
 *     of Sec 2.4: the line between the centres x_L, x_R crosses the face at
 *     x_L + theta d (d = x_R - x_L, theta = ((x_b - x_L) . n) / (d . n)),
 *     phi_b = (1 - theta) phi_L + theta phi_R + gbar . (x_b - x_L - theta d)
 *     with gbar the theta-blend of the two cells' gradients, and the face
 *     gradient g = gbar + ((phi_R - phi_L) - gbar . d) n / (d . n), so that
 *     phi(x_b - h xi) = phi_b - h xi . g.  Cell gradients: central
 *     differences along the two mesh lines, mapped by the inverse Jacobian of
 *     the centre positions (one-sided at the outer ghost layer of a side that
 *     is not periodic).  DVBE_RECON_UPWIND_CELL: phi_C + (x_b - h xi - x_C) .
 *     grad phi_C;
 *   - ghost centres: the first inner centre mirrored across the boundary
 *     face; wall extrapolation factor e = ((x_g - x_1) . n) / ((x_1 - x_2) .
 *     n); the rules of Sec 2.5 with the face's own normal; symmetry sides
 *     need faces normal to x or y; boundary segments are chosen by the face
 *     midpoint's y (W, E) or x (S, N); a periodic pair of sides must be
 *     translates of each other.
 * A tensor mesh given this way steps as dvbe_mesh_create's up to rounding.
 * Solvers on a quadrilateral mesh run the multi-pass step
 * (DVBE_PATH_MULTIPASS; DVBE_F64 or DVBE_F32 storage, otherwise
 * DVBE_ERR_UNSUPPORTED); batches take tensor meshes only. */
DVBE_API dvbe_status dvbe_mesh_create_quad(int nx, int ny, const double *X, const double *Y,
                                           dvbe_mesh *out);
/* Cell centres and volumes of either kind of mesh, each [ny][nx] (any may be
 * NULL). */
DVBE_API dvbe_status dvbe_mesh_cells(dvbe_mesh mesh, double *xc, double *yc, double *vol);
/* n+1 faces: uniform on [a, b]; tanh-clustered toward both ends,
 * a + (b-a)(1 + tanh(beta(2s-1))/tanh(beta))/2 with s = i/n; geometric from a
 * with first width d0 and growth ratio. */
DVBE_API dvbe_status dvbe_faces_uniform(int n, double a, double b, double *out);
DVBE_API dvbe_status dvbe_faces_tanh(int n, double a, double b, double beta, double *out);
DVBE_API dvbe_status dvbe_faces_geometric(int n, double a, double d0, double ratio, double *out);
/* Eq. eq:cfl: dt = cfl * dx_min / (sqrt(6) c_s), dx_min the smallest cell
 * width of the mesh in either direction (on a quadrilateral mesh, the
 * shortest cell edge). */
DVBE_API dvbe_status dvbe_dt_from_cfl(dvbe_mesh mesh, double RT, double cfl, double *dt);

/* ---- device memory ------------------------------------------------------ */

/* Install a device allocator used for every later allocation (for instance a
 * caching allocator).  alloc returns NULL on failure; free_ receives what
 * alloc returned.  Pass NULL, NULL to return to cudaMalloc / cudaFree.
 * Process-wide; call it while no solver or batch exists. */
typedef void *(*dvbe_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dvbe_free_fn)(void *ptr, void *stream, void *ctx);
DVBE_API dvbe_status dvbe_set_allocator(dvbe_alloc_fn alloc, dvbe_free_fn free_, void *ctx);

/* ---- one solver ----------------------------------------------------------- */

/* Validates the parameters (DVBE_ERR_CFL when the CFL number dt |xi|_max /
 * dx_min is >= 1 without allow_cfl_ge_1), copies the mesh and the boundary
 * segments, allocates two device copies of f_tilde and the geometry
 * tables.  The distribution starts at rest equilibrium (f_tilde = w rho0). */
DVBE_API dvbe_status dvbe_solver_create(const dvbe_params *params, dvbe_solver *out);
DVBE_API void dvbe_solver_destroy(dvbe_solver s);

/* f_tilde = f_eq(rho, u) (Eq. equilibrium); fields [ny][nx]. */
DVBE_API dvbe_status dvbe_init_equilibrium(dvbe_solver s, const double *rho, const double *ux,
                                  const double *uy);
/* Sec 3.1: f = f_eq - tau (d_t f_eq + xi . grad f_eq) with the derivatives of
 * f_eq taken through (rho, u) from d[9] = (rho_t, ux_t, uy_t, rho_x, ux_x,
 * uy_x, rho_y, ux_y, uy_y), then f_tilde = f - dt/2 Omega(f). */
DVBE_API dvbe_status dvbe_init_chapman_enskog(dvbe_solver s, const double *rho, const double *ux,
                                     const double *uy, const double *const *d);
/* Set / read f_tilde [9][ny][nx]. */
DVBE_API dvbe_status dvbe_init_f(dvbe_solver s, const double *f_tilde);
DVBE_API dvbe_status dvbe_get_f(dvbe_solver s, double *f_tilde);

/* Advance nsteps time steps (Eq. eq_update for DUGKS, Eq. lwfv for BKG, the
 * same finite-volume update with the collision-free faces of Eqs. cfd1 /
 * cfd2 for DVBE_CFREE_*).
 * Launches are queued on the solver's stream; the call then waits for them
 * and returns DVBE_ERR_DIVERGED if any step met a non-finite or non-positive
 * density (the state is left as it is). */
DVBE_API dvbe_status dvbe_step(dvbe_solver s, long long nsteps);
/* Same launches without the final wait and check. */
DVBE_API dvbe_status dvbe_step_async(dvbe_solver s, long long nsteps);
/* Wait for queued work; DVBE_ERR_DIVERGED as for dvbe_step. */
DVBE_API dvbe_status dvbe_sync(dvbe_solver s);
/* Steps taken since creation or the last init. */
DVBE_API dvbe_status dvbe_step_count(dvbe_solver s, long long *nsteps);

/* Density and velocity from f_tilde (Eq. macro_var), fields [ny][nx]. */
DVBE_API dvbe_status dvbe_get_moments(dvbe_solver s, double *rho, double *ux, double *uy);
/* FP64 sums out[0] = sum rho |V|, out[1] = sum rho u_x |V|, out[2] = sum rho u_y |V|
 * (deterministic order). */
DVBE_API dvbe_status dvbe_conserved(dvbe_solver s, double out[3]);
/* Relative velocity change since the previous call (FP64, deterministic):
 * r = ||u - u_prev||_2 / ||u||_2 over cells; the first call returns +inf. */
DVBE_API dvbe_status dvbe_residual(dvbe_solver s, double *r);
/* Sec 3.1: E_u = ||u - u_a||_2 / ||u_a||_2 over cells, FP64. ua, va [ny][nx]. */
DVBE_API dvbe_status dvbe_l2_error_u(dvbe_solver s, const double *ua, const double *va,
                            double *eu);

/* Launch shape: cells per warp row are fixed at 30 (32 lanes less two halo
 * columns); strip_rows = rows one warp marches through; warps_per_block;
 * blocks = grid size (0: enough for every strip).  graph_chunk > 0 replays
 * CUDA graphs of that many steps inside dvbe_step. */
typedef struct {
  int strip_rows;
  int warps_per_block;
  int blocks;
  int graph_chunk;
} dvbe_launch;
DVBE_API dvbe_status dvbe_get_launch(dvbe_solver s, dvbe_launch *out);
DVBE_API dvbe_status dvbe_set_launch(dvbe_solver s, const dvbe_launch *in);
/* Time each candidate launch shape on this solver's own state for `steps`
 * steps and keep the fastest; the state is restored afterwards.  best_ms
 * (may be NULL) receives the fastest time per step.  Candidates: strip
 * heights from 8 to 256 rows and the heights that make the inner strips fill
 * a whole number of waves of resident warps, with 2, 4 or 8 warps per block,
 * each with a grid of one block per strip group or one wave of blocks.  The
 * choice is cached (dvbe_set_autotune_cache) under the scheme, precision,
 * mesh size and periodicity, GPU model and library build: a later call with
 * the same key takes the cached shape without timing anything.  A solver on
 * the multi-pass path has no launch shape: the call returns at once with
 * best_ms = 0. */
DVBE_API dvbe_status dvbe_autotune(dvbe_solver s, int steps, double *best_ms);
/* Autotuner cache file (JSON).  NULL: no cache; "": the default, which is
 * $DVBE_AUTOTUNE_CACHE if set (empty: no cache), else
 * $XDG_CACHE_HOME/dvbe/autotune.json, else $HOME/.cache/dvbe/autotune.json.
 * Process-wide. */
DVBE_API dvbe_status dvbe_set_autotune_cache(const char *path);

/* Device view of the current f_tilde (for timing and inspection): pointer to
 * column 0 of row 0 of field 0, row pitch in elements, elements per field,
 * element size; element (a, j, i) is at ptr + a * plane + j * pitch + i.  On
 * a mesh periodic in x the rows carry halo columns (copies of the columns at
 * the other end) just before column 0 and just after column nx-1. */
DVBE_API dvbe_status dvbe_device_state(dvbe_solver s, void **ptr, long long *pitch,
                              long long *plane, int *elem_bytes);
/* Kernel launches issued since creation (every step kernel, init, reduction).
 * A step is one launch, or two on meshes with inner strips and boundary
 * strips: the strips that touch no boundary run in a kernel compiled without
 * boundary code, the others in a second kernel at the same time.  On a mesh
 * periodic in both directions every strip is inner (one launch), except for
 * FP32 and 16-bit storage at an odd nx. */
DVBE_API dvbe_status dvbe_launch_count(dvbe_solver s, long long *count);

/* Spatial decomposition (the paper has none; its FV form on cells V_k and
 * their faces, Sec 2.2, is what lets a mesh be split into blocks).  One
 * line of cells of all nine fields moved between the solver's f_tilde and a
 * dense device buffer [9][hi-lo] of the solver's storage element (values as
 * stored): axis 0 is column `index` over rows lo..hi-1, axis 1 row `index`
 * over columns lo..hi-1.  Used to exchange the halo ring of a block with its
 * neighbours between steps.  The calls wait for the copy.  A line outside
 * the mesh: DVBE_ERR_INVALID_ARG. */
DVBE_API dvbe_status dvbe_pack_line(dvbe_solver s, int axis, int index, int lo, int hi, void *dev_buf);
DVBE_API dvbe_status dvbe_unpack_line(dvbe_solver s, int axis, int index, int lo, int hi,
                                      const void *dev_buf);
/* dvbe_conserved over the window of cells [i0, i0+nx) x [j0, j0+ny) (FP64,
 * deterministic order): the owned cells of a block. */
DVBE_API dvbe_status dvbe_conserved_window(dvbe_solver s, int i0, int j0, int nx, int ny, double out[3]);

/* Checkpoint and restart (the paper has no counterpart).  The device storage
 * of f_tilde exactly as stored ([9][ny][pitch] elements of the solver's
 * precision, padding included), so a solver of the same problem restarted
 * from it continues bit for bit, whatever the storage mode (dvbe_get_f /
 * dvbe_init_f round-trip exactly only for DVBE_F64 and DVBE_F32).
 * dvbe_state_bytes gives the size; save copies it to host memory the caller
 * owns (and the step count to *step, may be NULL); load copies it back and
 * sets the step count.  A buffer of another size: DVBE_ERR_INVALID_ARG. */
DVBE_API dvbe_status dvbe_state_bytes(dvbe_solver s, size_t *bytes);
DVBE_API dvbe_status dvbe_save_state(dvbe_solver s, void *host, size_t bytes, long long *step);
DVBE_API dvbe_status dvbe_load_state(dvbe_solver s, const void *host, size_t bytes, long long step);

/* Failure detection of the step kernel (the paper has no counterpart).  Each
 * warp stages rows through asynchronous copies completed on mbarriers; a copy
 * not complete at its first test is polled at most `polls` more times, after
 * which the warp stops fetching, waits (bounded) for the copies it has in
 * flight, and leaves; the step then returns DVBE_ERR_TIMEOUT and the state is
 * not a valid time level (re-initialise it).  The default is
 * DVBE_DEFAULT_WAIT_LIMIT polls, and every wait also gives up after about a
 * second of SM clock cycles, far longer than any copy takes.  0 serves tests
 * of the failure path: every wait gives up at once, so each warp stops at
 * its first fetch.  polls < 0: DVBE_ERR_INVALID_ARG.  Waits for queued work
 * first. */
#define DVBE_DEFAULT_WAIT_LIMIT 16777216LL
DVBE_API dvbe_status dvbe_set_wait_limit(dvbe_solver s, long long polls);

/* Allocation-free variant of dvbe_conserved.  The paper has no counterpart:
 * this is an interface for callers that cannot allocate device memory, such as
 * a framework that reserves all GPU memory for its own pool before the run, or
 * a time-critical loop in which cudaMalloc / cudaFree must not run (cudaFree
 * waits for the whole device).  It allocates nothing: the caller passes
 * device pointers to f_tilde (storage `precision`, layout [9][ny][pitch] with
 * element offsets, as dvbe_device_state reports it), to the cell widths
 * dx[nx] and dy[ny], and to out[3], which receives sum rho |V|, sum rho u_x |V|
 * and sum rho u_y |V| in FP64.  RT, rho0 and dev_scale are those of the
 * solver that produced f_tilde.  Work is queued on `stream` (a cudaStream_t,
 * NULL for the legacy default stream) and the call returns without waiting.
 * Partial sums go to one fixed device array of 8192 x 3 doubles (192 KB) that
 * every GPU loading the library keeps until exit; meshes of more than
 * 33,554,432 cells (8192 x 4096) are rejected with DVBE_ERR_INVALID_ARG.
 * Every call on a device shares that array and overwrites the slots it uses
 * before reading them (nothing needs clearing), so calls that overlap on the
 * GPU race.  The first call on each device resolves the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream
 * capture. */
DVBE_API dvbe_status dvbe_conserved_noalloc(const void *f_tilde, int precision, int nx, int ny,
                                            long long pitch, const double *dx, const double *dy,
                                            double RT, double rho0, double dev_scale, double *out,
                                            void *stream);

/* ---- batched form --------------------------------------------------------- */

/* Many independent cases of uneven size stepped together: every step is one
 * persistent launch per scheme over a work queue of all cases' strips.
 * All cases must share one precision.  Each case keeps its own divergence
 * status; a diverged case stops being stepped. */
DVBE_API dvbe_status dvbe_batch_create(const dvbe_params *cases, int ncases, dvbe_batch *out);
DVBE_API void dvbe_batch_destroy(dvbe_batch b);
DVBE_API dvbe_status dvbe_batch_init_equilibrium(dvbe_batch b, int icase, const double *rho,
                                        const double *ux, const double *uy);
/* nsteps steps, replayed as CUDA graphs of graph_chunk steps (0: no graph). */
DVBE_API dvbe_status dvbe_batch_step(dvbe_batch b, long long nsteps, int graph_chunk);
/* DVBE_OK or DVBE_ERR_DIVERGED for one case (waits for queued work). */
DVBE_API dvbe_status dvbe_batch_case_status(dvbe_batch b, int icase);
DVBE_API dvbe_status dvbe_batch_get_moments(dvbe_batch b, int icase, double *rho, double *ux,
                                   double *uy);
DVBE_API dvbe_status dvbe_batch_get_f(dvbe_batch b, int icase, double *f_tilde);
DVBE_API dvbe_status dvbe_batch_set_launch(dvbe_batch b, const dvbe_launch *in);
DVBE_API dvbe_status dvbe_batch_autotune(dvbe_batch b, int steps, double *best_ms);
DVBE_API dvbe_status dvbe_batch_launch_count(dvbe_batch b, long long *count);
/* dvbe_set_wait_limit for every case of a batch; a case whose wait ran out
 * reports DVBE_ERR_TIMEOUT from dvbe_batch_case_status. */
DVBE_API dvbe_status dvbe_batch_set_wait_limit(dvbe_batch b, long long polls);

/* ---- misc --------------------------------------------------------------- */

/* Thread-local text of the last failure ("" if none). */
DVBE_API const char *dvbe_last_error(void);
/* Build identification ("libdvbe <arch>"). */
DVBE_API const char *dvbe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DVBE_H */
