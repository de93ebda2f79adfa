/*
 * Plain FP64 CPU oracle for the D2Q9 DUGKS / BKG finite-volume step.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper (Zhu, Wang, Guo, "Performance evaluation of the general
 * characteristics based off-lattice Boltzmann and DUGKS methods ...",
 * arXiv 1511.00242).  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Every routine is written for clarity: nested loops, explicit ghost and
 * face arrays, no blocking, no fusion.  Section / equation references are to
 * the paper:
 *   Sec 2.1  D2Q9 velocity set, equilibrium, moments, nu = tau RT
 *   Sec 2.2  DUGKS (Eqs. dugks_fv, eq_raw, eq_update, eq_flux, eq_charraw,
 *            eq_trans_2, eq_char, eq:cfl)
 *   Sec 2.3  BKG (Eqs. split_a/b, splic_c, bkg_collision, bkgfd,
 *            central_schemes, lwfv, G, bkg_fb, bkg_fv, f_left)
 *   Sec 2.5  no-slip wall: ghost cells + half-way bounce-back
 *   Sec 3.1  Taylor-Green set-up, Chapman-Enskog initial state, E_u
 *
 * Parity pins for each function are listed in tests/test_oracle_pins.py.
 * Three rules are readings where the paper is silent; each is pinned by a
 * consequence derived by hand rather than by the paper:
 *   - the diffuse-reflection wall: the slip length of plane Couette flow,
 *     tau c (BKG, the exact DVBE result) and (tau + h/2) c (DUGKS);
 *   - the free-stream face: the mass that leaves a channel in the first
 *     step, in closed form, and relaxation to the free stream;
 *   - the corner-ghost fill order: a box symmetric under a 180-degree
 *     rotation stays symmetric (this pins the corners against one-sided
 *     mistakes, not the order itself, which is a convention).
 */
#ifndef DVBE_ORACLE_H
#define DVBE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* DUGKS (Sec 2.2), BKG (Sec 2.3), and the two collision-free face values
 * of Sec 2.4: the upwind value f^n(x_b - h xi) (Eq. cfd2) and the central
 * value f^n(x_b) (Eq. cfd1), both from the cell f^n with no collision term
 * in the flux. */
enum { ORC_DUGKS = 0, ORC_BKG = 1, ORC_CFREE_UPWIND = 2, ORC_CFREE_CENTRAL = 3 };

enum {
  ORC_BC_PERIODIC = 0,
  ORC_BC_WALL_BOUNCEBACK = 1,
  ORC_BC_WALL_DIFFUSE = 2,
  ORC_BC_INFLOW_EQ = 3,
  ORC_BC_OUTFLOW_ZG = 4,
  ORC_BC_SYMMETRY = 5,
  ORC_BC_OUTFLOW_NEQ = 6 /* outflow at the segment's density: equilibrium part at rho_s,
                            non-equilibrium part extrapolated (zero gradient) */
};

enum { ORC_SIDE_W = 0, ORC_SIDE_E = 1, ORC_SIDE_S = 2, ORC_SIDE_N = 3 };

/* Reconstruction of the face value phi(x_b - h xi).  ORC_RECON_LINEAR: the
 * linear interpolation between the two cells of the face (Eqs. eq_char,
 * f_left).  ORC_RECON_UPWIND_CELL: the alternative of the traditional upwind
 * FV schemes Sec 2.4 contrasts: the upwind cell C's value carried to the foot
 * point with C's central-difference gradient, phi_C + (x_b - h xi - x_C) .
 * grad phi_C.  Directions along the face (xi . n = 0), and faces on a
 * non-periodic side of the mesh (whose upwind cell would be a ghost), take
 * the linear reconstruction. */
enum { ORC_RECON_LINEAR = 0, ORC_RECON_UPWIND_CELL = 1 };

/* One boundary segment on a side: faces whose centre coordinate along the
 * side lies in [s0, s1) take this condition.  (rho, ux, uy) is the wall
 * velocity (walls) or the free-stream state (inflow). */
typedef struct {
  int kind;
  double s0, s1;
  double rho, ux, uy;
} orc_bc_segment;

/* The problem as the paper states it: mesh (face coordinates of a tensor
 * mesh), velocity model (RT), relaxation time tau, time step dt, scheme and
 * boundary conditions.  Arrays are borrowed, never freed. */
typedef struct {
  int nx, ny;
  const double *xf; /* nx+1 x-face coordinates, strictly increasing */
  const double *yf; /* ny+1 y-face coordinates, strictly increasing */
  double RT, tau, dt;
  int scheme;       /* ORC_DUGKS, ORC_BKG, ORC_CFREE_UPWIND or ORC_CFREE_CENTRAL */
  int nbc[4];       /* segments per side, W E S N */
  const orc_bc_segment *bc[4];
  int recon;        /* ORC_RECON_LINEAR (default) or ORC_RECON_UPWIND_CELL */
} orc_problem;

/* Status codes: 0 ok, <0 bad argument. */
#define ORC_OK 0
#define ORC_EINVAL (-1)

/* Sec 2.1: velocity set xi[9][2], weights w[9], reverse directions opp[9]. */
int orc_d2q9(double RT, double *xi, double *w, int *opp);
/* Sec 2.1, Eq. equilibrium. */
void orc_equilibrium(double RT, double rho, double ux, double uy, double *feq);

/* Mesh helpers (face coordinates). */
int orc_faces_uniform(int n, double a, double b, double *out);
int orc_faces_tanh(int n, double a, double b, double beta, double *out);
int orc_faces_geometric(int n, double a, double d0, double ratio, double *out);
/* Eq. eq:cfl with dx the smallest cell width in either direction. */
int orc_dt_from_cfl(int nx, int ny, const double *xf, const double *yf,
                    double RT, double cfl, double *dt);

/* Initial states.  Host arrays: fields [ny][nx], f_tilde [9][ny][nx]. */
int orc_init_equilibrium(const orc_problem *p, const double *rho,
                         const double *ux, const double *uy, double *f_tilde);
/* Sec 3.1: f = f_eq - tau (d_t f_eq + xi . grad f_eq), with the derivative of
 * f_eq taken through (rho, u) by the chain rule from the supplied field
 * derivatives; then f_tilde = f - dt/2 Omega(f).  d is 9 arrays [ny][nx]:
 * rho_t, ux_t, uy_t, rho_x, ux_x, uy_x, rho_y, ux_y, uy_y. */
int orc_init_chapman_enskog(const orc_problem *p, const double *rho,
                            const double *ux, const double *uy,
                            const double *const *d, double *f_tilde);

/* The explicit time step (DUGKS or BKG in finite-volume form), nsteps times,
 * in place on f_tilde [9][ny][nx]. */
int orc_step(const orc_problem *p, double *f_tilde, long long nsteps);
/* BKG in its finite-difference Lax-Wendroff form (Eqs. bkgfd and
 * central_schemes); uniform periodic meshes only. */
int orc_step_bkg_fd(const orc_problem *p, double *f_tilde, long long nsteps);
/* Brute force from the implicit (trapezoidal) forms, Eqs. eq_raw and
 * eq_charraw (DUGKS) or splic_c then bkgfd (BKG), on the ORIGINAL
 * distribution f [9][ny][nx]; periodic meshes only.  The implicit relations
 * are solved by fixed-point iteration until the residual is at rounding
 * level (8 eps (1 + k/tau) max|rhs|). */
int orc_step_implicit(const orc_problem *p, double *f, long long nsteps);

/* f_tilde = f - dt/2 Omega(f) (transform of Sec 2.2), element-wise. */
int orc_tilde_from_f(const orc_problem *p, const double *f, double *f_tilde);

/* Diagnostics. */
int orc_moments(const orc_problem *p, const double *f_tilde, double *rho,
                double *ux, double *uy);
/* out[0] = sum rho |V|, out[1..2] = sum rho u |V|. */
int orc_conserved(const orc_problem *p, const double *f_tilde, double *out);
/* Sec 3.1: E_u = sqrt(sum |u_n - u_a|^2) / sqrt(sum |u_a|^2) over cells. */
int orc_l2_error_u(const orc_problem *p, const double *f_tilde,
                   const double *ua, const double *va, double *eu);

/* ---- curvilinear structured meshes (general quadrilateral cells) -------
 * The FV form of Sec 2.2 on cells V_k with faces of any orientation: cell
 * (i, j) has the vertices (i, j), (i+1, j), (i+1, j+1), (i, j+1) of the
 * vertex arrays X, Y [(ny+1)][(nx+1)] (counter-clockwise).  Readings (the
 * paper states the method for general cells but gives the reconstruction
 * only on uniform meshes):
 *   - cell centre: the mean of its four vertices; volume: its area;
 *   - face: the edge between two cells, with midpoint x_b, unit normal n
 *     (pointing to increasing i on x-faces, increasing j on y-faces) and
 *     area A = its length;
 *   - cell gradient: central differences along the two mesh lines through
 *     the centre, grad phi = J^-T (phi_i, phi_j) with J the Jacobian of the
 *     centre positions along those lines (one-sided toward the inside at
 *     the outer ghost layer of a non-periodic side);
 *   - face value (linear), the uniform-mesh split of Sec 2.4 (normal slope
 *     from the two cells, tangential slope from their gradients) carried
 *     over: with d = x_R - x_L, the line between the centres crosses the
 *     face at x_L + theta d, theta = ((x_b - x_L) . n) / (d . n), and
 *     o = x_b - (x_L + theta d) lies along the face; phi_b = (1 - theta)
 *     phi_L + theta phi_R + gbar . o with gbar = (1 - theta) grad phi_L +
 *     theta grad phi_R; the face gradient g = gbar + ((phi_R - phi_L) -
 *     gbar . d) n / (d . n) keeps gbar's tangential part and takes the
 *     two-point difference along d; phi(x_b - h xi) = phi_b - h xi . g.
 *     The upwind-cell value is phi_C + (x_b - h xi - x_C) . grad phi_C.  On
 *     a tensor mesh both equal the tensor oracle's (o = 0, d along n);
 *   - ghost cells: the first inner centre mirrored across the boundary face,
 *     values by the side's rule with the wall extrapolation factor
 *     e = ((x_g - x_1) . n) / ((x_1 - x_2) . n) (the ratio of the distances
 *     to the wall); corners as on tensor meshes (x sides first, then y
 *     sides over the padded width);
 *   - boundary faces: the rules of Sec 2.5 with the face's own normal (the
 *     symmetry rule needs a face normal along x or y, and mirrors across
 *     that axis); segments by the face centre's y (W, E) or x (S, N);
 *     periodic sides: the opposite side is a translate of it.
 * Parity unpinned by the paper (the readings above are checked by the
 * invariants of tests/test_oracle_pins.py and by reduction to the tensor
 * oracle). */
typedef struct {
  int nx, ny;
  const double *X, *Y; /* vertex coordinates [(ny+1)][(nx+1)] */
  double RT, tau, dt;
  int scheme, recon;
  int nbc[4];
  const orc_bc_segment *bc[4];
} orc_quad_problem;

/* Cell centres xc, yc and volumes vol, each [ny][nx] (any may be NULL). */
int orc_quad_geometry(const orc_quad_problem *p, double *xc, double *yc, double *vol);
/* The explicit step on the quad mesh, nsteps times, in place. */
int orc_quad_step(const orc_quad_problem *p, double *f_tilde, long long nsteps);
/* out[0] = sum rho |V|, out[1..2] = sum rho u |V| over the quad cells. */
int orc_quad_conserved(const orc_quad_problem *p, const double *f_tilde, double *out);
/* Eq. eq:cfl with dx the shortest face of the mesh. */
int orc_quad_dt_from_cfl(const orc_quad_problem *p, double cfl, double *dt);

#ifdef __cplusplus
}
#endif
#endif
