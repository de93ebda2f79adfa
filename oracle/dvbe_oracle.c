/*
 * Plain FP64 CPU oracle for the D2Q9 DUGKS / BKG finite-volume step.
 * TEST INFRASTRUCTURE ONLY: see dvbe_oracle.h for who may use it.
 *
 * The step is written in the paper's order with explicit arrays:
 *   1. cell moments and equilibrium               (Sec 2.1, Eq. macro_var)
 *   2. phi = f_bar^+ (DUGKS), f_tilde^+ (BKG) or the cell f^n (collision-free
 *      faces of Eqs. cfd1 / cfd2)               (Eqs. eq_trans_2, bkg_collision)
 *   3. ghost layer of phi                         (Sec 2.5)
 *   4. face values phi(x_b - h xi) by linear reconstruction
 *                                                 (Eqs. eq_char, bkg_fb, f_left);
 *      phi(x_b) for the central collision-free face (Eq. cfd1)
 *   5. wall / inflow treatment at boundary faces  (Sec 2.5)
 *   6. DUGKS: face moments, back-transform to f   (Sec 2.2 after Eq. eq_char)
 *   7. flux and update                            (Eqs. eq_update, eq_flux, lwfv, bkg_fv)
 *
 * Readings taken where the paper is silent (each also pinned or marked in the
 * tests):
 *   - The closed forms of the transforms are derived here from their
 *     definitions (f_tilde = f - dt/2 Omega, f_bar^+ = f + h/2 Omega, ...):
 *       f        = (2 tau f_tilde + dt f_eq) / (2 tau + dt)
 *       f_bar^+  = ((2 tau - h) f_tilde + 3 h f_eq) / (2 tau + dt)
 *       f_tilde^+= ((2 tau - dt) f_tilde + 2 dt f_eq) / (2 tau + dt)
 *       f (face) = (2 tau f_bar + h f_eq) / (2 tau + h)
 *     Pinned by orc_step_implicit, which solves the implicit forms directly.
 *   - Linear reconstruction on a tensor mesh: at an x-face between cells L, R
 *     with theta = (x_b - x_L)/(x_R - x_L): value (1-theta) phi_L + theta phi_R,
 *     normal slope (phi_R - phi_L)/(x_R - x_L), tangential slope the theta
 *     blend of the two cells' central differences; the foot value is
 *     value - h (xi . slope).  On a uniform mesh this is exactly Eq. f_left.
 *   - Flux sign: the update subtracts the outward flux (Eq. bkg_fv).
 *   - Wall ghosts: linear extrapolation from the first two inner centres to
 *     the mirror point of the first centre.  Corner ghosts: x sides are filled
 *     first (interior rows), then y sides over the full padded width.
 *   - Bounce-back uses the formula of Sec 2.5 literally (no density factor).
 *   - Diffuse wall (the paper has none): the incoming values are
 *     f_eq(rho_w, U_w) with rho_w making the normal mass flux through the
 *     face zero.  Pinned by the Couette slip length.
 *   - Free stream / inflow (Sec 3.3): ghosts are f_eq(rho_inf, U_inf) and,
 *     at the boundary face, the distributions entering the domain are set
 *     to it (those leaving keep their reconstructed values); outflow:
 *     zero-gradient ghosts; symmetry: mirrored ghosts.
 *   - Outflow at a set density (not in the paper; an option beside the
 *     zero-gradient outflow): the ghost is the first inner value with its
 *     equilibrium part taken at the segment's density, f_eq(rho_s, u_1)
 *     + (phi_1 - f_eq(rho_1, u_1)).  It holds the outlet at that density;
 *     on the flat plate at small dt/tau it stays bounded where the
 *     zero-gradient outflow diverges.
 */
#include "dvbe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Velocity model, Sec 2.1                                            */
/* ------------------------------------------------------------------ */

typedef struct {
  double c, cs2;
  double xi[9][2];
  double w[9];
  int opp[9];  /* reverse direction: xi_opp = -xi            */
  int mirx[9]; /* mirror across an x-normal face: xi_x -> -xi_x */
  int miry[9]; /* mirror across a y-normal face: xi_y -> -xi_y  */
} vset;

static void make_vset(double RT, vset *v) {
  const double pi = acos(-1.0);
  v->cs2 = RT;
  v->c = sqrt(3.0 * RT);
  for (int a = 0; a < 9; ++a) {
    double ex, ey;
    if (a == 0) {
      ex = 0.0;
      ey = 0.0;
    } else if (a <= 4) {
      double th = (a - 1) * pi / 2.0;
      ex = cos(th);
      ey = sin(th);
    } else {
      double th = (2 * a - 9) * pi / 4.0;
      ex = sqrt(2.0) * cos(th);
      ey = sqrt(2.0) * sin(th);
    }
    /* The nine velocities are c times points of the integer lattice; rounding
     * removes the 1e-16 residue that cos(pi/2) and friends leave. */
    v->xi[a][0] = v->c * (double)lround(ex);
    v->xi[a][1] = v->c * (double)lround(ey);
    v->w[a] = (a == 0) ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  for (int a = 0; a < 9; ++a) {
    for (int b = 0; b < 9; ++b) {
      if (v->xi[b][0] == -v->xi[a][0] && v->xi[b][1] == -v->xi[a][1]) v->opp[a] = b;
      if (v->xi[b][0] == -v->xi[a][0] && v->xi[b][1] == v->xi[a][1]) v->mirx[a] = b;
      if (v->xi[b][0] == v->xi[a][0] && v->xi[b][1] == -v->xi[a][1]) v->miry[a] = b;
    }
  }
}

/* Eq. equilibrium. */
static void feq_of(const vset *v, double rho, double ux, double uy, double *feq) {
  double usq = ux * ux + uy * uy;
  for (int a = 0; a < 9; ++a) {
    double eu = v->xi[a][0] * ux + v->xi[a][1] * uy;
    feq[a] = v->w[a] * rho *
             (1.0 + eu / v->cs2 + (eu * eu) / (2.0 * v->cs2 * v->cs2) -
              usq / (2.0 * v->cs2));
  }
}

/* Eqs. macro / macro_var. */
static void moments_of(const vset *v, const double *f9, double *rho, double *ux,
                       double *uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < 9; ++a) {
    r += f9[a];
    jx += v->xi[a][0] * f9[a];
    jy += v->xi[a][1] * f9[a];
  }
  *rho = r;
  *ux = jx / r;
  *uy = jy / r;
}

/* Omega(f) = (f_eq - f)/tau with f_eq from f's own moments (Eq. BGK_discrete). */
static void omega_of(const vset *v, double tau, const double *f9, double *om) {
  double rho, ux, uy, feq[9];
  moments_of(v, f9, &rho, &ux, &uy);
  feq_of(v, rho, ux, uy, feq);
  for (int a = 0; a < 9; ++a) om[a] = (feq[a] - f9[a]) / tau;
}

int orc_d2q9(double RT, double *xi, double *w, int *opp) {
  if (!(RT > 0.0) || !xi || !w || !opp) return ORC_EINVAL;
  vset v;
  make_vset(RT, &v);
  for (int a = 0; a < 9; ++a) {
    xi[2 * a] = v.xi[a][0];
    xi[2 * a + 1] = v.xi[a][1];
    w[a] = v.w[a];
    opp[a] = v.opp[a];
  }
  return ORC_OK;
}

void orc_equilibrium(double RT, double rho, double ux, double uy, double *feq) {
  vset v;
  make_vset(RT, &v);
  feq_of(&v, rho, ux, uy, feq);
}

/* ------------------------------------------------------------------ */
/* Mesh                                                               */
/* ------------------------------------------------------------------ */

int orc_faces_uniform(int n, double a, double b, double *out) {
  if (n < 1 || !(b > a) || !out) return ORC_EINVAL;
  for (int i = 0; i <= n; ++i) out[i] = a + (b - a) * (double)i / (double)n;
  return ORC_OK;
}

int orc_faces_tanh(int n, double a, double b, double beta, double *out) {
  if (n < 1 || !(b > a) || !(beta > 0.0) || !out) return ORC_EINVAL;
  for (int i = 0; i <= n; ++i) {
    double s = (double)i / (double)n;
    out[i] = a + (b - a) * 0.5 * (1.0 + tanh(beta * (2.0 * s - 1.0)) / tanh(beta));
  }
  return ORC_OK;
}

int orc_faces_geometric(int n, double a, double d0, double ratio, double *out) {
  if (n < 1 || !(d0 > 0.0) || !(ratio > 0.0) || !out) return ORC_EINVAL;
  for (int i = 0; i <= n; ++i) {
    if (ratio == 1.0)
      out[i] = a + d0 * (double)i;
    else
      out[i] = a + d0 * (pow(ratio, (double)i) - 1.0) / (ratio - 1.0);
  }
  return ORC_OK;
}

int orc_dt_from_cfl(int nx, int ny, const double *xf, const double *yf, double RT,
                    double cfl, double *dt) {
  if (nx < 1 || ny < 1 || !xf || !yf || !(RT > 0.0) || !(cfl > 0.0) || !dt)
    return ORC_EINVAL;
  double dmin = INFINITY;
  for (int i = 0; i < nx; ++i) {
    double d = xf[i + 1] - xf[i];
    if (!(d > 0.0)) return ORC_EINVAL;
    if (d < dmin) dmin = d;
  }
  for (int j = 0; j < ny; ++j) {
    double d = yf[j + 1] - yf[j];
    if (!(d > 0.0)) return ORC_EINVAL;
    if (d < dmin) dmin = d;
  }
  /* Eq. eq:cfl: |xi|_max = sqrt(6) c_s for D2Q9. */
  *dt = cfl * dmin / (sqrt(6.0) * sqrt(RT));
  return ORC_OK;
}

/* Cell centres with one ghost centre per side.  Non-periodic sides put the
 * ghost centre at the mirror image of the first inner centre; periodic sides
 * at the shifted image of the opposite inner centre. */
typedef struct {
  int nx, ny, per_x, per_y;
  const double *xf, *yf;
  double *xcb, *ycb; /* storage, index shifted by one */
  double *xc, *yc;   /* xc[-1..nx], yc[-1..ny] */
  const orc_bc_segment **segW, **segE, **segS, **segN; /* per boundary face */
} geom;

static void geom_free(geom *g) {
  free(g->xcb);
  free(g->ycb);
  free((void *)g->segW);
  free((void *)g->segE);
  free((void *)g->segS);
  free((void *)g->segN);
  memset(g, 0, sizeof(*g));
}

static const orc_bc_segment *seg_at(const orc_problem *p, int side, double t) {
  for (int k = 0; k < p->nbc[side]; ++k) {
    const orc_bc_segment *s = &p->bc[side][k];
    if (t >= s->s0 && t < s->s1) return s;
  }
  return NULL;
}

static int kind_valid(int k) { return k >= ORC_BC_PERIODIC && k <= ORC_BC_OUTFLOW_NEQ; }

static int geom_build(const orc_problem *p, geom *g) {
  memset(g, 0, sizeof(*g));
  if (!p || p->nx < 2 || p->ny < 2 || !p->xf || !p->yf) return ORC_EINVAL;
  if (!(p->RT > 0.0) || !(p->tau > 0.0) || !(p->dt > 0.0)) return ORC_EINVAL;
  if (p->scheme < ORC_DUGKS || p->scheme > ORC_CFREE_CENTRAL) return ORC_EINVAL;
  if (p->recon != ORC_RECON_LINEAR && p->recon != ORC_RECON_UPWIND_CELL) return ORC_EINVAL;
  for (int i = 0; i < p->nx; ++i)
    if (!(p->xf[i + 1] > p->xf[i])) return ORC_EINVAL;
  for (int j = 0; j < p->ny; ++j)
    if (!(p->yf[j + 1] > p->yf[j])) return ORC_EINVAL;
  int per[4];
  for (int s = 0; s < 4; ++s) {
    if (p->nbc[s] < 1 || !p->bc[s]) return ORC_EINVAL;
    per[s] = 0;
    for (int k = 0; k < p->nbc[s]; ++k) {
      if (!kind_valid(p->bc[s][k].kind)) return ORC_EINVAL;
      if (p->bc[s][k].kind == ORC_BC_PERIODIC) per[s] = 1;
    }
    if (per[s] && p->nbc[s] != 1) return ORC_EINVAL;
  }
  if (per[ORC_SIDE_W] != per[ORC_SIDE_E] || per[ORC_SIDE_S] != per[ORC_SIDE_N])
    return ORC_EINVAL;
  int nx = p->nx, ny = p->ny;
  g->nx = nx;
  g->ny = ny;
  g->per_x = per[ORC_SIDE_W];
  g->per_y = per[ORC_SIDE_S];
  g->xf = p->xf;
  g->yf = p->yf;
  g->xcb = (double *)malloc(sizeof(double) * (nx + 2));
  g->ycb = (double *)malloc(sizeof(double) * (ny + 2));
  g->segW = (const orc_bc_segment **)calloc(ny, sizeof(void *));
  g->segE = (const orc_bc_segment **)calloc(ny, sizeof(void *));
  g->segS = (const orc_bc_segment **)calloc(nx, sizeof(void *));
  g->segN = (const orc_bc_segment **)calloc(nx, sizeof(void *));
  if (!g->xcb || !g->ycb || !g->segW || !g->segE || !g->segS || !g->segN) {
    geom_free(g);
    return ORC_EINVAL;
  }
  g->xc = g->xcb + 1;
  g->yc = g->ycb + 1;
  for (int i = 0; i < nx; ++i) g->xc[i] = 0.5 * (p->xf[i] + p->xf[i + 1]);
  for (int j = 0; j < ny; ++j) g->yc[j] = 0.5 * (p->yf[j] + p->yf[j + 1]);
  double Lx = p->xf[nx] - p->xf[0], Ly = p->yf[ny] - p->yf[0];
  if (g->per_x) {
    g->xc[-1] = g->xc[nx - 1] - Lx;
    g->xc[nx] = g->xc[0] + Lx;
  } else {
    g->xc[-1] = 2.0 * p->xf[0] - g->xc[0];
    g->xc[nx] = 2.0 * p->xf[nx] - g->xc[nx - 1];
  }
  if (g->per_y) {
    g->yc[-1] = g->yc[ny - 1] - Ly;
    g->yc[ny] = g->yc[0] + Ly;
  } else {
    g->yc[-1] = 2.0 * p->yf[0] - g->yc[0];
    g->yc[ny] = 2.0 * p->yf[ny] - g->yc[ny - 1];
  }
  for (int j = 0; j < ny; ++j) {
    g->segW[j] = seg_at(p, ORC_SIDE_W, g->yc[j]);
    g->segE[j] = seg_at(p, ORC_SIDE_E, g->yc[j]);
    if (g->per_x) g->segW[j] = g->segE[j] = NULL;
    else if (!g->segW[j] || !g->segE[j]) {
      geom_free(g);
      return ORC_EINVAL;
    }
  }
  for (int i = 0; i < nx; ++i) {
    g->segS[i] = seg_at(p, ORC_SIDE_S, g->xc[i]);
    g->segN[i] = seg_at(p, ORC_SIDE_N, g->xc[i]);
    if (g->per_y) g->segS[i] = g->segN[i] = NULL;
    else if (!g->segS[i] || !g->segN[i]) {
      geom_free(g);
      return ORC_EINVAL;
    }
    if (!g->per_y && (g->segS[i]->kind == ORC_BC_PERIODIC ||
                      g->segN[i]->kind == ORC_BC_PERIODIC)) {
      geom_free(g);
      return ORC_EINVAL;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Ghost layer (Sec 2.5 and the inflow/outflow/symmetry of Sec 3.3)   */
/* ------------------------------------------------------------------ */

/* Padded array of 9 fields over i = -1..nx, j = -1..ny. */
#define PIDX(g, i, j) (((j) + 1) * ((g)->nx + 2) + ((i) + 1))

static void ghost_rule(const vset *v, const orc_bc_segment *s, double e, const int *mir,
                       const double *p1, const double *p2, double *pg) {
  switch (s->kind) {
    case ORC_BC_WALL_BOUNCEBACK:
    case ORC_BC_WALL_DIFFUSE:
      /* linear extrapolation from the first two inner centres */
      for (int a = 0; a < 9; ++a) pg[a] = p1[a] + e * (p1[a] - p2[a]);
      break;
    case ORC_BC_INFLOW_EQ:
      feq_of(v, s->rho, s->ux, s->uy, pg);
      break;
    case ORC_BC_OUTFLOW_ZG:
      for (int a = 0; a < 9; ++a) pg[a] = p1[a];
      break;
    case ORC_BC_OUTFLOW_NEQ: {
      /* the first inner value with its equilibrium part moved from rho_1 to
         the segment's density at the same velocity:
         pg = p1 + f_eq(rho_s, u_1) - f_eq(rho_1, u_1) */
      double r1, ux1, uy1, e1[9], es[9];
      moments_of(v, p1, &r1, &ux1, &uy1);
      feq_of(v, r1, ux1, uy1, e1);
      feq_of(v, s->rho, ux1, uy1, es);
      for (int a = 0; a < 9; ++a) pg[a] = p1[a] + (es[a] - e1[a]);
      break;
    }
    case ORC_BC_SYMMETRY:
      for (int a = 0; a < 9; ++a) pg[a] = p1[mir[a]];
      break;
    default:
      break;
  }
}

static void fill_ghosts(const vset *v, const geom *g, double *P) {
  const int nx = g->nx, ny = g->ny;
  const size_t plane = (size_t)(nx + 2) * (ny + 2);
  double p1[9], p2[9], pg[9];
  /* extrapolation factors e = (x_g - x_1)/(x_1 - x_2) per side */
  const double eW = (g->xc[-1] - g->xc[0]) / (g->xc[0] - g->xc[1]);
  const double eE = (g->xc[nx] - g->xc[nx - 1]) / (g->xc[nx - 1] - g->xc[nx - 2]);
  const double eS = (g->yc[-1] - g->yc[0]) / (g->yc[0] - g->yc[1]);
  const double eN = (g->yc[ny] - g->yc[ny - 1]) / (g->yc[ny - 1] - g->yc[ny - 2]);

  /* x sides first, interior rows only */
  for (int j = 0; j < ny; ++j) {
    for (int side = 0; side < 2; ++side) {
      int ig = side == 0 ? -1 : nx;
      int i1 = side == 0 ? 0 : nx - 1;
      int i2 = side == 0 ? 1 : nx - 2;
      if (g->per_x) {
        int src = side == 0 ? nx - 1 : 0;
        for (int a = 0; a < 9; ++a) P[a * plane + PIDX(g, ig, j)] = P[a * plane + PIDX(g, src, j)];
        continue;
      }
      for (int a = 0; a < 9; ++a) {
        p1[a] = P[a * plane + PIDX(g, i1, j)];
        p2[a] = P[a * plane + PIDX(g, i2, j)];
      }
      const orc_bc_segment *s = side == 0 ? g->segW[j] : g->segE[j];
      ghost_rule(v, s, side == 0 ? eW : eE, v->mirx, p1, p2, pg);
      for (int a = 0; a < 9; ++a) P[a * plane + PIDX(g, ig, j)] = pg[a];
    }
  }
  /* then y sides over the full padded width (corners included) */
  for (int i = -1; i <= nx; ++i) {
    int ic = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
    for (int side = 0; side < 2; ++side) {
      int jg = side == 0 ? -1 : ny;
      int j1 = side == 0 ? 0 : ny - 1;
      int j2 = side == 0 ? 1 : ny - 2;
      if (g->per_y) {
        int src = side == 0 ? ny - 1 : 0;
        for (int a = 0; a < 9; ++a) P[a * plane + PIDX(g, i, jg)] = P[a * plane + PIDX(g, i, src)];
        continue;
      }
      for (int a = 0; a < 9; ++a) {
        p1[a] = P[a * plane + PIDX(g, i, j1)];
        p2[a] = P[a * plane + PIDX(g, i, j2)];
      }
      const orc_bc_segment *s = side == 0 ? g->segS[ic] : g->segN[ic];
      ghost_rule(v, s, side == 0 ? eS : eN, v->miry, p1, p2, pg);
      for (int a = 0; a < 9; ++a) P[a * plane + PIDX(g, i, jg)] = pg[a];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Face values                                                        */
/* ------------------------------------------------------------------ */

/* Cell centre and padded-array column of cell c along x, for c = -2 .. nx+1:
 * beyond the ghost layer only on a periodic mesh, by the wrap. */
static double xcell(const geom *g, int c, int *col) {
  const double Lx = g->xf[g->nx] - g->xf[0];
  if (c < -1) {
    *col = c + g->nx;
    return g->xc[c + g->nx] - Lx;
  }
  if (c > g->nx) {
    *col = c - g->nx;
    return g->xc[c - g->nx] + Lx;
  }
  *col = c;
  return g->xc[c];
}
static double ycell(const geom *g, int c, int *row) {
  const double Ly = g->yf[g->ny] - g->yf[0];
  if (c < -1) {
    *row = c + g->ny;
    return g->yc[c + g->ny] - Ly;
  }
  if (c > g->ny) {
    *row = c - g->ny;
    return g->yc[c - g->ny] + Ly;
  }
  *row = c;
  return g->yc[c];
}

/* phi(x_b - h xi) at the x-face i (between cells i-1 and i), row j. */
static void recon_xface(const vset *v, const geom *g, const double *P, int i, int j,
                        double h, int recon, double *out) {
  const size_t plane = (size_t)(g->nx + 2) * (g->ny + 2);
  double xl = g->xc[i - 1], xr = g->xc[i], xb = g->xf[i];
  double th = (xb - xl) / (xr - xl);
  double ylo = g->yc[j - 1], yhi = g->yc[j + 1];
  const int upwind_ok = recon == ORC_RECON_UPWIND_CELL && (g->per_x || (i > 0 && i < g->nx));
  for (int a = 0; a < 9; ++a) {
    const double *Pa = P + a * plane;
    if (upwind_ok && v->xi[a][0] != 0.0) {
      /* upwind cell C and its central differences along x and y */
      const int C = v->xi[a][0] > 0.0 ? i - 1 : i;
      int cm, cp, cc;
      const double xm = xcell(g, C - 1, &cm), xp = xcell(g, C + 1, &cp), xC = xcell(g, C, &cc);
      const double gx = (Pa[PIDX(g, cp, j)] - Pa[PIDX(g, cm, j)]) / (xp - xm);
      const double gy = (Pa[PIDX(g, cc, j + 1)] - Pa[PIDX(g, cc, j - 1)]) / (yhi - ylo);
      out[a] = Pa[PIDX(g, cc, j)] + (xb - h * v->xi[a][0] - xC) * gx - h * v->xi[a][1] * gy;
      continue;
    }
    double pl = Pa[PIDX(g, i - 1, j)], pr = Pa[PIDX(g, i, j)];
    double gl = (Pa[PIDX(g, i - 1, j + 1)] - Pa[PIDX(g, i - 1, j - 1)]) / (yhi - ylo);
    double gr = (Pa[PIDX(g, i, j + 1)] - Pa[PIDX(g, i, j - 1)]) / (yhi - ylo);
    double value = (1.0 - th) * pl + th * pr;
    double slope_n = (pr - pl) / (xr - xl);
    double slope_t = (1.0 - th) * gl + th * gr;
    out[a] = value - h * (v->xi[a][0] * slope_n + v->xi[a][1] * slope_t);
  }
}

/* phi(x_b - h xi) at the y-face j (between rows j-1 and j), column i. */
static void recon_yface(const vset *v, const geom *g, const double *P, int i, int j,
                        double h, int recon, double *out) {
  const size_t plane = (size_t)(g->nx + 2) * (g->ny + 2);
  double yl = g->yc[j - 1], yr = g->yc[j], yb = g->yf[j];
  double th = (yb - yl) / (yr - yl);
  double xlo = g->xc[i - 1], xhi = g->xc[i + 1];
  const int upwind_ok = recon == ORC_RECON_UPWIND_CELL && (g->per_y || (j > 0 && j < g->ny));
  for (int a = 0; a < 9; ++a) {
    const double *Pa = P + a * plane;
    if (upwind_ok && v->xi[a][1] != 0.0) {
      const int C = v->xi[a][1] > 0.0 ? j - 1 : j;
      int rm, rp, rc;
      const double ym = ycell(g, C - 1, &rm), yp = ycell(g, C + 1, &rp), yC = ycell(g, C, &rc);
      const double gy = (Pa[PIDX(g, i, rp)] - Pa[PIDX(g, i, rm)]) / (yp - ym);
      const double gx = (Pa[PIDX(g, i + 1, rc)] - Pa[PIDX(g, i - 1, rc)]) / (xhi - xlo);
      out[a] = Pa[PIDX(g, i, rc)] + (yb - h * v->xi[a][1] - yC) * gy - h * v->xi[a][0] * gx;
      continue;
    }
    double pl = Pa[PIDX(g, i, j - 1)], pr = Pa[PIDX(g, i, j)];
    double gl = (Pa[PIDX(g, i + 1, j - 1)] - Pa[PIDX(g, i - 1, j - 1)]) / (xhi - xlo);
    double gr = (Pa[PIDX(g, i + 1, j)] - Pa[PIDX(g, i - 1, j)]) / (xhi - xlo);
    double value = (1.0 - th) * pl + th * pr;
    double slope_n = (pr - pl) / (yr - yl);
    double slope_t = (1.0 - th) * gl + th * gr;
    out[a] = value - h * (v->xi[a][0] * slope_t + v->xi[a][1] * slope_n);
  }
}

/* Sec 2.5 at a boundary face; n = outward normal of the fluid domain. */
static void face_bc(const vset *v, const orc_bc_segment *s, double nxo, double nyo,
                    double *val) {
  double orig[9];
  memcpy(orig, val, sizeof(orig));
  switch (s->kind) {
    case ORC_BC_WALL_BOUNCEBACK:
      for (int a = 0; a < 9; ++a) {
        double xn = v->xi[a][0] * nxo + v->xi[a][1] * nyo;
        if (xn > 0.0) {
          double xu = v->xi[a][0] * s->ux + v->xi[a][1] * s->uy;
          val[v->opp[a]] = orig[a] - 2.0 * v->w[a] * xu / v->cs2;
        }
      }
      break;
    case ORC_BC_WALL_DIFFUSE: {
      double f1[9], num = 0.0, den = 0.0;
      feq_of(v, 1.0, s->ux, s->uy, f1);
      for (int a = 0; a < 9; ++a) {
        double xn = v->xi[a][0] * nxo + v->xi[a][1] * nyo;
        if (xn > 0.0) num += xn * orig[a];
        if (xn < 0.0) den += -xn * f1[a];
      }
      double rw = num / den;
      for (int a = 0; a < 9; ++a) {
        double xn = v->xi[a][0] * nxo + v->xi[a][1] * nyo;
        if (xn < 0.0) val[a] = rw * f1[a];
      }
      break;
    }
    case ORC_BC_INFLOW_EQ: {
      /* free stream: what enters the domain is the free-stream equilibrium;
         what leaves keeps its reconstructed value */
      double fe[9];
      feq_of(v, s->rho, s->ux, s->uy, fe);
      for (int a = 0; a < 9; ++a) {
        double xn = v->xi[a][0] * nxo + v->xi[a][1] * nyo;
        if (xn < 0.0) val[a] = fe[a];
      }
      break;
    }
    default:
      break;
  }
}

/* DUGKS: from f_bar at the face to the original f (Eq. eq_trans_2 inverted,
 * with the face moments of f_bar).  BKG: the face value is f already (Eq. bkg_fb). */
static void face_to_f(const vset *v, const orc_problem *p, double *val) {
  if (p->scheme != ORC_DUGKS) return;
  const double h = 0.5 * p->dt, tau = p->tau;
  double rho, ux, uy, fe[9];
  moments_of(v, val, &rho, &ux, &uy);
  feq_of(v, rho, ux, uy, fe);
  for (int a = 0; a < 9; ++a) val[a] = (2.0 * tau * val[a] + h * fe[a]) / (2.0 * tau + h);
}

/* ------------------------------------------------------------------ */
/* The explicit step                                                  */
/* ------------------------------------------------------------------ */

/* Sec 2.2 cell stage of one direction: f_tilde^+ and the value phi the
 * faces reconstruct (f_bar^+ for DUGKS, f_tilde^+ for BKG, the cell f^n for
 * the collision-free faces of Eqs. cfd1 / cfd2). */
static void cell_stage(int scheme, double tau, double dt, double f, double fe, double *tplus,
                       double *phi) {
  const double h = 0.5 * dt;
  *tplus = ((2.0 * tau - dt) * f + 2.0 * dt * fe) / (2.0 * tau + dt);
  if (scheme == ORC_DUGKS)
    *phi = ((2.0 * tau - h) * f + 3.0 * h * fe) / (2.0 * tau + dt);
  else if (scheme == ORC_BKG)
    *phi = *tplus;
  else /* collision-free faces: the cell f^n itself */
    *phi = (2.0 * tau * f + dt * fe) / (2.0 * tau + dt);
}

/* Distance h the face value is taken back along the characteristic; the
 * central collision-free face takes phi at x_b itself. */
static double face_shift(int scheme, double h) { return scheme == ORC_CFREE_CENTRAL ? 0.0 : h; }

static int step_once(const orc_problem *p, const vset *v, const geom *g, double *ft,
                     double *P, double *TP, double *FX, double *FY) {
  const int nx = g->nx, ny = g->ny;
  const size_t n = (size_t)nx * ny, plane = (size_t)(nx + 2) * (ny + 2);
  const double dt = p->dt, tau = p->tau, h = 0.5 * dt;
  double f9[9], fe[9], rho, ux, uy, val[9];

  /* 1-2: cell moments, equilibrium, phi and f_tilde^+ */
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)j * nx + i;
      for (int a = 0; a < 9; ++a) f9[a] = ft[a * n + k];
      moments_of(v, f9, &rho, &ux, &uy);
      feq_of(v, rho, ux, uy, fe);
      for (int a = 0; a < 9; ++a) {
        double tplus, phi;
        cell_stage(p->scheme, tau, dt, f9[a], fe[a], &tplus, &phi);
        TP[a * n + k] = tplus;
        P[a * plane + PIDX(g, i, j)] = phi;
      }
    }
  }
  /* 3: ghost layer */
  fill_ghosts(v, g, P);

  /* 4-6: x-faces i = 0..nx, rows 0..ny-1; the central collision-free face
     takes phi at x_b itself (no shift along the characteristic) */
  const double hs = face_shift(p->scheme, h);
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i <= nx; ++i) {
      recon_xface(v, g, P, i, j, hs, p->recon, val);
      if (!g->per_x && i == 0) face_bc(v, g->segW[j], -1.0, 0.0, val);
      if (!g->per_x && i == nx) face_bc(v, g->segE[j], 1.0, 0.0, val);
      face_to_f(v, p, val);
      for (int a = 0; a < 9; ++a) FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i] = val[a];
    }
  }
  /* y-faces j = 0..ny, columns 0..nx-1 */
  for (int j = 0; j <= ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      recon_yface(v, g, P, i, j, hs, p->recon, val);
      if (!g->per_y && j == 0) face_bc(v, g->segS[i], 0.0, -1.0, val);
      if (!g->per_y && j == ny) face_bc(v, g->segN[i], 0.0, 1.0, val);
      face_to_f(v, p, val);
      for (int a = 0; a < 9; ++a) FY[(size_t)a * nx * (ny + 1) + (size_t)j * nx + i] = val[a];
    }
  }
  /* 7: f_tilde^{n+1} = f_tilde^+ - dt/|V| sum_faces (xi . n_out) A f_face */
  for (int j = 0; j < ny; ++j) {
    double dy = g->yf[j + 1] - g->yf[j];
    for (int i = 0; i < nx; ++i) {
      double dx = g->xf[i + 1] - g->xf[i];
      double vol = dx * dy;
      size_t k = (size_t)j * nx + i;
      for (int a = 0; a < 9; ++a) {
        double fw = FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i];
        double fE = FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i + 1];
        double fs = FY[(size_t)a * nx * (ny + 1) + (size_t)j * nx + i];
        double fn = FY[(size_t)a * nx * (ny + 1) + (size_t)(j + 1) * nx + i];
        double out_flux = v->xi[a][0] * dy * (fE - fw) + v->xi[a][1] * dx * (fn - fs);
        ft[a * n + k] = TP[a * n + k] - dt / vol * out_flux;
      }
    }
  }
  return ORC_OK;
}

int orc_step(const orc_problem *p, double *f_tilde, long long nsteps) {
  if (!f_tilde || nsteps < 0) return ORC_EINVAL;
  geom g;
  int rc = geom_build(p, &g);
  if (rc) return rc;
  vset v;
  make_vset(p->RT, &v);
  const int nx = p->nx, ny = p->ny;
  double *P = (double *)calloc((size_t)9 * (nx + 2) * (ny + 2), sizeof(double));
  double *TP = (double *)calloc((size_t)9 * nx * ny, sizeof(double));
  double *FX = (double *)calloc((size_t)9 * (nx + 1) * ny, sizeof(double));
  double *FY = (double *)calloc((size_t)9 * nx * (ny + 1), sizeof(double));
  if (!P || !TP || !FX || !FY) rc = ORC_EINVAL;
  for (long long s = 0; s < nsteps && !rc; ++s) rc = step_once(p, &v, &g, f_tilde, P, TP, FX, FY);
  free(P);
  free(TP);
  free(FX);
  free(FY);
  geom_free(&g);
  return rc;
}

/* ------------------------------------------------------------------ */
/* BKG, finite-difference Lax-Wendroff form (Eqs. bkgfd, central_schemes) */
/* ------------------------------------------------------------------ */

static int uniform_spacing(const double *f, int n, double *d) {
  double d0 = f[1] - f[0];
  for (int i = 1; i < n; ++i)
    if (fabs((f[i + 1] - f[i]) - d0) > 1e-12 * fabs(d0)) return 0;
  *d = (f[n] - f[0]) / (double)n;
  return 1;
}

static void lw_fd_periodic(const vset *v, int nx, int ny, double dx1, double dx2,
                           double dt, const double *phi, double *out) {
  const size_t n = (size_t)nx * ny;
  for (int a = 0; a < 9; ++a) {
    const double *F = phi + a * n;
    double x1 = v->xi[a][0], x2 = v->xi[a][1];
    for (int m = 0; m < ny; ++m) {
      int mp = (m + 1) % ny, mm = (m + ny - 1) % ny;
      for (int l = 0; l < nx; ++l) {
        int lp = (l + 1) % nx, lm = (l + nx - 1) % nx;
        double c = F[(size_t)m * nx + l];
        double d1 = (F[(size_t)m * nx + lp] - F[(size_t)m * nx + lm]) / (2.0 * dx1);
        double d2 = (F[(size_t)mp * nx + l] - F[(size_t)mm * nx + l]) / (2.0 * dx2);
        double d11 = (F[(size_t)m * nx + lp] + F[(size_t)m * nx + lm] - 2.0 * c) / (dx1 * dx1);
        double d22 = (F[(size_t)mp * nx + l] + F[(size_t)mm * nx + l] - 2.0 * c) / (dx2 * dx2);
        double d12 = (F[(size_t)mp * nx + lp] - F[(size_t)mp * nx + lm] -
                      F[(size_t)mm * nx + lp] + F[(size_t)mm * nx + lm]) /
                     (4.0 * dx1 * dx2);
        out[a * n + (size_t)m * nx + l] =
            c - dt * (x1 * d1 + x2 * d2) +
            0.5 * dt * dt * (x1 * x1 * d11 + 2.0 * x1 * x2 * d12 + x2 * x2 * d22);
      }
    }
  }
}

int orc_step_bkg_fd(const orc_problem *p, double *f_tilde, long long nsteps) {
  if (!f_tilde || nsteps < 0) return ORC_EINVAL;
  geom g;
  int rc = geom_build(p, &g);
  if (rc) return rc;
  double dx1, dx2;
  if (!g.per_x || !g.per_y || !uniform_spacing(p->xf, p->nx, &dx1) ||
      !uniform_spacing(p->yf, p->ny, &dx2)) {
    geom_free(&g);
    return ORC_EINVAL;
  }
  vset v;
  make_vset(p->RT, &v);
  const int nx = p->nx, ny = p->ny;
  const size_t n = (size_t)nx * ny;
  const double dt = p->dt, tau = p->tau;
  double *phi = (double *)malloc(sizeof(double) * 9 * n);
  if (!phi) rc = ORC_EINVAL;
  for (long long s = 0; s < nsteps && !rc; ++s) {
    for (size_t k = 0; k < n; ++k) {
      double f9[9], fe[9], rho, ux, uy;
      for (int a = 0; a < 9; ++a) f9[a] = f_tilde[a * n + k];
      moments_of(&v, f9, &rho, &ux, &uy);
      feq_of(&v, rho, ux, uy, fe);
      /* Eq. bkg_collision: the collision step gives f_tilde^+ */
      for (int a = 0; a < 9; ++a)
        phi[a * n + k] = ((2.0 * tau - dt) * f9[a] + 2.0 * dt * fe[a]) / (2.0 * tau + dt);
    }
    lw_fd_periodic(&v, nx, ny, dx1, dx2, dt, phi, f_tilde);
  }
  free(phi);
  geom_free(&g);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Brute force from the implicit forms                                */
/* ------------------------------------------------------------------ */

/* Solve out - k Omega(out) = rhs for out by the damped fixed point
 * out <- (rhs + (k/tau) f_eq(out)) / (1 + k/tau). */
static int solve_implicit(const vset *v, double tau, double k, const double *rhs,
                          double *out) {
  double scale = 0.0, om[9];
  for (int a = 0; a < 9; ++a) {
    out[a] = rhs[a];
    if (fabs(rhs[a]) > scale) scale = fabs(rhs[a]);
  }
  for (int it = 0; it < 200; ++it) {
    double rho, ux, uy, fe[9];
    moments_of(v, out, &rho, &ux, &uy);
    feq_of(v, rho, ux, uy, fe);
    for (int a = 0; a < 9; ++a) out[a] = (rhs[a] + (k / tau) * fe[a]) / (1.0 + k / tau);
    omega_of(v, tau, out, om);
    double res = 0.0;
    for (int a = 0; a < 9; ++a) {
      double r = fabs(out[a] - k * om[a] - rhs[a]);
      if (r > res) res = r;
    }
    /* rounding level of the residual expression itself */
    if (res <= 8.0 * 2.220446049250313e-16 * (1.0 + k / tau) * scale) return ORC_OK;
  }
  return ORC_EINVAL;
}

int orc_tilde_from_f(const orc_problem *p, const double *f, double *f_tilde) {
  if (!p || !f || !f_tilde || p->nx < 1 || p->ny < 1 || !(p->tau > 0.0)) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  for (size_t k = 0; k < n; ++k) {
    double f9[9], om[9];
    for (int a = 0; a < 9; ++a) f9[a] = f[a * n + k];
    omega_of(&v, p->tau, f9, om);
    for (int a = 0; a < 9; ++a) f_tilde[a * n + k] = f9[a] - 0.5 * p->dt * om[a];
  }
  return ORC_OK;
}

static int implicit_dugks_once(const orc_problem *p, const vset *v, const geom *g,
                               double *f, double *P, double *TP, double *FX, double *FY) {
  const int nx = g->nx, ny = g->ny;
  const size_t n = (size_t)nx * ny, plane = (size_t)(nx + 2) * (ny + 2);
  const double dt = p->dt, tau = p->tau, h = 0.5 * dt;
  double f9[9], om[9], val[9], F[9];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t k = (size_t)j * nx + i;
      for (int a = 0; a < 9; ++a) f9[a] = f[a * n + k];
      omega_of(v, tau, f9, om);
      for (int a = 0; a < 9; ++a) {
        P[a * plane + PIDX(g, i, j)] = f9[a] + 0.5 * h * om[a]; /* f_bar^+ */
        TP[a * n + k] = f9[a] + 0.5 * dt * om[a];                /* f + dt/2 Omega */
      }
    }
  fill_ghosts(v, g, P);
  /* Eq. eq_charraw along the characteristic: F - h/2 Omega(F) = f_bar^+(foot) */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      recon_xface(v, g, P, i, j, h, p->recon, val);
      if (solve_implicit(v, tau, 0.5 * h, val, F)) return ORC_EINVAL;
      for (int a = 0; a < 9; ++a) FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i] = F[a];
    }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      recon_yface(v, g, P, i, j, h, p->recon, val);
      if (solve_implicit(v, tau, 0.5 * h, val, F)) return ORC_EINVAL;
      for (int a = 0; a < 9; ++a) FY[(size_t)a * nx * (ny + 1) + (size_t)j * nx + i] = F[a];
    }
  /* Eq. eq_raw: f^{n+1} - dt/2 Omega(f^{n+1}) = f^n + dt/2 Omega(f^n) + dt/|V| F_in */
  for (int j = 0; j < ny; ++j) {
    double dy = g->yf[j + 1] - g->yf[j];
    for (int i = 0; i < nx; ++i) {
      double dx = g->xf[i + 1] - g->xf[i];
      size_t k = (size_t)j * nx + i;
      double rhs[9];
      for (int a = 0; a < 9; ++a) {
        double fw = FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i];
        double fE = FX[(size_t)a * (nx + 1) * ny + (size_t)j * (nx + 1) + i + 1];
        double fs = FY[(size_t)a * nx * (ny + 1) + (size_t)j * nx + i];
        double fn = FY[(size_t)a * nx * (ny + 1) + (size_t)(j + 1) * nx + i];
        double flux_in = -(v->xi[a][0] * dy * (fE - fw) + v->xi[a][1] * dx * (fn - fs));
        rhs[a] = TP[a * n + k] + dt / (dx * dy) * flux_in;
      }
      if (solve_implicit(v, tau, 0.5 * dt, rhs, F)) return ORC_EINVAL;
      for (int a = 0; a < 9; ++a) f[a * n + k] = F[a];
    }
  }
  return ORC_OK;
}

static int implicit_bkg_once(const orc_problem *p, const vset *v, const geom *g,
                             double dx1, double dx2, double *f, double *ts, double *tn) {
  const int nx = g->nx, ny = g->ny;
  const size_t n = (size_t)nx * ny;
  const double dt = p->dt, tau = p->tau;
  double f9[9], om[9], rhs[9], fs[9];
  for (size_t k = 0; k < n; ++k) {
    for (int a = 0; a < 9; ++a) f9[a] = f[a * n + k];
    /* Eq. splic_c: f* - dt/2 Omega(f*) = f^n + dt/2 Omega(f^n) */
    omega_of(v, tau, f9, om);
    for (int a = 0; a < 9; ++a) rhs[a] = f9[a] + 0.5 * dt * om[a];
    if (solve_implicit(v, tau, 0.5 * dt, rhs, fs)) return ORC_EINVAL;
    /* f_tilde* = f* - dt/2 Omega(f*) */
    omega_of(v, tau, fs, om);
    for (int a = 0; a < 9; ++a) ts[a * n + k] = fs[a] - 0.5 * dt * om[a];
  }
  /* Eq. split_b by Lax-Wendroff (Eq. bkgfd) */
  lw_fd_periodic(v, nx, ny, dx1, dx2, dt, ts, tn);
  /* back to the original distribution: f - dt/2 Omega(f) = f_tilde */
  for (size_t k = 0; k < n; ++k) {
    for (int a = 0; a < 9; ++a) rhs[a] = tn[a * n + k];
    if (solve_implicit(v, tau, 0.5 * dt, rhs, fs)) return ORC_EINVAL;
    for (int a = 0; a < 9; ++a) f[a * n + k] = fs[a];
  }
  return ORC_OK;
}

int orc_step_implicit(const orc_problem *p, double *f, long long nsteps) {
  if (!f || nsteps < 0) return ORC_EINVAL;
  if (!p || (p->scheme != ORC_DUGKS && p->scheme != ORC_BKG)) return ORC_EINVAL;
  geom g;
  int rc = geom_build(p, &g);
  if (rc) return rc;
  if (!g.per_x || !g.per_y) {
    geom_free(&g);
    return ORC_EINVAL;
  }
  vset v;
  make_vset(p->RT, &v);
  const int nx = p->nx, ny = p->ny;
  const size_t n = (size_t)nx * ny;
  if (p->scheme == ORC_DUGKS) {
    double *P = (double *)calloc((size_t)9 * (nx + 2) * (ny + 2), sizeof(double));
    double *TP = (double *)calloc(9 * n, sizeof(double));
    double *FX = (double *)calloc((size_t)9 * (nx + 1) * ny, sizeof(double));
    double *FY = (double *)calloc((size_t)9 * nx * (ny + 1), sizeof(double));
    if (!P || !TP || !FX || !FY) rc = ORC_EINVAL;
    for (long long s = 0; s < nsteps && !rc; ++s)
      rc = implicit_dugks_once(p, &v, &g, f, P, TP, FX, FY);
    free(P);
    free(TP);
    free(FX);
    free(FY);
  } else {
    double dx1, dx2;
    if (!uniform_spacing(p->xf, nx, &dx1) || !uniform_spacing(p->yf, ny, &dx2)) {
      geom_free(&g);
      return ORC_EINVAL;
    }
    double *ts = (double *)malloc(sizeof(double) * 9 * n);
    double *tn = (double *)malloc(sizeof(double) * 9 * n);
    if (!ts || !tn) rc = ORC_EINVAL;
    for (long long s = 0; s < nsteps && !rc; ++s)
      rc = implicit_bkg_once(p, &v, &g, dx1, dx2, f, ts, tn);
    free(ts);
    free(tn);
  }
  geom_free(&g);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Initial states                                                     */
/* ------------------------------------------------------------------ */

int orc_init_equilibrium(const orc_problem *p, const double *rho, const double *ux,
                         const double *uy, double *f_tilde) {
  if (!p || !rho || !ux || !uy || !f_tilde || p->nx < 1 || p->ny < 1) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  double fe[9];
  for (size_t k = 0; k < n; ++k) {
    feq_of(&v, rho[k], ux[k], uy[k], fe);
    for (int a = 0; a < 9; ++a) f_tilde[a * n + k] = fe[a];
  }
  return ORC_OK;
}

int orc_init_chapman_enskog(const orc_problem *p, const double *rho, const double *ux,
                            const double *uy, const double *const *d, double *f_tilde) {
  if (!p || !rho || !ux || !uy || !d || !f_tilde || p->nx < 1 || p->ny < 1) return ORC_EINVAL;
  for (int q = 0; q < 9; ++q)
    if (!d[q]) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  const double cs2 = v.cs2, tau = p->tau, dt = p->dt;
  for (size_t k = 0; k < n; ++k) {
    double r = rho[k], u = ux[k], w = uy[k];
    double fe[9], f9[9], om[9];
    feq_of(&v, r, u, w, fe);
    for (int a = 0; a < 9; ++a) {
      double cx = v.xi[a][0], cy = v.xi[a][1];
      double eu = cx * u + cy * w;
      /* partial derivatives of Eq. equilibrium with respect to rho, u_x, u_y */
      double d_rho = fe[a] / r;
      double d_ux = v.w[a] * r * (cx / cs2 + eu * cx / (cs2 * cs2) - u / cs2);
      double d_uy = v.w[a] * r * (cy / cs2 + eu * cy / (cs2 * cs2) - w / cs2);
      double dt_feq = d_rho * d[0][k] + d_ux * d[1][k] + d_uy * d[2][k];
      double dx_feq = d_rho * d[3][k] + d_ux * d[4][k] + d_uy * d[5][k];
      double dy_feq = d_rho * d[6][k] + d_ux * d[7][k] + d_uy * d[8][k];
      f9[a] = fe[a] - tau * (dt_feq + cx * dx_feq + cy * dy_feq);
    }
    omega_of(&v, tau, f9, om);
    for (int a = 0; a < 9; ++a) f_tilde[a * n + k] = f9[a] - 0.5 * dt * om[a];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Diagnostics                                                        */
/* ------------------------------------------------------------------ */

int orc_moments(const orc_problem *p, const double *f_tilde, double *rho, double *ux,
                double *uy) {
  if (!p || !f_tilde || !rho || !ux || !uy || p->nx < 1 || p->ny < 1) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  for (size_t k = 0; k < n; ++k) {
    double f9[9];
    for (int a = 0; a < 9; ++a) f9[a] = f_tilde[a * n + k];
    moments_of(&v, f9, &rho[k], &ux[k], &uy[k]);
  }
  return ORC_OK;
}

int orc_conserved(const orc_problem *p, const double *f_tilde, double *out) {
  if (!p || !f_tilde || !out || p->nx < 1 || p->ny < 1 || !p->xf || !p->yf) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  double m = 0.0, jx = 0.0, jy = 0.0;
  for (int j = 0; j < p->ny; ++j)
    for (int i = 0; i < p->nx; ++i) {
      size_t k = (size_t)j * p->nx + i;
      double vol = (p->xf[i + 1] - p->xf[i]) * (p->yf[j + 1] - p->yf[j]);
      for (int a = 0; a < 9; ++a) {
        double fa = f_tilde[a * n + k];
        m += fa * vol;
        jx += v.xi[a][0] * fa * vol;
        jy += v.xi[a][1] * fa * vol;
      }
    }
  out[0] = m;
  out[1] = jx;
  out[2] = jy;
  return ORC_OK;
}

int orc_l2_error_u(const orc_problem *p, const double *f_tilde, const double *ua,
                   const double *va, double *eu) {
  if (!p || !f_tilde || !ua || !va || !eu || p->nx < 1 || p->ny < 1) return ORC_EINVAL;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  double num = 0.0, den = 0.0;
  for (size_t k = 0; k < n; ++k) {
    double f9[9], rho, ux, uy;
    for (int a = 0; a < 9; ++a) f9[a] = f_tilde[a * n + k];
    moments_of(&v, f9, &rho, &ux, &uy);
    num += (ux - ua[k]) * (ux - ua[k]) + (uy - va[k]) * (uy - va[k]);
    den += ua[k] * ua[k] + va[k] * va[k];
  }
  *eu = sqrt(num) / sqrt(den);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Curvilinear structured meshes (readings in dvbe_oracle.h)            */
/* ------------------------------------------------------------------ */

typedef struct {
  int nx, ny, per_x, per_y;
  double Px[2], Py[2]; /* translation from side W to E, from S to N (periodic) */
  double *cx, *cy;     /* padded centres, i = -2 .. nx+1, j = -2 .. ny+1 */
  double *vol;         /* [ny][nx] */
  /* x-faces [ny][nx+1], y-faces [ny+1][nx]: midpoint, unit normal, area */
  double *xbx, *xby, *xnx, *xny, *xA;
  double *ybx, *yby, *ynx, *yny, *yA;
  const orc_bc_segment **segW, **segE, **segS, **segN;
} qgeom;

#define QIDX(g, i, j) ((size_t)((j) + 2) * ((g)->nx + 4) + (size_t)((i) + 2))
#define QV(p, i, j) ((size_t)(j) * ((p)->nx + 1) + (size_t)(i))

static void qgeom_free(qgeom *g) {
  double *arrs[] = {g->cx, g->cy, g->vol, g->xbx, g->xby, g->xnx, g->xny, g->xA,
                    g->ybx, g->yby, g->ynx, g->yny, g->yA};
  for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) free(arrs[k]);
  free((void *)g->segW);
  free((void *)g->segE);
  free((void *)g->segS);
  free((void *)g->segN);
  memset(g, 0, sizeof(*g));
}

/* Mirror of point (x, y) across the line through (bx, by) with unit normal n. */
static void mirror(double x, double y, double bx, double by, double nx_, double ny_,
                   double *mx, double *my) {
  const double s = (x - bx) * nx_ + (y - by) * ny_;
  *mx = x - 2.0 * s * nx_;
  *my = y - 2.0 * s * ny_;
}

static int axis_normal(double nx_, double ny_) {
  return fabs(fabs(nx_) - 1.0) <= 1e-12 || fabs(fabs(ny_) - 1.0) <= 1e-12;
}

static int qgeom_build(const orc_quad_problem *p, qgeom *g) {
  memset(g, 0, sizeof(*g));
  if (!p || p->nx < 2 || p->ny < 2 || !p->X || !p->Y) return ORC_EINVAL;
  if (!(p->RT > 0.0) || !(p->tau > 0.0) || !(p->dt > 0.0)) return ORC_EINVAL;
  if (p->scheme < ORC_DUGKS || p->scheme > ORC_CFREE_CENTRAL) return ORC_EINVAL;
  if (p->recon != ORC_RECON_LINEAR && p->recon != ORC_RECON_UPWIND_CELL) return ORC_EINVAL;
  int per[4];
  for (int s = 0; s < 4; ++s) {
    if (p->nbc[s] < 1 || !p->bc[s]) return ORC_EINVAL;
    per[s] = 0;
    for (int k = 0; k < p->nbc[s]; ++k) {
      if (!kind_valid(p->bc[s][k].kind)) return ORC_EINVAL;
      if (p->bc[s][k].kind == ORC_BC_PERIODIC) per[s] = 1;
    }
    if (per[s] && p->nbc[s] != 1) return ORC_EINVAL;
  }
  if (per[ORC_SIDE_W] != per[ORC_SIDE_E] || per[ORC_SIDE_S] != per[ORC_SIDE_N]) return ORC_EINVAL;
  const int nx = p->nx, ny = p->ny;
  g->nx = nx;
  g->ny = ny;
  g->per_x = per[ORC_SIDE_W];
  g->per_y = per[ORC_SIDE_S];
  const size_t np = (size_t)(nx + 4) * (ny + 4), nfx = (size_t)(nx + 1) * ny, nfy = (size_t)nx * (ny + 1);
  g->cx = calloc(np, sizeof(double));
  g->cy = calloc(np, sizeof(double));
  g->vol = calloc((size_t)nx * ny, sizeof(double));
  double **fx[5] = {&g->xbx, &g->xby, &g->xnx, &g->xny, &g->xA};
  double **fy[5] = {&g->ybx, &g->yby, &g->ynx, &g->yny, &g->yA};
  for (int q = 0; q < 5; ++q) {
    *fx[q] = calloc(nfx, sizeof(double));
    *fy[q] = calloc(nfy, sizeof(double));
  }
  g->segW = calloc(ny, sizeof(void *));
  g->segE = calloc(ny, sizeof(void *));
  g->segS = calloc(nx, sizeof(void *));
  g->segN = calloc(nx, sizeof(void *));
  if (!g->cx || !g->cy || !g->vol || !g->xA || !g->yA || !g->segW || !g->segE || !g->segS || !g->segN) {
    qgeom_free(g);
    return ORC_EINVAL;
  }
  const double *X = p->X, *Y = p->Y;
  /* periodic translations */
  g->Px[0] = X[QV(p, nx, 0)] - X[QV(p, 0, 0)];
  g->Px[1] = Y[QV(p, nx, 0)] - Y[QV(p, 0, 0)];
  g->Py[0] = X[QV(p, 0, ny)] - X[QV(p, 0, 0)];
  g->Py[1] = Y[QV(p, 0, ny)] - Y[QV(p, 0, 0)];
  /* cells */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x0 = X[QV(p, i, j)], x1 = X[QV(p, i + 1, j)], x2 = X[QV(p, i + 1, j + 1)], x3 = X[QV(p, i, j + 1)];
      const double y0 = Y[QV(p, i, j)], y1 = Y[QV(p, i + 1, j)], y2 = Y[QV(p, i + 1, j + 1)], y3 = Y[QV(p, i, j + 1)];
      g->cx[QIDX(g, i, j)] = 0.25 * (x0 + x1 + x2 + x3);
      g->cy[QIDX(g, i, j)] = 0.25 * (y0 + y1 + y2 + y3);
      const double area = 0.5 * ((x0 * y1 - x1 * y0) + (x1 * y2 - x2 * y1) + (x2 * y3 - x3 * y2) + (x3 * y0 - x0 * y3));
      if (!(area > 0.0)) {
        qgeom_free(g);
        return ORC_EINVAL;
      }
      g->vol[(size_t)j * nx + i] = area;
    }
  /* faces */
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k <= nx; ++k) {
      const double ax = X[QV(p, k, j)], ay = Y[QV(p, k, j)], bx = X[QV(p, k, j + 1)], by = Y[QV(p, k, j + 1)];
      const double tx = bx - ax, ty = by - ay, len = sqrt(tx * tx + ty * ty);
      const size_t f = (size_t)j * (nx + 1) + k;
      g->xbx[f] = 0.5 * (ax + bx);
      g->xby[f] = 0.5 * (ay + by);
      g->xnx[f] = ty / len;
      g->xny[f] = -tx / len;
      g->xA[f] = len;
    }
  for (int k = 0; k <= ny; ++k)
    for (int i = 0; i < nx; ++i) {
      const double ax = X[QV(p, i, k)], ay = Y[QV(p, i, k)], bx = X[QV(p, i + 1, k)], by = Y[QV(p, i + 1, k)];
      const double tx = bx - ax, ty = by - ay, len = sqrt(tx * tx + ty * ty);
      const size_t f = (size_t)k * nx + i;
      g->ybx[f] = 0.5 * (ax + bx);
      g->yby[f] = 0.5 * (ay + by);
      g->ynx[f] = -ty / len;
      g->yny[f] = tx / len;
      g->yA[f] = len;
    }
  /* ghost centres: x sides over the inner rows, then y sides over the padded width */
  for (int j = 0; j < ny; ++j) {
    if (g->per_x) {
      for (int l = 1; l <= 2; ++l) {
        g->cx[QIDX(g, -l, j)] = g->cx[QIDX(g, nx - l, j)] - g->Px[0];
        g->cy[QIDX(g, -l, j)] = g->cy[QIDX(g, nx - l, j)] - g->Px[1];
        g->cx[QIDX(g, nx - 1 + l, j)] = g->cx[QIDX(g, l - 1, j)] + g->Px[0];
        g->cy[QIDX(g, nx - 1 + l, j)] = g->cy[QIDX(g, l - 1, j)] + g->Px[1];
      }
    } else {
      for (int side = 0; side < 2; ++side) {
        const int i1 = side == 0 ? 0 : nx - 1, ig = side == 0 ? -1 : nx, ig2 = side == 0 ? -2 : nx + 1;
        const size_t f = (size_t)j * (nx + 1) + (side == 0 ? 0 : nx);
        mirror(g->cx[QIDX(g, i1, j)], g->cy[QIDX(g, i1, j)], g->xbx[f], g->xby[f], g->xnx[f], g->xny[f],
               &g->cx[QIDX(g, ig, j)], &g->cy[QIDX(g, ig, j)]);
        g->cx[QIDX(g, ig2, j)] = 2.0 * g->cx[QIDX(g, ig, j)] - g->cx[QIDX(g, i1, j)];
        g->cy[QIDX(g, ig2, j)] = 2.0 * g->cy[QIDX(g, ig, j)] - g->cy[QIDX(g, i1, j)];
      }
    }
  }
  for (int i = -2; i <= nx + 1; ++i) {
    if (g->per_y) {
      for (int l = 1; l <= 2; ++l) {
        g->cx[QIDX(g, i, -l)] = g->cx[QIDX(g, i, ny - l)] - g->Py[0];
        g->cy[QIDX(g, i, -l)] = g->cy[QIDX(g, i, ny - l)] - g->Py[1];
        g->cx[QIDX(g, i, ny - 1 + l)] = g->cx[QIDX(g, i, l - 1)] + g->Py[0];
        g->cy[QIDX(g, i, ny - 1 + l)] = g->cy[QIDX(g, i, l - 1)] + g->Py[1];
      }
    } else {
      const int ic = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
      for (int side = 0; side < 2; ++side) {
        const int j1 = side == 0 ? 0 : ny - 1, jg = side == 0 ? -1 : ny, jg2 = side == 0 ? -2 : ny + 1;
        const size_t f = (size_t)(side == 0 ? 0 : ny) * nx + ic;
        mirror(g->cx[QIDX(g, i, j1)], g->cy[QIDX(g, i, j1)], g->ybx[f], g->yby[f], g->ynx[f], g->yny[f],
               &g->cx[QIDX(g, i, jg)], &g->cy[QIDX(g, i, jg)]);
        g->cx[QIDX(g, i, jg2)] = 2.0 * g->cx[QIDX(g, i, jg)] - g->cx[QIDX(g, i, j1)];
        g->cy[QIDX(g, i, jg2)] = 2.0 * g->cy[QIDX(g, i, jg)] - g->cy[QIDX(g, i, j1)];
      }
    }
  }
  /* boundary segments by face centre; symmetry needs an axis-aligned face */
  for (int j = 0; j < ny; ++j) {
    if (g->per_x) continue;
    const size_t fw = (size_t)j * (nx + 1), fe = fw + nx;
    for (int k = 0; k < p->nbc[ORC_SIDE_W]; ++k)
      if (g->xby[fw] >= p->bc[ORC_SIDE_W][k].s0 && g->xby[fw] < p->bc[ORC_SIDE_W][k].s1) {
        g->segW[j] = &p->bc[ORC_SIDE_W][k];
        break;
      }
    for (int k = 0; k < p->nbc[ORC_SIDE_E]; ++k)
      if (g->xby[fe] >= p->bc[ORC_SIDE_E][k].s0 && g->xby[fe] < p->bc[ORC_SIDE_E][k].s1) {
        g->segE[j] = &p->bc[ORC_SIDE_E][k];
        break;
      }
    if (!g->segW[j] || !g->segE[j] || g->segW[j]->kind == ORC_BC_PERIODIC || g->segE[j]->kind == ORC_BC_PERIODIC ||
        (g->segW[j]->kind == ORC_BC_SYMMETRY && !axis_normal(g->xnx[fw], g->xny[fw])) ||
        (g->segE[j]->kind == ORC_BC_SYMMETRY && !axis_normal(g->xnx[fe], g->xny[fe]))) {
      qgeom_free(g);
      return ORC_EINVAL;
    }
  }
  for (int i = 0; i < nx; ++i) {
    if (g->per_y) continue;
    const size_t fs = (size_t)i, fn = (size_t)ny * nx + i;
    for (int k = 0; k < p->nbc[ORC_SIDE_S]; ++k)
      if (g->ybx[fs] >= p->bc[ORC_SIDE_S][k].s0 && g->ybx[fs] < p->bc[ORC_SIDE_S][k].s1) {
        g->segS[i] = &p->bc[ORC_SIDE_S][k];
        break;
      }
    for (int k = 0; k < p->nbc[ORC_SIDE_N]; ++k)
      if (g->ybx[fn] >= p->bc[ORC_SIDE_N][k].s0 && g->ybx[fn] < p->bc[ORC_SIDE_N][k].s1) {
        g->segN[i] = &p->bc[ORC_SIDE_N][k];
        break;
      }
    if (!g->segS[i] || !g->segN[i] || g->segS[i]->kind == ORC_BC_PERIODIC || g->segN[i]->kind == ORC_BC_PERIODIC ||
        (g->segS[i]->kind == ORC_BC_SYMMETRY && !axis_normal(g->ynx[fs], g->yny[fs])) ||
        (g->segN[i]->kind == ORC_BC_SYMMETRY && !axis_normal(g->ynx[fn], g->yny[fn]))) {
      qgeom_free(g);
      return ORC_EINVAL;
    }
  }
  return ORC_OK;
}

/* Extrapolation factor e = ((x_g - x_1) . n) / ((x_1 - x_2) . n), n the
 * boundary face's normal: the ratio of the distances to the wall. */
static double qext(const qgeom *g, size_t cg, size_t c1, size_t c2, double nx_, double ny_) {
  const double dx = g->cx[c1] - g->cx[c2], dy = g->cy[c1] - g->cy[c2];
  return ((g->cx[cg] - g->cx[c1]) * nx_ + (g->cy[cg] - g->cy[c1]) * ny_) / (dx * nx_ + dy * ny_);
}

/* Mirror map of a symmetry face: the one of the axis its normal lies on. */
static const int *qmir(const vset *v, double nx_) { return fabs(nx_) > 0.5 ? v->mirx : v->miry; }

static void qfill_ghosts(const vset *v, const qgeom *g, double *P) {
  const int nx = g->nx, ny = g->ny;
  const size_t plane = (size_t)(nx + 4) * (ny + 4);
  double p1[9], p2[9], pg[9];
  for (int j = 0; j < ny; ++j) {
    for (int side = 0; side < 2; ++side) {
      if (g->per_x) {
        for (int l = 1; l <= 2; ++l) {
          const int ig = side == 0 ? -l : nx - 1 + l, src = side == 0 ? nx - l : l - 1;
          for (int a = 0; a < 9; ++a) P[a * plane + QIDX(g, ig, j)] = P[a * plane + QIDX(g, src, j)];
        }
        continue;
      }
      const int ig = side == 0 ? -1 : nx, i1 = side == 0 ? 0 : nx - 1, i2 = side == 0 ? 1 : nx - 2;
      for (int a = 0; a < 9; ++a) {
        p1[a] = P[a * plane + QIDX(g, i1, j)];
        p2[a] = P[a * plane + QIDX(g, i2, j)];
      }
      const size_t f = (size_t)j * (nx + 1) + (side == 0 ? 0 : nx);
      const double e = qext(g, QIDX(g, ig, j), QIDX(g, i1, j), QIDX(g, i2, j), g->xnx[f], g->xny[f]);
      ghost_rule(v, side == 0 ? g->segW[j] : g->segE[j], e, qmir(v, g->xnx[f]), p1, p2, pg);
      for (int a = 0; a < 9; ++a) P[a * plane + QIDX(g, ig, j)] = pg[a];
    }
  }
  const int ilo = g->per_x ? -2 : -1, ihi = g->per_x ? nx + 1 : nx;
  for (int i = ilo; i <= ihi; ++i) {
    const int ic = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
    for (int side = 0; side < 2; ++side) {
      if (g->per_y) {
        for (int l = 1; l <= 2; ++l) {
          const int jg = side == 0 ? -l : ny - 1 + l, src = side == 0 ? ny - l : l - 1;
          for (int a = 0; a < 9; ++a) P[a * plane + QIDX(g, i, jg)] = P[a * plane + QIDX(g, i, src)];
        }
        continue;
      }
      const int jg = side == 0 ? -1 : ny, j1 = side == 0 ? 0 : ny - 1, j2 = side == 0 ? 1 : ny - 2;
      for (int a = 0; a < 9; ++a) {
        p1[a] = P[a * plane + QIDX(g, i, j1)];
        p2[a] = P[a * plane + QIDX(g, i, j2)];
      }
      const size_t f = (size_t)(side == 0 ? 0 : ny) * nx + ic;
      const double e = qext(g, QIDX(g, i, jg), QIDX(g, i, j1), QIDX(g, i, j2), g->ynx[f], g->yny[f]);
      ghost_rule(v, side == 0 ? g->segS[ic] : g->segN[ic], e, qmir(v, g->ynx[f]), p1, p2, pg);
      for (int a = 0; a < 9; ++a) P[a * plane + QIDX(g, i, jg)] = pg[a];
    }
  }
}

/* Gradient of field Pa at padded cell (i, j) by central differences along
 * the two mesh lines (one-sided toward the inside at the outer layer of a
 * non-periodic side), grad = J^-T (d_i, d_j). */
static void qgrad(const qgeom *g, const double *Pa, int i, int j, double *gx, double *gy) {
  int im = i - 1, ip = i + 1, jm = j - 1, jp = j + 1;
  if (!g->per_x && i <= -1) im = i;
  if (!g->per_x && i >= g->nx) ip = i;
  if (!g->per_y && j <= -1) jm = j;
  if (!g->per_y && j >= g->ny) jp = j;
  const double pi = Pa[QIDX(g, ip, j)] - Pa[QIDX(g, im, j)];
  const double pj = Pa[QIDX(g, i, jp)] - Pa[QIDX(g, i, jm)];
  const double xi_ = g->cx[QIDX(g, ip, j)] - g->cx[QIDX(g, im, j)];
  const double yi_ = g->cy[QIDX(g, ip, j)] - g->cy[QIDX(g, im, j)];
  const double xj_ = g->cx[QIDX(g, i, jp)] - g->cx[QIDX(g, i, jm)];
  const double yj_ = g->cy[QIDX(g, i, jp)] - g->cy[QIDX(g, i, jm)];
  const double det = xi_ * yj_ - yi_ * xj_;
  *gx = (pi * yj_ - yi_ * pj) / det;
  *gy = (xi_ * pj - pi * xj_) / det;
}

/* phi(x_b - h xi) at a face with midpoint (bx, by) and unit normal n between
 * padded cells L and R; upwind: the upwind-cell form is allowed here. */
static void qrecon(const vset *v, const qgeom *g, const double *P, int iL, int jL, int iR, int jR,
                   double bx, double by, double nx_, double ny_, double h, int upwind, double *out) {
  const size_t plane = (size_t)(g->nx + 4) * (g->ny + 4);
  const size_t L = QIDX(g, iL, jL), R = QIDX(g, iR, jR);
  const double dx = g->cx[R] - g->cx[L], dy = g->cy[R] - g->cy[L], dn = dx * nx_ + dy * ny_;
  const double th = ((bx - g->cx[L]) * nx_ + (by - g->cy[L]) * ny_) / dn;
  const double ox = bx - (g->cx[L] + th * dx), oy = by - (g->cy[L] + th * dy);
  for (int a = 0; a < 9; ++a) {
    const double *Pa = P + a * plane;
    const double xn = v->xi[a][0] * nx_ + v->xi[a][1] * ny_;
    if (upwind && xn != 0.0) {
      const int iC = xn > 0.0 ? iL : iR, jC = xn > 0.0 ? jL : jR;
      const size_t C = QIDX(g, iC, jC);
      double gx, gy;
      qgrad(g, Pa, iC, jC, &gx, &gy);
      out[a] = Pa[C] + (bx - h * v->xi[a][0] - g->cx[C]) * gx + (by - h * v->xi[a][1] - g->cy[C]) * gy;
      continue;
    }
    double glx, gly, grx, gry;
    qgrad(g, Pa, iL, jL, &glx, &gly);
    qgrad(g, Pa, iR, jR, &grx, &gry);
    const double gbx = (1.0 - th) * glx + th * grx, gby = (1.0 - th) * gly + th * gry;
    const double pb = (1.0 - th) * Pa[L] + th * Pa[R] + gbx * ox + gby * oy;
    const double corr = ((Pa[R] - Pa[L]) - (gbx * dx + gby * dy)) / dn;
    const double gfx = gbx + corr * nx_, gfy = gby + corr * ny_;
    out[a] = pb - h * (v->xi[a][0] * gfx + v->xi[a][1] * gfy);
  }
}

static int qstep_once(const orc_quad_problem *p, const vset *v, const qgeom *g, double *ft,
                      double *P, double *TP, double *FX, double *FY) {
  const int nx = g->nx, ny = g->ny;
  const size_t n = (size_t)nx * ny, plane = (size_t)(nx + 4) * (ny + 4);
  const size_t nfx = (size_t)(nx + 1) * ny, nfy = (size_t)nx * (ny + 1);
  const double dt = p->dt, tau = p->tau, h = 0.5 * dt;
  double f9[9], fe[9], rho, ux, uy, val[9];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)j * nx + i;
      for (int a = 0; a < 9; ++a) f9[a] = ft[a * n + k];
      moments_of(v, f9, &rho, &ux, &uy);
      feq_of(v, rho, ux, uy, fe);
      for (int a = 0; a < 9; ++a) {
        double tplus, phi;
        cell_stage(p->scheme, tau, dt, f9[a], fe[a], &tplus, &phi);
        TP[a * n + k] = tplus;
        P[a * plane + QIDX(g, i, j)] = phi;
      }
    }
  qfill_ghosts(v, g, P);
  const double hs = face_shift(p->scheme, h);
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k <= nx; ++k) {
      const size_t f = (size_t)j * (nx + 1) + k;
      const int upw = p->recon == ORC_RECON_UPWIND_CELL && (g->per_x || (k > 0 && k < nx));
      qrecon(v, g, P, k - 1, j, k, j, g->xbx[f], g->xby[f], g->xnx[f], g->xny[f], hs, upw, val);
      if (!g->per_x && k == 0) face_bc(v, g->segW[j], -g->xnx[f], -g->xny[f], val);
      if (!g->per_x && k == nx) face_bc(v, g->segE[j], g->xnx[f], g->xny[f], val);
      face_to_f(v, (const orc_problem *)&(orc_problem){.dt = p->dt, .tau = p->tau, .scheme = p->scheme}, val);
      for (int a = 0; a < 9; ++a) FX[(size_t)a * nfx + f] = val[a];
    }
  for (int k = 0; k <= ny; ++k)
    for (int i = 0; i < nx; ++i) {
      const size_t f = (size_t)k * nx + i;
      const int upw = p->recon == ORC_RECON_UPWIND_CELL && (g->per_y || (k > 0 && k < ny));
      qrecon(v, g, P, i, k - 1, i, k, g->ybx[f], g->yby[f], g->ynx[f], g->yny[f], hs, upw, val);
      if (!g->per_y && k == 0) face_bc(v, g->segS[i], -g->ynx[f], -g->yny[f], val);
      if (!g->per_y && k == ny) face_bc(v, g->segN[i], g->ynx[f], g->yny[f], val);
      face_to_f(v, (const orc_problem *)&(orc_problem){.dt = p->dt, .tau = p->tau, .scheme = p->scheme}, val);
      for (int a = 0; a < 9; ++a) FY[(size_t)a * nfy + f] = val[a];
    }
  /* f_tilde^{n+1} = f_tilde^+ - dt/|V| sum_faces (xi . n_out) A f_face */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)j * nx + i;
      const size_t fw = (size_t)j * (nx + 1) + i, fe_ = fw + 1, fs = (size_t)j * nx + i, fn = fs + nx;
      for (int a = 0; a < 9; ++a) {
        const double x0 = v->xi[a][0], x1 = v->xi[a][1];
        const double out_flux =
            (x0 * g->xnx[fe_] + x1 * g->xny[fe_]) * g->xA[fe_] * FX[(size_t)a * nfx + fe_] -
            (x0 * g->xnx[fw] + x1 * g->xny[fw]) * g->xA[fw] * FX[(size_t)a * nfx + fw] +
            (x0 * g->ynx[fn] + x1 * g->yny[fn]) * g->yA[fn] * FY[(size_t)a * nfy + fn] -
            (x0 * g->ynx[fs] + x1 * g->yny[fs]) * g->yA[fs] * FY[(size_t)a * nfy + fs];
        ft[a * n + k] = TP[a * n + k] - dt / g->vol[k] * out_flux;
      }
    }
  return ORC_OK;
}

int orc_quad_step(const orc_quad_problem *p, double *f_tilde, long long nsteps) {
  if (!f_tilde || nsteps < 0) return ORC_EINVAL;
  qgeom g;
  int rc = qgeom_build(p, &g);
  if (rc) return rc;
  vset v;
  make_vset(p->RT, &v);
  const int nx = p->nx, ny = p->ny;
  double *P = calloc((size_t)9 * (nx + 4) * (ny + 4), sizeof(double));
  double *TP = calloc((size_t)9 * nx * ny, sizeof(double));
  double *FX = calloc((size_t)9 * (nx + 1) * ny, sizeof(double));
  double *FY = calloc((size_t)9 * nx * (ny + 1), sizeof(double));
  if (!P || !TP || !FX || !FY) rc = ORC_EINVAL;
  for (long long s = 0; s < nsteps && !rc; ++s) rc = qstep_once(p, &v, &g, f_tilde, P, TP, FX, FY);
  free(P);
  free(TP);
  free(FX);
  free(FY);
  qgeom_free(&g);
  return rc;
}

int orc_quad_geometry(const orc_quad_problem *p, double *xc, double *yc, double *vol) {
  qgeom g;
  int rc = qgeom_build(p, &g);
  if (rc) return rc;
  for (int j = 0; j < p->ny; ++j)
    for (int i = 0; i < p->nx; ++i) {
      const size_t k = (size_t)j * p->nx + i;
      if (xc) xc[k] = g.cx[QIDX(&g, i, j)];
      if (yc) yc[k] = g.cy[QIDX(&g, i, j)];
      if (vol) vol[k] = g.vol[k];
    }
  qgeom_free(&g);
  return ORC_OK;
}

int orc_quad_conserved(const orc_quad_problem *p, const double *f_tilde, double *out) {
  if (!f_tilde || !out) return ORC_EINVAL;
  qgeom g;
  int rc = qgeom_build(p, &g);
  if (rc) return rc;
  vset v;
  make_vset(p->RT, &v);
  const size_t n = (size_t)p->nx * p->ny;
  double m = 0.0, jx = 0.0, jy = 0.0;
  for (size_t k = 0; k < n; ++k)
    for (int a = 0; a < 9; ++a) {
      const double fa = f_tilde[a * n + k];
      m += fa * g.vol[k];
      jx += v.xi[a][0] * fa * g.vol[k];
      jy += v.xi[a][1] * fa * g.vol[k];
    }
  out[0] = m;
  out[1] = jx;
  out[2] = jy;
  qgeom_free(&g);
  return ORC_OK;
}

int orc_quad_dt_from_cfl(const orc_quad_problem *p, double cfl, double *dt) {
  if (!p || !dt || !(cfl > 0.0) || !(p->RT > 0.0)) return ORC_EINVAL;
  double dmin = INFINITY;
  for (int j = 0; j <= p->ny; ++j)
    for (int i = 0; i <= p->nx; ++i) {
      if (i < p->nx) {
        const double dx = p->X[QV(p, i + 1, j)] - p->X[QV(p, i, j)], dy = p->Y[QV(p, i + 1, j)] - p->Y[QV(p, i, j)];
        const double l = sqrt(dx * dx + dy * dy);
        if (l < dmin) dmin = l;
      }
      if (j < p->ny) {
        const double dx = p->X[QV(p, i, j + 1)] - p->X[QV(p, i, j)], dy = p->Y[QV(p, i, j + 1)] - p->Y[QV(p, i, j)];
        const double l = sqrt(dx * dx + dy * dy);
        if (l < dmin) dmin = l;
      }
    }
  *dt = cfl * dmin / (sqrt(6.0) * sqrt(p->RT));
  return ORC_OK;
}
