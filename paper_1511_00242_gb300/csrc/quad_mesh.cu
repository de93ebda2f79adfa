// Curvilinear structured meshes of general quadrilateral cells: creation,
// validation and the geometry tables of the multi-pass step.
//
// The FV form of Sec 2.2 holds for cells V_k with faces of any orientation;
// Sec 2.4 writes the face reconstruction on uniform meshes only.  The tables
// below carry the reconstruction over with the slope split along the face
// normal: the two-point difference between the cell centres gives the
// normal part, the cells' mesh-line gradients the tangential part (the
// uniform-mesh form when the mesh is a tensor mesh).  Ghost centres are the
// first inner centres mirrored across the boundary face.
#include <cmath>
#include <new>

#include "capi_common.h"

namespace dvbe {

namespace {

struct P2 {
  double x, y;
};
inline P2 operator-(P2 a, P2 b) { return {a.x - b.x, a.y - b.y}; }
inline P2 operator+(P2 a, P2 b) { return {a.x + b.x, a.y + b.y}; }
inline P2 operator*(double s, P2 a) { return {s * a.x, s * a.y}; }
inline double dot(P2 a, P2 b) { return a.x * b.x + a.y * b.y; }

// Geometry of one mesh: padded centres (two ghost layers) and the faces.
struct Geo {
  int nx, ny;
  bool per_x, per_y;
  std::vector<P2> c;            // [(ny+4)(nx+4)]
  std::vector<P2> xb, xn, yb, yn; // face midpoints and unit normals
  std::vector<double> xa, ya;   // face lengths
  P2 px{0, 0}, py{0, 0};        // periodic translations W -> E, S -> N
  long long at(int i, int j) const { return (long long)(j + 2) * (nx + 4) + (i + 2); }
  P2 &C(int i, int j) { return c[at(i, j)]; }
  long long xf(int k, int j) const { return (long long)j * (nx + 1) + k; }
  long long yf(int i, int k) const { return (long long)k * nx + i; }
};

P2 vtx(const dvbe_mesh_ &m, int i, int j) {
  const size_t v = (size_t)j * (m.nx + 1) + i;
  return {m.X[v], m.Y[v]};
}

// Mirror image of p across the line through b with unit normal n.
P2 reflect(P2 p, P2 b, P2 n) { return p - (2.0 * dot(p - b, n)) * n; }

void build_geo(const dvbe_mesh_ &m, bool per_x, bool per_y, Geo &g) {
  const int nx = m.nx, ny = m.ny;
  g.nx = nx;
  g.ny = ny;
  g.per_x = per_x;
  g.per_y = per_y;
  g.c.assign((size_t)(nx + 4) * (ny + 4), P2{0, 0});
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      g.C(i, j) = 0.25 * (vtx(m, i, j) + vtx(m, i + 1, j) + vtx(m, i + 1, j + 1) + vtx(m, i, j + 1));
  g.xb.resize((size_t)(nx + 1) * ny);
  g.xn.resize(g.xb.size());
  g.xa.resize(g.xb.size());
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k <= nx; ++k) {
      const P2 a = vtx(m, k, j), b = vtx(m, k, j + 1), t = b - a;
      const double len = std::sqrt(dot(t, t));
      g.xb[g.xf(k, j)] = 0.5 * (a + b);
      g.xn[g.xf(k, j)] = {t.y / len, -t.x / len}; // towards increasing i
      g.xa[g.xf(k, j)] = len;
    }
  g.yb.resize((size_t)nx * (ny + 1));
  g.yn.resize(g.yb.size());
  g.ya.resize(g.yb.size());
  for (int k = 0; k <= ny; ++k)
    for (int i = 0; i < nx; ++i) {
      const P2 a = vtx(m, i, k), b = vtx(m, i + 1, k), t = b - a;
      const double len = std::sqrt(dot(t, t));
      g.yb[g.yf(i, k)] = 0.5 * (a + b);
      g.yn[g.yf(i, k)] = {-t.y / len, t.x / len}; // towards increasing j
      g.ya[g.yf(i, k)] = len;
    }
  g.px = vtx(m, nx, 0) - vtx(m, 0, 0);
  g.py = vtx(m, 0, ny) - vtx(m, 0, 0);
  // ghost centres: x sides over the inner rows, then y sides over the
  // padded width (the corner ghosts from the x ghosts)
  for (int j = 0; j < ny; ++j) {
    if (per_x) {
      for (int l = 1; l <= 2; ++l) {
        g.C(-l, j) = g.C(nx - l, j) - g.px;
        g.C(nx - 1 + l, j) = g.C(l - 1, j) + g.px;
      }
    } else {
      g.C(-1, j) = reflect(g.C(0, j), g.xb[g.xf(0, j)], g.xn[g.xf(0, j)]);
      g.C(nx, j) = reflect(g.C(nx - 1, j), g.xb[g.xf(nx, j)], g.xn[g.xf(nx, j)]);
    }
  }
  const int ilo = per_x ? -2 : -1, ihi = per_x ? nx + 1 : nx;
  for (int i = ilo; i <= ihi; ++i) {
    if (per_y) {
      for (int l = 1; l <= 2; ++l) {
        g.C(i, -l) = g.C(i, ny - l) - g.py;
        g.C(i, ny - 1 + l) = g.C(i, l - 1) + g.py;
      }
    } else {
      const int ic = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
      g.C(i, -1) = reflect(g.C(i, 0), g.yb[g.yf(ic, 0)], g.yn[g.yf(ic, 0)]);
      g.C(i, ny) = reflect(g.C(i, ny - 1), g.yb[g.yf(ic, ny)], g.yn[g.yf(ic, ny)]);
    }
  }
}

bool along_axis(P2 n) { return std::fabs(std::fabs(n.x) - 1.0) <= 1e-12 || std::fabs(std::fabs(n.y) - 1.0) <= 1e-12; }

int seg_of(const std::vector<dvbe_bc_segment> &segs, double t) {
  for (size_t k = 0; k < segs.size(); ++k)
    if (t >= segs[k].s0 && t < segs[k].s1) return (int)k;
  return -1;
}

} // namespace

dvbe_status quad_tables(const dvbe_mesh_ &m, Problem &pb) {
  const int nx = m.nx, ny = m.ny;
  // periodic pairs must be translates of each other
  {
    double ext = 0;
    for (size_t v = 0; v < m.X.size(); ++v) ext = std::max(ext, std::max(std::fabs(m.X[v]), std::fabs(m.Y[v])));
    const double tol = 1e-12 * std::max(ext, 1.0);
    const P2 px = vtx(m, nx, 0) - vtx(m, 0, 0), py = vtx(m, 0, ny) - vtx(m, 0, 0);
    if (pb.per_x)
      for (int j = 0; j <= ny; ++j) {
        const P2 d = vtx(m, nx, j) - vtx(m, 0, j) - px;
        if (std::fabs(d.x) > tol || std::fabs(d.y) > tol)
          return fail(DVBE_ERR_INVALID_ARG, "periodic W and E sides are not translates of each other");
      }
    if (pb.per_y)
      for (int i = 0; i <= nx; ++i) {
        const P2 d = vtx(m, i, ny) - vtx(m, i, 0) - py;
        if (std::fabs(d.x) > tol || std::fabs(d.y) > tol)
          return fail(DVBE_ERR_INVALID_ARG, "periodic S and N sides are not translates of each other");
      }
  }
  Geo g;
  build_geo(m, pb.per_x, pb.per_y, g);

  QuadHost &q = pb.q;
  const double c = pb.c, h = 0.5 * pb.dt;
  q.eshift = pb.user_scheme == DVBE_CFREE_CENTRAL ? 0.0 : 1.0;
  q.s = q.eshift > 0 ? h * c : 1.0;
  const double s = q.s;

  // cell gradients: s J^-T of the central differences along the mesh lines
  const long long pp = (long long)(nx + 4) * (ny + 4);
  q.jinv.assign(4 * pp, 0.0);
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      const int im = (!pb.per_x && i <= -1) ? i : i - 1, ip = (!pb.per_x && i >= nx) ? i : i + 1;
      const int jm = (!pb.per_y && j <= -1) ? j : j - 1, jp = (!pb.per_y && j >= ny) ? j : j + 1;
      const P2 di = g.C(ip, j) - g.C(im, j), dj = g.C(i, jp) - g.C(i, jm);
      const double det = di.x * dj.y - di.y * dj.x;
      if (!(std::fabs(det) > 0)) continue; // unused corner of the padded array
      const long long k = g.at(i, j);
      q.jinv[0 * pp + k] = s * dj.y / det;
      q.jinv[1 * pp + k] = -s * di.y / det;
      q.jinv[2 * pp + k] = -s * dj.x / det;
      q.jinv[3 * pp + k] = s * di.x / det;
    }

  // face tables
  auto face = [&](std::vector<double> &t, long long nf, long long f, P2 cl, P2 cr, P2 b, P2 n, double len) {
    const P2 d = cr - cl;
    const double dn = dot(d, n), th = dot(b - cl, n) / dn;
    const P2 o = b - (cl + th * d);
    const double v[kQF] = {th, o.x / s, o.y / s, d.x / s, d.y / s, n.x * s / dn, n.y * s / dn,
                           (b - cl).x / s, (b - cl).y / s, n.x, n.y, n.x * len, n.y * len};
    for (int r = 0; r < kQF; ++r) t[(size_t)r * nf + f] = v[r];
    return dn > 0;
  };
  const long long nfx = (long long)(nx + 1) * ny, nfy = (long long)nx * (ny + 1);
  q.fx.assign((size_t)kQF * nfx, 0.0);
  q.fy.assign((size_t)kQF * nfy, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k <= nx; ++k) {
      const long long f = g.xf(k, j);
      if (!face(q.fx, nfx, f, g.C(k - 1, j), g.C(k, j), g.xb[f], g.xn[f], g.xa[f]))
        return fail(DVBE_ERR_INVALID_ARG, "a cell centre lies across its own face (mesh too distorted)");
    }
  for (int k = 0; k <= ny; ++k)
    for (int i = 0; i < nx; ++i) {
      const long long f = g.yf(i, k);
      if (!face(q.fy, nfy, f, g.C(i, k - 1), g.C(i, k), g.yb[f], g.yn[f], g.ya[f]))
        return fail(DVBE_ERR_INVALID_ARG, "a cell centre lies across its own face (mesh too distorted)");
    }

  // cell volumes (shoelace) and the update factor dt c / |V|
  q.vol.resize((size_t)nx * ny);
  q.vs.resize(q.vol.size());
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const P2 v[4] = {vtx(m, i, j), vtx(m, i + 1, j), vtx(m, i + 1, j + 1), vtx(m, i, j + 1)};
      double a2 = 0;
      for (int r = 0; r < 4; ++r) a2 += v[r].x * v[(r + 1) % 4].y - v[(r + 1) % 4].x * v[r].y;
      q.vol[(size_t)j * nx + i] = 0.5 * a2;
      q.vs[(size_t)j * nx + i] = pb.dt * c / (0.5 * a2);
    }

  // ghosts: extrapolation factor along the wall normal, mirror axis,
  // outward normals and segments of the boundary faces
  q.ext.assign(2 * (size_t)ny + 2 * (size_t)(nx + 4), 0.0);
  q.mir.assign(q.ext.size(), 0);
  q.bn.assign(4 * (size_t)ny + 4 * (size_t)nx, 0.0);
  for (int side = 0; side < 4; ++side) pb.segid[side].assign(side < 2 ? ny : nx, 0);
  auto ext_of = [](P2 xg, P2 x1, P2 x2, P2 n) { return dot(xg - x1, n) / dot(x1 - x2, n); };
  auto check_seg = [&](int side, int k, double t, P2 n) -> dvbe_status {
    const int sg = seg_of(pb.bc[side], t);
    if (sg < 0) return fail(DVBE_ERR_INVALID_ARG, "a boundary face is not covered by any segment");
    if (pb.bc[side][sg].kind == DVBE_BC_PERIODIC)
      return fail(DVBE_ERR_INVALID_ARG, "periodic segment on a non-periodic side");
    if (pb.bc[side][sg].kind == DVBE_BC_SYMMETRY && !along_axis(n))
      return fail(DVBE_ERR_INVALID_ARG, "a symmetry side needs faces normal to x or y");
    pb.segid[side][k] = (unsigned char)sg;
    return DVBE_OK;
  };
  if (!pb.per_x)
    for (int side = 0; side < 2; ++side)
      for (int j = 0; j < ny; ++j) {
        const int ig = side == 0 ? -1 : nx, i1 = side == 0 ? 0 : nx - 1, i2 = side == 0 ? 1 : nx - 2;
        const long long f = g.xf(side == 0 ? 0 : nx, j);
        const P2 n = g.xn[f], no = side == 0 ? -1.0 * n : n;
        q.ext[(size_t)side * ny + j] = ext_of(g.C(ig, j), g.C(i1, j), g.C(i2, j), n);
        q.mir[(size_t)side * ny + j] = std::fabs(n.x) > 0.5;
        q.bn[(size_t)side * 2 * ny + 2 * j] = no.x;
        q.bn[(size_t)side * 2 * ny + 2 * j + 1] = no.y;
        dvbe_status st = check_seg(side, j, g.xb[f].y, n);
        if (st != DVBE_OK) return st;
      }
  if (!pb.per_y) {
    const size_t e0 = 2 * (size_t)ny, b0 = 4 * (size_t)ny;
    for (int side = 0; side < 2; ++side) {
      for (int i = -1; i <= nx; ++i) {
        const int ic = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
        const int jg = side == 0 ? -1 : ny, j1 = side == 0 ? 0 : ny - 1, j2 = side == 0 ? 1 : ny - 2;
        const P2 n = g.yn[g.yf(ic, side == 0 ? 0 : ny)];
        q.ext[e0 + (size_t)side * (nx + 4) + (i + 2)] = ext_of(g.C(i, jg), g.C(i, j1), g.C(i, j2), n);
        q.mir[e0 + (size_t)side * (nx + 4) + (i + 2)] = std::fabs(n.x) > 0.5;
      }
      for (int i = 0; i < nx; ++i) {
        const long long f = g.yf(i, side == 0 ? 0 : ny);
        const P2 n = g.yn[f], no = side == 0 ? -1.0 * n : n;
        q.bn[b0 + (size_t)side * 2 * nx + 2 * i] = no.x;
        q.bn[b0 + (size_t)side * 2 * nx + 2 * i + 1] = no.y;
        dvbe_status st = check_seg(2 + side, i, g.yb[f].x, n);
        if (st != DVBE_OK) return st;
      }
    }
  }
  return DVBE_OK;
}

} // namespace dvbe

using dvbe::fail;

extern "C" {

dvbe_status dvbe_mesh_create_quad(int nx, int ny, const double *X, const double *Y, dvbe_mesh *out) {
  if (!out || !X || !Y) return fail(DVBE_ERR_INVALID_ARG, "NULL pointer");
  *out = nullptr;
  if (nx < 2 || ny < 2) return fail(DVBE_ERR_INVALID_ARG, "nx and ny must be >= 2");
  if ((long long)nx * ny > (1LL << 31)) return fail(DVBE_ERR_INVALID_ARG, "mesh too large");
  const size_t nv = (size_t)(nx + 1) * (ny + 1);
  for (size_t v = 0; v < nv; ++v)
    if (!std::isfinite(X[v]) || !std::isfinite(Y[v]))
      return fail(DVBE_ERR_INVALID_ARG, "vertex coordinates must be finite");
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t v[4] = {(size_t)j * (nx + 1) + i, (size_t)j * (nx + 1) + i + 1,
                           (size_t)(j + 1) * (nx + 1) + i + 1, (size_t)(j + 1) * (nx + 1) + i};
      double a2 = 0;
      for (int r = 0; r < 4; ++r) a2 += X[v[r]] * Y[v[(r + 1) % 4]] - X[v[(r + 1) % 4]] * Y[v[r]];
      if (!(a2 > 0))
        return fail(DVBE_ERR_INVALID_ARG, "cell (" + std::to_string(i) + ", " + std::to_string(j) +
                                              ") has no positive area (vertices must run counter-clockwise)");
    }
  dvbe_mesh m = new (std::nothrow) dvbe_mesh_;
  if (!m) return fail(DVBE_ERR_OOM, "host allocation failed");
  m->nx = nx;
  m->ny = ny;
  m->quad = true;
  m->X.assign(X, X + nv);
  m->Y.assign(Y, Y + nv);
  // stand-in face coordinates (cell indices) for the code that sizes tables
  m->xf.resize(nx + 1);
  m->yf.resize(ny + 1);
  for (int i = 0; i <= nx; ++i) m->xf[i] = i;
  for (int j = 0; j <= ny; ++j) m->yf[j] = j;
  *out = m;
  return DVBE_OK;
}

dvbe_status dvbe_mesh_cells(dvbe_mesh m, double *xc, double *yc, double *vol) {
  if (!m) return fail(DVBE_ERR_INVALID_ARG, "NULL mesh");
  const int nx = m->nx, ny = m->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)j * nx + i;
      if (!m->quad) {
        if (xc) xc[k] = 0.5 * (m->xf[i] + m->xf[i + 1]);
        if (yc) yc[k] = 0.5 * (m->yf[j] + m->yf[j + 1]);
        if (vol) vol[k] = (m->xf[i + 1] - m->xf[i]) * (m->yf[j + 1] - m->yf[j]);
        continue;
      }
      const dvbe::P2 v[4] = {dvbe::vtx(*m, i, j), dvbe::vtx(*m, i + 1, j), dvbe::vtx(*m, i + 1, j + 1),
                             dvbe::vtx(*m, i, j + 1)};
      double a2 = 0;
      for (int r = 0; r < 4; ++r) a2 += v[r].x * v[(r + 1) % 4].y - v[(r + 1) % 4].x * v[r].y;
      if (xc) xc[k] = 0.25 * (v[0].x + v[1].x + v[2].x + v[3].x);
      if (yc) yc[k] = 0.25 * (v[0].y + v[1].y + v[2].y + v[3].y);
      if (vol) vol[k] = 0.5 * a2;
    }
  return DVBE_OK;
}

} // extern "C"

namespace dvbe {

double quad_min_edge(const dvbe_mesh_ &m) {
  double dmin = INFINITY;
  for (int j = 0; j <= m.ny; ++j)
    for (int i = 0; i <= m.nx; ++i) {
      if (i < m.nx) {
        const P2 t = vtx(m, i + 1, j) - vtx(m, i, j);
        dmin = std::min(dmin, std::sqrt(dot(t, t)));
      }
      if (j < m.ny) {
        const P2 t = vtx(m, i, j + 1) - vtx(m, i, j);
        dmin = std::min(dmin, std::sqrt(dot(t, t)));
      }
    }
  return dmin;
}

} // namespace dvbe
