// Multi-pass FP64 step with face arrays: the form of the step the paper's
// implementation keeps ("two sets of additional DFs and macro variables at
// cell faces", Sec 3.1), one kernel per stage, for the reconstruction
// variants the fused strip kernel does not carry.
//
//   1. cell stage: phi (f_bar^+ for DUGKS, f_tilde^+ for BKG, the cell f^n
//      for the collision-free faces) into a padded array with two ghost
//      layers, and f_tilde^+ of every cell;
//   2. ghost layers: x sides over the inner rows, then y sides over the
//      padded width (Sec 2.5; periodic sides copy two layers);
//   3. x faces, 4. y faces: phi at x_b - h xi by the linear reconstruction
//      (Eqs. eq_char, f_left) or the upwind-cell one (phi_C + (x_b - h xi -
//      x_C) . grad phi_C, central-difference gradient of the upwind cell C;
//      directions along the face and faces on non-periodic sides keep the
//      linear one), the boundary face rules, and for DUGKS the face moments
//      and back-transform to f (Sec 2.2);
//   5. update f_tilde^{n+1} = f_tilde^+ - dt/|V| sum (xi . n) A f_face.
//
// Everything is FP64 on f_tilde itself; the geometry tables are those of
// the fused kernel (CaseArgs) plus the foot offsets of the upwind cells.
// Quadrilateral meshes run the same stages with their own ghost, face and
// update kernels (tables of quad_mesh.cu).
#include "capi_common.h"
#include "step_kernel.cuh"

namespace dvbe {
namespace mp {

using dev::EX;
using dev::EY;
using dev::WGT;

constexpr int T = 256;

// Padded index of cell (i, j), i in -2 .. nx+1, j in -2 .. ny+1.
__device__ __forceinline__ long long pidx(const MPArgs &m, int i, int j) {
  return (long long)(j + 2) * (m.nx + 4) + (i + 2);
}

__device__ __forceinline__ void feq9(double rho, double Ux, double Uy, double *f) {
  // Eq. equilibrium with U = u / c: w rho (1 + 3 e.U + 4.5 (e.U)^2 - 1.5 |U|^2)
  const double u2 = Ux * Ux + Uy * Uy;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double eu = EX(a) * Ux + EY(a) * Uy;
    f[a] = WGT(a) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u2);
  }
}

__device__ __forceinline__ void mom9(const double *f, double &rho, double &Ux, double &Uy) {
  double r = 0, mx = 0, my = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    r += f[a];
    mx += EX(a) * f[a];
    my += EY(a) * f[a];
  }
  rho = r;
  Ux = mx / r;
  Uy = my / r;
}

__global__ void k_stage(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const double *f = (const double *)A.fin;
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const long long idx = (long long)j * A.pitch + i;
    double d[9], fe[9], rho, Ux, Uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) d[a] = f[a * A.plane + idx];
    mom9(d, rho, Ux, Uy);
    if (!(rho > 0 && rho < 1e30)) atomicOr(A.flag, 1u);
    feq9(rho, Ux, Uy, fe);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      m.phi[a * m.pplane + pidx(m, i, j)] = d[a] + A.b_phi * (fe[a] - d[a]);
      m.tp[a * n + k] = d[a] + m.b_tp * (fe[a] - d[a]);
    }
  }
}

__global__ void k_ghost_x(CaseArgs A, MPArgs m) {
  const int j = blockIdx.x * T + threadIdx.x;
  if (j >= A.ny) return;
  double *P = m.phi;
  for (int side = 0; side < 2; ++side) {
    if (A.per_x) {
      for (int l = 1; l <= 2; ++l) {
        const int ig = side == 0 ? -l : A.nx - 1 + l, src = side == 0 ? A.nx - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = P[a * m.pplane + pidx(m, src, j)];
      }
      continue;
    }
    const int ig = side == 0 ? -1 : A.nx, i1 = side == 0 ? 0 : A.nx - 1, i2 = side == 0 ? 1 : A.nx - 2;
    double p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i1, j)];
      p2[a] = P[a * m.pplane + pidx(m, i2, j)];
      g[a] = 0.0;
    }
    dev::apply_ghost<double, true>(A.seg[side][A.segid[side][j]], A.ext[side], 0.0, p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = g[a];
  }
}

__global__ void k_ghost_y(CaseArgs A, MPArgs m) {
  const int i = blockIdx.x * T + threadIdx.x - 2; // -2 .. nx+1
  if (i > A.nx + 1) return;
  double *P = m.phi;
  const int ic = min(max(i, 0), A.nx - 1);
  for (int side = 2; side < 4; ++side) {
    if (A.per_y) {
      for (int l = 1; l <= 2; ++l) {
        const int jg = side == 2 ? -l : A.ny - 1 + l, src = side == 2 ? A.ny - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = P[a * m.pplane + pidx(m, i, src)];
      }
      continue;
    }
    const int jg = side == 2 ? -1 : A.ny, j1 = side == 2 ? 0 : A.ny - 1, j2 = side == 2 ? 1 : A.ny - 2;
    double p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i, j1)];
      p2[a] = P[a * m.pplane + pidx(m, i, j2)];
      g[a] = 0.0;
    }
    dev::apply_ghost<double, false>(A.seg[side][A.segid[side][ic]], A.ext[side], 0.0, p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = g[a];
  }
}

// DUGKS face moments and back-transform f = f_bar + q (f_eq - f_bar).
__device__ __forceinline__ void dugks_back(const CaseArgs &A, double *F) {
  double rho, Ux, Uy, fe[9];
  mom9(F, rho, Ux, Uy);
  feq9(rho, Ux, Uy, fe);
#pragma unroll
  for (int a = 0; a < 9; ++a) F[a] += A.q_face * (fe[a] - F[a]);
}

// x-face k between cells k-1 and k, row j.  Tables: xfth[k+1] theta and
// xfs[k+1] = h c / (x_k - x_{k-1}) (CaseArgs, FP64); m.xg[c+2] = h c /
// (x_{c+1} - x_{c-1}) for cells c = -2 .. nx+1 (m.yg likewise); m.xoff[2k],
// [2k+1] = (x_b - x_C) / (h c) for C = k-1 and C = k.
__global__ void k_faces_x(CaseArgs A, MPArgs m) {
  const long long n = (long long)(A.nx + 1) * A.ny;
  const double *xfth = (const double *)A.xfth, *xfs = (const double *)A.xfs;
  const double *P = m.phi;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int j = (int)(t / (A.nx + 1)), k = (int)(t % (A.nx + 1));
    const double th = xfth[k + 1], s = xfs[k + 1], ty = m.yg[j + 2];
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_x || (k > 0 && k < A.nx));
    double F[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double *Pa = P + a * m.pplane;
      if (upw && EX(a) != 0) {
        const int C = EX(a) > 0 ? k - 1 : k;
        const double gx = (Pa[pidx(m, C + 1, j)] - Pa[pidx(m, C - 1, j)]) * m.xg[C + 2];
        const double gy = (Pa[pidx(m, C, j + 1)] - Pa[pidx(m, C, j - 1)]) * ty;
        const double off = m.xoff[2 * k + (EX(a) > 0 ? 0 : 1)];
        F[a] = Pa[pidx(m, C, j)] + (off - EX(a)) * gx - EY(a) * gy;
        continue;
      }
      const double pl = Pa[pidx(m, k - 1, j)], pr = Pa[pidx(m, k, j)];
      const double gl = (Pa[pidx(m, k - 1, j + 1)] - Pa[pidx(m, k - 1, j - 1)]) * ty;
      const double gr = (Pa[pidx(m, k, j + 1)] - Pa[pidx(m, k, j - 1)]) * ty;
      F[a] = (1.0 - th) * pl + th * pr - EX(a) * s * (pr - pl) - EY(a) * ((1.0 - th) * gl + th * gr);
    }
    if (!A.per_x && (k == 0 || k == A.nx)) {
      const int side = k == 0 ? 0 : 1;
      dev::face_bc<double>(A.seg[side][A.segid[side][j]], side == 0 ? -1 : 1, 0, 0.0, F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) m.fx[a * n + t] = F[a];
  }
}

__global__ void k_faces_y(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * (A.ny + 1);
  const double *yfth = (const double *)A.yfth, *yfs = (const double *)A.yfs;
  const double *P = m.phi;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int k = (int)(t / A.nx), i = (int)(t % A.nx);
    const double th = yfth[k + 1], s = yfs[k + 1], tx = m.xg[i + 2];
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_y || (k > 0 && k < A.ny));
    double F[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double *Pa = P + a * m.pplane;
      if (upw && EY(a) != 0) {
        const int C = EY(a) > 0 ? k - 1 : k;
        const double gy = (Pa[pidx(m, i, C + 1)] - Pa[pidx(m, i, C - 1)]) * m.yg[C + 2];
        const double gx = (Pa[pidx(m, i + 1, C)] - Pa[pidx(m, i - 1, C)]) * tx;
        const double off = m.yoff[2 * k + (EY(a) > 0 ? 0 : 1)];
        F[a] = Pa[pidx(m, i, C)] + (off - EY(a)) * gy - EX(a) * gx;
        continue;
      }
      const double pl = Pa[pidx(m, i, k - 1)], pr = Pa[pidx(m, i, k)];
      const double gl = (Pa[pidx(m, i + 1, k - 1)] - Pa[pidx(m, i - 1, k - 1)]) * tx;
      const double gr = (Pa[pidx(m, i + 1, k)] - Pa[pidx(m, i - 1, k)]) * tx;
      F[a] = (1.0 - th) * pl + th * pr - EY(a) * s * (pr - pl) - EX(a) * ((1.0 - th) * gl + th * gr);
    }
    if (!A.per_y && (k == 0 || k == A.ny)) {
      const int side = k == 0 ? 2 : 3;
      dev::face_bc<double>(A.seg[side][A.segid[side][i]], 0, side == 2 ? -1 : 1, 0.0, F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) m.fy[a * n + t] = F[a];
  }
}

__global__ void k_update(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const long long nfx = (long long)(A.nx + 1) * A.ny, nfy = (long long)A.nx * (A.ny + 1);
  const double *xcu = (const double *)A.xcu, *ycu = (const double *)A.ycu;
  double *fo = (double *)A.fout;
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const double cx = xcu[i + 1], cy = ycu[j + 1];
    const long long w = (long long)j * (A.nx + 1) + i, s = (long long)j * A.nx + i;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      double v = m.tp[a * n + k];
      if (EX(a) != 0) v -= cx * EX(a) * (m.fx[a * nfx + w + 1] - m.fx[a * nfx + w]);
      if (EY(a) != 0) v -= cy * EY(a) * (m.fy[a * nfy + s + A.nx] - m.fy[a * nfy + s]);
      fo[a * A.plane + (long long)j * A.pitch + i] = v;
    }
  }
}

// ---- quadrilateral meshes -------------------------------------------------
//
// Tables (QuadHost, lengths over s = h c): per padded cell s J^-T, per face
// theta, the offset o of the face midpoint from the centre line, d = x_R -
// x_L, the correction direction n s / (d . n), x_b - x_L, the unit normal n
// and n A.  The face value is
//   linear:      phi_b - e . g,  phi_b = (1 - theta) phi_L + theta phi_R + gbar . o,
//                g = gbar + ((phi_R - phi_L) - gbar . d) n s / (d . n)
//   upwind cell: phi_C + ((x_b - x_C) / s - e) . grad_C
// with gbar the theta-blend of the cells' gradients (all scaled by s) and
// e = xi / c; the central collision-free face drops the e . g term.

// s grad phi at padded cell (i, j): central differences along the mesh
// lines, one-sided at the outer ghost layer of a side that is not periodic.
__device__ __forceinline__ void qgrad(const CaseArgs &A, const MPArgs &m, const double *Pa, int i,
                                      int j, double &gx, double &gy) {
  const int im = (!A.per_x && i <= -1) ? i : i - 1, ip = (!A.per_x && i >= A.nx) ? i : i + 1;
  const int jm = (!A.per_y && j <= -1) ? j : j - 1, jp = (!A.per_y && j >= A.ny) ? j : j + 1;
  const double di = Pa[pidx(m, ip, j)] - Pa[pidx(m, im, j)];
  const double dj = Pa[pidx(m, i, jp)] - Pa[pidx(m, i, jm)];
  const long long c = pidx(m, i, j);
  gx = m.jinv[c] * di + m.jinv[m.pplane + c] * dj;
  gy = m.jinv[2 * m.pplane + c] * di + m.jinv[3 * m.pplane + c] * dj;
}

// Sec 2.5 at a boundary face with outward normal (nxo, nyo) of any
// orientation: full f (FP64).  Only directions crossing the face change.
__device__ __forceinline__ void qface_bc(const SegParam &sp, double nxo, double nyo, double (&F)[9]) {
  if (sp.kind == DVBE_BC_WALL_BOUNCEBACK) {
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (EX(a) * nxo + EY(a) * nyo > 0)
        F[dev::OPP(a)] = F[a] - 6.0 * WGT(a) * (EX(a) * sp.ux + EY(a) * sp.uy);
  } else if (sp.kind == DVBE_BC_WALL_DIFFUSE) {
    double f1[9];
    feq9(1.0, sp.ux, sp.uy, f1);
    double num = 0, den = 0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const double en = EX(a) * nxo + EY(a) * nyo;
      if (en > 0) num += en * F[a];
      if (en < 0) den -= en * f1[a];
    }
    const double rw = num / den;
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (EX(a) * nxo + EY(a) * nyo < 0) F[a] = rw * f1[a];
  } else if (sp.kind == DVBE_BC_INFLOW_EQ) {
    double fe[9];
    feq9(sp.rho, sp.ux, sp.uy, fe);
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (EX(a) * nxo + EY(a) * nyo < 0) F[a] = fe[a];
  }
}

__global__ void k_qghost_x(CaseArgs A, MPArgs m) {
  const int j = blockIdx.x * T + threadIdx.x;
  if (j >= A.ny) return;
  double *P = m.phi;
  for (int side = 0; side < 2; ++side) {
    if (A.per_x) {
      for (int l = 1; l <= 2; ++l) {
        const int ig = side == 0 ? -l : A.nx - 1 + l, src = side == 0 ? A.nx - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = P[a * m.pplane + pidx(m, src, j)];
      }
      continue;
    }
    const int ig = side == 0 ? -1 : A.nx, i1 = side == 0 ? 0 : A.nx - 1, i2 = side == 0 ? 1 : A.nx - 2;
    double p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i1, j)];
      p2[a] = P[a * m.pplane + pidx(m, i2, j)];
      g[a] = 0.0;
    }
    const long long q = (long long)side * A.ny + j;
    const SegParam &sp = A.seg[side][A.segid[side][j]];
    if (m.qmir[q])
      dev::apply_ghost<double, true>(sp, m.qext[q], 0.0, p1, p2, g);
    else
      dev::apply_ghost<double, false>(sp, m.qext[q], 0.0, p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = g[a];
  }
}

__global__ void k_qghost_y(CaseArgs A, MPArgs m) {
  const int lo = A.per_x ? -2 : -1, hi = A.per_x ? A.nx + 1 : A.nx;
  const int i = blockIdx.x * T + threadIdx.x + lo;
  if (i > hi) return;
  double *P = m.phi;
  const int ic = min(max(i, 0), A.nx - 1);
  for (int side = 2; side < 4; ++side) {
    if (A.per_y) {
      for (int l = 1; l <= 2; ++l) {
        const int jg = side == 2 ? -l : A.ny - 1 + l, src = side == 2 ? A.ny - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = P[a * m.pplane + pidx(m, i, src)];
      }
      continue;
    }
    const int jg = side == 2 ? -1 : A.ny, j1 = side == 2 ? 0 : A.ny - 1, j2 = side == 2 ? 1 : A.ny - 2;
    double p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i, j1)];
      p2[a] = P[a * m.pplane + pidx(m, i, j2)];
      g[a] = 0.0;
    }
    const long long q = 2LL * A.ny + (long long)(side - 2) * (A.nx + 4) + (i + 2);
    const SegParam &sp = A.seg[side][A.segid[side][ic]];
    if (m.qmir[q])
      dev::apply_ghost<double, true>(sp, m.qext[q], 0.0, p1, p2, g);
    else
      dev::apply_ghost<double, false>(sp, m.qext[q], 0.0, p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = g[a];
  }
}

// One face between padded cells L = (iL, jL) and R = (iR, jR); tab[r * nf + f]
// its tables.  Writes the nine face values phi(x_b - h xi).
__device__ __forceinline__ void qface(const CaseArgs &A, const MPArgs &m, const double *tab,
                                      long long nf, long long f, int iL, int jL, int iR, int jR,
                                      bool upwind, double (&F)[9]) {
  const double th = tab[QF_TH * nf + f], ox = tab[QF_OX * nf + f], oy = tab[QF_OY * nf + f];
  const double dx = tab[QF_DX * nf + f], dy = tab[QF_DY * nf + f];
  const double tx = tab[QF_TX * nf + f], ty = tab[QF_TY * nf + f];
  const double bx = tab[QF_BX * nf + f], by = tab[QF_BY * nf + f];
  const double nx = tab[QF_NX * nf + f], ny = tab[QF_NY * nf + f];
  const long long L = pidx(m, iL, jL), R = pidx(m, iR, jR);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double *Pa = m.phi + a * m.pplane;
    const double en = EX(a) * nx + EY(a) * ny;
    if (upwind && en != 0) {
      double gx, gy;
      if (en > 0) {
        qgrad(A, m, Pa, iL, jL, gx, gy);
        F[a] = Pa[L] + (bx - EX(a)) * gx + (by - EY(a)) * gy;
      } else {
        qgrad(A, m, Pa, iR, jR, gx, gy);
        F[a] = Pa[R] + (bx - dx - EX(a)) * gx + (by - dy - EY(a)) * gy;
      }
      continue;
    }
    double glx, gly, grx, gry;
    qgrad(A, m, Pa, iL, jL, glx, gly);
    qgrad(A, m, Pa, iR, jR, grx, gry);
    const double gbx = (1.0 - th) * glx + th * grx, gby = (1.0 - th) * gly + th * gry;
    const double pb = (1.0 - th) * Pa[L] + th * Pa[R] + gbx * ox + gby * oy;
    const double corr = (Pa[R] - Pa[L]) - (gbx * dx + gby * dy);
    const double gfx = gbx + corr * tx, gfy = gby + corr * ty;
    F[a] = pb - m.eshift * (EX(a) * gfx + EY(a) * gfy);
  }
}

__global__ void k_qfaces_x(CaseArgs A, MPArgs m) {
  const long long n = (long long)(A.nx + 1) * A.ny;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int j = (int)(t / (A.nx + 1)), k = (int)(t % (A.nx + 1));
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_x || (k > 0 && k < A.nx));
    double F[9];
    qface(A, m, m.qfx, n, t, k - 1, j, k, j, upw, F);
    if (!A.per_x && (k == 0 || k == A.nx)) {
      const int side = k == 0 ? 0 : 1;
      const double *bn = m.qbn + (long long)side * 2 * A.ny + 2 * j;
      qface_bc(A.seg[side][A.segid[side][j]], bn[0], bn[1], F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) m.fx[a * n + t] = F[a];
  }
}

__global__ void k_qfaces_y(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * (A.ny + 1);
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int k = (int)(t / A.nx), i = (int)(t % A.nx);
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_y || (k > 0 && k < A.ny));
    double F[9];
    qface(A, m, m.qfy, n, t, i, k - 1, i, k, upw, F);
    if (!A.per_y && (k == 0 || k == A.ny)) {
      const int side = k == 0 ? 2 : 3;
      const double *bn = m.qbn + 4LL * A.ny + (long long)(side - 2) * 2 * A.nx + 2 * i;
      qface_bc(A.seg[side][A.segid[side][i]], bn[0], bn[1], F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) m.fy[a * n + t] = F[a];
  }
}

// f_tilde^{n+1} = f_tilde^+ - dt c / |V| sum over the faces of (e . n_out A) f_face
__global__ void k_qupdate(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const long long nfx = (long long)(A.nx + 1) * A.ny, nfy = (long long)A.nx * (A.ny + 1);
  const double *ax = m.qfx + QF_AX * nfx, *ay = m.qfx + QF_AY * nfx;
  const double *bx = m.qfy + QF_AX * nfy, *by = m.qfy + QF_AY * nfy;
  double *fo = (double *)A.fout;
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const long long w = (long long)j * (A.nx + 1) + i, s = (long long)j * A.nx + i, nn = s + A.nx;
    const double vs = m.vs[k];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double flux = (EX(a) * ax[w + 1] + EY(a) * ay[w + 1]) * m.fx[a * nfx + w + 1] -
                          (EX(a) * ax[w] + EY(a) * ay[w]) * m.fx[a * nfx + w] +
                          (EX(a) * bx[nn] + EY(a) * by[nn]) * m.fy[a * nfy + nn] -
                          (EX(a) * bx[s] + EY(a) * by[s]) * m.fy[a * nfy + s];
      fo[a * A.plane + (long long)j * A.pitch + i] = m.tp[a * n + k] - vs * flux;
    }
  }
}

int grid(long long n) {
  long long g = (n + T - 1) / T;
  return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

} // namespace mp

cudaError_t launch_multipass(const CaseArgs &a, const MPArgs &m, cudaStream_t s) {
  using namespace mp;
  if (m.quad) {
    k_stage<<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
    k_qghost_x<<<grid(a.ny), T, 0, s>>>(a, m);
    k_qghost_y<<<grid(a.nx + 4), T, 0, s>>>(a, m);
    k_qfaces_x<<<grid((long long)(a.nx + 1) * a.ny), T, 0, s>>>(a, m);
    k_qfaces_y<<<grid((long long)a.nx * (a.ny + 1)), T, 0, s>>>(a, m);
    k_qupdate<<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
    return cudaGetLastError();
  }
  k_stage<<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
  k_ghost_x<<<grid(a.ny), T, 0, s>>>(a, m);
  k_ghost_y<<<grid(a.nx + 4), T, 0, s>>>(a, m);
  k_faces_x<<<grid((long long)(a.nx + 1) * a.ny), T, 0, s>>>(a, m);
  k_faces_y<<<grid((long long)a.nx * (a.ny + 1)), T, 0, s>>>(a, m);
  k_update<<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
  return cudaGetLastError();
}

} // namespace dvbe
