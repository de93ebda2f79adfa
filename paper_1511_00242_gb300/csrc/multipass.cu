// Multi-pass step with face arrays, one kernel per stage: the form of the
// paper's own implementation, which holds extra arrays of distributions and
// moments at the cell faces (Sec 3.1).  It carries the reconstruction
// variants and the quadrilateral meshes the fused strip kernel does not.
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
// The arithmetic is on f_tilde itself, in the storage's precision: FP64, or
// FP32 (absolute storage; the equilibrium then takes the exact-sum weights
// of EqCoef, so the collision keeps mass and momentum up to unbiased
// rounding).  The geometry tables are those of the fused kernel (CaseArgs)
// plus the foot offsets of the upwind cells, all in that precision.
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

// Equilibrium weights in the arithmetic's precision: FP64 the rounded 4/9,
// 1/9, 1/36; FP32 the exact-sum weights of EqCoef (their sum is 1 in FP32).
template <typename R> __device__ __forceinline__ R wgt(int a);
template <> __device__ __forceinline__ double wgt<double>(int a) { return WGT(a); }
template <> __device__ __forceinline__ float wgt<float>(int a) {
  using C = dev::EqCoef<float>;
  return a == 0 ? C::W0 : (a <= 4 ? C::W1 : C::W2);
}

template <typename R> __device__ __forceinline__ void feq9(R rho, R Ux, R Uy, R *f) {
  // Eq. equilibrium with U = u / c: w rho (1 + 3 e.U + 4.5 (e.U)^2 - 1.5 |U|^2)
  const R u2 = Ux * Ux + Uy * Uy;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const R eu = R(EX(a)) * Ux + R(EY(a)) * Uy;
    f[a] = wgt<R>(a) * rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * u2);
  }
}

template <typename R> __device__ __forceinline__ void mom9(const R *f, R &rho, R &Ux, R &Uy) {
  R r = 0, mx = 0, my = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    r += f[a];
    mx += R(EX(a)) * f[a];
    my += R(EY(a)) * f[a];
  }
  rho = r;
  Ux = mx / r;
  Uy = my / r;
}

template <typename R> __global__ void k_stage(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const R *f = (const R *)A.fin;
  R *phi = (R *)m.phi, *tp = (R *)m.tp;
  const R bphi = R(A.b_phi), btp = R(m.b_tp);
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const long long idx = (long long)j * A.pitch + i;
    R d[9], fe[9], rho, Ux, Uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) d[a] = f[a * A.plane + idx];
    mom9(d, rho, Ux, Uy);
    if (!(rho > R(0) && rho < R(1e30))) atomicOr(A.flag, 1u);
    feq9(rho, Ux, Uy, fe);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      phi[a * m.pplane + pidx(m, i, j)] = d[a] + bphi * (fe[a] - d[a]);
      tp[a * n + k] = d[a] + btp * (fe[a] - d[a]);
    }
  }
}

template <typename R> __global__ void k_ghost_x(CaseArgs A, MPArgs m) {
  const int j = blockIdx.x * T + threadIdx.x;
  if (j >= A.ny) return;
  R *P = (R *)m.phi;
  for (int side = 0; side < 2; ++side) {
    if (A.per_x) {
      for (int l = 1; l <= 2; ++l) {
        const int ig = side == 0 ? -l : A.nx - 1 + l, src = side == 0 ? A.nx - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = P[a * m.pplane + pidx(m, src, j)];
      }
      continue;
    }
    const int ig = side == 0 ? -1 : A.nx, i1 = side == 0 ? 0 : A.nx - 1, i2 = side == 0 ? 1 : A.nx - 2;
    R p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i1, j)];
      p2[a] = P[a * m.pplane + pidx(m, i2, j)];
      g[a] = R(0);
    }
    dev::apply_ghost<R, true>(A.seg[side][A.segid[side][j]], R(A.ext[side]), R(0), p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = g[a];
  }
}

template <typename R> __global__ void k_ghost_y(CaseArgs A, MPArgs m) {
  const int i = blockIdx.x * T + threadIdx.x - 2; // -2 .. nx+1
  if (i > A.nx + 1) return;
  R *P = (R *)m.phi;
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
    R p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i, j1)];
      p2[a] = P[a * m.pplane + pidx(m, i, j2)];
      g[a] = R(0);
    }
    dev::apply_ghost<R, false>(A.seg[side][A.segid[side][ic]], R(A.ext[side]), R(0), p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = g[a];
  }
}

// DUGKS face moments and back-transform f = f_bar + q (f_eq - f_bar).
template <typename R> __device__ __forceinline__ void dugks_back(const CaseArgs &A, R *F) {
  R rho, Ux, Uy, fe[9];
  mom9(F, rho, Ux, Uy);
  feq9(rho, Ux, Uy, fe);
  const R q = R(A.q_face);
#pragma unroll
  for (int a = 0; a < 9; ++a) F[a] += q * (fe[a] - F[a]);
}

// x-face k between cells k-1 and k, row j.  Tables: xfth[k+1] theta and
// xfs[k+1] = h c / (x_k - x_{k-1}) (CaseArgs, FP64); m.xg[c+2] = h c /
// (x_{c+1} - x_{c-1}) for cells c = -2 .. nx+1 (m.yg likewise); m.xoff[2k],
// [2k+1] = (x_b - x_C) / (h c) for C = k-1 and C = k.
template <typename R> __global__ void k_faces_x(CaseArgs A, MPArgs m) {
  const long long n = (long long)(A.nx + 1) * A.ny;
  const R *xfth = (const R *)A.xfth, *xfs = (const R *)A.xfs;
  const R *P = (const R *)m.phi;
  const R *xg = (const R *)m.xg, *yg = (const R *)m.yg, *xoff = (const R *)m.xoff;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int j = (int)(t / (A.nx + 1)), k = (int)(t % (A.nx + 1));
    const R th = xfth[k + 1], s = xfs[k + 1], ty = yg[j + 2];
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_x || (k > 0 && k < A.nx));
    R F[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R *Pa = P + a * m.pplane;
      if (upw && EX(a) != 0) {
        const int C = EX(a) > 0 ? k - 1 : k;
        const R gx = (Pa[pidx(m, C + 1, j)] - Pa[pidx(m, C - 1, j)]) * xg[C + 2];
        const R gy = (Pa[pidx(m, C, j + 1)] - Pa[pidx(m, C, j - 1)]) * ty;
        const R off = xoff[2 * k + (EX(a) > 0 ? 0 : 1)];
        F[a] = Pa[pidx(m, C, j)] + (off - R(EX(a))) * gx - R(EY(a)) * gy;
        continue;
      }
      const R pl = Pa[pidx(m, k - 1, j)], pr = Pa[pidx(m, k, j)];
      const R gl = (Pa[pidx(m, k - 1, j + 1)] - Pa[pidx(m, k - 1, j - 1)]) * ty;
      const R gr = (Pa[pidx(m, k, j + 1)] - Pa[pidx(m, k, j - 1)]) * ty;
      F[a] = (R(1) - th) * pl + th * pr - R(EX(a)) * s * (pr - pl) - R(EY(a)) * ((R(1) - th) * gl + th * gr);
    }
    if (!A.per_x && (k == 0 || k == A.nx)) {
      const int side = k == 0 ? 0 : 1;
      dev::face_bc<R>(A.seg[side][A.segid[side][j]], side == 0 ? -1 : 1, 0, R(0), F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) ((R *)m.fx)[a * n + t] = F[a];
  }
}

template <typename R> __global__ void k_faces_y(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * (A.ny + 1);
  const R *yfth = (const R *)A.yfth, *yfs = (const R *)A.yfs;
  const R *P = (const R *)m.phi;
  const R *xg = (const R *)m.xg, *yg = (const R *)m.yg, *yoff = (const R *)m.yoff;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int k = (int)(t / A.nx), i = (int)(t % A.nx);
    const R th = yfth[k + 1], s = yfs[k + 1], tx = xg[i + 2];
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_y || (k > 0 && k < A.ny));
    R F[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R *Pa = P + a * m.pplane;
      if (upw && EY(a) != 0) {
        const int C = EY(a) > 0 ? k - 1 : k;
        const R gy = (Pa[pidx(m, i, C + 1)] - Pa[pidx(m, i, C - 1)]) * yg[C + 2];
        const R gx = (Pa[pidx(m, i + 1, C)] - Pa[pidx(m, i - 1, C)]) * tx;
        const R off = yoff[2 * k + (EY(a) > 0 ? 0 : 1)];
        F[a] = Pa[pidx(m, i, C)] + (off - R(EY(a))) * gy - R(EX(a)) * gx;
        continue;
      }
      const R pl = Pa[pidx(m, i, k - 1)], pr = Pa[pidx(m, i, k)];
      const R gl = (Pa[pidx(m, i + 1, k - 1)] - Pa[pidx(m, i - 1, k - 1)]) * tx;
      const R gr = (Pa[pidx(m, i + 1, k)] - Pa[pidx(m, i - 1, k)]) * tx;
      F[a] = (R(1) - th) * pl + th * pr - R(EY(a)) * s * (pr - pl) - R(EX(a)) * ((R(1) - th) * gl + th * gr);
    }
    if (!A.per_y && (k == 0 || k == A.ny)) {
      const int side = k == 0 ? 2 : 3;
      dev::face_bc<R>(A.seg[side][A.segid[side][i]], 0, side == 2 ? -1 : 1, R(0), F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) ((R *)m.fy)[a * n + t] = F[a];
  }
}

template <typename R> __global__ void k_update(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const long long nfx = (long long)(A.nx + 1) * A.ny, nfy = (long long)A.nx * (A.ny + 1);
  const R *xcu = (const R *)A.xcu, *ycu = (const R *)A.ycu;
  const R *tp = (const R *)m.tp, *fx = (const R *)m.fx, *fy = (const R *)m.fy;
  R *fo = (R *)A.fout;
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const R cx = xcu[i + 1], cy = ycu[j + 1];
    const long long w = (long long)j * (A.nx + 1) + i, s = (long long)j * A.nx + i;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      R v = tp[a * n + k];
      if (EX(a) != 0) v -= cx * R(EX(a)) * (fx[a * nfx + w + 1] - fx[a * nfx + w]);
      if (EY(a) != 0) v -= cy * R(EY(a)) * (fy[a * nfy + s + A.nx] - fy[a * nfy + s]);
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
template <typename R>
__device__ __forceinline__ void qgrad(const CaseArgs &A, const MPArgs &m, const R *Pa, int i, int j,
                                      R &gx, R &gy) {
  const int im = (!A.per_x && i <= -1) ? i : i - 1, ip = (!A.per_x && i >= A.nx) ? i : i + 1;
  const int jm = (!A.per_y && j <= -1) ? j : j - 1, jp = (!A.per_y && j >= A.ny) ? j : j + 1;
  const R di = Pa[pidx(m, ip, j)] - Pa[pidx(m, im, j)];
  const R dj = Pa[pidx(m, i, jp)] - Pa[pidx(m, i, jm)];
  const long long c = pidx(m, i, j);
  const R *J = (const R *)m.jinv;
  gx = J[c] * di + J[m.pplane + c] * dj;
  gy = J[2 * m.pplane + c] * di + J[3 * m.pplane + c] * dj;
}

// Sec 2.5 at a boundary face with outward normal (nxo, nyo) of any
// orientation, on full f.  Only directions crossing the face change.
template <typename R> __device__ __forceinline__ void qface_bc(const SegParam &sp, R nxo, R nyo, R (&F)[9]) {
  if (sp.kind == DVBE_BC_WALL_BOUNCEBACK) {
    const R ux = R(sp.ux), uy = R(sp.uy);
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (R(EX(a)) * nxo + R(EY(a)) * nyo > R(0))
        F[dev::OPP(a)] = F[a] - R(6.0 * WGT(a)) * (R(EX(a)) * ux + R(EY(a)) * uy);
  } else if (sp.kind == DVBE_BC_WALL_DIFFUSE) {
    R f1[9];
    feq9(R(1), R(sp.ux), R(sp.uy), f1);
    R num = 0, den = 0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const R en = R(EX(a)) * nxo + R(EY(a)) * nyo;
      if (en > R(0)) num += en * F[a];
      if (en < R(0)) den -= en * f1[a];
    }
    const R rw = num / den;
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (R(EX(a)) * nxo + R(EY(a)) * nyo < R(0)) F[a] = rw * f1[a];
  } else if (sp.kind == DVBE_BC_INFLOW_EQ) {
    R fe[9];
    feq9(R(sp.rho), R(sp.ux), R(sp.uy), fe);
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (R(EX(a)) * nxo + R(EY(a)) * nyo < R(0)) F[a] = fe[a];
  }
}

template <typename R> __global__ void k_qghost_x(CaseArgs A, MPArgs m) {
  const int j = blockIdx.x * T + threadIdx.x;
  if (j >= A.ny) return;
  R *P = (R *)m.phi;
  const R *ext = (const R *)m.qext;
  for (int side = 0; side < 2; ++side) {
    if (A.per_x) {
      for (int l = 1; l <= 2; ++l) {
        const int ig = side == 0 ? -l : A.nx - 1 + l, src = side == 0 ? A.nx - l : l - 1;
        for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = P[a * m.pplane + pidx(m, src, j)];
      }
      continue;
    }
    const int ig = side == 0 ? -1 : A.nx, i1 = side == 0 ? 0 : A.nx - 1, i2 = side == 0 ? 1 : A.nx - 2;
    R p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i1, j)];
      p2[a] = P[a * m.pplane + pidx(m, i2, j)];
      g[a] = R(0);
    }
    const long long q = (long long)side * A.ny + j;
    const SegParam &sp = A.seg[side][A.segid[side][j]];
    if (m.qmir[q])
      dev::apply_ghost<R, true>(sp, ext[q], R(0), p1, p2, g);
    else
      dev::apply_ghost<R, false>(sp, ext[q], R(0), p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, ig, j)] = g[a];
  }
}

template <typename R> __global__ void k_qghost_y(CaseArgs A, MPArgs m) {
  const int lo = A.per_x ? -2 : -1, hi = A.per_x ? A.nx + 1 : A.nx;
  const int i = blockIdx.x * T + threadIdx.x + lo;
  if (i > hi) return;
  R *P = (R *)m.phi;
  const R *ext = (const R *)m.qext;
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
    R p1[9], p2[9], g[9];
    for (int a = 0; a < 9; ++a) {
      p1[a] = P[a * m.pplane + pidx(m, i, j1)];
      p2[a] = P[a * m.pplane + pidx(m, i, j2)];
      g[a] = R(0);
    }
    const long long q = 2LL * A.ny + (long long)(side - 2) * (A.nx + 4) + (i + 2);
    const SegParam &sp = A.seg[side][A.segid[side][ic]];
    if (m.qmir[q])
      dev::apply_ghost<R, true>(sp, ext[q], R(0), p1, p2, g);
    else
      dev::apply_ghost<R, false>(sp, ext[q], R(0), p1, p2, g);
    for (int a = 0; a < 9; ++a) P[a * m.pplane + pidx(m, i, jg)] = g[a];
  }
}

// One face between padded cells L = (iL, jL) and R = (iR, jR); tab[r * nf + f]
// its tables.  Writes the nine face values phi(x_b - h xi).
template <typename R>
__device__ __forceinline__ void qface(const CaseArgs &A, const MPArgs &m, const R *tab, long long nf,
                                      long long f, int iL, int jL, int iR, int jR, bool upwind,
                                      R (&F)[9]) {
  const R th = tab[QF_TH * nf + f], ox = tab[QF_OX * nf + f], oy = tab[QF_OY * nf + f];
  const R dx = tab[QF_DX * nf + f], dy = tab[QF_DY * nf + f];
  const R tx = tab[QF_TX * nf + f], ty = tab[QF_TY * nf + f];
  const R bx = tab[QF_BX * nf + f], by = tab[QF_BY * nf + f];
  const R nx = tab[QF_NX * nf + f], ny = tab[QF_NY * nf + f];
  const R es = R(m.eshift);
  const long long cl = pidx(m, iL, jL), cr = pidx(m, iR, jR);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const R *Pa = (const R *)m.phi + a * m.pplane;
    const R ex = R(EX(a)), ey = R(EY(a));
    const R en = ex * nx + ey * ny;
    if (upwind && en != R(0)) {
      R gx, gy;
      if (en > R(0)) {
        qgrad(A, m, Pa, iL, jL, gx, gy);
        F[a] = Pa[cl] + (bx - ex) * gx + (by - ey) * gy;
      } else {
        qgrad(A, m, Pa, iR, jR, gx, gy);
        F[a] = Pa[cr] + (bx - dx - ex) * gx + (by - dy - ey) * gy;
      }
      continue;
    }
    R glx, gly, grx, gry;
    qgrad(A, m, Pa, iL, jL, glx, gly);
    qgrad(A, m, Pa, iR, jR, grx, gry);
    const R gbx = (R(1) - th) * glx + th * grx, gby = (R(1) - th) * gly + th * gry;
    const R pb = (R(1) - th) * Pa[cl] + th * Pa[cr] + gbx * ox + gby * oy;
    const R corr = (Pa[cr] - Pa[cl]) - (gbx * dx + gby * dy);
    const R gfx = gbx + corr * tx, gfy = gby + corr * ty;
    F[a] = pb - es * (ex * gfx + ey * gfy);
  }
}

template <typename R> __global__ void k_qfaces_x(CaseArgs A, MPArgs m) {
  const long long n = (long long)(A.nx + 1) * A.ny;
  const R *bnt = (const R *)m.qbn;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int j = (int)(t / (A.nx + 1)), k = (int)(t % (A.nx + 1));
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_x || (k > 0 && k < A.nx));
    R F[9];
    qface(A, m, (const R *)m.qfx, n, t, k - 1, j, k, j, upw, F);
    if (!A.per_x && (k == 0 || k == A.nx)) {
      const int side = k == 0 ? 0 : 1;
      const R *bn = bnt + (long long)side * 2 * A.ny + 2 * j;
      qface_bc(A.seg[side][A.segid[side][j]], bn[0], bn[1], F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) ((R *)m.fx)[a * n + t] = F[a];
  }
}

template <typename R> __global__ void k_qfaces_y(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * (A.ny + 1);
  const R *bnt = (const R *)m.qbn;
  for (long long t = blockIdx.x * (long long)T + threadIdx.x; t < n; t += (long long)gridDim.x * T) {
    const int k = (int)(t / A.nx), i = (int)(t % A.nx);
    const bool upw = m.recon == DVBE_RECON_UPWIND_CELL && (A.per_y || (k > 0 && k < A.ny));
    R F[9];
    qface(A, m, (const R *)m.qfy, n, t, i, k - 1, i, k, upw, F);
    if (!A.per_y && (k == 0 || k == A.ny)) {
      const int side = k == 0 ? 2 : 3;
      const R *bn = bnt + 4LL * A.ny + (long long)(side - 2) * 2 * A.nx + 2 * i;
      qface_bc(A.seg[side][A.segid[side][i]], bn[0], bn[1], F);
    }
    if (m.scheme == SC_DUGKS) dugks_back(A, F);
#pragma unroll
    for (int a = 0; a < 9; ++a) ((R *)m.fy)[a * n + t] = F[a];
  }
}

// f_tilde^{n+1} = f_tilde^+ - dt c / |V| sum over the faces of (e . n_out A) f_face
template <typename R> __global__ void k_qupdate(CaseArgs A, MPArgs m) {
  const long long n = (long long)A.nx * A.ny;
  const long long nfx = (long long)(A.nx + 1) * A.ny, nfy = (long long)A.nx * (A.ny + 1);
  const R *qfx = (const R *)m.qfx, *qfy = (const R *)m.qfy;
  const R *ax = qfx + QF_AX * nfx, *ay = qfx + QF_AY * nfx;
  const R *bx = qfy + QF_AX * nfy, *by = qfy + QF_AY * nfy;
  const R *tp = (const R *)m.tp, *fx = (const R *)m.fx, *fy = (const R *)m.fy, *vsc = (const R *)m.vs;
  R *fo = (R *)A.fout;
  for (long long k = blockIdx.x * (long long)T + threadIdx.x; k < n; k += (long long)gridDim.x * T) {
    const int j = (int)(k / A.nx), i = (int)(k % A.nx);
    const long long w = (long long)j * (A.nx + 1) + i, s = (long long)j * A.nx + i, nn = s + A.nx;
    const R vs = vsc[k];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R ex = R(EX(a)), ey = R(EY(a));
      const R flux = (ex * ax[w + 1] + ey * ay[w + 1]) * fx[a * nfx + w + 1] -
                     (ex * ax[w] + ey * ay[w]) * fx[a * nfx + w] +
                     (ex * bx[nn] + ey * by[nn]) * fy[a * nfy + nn] -
                     (ex * bx[s] + ey * by[s]) * fy[a * nfy + s];
      fo[a * A.plane + (long long)j * A.pitch + i] = tp[a * n + k] - vs * flux;
    }
  }
}

int grid(long long n) {
  long long g = (n + T - 1) / T;
  return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

} // namespace mp

template <typename R> static cudaError_t launch_mp(const CaseArgs &a, const MPArgs &m, cudaStream_t s) {
  using namespace mp;
  if (m.quad) {
    k_stage<R><<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
    k_qghost_x<R><<<grid(a.ny), T, 0, s>>>(a, m);
    k_qghost_y<R><<<grid(a.nx + 4), T, 0, s>>>(a, m);
    k_qfaces_x<R><<<grid((long long)(a.nx + 1) * a.ny), T, 0, s>>>(a, m);
    k_qfaces_y<R><<<grid((long long)a.nx * (a.ny + 1)), T, 0, s>>>(a, m);
    k_qupdate<R><<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
    return cudaGetLastError();
  }
  k_stage<R><<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
  k_ghost_x<R><<<grid(a.ny), T, 0, s>>>(a, m);
  k_ghost_y<R><<<grid(a.nx + 4), T, 0, s>>>(a, m);
  k_faces_x<R><<<grid((long long)(a.nx + 1) * a.ny), T, 0, s>>>(a, m);
  k_faces_y<R><<<grid((long long)a.nx * (a.ny + 1)), T, 0, s>>>(a, m);
  k_update<R><<<grid((long long)a.nx * a.ny), T, 0, s>>>(a, m);
  return cudaGetLastError();
}

cudaError_t launch_multipass(const CaseArgs &a, const MPArgs &m, cudaStream_t s) {
  return m.elem == 8 ? launch_mp<double>(a, m, s) : launch_mp<float>(a, m, s);
}

} // namespace dvbe
