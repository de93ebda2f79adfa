// Fused D2Q9 finite-volume step (DUGKS, Sec 2.2; BKG, Sec 2.3) for sm_103a.
//
// Work decomposition.  A warp owns a strip of 32 consecutive columns
// (output columns i0 .. i0+29 plus one halo column on each side) and marches
// up through H rows.  Each lane keeps the reconstruction variable phi of its
// own column for rows j-1, j, j+1 in registers; values of the neighbouring
// columns come from warp shuffles.  Nothing goes through shared memory and no
// block-wide barrier is needed.  Per row and lane:
//   1. load f_tilde of row j+1 (9 coalesced loads), cell stage:
//      rho, u (Eq. macro_var), f_eq (Eq. equilibrium),
//      phi = f_bar^+ (DUGKS, Eq. eq_trans_2) or f_tilde^+ (BKG, Eq. bkg_collision)
//   2. ghost values of phi at non-periodic sides (Sec 2.5)
//   3. the x-face west of the lane's cell: phi(x_b - h xi) by linear
//      reconstruction (Eqs. eq_char / bkg_fb; on a uniform mesh Eq. f_left),
//      split into a left part computed by the left lane and a right part,
//   4. the y-face north of the cell (the south face is the previous row's
//      north face, kept in registers),
//   5. boundary faces: bounce-back / diffuse wall / inflow (Sec 2.5),
//   6. DUGKS: face moments, f_eq at the face and the back-transform to f,
//   7. update f_tilde^{n+1} = f_tilde^+ - dt/|V| sum (xi . n) A f_face
//      (Eqs. eq_update, lwfv, bkg_fv) and store.
// Every face is computed once.  All arithmetic is on deviations
// delta = f_tilde - w_alpha rho0: transforms, reconstruction and the flux
// difference are affine with weights summing to one, so the constant drops
// out and rounding scales with the deviation, not with f_tilde itself.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace dvbe {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// D2Q9 lattice directions (xi = c e, Sec 2.1) and weights.
__host__ __device__ constexpr int EX(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EY(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr double WGT(int a) {
  return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int OPP(int a) {
  return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}
__host__ __device__ constexpr int MIRX(int a) { // e_x -> -e_x
  return a == 1 ? 3 : a == 3 ? 1 : a == 5 ? 6 : a == 6 ? 5 : a == 7 ? 8 : a == 8 ? 7 : a;
}
__host__ __device__ constexpr int MIRY(int a) { // e_y -> -e_y
  return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}

// ---- storage --------------------------------------------------------------

template <int ST> struct StoreT;
template <> struct StoreT<ST_F64> {
  using T = double;
  using Real = double;
  static constexpr bool DEV = false;
};
template <> struct StoreT<ST_F32> {
  using T = float;
  using Real = float;
  static constexpr bool DEV = false;
};
template <> struct StoreT<ST_F32_DEV> {
  using T = float;
  using Real = float;
  static constexpr bool DEV = true;
};
template <> struct StoreT<ST_F16_DEV> {
  using T = __half;
  using Real = float;
  static constexpr bool DEV = true;
};
template <> struct StoreT<ST_BF16_DEV> {
  using T = __nv_bfloat16;
  using Real = float;
  static constexpr bool DEV = true;
};

__device__ __forceinline__ double to_real(double x) { return x; }
__device__ __forceinline__ float to_real(float x) { return x; }
__device__ __forceinline__ float to_real(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_real(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T> __device__ __forceinline__ T from_real(double x);
template <> __device__ __forceinline__ double from_real<double>(double x) { return x; }
template <typename T> __device__ __forceinline__ T from_realf(float x);
template <> __device__ __forceinline__ float from_realf<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_realf<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_realf<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
__device__ __forceinline__ void store_real(double *p, double v) { *p = v; }
template <typename T> __device__ __forceinline__ void store_real(T *p, float v) {
  *p = from_realf<T>(v);
}

__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }

// Weight class of a direction: 0 rest, 1 axis, 2 diagonal.
__host__ __device__ constexpr int WCLS(int a) { return a == 0 ? 0 : (a <= 4 ? 1 : 2); }

// Per-case constants in compute precision.
template <typename Real> struct K {
  Real rho0;
  Real wr[3];  // w rho0 per weight class
  Real sc[3];  // storage scale per weight class (DEV)
  Real isc[3]; // 1 / storage scale
};

template <int ST, typename Real, typename T>
__device__ __forceinline__ Real load_delta(const T *p, int a, const K<Real> &k) {
  Real v = to_real(*p);
  if constexpr (StoreT<ST>::DEV)
    return v * k.sc[WCLS(a)];
  else
    return v - k.wr[WCLS(a)];
}

template <int ST, typename Real, typename T>
__device__ __forceinline__ void store_delta(T *p, int a, Real d, const K<Real> &k) {
  if constexpr (StoreT<ST>::DEV)
    store_real(p, d * k.isc[WCLS(a)]);
  else
    store_real(p, d + k.wr[WCLS(a)]);
}

// delta_eq_alpha = f_eq_alpha - w rho0 = w (rho' + rho P(e.U)) with
// P = 3 eU + 4.5 eU^2 - 1.5 |U|^2 and U = u / c (Eq. equilibrium, c_s^2 = c^2/3).
template <typename Real>
__device__ __forceinline__ Real deq_of(int a, Real rp, Real rho, Real Ux, Real Uy, Real u15) {
  Real eU = Real(EX(a)) * Ux + Real(EY(a)) * Uy;
  Real P = eU * (Real(3) + Real(4.5) * eU) - u15;
  return Real(WGT(a)) * (rp + rho * P);
}

// Moments of a 9-vector of deviations: rho' = sum d, U = (sum e d) / rho.
template <typename Real>
__device__ __forceinline__ void moments(const Real (&d)[9], Real rho0, Real &rp, Real &rho,
                                        Real &Ux, Real &Uy) {
  rp = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
  Real mx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
  Real my = (d[2] - d[4]) + (d[5] - d[8]) + (d[6] - d[7]);
  rho = rho0 + rp;
  Real ri = rcp(rho);
  Ux = mx * ri;
  Uy = my * ri;
}

// Ghost rule for one ghost cell from the first (p1) and second (p2) inner cell.
template <typename Real, bool XSIDE>
__device__ __forceinline__ void apply_ghost(const SegParam &sp, Real e, Real rho0,
                                            const Real (&p1)[9], const Real (&p2)[9],
                                            Real (&g)[9]) {
  const int kind = sp.kind;
  if (kind == DVBE_BC_WALL_BOUNCEBACK || kind == DVBE_BC_WALL_DIFFUSE) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[a] + e * (p1[a] - p2[a]);
  } else if (kind == DVBE_BC_INFLOW_EQ) {
    Real rho = Real(sp.rho), Ux = Real(sp.ux), Uy = Real(sp.uy);
    Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = deq_of<Real>(a, rho - rho0, rho, Ux, Uy, u15);
  } else if (kind == DVBE_BC_OUTFLOW_ZG) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[a];
  } else if (kind == DVBE_BC_SYMMETRY) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[XSIDE ? MIRX(a) : MIRY(a)];
  }
}

// Boundary face treatment (Sec 2.5) on face values fb (deviations), outward
// normal (nx_o, ny_o) of the fluid.  NEED(a) tells which directions the
// caller has computed (BKG skips the ones with zero normal velocity).
template <typename Real>
__device__ __forceinline__ void face_bc(const SegParam &sp, int nxo, int nyo, Real rho0,
                                        Real (&fb)[9]) {
  const int kind = sp.kind;
  if (kind == DVBE_BC_WALL_BOUNCEBACK) {
    // incoming reverse = outgoing - 2 w (xi . U_w) / c_s^2 = outgoing - 6 w (e . U_w / c)
    Real ux = Real(sp.ux), uy = Real(sp.uy);
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      if (EX(a) * nxo + EY(a) * nyo > 0)
        fb[OPP(a)] = fb[a] - Real(6.0 * WGT(a)) * (Real(EX(a)) * ux + Real(EY(a)) * uy);
    }
  } else if (kind == DVBE_BC_WALL_DIFFUSE) {
    // incoming = rho_w f_eq(1, U_w), rho_w from zero normal mass flux
    Real Ux = Real(sp.ux), Uy = Real(sp.uy);
    Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
    Real num = 0, den = 0;
    Real f1[9];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      Real eU = Real(EX(a)) * Ux + Real(EY(a)) * Uy;
      f1[a] = Real(WGT(a)) * (Real(1) + eU * (Real(3) + Real(4.5) * eU) - u15);
      int en = EX(a) * nxo + EY(a) * nyo;
      if (en > 0) num += Real(en) * (fb[a] + Real(WGT(a)) * rho0);
      if (en < 0) den += Real(-en) * f1[a];
    }
    Real rw = num / den;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      if (EX(a) * nxo + EY(a) * nyo < 0) fb[a] = rw * f1[a] - Real(WGT(a)) * rho0;
    }
  } else if (kind == DVBE_BC_INFLOW_EQ) {
    Real rho = Real(sp.rho), Ux = Real(sp.ux), Uy = Real(sp.uy);
    Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
    for (int a = 0; a < 9; ++a) fb[a] = deq_of<Real>(a, rho - rho0, rho, Ux, Uy, u15);
  }
}

// DUGKS: face moments of f_bar, f_eq there and f = p f_bar + q f_eq for the
// directions crossing the face (AXIS 0: x-face, e_x != 0; 1: y-face).
template <typename Real, int AXIS>
__device__ __forceinline__ void dugks_face(Real (&fb)[9], Real rho0, Real p, Real q) {
  Real rp, rho, Ux, Uy;
  moments(fb, rho0, rp, rho, Ux, Uy);
  Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if ((AXIS == 0 ? EX(a) : EY(a)) != 0) fb[a] = p * fb[a] + q * deq_of<Real>(a, rp, rho, Ux, Uy, u15);
  }
}

template <int SCHEME> __host__ __device__ constexpr bool needx(int a) {
  return SCHEME == SC_DUGKS ? true : EX(a) != 0;
}
template <int SCHEME> __host__ __device__ constexpr bool needy(int a) {
  return SCHEME == SC_DUGKS ? true : EY(a) != 0;
}

// ---- the strip ---------------------------------------------------------------

template <int SCHEME, int ST> struct Strip {
  using S = StoreT<ST>;
  using Real = typename S::Real;
  using T = typename S::T;
  static constexpr bool DUG = SCHEME == SC_DUGKS;
  static constexpr bool FD = SCHEME == SC_BKG_FD;

  const CaseArgs &A;
  K<Real> k;
  int lane, i, lc, nx, ny;
  bool per_x, per_y, touchW, touchE, out_lane;
  Real a_phi, b_phi, a_tp, b_tp, p_face, q_face;
  // x-face coefficients of this lane: right part of its west face, left part
  // of its east face; tangential / update factors of its column.
  Real cR[3], cL[3], tR0, tL0, txc, cxu;
  // BKG-FD stencil factors
  Real kx1, kx2, ky1, ky2, kxy;
  int segS, segN;
  const T *fin;
  T *fout;
  bool bad;

  __device__ __forceinline__ Strip(const CaseArgs &args, int lane_) : A(args), lane(lane_) {}

  __device__ __forceinline__ void setup(int sx) {
    nx = A.nx;
    ny = A.ny;
    per_x = A.per_x;
    per_y = A.per_y;
    const int i0 = sx * kStripCols;
    i = i0 - 1 + lane;
    if (i >= 0 && i < nx)
      lc = i;
    else if (per_x && i == -1)
      lc = nx - 1;
    else if (per_x && i == nx)
      lc = 0;
    else
      lc = -1;
    touchW = !per_x && i0 == 0;
    touchE = !per_x && i0 + kStripCols >= nx;
    out_lane = lane >= 1 && lane <= kStripCols && i < nx;
    const int ic = min(max(i, -1), nx);
    const Real *xfth = (const Real *)A.xfth, *xfs = (const Real *)A.xfs;
    const Real *xct = (const Real *)A.xct, *xcu = (const Real *)A.xcu;
    Real thW = xfth[ic + 1], sW = xfs[ic + 1], thE = xfth[ic + 2], sE = xfs[ic + 2];
    cR[0] = thW + sW; // e_x = -1
    cR[1] = thW;
    cR[2] = thW - sW;
    cL[0] = (Real(1) - thE) - sE;
    cL[1] = Real(1) - thE;
    cL[2] = (Real(1) - thE) + sE;
    tR0 = thW;
    tL0 = Real(1) - thE;
    txc = xct[ic + 1];
    cxu = xcu[ic + 1];
    const int icc = min(max(i, 0), nx - 1);
    segS = per_y ? 0 : A.segid[2][icc];
    segN = per_y ? 0 : A.segid[3][icc];
    k.rho0 = Real(A.rho0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double w = c == 0 ? WGT(0) : (c == 1 ? WGT(1) : WGT(5));
      k.wr[c] = Real(w * A.rho0);
      k.sc[c] = Real(A.dev_sigma * w * A.rho0);
      k.isc[c] = Real(1.0 / (A.dev_sigma * w * A.rho0));
    }
    a_phi = Real(A.a_phi);
    b_phi = Real(A.b_phi);
    a_tp = Real(A.a_tp);
    b_tp = Real(A.b_tp);
    p_face = Real(A.p_face);
    q_face = Real(A.q_face);
    if constexpr (FD) {
      Real nux = Real(A.fd_nux), nuy = Real(A.fd_nuy);
      kx1 = Real(0.5) * nux;
      kx2 = Real(0.5) * nux * nux;
      ky1 = Real(0.5) * nuy;
      ky2 = Real(0.5) * nuy * nuy;
      kxy = Real(0.25) * nux * nuy;
    }
    fin = (const T *)A.fin;
    fout = (T *)A.fout;
  }

  // Row r (0 <= r < ny): load, cell stage, x ghosts.
  __device__ __forceinline__ void produce(int r, Real (&phi)[9], Real (&tp)[9]) {
    if (lc >= 0) {
      const T *p = fin + (long long)r * A.pitch + lc;
      Real d[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) d[a] = load_delta<ST, Real>(p + a * A.plane, a, k);
      Real rp, rho, Ux, Uy;
      moments(d, k.rho0, rp, rho, Ux, Uy);
      bad |= !(rho > Real(0) && rho < Real(1e30));
      Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        Real de = deq_of<Real>(a, rp, rho, Ux, Uy, u15);
        phi[a] = a_phi * d[a] + b_phi * de;
        if constexpr (DUG) tp[a] = a_tp * d[a] + b_tp * de;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        phi[a] = Real(0);
        if constexpr (DUG) tp[a] = Real(0);
      }
    }
    if (touchW || touchE) ghost_x(r, phi);
  }

  __device__ __forceinline__ void ghost_x(int r, Real (&phi)[9]) {
    Real q1[9], q2[9];
    if (touchW) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        q1[a] = __shfl_down_sync(kFull, phi[a], 1);
        q2[a] = __shfl_down_sync(kFull, phi[a], 2);
      }
      if (i == -1) apply_ghost<Real, true>(A.seg[0][A.segid[0][r]], Real(A.ext[0]), k.rho0, q1, q2, phi);
    }
    if (touchE) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        q1[a] = __shfl_up_sync(kFull, phi[a], 1);
        q2[a] = __shfl_up_sync(kFull, phi[a], 2);
      }
      if (i == nx) apply_ghost<Real, true>(A.seg[1][A.segid[1][r]], Real(A.ext[1]), k.rho0, q1, q2, phi);
    }
  }

  // Ghost row from the first (p1) and second (p2) inner rows; side 2 = S, 3 = N.
  __device__ __forceinline__ void ghost_row(int side, const Real (&p1)[9], const Real (&p2)[9],
                                            Real (&g)[9]) {
    const SegParam &sp = A.seg[side][side == 2 ? segS : segN];
    apply_ghost<Real, false>(sp, Real(A.ext[side]), k.rho0, p1, p2, g);
  }

  // Flux values of the x-face west of this lane's cell at row j.
  __device__ __forceinline__ void xface(int j, const Real (&Pm)[9], const Real (&P0)[9],
                                        const Real (&Pp)[9], Real (&F)[9]) {
    const Real tyc = ((const Real *)A.yct)[j + 1];
    const Real tL = tyc * tL0, tR = tyc * tR0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (!needx<SCHEME>(a)) continue;
      Real Lp = P0[a] * cL[EX(a) + 1];
      Real Rp = P0[a] * cR[EX(a) + 1];
      if (EY(a) != 0) {
        Real dy = Pp[a] - Pm[a];
        Lp -= Real(EY(a)) * tL * dy;
        Rp -= Real(EY(a)) * tR * dy;
      }
      F[a] = __shfl_up_sync(kFull, Lp, 1) + Rp;
    }
    if (!per_x && (i == 0 || i == nx)) {
      const int side = i == 0 ? 0 : 1;
      face_bc<Real>(A.seg[side][A.segid[side][j]], side == 0 ? -1 : 1, 0, k.rho0, F);
    }
    if constexpr (DUG) dugks_face<Real, 0>(F, k.rho0, p_face, q_face);
  }

  // Flux values of the y-face kf (between rows kf-1 and kf) at this column;
  // Pl = phi of row kf-1, Pu = phi of row kf.
  __device__ __forceinline__ void yface(int kf, const Real (&Pl)[9], const Real (&Pu)[9],
                                        Real (&F)[9]) {
    const Real th = ((const Real *)A.yfth)[kf + 1], s = ((const Real *)A.yfs)[kf + 1];
    const Real a0 = Real(1) - th, b0 = th;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (!needy<SCHEME>(a)) continue;
      Real B = a0 * Pl[a] + b0 * Pu[a];
      Real own;
      if (EY(a) == 0)
        own = B;
      else if (EY(a) > 0)
        own = (a0 + s) * Pl[a] + (b0 - s) * Pu[a];
      else
        own = (a0 - s) * Pl[a] + (b0 + s) * Pu[a];
      if (EX(a) != 0) {
        Real Bn = __shfl_down_sync(kFull, B, 1);
        Real Bs = __shfl_up_sync(kFull, B, 1);
        own -= Real(EX(a)) * txc * (Bn - Bs);
      }
      F[a] = own;
    }
    if (!per_y && (kf == 0 || kf == ny)) {
      const int side = kf == 0 ? 2 : 3;
      face_bc<Real>(A.seg[side][side == 2 ? segS : segN], 0, side == 2 ? -1 : 1, k.rho0, F);
    }
    if constexpr (DUG) dugks_face<Real, 1>(F, k.rho0, p_face, q_face);
  }

  // One row of the finite-volume update.
  __device__ __forceinline__ void update_fv(int j, const Real (&T0)[9], const Real (&FW)[9],
                                            const Real (&FS)[9], const Real (&FN)[9]) {
    const Real cyu = ((const Real *)A.ycu)[j + 1];
    Real v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      v[a] = T0[a];
      if (EX(a) != 0) {
        Real FE = __shfl_down_sync(kFull, FW[a], 1);
        v[a] -= Real(EX(a)) * cxu * (FE - FW[a]);
      }
      if (EY(a) != 0) v[a] -= Real(EY(a)) * cyu * (FN[a] - FS[a]);
    }
    if (out_lane) {
      T *p = fout + (long long)j * A.pitch + i;
#pragma unroll
      for (int a = 0; a < 9; ++a) store_delta<ST, Real>(p + a * A.plane, a, v[a], k);
    }
  }

  // One row of the Lax-Wendroff stencil (Eqs. bkgfd, central_schemes).
  __device__ __forceinline__ void update_fd(int j, const Real (&Pm)[9], const Real (&P0)[9],
                                            const Real (&Pp)[9]) {
    Real v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int ex = EX(a), ey = EY(a);
      // weights C[di][dj] of phi(i+di, j+dj): centre 1 - nx^2 - ny^2;
      // (+-1,0): -+nx/2 + nx^2/2; (0,+-1): -+ny/2 + ny^2/2; corners +-nx ny/4
      const Real cxm = ex ? (Real(ex) * kx1 + kx2) : Real(0); // di = -1
      const Real cxp = ex ? (kx2 - Real(ex) * kx1) : Real(0); // di = +1
      const Real cym = ey ? (Real(ey) * ky1 + ky2) : Real(0);
      const Real cyp = ey ? (ky2 - Real(ey) * ky1) : Real(0);
      const Real cc = Real(1) - (ex ? Real(2) * kx2 : Real(0)) - (ey ? Real(2) * ky2 : Real(0));
      Real M = cc * P0[a];
      if (ey) M += cym * Pm[a] + cyp * Pp[a];
      if (ex) {
        // column parts for the neighbours: this column is di = +1 for the
        // left neighbour and di = -1 for the right one
        Real forL = cxp * P0[a], forR = cxm * P0[a];
        if (ey) {
          const Real kc = Real(ex * ey) * kxy;
          forL += kc * (Pp[a] - Pm[a]);
          forR -= kc * (Pp[a] - Pm[a]);
        }
        M += __shfl_down_sync(kFull, forL, 1) + __shfl_up_sync(kFull, forR, 1);
      }
      v[a] = M;
    }
    if (out_lane) {
      T *p = fout + (long long)j * A.pitch + i;
#pragma unroll
      for (int a = 0; a < 9; ++a) store_delta<ST, Real>(p + a * A.plane, a, v[a], k);
    }
  }

  // One full row: produce row j+1 into Pc (unless have_next), faces, update.
  // Pa, Pb, Pc = phi of rows j-1, j, j+1 (Tb, Tc: f_tilde^+ of rows j, j+1).
  __device__ __forceinline__ void row(int j, bool have_next, Real (&Pa)[9], Real (&Pb)[9],
                                      Real (&Pc)[9], Real (&Tb)[9], Real (&Tc)[9], Real (&FS)[9]) {
    if (!have_next) {
      if (j + 1 < ny)
        produce(j + 1, Pc, Tc);
      else if (per_y)
        produce(0, Pc, Tc);
      else
        ghost_row(3, Pb, Pa, Pc);
    }
    if constexpr (FD) {
      update_fd(j, Pa, Pb, Pc);
    } else {
      Real FW[9], FN[9];
      xface(j, Pa, Pb, Pc, FW);
      yface(j + 1, Pb, Pc, FN);
      update_fv(j, DUG ? Tb : Pb, FW, FS, FN);
#pragma unroll
      for (int a = 0; a < 9; ++a) FS[a] = FN[a];
    }
  }

  __device__ __forceinline__ void run(int sx, int sy) {
    setup(sx);
    const int j0 = sy * A.H;
    const int jend = min(j0 + A.H, ny);
    Real P0[9], P1[9], P2[9], T0[9], T1[9], T2[9], FS[9];
    bool have_next;
    // prologue: rows j0-1 (P0) and j0 (P1) [and j0+1 (P2) at a ghost bottom]
    if (j0 == 0 && !per_y) {
      produce(0, P1, T1);
      produce(1, P2, T2);
      ghost_row(2, P1, P2, P0);
      have_next = true;
    } else {
      produce(j0 == 0 ? ny - 1 : j0 - 1, P0, T0);
      produce(j0, P1, T1);
      have_next = false;
    }
    if constexpr (!FD) yface(j0, P0, P1, FS);
    // rows, unrolled by three so that the phi / f_tilde^+ registers rotate
    // without copies
    int j = j0;
    while (true) {
      if (j >= jend) break;
      row(j, have_next, P0, P1, P2, T1, T2, FS);
      have_next = false;
      if (++j >= jend) break;
      row(j, false, P1, P2, P0, T2, T0, FS);
      if (++j >= jend) break;
      row(j, false, P2, P0, P1, T0, T1, FS);
      ++j;
    }
  }
};

template <int SCHEME, int ST>
__global__ void __launch_bounds__(256) k_step(const __grid_constant__ CaseArgs A) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nitems = (long long)A.strips_x * A.strips_y;
  Strip<SCHEME, ST> s(A, lane);
  s.bad = false;
  for (long long it = gw; it < nitems; it += nw) s.run((int)(it % A.strips_x), (int)(it / A.strips_x));
  if (__any_sync(kFull, s.bad) && lane == 0) atomicOr(A.flag, 1u);
}

// Batched form: warps take strips of all cases from one queue.
template <int SCHEME, int ST>
__global__ void __launch_bounds__(256)
    k_step_batch(const CaseArgs *__restrict__ cases, const long long *__restrict__ prefix,
                 int ncases, long long nitems, unsigned long long *queue) {
  const int lane = threadIdx.x & 31;
  while (true) {
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd(queue, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= nitems) break;
    // case c with prefix[c] <= item < prefix[c+1]
    int lo = 0, hi = ncases;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (prefix[mid] <= item)
        lo = mid;
      else
        hi = mid;
    }
    const CaseArgs &A = cases[lo];
    // diverged case: no longer stepped (read once, so the warp decides as one)
    unsigned dead = 0;
    if (lane == 0) dead = *(volatile unsigned *)A.flag;
    if (__shfl_sync(kFull, dead, 0)) continue;
    const long long local = item - prefix[lo];
    Strip<SCHEME, ST> s(A, lane);
    s.bad = false;
    s.run((int)(local % A.strips_x), (int)(local / A.strips_x));
    if (__any_sync(kFull, s.bad) && lane == 0) atomicOr(A.flag, 1u);
  }
}

} // namespace dev

template <int ST>
cudaError_t launch_step_impl(int scheme, const CaseArgs &a, int blocks, int wpb, cudaStream_t s) {
  dim3 block(32 * wpb);
  const long long nitems = (long long)a.strips_x * a.strips_y;
  if (blocks <= 0) blocks = (int)((nitems + wpb - 1) / wpb);
  if (scheme == SC_DUGKS)
    dev::k_step<SC_DUGKS, ST><<<blocks, block, 0, s>>>(a);
  else if (scheme == SC_BKG_FV)
    dev::k_step<SC_BKG_FV, ST><<<blocks, block, 0, s>>>(a);
  else
    dev::k_step<SC_BKG_FD, ST><<<blocks, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <int ST>
cudaError_t launch_batch_impl(int scheme, const CaseArgs *d_cases, const long long *d_prefix,
                              int ncases, long long nitems, unsigned long long *d_queue,
                              int blocks, int wpb, cudaStream_t s) {
  dim3 block(32 * wpb);
  auto kern = scheme == SC_DUGKS ? dev::k_step_batch<SC_DUGKS, ST> : dev::k_step_batch<SC_BKG_FV, ST>;
  if (blocks <= 0) {
    // persistent grid: as many blocks as fit on the GPU at once
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block.x, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    blocks = (per_sm > 0 ? per_sm : 1) * sms;
  }
  kern<<<blocks, block, 0, s>>>(d_cases, d_prefix, ncases, nitems, d_queue);
  return cudaGetLastError();
}

} // namespace dvbe
